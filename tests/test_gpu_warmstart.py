"""GPU tests of the learned warm start: the network's kernels against the FP64 CPU network
oracle, training progress, and what the trained network gains over the cold start."""
import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _net_and_data(n_in=93, width=256, n_out=8, rows=64, seed=0):
    import torch

    rng = np.random.default_rng(seed)
    net = moc.Mlp(n_in, width, n_out, seed=seed)
    norm = (rng.normal(0, 0.2, n_in), rng.uniform(0.5, 2.0, n_in), rng.normal(0, 0.2, n_out), rng.uniform(0.5, 2.0, n_out))
    net.set_normalization(*norm)
    x = rng.normal(0, 1, (rows, n_in)).astype(np.float32)
    y = rng.normal(0, 1, (rows, n_out)).astype(np.float32)
    return net, norm, x, y, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()


@pytest.mark.parametrize("rows,width,n_out", [(64, 256, 8), (300, 512, 40)])
def test_forward_and_gradients_match_cpu_oracle(rows, width, n_out):
    """The network's tensor-core forward and backward passes (tiles of 128 rows and 256 columns,
    partial tiles at both edges) against the FP64 network oracle."""
    import torch

    net, norm, x, y, xd, yd = _net_and_data(width=width, n_out=n_out, rows=rows)
    p = net.get_params().astype(np.float64)
    out = torch.empty((x.shape[0], n_out), dtype=torch.float32, device="cuda")
    net.forward(xd, out, x.shape[0])
    torch.cuda.synchronize()
    ref, _ = MO.forward(p, net.dims, x, norm, bf16=True)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=2e-5, atol=2e-5)
    g, loss = net.gradients(xd, yd, x.shape[0])
    lref, gref = MO.loss_and_grad(p, net.dims, x, y, norm, bf16=True)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    # per layer: error relative to the layer's largest gradient entry
    o = 0
    for l in range(4):
        nw = net.dims[l + 1] * net.dims[l] + net.dims[l + 1]
        err = np.abs(g[o:o + nw] - gref[o:o + nw]).max() / np.abs(gref[o:o + nw]).max()
        assert err < 1e-4, (l, err)
        o += nw


def test_training_reduces_loss_on_a_smooth_target():
    import torch

    rng = np.random.default_rng(3)
    n_in, n_out, rows = 16, 4, 4096
    net = moc.Mlp(n_in, 128, n_out, seed=1)
    x = rng.normal(0, 1, (rows, n_in)).astype(np.float32)
    A = rng.normal(0, 0.5, (n_in, n_out))
    y = (np.tanh(x @ A) + 0.1 * (x[:, :n_out] ** 2)).astype(np.float32)
    net.set_normalization(np.zeros(n_in), np.ones(n_in), y.mean(0), y.std(0))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    first = net.train_step(xd, yd, rows, 2e-3, want_loss=True)
    for _ in range(300):
        last = net.train_step(xd, yd, rows, 2e-3, want_loss=True)
    assert last < 0.05 * first, (first, last)


def test_learned_start_needs_fewer_outers_than_cold():
    from paper_2607_01591_gb300 import warmstart

    r = warmstart.run(n_train=48, n_eval=6, n_eval_fp64=1, rows_per_instance=400, epochs=30, out="", lattice=3)
    print(r)
    # the trained network's start needs fewer outers than the cold start
    assert r["warm_fp32"]["outers_mean"] < r["cold_fp32"]["outers_mean"]


def test_shipped_network_beats_the_ablation_and_the_cold_start():
    """The network the package ships (trained on the GPU by the library's own kernels on 2000
    perturbed assembly instances), on held-out instances it never saw: its start needs fewer
    outers to |k - k_ref| <= 5 pcm than the training-mean solution without a network (the
    ablation), which in turn needs fewer than the cold start."""
    from paper_2607_01591_gb300 import warmstart
    from paper_2607_01591_gb300 import workloads as W

    base = warmstart.assembly_base()
    ws = warmstart.WarmStart(W.assembly_problem(), base, W.guide_tube_positions())
    ws.load(warmstart.SHIPPED)
    mean_pred = ws.mean_solution([W.perturbed_xs(base, warmstart.TRAIN_SEED + i) for i in range(10)])
    held = [W.perturbed_xs(base, warmstart.HELD_OUT_SEED + 5000 + i) for i in range(8)]
    r = warmstart.evaluate(ws, held, mean_pred, n_fp64=0)
    print(r)
    assert r["warm_fp32"]["outers_mean"] < r["mean_solution_fp32"]["outers_mean"] < r["cold_fp32"]["outers_mean"]
    assert r["warm_initial_k_err_pcm_mean"] < r["mean_solution_initial_k_err_pcm_mean"]
