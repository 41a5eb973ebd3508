"""The network forward pass that allocates nothing (moc_mlp_forward_noalloc), for callers that
may not call cudaMalloc -- e.g. code running under CUDA graph capture or inside a solver that
owns all device memory through its own pool. It must give the same result as the ordinary forward
pass on consecutive calls, although every call reuses one fixed device workspace, and it must
refuse a batch larger than that workspace instead of overrunning it. Collected last on purpose."""
import numpy as np
import pytest

from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu

NOALLOC_FLOATS = 2 * 1024 * 1024


def test_noalloc_forward_matches_forward_on_consecutive_calls():
    import torch

    build()
    rng = np.random.default_rng(11)
    n_in, width, n_out = 93, 256, 8
    net = moc.Mlp(n_in, width, n_out, seed=5)
    net.set_normalization(rng.normal(0, 0.2, n_in), rng.uniform(0.5, 2, n_in), rng.normal(0, 0.2, n_out),
                          rng.uniform(0.5, 2, n_out))
    per_row = n_in + 2 * width * 3 + n_out
    max_rows = NOALLOC_FLOATS // per_row
    for rows in (max_rows, 257):            # two calls in a row, different sizes and inputs
        x = torch.from_numpy(rng.normal(0, 1, (rows, n_in)).astype(np.float32)).cuda()
        y_ref = torch.empty((rows, n_out), dtype=torch.float32, device="cuda")
        y = torch.full((rows, n_out), float("nan"), dtype=torch.float32, device="cuda")
        net.forward(x, y_ref, rows)
        net.forward_noalloc(x, y, rows)
        torch.cuda.synchronize()
        np.testing.assert_allclose(y.cpu().numpy(), y_ref.cpu().numpy(), rtol=2e-5, atol=2e-5)
    # a batch beyond the fixed workspace is refused with an error, not run
    x = torch.zeros((max_rows + 1, n_in), dtype=torch.float32, device="cuda")
    y = torch.zeros((max_rows + 1, n_out), dtype=torch.float32, device="cuda")
    with pytest.raises(moc.MocError) as e:
        net.forward_noalloc(x, y, max_rows + 1)
    assert e.value.code == -1
