"""The remaining boundary calls on the GPU: tracks supplied by the caller (moc_set_tracks), one
outer with caller-owned device flux arrays (moc_sweep_dev), and the timing statistics
(moc_get_stats)."""
import numpy as np
import pytest

from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _prob():
    return W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)


def test_caller_tracks_iterate_like_generated_ones():
    prob = _prob()
    a = moc.Moc.from_problem(prob, precision="fp64")
    tr, q = a.tracks(), a.quadrature(prob.n_azim // 2)
    b = moc.Moc(0, "fp64")
    b.set_mesh(prob.mesh)
    b.set_quadrature(prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w)
    b.set_tracks(tr["seg_off"], tr["seg_region"], tr["seg_len"], tr["track_dir"], q["omega"], q["delta"], tr["link"])
    b.set_xs(prob.xs)
    ka, _ = a.outer(6)
    kb, _ = b.outer(6)
    assert abs(ka - kb) <= 1e-12 * ka
    np.testing.assert_allclose(b.get_state()[0], a.get_state()[0], rtol=1e-11)
    with pytest.raises(moc.MocError):      # the directions' angles are unknown
        b.set_scattering(W.anisotropic_moments(prob.xs, 1, [0.1, 0.1, 0.1]))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sweep_dev_matches_outer(precision):
    import torch
    prob = _prob()
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 2e-6
    a = moc.Moc.from_problem(prob, precision=precision)
    b = moc.Moc.from_problem(prob, precision=precision)
    R, G = prob.mesh.n_tri, prob.xs.n_groups
    # continuing from the context's own flux
    out = torch.empty((R, G), dtype=dt, device="cuda")
    stream = torch.cuda.Stream()
    a.outer(2)
    b.outer(1)
    b.sweep_dev(None, out, stream)
    stream.synchronize()
    phi_a, ka = a.get_state()
    kb, _ = b.outer(0)
    assert abs(ka - kb) <= tol * ka
    np.testing.assert_allclose(out.cpu().double().numpy(), phi_a, rtol=10 * tol)
    # feeding the returned (normalised) flux back in continues the same iteration
    out2 = torch.empty_like(out)
    b.sweep_dev(out, out2, None)
    a.outer(1)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out2.cpu().double().numpy(), a.get_state()[0], rtol=10 * tol)


def test_stats_report_the_timed_sweeps():
    prob = W.assembly_problem()
    m = moc.Moc.from_problem(prob)
    m.outer(2)
    m.enable_timing(True)
    m.outer(5, read=False)
    ms, ups = m.stats()
    assert 0.0 < ms < 100.0
    _, per_sweep, _ = m.work()
    assert abs(ups - per_sweep / (ms * 1e-3)) <= 1e-9 * ups


def test_set_xs_rejects_negative_absorption():
    prob = _prob()
    m = moc.Moc.from_problem(prob, precision="fp32", with_xs=False)
    xs = prob.xs
    bad = W.CrossSections(xs.sigma_t, xs.nu_sigma_f, xs.chi, xs.sigma_s * 1.2)
    with pytest.raises(moc.MocError) as e:
        m.set_xs(bad)
    assert e.value.code == -1 and "scattering" in str(e.value)
    m.set_xs(xs)


def test_history_records_every_check():
    prob = _prob()
    a = moc.Moc.from_problem(prob, precision="fp64")
    k, n, r, ok = a.power_iterate(tol_k=1e-7, tol_flux=1e-6, max_outer=400, check_every=5)
    h = a.history()
    assert ok and h.shape == (n // 5, 4)
    np.testing.assert_array_equal(h[:, 0], 5.0 * np.arange(1, n // 5 + 1))
    assert h[-1, 1] == k and h[-1, 3] == r
    assert abs(h[-1, 1] - h[-1, 2]) <= 1e-7 and h[-1, 3] <= 1e-6
    assert not (abs(h[-2, 1] - h[-2, 2]) <= 1e-7 and h[-2, 3] <= 1e-6)   # the previous check had not converged
    # the same iteration driven five outers at a time gives the same records
    b = moc.Moc.from_problem(prob, precision="fp64")
    for _ in range(3):
        b.outer(5)
    b.outer(0)                                  # a read without outers records nothing
    np.testing.assert_allclose(b.history(), h[:3], rtol=1e-12)
    assert a.history(2).shape == (2, 4) and np.array_equal(a.history(2), h[-2:])
    a.set_state(None, 1.0)                      # a new start clears the record
    assert a.history().shape == (0, 4)


def test_history_ring_keeps_the_last_4096_checks_in_order():
    m = moc.Moc.from_problem(W.pin_cell_problem(), precision="fp32")
    _, n, _, ok = m.power_iterate(tol_k=0.0, tol_flux=0.0, max_outer=4100, check_every=1, raise_on_fail=False)
    assert not ok and n == 4100
    h = m.history()
    assert h.shape == (4096, 4)
    np.testing.assert_array_equal(h[:, 0], np.arange(5, 4101, dtype=float))   # oldest first after wrapping
    assert np.array_equal(m.history(3), h[-3:])


def test_rate_probes_measure_positive_rates():
    """Every hardware rate probe runs, reports the device's multiprocessor count, positive lane
    rates, and sector rates consistent with its access shape."""
    for kind in moc.PROBES:
        r = moc.probe_rate(kind, 0)
        assert r["sm_count"] > 0
        assert r["lane_ops_per_s"] > 0, kind
        if kind in ("ffma", "dfma"):
            assert r["sectors_per_s"] == 0.0
        else:
            per = {"red_f32x4_pair": 0.5, "red_f32_row8": 0.125}.get(kind, 1.0)
            assert abs(r["sectors_per_s"] - per * r["lane_ops_per_s"]) <= 1e-9 * r["lane_ops_per_s"], kind
