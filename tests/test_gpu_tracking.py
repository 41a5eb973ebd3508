"""Segmentation on the GPU (moc_generate_tracks_device) against the host walk: the same code in
IEEE double arithmetic without contracted multiply-adds on both sides, so every track, segment,
link and area must be bit-identical. The host walk itself is pinned against the oracle's
clip-based segmentation in test_abi_host.py."""
import numpy as np
import pytest

from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _core1(n_azim, spacing):
    xs = W.synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, 4,
                        fuel_scales=[1.0, 0.95, 1.05, 0.9])
    return W.Problem(W.core_mesh(1), xs, n_azim, spacing, tol=1e-6, name="core1", seed=4)


CASES = {
    "pin": lambda: W.pin_cell_problem(),
    "pin_vacuum": lambda: W.Problem(W.with_bc(W.pin_cell_mesh(), (0, 0, 0, 0)), W.synthetic_xs(["fuel", "moderator"], 7, 1), 16, 0.05),
    "lattice3_mixed_bc": lambda: W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03),
    "grid": lambda: W.Problem(W.grid_mesh(5, 3, 2.0, 1.0), W.synthetic_xs(["fuel"], 2, 1), 8, 0.07),
    "hex7_concave": lambda: W.Problem(W.hex_core_mesh(n_sub=4, n_rings=1), W.synthetic_xs(["fuel", "fuel", "coolant"], 3, 1), 12, 0.3),
    "hex7_back_projection": lambda: W.Problem(W.hex_core_mesh(n_sub=4, n_rings=1), W.synthetic_xs(["fuel", "fuel", "coolant"], 3, 1), 12, 0.3, ray_layout=1),
    "assembly": lambda: W.assembly_problem(),
    "core1": lambda: _core1(16, 0.05),
    "core1_45deg": lambda: _core1(12, 0.2),        # rays along cell diagonals and through vertices
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_device_tracks_are_bit_identical(case):
    prob = CASES[case]()
    h = moc.Moc.from_problem(prob, with_xs=False)
    d = moc.Moc.from_problem(prob, with_xs=False, device_tracking=True)
    assert h.track_counts() == d.track_counts()
    a, b = h.tracks(), d.tracks()
    for key in ("seg_off", "seg_region", "seg_len", "track_dir", "track_xy", "link"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(h.areas(), d.areas())


def test_device_tracking_runs_the_solver():
    """A context tracked on the device iterates like one tracked on the host (equal up to the
    order of the sweep's atomic additions, which differs from run to run anyway)."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    h = moc.Moc.from_problem(prob, precision="fp64")
    d = moc.Moc.from_problem(prob, precision="fp64", device_tracking=True)
    kh, _ = h.outer(5)
    kd, _ = d.outer(5)
    assert abs(kh - kd) <= 1e-13 * kh
    np.testing.assert_allclose(d.get_state()[0], h.get_state()[0], rtol=1e-12)


@pytest.mark.parametrize("case", ["hex7_back_projection", "core1"])
def test_device_tracked_solve_matches_oracle(case):
    """Geometry segmented on the GPU, solved on the GPU, compared with the oracle's own clip-based
    segmentation and sweep (not with the host walk): back-projected rays on the concave hexagon
    cluster (vacuum) and cyclic modular rays on one assembly with its reflector band (reflective
    -x/-y, vacuum +x/+y). FP64, outers from the same random state compared after each."""
    import oracle

    prob = CASES[case]()
    if case == "hex7_back_projection":
        prob.xs = W.synthetic_xs(["fuel", "fuel", "coolant"], 7, 9, sigt_range=(0.05, 0.6))
    o = oracle.Oracle.from_problem(prob, threads=8)
    m = moc.Moc.from_problem(prob, precision="fp64", device_tracking=True)
    assert m.track_counts() == (o.n_tracks, o.n_segments)
    rng = np.random.default_rng(41)
    G = prob.xs.n_groups
    phi0 = rng.uniform(0.5, 1.5, (prob.mesh.n_tri, G))
    psi0 = rng.uniform(0.0, 0.2, (o.n_tracks, 2, len(prob.sin_theta), G))
    o.set_state(phi0, 1.05, psi0)
    o.normalise()
    m.set_state(phi0, 1.05, psi0)
    for it in range(3):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        phig, _ = m.get_state()
        assert abs(kg - ko) <= 1e-11 * ko, (it, kg, ko)
        err = float(np.max(np.abs(phig - phio) / np.maximum(np.abs(phio), 1e-300)))
        assert err <= 1e-10, (it, err)
