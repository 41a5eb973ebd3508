"""C-ABI library: loads, exports every declared symbol, and its host-side geometry (half-edge
walk segmentation, links, tracked areas) agrees with the oracle's clip-based segmentation.
No GPU is needed: these use host-only contexts (device = -1)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return moc.load_library()


def test_library_exports_every_header_symbol(lib):
    names = moc.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def _compare_tracks(prob):
    m = moc.Moc.from_problem(prob, device=-1)
    o = oracle.Oracle.from_problem(prob, with_xs=False)
    a, b = m.tracks(), o.tracks()
    assert m.track_counts() == (o.n_tracks, o.n_segments)
    assert np.array_equal(a["seg_off"], b["seg_off"])
    assert np.array_equal(a["seg_region"], b["seg_region"])
    np.testing.assert_allclose(a["seg_len"], b["seg_len"], rtol=0, atol=1e-11)
    assert np.array_equal(a["track_dir"], b["track_dir"])
    np.testing.assert_allclose(a["track_xy"], b["track_xy"], rtol=0, atol=1e-11)
    assert np.array_equal(a["link"], b["link"])
    np.testing.assert_allclose(m.areas(), o.areas(), rtol=1e-11)
    q1, q2 = m.quadrature(o.n_dir), o.quadrature()
    for k in ("phi", "delta", "omega"):
        np.testing.assert_allclose(q1[k], q2[k], rtol=1e-14)


@pytest.mark.parametrize("case", ["pin", "pin_vacuum", "lattice3", "lattice3_mixed_bc", "grid", "hex7", "hex1",
                                  "pin_back_projection", "hex7_back_projection", "grid_back_projection"])
def test_host_segmentation_matches_oracle(lib, case):
    if case == "pin":
        prob = W.pin_cell_problem()
    elif case == "pin_vacuum":
        prob = W.pin_cell_problem()
        prob.mesh = W.with_bc(prob.mesh, (0, 0, 0, 0))
    elif case == "lattice3":
        prob = W.small_lattice_problem(3)
    elif case == "lattice3_mixed_bc":
        prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    elif case == "grid":
        prob = W.Problem(W.grid_mesh(5, 3, 2.0, 1.0), W.synthetic_xs(["fuel"], 2, 1), 8, 0.07)
    elif case == "hex7":
        prob = W.Problem(W.hex_core_mesh(n_sub=4, n_rings=1), W.synthetic_xs(["fuel", "fuel", "coolant"], 3, 1), 12, 0.3)
    elif case == "hex1":
        prob = W.Problem(W.hex_core_mesh(n_sub=6, n_rings=0), W.synthetic_xs(["fuel", "fuel", "coolant"], 3, 1), 8, 0.2)
    elif case == "pin_back_projection":
        prob = W.pin_cell_problem()
        prob.mesh = W.with_bc(prob.mesh, (0, 0, 0, 0))
        prob.ray_layout = 1
    elif case == "hex7_back_projection":
        prob = W.Problem(W.hex_core_mesh(n_sub=4, n_rings=1), W.synthetic_xs(["fuel", "fuel", "coolant"], 3, 1), 12, 0.3,
                         ray_layout=1)
    else:
        prob = W.Problem(W.grid_mesh(5, 3, 2.0, 1.0, bc=(0, 0, 0, 0)), W.synthetic_xs(["fuel"], 2, 1), 12, 0.07,
                         ray_layout=1)
    _compare_tracks(prob)


def test_rays_along_mesh_edges_are_traced_without_gaps(lib):
    """12 azimuths put one direction at exactly 45 degrees, along the diagonals of the reflector's
    square cells: rays run along edges and through vertices. Host walk and oracle must agree
    (before edge tests were evaluated from a canonical endpoint, such rays lost pieces)."""
    xs = W.synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, 4,
                        fuel_scales=[1.0, 0.95, 1.05, 0.9])
    _compare_tracks(W.Problem(W.core_mesh(1), xs, 12, 0.2, tol=1e-6, name="core1", seed=4))


def test_back_projection_rejects_reflective_walls(lib):
    prob = W.pin_cell_problem()
    prob.ray_layout = 1
    with pytest.raises(moc.MocError):
        moc.Moc.from_problem(prob, device=-1)


def test_bad_inputs_are_rejected(lib):
    m = moc.Moc(device=-1)
    mesh = W.grid_mesh(2, 2, 1.0, 1.0)
    bad = W.Mesh(mesh.xy, mesh.tri[:, ::-1].copy(), mesh.mat, mesh.bbox, mesh.bc)   # clockwise
    with pytest.raises(moc.MocError) as e:
        m.set_mesh(bad)
    assert e.value.code == -1
    bad2 = W.Mesh(mesh.xy, mesh.tri.copy(), mesh.mat, mesh.bbox, mesh.bc)
    bad2.tri[0, 0] = 10_000
    with pytest.raises(moc.MocError):
        m.set_mesh(bad2)
    # three triangles on one edge: not conforming
    dup = W.Mesh(mesh.xy, np.concatenate([mesh.tri, mesh.tri[:1]]), np.concatenate([mesh.mat, mesh.mat[:1]]),
                 mesh.bbox, mesh.bc)
    with pytest.raises(moc.MocError):
        m.set_mesh(dup)
    m.set_mesh(mesh)
    with pytest.raises(moc.MocError):
        m.set_quadrature(6, 0.1, W.TY3_SIN_THETA, W.TY3_WEIGHT)       # not a multiple of 4
    with pytest.raises(moc.MocError):
        m.set_quadrature(8, 0.1, W.TY3_SIN_THETA, W.TY3_WEIGHT * 2)   # weights must sum to 1
    with pytest.raises(moc.MocError) as e:
        m.generate_tracks()                                            # no quadrature yet
    assert e.value.code == -4
    m.set_quadrature(8, 0.1, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    m.generate_tracks()
    # GPU work on a host-only context is refused with a message, not a crash
    with pytest.raises(moc.MocError) as e:
        m.set_xs(W.synthetic_xs(["fuel"], 2, 1))
    assert e.value.code == -4
    assert "host-only" in str(e.value)


def _caller_tracks(prob):
    a = moc.Moc.from_problem(prob, device=-1)
    tr = a.tracks()
    q = a.quadrature(prob.n_azim // 2)
    return a, tr, q


def test_set_tracks_reproduces_generated_tracks(lib):
    """Tracks generated by one context and handed to another through moc_set_tracks give the same
    segments, links and (to rounding) tracked areas."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    a, tr, q = _caller_tracks(prob)
    b = moc.Moc(-1, "fp32")
    b.set_mesh(prob.mesh)
    b.set_quadrature(prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w)
    b.set_tracks(tr["seg_off"], tr["seg_region"], tr["seg_len"], tr["track_dir"], q["omega"], q["delta"], tr["link"])
    tb = b.tracks()
    for key in ("seg_off", "seg_region", "seg_len", "track_dir", "link"):
        assert np.array_equal(tb[key], tr[key]), key
    np.testing.assert_allclose(b.areas(), a.areas(), rtol=1e-13)


def test_set_tracks_validates(lib):
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    a, tr, q = _caller_tracks(prob)
    b = moc.Moc(-1, "fp32")
    b.set_mesh(prob.mesh)
    b.set_quadrature(prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w)
    args = [tr["seg_off"], tr["seg_region"], tr["seg_len"], tr["track_dir"], q["omega"], q["delta"], tr["link"]]
    bad_link = tr["link"].copy()
    e = bad_link[bad_link >= 0][0]
    bad_link[bad_link == -1] = e          # an incoming end fed twice
    bad_len = tr["seg_len"].copy()
    bad_len[3] = -1.0
    bad_reg = tr["seg_region"].copy()
    bad_reg[5] = prob.mesh.n_tri
    for i, v in ((6, bad_link), (2, bad_len), (1, bad_reg)):
        a2 = list(args)
        a2[i] = v
        with pytest.raises(moc.MocError) as err:
            b.set_tracks(*a2)
        assert err.value.code == -1


@pytest.mark.parametrize("tol_k,tol_flux,max_outer,check_every",
                         [(float("nan"), 1e-6, 10, 1), (-1e-6, 1e-6, 10, 1), (1e-6, float("nan"), 10, 1),
                          (1e-6, -1.0, 10, 1), (1e-6, 1e-6, 0, 1), (1e-6, 1e-6, 10, 0)])
def test_power_iterate_rejects_bad_arguments(lib, tol_k, tol_flux, max_outer, check_every):
    """Tolerances that can never be met (NaN, negative) and empty loops are argument errors, checked
    before anything else (so also on a host-only context)."""
    m = moc.Moc.from_problem(W.pin_cell_problem(), device=-1)
    with pytest.raises(moc.MocError) as e:
        m.power_iterate(tol_k, tol_flux, max_outer, check_every=check_every)
    assert e.value.code == -1
    # valid arguments on a host-only context: a state error, not an argument error
    with pytest.raises(moc.MocError) as e:
        m.power_iterate(1e-6, 1e-6, 10, check_every=1)
    assert e.value.code == -4


def test_rate_probe_rejects_unknown_kinds_and_devices(lib):
    """The rate probes validate their arguments before touching a device."""
    import ctypes

    d = ctypes.c_double()
    assert lib.moc_probe_rate(0, -1, ctypes.byref(d), None, None) == -1
    assert lib.moc_probe_rate(0, len(moc.PROBES), ctypes.byref(d), None, None) == -1
    assert lib.moc_probe_rate(-1, 0, ctypes.byref(d), None, None) == -1
