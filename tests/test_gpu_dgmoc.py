"""DGMOC on the GPU (moc_set_axial) against the oracle's DGMOC (Sec. 2.2, Alg. 2), all through
the C ABI: outer by outer from the same flat start, converged k, the fixed-source slab, and
symmetry at the full assembly size."""
import numpy as np
import pytest

import oracle
from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _case(bc_xy=(1, 0, 1, 0)):
    prob = W.small_lattice_problem(3, bc=bc_xy, n_azim=8, ray_spacing=0.1)
    nz = 3
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[-1] = prob.mesh.mat.max()            # top plane of the last material (moderator)
    dz = np.array([1.1, 2.0, 0.6])
    return prob, dz, mat3


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("bcz", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_outers_match_oracle_fp64(bcz):
    prob, dz, mat3 = _case()
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=bcz)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_axial(dz, mat3, bc=bcz)
    for it in range(5):
        o.outer()
        k, _ = m.outer(1)
        po, ko = o.flux3()
        pg, kg = m.get_state()
        assert abs(k - ko) <= 1e-11 * ko and kg == k
        assert _rel(pg[:, :, 0], po[:, :, 0]) <= 1e-11, it
        assert np.abs(pg[:, :, 1] - po[:, :, 1]).max() <= 1e-11 * np.abs(po[:, :, 0]).max(), it


def test_outers_match_oracle_fp32():
    prob, dz, mat3 = _case()
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=(1, 0))
    m = moc.Moc.from_problem(prob, precision="fp32")
    m.set_axial(dz, mat3, bc=(1, 0))
    for _ in range(4):
        o.outer()
    k, _ = m.outer(4)
    po, ko = o.flux3()
    pg, _ = m.get_state()
    # FP32 rounding of per-segment moments accumulated by atomics over ~1e2 segments per element
    assert abs(k - ko) <= 2e-5 * ko
    assert _rel(pg[:, :, 0], po[:, :, 0]) <= 5e-5
    assert np.abs(pg[:, :, 1] - po[:, :, 1]).max() <= 5e-5 * np.abs(po[:, :, 0]).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 5e-5)])
def test_converged_k_matches_oracle(precision, tol):
    prob, dz, mat3 = _case((0, 0, 0, 0))
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=(0, 0))
    ko, _, _, ok = o.iterate(tol_k=1e-10, tol_f=1e-8, max_outer=2000)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_axial(dz, mat3, bc=(0, 0))
    kg, n, r, okg = m.power_iterate(tol_k=1e-10 if precision == "fp64" else 1e-7,
                                    tol_flux=1e-8 if precision == "fp64" else 1e-5, max_outer=2000)
    assert ok and okg and abs(kg - ko) <= tol * ko
    pg, _ = m.get_state()
    po, _ = o.flux3()
    assert _rel(pg[:, :, 0], po[:, :, 0]) <= (1e-7 if precision == "fp64" else 2e-4)


def test_fixed_source_slab_matches_oracle():
    mesh = W.grid_mesh(1, 1, 4.0, 4.0, bc=(1, 1, 1, 1))
    xs = W.CrossSections(np.array([[1.0]]), np.zeros((1, 1)), np.zeros((1, 1)), np.array([[[0.6]]]))
    prob = W.Problem(mesh, xs, 8, 0.5, fixed_source=np.ones((mesh.n_tri, 1)))
    dz = np.full(16, 0.25)
    o = oracle.Oracle.from_problem(prob)
    o.set_axial(dz, bc=(0, 0))
    o.iterate(eigen=False, tol_f=1e-12, max_outer=2000)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_axial(dz, bc=(0, 0))
    _, _, _, ok = m.power_iterate(tol_k=1.0, tol_flux=1e-12, max_outer=2000)
    assert ok
    np.testing.assert_allclose(m.get_state()[0], o.flux3()[0], rtol=1e-10, atol=1e-12)


def test_axial_mode_switches_and_rejections():
    prob, dz, mat3 = _case()
    m = moc.Moc.from_problem(prob, precision="fp64")
    k2, _ = m.outer(3)
    m.set_axial(dz, mat3)
    with pytest.raises(moc.MocError):
        m.set_state(np.ones((3, prob.mesh.n_tri, 2, prob.xs.n_groups)), 1.0,
                    np.zeros((m.track_counts()[0], 2, m.n_polar, prob.xs.n_groups)))
    with pytest.raises(moc.MocError):
        m.set_scattering(W.anisotropic_moments(prob.xs, 1, [0.1] * prob.xs.n_mat))
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    with pytest.raises(moc.MocError):
        m.set_cmfd(cell, nc)
    with pytest.raises(moc.MocError):
        m.set_axial(np.array([1.0, -1.0]))
    # planes thinner than 1e-9 cm are refused (they would push the per-update 1/D of the FP32
    # sweep outside the approximate division's range)
    with pytest.raises(moc.MocError) as e:
        m.set_axial(np.array([1.0, 1e-10]))
    assert e.value.code == -1
    with pytest.raises(moc.MocError):
        m.set_axial(dz, np.full_like(mat3, 99))
    # a state set in the DG layout round-trips
    m.set_axial(dz, mat3)
    m.outer(2)
    phi, k = m.get_state()
    m2 = moc.Moc.from_problem(prob, precision="fp64")
    m2.set_axial(dz, mat3)
    m2.set_state(phi, k)
    np.testing.assert_allclose(m2.get_state()[0], phi, rtol=1e-14)
    # back to the planar method
    m.set_axial([])
    assert m.get_state()[0].shape == (prob.mesh.n_tri, prob.xs.n_groups)
    assert abs(m.outer(3)[0] - k2) <= 1e-12 * k2


@pytest.mark.parametrize("precision", ["fp32"])
def test_full_assembly_symmetric_stack(precision):
    """The benchmark's extruded assembly (8 planes, vacuum top and bottom, a reflector plane at
    each end): plane averages mirror about the mid-plane and the linear moments change sign (a
    property of the exact and the discrete solution at any size)."""
    prob = W.assembly_problem()
    nz = 8
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[0] = mat3[-1] = prob.mesh.mat.max()
    dz = np.array([5.0] + [10.0] * 6 + [5.0])
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_axial(dz, mat3, bc=(0, 0))
    k, _ = m.outer(6)
    phi, _ = m.get_state()
    assert np.isfinite(k) and np.all(phi[:, :, 0] > 0)
    scale = np.abs(phi[:, :, 0]).max()
    assert np.abs(phi[::-1, :, 0] - phi[:, :, 0]).max() <= 2e-5 * scale
    assert np.abs(phi[::-1, :, 1] + phi[:, :, 1]).max() <= 2e-5 * scale


def test_plane_by_plane_variant_matches_oracle():
    """14 FP64 planes need more shared memory per block than the plane-inner sweep takes, so the
    library runs the plane-by-plane sweep with its interface buffer in device memory."""
    prob, _, _ = _case()
    nz = 14
    rng = np.random.default_rng(5)
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[rng.random(nz) < 0.3] = prob.mesh.mat.max()
    dz = rng.uniform(0.3, 2.0, nz)
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=(1, 1))
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_axial(dz, mat3, bc=(1, 1))
    for _ in range(3):
        o.outer()
    k, _ = m.outer(3)
    po, ko = o.flux3()
    pg, _ = m.get_state()
    assert abs(k - ko) <= 1e-11 * ko
    assert _rel(pg[:, :, 0], po[:, :, 0]) <= 1e-11
    assert np.abs(pg[:, :, 1] - po[:, :, 1]).max() <= 1e-11 * np.abs(po[:, :, 0]).max()


def _outers_vs_oracle(prob, dz, mat3, bc, n=3, threads=8):
    o = oracle.Oracle.from_problem(prob, threads=threads)
    o.set_axial(dz, mat3, bc=bc)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_axial(dz, mat3, bc=bc)
    for _ in range(n):
        o.outer(prob.fixed_source is None)
    k, _ = m.outer(n)
    po, ko = o.flux3()
    pg, _ = m.get_state()
    assert prob.fixed_source is not None or abs(k - ko) <= 1e-11 * ko
    assert _rel(pg[:, :, 0], po[:, :, 0]) <= 1e-11
    assert np.abs(pg[:, :, 1] - po[:, :, 1]).max() <= 1e-11 * np.abs(po[:, :, 0]).max()


@pytest.mark.parametrize("n_polar", [1, 2, 4])
def test_polar_counts_match_oracle(n_polar):
    """every compiled polar count of the sweep (3 is covered above)"""
    prob, dz, mat3 = _case()
    st = {1: [0.8], 2: [0.35, 0.9], 4: [0.1, 0.4, 0.7, 0.95]}[n_polar]
    w = np.full(n_polar, 1.0 / n_polar)
    prob = W.Problem(prob.mesh, prob.xs, prob.n_azim, prob.ray_spacing, np.array(st), w)
    _outers_vs_oracle(prob, dz, mat3, (1, 0))


def test_one_plane_many_groups_and_back_projection():
    """one plane (both faces reflective), 33 groups (threads per track beyond a warp's quarter);
    then back-projected rays on the concave 7-hexagon cluster (vacuum) with 2 planes"""
    mesh = W.grid_mesh(3, 3, 3.0, 3.0, bc=(1, 0, 1, 0), mat_fn=lambda i, j: (i + j) % 2)
    xs = W.synthetic_xs(["fuel", "moderator"], 33, 12)
    prob = W.Problem(mesh, xs, 8, 0.2)
    _outers_vs_oracle(prob, np.array([3.0]), None, (1, 1), n=2)
    mesh = W.hex_core_mesh(n_sub=4, n_rings=1)
    xs = W.synthetic_xs(["fuel", "fuel", "coolant"], 7, 9, sigt_range=(0.05, 0.6))
    prob = W.Problem(mesh, xs, 12, 0.3, ray_layout=1)
    _outers_vs_oracle(prob, np.array([2.0, 1.0]), None, (0, 0), n=3)


@pytest.mark.parametrize("bcz", [(1, 0), (0, 1)])
def test_axial_acceleration_outers_match_oracle(bcz):
    """accelerated outers (planes as coarse cells) from the flat start, compared after each"""
    prob, dz, mat3 = _case()
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=bcz)
    o.set_dg_cmfd(6, 3, 1.2)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_axial(dz, mat3, bc=bcz)
    m.set_dg_cmfd(6, 3, 1.2)
    for it in range(4):
        o.outer()
        k, _ = m.outer(1)
        po, ko = o.flux3()
        pg, _ = m.get_state()
        assert abs(k - ko) <= 1e-10 * ko, (it, k, ko)
        assert _rel(pg[:, :, 0], po[:, :, 0]) <= 1e-10, it
        assert np.abs(pg[:, :, 1] - po[:, :, 1]).max() <= 1e-10 * np.abs(po[:, :, 0]).max(), it


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 5e-5)])
def test_axial_acceleration_reaches_the_plain_limit_faster(precision, tol):
    """a pin cell stacked in 4 planes of 3 cm (moderator on top, reflective bottom): the accelerated
    GPU iteration reaches the oracle's accelerated limit (pinned to the plain iteration's fixed
    point) in a fraction of the outers the plain GPU iteration needs. Flux bar: the stopping
    residual (1e-10 in FP64) over the gap of the accelerated iteration's spectrum."""
    pin = W.pin_cell_problem()
    prob = W.Problem(pin.mesh, pin.xs, 8, 0.1)
    nz = 4
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[-1] = prob.mesh.mat.max()
    dz = np.full(nz, 3.0)
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_axial(dz, mat3, bc=(1, 0))
    o.set_dg_cmfd(8, 4, 1.0)
    ko, _, _, ok = o.iterate(tol_k=1e-12, tol_f=1e-10, max_outer=2000)
    tk, tf = (1e-12, 1e-10) if precision == "fp64" else (1e-7, 1e-5)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_axial(dz, mat3, bc=(1, 0))
    m.set_dg_cmfd(8, 4, 1.0)
    kg, n_acc, _, okg = m.power_iterate(tol_k=tk, tol_flux=tf, max_outer=2000)
    assert ok and okg and abs(kg - ko) <= tol * ko
    assert _rel(m.get_state()[0][:, :, 0], o.flux3()[0][:, :, 0]) <= (1e-8 if precision == "fp64" else 3e-4)
    p = moc.Moc.from_problem(prob, precision=precision)
    p.set_axial(dz, mat3, bc=(1, 0))
    _, n_plain, _, _ = p.power_iterate(tol_k=tk, tol_flux=tf, max_outer=3 * n_acc, raise_on_fail=False)
    assert n_plain >= 3 * n_acc - 10, (n_acc, n_plain)   # plain needs at least three times as many


def test_full_assembly_infinite_medium():
    """The benchmark's mesh, tracks and launch configuration (17x17 assembly, 9.1M segments,
    8 planes, plane-inner sweep, FP32) with one material everywhere and every face reflective,
    iterated with the axial acceleration: the closed-form k-infinity, a flat plane-average flux
    and zero slopes, at full size."""
    base = W.assembly_problem()
    xs = W.synthetic_xs(["fuel"], 7, 31)
    prob = W.Problem(W.one_material(base.mesh), xs, base.n_azim, base.ray_spacing)
    M = np.diag(xs.sigma_t[0]) - xs.sigma_s[0].T
    kinf = float(xs.nu_sigma_f[0] @ np.linalg.solve(M, xs.chi[0]))
    m = moc.Moc.from_problem(prob, precision="fp32")
    m.set_axial(np.full(8, 10.71), bc=(1, 1))
    m.set_dg_cmfd(8, 4, 1.0)
    k, n, r, ok = m.power_iterate(tol_k=1e-8, tol_flux=1e-6, max_outer=400)
    assert ok and abs(k - kinf) <= 2e-6 * kinf, (k, kinf, n)
    phi, _ = m.get_state()
    spec = phi[:, :, 0, :].reshape(-1, 7)
    np.testing.assert_allclose(spec, np.broadcast_to(spec.mean(axis=0), spec.shape), rtol=2e-5)
    assert np.abs(phi[:, :, 1]).max() <= 2e-5 * np.abs(spec).max()


def test_axial_acceleration_is_for_eigenvalue_mode_only():
    """a fixed-source DGMOC iteration with the acceleration switched on is the plain one"""
    mesh = W.grid_mesh(2, 2, 2.0, 2.0, bc=(1, 0, 1, 0))
    xs = W.CrossSections(np.array([[1.0]]), np.zeros((1, 1)), np.zeros((1, 1)), np.array([[[0.5]]]))
    prob = W.Problem(mesh, xs, 8, 0.2, fixed_source=np.ones((mesh.n_tri, 1)))
    res = []
    for acc in (False, True):
        m = moc.Moc.from_problem(prob, precision="fp64")
        m.set_axial(np.full(3, 1.0), bc=(0, 0))
        if acc:
            m.set_dg_cmfd(8, 4, 1.0)
        m.outer(5)
        res.append(m.get_state()[0])
    # equal up to the order of the tally atomics
    np.testing.assert_allclose(res[1], res[0], rtol=1e-12, atol=1e-14 * np.abs(res[0]).max())
