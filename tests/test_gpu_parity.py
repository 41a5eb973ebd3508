"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle on the same
seeded inputs. Bars: FP64 mode |dk| <= 2 pcm and max relative region-flux error <= 1e-5
(tighter where both sides run the same outers from the same state); FP32 modes are reported
and held to looser bars that follow from FP32 arithmetic."""
import os

import numpy as np
import pytest

import oracle
from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu

PCM = 1e-5
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _oracle(prob):
    return oracle.Oracle.from_problem(prob, threads=min(NCPU, 16))


def test_pin_cell_converged_fp64():
    prob = W.pin_cell_problem()
    o = _oracle(prob)
    ko, no, _, conv = o.iterate(True, 1e-11, 1e-10, 20000)
    assert conv
    phio, _ = o.get_state()
    m = moc.Moc.from_problem(prob, precision="fp64")
    kg, ng, rg, convg = m.power_iterate(1e-11, 1e-10, 20000, check_every=1)
    assert convg
    phig, _ = m.get_state()
    assert abs(kg - ko) <= 2 * PCM
    assert _rel(phig, phio) <= 1e-5
    # both iterate the same discrete operator: much closer than the bar, same outer count
    assert abs(kg - ko) < 1e-9 and _rel(phig, phio) < 1e-8
    assert ng == no


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_plain"])
def test_same_outers_from_same_state(precision):
    """Random flux, k and boundary flux on both sides; then 6 outers each, compared after every
    outer (exercises every link, the normalisation and the k update)."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    o = _oracle(prob)
    m = moc.Moc.from_problem(prob, precision=precision)
    rng = np.random.default_rng(5)
    T, _ = m.track_counts()
    phi0 = rng.uniform(0.5, 1.5, (prob.mesh.n_tri, prob.xs.n_groups))
    psi0 = rng.uniform(0.0, 0.2, (T, 2, 3, prob.xs.n_groups))
    o.set_state(phi0, 1.1, psi0)
    o.normalise()
    m.set_state(phi0, 1.1, psi0)
    tol_phi = {"fp64": 1e-11, "fp32": 2e-5, "fp32_plain": 5e-5}[precision]
    tol_k = {"fp64": 1e-12, "fp32": 2e-6, "fp32_plain": 5e-6}[precision]
    for it in range(6):
        ro = o.outer(True)
        kg, rg = m.outer(1)
        phio, ko = o.get_state()
        phig, kg2 = m.get_state()
        assert kg == kg2
        assert abs(kg - ko) <= tol_k, (it, kg, ko)
        assert _rel(phig, phio) <= tol_phi, (it, _rel(phig, phio))
        assert abs(rg - ro) <= max(1e-9, 10 * tol_phi) * max(1.0, ro), (it, rg, ro)


def test_fixed_source_vacuum_fp64():
    prob = W.pin_cell_problem()
    prob.mesh = W.with_bc(prob.mesh, (0, 0, 0, 0))
    xs = prob.xs
    prob.xs = W.CrossSections(xs.sigma_t, np.zeros_like(xs.nu_sigma_f), xs.chi, xs.sigma_s)
    S = np.zeros((prob.mesh.n_tri, 7))
    S[prob.mesh.mat == 0, 0] = 1.0
    prob.fixed_source = S
    o = _oracle(prob)
    o.set_state(np.zeros_like(S), 1.0, None)
    _, no, _, conv = o.iterate(False, 0.0, 1e-12, 5000)
    assert conv
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_state(np.zeros_like(S), 1.0, None)
    _, ng, _, convg = m.power_iterate(0.0, 1e-12, 5000, check_every=1)
    assert convg and ng == no
    assert _rel(m.get_state()[0], o.get_state()[0]) < 1e-9


def test_fp32_converged_error_is_small():
    prob = W.pin_cell_problem()
    o = _oracle(prob)
    ko, _, _, _ = o.iterate(True, 1e-10, 1e-10, 20000)
    phio, _ = o.get_state()
    errs = {}
    for prec in ("fp32", "fp32_plain"):
        m = moc.Moc.from_problem(prob, precision=prec)
        kg, ng, _, conv = m.power_iterate(1e-7, 1e-6, 20000, check_every=5)
        assert conv
        errs[prec] = (abs(kg - ko), _rel(m.get_state()[0], phio))
    assert errs["fp32"][0] < 0.5 * PCM and errs["fp32"][1] < 1e-4, errs


def test_checkpoint_resume_reproduces_iterates():
    prob = W.small_lattice_problem(3)
    a = moc.Moc.from_problem(prob, precision="fp64")
    a.outer(7)
    phi, k, psi = a.get_state(with_psi=True)
    a.outer(5)
    ref = a.get_state()
    b = moc.Moc.from_problem(prob, precision="fp64")
    b.set_state(phi, k, psi)
    b.outer(5)
    got = b.get_state()
    assert abs(got[1] - ref[1]) < 1e-13
    assert _rel(got[0], ref[0]) < 1e-11


def test_edge_cases():
    # two triangles, one group, one polar angle, vacuum: smallest problem
    mesh = W.grid_mesh(1, 1, 1.0, 1.0, bc=(0, 0, 0, 0))
    xs = W.CrossSections(np.array([[0.5]]), np.array([[0.9]]), np.array([[1.0]]), np.array([[[0.2]]]))
    prob = W.Problem(mesh, xs, 4, 0.3, sin_theta=np.array([0.8]), polar_w=np.array([1.0]))
    o = _oracle(prob)
    m = moc.Moc.from_problem(prob, precision="fp64")
    for _ in range(4):
        o.outer(True)
        m.outer(1)
    assert abs(m.get_state()[1] - o.get_state()[1]) < 1e-13
    # many groups (not a multiple of the padding), several polar angles, hexagonal mesh with gaps
    mesh = W.hex_core_mesh(n_sub=4, n_rings=1)
    xs = W.synthetic_xs(["fuel", "fuel", "coolant"], 33, 9, sigt_range=(0.05, 0.6))
    prob = W.Problem(mesh, xs, 12, 0.3)
    o = _oracle(prob)
    m = moc.Moc.from_problem(prob, precision="fp64")
    for _ in range(3):
        o.outer(True)
        m.outer(1)
    assert _rel(m.get_state()[0], o.get_state()[0]) < 1e-11
    # no ray crosses a tiny mesh in the corner of a big box -> geometry error, no crash
    tiny = W.grid_mesh(1, 1, 1e-3, 1e-3, bc=(0, 0, 0, 0))
    tiny.bbox = (0.0, 10.0, 0.0, 10.0)
    mm = moc.Moc(0, "fp64")
    mm.set_mesh(tiny)
    mm.set_quadrature(4, 1.0, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    with pytest.raises(moc.MocError) as e:
        mm.generate_tracks()
    assert e.value.code == -7


def test_status_codes_without_faults():
    prob = W.small_lattice_problem(3)
    m = moc.Moc.from_problem(prob, precision="fp64")
    k, n, r, conv = m.power_iterate(1e-14, 1e-14, 4, check_every=2, raise_on_fail=False)
    assert not conv and n == 4
    # eigenvalue mode without any fission: the k update is not finite -> status, not a fault
    xs = prob.xs
    m.set_xs(W.CrossSections(xs.sigma_t, np.zeros_like(xs.nu_sigma_f), xs.chi, xs.sigma_s))
    with pytest.raises(moc.MocError) as e:
        m.power_iterate(1e-6, 1e-6, 4, check_every=1)
    assert e.value.code == -6


def test_fp32_exponential_exhaustive():
    """Every FP32 tau in [0, 80]: relative error of the library's 1 - exp(-tau) against FP64."""
    lo = 0
    hi = int(np.array(80.0, np.float32).view(np.int32))
    worst = 0.0
    chunk = 1 << 24
    for start in range(lo, hi + 1, chunk):
        bits = np.arange(start, min(start + chunk, hi + 1), dtype=np.int32)
        tau = bits.view(np.float32)
        got32 = moc.eval_one_minus_exp_f32(tau)
        # the packed form (two values per f32x2 instruction, the many-group sweep's) is the same
        # function bit for bit
        np.testing.assert_array_equal(moc.eval_one_minus_exp_f32(tau, packed=True).view(np.int32),
                                      got32.view(np.int32))
        got = got32.astype(np.float64)
        ref = -np.expm1(-tau.astype(np.float64))
        nz = ref > 0
        err = np.abs(got[nz] - ref[nz]) / ref[nz]
        worst = max(worst, float(err.max()))
    # stated bound: 3 ulp of FP32 (2^-23 ~ 1.19e-7 per ulp)
    assert worst < 3 * 2.0 ** -23, worst
    print(f"max relative error of FP32 1-exp(-tau) over [0, 80]: {worst:.3e} ({worst / 2**-23:.2f} ulp)")


def test_assembly_full_size_fp64_and_fp32():
    """17x17 assembly at full size: 20 outers from the default state, GPU vs oracle."""
    prob = W.assembly_problem()
    o = _oracle(prob)
    o.normalise()
    for _ in range(20):
        o.outer(True)
    phio, ko = o.get_state()
    for prec, tk, tf in (("fp64", 2 * PCM, 1e-5), ("fp32", 2 * PCM, 2e-4)):
        m = moc.Moc.from_problem(prob, precision=prec)
        m.outer(20)
        phig, kg = m.get_state()
        print(prec, "dk", kg - ko, "max rel flux err", _rel(phig, phio))
        assert abs(kg - ko) <= tk
        assert _rel(phig, phio) <= tf


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_plain"])
def test_core_and_hex_geometries_reduced_quadrature(precision):
    """The 3x3-assembly core (vacuum on two sides, 7 groups) and the 19-hexagon core (vacuum,
    33 groups: the chunked FP32 kernel) at full mesh size with a coarse quadrature, 3 outers
    from the default state, GPU vs oracle."""
    tol = {"fp64": (1e-12, 1e-10), "fp32": (5e-6, 5e-5), "fp32_plain": (1e-5, 1e-4)}[precision]
    for prob in (W.core_problem(), W.hex_core_problem()):
        prob.n_azim, prob.ray_spacing = 8, 0.25
        o = _oracle(prob)
        o.normalise()
        for _ in range(3):
            o.outer(True)
        phio, ko = o.get_state()
        m = moc.Moc.from_problem(prob, precision=precision)
        m.outer(3)
        phig, kg = m.get_state()
        assert abs(kg - ko) <= tol[0] * ko, (prob.name, kg, ko)
        assert _rel(phig, phio) <= tol[1], (prob.name, _rel(phig, phio))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_core_full_size_sampled_regions(precision):
    """The 3x3-assembly core at full size (64 azimuths, 0.01 cm: 4.7e8 segments) in the launch
    configuration bench.py times: one fixed-source outer from a random state on the GPU, checked
    region by region against the oracle, which sweeps only the rays crossing the sampled regions."""
    prob = W.core_problem()
    xs = W.CrossSections(prob.xs.sigma_t, np.zeros_like(prob.xs.nu_sigma_f), prob.xs.chi, prob.xs.sigma_s)
    R, G = prob.mesh.n_tri, xs.n_groups
    rng = np.random.default_rng(17)
    S = rng.uniform(0.0, 1.0, (R, G))
    phi0 = rng.uniform(0.5, 1.5, (R, G))
    m = moc.Moc.from_problem(prob, precision=precision, with_xs=False)
    T, _ = m.track_counts()
    psi0 = rng.uniform(0.0, 0.2, (T, 2, 3, G))
    m.set_xs(xs)
    m.set_fixed_source(S)
    m.set_state(phi0, 1.0, psi0)
    m.outer(1)
    phig, _ = m.get_state()
    m.close()
    # regions spread over fuel, clad, moderator and reflector, plus the smallest ones
    by_mat = [rng.choice(np.nonzero(prob.mesh.mat == k)[0], 5, replace=False) for k in range(7)]
    sample = np.unique(np.concatenate(by_mat + [np.argsort(prob.mesh.areas())[:5]]))
    ref, area = oracle.sample_fixed_source(prob.mesh, prob.n_azim, prob.ray_spacing, prob.sin_theta,
                                           prob.polar_w, xs, S, phi0, psi0, sample)
    tol = 1e-10 if precision == "fp64" else 2e-5
    assert _rel(phig[sample], ref) <= tol, _rel(phig[sample], ref)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-5), ("fp32_plain", 2e-5)])
def test_hex_core_full_size_sampled_regions(precision, tol):
    """The 19-hexagon core at its benchmarked size (1.5M triangles, 33 groups, 48 azimuths, 0.02 cm:
    1.3e8 segments; FP32 runs the four-group chunked sweep), vacuum everywhere: one fixed-source
    outer from a random flux on the GPU, checked region by region against the oracle, which sweeps
    only the rays crossing the sampled regions (each in-mesh chord with zero inflow)."""
    prob = W.hex_core_problem()
    xs = W.CrossSections(prob.xs.sigma_t, np.zeros_like(prob.xs.nu_sigma_f), prob.xs.chi, prob.xs.sigma_s)
    R, G = prob.mesh.n_tri, xs.n_groups
    rng = np.random.default_rng(23)
    S = rng.uniform(0.0, 1.0, (R, G))
    phi0 = rng.uniform(0.5, 1.5, (R, G))
    m = moc.Moc.from_problem(prob, precision=precision, with_xs=False)
    m.set_xs(xs)
    m.set_fixed_source(S)
    m.set_state(phi0, 1.0, None)
    m.outer(1)
    phig, _ = m.get_state()
    m.close()
    # regions of every material, the smallest ones and ones at the core's outer edge
    by_mat = [rng.choice(np.nonzero(prob.mesh.mat == k)[0], 6, replace=False) for k in range(xs.n_mat)]
    c = prob.mesh.centroids()
    edge = np.argsort(-np.hypot(c[:, 0] - c[:, 0].mean(), c[:, 1] - c[:, 1].mean()))[:6]
    sample = np.unique(np.concatenate(by_mat + [np.argsort(prob.mesh.areas())[:6], edge]))
    ref, _ = oracle.sample_fixed_source(prob.mesh, prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w,
                                        xs, S, phi0, np.zeros((1, 2, 3, G)), sample)
    err = _rel(phig[sample], ref)
    print(precision, "sampled regions", sample.size, "max rel flux err", err)
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["fp32", "fp32_plain"])
@pytest.mark.parametrize("n_polar,G", [(1, 1), (2, 3), (4, 5), (3, 8), (3, 9), (3, 10), (3, 11), (3, 12), (3, 13)])
def test_fp32_kernel_variants(precision, n_polar, G):
    """Every FP32 sweep variant (polar counts without the specialised kernel, group counts on both
    sides of 8, and above it every remainder of G / 4: four-group lanes with tails of 1, 2, 3 or
    no groups) against the oracle after 4 outers, mixed boundary conditions."""
    sin_t = {1: [0.8], 2: [0.3, 0.85], 3: list(W.TY3_SIN_THETA), 4: [0.1, 0.4, 0.7, 0.95]}[n_polar]
    wts = {1: [1.0], 2: [0.4, 0.6], 3: list(W.TY3_WEIGHT), 4: [0.1, 0.2, 0.3, 0.4]}[n_polar]
    mesh = W.lattice_mesh(3, guide_tubes=False, bc=(1, 0, 1, 1))
    xs = W.synthetic_xs(["fuel", "clad", "moderator"], G, 40 + G)
    prob = W.Problem(mesh, xs, 12, 0.05, sin_theta=np.array(sin_t), polar_w=np.array(wts))
    o = _oracle(prob)
    o.normalise()
    m = moc.Moc.from_problem(prob, precision=precision)
    for _ in range(4):
        o.outer(True)
    m.outer(4)
    phio, ko = o.get_state()
    phig, kg = m.get_state()
    assert abs(kg - ko) <= 5e-6 * ko, (kg, ko)
    assert _rel(phig, phio) <= 1e-4, _rel(phig, phio)


@pytest.mark.parametrize("cell_size,omega", [(1.26, 1.0), (1.26, 1.6), (0.63, 1.4)])
def test_cmfd_outers_match_oracle_fp64(cell_size, omega):
    """Accelerated outers from the same random state, GPU FP64 vs oracle, compared after each
    (Gauss-Seidel and over-relaxed coarse sweeps; pin and half-pin cells)."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    cell, nc = W.grid_cells(prob.mesh, cell_size)
    o = _oracle(prob)
    o.set_cmfd(cell, nc, 5, 4, omega)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_cmfd(cell, nc, 5, 4, omega)
    rng = np.random.default_rng(8)
    T, _ = m.track_counts()
    phi0 = rng.uniform(0.5, 1.5, (prob.mesh.n_tri, prob.xs.n_groups))
    psi0 = rng.uniform(0.0, 0.2, (T, 2, 3, prob.xs.n_groups))
    o.set_state(phi0, 1.1, psi0)
    o.normalise()
    m.set_state(phi0, 1.1, psi0)
    for it in range(5):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        phig, _ = m.get_state()
        assert abs(kg - ko) <= 1e-10 * ko, (it, kg, ko)
        assert _rel(phig, phio) <= 1e-9, (it, _rel(phig, phio))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cmfd_converges_to_the_unaccelerated_solution(precision):
    prob = W.small_lattice_problem(5, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.04)
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    ref = moc.Moc.from_problem(prob, precision="fp64")
    kr, nr, _, cr = ref.power_iterate(1e-11, 1e-10, 50000, check_every=10)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_cmfd(cell, nc, 6, 6)
    tol = (1e-10, 1e-9) if precision == "fp64" else (1e-7, 1e-6)
    k, n, _, c = m.power_iterate(tol[0], tol[1], 50000, check_every=1)
    assert cr and c
    assert n < nr / 2, (n, nr)
    assert abs(k - kr) <= (1e-9 if precision == "fp64" else 2e-6) * kr
    assert _rel(m.get_state()[0], ref.get_state()[0]) <= (1e-7 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cmfd_early_stop_reaches_the_same_solution(precision):
    """The coarse power iteration stopped once k and the coarse source settle (a production mode):
    the converged solution is still the unaccelerated one, and the coarse iterations run are far
    fewer than the fixed count would run."""
    prob = W.small_lattice_problem(5, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.04)
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    ref = moc.Moc.from_problem(prob, precision="fp64")
    kr, _, _, cr = ref.power_iterate(1e-11, 1e-10, 50000, check_every=10)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_cmfd(cell, nc, 60, 6)
    m.set_cmfd_tolerance(1e-9 if precision == "fp64" else 1e-6)
    m.set_state(None, 1.0)
    tol = (1e-10, 1e-9) if precision == "fp64" else (1e-7, 1e-6)
    k, n, _, c = m.power_iterate(tol[0], tol[1], 50000, check_every=1)
    used = m.cmfd_iterations()
    assert cr and c
    assert used < 60 * n / 2, (used, n)
    assert abs(k - kr) <= (1e-9 if precision == "fp64" else 2e-6) * kr
    assert _rel(m.get_state()[0], ref.get_state()[0]) <= (1e-7 if precision == "fp64" else 1e-4)
    with pytest.raises(moc.MocError):
        m.set_cmfd_tolerance(-1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cmfd_reflector_core_converges_to_the_oracle(precision):
    """One assembly with the reflector band, pin-size coarse cells, reflective -x/-y: the
    accelerated GPU iteration converges to the oracle's accelerated limit, which the oracle pins
    as a fixed point of the plain transport iteration."""
    xs = W.synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, 4,
                        fuel_scales=[1.0, 0.95, 1.05, 0.9])
    prob = W.Problem(W.core_mesh(1), xs, 16, 0.2, tol=1e-6, name="core1", seed=4)
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    o = _oracle(prob)
    o.set_cmfd(cell, nc, 20, 20)
    ko, _, _, co = o.iterate(True, 1e-11, 1e-9, 80)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_cmfd(cell, nc, 20, 20)
    tol = (1e-11, 1e-9) if precision == "fp64" else (1e-7, 2e-6)
    k, n, r, c = m.power_iterate(tol[0], tol[1], 400, check_every=1)
    assert co and c, (n, r)
    assert abs(k - ko) <= (1e-9 if precision == "fp64" else 2e-6) * ko, (k, ko)
    assert _rel(m.get_state()[0], o.get_state()[0]) <= (1e-7 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_back_projection_outers_match_oracle(precision, tol):
    """Back-projected rays on the concave 7-hexagon cluster (vacuum): outers from the same random
    state, GPU vs oracle, compared after each."""
    mesh = W.hex_core_mesh(n_sub=4, n_rings=1)
    xs = W.synthetic_xs(["fuel", "fuel", "coolant"], 7, 9, sigt_range=(0.05, 0.6))
    prob = W.Problem(mesh, xs, 12, 0.3, ray_layout=1)
    o = _oracle(prob)
    m = moc.Moc.from_problem(prob, precision=precision)
    rng = np.random.default_rng(21)
    phi0 = rng.uniform(0.5, 1.5, (mesh.n_tri, 7))
    o.set_state(phi0, 1.05, None)
    o.normalise()
    m.set_state(phi0, 1.05, None)
    for it in range(4):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        assert abs(kg - ko) <= tol * ko, (it, kg, ko)
        assert _rel(m.get_state()[0], phio) <= 10 * tol, (it, _rel(m.get_state()[0], phio))


def test_cmfd_full_assembly_outers_match_oracle():
    """The bench's full-size assembly with CMFD on its 289 pin cells: 3 accelerated outers from the
    cold start, GPU FP64 vs oracle after each."""
    prob = W.assembly_problem()
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    o = _oracle(prob)
    o.set_cmfd(cell, nc, 6, 6, 1.0)
    o.normalise()
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_cmfd(cell, nc, 6, 6, 1.0)
    for it in range(3):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        assert abs(kg - ko) <= 1e-10 * ko, (it, kg, ko)
        assert _rel(m.get_state()[0], phio) <= 1e-9, (it, _rel(m.get_state()[0], phio))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_cmfd_cluster_solve_matches_oracle(precision, tol):
    """4,624 half-pin coarse cells (one assembly + reflector band): the coarse solve runs on a
    thread-block cluster; 3 accelerated outers from the cold start vs the oracle."""
    xs = W.synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, 4,
                        fuel_scales=[1.0, 0.95, 1.05, 0.9])
    prob = W.Problem(W.core_mesh(1), xs, 16, 0.2, tol=1e-6, name="core1", seed=4)
    cell, nc = W.grid_cells(prob.mesh, 0.63)
    assert nc >= 1024
    o = _oracle(prob)
    o.set_cmfd(cell, nc, 5, 3, 1.4)
    o.normalise()
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_cmfd(cell, nc, 5, 3, 1.4)
    for it in range(3):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        phig = m.get_state()[0]
        assert abs(kg - ko) <= tol * ko, (it, kg, ko)
        # the reflector's far corner holds fluxes 1e-9 of the peak: relative to max(|phi|, 1e-6 peak)
        err = float(np.max(np.abs(phig - phio) / np.maximum(np.abs(phio), 1e-6 * np.abs(phio).max())))
        assert err <= 10 * tol, (it, err)
