"""Pins of the oracle's DGMOC (Sec. 2.2 DGMOC formulation, Alg. 2) against facts fixed outside it:
the matrix exponential of a library, the exact solution of the segment's linear system, the
analytic slab solution and a fine-mesh slab transport solver the method must converge to, the
infinite-medium multiplication factor, global neutron balance and the planar limit."""
import numpy as np
import pytest

import oracle
from paper_2607_01591_gb300 import workloads as W

MU = np.sqrt(1.0 - W.TY3_SIN_THETA ** 2)


def test_expm2_matches_scipy():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    for _ in range(40):
        M = rng.normal(size=(2, 2)) * rng.uniform(0.01, 8.0)
        R = sl.expm(M)
        np.testing.assert_allclose(oracle.expm2(M), R, rtol=1e-12, atol=1e-13 * np.abs(R).max())
    # the DG operator's form (complex eigenvalues, damped rotation), thin to optically thick
    for c, l in ((3.0, 0.7), (0.05, 0.01), (20.0, 2.0), (0.5, 30.0)):
        K = np.array([[1 + c, c], [-3 * c, 1 + 3 * c]])
        R = sl.expm(-l * K)
        np.testing.assert_allclose(oracle.expm2(-l * K), R, rtol=1e-10, atol=1e-11 * np.abs(R).max() + 1e-300)


def test_segment_solves_its_linear_system():
    """y' = r - K y along the segment with the system of the DG weak form (upwind inflow psi_in):
    the end value and the integral agree with a tight numerical integration."""
    si = pytest.importorskip("scipy.integrate")
    st, mu, h, sig, q0, q1, psi_in, L = 0.537707, MU[1], 0.8, 1.3, 0.4, -0.15, 0.9, 0.37
    c = mu / h
    K = np.array([[sig + c, c], [-3 * c, sig + 3 * c]]) / st
    r = np.array([q0 + c * psi_in, q1 - 3 * c * psi_in]) / st
    y0 = np.array([0.6, 0.2])

    def f(s, z):
        return np.concatenate([r - K @ z[:2], z[:2]])

    sol = si.solve_ivp(f, (0.0, L), np.concatenate([y0, [0.0, 0.0]]), rtol=1e-12, atol=1e-14, method="DOP853")
    y1, yi = oracle.dg_segment(y0, psi_in, L, st, mu, h, sig, q0, q1)
    np.testing.assert_allclose(y1, sol.y[:2, -1], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(yi, sol.y[2:, -1], rtol=1e-10, atol=1e-13)


def _slab_oracle(Nz, sig, c, Z=4.0, S=1.0):
    mesh = W.grid_mesh(1, 1, 4.0, 4.0, bc=(1, 1, 1, 1))
    xs = W.CrossSections(np.array([[sig]]), np.zeros((1, 1)), np.zeros((1, 1)), np.array([[[c * sig]]]))
    o = oracle.Oracle(mesh, 8, 0.5, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    o.set_fixed_source(np.full((mesh.n_tri, 1), S))
    o.set_axial(np.full(Nz, Z / Nz), bc=(0, 0))
    _, _, _, ok = o.iterate(eigen=False, tol_f=1e-13, max_outer=3000)
    assert ok
    phi, _ = o.flux3()
    # x-y uniform: every region of a plane has the same moments
    np.testing.assert_allclose(phi[:, 1], phi[:, 0], rtol=1e-12, atol=1e-14)
    return phi[:, 0, :, 0]


def _plane_moments(zf, phif, Nz, Z):
    """plane average and Legendre (xi) coefficient of a finely resolved profile"""
    out = np.zeros((Nz, 2))
    h = Z / Nz
    for i in range(Nz):
        m = (zf >= i * h) & (zf < (i + 1) * h)
        xi = (zf[m] - (i + 0.5) * h) / (0.5 * h)
        out[i, 0] = phif[m].mean()
        out[i, 1] = 1.5 * 2.0 * np.mean(phif[m] * xi)
    return out


def test_slab_absorber_converges_to_the_analytic_solution():
    """x-y uniform, reflective sides, vacuum top and bottom, pure absorber with a uniform source:
    the discrete-ordinates slab solution is psi = q/sig (1 - exp(-sig z/mu)) upward (z from the top
    downward). The DG moments converge to its plane moments at second order."""
    Z, sig = 4.0, 1.0
    q = 1.0 / (4 * np.pi)
    x, wq = np.polynomial.legendre.leggauss(40)
    errs = []
    for Nz in (8, 16, 32, 64):
        phi = _slab_oracle(Nz, sig, 0.0, Z)
        h = Z / Nz
        ref = np.zeros((Nz, 2))
        for i in range(Nz):
            z = i * h + (x + 1) * h / 2
            f = sum(2 * np.pi * w * (q / sig) * (2 - np.exp(-sig * z / m) - np.exp(-sig * (Z - z) / m))
                    for w, m in zip(W.TY3_WEIGHT, MU))
            ref[i] = 0.5 * np.sum(wq * f), 1.5 * np.sum(wq * f * x)
        errs.append(np.abs(phi - ref).max(axis=0) / ref[:, 0].max())
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order[1:, 0] >= 1.9), errs          # plane averages
    assert np.all(order[1:, 1] >= 1.5), errs          # linear moments
    assert errs[-1, 0] < 5e-5 and errs[-1, 1] < 2e-3


def _fine_slab(sig, c, Z=4.0, S=1.0, n=8192):
    """Slab discrete ordinates with the same polar set, step characteristics on a fine mesh,
    source iteration to convergence (an independent textbook solver). Cell-edge fluxes follow
    the linear recurrence psi_{i+1} = e^{-x} psi_i + (q_i/sig)(1 - e^{-x}), x = sig h/mu; the cell
    average is q/sig + (psi_in - q/sig)(1 - e^{-x})/x."""
    sg = pytest.importorskip("scipy.signal")
    h = Z / n
    phi = np.zeros(n)
    for _ in range(400):
        q = (c * sig * phi + S) / (4 * np.pi)
        new = np.zeros(n)
        for w, m in zip(W.TY3_WEIGHT, MU):
            x = sig * h / m
            a, f = np.exp(-x), -np.expm1(-x)
            for qq in (q, q[::-1]):
                edge = sg.lfilter([0.0, f], [1.0, -a], qq / sig)        # psi entering cell i
                avg = qq / sig + (edge - qq / sig) * f / x
                new += 2 * np.pi * w * (avg if qq is q else avg[::-1])
        if np.max(np.abs(new - phi)) <= 1e-12 * np.max(new):
            return (np.arange(n) + 0.5) * h, new
        phi = new
    raise AssertionError("fine slab solver did not converge")


def test_slab_with_scattering_converges_to_a_fine_transport_solution():
    Z, sig, c = 4.0, 1.0, 0.6
    zf, pf = _fine_slab(sig, c, Z)
    errs = []
    for Nz in (16, 32, 64):
        phi = _slab_oracle(Nz, sig, c, Z)
        ref = _plane_moments(zf, pf, Nz, Z)
        errs.append(np.abs(phi - ref).max(axis=0) / ref[:, 0].max())
    errs = np.array(errs)
    assert np.all(np.log2(errs[0] / errs[1]) >= 1.5) and np.all(np.log2(errs[1] / errs[2]) >= 1.5), errs
    assert errs[-1, 0] < 1e-4 and errs[-1, 1] < 3e-3


def test_infinite_medium_keeps_k_inf():
    xs = W.synthetic_xs(["fuel"], 4, seed=7)
    mesh = W.one_material(W.grid_mesh(2, 2, 2.0, 2.0, bc=(1, 1, 1, 1)))
    o = oracle.Oracle(mesh, 8, 0.2, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    o.set_axial(np.array([0.5, 1.0, 0.7]), bc=(1, 1))
    k, n, r, ok = o.iterate(tol_k=1e-12, tol_f=1e-11, max_outer=400)
    M = np.diag(xs.sigma_t[0]) - xs.sigma_s[0].T
    kinf = float(xs.nu_sigma_f[0] @ np.linalg.solve(M, xs.chi[0]))
    assert ok and abs(k - kinf) < 1e-10
    phi, _ = o.flux3()
    assert np.abs(phi[:, :, 1]).max() < 1e-12                      # no axial slope
    np.testing.assert_allclose(phi[:, :, 0], np.broadcast_to(phi[0, 0, 0], phi[:, :, 0].shape), rtol=1e-10)


def _lattice3d(nz_mats=True):
    prob = W.small_lattice_problem(3, bc=(0, 0, 0, 0), n_azim=8, ray_spacing=0.2)
    o = oracle.Oracle.from_problem(prob, threads=8)
    mat3 = np.tile(prob.mesh.mat, (3, 1))
    if nz_mats:
        mat3[-1] = prob.mesh.mat.max()
    return prob, o, mat3


def test_global_balance_with_vacuum_boundaries():
    """At convergence: production / k = absorption + radial, bottom and top leakage."""
    prob, o, mat3 = _lattice3d()
    dz = np.array([1.0, 2.0, 1.0])
    o.set_axial(dz, mat3, bc=(0, 0))
    k, n, r, ok = o.iterate(tol_k=1e-11, tol_f=1e-9, max_outer=2000)
    assert ok
    phi, _ = o.flux3()
    A, xs = o.areas(), prob.xs
    absr = prod = 0.0
    for z in range(3):
        for i in range(prob.mesh.n_tri):
            m, ph = mat3[z, i], phi[z, i, 0]
            absr += A[i] * dz[z] * (xs.sigma_t[m] - xs.sigma_s[m].sum(1)) @ ph
            prod += A[i] * dz[z] * xs.nu_sigma_f[m] @ ph
    L = o.leakage3()
    assert np.all(L > 0)
    assert abs(prod / k - absr - L.sum()) <= 5e-9 * prod / k


def test_symmetric_stack_gives_symmetric_moments():
    """vacuum top and bottom, materials mirrored about the mid-plane: plane averages mirror, the
    linear moments change sign"""
    prob, o, mat3 = _lattice3d(False)
    mat3[0] = mat3[2] = prob.mesh.mat.max()
    o.set_axial(np.array([0.7, 1.5, 0.7]), mat3, bc=(0, 0))
    for _ in range(6):
        o.outer()
    phi, _ = o.flux3()
    np.testing.assert_allclose(phi[2, :, 0], phi[0, :, 0], rtol=1e-12)
    np.testing.assert_allclose(phi[2, :, 1], -phi[0, :, 1], rtol=1e-10, atol=1e-14)
    assert np.abs(phi[1, :, 1]).max() < 1e-12 * np.abs(phi[1, :, 0]).max()


def test_thick_planes_approach_the_planar_method():
    """One plane with reflective top and bottom: as the plane grows thick the axial coupling
    (mu/dz) vanishes and k tends to the planar method's."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=8, ray_spacing=0.2)
    o2 = oracle.Oracle.from_problem(prob, threads=8)
    k2, _, _, ok2 = o2.iterate(tol_k=1e-11, tol_f=1e-9, max_outer=2000)
    diffs = []
    for h in (10.0, 1000.0):
        o = oracle.Oracle.from_problem(prob, threads=8)
        o.set_axial(np.array([h]), bc=(1, 1))
        k, _, _, ok = o.iterate(tol_k=1e-11, tol_f=1e-9, max_outer=2000)
        assert ok
        diffs.append(abs(k - k2))
    assert ok2 and diffs[1] < 1e-6 and diffs[1] < diffs[0] / 30


def _pin_stack(nz=4, h=3.0, bc=(0, 0)):
    pin = W.pin_cell_problem()
    prob = W.Problem(pin.mesh, pin.xs, 8, 0.1)
    o = oracle.Oracle.from_problem(prob, threads=8)
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[-1] = prob.mesh.mat.max()
    o.set_axial(np.full(nz, h), mat3, bc=bc)
    return o


def test_axial_acceleration_converges_to_the_transport_solution():
    """The accelerated iteration's limit is a fixed point of the plain DGMOC iteration (the coarse
    operator reproduces the sweep's currents, so it changes nothing at the transport solution),
    and it gets there in far fewer outers than the plain iteration."""
    o = _pin_stack(bc=(1, 0))
    o.set_dg_cmfd(8, 4, 1.0)
    k, n_acc, r, ok = o.iterate(tol_k=1e-12, tol_f=1e-10, max_outer=2000)
    assert ok
    phi, _ = o.flux3()
    o.set_dg_cmfd(0)
    o.outer()
    phi1, k1 = o.flux3()
    assert abs(k1 - k) <= 1e-10 and np.abs(phi1 - phi).max() <= 1e-9 * np.abs(phi).max()
    p = _pin_stack(bc=(1, 0))
    kp, n_plain, _, okp = p.iterate(tol_k=1e-12, tol_f=1e-10, max_outer=5000)
    assert okp and abs(kp - k) <= 1e-10
    assert n_acc * 3 < n_plain, (n_acc, n_plain)
