"""Pins of the CPU oracle against facts other than itself (no GPU).

Each test checks the oracle against mathematics or geometry it does not compute the same way:
closed-form infinite-medium eigenvalues and fluxes, exact path integrals evaluated in extended
precision, an independent brute-force segmentation, direct angular/spatial integration of the
exact characteristic solution, global neutron balance, and mirror symmetry.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2607_01591_gb300 import workloads as W

FOUR_PI = 4.0 * math.pi


def _xs_one(G, seed, kind="fuel"):
    xs = W.synthetic_xs([kind], G, seed)
    return xs


def _closed_form_kinf(xs, m=0):
    """k_inf = nuSigma_f^T (diag Sigma_t - S^T)^{-1} chi, S[g'][g] = Sigma_s g'->g."""
    M = np.diag(xs.sigma_t[m]) - xs.sigma_s[m].T
    spec = np.linalg.solve(M, xs.chi[m])
    return float(xs.nu_sigma_f[m] @ spec), spec


# ------------------------------------------------------------------------------ quadrature

def test_azimuthal_weights_and_spacing():
    mesh = W.pin_cell_mesh()
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    q = o.quadrature()
    # weights over the full 2 pi set (each stored direction stands for itself and its reverse)
    assert abs(2.0 * q["omega"].sum() - 1.0) < 1e-14
    np.testing.assert_allclose(q["omega"], q["omega"][::-1], rtol=1e-13)      # phi <-> pi - phi
    # cyclic condition: tan(phi) = H nx / (W ny); spacing no larger than requested
    Wd = mesh.bbox[1] - mesh.bbox[0]
    np.testing.assert_allclose(np.tan(q["phi"][:4]), Wd * q["nx"][:4] / (Wd * q["ny"][:4]), rtol=1e-13)
    assert (q["delta"] <= 0.05 + 1e-15).all()
    # the azimuthal quadrature integrates cos^2 over the circle to ~1/2
    phis = np.concatenate([q["phi"], q["phi"] + math.pi])
    om = np.concatenate([q["omega"], q["omega"]])
    assert abs((om * np.cos(phis) ** 2).sum() - 0.5) < 5e-3


def test_polar_set_is_a_hemisphere_quadrature():
    # weights normalised to one hemisphere; mean of sin(theta) over the hemisphere is pi/4
    assert abs(W.TY3_WEIGHT.sum() - 1.0) < 1e-6
    assert abs((W.TY3_WEIGHT * W.TY3_SIN_THETA).sum() - math.pi / 4) < 1e-4


# ------------------------------------------------------------------------------ geometry

def _track_lines(o):
    q = o.quadrature()
    tr = o.tracks()
    return q, tr


def test_parallel_track_spacing_matches_effective_spacing():
    mesh = W.pin_cell_mesh()
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    q, tr = _track_lines(o)
    xmin, xmax, ymin, ymax = mesh.bbox
    corners = np.array([[xmin, ymin], [xmax, ymin], [xmin, ymax], [xmax, ymax]])
    for j in range(o.n_dir):
        sel = tr["track_dir"] == j
        assert sel.sum() == q["nx"][j] + q["ny"][j]
        ph = q["phi"][j]
        nrm = np.array([-math.sin(ph), math.cos(ph)])
        u = np.array([math.cos(ph), math.sin(ph)])
        st = tr["track_xy"][sel, :2]
        en = tr["track_xy"][sel, 2:]
        d = en - st
        # every track runs along its direction
        np.testing.assert_allclose(d / np.linalg.norm(d, axis=1)[:, None], np.tile(u, (sel.sum(), 1)), atol=1e-12)
        c = np.sort(st @ nrm)
        np.testing.assert_allclose(np.diff(c), q["delta"][j], rtol=1e-9)
        # the family covers the box: first/last offsets half a spacing inside the box's extent
        cc = corners @ nrm
        assert abs(c[0] - cc.min() - q["delta"][j] / 2) < 1e-9
        assert abs(cc.max() - c[-1] - q["delta"][j] / 2) < 1e-9


def _brute_force_pieces(mesh, p0, u, L):
    """Segmentation by a different algorithm: intersect the line with every mesh edge, sort the
    crossing parameters, and classify each sub-interval by locating its midpoint."""
    tri = mesh.tri
    xy = mesh.xy
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.unique(np.sort(e, 1), axis=0)
    a = xy[e[:, 0]]
    b = xy[e[:, 1]]
    dvec = b - a
    den = u[0] * dvec[:, 1] - u[1] * dvec[:, 0]
    ap = a - p0
    ok = den != 0
    s = np.where(ok, (ap[:, 0] * dvec[:, 1] - ap[:, 1] * dvec[:, 0]) / np.where(ok, den, 1), np.nan)
    t = np.where(ok, (ap[:, 0] * u[1] - ap[:, 1] * u[0]) / np.where(ok, den, 1), np.nan)
    hit = ok & (t >= -1e-12) & (t <= 1 + 1e-12) & (s > 0) & (s < L)
    cuts = np.unique(np.concatenate([[0.0, L], s[hit]]))
    P = xy[tri]
    pieces = []
    for s0, s1 in zip(cuts[:-1], cuts[1:]):
        if s1 - s0 < 1e-12:
            continue
        m = p0 + 0.5 * (s0 + s1) * u
        c0 = (P[:, 1, 0] - P[:, 0, 0]) * (m[1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (m[0] - P[:, 0, 0])
        c1 = (P[:, 2, 0] - P[:, 1, 0]) * (m[1] - P[:, 1, 1]) - (P[:, 2, 1] - P[:, 1, 1]) * (m[0] - P[:, 1, 0])
        c2 = (P[:, 0, 0] - P[:, 2, 0]) * (m[1] - P[:, 2, 1]) - (P[:, 0, 1] - P[:, 2, 1]) * (m[0] - P[:, 2, 0])
        inside = np.nonzero((c0 > 0) & (c1 > 0) & (c2 > 0))[0]
        assert len(inside) <= 1
        pieces.append((s0, s1, int(inside[0]) if len(inside) else -1))
    # merge consecutive pieces in the same triangle
    merged = []
    for p in pieces:
        if merged and merged[-1][2] == p[2]:
            merged[-1] = (merged[-1][0], p[1], p[2])
        else:
            merged.append(p)
    return merged


@pytest.mark.parametrize("which", ["grid", "pin", "hex7", "hex7_back_projection", "pin_back_projection"])
def test_segmentation_matches_brute_force(which):
    if which == "grid":
        mesh = W.grid_mesh(2, 2, 1.0, 1.0)
        o = oracle.Oracle(mesh, 8, 0.15, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    elif which == "pin":
        mesh = W.pin_cell_mesh()
        o = oracle.Oracle(mesh, 8, 0.1, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    elif which == "pin_back_projection":
        mesh = W.with_bc(W.pin_cell_mesh(), (0, 0, 0, 0))
        o = oracle.Oracle(mesh, 12, 0.1, W.TY3_SIN_THETA, W.TY3_WEIGHT, ray_layout=1)
    else:
        mesh = W.hex_core_mesh(n_sub=2, n_rings=1)     # 7 hexagons: concave outline, gaps in rays
        o = oracle.Oracle(mesh, 8 if which == "hex7" else 12, 1.0, W.TY3_SIN_THETA, W.TY3_WEIGHT,
                          ray_layout=0 if which == "hex7" else 1)
    q, tr = _track_lines(o)
    xmin, xmax, ymin, ymax = mesh.bbox
    n_checked = 0
    for t in range(o.n_tracks):
        j = tr["track_dir"][t]
        ph = q["phi"][j]
        u = np.array([math.cos(ph), math.sin(ph)])
        st = tr["track_xy"][t, :2]
        # extend the track's line to the whole box
        sb = []
        for (lim, comp) in ((xmin, 0), (xmax, 0), (ymin, 1), (ymax, 1)):
            if u[comp] != 0:
                sb.append((lim - st[comp]) / u[comp])
        sb = np.array(sb)
        s_back = sb[sb <= 1e-12].max()
        s_fwd = sb[sb >= -1e-12]
        p0 = st + s_back * u
        L = min(x for x in (sb - s_back) if x > 1e-9)
        pieces = _brute_force_pieces(mesh, p0, u, L)
        # find the run of in-mesh pieces that starts at this track's start
        s_start = -s_back
        runs, cur = [], []
        for p in pieces:
            if p[2] < 0:
                if cur:
                    runs.append(cur)
                cur = []
            else:
                cur.append(p)
        if cur:
            runs.append(cur)
        run = [r for r in runs if abs(r[0][0] - s_start) < 1e-9]
        assert len(run) == 1, (t, s_start, [r[0][0] for r in runs])
        run = run[0]
        s0, s1 = tr["seg_off"][t], tr["seg_off"][t + 1]
        reg = tr["seg_region"][s0:s1]
        ln = tr["seg_len"][s0:s1]
        assert list(reg) == [p[2] for p in run]
        np.testing.assert_allclose(ln, [p[1] - p[0] for p in run], rtol=0, atol=1e-11)
        n_checked += 1
    assert n_checked == o.n_tracks


def _reflect(u, wall):
    v = u.copy()
    if wall <= 1:
        v[0] = -v[0]
    else:
        v[1] = -v[1]
    return v


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 0, 1, 0), (0, 0, 0, 0)])
def test_links_reflect_at_walls(bc):
    mesh = W.with_bc(W.pin_cell_mesh(), bc)
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    q, tr = _track_lines(o)
    xmin, xmax, ymin, ymax = mesh.bbox
    link = tr["link"]
    seen = np.zeros(2 * o.n_tracks, int)
    for t in range(o.n_tracks):
        ph = q["phi"][tr["track_dir"][t]]
        for d in range(2):
            u = np.array([math.cos(ph), math.sin(ph)]) * (1 if d == 0 else -1)
            out_pt = tr["track_xy"][t, 2:] if d == 0 else tr["track_xy"][t, :2]
            wall = int(np.argmin([abs(out_pt[0] - xmin), abs(out_pt[0] - xmax), abs(out_pt[1] - ymin), abs(out_pt[1] - ymax)]))
            e = link[t, d]
            if bc[wall] == 0:
                assert e == -1
                continue
            assert e >= 0
            seen[e] += 1
            t2, d2 = divmod(int(e), 2)
            ph2 = q["phi"][tr["track_dir"][t2]]
            u2 = np.array([math.cos(ph2), math.sin(ph2)]) * (1 if d2 == 0 else -1)
            in_pt = tr["track_xy"][t2, :2] if d2 == 0 else tr["track_xy"][t2, 2:]
            np.testing.assert_allclose(in_pt, out_pt, atol=1e-12)
            np.testing.assert_allclose(u2, _reflect(u, wall), atol=1e-12)
    assert seen.max() <= 1
    if all(b == 1 for b in bc):
        assert (seen == 1).all()          # a bijection of track ends


def test_back_projection_quadrature_and_ray_offsets():
    """Back projection: nominal angles, equal weights, and per direction n = ceil(extent/delta)
    parallel rays at offsets (i + 1/2) * extent/n across the mesh's projection on the normal."""
    mesh = W.grid_mesh(3, 2, 1.5, 1.0, bc=(0, 0, 0, 0))      # convex: every ray crosses the mesh
    A, sp = 12, 0.07
    o = oracle.Oracle(mesh, A, sp, W.TY3_SIN_THETA, W.TY3_WEIGHT, ray_layout=1)
    q, tr = _track_lines(o)
    np.testing.assert_allclose(q["phi"], 2 * math.pi * (np.arange(A // 2) + 0.5) / A, rtol=1e-15)
    np.testing.assert_allclose(q["omega"], 1.0 / A, rtol=1e-13)
    for j in range(o.n_dir):
        ph = q["phi"][j]
        nrm = np.array([-math.sin(ph), math.cos(ph)])
        ext = mesh.xy @ nrm
        n = math.ceil((ext.max() - ext.min()) / sp)
        assert abs(q["delta"][j] - (ext.max() - ext.min()) / n) < 1e-13 and q["delta"][j] <= sp
        sel = tr["track_dir"] == j
        assert sel.sum() == n
        c = np.sort(tr["track_xy"][sel, :2] @ nrm)
        np.testing.assert_allclose(c, ext.min() + (np.arange(n) + 0.5) * q["delta"][j], rtol=0, atol=1e-12)
        # every track spans the mesh: it starts and ends on the mesh outline
        for st in tr["track_xy"][sel]:
            for x, y in (st[:2], st[2:]):
                assert min(abs(x - 0.0), abs(x - 1.5), abs(y - 0.0), abs(y - 1.0)) < 1e-12


def test_back_projection_areas_converge():
    mesh = W.with_bc(W.pin_cell_mesh(), (0, 0, 0, 0))
    exact = mesh.areas()
    errs = []
    for sp in (0.05, 0.01, 0.002):
        o = oracle.Oracle(mesh, 16, sp, W.TY3_SIN_THETA, W.TY3_WEIGHT, ray_layout=1)
        errs.append(np.abs(o.areas() / exact - 1).max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


def test_back_projection_needs_vacuum_walls():
    with pytest.raises(RuntimeError):
        oracle.Oracle(W.pin_cell_mesh(), 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT, ray_layout=1)


def test_tracked_area_total_and_convergence():
    mesh = W.pin_cell_mesh()
    exact = mesh.areas()
    errs = []
    for sp in (0.05, 0.01, 0.002):
        o = oracle.Oracle(mesh, 16, sp, W.TY3_SIN_THETA, W.TY3_WEIGHT)
        a = o.areas()
        # cyclic tracks cover the box exactly: the total equals the box area
        assert abs(a.sum() / exact.sum() - 1) < 1e-13
        errs.append(np.abs(a / exact - 1).max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


# ------------------------------------------------------------------------------ characteristics

def test_track_sweep_matches_exact_path_integral():
    rng = np.random.default_rng(7)
    mpmath.mp.dps = 40
    for trial in range(20):
        n = int(rng.integers(1, 30))
        sig = rng.uniform(0.01, 3.0, n)
        ln = 10 ** rng.uniform(-7, 0.5, n)
        qr = rng.uniform(0.0, 2.0, n)
        sin_t = float(rng.choice(W.TY3_SIN_THETA))
        psi0 = float(rng.uniform(0, 3))
        got = oracle.track_sweep(sig, qr, ln, sin_t, psi0)
        tau = [mpmath.mpf(float(s)) * mpmath.mpf(float(l)) / mpmath.mpf(sin_t) for s, l in zip(sig, ln)]
        for k in range(n):
            # psi after segment k = psi0 e^{-sum tau} + sum_m qr_m (1 - e^{-tau_m}) e^{-sum_{m<j<=k} tau_j}
            tot = mpmath.mpf(psi0) * mpmath.exp(-mpmath.fsum(tau[:k + 1]))
            for m in range(k + 1):
                tot += mpmath.mpf(float(qr[m])) * (1 - mpmath.exp(-tau[m])) * mpmath.exp(-mpmath.fsum(tau[m + 1:k + 1]))
            assert abs(got[k] - float(tot)) <= 1e-14 * max(1.0, abs(float(tot))), (trial, k)


def test_one_sweep_flux_equals_direct_angular_integration():
    """phi after one sweep from zero inflow equals the direct integral of the exact angular flux:
    phi_i = (1/A_i) sum_{a,p} 4 pi omega_a w_p delta_a sum_{k in i} int_segment psi ds."""
    mesh = W.grid_mesh(2, 2, 1.0, 1.0, bc=(0, 0, 0, 0), mat_fn=lambda i, j: (i + j) % 2)
    G = 2
    xs = W.CrossSections(np.array([[1.3, 0.7], [0.4, 2.2]]), np.zeros((2, G)), np.zeros((2, G)),
                         np.zeros((2, G, G)))
    S = np.random.default_rng(3).uniform(0.5, 2.0, (mesh.n_tri, G))
    o = oracle.Oracle(mesh, 8, 0.2, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    o.set_fixed_source(S)
    o.set_state(np.zeros((mesh.n_tri, G)), 1.0, None)
    o.outer(eigen=False)
    phi, _ = o.get_state()
    q, tr = _track_lines(o)
    area = o.areas()
    Q = S / FOUR_PI
    num = np.zeros((mesh.n_tri, G))
    for t in range(o.n_tracks):
        j = tr["track_dir"][t]
        segs = list(zip(tr["seg_region"][tr["seg_off"][t]:tr["seg_off"][t + 1]],
                        tr["seg_len"][tr["seg_off"][t]:tr["seg_off"][t + 1]]))
        for d in range(2):
            order = segs if d == 0 else segs[::-1]
            for p, (sn, wp) in enumerate(zip(W.TY3_SIN_THETA, W.TY3_WEIGHT)):
                for g in range(G):
                    taus = [xs.sigma_t[mesh.mat[r], g] * l / sn for r, l in order]
                    for k, (r, l) in enumerate(order):
                        # entering flux by the explicit sum over upstream segments
                        psi_k = 0.0
                        for m in range(k):
                            rm = order[m][0]
                            sm = xs.sigma_t[mesh.mat[rm], g]
                            psi_k += Q[rm, g] / sm * (1 - math.exp(-taus[m])) * math.exp(-sum(taus[m + 1:k]))
                        sg = xs.sigma_t[mesh.mat[r], g]
                        f = lambda x: psi_k * math.exp(-sg * x / sn) + Q[r, g] / sg * (1 - math.exp(-sg * x / sn))
                        val, _ = integrate.quad(f, 0.0, l, epsabs=1e-15, epsrel=1e-13)
                        num[r, g] += FOUR_PI * q["omega"][j] * wp * q["delta"][j] * val
    ref = num / area[:, None]
    np.testing.assert_allclose(phi, ref, rtol=1e-10)


# ------------------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("G,seed", [(1, 11), (7, 12)])
def test_infinite_medium_eigenvalue(G, seed):
    mesh = W.one_material(W.pin_cell_mesh())
    xs = _xs_one(G, seed)
    kinf, spec = _closed_form_kinf(xs)
    if G == 1:
        # one group: k = nuSigma_f / (Sigma_t - Sigma_s)
        assert abs(kinf - xs.nu_sigma_f[0, 0] / (xs.sigma_t[0, 0] - xs.sigma_s[0, 0, 0])) < 1e-13
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    k, n, r, conv = o.iterate(True, 1e-13, 1e-12, 20000)
    assert conv
    assert abs(k - kinf) < 1e-10
    phi, _ = o.get_state()
    # spatially flat, with the infinite-medium spectrum
    np.testing.assert_allclose(phi, np.tile(phi[0], (mesh.n_tri, 1)), rtol=1e-10)
    np.testing.assert_allclose(phi[0] / phi[0].sum(), spec / spec.sum(), rtol=1e-10)


def test_infinite_medium_fixed_source():
    mesh = W.one_material(W.pin_cell_mesh())
    xs = W.synthetic_xs(["moderator"], 4, 21)
    S = np.tile(np.array([1.0, 0.5, 0.2, 0.0]), (mesh.n_tri, 1))
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    o.set_fixed_source(S)
    k, n, r, conv = o.iterate(False, 0.0, 1e-13, 20000)
    assert conv
    phi, _ = o.get_state()
    ref = np.linalg.solve(np.diag(xs.sigma_t[0]) - xs.sigma_s[0].T, S[0])
    np.testing.assert_allclose(phi, np.tile(ref, (mesh.n_tri, 1)), rtol=1e-10)
    # one-group pure absorber: phi = S / Sigma_t
    xs1 = W.CrossSections(np.array([[0.8]]), np.zeros((1, 1)), np.zeros((1, 1)), np.zeros((1, 1, 1)))
    o1 = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o1.set_xs(xs1)
    o1.set_fixed_source(np.full((mesh.n_tri, 1), 2.0))
    o1.iterate(False, 0.0, 1e-14, 1000)
    phi1, _ = o1.get_state()
    np.testing.assert_allclose(phi1, 2.0 / 0.8, rtol=1e-12)


# ------------------------------------------------------------------------------ balance, symmetry

@pytest.mark.parametrize("bc,layout", [((0, 0, 0, 0), 0), ((1, 0, 1, 0), 0), ((1, 1, 1, 1), 0), ((0, 0, 0, 0), 1)])
def test_global_neutron_balance(bc, layout):
    """At convergence: absorption + leakage = production / k, with production normalised to 1
    (modular and back-projected rays)."""
    prob = W.pin_cell_problem()
    mesh = W.with_bc(prob.mesh, bc)
    xs = prob.xs
    if bc == (0, 0, 0, 0):
        xs = W.CrossSections(xs.sigma_t, xs.nu_sigma_f * 4.0, xs.chi, xs.sigma_s)
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT, ray_layout=layout)
    o.set_xs(xs)
    k, n, r, conv = o.iterate(True, 1e-13, 1e-12, 50000)
    assert conv
    phi, _ = o.get_state()
    A = o.areas()
    sa = xs.sigma_t - xs.sigma_s.sum(2)            # absorption = total - out-scatter
    absorption = float((A[:, None] * sa[mesh.mat] * phi).sum())
    production = float((A[:, None] * xs.nu_sigma_f[mesh.mat] * phi).sum())
    leak = float(o.leakage().sum())
    assert abs(production - 1.0) < 1e-12
    if all(b == 1 for b in bc):
        assert abs(leak) == 0.0
    else:
        assert leak > 0
    assert abs((absorption + leak) * k - production) < 1e-9


def _d4_permutations(mesh):
    c = mesh.centroids()
    maps = [lambda x, y: (-x, y), lambda x, y: (x, -y), lambda x, y: (y, x), lambda x, y: (-y, -x)]
    perms = []
    for f in maps:
        tx, ty = f(c[:, 0], c[:, 1])
        tc = np.stack([tx, ty], 1)
        d = ((tc[:, None, :] - c[None, :, :]) ** 2).sum(-1)
        p = d.argmin(1)
        assert d[np.arange(len(p)), p].max() < 1e-20
        perms.append(p)
    return perms


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (0, 0, 0, 0)])
def test_mirror_symmetry(bc):
    prob = W.pin_cell_problem()
    mesh = W.with_bc(prob.mesh, bc)
    xs = prob.xs
    if bc == (0, 0, 0, 0):
        xs = W.CrossSections(xs.sigma_t, xs.nu_sigma_f * 4.0, xs.chi, xs.sigma_s)
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    k, n, r, conv = o.iterate(True, 1e-13, 1e-12, 50000)
    assert conv
    phi, _ = o.get_state()
    for p in _d4_permutations(mesh):
        np.testing.assert_allclose(phi[p], phi, rtol=1e-9)


def test_thread_count_does_not_change_results():
    prob = W.small_lattice_problem(3, n_azim=8, ray_spacing=0.08)
    res = []
    for th in (1, 3):
        o = oracle.Oracle.from_problem(prob, threads=th)
        for _ in range(5):
            o.outer(True)
        res.append(o.get_state())
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


# ------------------------------------------------------------------------------ warm-start network

def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp_oracle as MO

    rng = np.random.default_rng(0)
    dims = [5, 8, 8, 8, 3]
    n_par = sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(4))
    p = rng.normal(0, 0.5, n_par)
    x = rng.normal(0, 1, (7, 5))
    y = rng.normal(0, 1, (7, 3))
    norm = (rng.normal(0, 0.1, 5), rng.uniform(0.5, 2, 5), rng.normal(0, 0.1, 3), rng.uniform(0.5, 2, 3))
    loss, g = MO.loss_and_grad(p, dims, x, y, norm, bf16=False)
    h = 1e-6
    fd = np.zeros(n_par)
    for i in range(n_par):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd[i] = (MO.loss_and_grad(pp, dims, x, y, norm, bf16=False)[0] -
                 MO.loss_and_grad(pm, dims, x, y, norm, bf16=False)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_bf16_rounding_is_round_to_nearest_even():
    from oracle import mlp_oracle as MO

    # 1 + 2^-8 lies exactly between bf16 neighbours 1 and 1 + 2^-7: ties go to even (1.0)
    assert MO.round_bf16(np.float32(1.0 + 2 ** -8)) == 1.0
    assert MO.round_bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6
    assert MO.round_bf16(np.float32(1.0 + 2 ** -8 + 2 ** -20)) == 1.0 + 2 ** -7
    assert MO.round_bf16(np.float32(-2.5)) == -2.5


# ------------------------------------------------------------------------------ CMFD acceleration

@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 0, 1, 0)])
def test_cmfd_keeps_the_converged_solution_and_needs_fewer_outers(bc):
    """The partial-current coarse balance reproduces the MOC currents, so the accelerated power
    iteration converges to the unaccelerated solution, in fewer outers."""
    prob = W.small_lattice_problem(3, bc=bc, n_azim=16, ray_spacing=0.05)
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    a = oracle.Oracle.from_problem(prob, threads=4)
    ka, na, _, ca = a.iterate(True, 1e-12, 1e-11, 20000)
    b = oracle.Oracle.from_problem(prob, threads=4)
    b.set_cmfd(cell, nc, 6, 6)
    kb, nb, _, cb = b.iterate(True, 1e-12, 1e-11, 20000)
    assert ca and cb
    assert abs(ka - kb) < 1e-10
    np.testing.assert_allclose(b.get_state()[0], a.get_state()[0], rtol=1e-8)
    assert nb < na / 2, (na, nb)


def test_cmfd_step_is_consistent_at_the_fixed_point():
    """From a converged unaccelerated state one accelerated outer leaves k and the flux unchanged:
    any error in the currents, homogenisation or coefficients would move them."""
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.05)
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    o = oracle.Oracle.from_problem(prob, threads=4)
    o.iterate(True, 1e-13, 1e-12, 20000)
    phi, k, psi = o.get_state(with_psi=True)
    o.set_cmfd(cell, nc, 8, 8)
    o.set_state(phi, k, psi)
    o.outer(True)
    phi2, k2 = o.get_state()
    assert abs(k2 - k) < 1e-10
    np.testing.assert_allclose(phi2, phi, rtol=1e-9)


def _reflector_core_1():
    """One assembly with the core's reflector band (reflective -x/-y, vacuum +x/+y), coarse
    quadrature: a case where leaving the reflective-wall currents out of the coarse balance made
    the accelerated iteration settle 2 pcm away from the transport solution."""
    xs = W.synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, 4,
                        fuel_scales=[1.0, 0.95, 1.05, 0.9])
    return W.Problem(W.core_mesh(1), xs, 16, 0.2, tol=1e-6, name="core1", seed=4)


def test_cmfd_settles_on_the_transport_solution_with_reflective_walls():
    """The accelerated iteration converges, and its limit is a fixed point of the plain transport
    iteration (one unaccelerated outer from it changes nothing)."""
    prob = _reflector_core_1()
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    o = oracle.Oracle.from_problem(prob, threads=7)
    o.set_cmfd(cell, nc, 20, 20)
    k, n, r, conv = o.iterate(True, 1e-11, 1e-9, 80)
    assert conv, (k, n, r)
    phi, k, psi = o.get_state(with_psi=True)
    o.set_cmfd(None)
    o.set_state(phi, k, psi)
    r1 = o.outer(True)
    phi1, k1 = o.get_state()
    assert r1 < 1e-8, r1
    assert abs(k1 - k) < 1e-10


# ------------------------------------------------------------------------------ anisotropic scattering

def test_legendre_polynomials():
    from scipy.special import eval_legendre
    rng = np.random.default_rng(3)
    for l in range(0, 7):
        for x in rng.uniform(-1, 1, 5):
            assert abs(oracle.legendre(l, x) - eval_legendre(l, x)) < 1e-14


def _bare_square_1g(size=4.0, n=8, st=1.0, c=0.9):
    mesh = W.grid_mesh(n, n, size, size, bc=(0, 0, 0, 0))
    xs = W.CrossSections(np.array([[st]]), np.array([[0.25]]), np.array([[1.0]]), np.array([[[c * st]]]))
    return mesh, xs


def _k_of(mesh, xs, ssl=None, tol=1e-10):
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    if ssl is not None:
        o.set_scattering(ssl)
    k, n, r, conv = o.iterate(True, tol, 10 * tol, 5000)
    assert conv
    return k, o


def test_p1_scattering_agrees_with_the_transport_correction():
    """Forward-peaked P1 scattering (mean cosine g) in a bare homogeneous square lowers k (more
    leakage) and lands close to the transport-corrected isotropic problem (Sigma_t - g Sigma_s,
    Sigma_s - g Sigma_s): a wrong sign or a missing (2l+1) fails one of the two."""
    mesh, xs = _bare_square_1g()
    g = 0.4
    k0, _ = _k_of(mesh, xs)
    k1, _ = _k_of(mesh, xs, W.anisotropic_moments(xs, 1, [g]))
    s = xs.sigma_s[0, 0, 0]
    xtc = W.CrossSections(xs.sigma_t - g * s, xs.nu_sigma_f, xs.chi, xs.sigma_s - g * s)
    ktc, _ = _k_of(mesh, xtc)
    assert k1 < ktc < k0, (k0, k1, ktc)
    assert abs(k1 - ktc) < 0.2 * abs(k0 - k1), (k0, k1, ktc)


def test_p1_infinite_medium_keeps_kinf_and_zero_moments_change_nothing():
    """All reflective, one material: the flat isotropic flux stays an exact fixed point with P1
    scattering, so k = k_inf; and Sigma_s,1 = 0 reproduces the isotropic iteration."""
    mesh = W.one_material(W.pin_cell_mesh())
    xs = _xs_one(7, 12)
    kinf, spec = _closed_form_kinf(xs)
    k, o = _k_of(mesh, xs, W.anisotropic_moments(xs, 1, [0.3]), tol=1e-12)
    assert abs(k - kinf) < 1e-9
    phi, _ = o.get_state()
    np.testing.assert_allclose(phi / phi[0], np.ones_like(phi), atol=1e-9)
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.05)
    a = oracle.Oracle.from_problem(prob)
    b = oracle.Oracle.from_problem(prob)
    b.set_scattering(np.zeros((1,) + prob.xs.sigma_s.shape))
    for _ in range(4):
        a.outer(True)
        b.outer(True)
    assert abs(a.get_state()[1] - b.get_state()[1]) < 1e-13
    np.testing.assert_allclose(b.get_state()[0], a.get_state()[0], rtol=1e-12)


def test_p1_global_balance_with_vacuum():
    """Odd Legendre terms integrate to zero over the (symmetric) quadrature, so absorption
    (Sigma_t - Sigma_s,0 out-scatter) + leakage = production / k still holds."""
    prob = W.pin_cell_problem()
    mesh = W.with_bc(prob.mesh, (0, 0, 0, 0))
    xs = W.CrossSections(prob.xs.sigma_t, prob.xs.nu_sigma_f * 4.0, prob.xs.chi, prob.xs.sigma_s)
    o = oracle.Oracle(mesh, 16, 0.05, W.TY3_SIN_THETA, W.TY3_WEIGHT)
    o.set_xs(xs)
    o.set_scattering(W.anisotropic_moments(xs, 1, [0.05, 0.3]))
    k, n, r, conv = o.iterate(True, 1e-13, 1e-12, 50000)
    assert conv
    phi, _ = o.get_state()
    A = o.areas()
    sa = xs.sigma_t - xs.sigma_s.sum(2)
    absorption = float((A[:, None] * sa[mesh.mat] * phi).sum())
    production = float((A[:, None] * xs.nu_sigma_f[mesh.mat] * phi).sum())
    leak = float(o.leakage().sum())
    assert abs((absorption + leak) * k - production) < 1e-9


# ------------------------------------------------------------------------------ sampled-region flux

@pytest.mark.parametrize("case", ["lattice_mixed_bc", "hex_cluster_vacuum"])
def test_sampled_fixed_source_flux_equals_the_full_outer(case):
    """The sampled-region check used at full size (only the rays crossing the sampled regions are
    laid down and swept) equals the whole oracle's fixed-source outer from the same state, on a
    rectangular lattice with mixed walls and on a concave 7-hexagon cluster whose rays leave and
    re-enter the mesh (every in-mesh chord a track with zero inflow)."""
    rng = np.random.default_rng(31)
    if case == "lattice_mixed_bc":
        prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.05)
    else:
        mesh = W.hex_core_mesh(n_sub=4, n_rings=1)
        prob = W.Problem(mesh, W.synthetic_xs(["fuel", "fuel", "coolant"], 5, 9, sigt_range=(0.05, 0.6)), 12, 0.2)
    xs = W.CrossSections(prob.xs.sigma_t, np.zeros_like(prob.xs.nu_sigma_f), prob.xs.chi, prob.xs.sigma_s)
    R, G = prob.mesh.n_tri, xs.n_groups
    o = oracle.Oracle.from_problem(prob, threads=2, with_xs=False)
    o.set_xs(xs)
    S = rng.uniform(0.0, 1.0, (R, G))
    phi0 = rng.uniform(0.5, 1.5, (R, G))
    psi0 = rng.uniform(0.0, 0.2, (o.n_tracks, 2, len(prob.sin_theta), G))
    o.set_fixed_source(S)
    o.set_state(phi0, 1.0, psi0)
    o.outer(False)
    full, _ = o.get_state()
    sample = np.unique(rng.choice(R, 25, replace=False))
    ref, area = oracle.sample_fixed_source(prob.mesh, prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w,
                                           xs, S, phi0, psi0, sample)
    np.testing.assert_allclose(area, o.areas()[sample], rtol=1e-12)
    np.testing.assert_allclose(ref, full[sample], rtol=1e-12)
