"""Seeded synthetic inputs: triangle meshes, multigroup cross sections, quadrature data.

This module produces INPUTS only: geometry (vertices, triangles, material ids), cross sections,
and the published polar quadrature table. It holds none of the transport method's arithmetic
(no track laydown, no segmentation, no sweep), so both the CUDA library and the CPU oracle may be
fed from it.

The paper's workloads (C5G7, ABTR, Empire, MSRE; Sec. 4, Tables 1-14) need benchmark geometry and
cross-section libraries that are not available, so these generators stand in for them with the
shapes the paper's MOC runs have: a square pin cell, a 17x17 lattice assembly, a 3x3-assembly core
with a reflector band, and a 19-assembly hexagonal core with 271 pins per assembly.

Every mesh is a conforming triangle mesh, counter-clockwise triangles, each triangle one flat
source region (Sec. 2.1: "FSR = one finite element").
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# Tabuchi-Yamamoto optimal 3-angle polar set (Yamamoto, Tabuchi, Sugimura, Endo, Ishizaki,
# J. Nucl. Sci. Technol. 44 (2007) 129): sin(theta_p) and weights over one hemisphere (sum 1).
TY3_SIN_THETA = np.array([0.166648, 0.537707, 0.932954], dtype=np.float64)
TY3_WEIGHT = np.array([0.046233, 0.283619, 0.670148], dtype=np.float64)

BC_VACUUM = 0
BC_REFLECTIVE = 1


@dataclasses.dataclass
class Mesh:
    xy: np.ndarray          # float64 [V, 2]
    tri: np.ndarray         # int32 [T, 3], counter-clockwise
    mat: np.ndarray         # int32 [T]
    bbox: Tuple[float, float, float, float]   # xmin, xmax, ymin, ymax
    bc: Tuple[int, int, int, int]              # x-, x+, y-, y+ : 0 vacuum, 1 reflective
    name: str = ""

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    def areas(self) -> np.ndarray:
        p = self.xy[self.tri]
        return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                      - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))

    def centroids(self) -> np.ndarray:
        return self.xy[self.tri].mean(axis=1)


@dataclasses.dataclass
class CrossSections:
    sigma_t: np.ndarray      # [M, G]
    nu_sigma_f: np.ndarray   # [M, G]
    chi: np.ndarray          # [M, G]
    sigma_s: np.ndarray      # [M, G_from, G_to]

    @property
    def n_mat(self) -> int:
        return int(self.sigma_t.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.sigma_t.shape[1])

    def absorption(self) -> np.ndarray:
        return self.sigma_t - self.sigma_s.sum(axis=2)


@dataclasses.dataclass
class Problem:
    mesh: Mesh
    xs: CrossSections
    n_azim: int
    ray_spacing: float
    sin_theta: np.ndarray = dataclasses.field(default_factory=lambda: TY3_SIN_THETA.copy())
    polar_w: np.ndarray = dataclasses.field(default_factory=lambda: TY3_WEIGHT.copy())
    tol: float = 1e-6
    name: str = ""
    seed: int = 0
    fixed_source: Optional[np.ndarray] = None   # [R, G] isotropic volumetric source, or None
    ray_layout: int = 0     # 0 cyclic modular rays over the bounding box, 1 back projection (vacuum only)


# ----------------------------------------------------------------------------------------------
# mesh assembly helpers
# ----------------------------------------------------------------------------------------------

class _MeshBuilder:
    """Collects triangles with exact-coordinate vertex merging (keys are rounded coordinates)."""

    def __init__(self, quantum: float = 1e-9):
        self.q = quantum
        self.keys: Dict[Tuple[int, int], int] = {}
        self.xy: List[Tuple[float, float]] = []
        self.tri: List[Tuple[int, int, int]] = []
        self.mat: List[int] = []

    def vid(self, x: float, y: float) -> int:
        k = (int(round(x / self.q)), int(round(y / self.q)))
        v = self.keys.get(k)
        if v is None:
            v = len(self.xy)
            self.keys[k] = v
            self.xy.append((x, y))
        return v

    def add(self, a, b, c, m: int):
        ia, ib, ic = self.vid(*a), self.vid(*b), self.vid(*c)
        ax, ay = self.xy[ia]
        bx, by = self.xy[ib]
        cx, cy = self.xy[ic]
        cr = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay)
        if cr < 0:
            ib, ic = ic, ib
        elif cr == 0:
            raise ValueError("degenerate triangle")
        self.tri.append((ia, ib, ic))
        self.mat.append(m)

    def mesh(self, bbox, bc, name) -> Mesh:
        return Mesh(np.asarray(self.xy, dtype=np.float64), np.asarray(self.tri, dtype=np.int32),
                    np.asarray(self.mat, dtype=np.int32), tuple(float(v) for v in bbox),
                    tuple(int(b) for b in bc), name)


# The 8 symmetries of the square (dihedral group D4) acting on (x, y).
_D4 = [
    lambda x, y: (x, y), lambda x, y: (y, x), lambda x, y: (-y, x), lambda x, y: (-x, y),
    lambda x, y: (-x, -y), lambda x, y: (-y, -x), lambda x, y: (y, -x), lambda x, y: (x, -y),
]

_H2 = math.sqrt(0.5)


def _pin_wedge(pitch: float, ring_radii: Sequence[float], ring_mats: Sequence[int],
               n_mod_layers: int, mod_mat: int):
    """Triangles of the 0..45 degree wedge of a pin cell centred at the origin.

    Ring boundaries are octagons (vertices every 45 degrees) whose circumradius keeps the area of
    the circle of the given radius. Between the outermost octagon and the cell square the
    moderator is split into `n_mod_layers` blended layers. The square carries nodes only at its
    corners and edge midpoints, so tiled pin cells are conforming.
    Returns a list of (p0, p1, p2, material).
    """
    h = 0.5 * pitch
    scale = math.sqrt(math.pi / (2.0 * math.sqrt(2.0)))   # octagon area 2*sqrt(2)*rho^2 = pi r^2
    rho = [r * scale for r in ring_radii]
    if rho[-1] >= h:
        raise ValueError("outer ring does not fit in the cell")
    out = []
    A = [(0.0, 0.0)]
    B = [(0.0, 0.0)]
    for r in rho:
        A.append((r, 0.0))
        B.append((r * _H2, r * _H2))
    # fuel / clad rings
    out.append((A[0], A[1], B[1], ring_mats[0]))
    for k in range(2, len(A)):
        m = ring_mats[k - 1]
        out.append((A[k - 1], A[k], B[k], m))
        out.append((A[k - 1], B[k], B[k - 1], m))
    # moderator layers blending the octagon into the square
    a0, b0 = A[-1], B[-1]
    prevA, prevB = a0, b0
    for j in range(1, n_mod_layers + 1):
        t = j / n_mod_layers
        if j == n_mod_layers:
            nA, nB = (h, 0.0), (h, h)
        else:
            nA = ((1 - t) * a0[0] + t * h, 0.0)
            s = (1 - t) * b0[0] + t * h
            nB = (s, s)
        out.append((prevA, nA, nB, mod_mat))
        out.append((prevA, nB, prevB, mod_mat))
        prevA, prevB = nA, nB
    return out


def _add_pin(mb: _MeshBuilder, wedge, cx: float, cy: float, mat_map=None):
    for g in _D4:
        for (p0, p1, p2, m) in wedge:
            q = [g(*p) for p in (p0, p1, p2)]
            mm = m if mat_map is None else mat_map.get(m, m)
            mb.add((cx + q[0][0], cy + q[0][1]), (cx + q[1][0], cy + q[1][1]),
                   (cx + q[2][0], cy + q[2][1]), mm)


# ----------------------------------------------------------------------------------------------
# geometry generators
# ----------------------------------------------------------------------------------------------

def pin_cell_mesh(pitch: float = 1.26, r_fuel: float = 0.54, n_fuel_rings: int = 8,
                  n_mod_layers: int = 5, bc=(1, 1, 1, 1)) -> Mesh:
    """Square pin cell centred at the origin: 8 equal-area fuel rings x 8 sectors, moderator
    layers to the square. Materials: 0 fuel, 1 moderator. 8 + 16*(rings-1) + 16*layers triangles.
    The mesh is exactly symmetric under x->-x, y->-y and x<->y."""
    radii = [r_fuel * math.sqrt(k / n_fuel_rings) for k in range(1, n_fuel_rings + 1)]
    wedge = _pin_wedge(pitch, radii, [0] * n_fuel_rings, n_mod_layers, 1)
    mb = _MeshBuilder()
    _add_pin(mb, wedge, 0.0, 0.0)
    h = 0.5 * pitch
    return mb.mesh((-h, h, -h, h), bc, "pin_cell")


def guide_tube_positions() -> List[Tuple[int, int]]:
    """25 moderator-filled positions of a 17x17 lattice, as (di, dj) offsets from the centre pin.

    A synthetic rule, not a benchmark layout: the centre plus the orbits under the 8 symmetries
    of the square of (3,0), (3,3), (6,0), (6,3) and (6,6): 1 + 4 + 4 + 4 + 8 + 4 = 25 positions."""
    pos = {(0, 0)}
    for a, b in [(3, 0), (3, 3), (6, 0), (6, 3), (6, 6)]:
        for g in _D4:
            x, y = g(a, b)
            pos.add((int(x), int(y)))
    out = sorted(pos)
    assert len(out) == 25
    return out


def assembly_pin_wedge(pitch: float = 1.26):
    """Coarser pin used in lattices: 4 equal-area fuel rings (r 0.46), 1 clad ring (to r 0.54),
    4 moderator layers: 136 triangles per pin. Materials: 0 fuel, 1 clad, 2 moderator."""
    r_f, r_c = 0.46, 0.54
    radii = [r_f * math.sqrt(k / 4) for k in range(1, 5)] + [r_c]
    return _pin_wedge(pitch, radii, [0, 0, 0, 0, 1], 4, 2)


def lattice_mesh(n: int = 17, pitch: float = 1.26, guide_tubes: bool = True,
                 bc=(1, 1, 1, 1)) -> Mesh:
    """n x n lattice of pins (n odd), centred at the origin. Guide-tube pins (17x17 only) have
    their fuel replaced by moderator. Materials: 0 fuel, 1 clad, 2 moderator."""
    if n % 2 != 1:
        raise ValueError("n must be odd")
    wedge = assembly_pin_wedge(pitch)
    gt = set(guide_tube_positions()) if (guide_tubes and n == 17) else set()
    mb = _MeshBuilder()
    c = n // 2
    for i in range(n):
        for j in range(n):
            di, dj = i - c, j - c
            mm = {0: 2} if (di, dj) in gt else None
            _add_pin(mb, wedge, di * pitch, dj * pitch, mm)
    h = 0.5 * n * pitch
    return mb.mesh((-h, h, -h, h), bc, f"lattice{n}")


def assembly_mesh() -> Mesh:
    """17x17 assembly, pitch 1.26 cm, 25 guide tubes, reflective on all sides (~39k triangles)."""
    m = lattice_mesh(17)
    m.name = "assembly17"
    return m


def core_mesh(n_asm: int = 3, refl_sub: int = 4) -> Mesh:
    """n_asm x n_asm assemblies in [0, n_asm*21.42]^2 plus a 21.42 cm reflector band on +x and +y.

    Reflective on -x and -y (symmetry planes), vacuum on +x and +y. The reflector is a grid of
    0.63 cm cells (half a pin pitch, so cell corners meet the pin-boundary nodes). A cell away
    from the assemblies is refl_sub x refl_sub squares, each cut into 2 triangles; a cell with an
    edge on an assembly face is a fan around its centre through its corners and the refl_sub-1
    intermediate nodes of its other edges, so the mesh stays conforming.
    Materials: 0-3 fuel variants, 4 clad, 5 moderator, 6 reflector.
    """
    pitch = 1.26
    asm_w = 17 * pitch
    wedge = assembly_pin_wedge(pitch)
    gt = set(guide_tube_positions())
    variant = [[0, 1, 2], [1, 3, 1], [2, 1, 0]]      # fixed synthetic fuel-variant pattern
    mb = _MeshBuilder()
    for ai in range(n_asm):
        for aj in range(n_asm):
            ox, oy = (ai + 0.5) * asm_w, (aj + 0.5) * asm_w
            v = variant[ai % 3][aj % 3]
            for i in range(17):
                for j in range(17):
                    di, dj = i - 8, j - 8
                    mm = {0: 5, 1: 4, 2: 5} if (di, dj) in gt else {0: v, 1: 4, 2: 5}
                    _add_pin(mb, wedge, ox + di * pitch, oy + dj * pitch, mm)
    core_w = n_asm * asm_w
    dom = core_w + asm_w
    cell = pitch / 2.0
    nc = int(round(dom / cell))
    nin = int(round(core_w / cell))
    k = refl_sub
    for ci in range(nc):
        for cj in range(nc):
            if ci < nin and cj < nin:
                continue
            x0, y0 = ci * cell, cj * cell
            face_l = (ci == nin and cj < nin)
            face_b = (cj == nin and ci < nin)
            if not (face_l or face_b):
                for a in range(k):
                    for b in range(k):
                        xa, xb = x0 + a * cell / k, x0 + (a + 1) * cell / k
                        ya, yb = y0 + b * cell / k, y0 + (b + 1) * cell / k
                        mb.add((xa, ya), (xb, ya), (xb, yb), 6)
                        mb.add((xa, ya), (xb, yb), (xa, yb), 6)
                continue
            x1, y1 = x0 + cell, y0 + cell
            xc, yc = x0 + 0.5 * cell, y0 + 0.5 * cell
            ring = []
            for a in range(k):                                   # bottom edge
                if a == 0 or not face_b:
                    ring.append((x0 + a * cell / k, y0))
            for a in range(k):                                   # right edge
                ring.append((x1, y0 + a * cell / k))
            for a in range(k):                                   # top edge
                ring.append((x1 - a * cell / k, y1))
            for a in range(k):                                   # left edge
                if a == 0 or not face_l:
                    ring.append((x0, y1 - a * cell / k))
            for q in range(len(ring)):
                mb.add((xc, yc), ring[q], ring[(q + 1) % len(ring)], 6)
    return mb.mesh((0.0, dom, 0.0, dom), (1, 0, 1, 0), "core3x3")


def _cube_round(q: np.ndarray, r: np.ndarray):
    x, z = q, r
    y = -x - z
    rx, ry, rz = np.round(x), np.round(y), np.round(z)
    dx, dy, dz = np.abs(rx - x), np.abs(ry - y), np.abs(rz - z)
    fix_x = (dx > dy) & (dx > dz)
    fix_y = (~fix_x) & (dy > dz)
    fix_z = ~(fix_x | fix_y)
    rx = np.where(fix_x, -ry - rz, rx)
    rz = np.where(fix_z, -rx - ry, rz)
    return rx.astype(np.int64), rz.astype(np.int64)


def hex_core_mesh(n_sub: int = 115, flat_to_flat: float = 14.6, n_rings: int = 2,
                  pin_rings: int = 10, pin_pitch: float = 0.74, pin_radius: float = 0.30) -> Mesh:
    """19 (n_rings=2) flat-topped hexagonal assemblies, each a uniform triangular subdivision of
    the hexagon (6*n_sub^2 triangles). All assemblies lie on one regular triangular lattice, so
    the mesh is conforming. Material by centroid: inside one of the 271 (10-ring) pin circles ->
    fuel (0 inner 7 assemblies, 1 outer ring), otherwise coolant (2). Vacuum on all sides."""
    F = flat_to_flat
    s = F / math.sqrt(3.0)
    a = s / n_sub
    e1 = np.array([a, 0.0])
    e2 = np.array([0.5 * a, 0.5 * math.sqrt(3.0) * a])
    # assembly lattice (Voronoi cells = flat-topped hexagons of apothem F/2)
    A1 = F * np.array([math.cos(math.pi / 6), math.sin(math.pi / 6)])
    A2 = F * np.array([0.0, 1.0])
    Ainv = np.linalg.inv(np.stack([A1, A2], axis=1))
    P1 = pin_pitch * np.array([1.0, 0.0])
    P2 = pin_pitch * np.array([0.5, 0.5 * math.sqrt(3.0)])
    Pinv = np.linalg.inv(np.stack([P1, P2], axis=1))
    extent = (n_rings + 1) * F
    umax = int(math.ceil(extent / a * 1.2)) + 2
    us = np.arange(-umax, umax + 1)
    tris = []
    mats = []
    for v in range(-umax, umax + 1):
        for up in (True, False):
            if up:
                c = (us[:, None] + 1.0 / 3.0) * e1 + (v + 1.0 / 3.0) * e2
            else:
                c = (us[:, None] + 2.0 / 3.0) * e1 + (v + 2.0 / 3.0) * e2
            qa = c @ Ainv.T
            aq, ar = _cube_round(qa[:, 0], qa[:, 1])
            hd = np.maximum(np.maximum(np.abs(aq), np.abs(ar)), np.abs(aq + ar))
            inside = hd <= n_rings
            if not inside.any():
                continue
            idx = np.nonzero(inside)[0]
            u = us[idx]
            if up:
                t = np.stack([np.stack([u, np.full_like(u, v)], 1), np.stack([u + 1, np.full_like(u, v)], 1),
                              np.stack([u, np.full_like(u, v + 1)], 1)], 1)
            else:
                t = np.stack([np.stack([u + 1, np.full_like(u, v)], 1), np.stack([u + 1, np.full_like(u, v + 1)], 1),
                              np.stack([u, np.full_like(u, v + 1)], 1)], 1)
            cc = c[idx]
            centre = aq[idx, None] * A1 + ar[idx, None] * A2
            local = cc - centre
            pq = local @ Pinv.T
            pq_, pr_ = _cube_round(pq[:, 0], pq[:, 1])
            pring = np.maximum(np.maximum(np.abs(pq_), np.abs(pr_)), np.abs(pq_ + pr_))
            pc = pq_[:, None] * P1 + pr_[:, None] * P2
            d2 = ((local - pc) ** 2).sum(1)
            fuel = (pring < pin_rings) & (d2 < pin_radius ** 2)
            outer = hd[idx] == n_rings
            m = np.where(fuel, np.where(outer, 1, 0), 2)
            tris.append(t)
            mats.append(m)
    T = np.concatenate(tris, 0)          # [n, 3, 2] lattice coords
    M = np.concatenate(mats, 0).astype(np.int32)
    flat = T.reshape(-1, 2)
    key = flat[:, 0] * (4 * umax + 10) + flat[:, 1]
    uniq, inv = np.unique(key, return_inverse=True)
    uv = np.zeros((uniq.shape[0], 2), dtype=np.int64)
    uv[inv] = flat
    xy = uv[:, 0:1] * e1 + uv[:, 1:2] * e2
    tri = inv.reshape(-1, 3).astype(np.int32)
    # lattice triangles (u,v),(u+1,v),(u,v+1) and (u+1,v),(u+1,v+1),(u,v+1) are both CCW
    xmin, ymin = xy.min(0)
    xmax, ymax = xy.max(0)
    return Mesh(xy, tri, M, (float(xmin), float(xmax), float(ymin), float(ymax)), (0, 0, 0, 0), "hexcore19")


# ----------------------------------------------------------------------------------------------
# cross sections
# ----------------------------------------------------------------------------------------------

def _kinf(sigma_t, nu_sigma_f, chi, sigma_s) -> float:
    """Infinite-medium multiplication of one material (used only to scale synthetic fission data)."""
    M = np.diag(sigma_t) - sigma_s.T
    return float(nu_sigma_f @ np.linalg.solve(M, chi))


def synthetic_xs(kinds: Sequence[str], G: int, seed: int, sigt_range=(0.2, 2.0),
                 kinf_target: float = 1.3, fuel_scales: Optional[Sequence[float]] = None) -> CrossSections:
    """Seeded synthetic multigroup data, one material per entry of `kinds` in
    {'fuel', 'clad', 'moderator', 'reflector', 'coolant'}.

    Sigma_t,g ~ U[sigt_range]; scattering ratio c_g in [0.5, 0.95] (moderator/reflector
    [0.85, 0.95]), so absorption >= 5% of Sigma_t; downscatter-only (lower triangular in
    from->to order) with a dominant within-group term; nu*Sigma_f only in fuel, scaled so the
    fuel's infinite-medium k is `kinf_target` (times the per-fuel scale factor); chi only in the
    top 3 groups."""
    rng = np.random.default_rng(seed)
    Mn = len(kinds)
    st = np.zeros((Mn, G))
    nsf = np.zeros((Mn, G))
    chi = np.zeros((Mn, G))
    ss = np.zeros((Mn, G, G))
    chi_top = rng.dirichlet([6.0, 3.0, 1.0]) if G >= 3 else np.ones(G) / G
    fuel_i = 0
    for m, kind in enumerate(kinds):
        st[m] = rng.uniform(sigt_range[0], sigt_range[1], G)
        if kind in ("moderator", "reflector"):
            c = rng.uniform(0.85, 0.95, G)
        elif kind == "fuel":
            c = rng.uniform(0.5, 0.8, G)
        else:
            c = rng.uniform(0.5, 0.95, G)
        for g in range(G):
            total_s = c[g] * st[m, g]
            if g == G - 1:
                ss[m, g, g] = total_s
                continue
            self_frac = rng.uniform(0.5, 0.9)
            rest = np.exp(-np.arange(G - g - 1) * rng.uniform(0.5, 1.5))
            rest = rest / rest.sum() * (1.0 - self_frac)
            ss[m, g, g] = self_frac * total_s
            ss[m, g, g + 1:] = rest * total_s
        ng = min(3, G)
        chi[m, :ng] = chi_top[:ng] / chi_top[:ng].sum()
        if kind == "fuel":
            sa = st[m] - ss[m].sum(1)
            nsf[m] = 2.45 * rng.uniform(0.3, 0.8, G) * sa
            k0 = _kinf(st[m], nsf[m], chi[m], ss[m])
            sc = kinf_target / k0
            if fuel_scales is not None:
                sc *= float(fuel_scales[fuel_i])
            nsf[m] *= sc
            fuel_i += 1
    return CrossSections(st, nsf, chi, ss)


def anisotropic_moments(xs: CrossSections, L: int, mean_cosine) -> np.ndarray:
    """Synthetic higher Legendre moments of the scattering matrices: Sigma_s,l = g^l Sigma_s,0
    with g the mean scattering cosine of each material (`mean_cosine`: one value per material,
    0 <= g < 1, forward-peaked for g > 0). Returns [L][M][G][G] for l = 1..L."""
    g = np.asarray(mean_cosine, dtype=np.float64)
    assert g.shape == (xs.n_mat,) and (g >= 0).all() and (g < 1).all()
    return np.stack([(g ** l)[:, None, None] * xs.sigma_s for l in range(1, L + 1)])


def perturbed_xs(base: CrossSections, seed: int, sigma: float = 0.1) -> CrossSections:
    """Per-material, per-group lognormal scaling (sigma) of absorption, each scattering row and
    nu*Sigma_f; Sigma_t is rebuilt as absorption + scattering so the data stay valid."""
    rng = np.random.default_rng(seed)
    M, G = base.sigma_t.shape
    sa = base.absorption() * rng.lognormal(0.0, sigma, (M, G))
    ss = base.sigma_s * rng.lognormal(0.0, sigma, (M, G, 1))
    nsf = base.nu_sigma_f * rng.lognormal(0.0, sigma, (M, G))
    st = sa + ss.sum(2)
    return CrossSections(st, nsf, base.chi.copy(), ss)


# ----------------------------------------------------------------------------------------------
# problem configurations
# ----------------------------------------------------------------------------------------------

def pin_cell_problem(seed: int = 1) -> Problem:
    """7-group square pin cell, pitch 1.26, fuel r 0.54, ~200 triangles, reflective,
    16 azimuths over 2 pi, TY-3 polar, ray spacing 0.05 cm, tolerance 1e-6."""
    mesh = pin_cell_mesh()
    xs = synthetic_xs(["fuel", "moderator"], 7, seed)
    return Problem(mesh, xs, 16, 0.05, tol=1e-6, name="pin_cell", seed=seed)


def assembly_problem(seed: int = 2, n_azim: int = 32, ray_spacing: float = 0.02) -> Problem:
    """7-group 17x17 assembly (~39k triangles), fuel/clad/moderator, reflective, 32 azimuths,
    TY-3 polar, ray spacing 0.02 cm."""
    mesh = assembly_mesh()
    xs = synthetic_xs(["fuel", "clad", "moderator"], 7, seed)
    return Problem(mesh, xs, n_azim, ray_spacing, tol=1e-6, name="assembly17", seed=seed)


def small_lattice_problem(n: int = 3, seed: int = 3, n_azim: int = 16, ray_spacing: float = 0.04,
                          G: int = 7, bc=(1, 1, 1, 1)) -> Problem:
    """n x n lattice of the assembly pin (no guide tubes), for fast parity cases."""
    mesh = lattice_mesh(n, guide_tubes=False, bc=bc)
    xs = synthetic_xs(["fuel", "clad", "moderator"], G, seed)
    return Problem(mesh, xs, n_azim, ray_spacing, tol=1e-8, name=f"lattice{n}", seed=seed)


def core_problem(seed: int = 4) -> Problem:
    """7-group 3x3-assembly core + reflector (~610k triangles), 4 fuel variants, vacuum +x/+y,
    reflective -x/-y, 64 azimuths, ray spacing 0.01 cm."""
    mesh = core_mesh()
    xs = synthetic_xs(["fuel", "fuel", "fuel", "fuel", "clad", "moderator", "reflector"], 7, seed,
                      fuel_scales=[1.0, 0.95, 1.05, 0.9])
    return Problem(mesh, xs, 64, 0.01, tol=1e-6, name="core3x3", seed=seed)


def hex_core_problem(seed: int = 5, n_sub: int = 115, n_rings: int = 2) -> Problem:
    """33-group fast-spectrum-like 19-assembly hexagonal core (~1.5M triangles), vacuum,
    48 azimuths, ray spacing 0.02 cm. n_rings = 1 keeps the central 7 assemblies (the same
    assemblies, cross sections and quadrature on a smaller core)."""
    mesh = hex_core_mesh(n_sub=n_sub, n_rings=n_rings)
    xs = synthetic_xs(["fuel", "fuel", "coolant"], 33, seed, sigt_range=(0.05, 0.6),
                      fuel_scales=[1.0, 0.9])
    return Problem(mesh, xs, 48, 0.02, tol=1e-6, name="hexcore19" if n_rings == 2 else f"hexcore{1 + 3 * n_rings * (n_rings + 1)}",
                   seed=seed)


def warm_start_instances(n: int, seed: int = 1000, base_seed: int = 2) -> List[CrossSections]:
    """XS of `n` assembly instances: the assembly's base data with seeded lognormal (sigma 0.1)
    per-material, per-group perturbations."""
    base = synthetic_xs(["fuel", "clad", "moderator"], 7, base_seed)
    return [perturbed_xs(base, seed + i) for i in range(n)]


def grid_mesh(nx: int, ny: int, width: float, height: float, bc=(1, 1, 1, 1), x0: float = 0.0,
              y0: float = 0.0, mat_fn=None) -> Mesh:
    """Structured nx x ny grid of rectangles, each cut into 2 triangles along alternating
    diagonals; material by `mat_fn(i, j)` (default 0). Small meshes for brute-force checks."""
    mb = _MeshBuilder()
    for i in range(nx):
        for j in range(ny):
            xa, xb = x0 + i * width / nx, x0 + (i + 1) * width / nx
            ya, yb = y0 + j * height / ny, y0 + (j + 1) * height / ny
            m = 0 if mat_fn is None else int(mat_fn(i, j))
            if (i + j) % 2 == 0:
                mb.add((xa, ya), (xb, ya), (xb, yb), m)
                mb.add((xa, ya), (xb, yb), (xa, yb), m)
            else:
                mb.add((xa, ya), (xb, ya), (xa, yb), m)
                mb.add((xb, ya), (xb, yb), (xa, yb), m)
    return mb.mesh((x0, x0 + width, y0, y0 + height), bc, f"grid{nx}x{ny}")


def one_material(mesh: Mesh) -> Mesh:
    """Copy of `mesh` with every triangle in material 0."""
    return Mesh(mesh.xy.copy(), mesh.tri.copy(), np.zeros_like(mesh.mat), mesh.bbox, mesh.bc, mesh.name)


def with_bc(mesh: Mesh, bc) -> Mesh:
    """Copy of `mesh` with other boundary conditions."""
    return Mesh(mesh.xy.copy(), mesh.tri.copy(), mesh.mat.copy(), mesh.bbox, tuple(int(b) for b in bc), mesh.name)


def grid_cells(mesh: Mesh, size: float):
    """Coarse cells for acceleration: each triangle goes to the square of side `size` (over the
    bounding box) that contains its centroid; empty squares are dropped. Returns (cell [n_tri],
    n_cells)."""
    c = mesh.centroids()
    xmin, xmax, ymin, ymax = mesh.bbox
    nx = max(1, int(math.ceil((xmax - xmin) / size - 1e-9)))
    i = np.clip(np.floor((c[:, 0] - xmin) / size).astype(np.int64), 0, nx - 1)
    j = np.clip(np.floor((c[:, 1] - ymin) / size).astype(np.int64), 0, 10 ** 9)
    key = j * nx + i
    uniq, inv = np.unique(key, return_inverse=True)
    return inv.astype(np.int32), int(uniq.size)
