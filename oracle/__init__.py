"""CPU FP64 oracle for the planar flat-source MOC sweep (test infrastructure).

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import
this package. It is an independent, plain restatement of the method (see moc_oracle.c for the
passages of the paper each step follows) and shares no code with the CUDA library.

The C source is compiled with gcc on first use (or by build()) into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moc_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_int, _d, ctypes.c_int, _i32, _i32, _d, _i32, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, _d, _d, ctypes.c_int, ctypes.c_char_p]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_error.restype = ctypes.c_char_p
        lib.orc_error.argtypes = [ctypes.c_void_p]
        lib.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_counts.argtypes = [ctypes.c_void_p, _i64, _i64, ctypes.POINTER(ctypes.c_int)]
        lib.orc_get_quadrature.argtypes = [ctypes.c_void_p, _d, _d, _d, _i32, _i32]
        lib.orc_get_tracks.argtypes = [ctypes.c_void_p, _i64, _i32, _d, _i32, _d, _i64]
        lib.orc_get_areas.argtypes = [ctypes.c_void_p, _d]
        lib.orc_set_xs.restype = ctypes.c_int
        lib.orc_set_xs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _d, _d, _d, _d]
        lib.orc_set_fixed_source.argtypes = [ctypes.c_void_p, _d]
        lib.orc_set_scattering.restype = ctypes.c_int
        lib.orc_set_scattering.argtypes = [ctypes.c_void_p, ctypes.c_int, _d]
        lib.orc_legendre.restype = ctypes.c_double
        lib.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_set_cmfd.restype = ctypes.c_int
        lib.orc_set_cmfd.argtypes = [ctypes.c_void_p, _i32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_set_state.argtypes = [ctypes.c_void_p, _d, ctypes.c_double, _d]
        lib.orc_get_state.argtypes = [ctypes.c_void_p, _d, _d, _d]
        lib.orc_get_q.argtypes = [ctypes.c_void_p, _d]
        lib.orc_get_tally.argtypes = [ctypes.c_void_p, _d]
        lib.orc_get_leakage.argtypes = [ctypes.c_void_p, _d]
        lib.orc_outer.restype = ctypes.c_double
        lib.orc_outer.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_normalise.argtypes = [ctypes.c_void_p]
        lib.orc_iterate.restype = ctypes.c_int
        lib.orc_iterate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, _d, ctypes.POINTER(ctypes.c_int), _d]
        lib.orc_set_axial.restype = ctypes.c_int
        lib.orc_set_axial.argtypes = [ctypes.c_void_p, ctypes.c_int, _d, _i32, ctypes.c_int, ctypes.c_int]
        lib.orc_get_flux3.argtypes = [ctypes.c_void_p, _d, _d]
        lib.orc_set_dg_cmfd.restype = ctypes.c_int
        lib.orc_set_dg_cmfd.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_get_leakage3.argtypes = [ctypes.c_void_p, _d]
        lib.orc_expm2.argtypes = [_d, _d]
        lib.orc_dg_segment.argtypes = [_d, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _d, _d]
        lib.orc_track_sweep.argtypes = [ctypes.c_int, _d, _d, _d, ctypes.c_double, ctypes.c_double, _d]
        lib.orc_sample_fixed_source.restype = ctypes.c_int
        lib.orc_sample_fixed_source.argtypes = [ctypes.c_int, _d, ctypes.c_int, _i32, _i32, _d, _i32, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, _d, _d, ctypes.c_int, ctypes.c_int,
                                                _d, _d, _d, _d, _d, ctypes.c_int, _i32, _d, _d]
        _lib = lib
        return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Oracle:
    """One problem: mesh + quadrature -> tracks; then cross sections, state and iterations."""

    def __init__(self, mesh, n_azim: int, ray_spacing: float, sin_theta, polar_w, threads: int = 1,
                 ray_layout: int = 0):
        lib = _load()
        self._lib = lib
        xy = _f64(mesh.xy)
        tri = _i32a(mesh.tri)
        mat = _i32a(mesh.mat)
        bbox = _f64(mesh.bbox)
        bc = _i32a(mesh.bc)
        st = _f64(sin_theta)
        pw = _f64(polar_w)
        err = ctypes.create_string_buffer(256)
        h = lib.orc_create(xy.shape[0], _p(xy, _d), tri.shape[0], _p(tri, _i32), _p(mat, _i32),
                           _p(bbox, _d), _p(bc, _i32), int(n_azim), float(ray_spacing), st.shape[0],
                           _p(st, _d), _p(pw, _d), int(ray_layout), err)
        if not h:
            raise RuntimeError("oracle: " + err.value.decode())
        self._h = ctypes.c_void_p(h)
        self.n_regions = int(tri.shape[0])
        self.n_polar = int(st.shape[0])
        self.G = 0
        T, S, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        lib.orc_counts(self._h, ctypes.byref(T), ctypes.byref(S), ctypes.byref(nd))
        self.n_tracks, self.n_segments, self.n_dir = T.value, S.value, nd.value
        lib.orc_set_threads(self._h, int(threads))

    @classmethod
    def from_problem(cls, prob, threads: int = 1, with_xs: bool = True) -> "Oracle":
        o = cls(prob.mesh, prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w, threads,
                getattr(prob, "ray_layout", 0))
        if with_xs:
            o.set_xs(prob.xs)
            if prob.fixed_source is not None:
                o.set_fixed_source(prob.fixed_source)
        return o

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_destroy(h)
            self._h = None

    def set_threads(self, n: int):
        self._lib.orc_set_threads(self._h, int(n))

    def quadrature(self) -> dict:
        n = self.n_dir
        phi, delta, omega = np.zeros(n), np.zeros(n), np.zeros(n)
        nx, ny = np.zeros(n, np.int32), np.zeros(n, np.int32)
        self._lib.orc_get_quadrature(self._h, _p(phi, _d), _p(delta, _d), _p(omega, _d), _p(nx, _i32), _p(ny, _i32))
        return dict(phi=phi, delta=delta, omega=omega, nx=nx, ny=ny)

    def tracks(self) -> dict:
        T, S = self.n_tracks, self.n_segments
        off = np.zeros(T + 1, np.int64)
        reg = np.zeros(S, np.int32)
        ln = np.zeros(S)
        dr = np.zeros(T, np.int32)
        xy = np.zeros((T, 4))
        link = np.zeros((T, 2), np.int64)
        self._lib.orc_get_tracks(self._h, _p(off, _i64), _p(reg, _i32), _p(ln, _d), _p(dr, _i32),
                                 _p(xy, _d), _p(link, _i64))
        return dict(seg_off=off, seg_region=reg, seg_len=ln, track_dir=dr, track_xy=xy, link=link)

    def areas(self) -> np.ndarray:
        a = np.zeros(self.n_regions)
        self._lib.orc_get_areas(self._h, _p(a, _d))
        return a

    def set_xs(self, xs):
        st, nsf, chi, ss = _f64(xs.sigma_t), _f64(xs.nu_sigma_f), _f64(xs.chi), _f64(xs.sigma_s)
        M, G = st.shape
        if self._lib.orc_set_xs(self._h, M, G, _p(st, _d), _p(nsf, _d), _p(chi, _d), _p(ss, _d)) != 0:
            raise RuntimeError("oracle: " + self._lib.orc_error(self._h).decode())
        self.G = G

    def set_fixed_source(self, S: Optional[np.ndarray]):
        if S is None:
            self._lib.orc_set_fixed_source(self._h, None)
        else:
            S = _f64(S)
            assert S.shape == (self.n_regions, self.G)
            self._lib.orc_set_fixed_source(self._h, _p(S, _d))

    def set_cmfd(self, cell=None, n_cells: int = 0, n_outer: int = 6, n_inner: int = 6, omega: float = 1.0):
        """Coarse-mesh acceleration on cells `cell` [R] (None disables); call after set_xs. Each
        outer runs n_outer coarse power iterations with n_inner over-relaxed (omega) sweeps per
        group."""
        if cell is None:
            self._lib.orc_set_cmfd(self._h, None, 0, 0, 0, 1.0)
            return
        c = _i32a(cell)
        self._lib.orc_set_cmfd(self._h, _p(c, _i32), int(n_cells), int(n_outer), int(n_inner), float(omega))
        self._cell = c

    def set_scattering(self, sigma_sl=None):
        """Anisotropic scattering: sigma_sl [L][M][G][G] holds Sigma_s,l (g' -> g) for l = 1..L;
        None restores isotropic scattering. Call after set_xs."""
        if sigma_sl is None:
            self._lib.orc_set_scattering(self._h, 0, None)
            return
        a = _f64(sigma_sl)
        rc = self._lib.orc_set_scattering(self._h, int(a.shape[0]), _p(a, _d))
        if rc:
            raise RuntimeError("oracle: " + self._lib.orc_error(self._h).decode())
        self._ssl = a

    def set_axial(self, dz, mat3=None, bc=(0, 0)):
        """DGMOC on len(dz) axial planes: mat3 [nz][R] materials (None: the planar ones in every
        plane), bc = (bottom, top), 0 vacuum 1 reflective. Call after set_xs; the state restarts
        flat. An empty dz returns to the planar method."""
        dz = _f64(dz)
        m3 = None if mat3 is None else _i32a(mat3)
        if m3 is not None:
            assert m3.shape == (dz.size, self.n_regions)
        rc = self._lib.orc_set_axial(self._h, int(dz.size), _p(dz, _d), None if m3 is None else _p(m3, _i32),
                                     int(bc[0]), int(bc[1]))
        if rc:
            raise RuntimeError("oracle: " + self._lib.orc_error(self._h).decode())
        self.nz = int(dz.size)
        self._dz, self._m3 = dz, m3

    def set_dg_cmfd(self, n_outer: int = 0, n_inner: int = 4, omega: float = 1.0):
        """Axial coarse-mesh acceleration of DGMOC (coarse cells = planes); n_outer = 0 disables."""
        if self._lib.orc_set_dg_cmfd(self._h, int(n_outer), int(n_inner), float(omega)):
            raise RuntimeError("oracle: " + self._lib.orc_error(self._h).decode())

    def flux3(self):
        """(phi [nz][R][2][G]: plane-average and linear moments, k)."""
        phi = np.zeros((self.nz, self.n_regions, 2, self.G))
        k = ctypes.c_double()
        self._lib.orc_get_flux3(self._h, _p(phi, _d), ctypes.byref(k))
        return phi, k.value

    def leakage3(self) -> np.ndarray:
        """[3][G] leakage of the last DGMOC sweep: radial, bottom, top."""
        a = np.zeros((3, self.G))
        self._lib.orc_get_leakage3(self._h, _p(a, _d))
        return a

    def set_state(self, phi=None, k: float = 1.0, psi=None):
        pp = None if phi is None else _f64(phi)
        ps = None if psi is None else _f64(psi)
        if pp is not None and getattr(self, "nz", 0):
            assert pp.size == self.nz * self.n_regions * 2 * self.G and ps is None
        elif pp is not None:
            assert pp.size == self.n_regions * self.G
        if ps is not None:
            assert ps.size == self.n_tracks * 2 * self.n_polar * self.G
        self._lib.orc_set_state(self._h, None if pp is None else _p(pp, _d), float(k),
                                None if ps is None else _p(ps, _d))

    def get_state(self, with_psi: bool = False):
        phi = np.zeros((self.n_regions, self.G))
        k = ctypes.c_double()
        psi = np.zeros((self.n_tracks, 2, self.n_polar, self.G)) if with_psi else None
        self._lib.orc_get_state(self._h, _p(phi, _d), ctypes.byref(k), None if psi is None else _p(psi, _d))
        return (phi, k.value, psi) if with_psi else (phi, k.value)

    def q(self) -> np.ndarray:
        a = np.zeros((self.n_regions, self.G))
        self._lib.orc_get_q(self._h, _p(a, _d))
        return a

    def tally(self) -> np.ndarray:
        a = np.zeros((self.n_regions, self.G))
        self._lib.orc_get_tally(self._h, _p(a, _d))
        return a

    def leakage(self) -> np.ndarray:
        a = np.zeros(self.G)
        self._lib.orc_get_leakage(self._h, _p(a, _d))
        return a

    def normalise(self):
        self._lib.orc_normalise(self._h)

    def outer(self, eigen: bool = True) -> float:
        return float(self._lib.orc_outer(self._h, 1 if eigen else 0))

    def iterate(self, eigen: bool = True, tol_k: float = 1e-6, tol_f: float = 1e-6, max_outer: int = 10000):
        k, n, r = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        rc = self._lib.orc_iterate(self._h, 1 if eigen else 0, float(tol_k), float(tol_f), int(max_outer),
                                   ctypes.byref(k), ctypes.byref(n), ctypes.byref(r))
        return k.value, n.value, r.value, rc == 0


def legendre(l: int, x: float) -> float:
    """The oracle's Legendre polynomial P_l(x)."""
    return float(_load().orc_legendre(int(l), float(x)))


def expm2(M) -> np.ndarray:
    """The oracle's exponential of a 2 x 2 matrix."""
    M = _f64(M).reshape(2, 2)
    E = np.zeros((2, 2))
    _load().orc_expm2(_p(M, _d), _p(E, _d))
    return E


def dg_segment(y0, psi_in, length, sin_theta, mu, h, sig, q0, q1s):
    """One DGMOC segment: (y at the end, segment integral of y) for y = (a, b)."""
    y0 = _f64(y0)
    y1, yi = np.zeros(2), np.zeros(2)
    _load().orc_dg_segment(_p(y0, _d), float(psi_in), float(length), float(sin_theta), float(mu), float(h),
                           float(sig), float(q0), float(q1s), _p(y1, _d), _p(yi, _d))
    return y1, yi


def track_sweep(sig, qr, length, sin_theta: float, psi_in: float) -> np.ndarray:
    """psi after each segment of one characteristic (one group, one polar angle)."""
    lib = _load()
    sig, qr, length = _f64(sig), _f64(qr), _f64(length)
    out = np.zeros(sig.shape[0])
    lib.orc_track_sweep(sig.shape[0], _p(sig, _d), _p(qr, _d), _p(length, _d), float(sin_theta),
                        float(psi_in), _p(out, _d))
    return out


def sample_fixed_source(mesh, n_azim, spacing, sin_theta, polar_w, xs, S, phi0, psi0, sample):
    """Flux of the sampled regions after one fixed-source outer from (phi0, psi0), computed from
    only the rays that cross them; also returns their tracked areas. Rectangular meshes, or any
    mesh whose walls are all vacuum (each in-mesh chord a track with zero inflow; psi0 unused)."""
    lib = _load()
    xy, tri, mat, bbox, bc = _f64(mesh.xy), _i32a(mesh.tri), _i32a(mesh.mat), _f64(mesh.bbox), _i32a(mesh.bc)
    st_, pw = _f64(sin_theta), _f64(polar_w)
    sig, ss = _f64(xs.sigma_t), _f64(xs.sigma_s)
    S, phi0, psi0 = _f64(S), _f64(phi0), _f64(psi0)
    sample = _i32a(sample)
    G = sig.shape[1]
    out = np.zeros((sample.size, G))
    area = np.zeros(sample.size)
    rc = lib.orc_sample_fixed_source(xy.shape[0], _p(xy, _d), tri.shape[0], _p(tri, _i32), _p(mat, _i32),
                                     _p(bbox, _d), _p(bc, _i32), int(n_azim), float(spacing), st_.size, _p(st_, _d), _p(pw, _d),
                                     sig.shape[0], G, _p(sig, _d), _p(ss, _d), _p(S, _d), _p(phi0, _d),
                                     _p(psi0, _d), sample.size, _p(sample, _i32), _p(out, _d), _p(area, _d))
    if rc != 0:
        raise RuntimeError(f"oracle sample_fixed_source failed ({rc})")
    return out, area
