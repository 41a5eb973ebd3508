"""Thin ctypes binding of the C ABI in include/moc_gb300.h (argument marshalling only).

Every step of the transport calculation runs in the CUDA library; this module converts numpy
arrays to pointers, checks status codes and raises MocError with the library's message. There
is no Python or CPU fallback: if the built library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmoc_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

MOC_FP64, MOC_FP32, MOC_FP32_PLAIN = 0, 1, 2
PRECISIONS = {"fp64": MOC_FP64, "fp32": MOC_FP32, "fp32_plain": MOC_FP32_PLAIN}
STATUS = {0: "MOC_OK", -1: "MOC_ERR_ARG", -2: "MOC_ERR_CUDA", -3: "MOC_ERR_OOM", -4: "MOC_ERR_STATE",
          -5: "MOC_ERR_NOT_CONVERGED", -6: "MOC_ERR_NONFINITE", -7: "MOC_ERR_GEOMETRY"}

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_lib = None
_lock = threading.Lock()


class MocError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def header_symbols() -> list:
    """Names of the functions declared in include/*.h."""
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            txt = open(os.path.join(INCLUDE, h)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(moc_\w+)\s*\(", txt, re.M))
    return sorted(names)


def load_library(path: Optional[str] = None):
    """Load the built library (raises OSError/ImportError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"CUDA library not built: {p} is missing (run paper_2607_01591_gb300.build.build())")
        lib = ctypes.CDLL(p)
        sig = {
            "moc_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _vp]),
            "moc_destroy": (None, [_vp]),
            "moc_last_error": (ctypes.c_char_p, [_vp]),
            "moc_set_mesh": (ctypes.c_int, [_vp, ctypes.c_int, _d, ctypes.c_int, _i32, _i32, _d, _i32]),
            "moc_set_quadrature": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _d, _d]),
            "moc_generate_tracks": (ctypes.c_int, [_vp]),
            "moc_set_tracks": (ctypes.c_int, [_vp, ctypes.c_int64, _i64, _i32, _d, _i32, _d, _d, _i32]),
            "moc_sweep_dev": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "moc_get_stats": (ctypes.c_int, [_vp, _d, _d]),
            "moc_get_history": (ctypes.c_int, [_vp, _d, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
            "moc_set_axial": (ctypes.c_int, [_vp, ctypes.c_int, _d, _i32, ctypes.c_int, ctypes.c_int]),
            "moc_set_dg_cmfd": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
            "moc_set_scattering": (ctypes.c_int, [_vp, ctypes.c_int, _d]),
            "moc_set_ray_layout": (ctypes.c_int, [_vp, ctypes.c_int]),
            "moc_generate_tracks_device": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
            "moc_get_track_counts": (ctypes.c_int, [_vp, _i64, _i64]),
            "moc_get_tracks": (ctypes.c_int, [_vp, _i64, _i32, _d, _i32, _d, _i64]),
            "moc_get_quadrature": (ctypes.c_int, [_vp, _d, _d, _d]),
            "moc_get_region_areas": (ctypes.c_int, [_vp, _d]),
            "moc_set_xs": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _d, _d, _d, _d]),
            "moc_set_fixed_source": (ctypes.c_int, [_vp, _d]),
            "moc_set_state": (ctypes.c_int, [_vp, _d, ctypes.c_double, _d]),
            "moc_get_state": (ctypes.c_int, [_vp, _d, _d, _d]),
            "moc_update_source": (ctypes.c_int, [_vp]),
            "moc_sweep": (ctypes.c_int, [_vp]),
            "moc_outer": (ctypes.c_int, [_vp, ctypes.c_int, _d, _d]),
            "moc_power_iterate": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                 _d, ctypes.POINTER(ctypes.c_int), _d]),
            "moc_enable_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
            "moc_get_timing": (ctypes.c_int, [_vp, _d, _i64]),
            "moc_get_work": (ctypes.c_int, [_vp, _i64, _i64, ctypes.POINTER(ctypes.c_int)]),
            "moc_synchronize": (ctypes.c_int, [_vp]),
            "moc_set_cmfd": (ctypes.c_int, [_vp, _i32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
            "moc_set_cmfd_tolerance": (ctypes.c_int, [_vp, ctypes.c_double]),
            "moc_get_cmfd_iterations": (ctypes.c_int, [_vp, _i64]),
            "moc_ws_features": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int, _vp]),
            "moc_ws_apply": (ctypes.c_int, [_vp, _vp, _d]),
            "moc_mlp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_uint64]),
            "moc_mlp_destroy": (None, [_vp]),
            "moc_mlp_last_error": (ctypes.c_char_p, [_vp]),
            "moc_mlp_dims": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _i64]),
            "moc_mlp_get_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
            "moc_mlp_set_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
            "moc_mlp_set_normalization": (ctypes.c_int, [_vp] + [ctypes.POINTER(ctypes.c_float)] * 4),
            "moc_mlp_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
            "moc_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_float,
                                                  ctypes.POINTER(ctypes.c_float), _vp]),
            "moc_mlp_gradients": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float),
                                                 ctypes.POINTER(ctypes.c_float), _vp]),
            "moc_mlp_forward_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
            "moc_eval_one_minus_exp_f32": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                                          ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
            "moc_eval_one_minus_exp_f32x2": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                                            ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
            "moc_probe_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _d, _d, ctypes.POINTER(ctypes.c_int)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(x) -> int:
    """Device address of a torch tensor (or an int address)."""
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


class Mlp:
    """The warm-start network of include/moc_mlp.h (bf16 weights, FP32 accumulate, Adam)."""

    def __init__(self, n_in: int, width: int = 256, n_out: int = 8, seed: int = 0, device: int = 0):
        self._lib = load_library()
        h = _vp()
        rc = self._lib.moc_mlp_create(ctypes.byref(h), int(device), int(n_in), int(width), int(n_out), int(seed))
        if rc != 0:
            raise MocError(rc, "moc_mlp_create failed")
        self._h = h
        dims = (ctypes.c_int * 5)()
        npar = ctypes.c_int64()
        self._lib.moc_mlp_dims(h, dims, ctypes.byref(npar))
        self.dims = list(dims)
        self.n_params = npar.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.moc_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise MocError(rc, self._lib.moc_mlp_last_error(self._h).decode())

    @staticmethod
    def _fp(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, np.float32)
        self._check(self._lib.moc_mlp_get_params(self._h, self._fp(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(self._lib.moc_mlp_set_params(self._h, self._fp(p)))

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (in_mean, in_std, out_mean, out_std)]
        self.norm = a
        self._check(self._lib.moc_mlp_set_normalization(self._h, *[self._fp(v) for v in a]))

    def forward(self, x, y, n: int, stream=None):
        self._check(self._lib.moc_mlp_forward(self._h, _vp(_ptr(x)), _vp(_ptr(y)), int(n),
                                              None if stream is None else _vp(stream)))

    def forward_noalloc(self, x, y, n: int, stream=None):
        """Forward pass in the library's fixed workspace; allocates nothing (moc_mlp_forward_noalloc)."""
        self._check(self._lib.moc_mlp_forward_noalloc(self._h, _vp(_ptr(x)), _vp(_ptr(y)), int(n),
                                                      None if stream is None else _vp(stream)))

    def train_step(self, x, y, n: int, lr: float, stream=None, want_loss: bool = False):
        loss = ctypes.c_float()
        self._check(self._lib.moc_mlp_train_step(self._h, _vp(_ptr(x)), _vp(_ptr(y)), int(n), float(lr),
                                                 ctypes.byref(loss) if want_loss else None,
                                                 None if stream is None else _vp(stream)))
        return loss.value if want_loss else None

    def gradients(self, x, y, n: int, stream=None):
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_float()
        self._check(self._lib.moc_mlp_gradients(self._h, _vp(_ptr(x)), _vp(_ptr(y)), int(n), self._fp(g),
                                                ctypes.byref(loss), None if stream is None else _vp(stream)))
        return g, loss.value


def eval_one_minus_exp_f32(tau: np.ndarray, device: int = 0, packed: bool = False) -> np.ndarray:
    """The library's FP32 1 - exp(-tau) evaluated on the GPU (packed: its f32x2 form)."""
    lib = load_library()
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    out = np.empty_like(tau)
    fp = ctypes.POINTER(ctypes.c_float)
    name = "moc_eval_one_minus_exp_f32x2" if packed else "moc_eval_one_minus_exp_f32"
    rc = getattr(lib, name)(int(device), tau.ctypes.data_as(fp), out.ctypes.data_as(fp), tau.size)
    if rc != 0:
        raise MocError(rc, name + " failed")
    return out


PROBES = ("ffma", "dfma", "red_f32", "red_f32x2", "red_f32x4", "red_f32x4_pair", "red_f32_row8", "atom_f32",
          "red_f64", "red_f32x4_hbm")


def probe_rate(kind: str, device: int = 0) -> dict:
    """One hardware rate probe of include/moc_probe.h: lane operations/s, 32-byte sectors/s and
    the device's multiprocessor count."""
    lib = load_library()
    ops, sec, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    rc = lib.moc_probe_rate(int(device), PROBES.index(kind), ctypes.byref(ops), ctypes.byref(sec), ctypes.byref(sms))
    if rc != 0:
        raise MocError(rc, f"moc_probe_rate({kind}) failed")
    return {"lane_ops_per_s": ops.value, "sectors_per_s": sec.value, "sm_count": sms.value}


class Moc:
    """One transport problem on one GPU (device >= 0) or host-only geometry (device = -1)."""

    def __init__(self, device: int = 0, precision: str = "fp32", stream: Optional[int] = None):
        self._lib = load_library()
        h = _vp()
        self.precision = precision
        rc = self._lib.moc_create(ctypes.byref(h), int(device), PRECISIONS[precision],
                                  None if stream is None else _vp(stream))
        if rc != 0:
            raise MocError(rc, "moc_create failed")
        self._h = h
        self.device = device
        self.G = 0
        self.n_polar = 0
        self.n_regions = 0

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.moc_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise MocError(rc, self._lib.moc_last_error(self._h).decode())

    # geometry -------------------------------------------------------------------------------
    def set_mesh(self, mesh):
        xy, tri, mat = _f64(mesh.xy), _i32a(mesh.tri), _i32a(mesh.mat)
        bbox, bc = _f64(mesh.bbox), _i32a(mesh.bc)
        self._check(self._lib.moc_set_mesh(self._h, xy.shape[0], _p(xy, _d), tri.shape[0], _p(tri, _i32),
                                           _p(mat, _i32), _p(bbox, _d), _p(bc, _i32)))
        self.n_regions = int(tri.shape[0])

    def set_quadrature(self, n_azim: int, spacing: float, sin_theta, polar_w):
        st, pw = _f64(sin_theta), _f64(polar_w)
        self._check(self._lib.moc_set_quadrature(self._h, int(n_azim), float(spacing), st.shape[0], _p(st, _d),
                                                 _p(pw, _d)))
        self.n_polar = int(st.shape[0])

    def generate_tracks(self):
        self._check(self._lib.moc_generate_tracks(self._h))

    def set_tracks(self, seg_off, seg_region, seg_len, track_azim, azim_weight, azim_spacing, link):
        """Tracks from the caller (see moc_set_tracks): segment CSR, direction per track, weights
        and spacings per direction, links [T][2] as 2 t' + d' or -1."""
        so = np.ascontiguousarray(seg_off, dtype=np.int64)
        sr, sl = _i32a(seg_region), _f64(seg_len)
        ta, aw, asp = _i32a(track_azim), _f64(azim_weight), _f64(azim_spacing)
        lk = _i32a(np.asarray(link).reshape(-1))
        self._check(self._lib.moc_set_tracks(self._h, int(so.size - 1), _p(so, _i64), _p(sr, _i32), _p(sl, _d),
                                             _p(ta, _i32), _p(aw, _d), _p(asp, _d), _p(lk, _i32)))

    def sweep_dev(self, phi_in=None, phi_out=None, stream=None):
        """One outer with caller-owned device flux tensors [n_tri][G] (torch CUDA tensors of the
        context's type, or None) on `stream` (a torch stream or None: the context's stream)."""
        def ptr(t):
            if t is None:
                return None
            assert t.is_cuda and t.is_contiguous() and t.numel() == self.n_regions * self.G
            return ctypes.c_void_p(t.data_ptr())
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(self._lib.moc_sweep_dev(self._h, st, ptr(phi_in), ptr(phi_out)))

    def history(self, max_entries: int = 4096) -> np.ndarray:
        """[n][4] rows (outers, k, k before the last outer, residual) of the recorded checks."""
        buf = np.zeros((max_entries, 4))
        n = ctypes.c_int()
        self._check(self._lib.moc_get_history(self._h, _p(buf, _d), int(max_entries), ctypes.byref(n)))
        return buf[: n.value].copy()

    def stats(self):
        """(average sweep ms, updates/s) over the sweeps timed since enable_timing(True)."""
        ms, ups = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.moc_get_stats(self._h, ctypes.byref(ms), ctypes.byref(ups)))
        return ms.value, ups.value

    def set_ray_layout(self, layout: int):
        """0: cyclic modular rays over the bounding box; 1: back projection (vacuum boundaries)."""
        self._check(self._lib.moc_set_ray_layout(self._h, int(layout)))

    def generate_tracks_device(self) -> float:
        """Tracks with the half-edge walk on the GPU (bit-identical to generate_tracks); returns the
        device time of the walk in ms."""
        ms = ctypes.c_double()
        self._check(self._lib.moc_generate_tracks_device(self._h, ctypes.byref(ms)))
        return ms.value

    def track_counts(self):
        T, S = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.moc_get_track_counts(self._h, ctypes.byref(T), ctypes.byref(S)))
        return T.value, S.value

    def tracks(self) -> dict:
        T, S = self.track_counts()
        off, reg, ln = np.zeros(T + 1, np.int64), np.zeros(S, np.int32), np.zeros(S)
        dr, xy, link = np.zeros(T, np.int32), np.zeros((T, 4)), np.zeros((T, 2), np.int64)
        self._check(self._lib.moc_get_tracks(self._h, _p(off, _i64), _p(reg, _i32), _p(ln, _d), _p(dr, _i32),
                                             _p(xy, _d), _p(link, _i64)))
        return dict(seg_off=off, seg_region=reg, seg_len=ln, track_dir=dr, track_xy=xy, link=link)

    def quadrature(self, n_dir: int) -> dict:
        phi, delta, omega = np.zeros(n_dir), np.zeros(n_dir), np.zeros(n_dir)
        self._check(self._lib.moc_get_quadrature(self._h, _p(phi, _d), _p(delta, _d), _p(omega, _d)))
        return dict(phi=phi, delta=delta, omega=omega)

    def areas(self) -> np.ndarray:
        a = np.zeros(self.n_regions)
        self._check(self._lib.moc_get_region_areas(self._h, _p(a, _d)))
        return a

    # physics --------------------------------------------------------------------------------
    def set_xs(self, xs):
        st, nsf, chi, ss = _f64(xs.sigma_t), _f64(xs.nu_sigma_f), _f64(xs.chi), _f64(xs.sigma_s)
        M, G = st.shape
        self._check(self._lib.moc_set_xs(self._h, M, G, _p(st, _d), _p(nsf, _d), _p(chi, _d), _p(ss, _d)))
        self.G = G
        self.nz = 0

    def set_fixed_source(self, S):
        S = _f64(S)
        if S is not None:
            assert S.shape == (self.n_regions, self.G)
        self._check(self._lib.moc_set_fixed_source(self._h, _p(S, _d)))

    def set_scattering(self, sigma_sl=None):
        """Anisotropic scattering: sigma_sl [L][M][G][G] = Sigma_s,l for l = 1..L (None: isotropic)."""
        if sigma_sl is None:
            self._check(self._lib.moc_set_scattering(self._h, 0, None))
            return
        a = _f64(sigma_sl)
        self._check(self._lib.moc_set_scattering(self._h, int(a.shape[0]), _p(a, _d)))

    def set_cmfd(self, cell=None, n_cells: int = 0, n_outer: int = 6, n_inner: int = 6, omega: float = 1.0):
        """CMFD acceleration on the coarse cells `cell` [n_tri] (None switches it off): per outer,
        n_outer coarse power iterations with n_inner over-relaxed (omega) sweeps per group."""
        if cell is None:
            self._check(self._lib.moc_set_cmfd(self._h, None, 0, 0, 0, 1.0))
            return
        cell = _i32a(cell)
        assert cell.size == self.n_regions
        self._check(self._lib.moc_set_cmfd(self._h, _p(cell, _i32), int(n_cells), int(n_outer), int(n_inner),
                                           float(omega)))

    def set_cmfd_tolerance(self, tol: float):
        """Stop each outer's coarse power iteration once k and the coarse fission source settle to
        tol (0: the fixed count of set_cmfd)."""
        self._check(self._lib.moc_set_cmfd_tolerance(self._h, float(tol)))

    def cmfd_iterations(self) -> int:
        """Coarse power iterations run since the last state reset, summed over outers."""
        n = ctypes.c_int64()
        self._check(self._lib.moc_get_cmfd_iterations(self._h, ctypes.byref(n)))
        return n.value

    def set_axial(self, dz, mat3=None, bc=(0, 0)):
        """DGMOC on len(dz) axial planes (empty: back to the planar method): mat3 [nz][R] materials
        (None: the mesh's in every plane), bc = (bottom, top), 0 vacuum 1 reflective. The flux of
        get_state/set_state is then [nz][R][2][G] (plane average, linear coefficient)."""
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        m3 = None if mat3 is None else np.ascontiguousarray(mat3, dtype=np.int32)
        if m3 is not None:
            assert m3.shape == (dz.size, self.n_regions)
        self._check(self._lib.moc_set_axial(self._h, int(dz.size), _p(dz, _d) if dz.size else None,
                                            None if m3 is None else _p(m3, _i32), int(bc[0]), int(bc[1])))
        self.nz = int(dz.size)

    def set_dg_cmfd(self, n_outer: int = 0, n_inner: int = 4, omega: float = 1.0):
        """Axial coarse-mesh acceleration of DGMOC (planes as coarse cells); n_outer = 0 disables.
        Call after set_axial."""
        self._check(self._lib.moc_set_dg_cmfd(self._h, int(n_outer), int(n_inner), float(omega)))

    def _phi_shape(self):
        nz = getattr(self, "nz", 0)
        return (nz, self.n_regions, 2, self.G) if nz else (self.n_regions, self.G)

    def set_state(self, phi=None, k: float = 1.0, psi=None):
        phi, psi = _f64(phi), _f64(psi)
        if phi is not None:
            assert phi.size == int(np.prod(self._phi_shape()))
        if psi is not None:
            T, _ = self.track_counts()
            assert psi.size == T * 2 * self.n_polar * self.G
        self._check(self._lib.moc_set_state(self._h, _p(phi, _d), float(k), _p(psi, _d)))

    def get_state(self, with_psi: bool = False, out=None):
        """(phi, k) or (phi, k, psi); `out` = (phi, psi or None) writes into caller arrays
        (float64, C-contiguous; pinned ones are written in place by the device)."""
        k = ctypes.c_double()
        if out is not None:
            phi, psi = out
            assert phi.dtype == np.float64 and phi.flags.c_contiguous and phi.size == int(np.prod(self._phi_shape()))
            with_psi = psi is not None
        else:
            phi = np.zeros(self._phi_shape())
            psi = None
            if with_psi:
                T, _ = self.track_counts()
                psi = np.zeros((T, 2, self.n_polar, self.G))
        self._check(self._lib.moc_get_state(self._h, _p(phi, _d), ctypes.byref(k), _p(psi, _d)))
        return (phi, k.value, psi) if with_psi else (phi, k.value)

    def update_source(self):
        self._check(self._lib.moc_update_source(self._h))

    def sweep(self):
        self._check(self._lib.moc_sweep(self._h))

    def outer(self, n: int = 1, read: bool = True):
        k, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.moc_outer(self._h, int(n), ctypes.byref(k) if read else None,
                                        ctypes.byref(r) if read else None))
        return (k.value, r.value) if read else None

    def power_iterate(self, tol_k: float = 1e-6, tol_flux: float = 1e-6, max_outer: int = 10000,
                      check_every: int = 10, raise_on_fail: bool = True):
        k, n, r = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        rc = self._lib.moc_power_iterate(self._h, float(tol_k), float(tol_flux), int(max_outer), int(check_every),
                                         ctypes.byref(k), ctypes.byref(n), ctypes.byref(r))
        if rc != 0 and (raise_on_fail or rc != -5):
            self._check(rc)
        return k.value, n.value, r.value, rc == 0

    def enable_timing(self, on: bool = True):
        self._check(self._lib.moc_enable_timing(self._h, 1 if on else 0))

    def timing(self):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self._lib.moc_get_timing(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def work(self):
        s, u, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        self._check(self._lib.moc_get_work(self._h, ctypes.byref(s), ctypes.byref(u), ctypes.byref(k)))
        return s.value, u.value, k.value

    def synchronize(self):
        self._check(self._lib.moc_synchronize(self._h))

    def ws_features(self, geo_ptr, n_geo: int, glob, feat_ptr):
        """Per-region network inputs on the device (see moc_ws_features)."""
        g = np.ascontiguousarray(glob, dtype=np.float32)
        self._check(self._lib.moc_ws_features(self._h, _vp(_ptr(geo_ptr)) if n_geo else None, int(n_geo),
                                              g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), g.size,
                                              _vp(_ptr(feat_ptr))))

    def ws_apply(self, pred_ptr) -> float:
        """Set the iterate from a network prediction on the device (see moc_ws_apply)."""
        k = ctypes.c_double()
        self._check(self._lib.moc_ws_apply(self._h, _vp(_ptr(pred_ptr)), ctypes.byref(k)))
        return k.value

    @classmethod
    def from_problem(cls, prob, device: int = 0, precision: str = "fp32", stream=None, with_xs: bool = True,
                     device_tracking: bool = False):
        m = cls(device, precision, stream)
        m.set_mesh(prob.mesh)
        m.set_quadrature(prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w)
        if getattr(prob, "ray_layout", 0):
            m.set_ray_layout(prob.ray_layout)
        if device_tracking:
            m.generate_tracks_device()
        else:
            m.generate_tracks()
        if with_xs and device >= 0:
            m.set_xs(prob.xs)
            if prob.fixed_source is not None:
                m.set_fixed_source(prob.fixed_source)
        return m
