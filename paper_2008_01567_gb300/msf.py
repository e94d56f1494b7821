"""Thin ctypes binding of libmsf.so (include/msf.h).

Argument marshalling only: every computation runs in the library's CUDA kernels.
Tensors are torch CUDA tensors (float32, contiguous); their device pointers and
the current CUDA stream are passed through.  There is no CPU fallback: if the
library is missing or the device is not sm_103, calls raise MsfError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmsf.so")

MSF_OK = 0
STATUS = {0: "MSF_OK", 1: "MSF_ERR_ARG", 2: "MSF_ERR_CUDA", 3: "MSF_ERR_NOMEM", 4: "MSF_ERR_TIMEOUT",
          5: "MSF_ERR_NUMERIC", 6: "MSF_ERR_UNSUPPORTED"}
MSF_XY_T, MSF_YZ_T, MSF_ZX_T = 0, 1, 2
MSF_PRIOR_QGGMRF, MSF_PRIOR_CNN = 0, 1
MSF_CONSENSUS_SUMS, MSF_CONSENSUS_WORK = 2432, 2434


class MsfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class msf_vol(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int),
                ("voxel", ctypes.c_double)]


class msf_geom(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_int), ("nv", ctypes.c_int), ("views", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double), ("dso", ctypes.c_double),
                ("dsd", ctypes.c_double), ("angles", ctypes.POINTER(ctypes.c_double))]


class msf_mrf(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("q", ctypes.c_double), ("T", ctypes.c_double),
                ("sigma_x", ctypes.c_double), ("b_temporal", ctypes.c_double)]


class msf_mace_desc(ctypes.Structure):
    _fields_ = [("proj", ctypes.c_void_p), ("prior", ctypes.c_int), ("K", ctypes.c_int),
                ("cnn", ctypes.c_void_p), ("mrf", msf_mrf), ("d_W", ctypes.c_void_p),
                ("d_X", ctypes.c_void_p), ("d_y", ctypes.c_void_p), ("d_lambda", ctypes.c_void_p),
                ("orient", ctypes.c_int)]


class msf_mace_params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("sigma", ctypes.c_double), ("mu", ctypes.c_double * 4),
                ("n_cg", ctypes.c_int), ("n_sweeps", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("n_icd", ctypes.c_int)]


# exported symbol -> (restype, argtypes)
_P, _I, _D, _Z, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_float
_SIGS = {
    "msf_last_error": (ctypes.c_char_p, []),
    "msf_version": (ctypes.c_char_p, []),
    "msf_profile_enable": (None, [_I]),
    "msf_profile_reset": (None, []),
    "msf_profile_read": (_I, [_I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(_D)]),
    "msf_projector_create": (_I, [ctypes.POINTER(msf_geom), ctypes.POINTER(msf_vol), ctypes.POINTER(_P)]),
    "msf_projector_destroy": (None, [_P]),
    "msf_projector_bytes": (_Z, [_P]),
    "msf_project": (_I, [_P, _P, _P, _P]),
    "msf_backproject": (_I, [_P, _P, _P, _P]),
    "msf_project_static": (_I, [ctypes.POINTER(msf_geom), ctypes.POINTER(msf_vol), _P, _P, _P]),
    "msf_weights": (_I, [_P, _P, _P, _Z, _D, _D, _P]),
    "msf_dataprox_create": (_I, [_P, ctypes.POINTER(_P)]),
    "msf_dataprox_destroy": (None, [_P]),
    "msf_prox_data": (_I, [_P, _P, _P, _P, _P, _D, _I, _P]),
    "msf_prox_data_icd": (_I, [_P, _P, _P, _P, _P, _D, _I, _P]),
    "msf_map_create": (_I, [_P, ctypes.POINTER(_P)]),
    "msf_map_destroy": (None, [_P]),
    "msf_map_solve": (_I, [_P, ctypes.POINTER(msf_mrf), _D, _P, _P, _P, _I, _I, _P]),
    "msf_map_cost": (_I, [_P, ctypes.POINTER(msf_mrf), _D, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "msf_fixcorr_create": (_I, [_P, ctypes.POINTER(_P)]),
    "msf_fixcorr_destroy": (None, [_P]),
    "msf_fixture_correct": (_I, [_P, _P, _P, _D, _D, _P, ctypes.POINTER(_D), _P]),
    "msf_prox_qggmrf": (_I, [ctypes.POINTER(msf_vol), ctypes.POINTER(msf_mrf), _P, _P, _D, _I, _P]),
    "msf_cnn_create": (_I, [ctypes.c_int64, ctypes.POINTER(_P)]),
    "msf_cnn_destroy": (None, [_P]),
    "msf_cnn_param_count": (_Z, []),
    "msf_cnn_set_params": (_I, [_P, _P, _Z]),
    "msf_cnn_get_params": (_I, [_P, _P, _Z]),
    "msf_denoise": (_I, [_P, _I, ctypes.POINTER(msf_vol), _P, _P, _P]),
    "msf_denoise_batch": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(msf_vol), ctypes.POINTER(_P),
                               ctypes.POINTER(_P), _P]),
    "msf_cnn_set_tuning": (_I, [_P, _I, ctypes.POINTER(msf_vol), _I, _I]),
    "msf_cnn_autotune": (_I, [_P, ctypes.POINTER(msf_vol), _P, _P, _P, ctypes.POINTER(_I)]),
    "msf_train_step": (_I, [_P, _P, _P, _I, _I, _I, _F, ctypes.POINTER(_F), _P]),
    "msf_cnn_train_reserve": (_I, [_P, ctypes.c_int64]),
    "msf_cnn_get_grads": (_I, [_P, _P, _Z]),
    "msf_cnn_train_trace": (_I, [_P, _I]),
    "msf_cnn_train_tensor": (_I, [_P, _I, _I, _P, _Z]),
    "msf_training_batch": (_I, [_P, ctypes.POINTER(msf_vol), _I, _I, _I, _D, _D, ctypes.c_uint64, _P, _P, _P]),
    "msf_mace_create": (_I, [ctypes.POINTER(msf_mace_desc), ctypes.POINTER(_P)]),
    "msf_mace_destroy": (None, [_P]),
    "msf_mace_step": (_I, [_P, ctypes.POINTER(msf_mace_params), ctypes.POINTER(_D), _P]),
    "msf_mace_set_counts": (_I, [_P, _P, _D, _D, _P]),
    "msf_mace_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "msf_mace_batch_destroy": (None, [_P]),
    "msf_mace_batch_step": (_I, [_P, ctypes.POINTER(msf_mace_params), ctypes.POINTER(_D), _P]),
    "msf_projector_autotune": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "msf_projector_set_tuning": (_I, [_P, _I, _I, _I]),
    "msf_mace_consensus": (_I, [_P, _P, _I, _Z, ctypes.POINTER(ctypes.c_double), ctypes.c_double, _P, _P]),
    "msf_selftest_wait": (_I, [ctypes.c_uint64, _P]),
    "msf_phantom_voxelize": (_I, [ctypes.POINTER(msf_vol), _P, _I, _I, _P, _P]),
    "msf_phantom_project": (_I, [_P, _P, _I, _P, _P]),
}

_lib = None


def lib():
    """Loads libmsf.so (built by paper_2008_01567_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MsfError(6, f"{LIB_PATH} is missing: run paper_2008_01567_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != MSF_OK:
        raise MsfError(st, lib().msf_last_error().decode())


def _ptr(t) -> int:
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _f32(t) -> int:
    import torch
    if t is not None and t.dtype != torch.float32:
        raise ValueError(f"expected float32, got {t.dtype}")
    return _ptr(t)


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def msf_profile_enable(on: bool):
    lib().msf_profile_enable(1 if on else 0)


def msf_profile_reset():
    lib().msf_profile_reset()


def msf_profile_read() -> dict:
    """{kernel name: (launches, total_ms)} since the last reset."""
    out = {}
    name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
    count = lib().msf_profile_read(-1, None, None, None)
    for i in range(count):
        lib().msf_profile_read(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms))
        out[name.value.decode()] = (n.value, ms.value)
    return out


def vol_of(scan) -> msf_vol:
    return msf_vol(scan.n, scan.n, scan.n, scan.nt, scan.vox)


# ------------------------------------------------------------------ projector


class Projector:
    """Owns an msf_projector plan for a synth.Scan-like description."""

    def __init__(self, scan, angles=None):
        ang = np.ascontiguousarray(scan.angles() if angles is None else angles, dtype=np.float64).ravel()
        self._angles = ang
        self.geom = msf_geom(scan.nu, scan.nv, scan.views, scan.pitch, scan.pitch, scan.dso, scan.dsd,
                             ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self.vol = vol_of(scan)
        self.scan = scan
        h = ctypes.c_void_p()
        _check(lib().msf_projector_create(ctypes.byref(self.geom), ctypes.byref(self.vol), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_projector_destroy(self.handle)
            self.handle = None

    __del__ = close

    def nbytes(self) -> int:
        return lib().msf_projector_bytes(self.handle)


def msf_project(proj: Projector, x, y, stream=None):
    _check(lib().msf_project(proj.handle, _f32(x), _f32(y), _stream(stream)))


def msf_backproject(proj: Projector, y, x, stream=None):
    _check(lib().msf_backproject(proj.handle, _f32(y), _f32(x), _stream(stream)))


def msf_project_static(scan, x, y, angles=None, stream=None):
    """Forward projection without a plan and without any device allocation
    (the ray table lives in the library's fixed static device array)."""
    ang = np.ascontiguousarray(scan.angles() if angles is None else angles, dtype=np.float64).ravel()
    geom = msf_geom(scan.nu, scan.nv, scan.views, scan.pitch, scan.pitch, scan.dso, scan.dsd,
                    ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    vol = vol_of(scan)
    _check(lib().msf_project_static(ctypes.byref(geom), ctypes.byref(vol), _f32(x), _f32(y), _stream(stream)))


def msf_weights(counts, y, lam, I0: float, c: float, stream=None):
    _check(lib().msf_weights(_f32(counts), _f32(y), _f32(lam), counts.numel(), I0, c, _stream(stream)))


class DataProx:
    def __init__(self, proj: Projector):
        h = ctypes.c_void_p()
        _check(lib().msf_dataprox_create(proj.handle, ctypes.byref(h)))
        self.handle = h
        self.proj = proj

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_dataprox_destroy(self.handle)
            self.handle = None

    __del__ = close


def msf_prox_data(dp: DataProx, y, lam, v, x, sigma: float, n_cg: int, stream=None):
    _check(lib().msf_prox_data(dp.handle, _f32(y), _f32(lam), _f32(v), _f32(x), sigma, n_cg, _stream(stream)))


def msf_prox_data_icd(dp: DataProx, y, lam, v, x, sigma: float, n_sweeps: int, stream=None):
    _check(lib().msf_prox_data_icd(dp.handle, _f32(y), _f32(lam), _f32(v), _f32(x), sigma, n_sweeps,
                                   _stream(stream)))


def msf_prox_qggmrf(vol: msf_vol, mrf: msf_mrf, v, x, sigma: float, n_sweeps: int, stream=None):
    _check(lib().msf_prox_qggmrf(ctypes.byref(vol), ctypes.byref(mrf), _f32(v), _f32(x), sigma, n_sweeps,
                                 _stream(stream)))


# ------------------------------------------------------------------ direct MAP


class MapSolver:
    """Owns an msf_map workspace for a projector's problem size."""

    def __init__(self, proj: Projector):
        h = ctypes.c_void_p()
        _check(lib().msf_map_create(proj.handle, ctypes.byref(h)))
        self.handle = h
        self.proj = proj

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_map_destroy(self.handle)
            self.handle = None

    __del__ = close


def msf_map_solve(ms: MapSolver, mrf: msf_mrf, beta: float, y, lam, x, n_outer: int, n_cg: int, stream=None):
    _check(lib().msf_map_solve(ms.handle, ctypes.byref(mrf), beta, _f32(y), _f32(lam), _f32(x), n_outer, n_cg,
                               _stream(stream)))


def msf_map_cost(ms: MapSolver, mrf: msf_mrf, beta: float, y, lam, x, stream=None) -> float:
    c = ctypes.c_double(0.0)
    _check(lib().msf_map_cost(ms.handle, ctypes.byref(mrf), beta, _f32(y), _f32(lam), _f32(x), ctypes.byref(c),
                              _stream(stream)))
    return c.value


# ------------------------------------------------------------------ fixture correction


class FixtureCorrector:
    """Owns an msf_fixcorr workspace for a projector's problem size."""

    def __init__(self, proj: Projector):
        h = ctypes.c_void_p()
        _check(lib().msf_fixcorr_create(proj.handle, ctypes.byref(h)))
        self.handle = h
        self.proj = proj

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_fixcorr_destroy(self.handle)
            self.handle = None

    __del__ = close


def msf_fixture_correct(fc: FixtureCorrector, y, x, r_mask: float, blur_sigma: float, ycorr, stream=None) -> float:
    c = ctypes.c_double(0.0)
    _check(lib().msf_fixture_correct(fc.handle, _f32(y), _f32(x), r_mask, blur_sigma, _f32(ycorr), ctypes.byref(c),
                                     _stream(stream)))
    return c.value


# ------------------------------------------------------------------ CNN


class Cnn:
    def __init__(self, max_pixels: int):
        h = ctypes.c_void_p()
        _check(lib().msf_cnn_create(int(max_pixels), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_cnn_destroy(self.handle)
            self.handle = None

    __del__ = close

    @staticmethod
    def param_count() -> int:
        return lib().msf_cnn_param_count()

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().msf_cnn_set_params(self.handle, a.ctypes.data, a.size))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.param_count(), dtype=np.float32)
        _check(lib().msf_cnn_get_params(self.handle, a.ctypes.data, a.size))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.zeros(self.param_count(), dtype=np.float32)
        _check(lib().msf_cnn_get_grads(self.handle, a.ctypes.data, a.size))
        return a

    def train_reserve(self, pixels: int):
        _check(lib().msf_cnn_train_reserve(self.handle, int(pixels)))

    def train_trace(self, on: bool):
        _check(lib().msf_cnn_train_trace(self.handle, 1 if on else 0))

    TT_ACT, TT_Z, TT_DZ, TT_DA, TT_R, TT_DR, TT_BN = range(7)

    def train_tensor(self, kind: int, layer: int, P: int) -> np.ndarray:
        """One tensor of the last training step as float64: [P][64] for
        activations and gradients (BF16 or FP32 on the device), [P] for R and
        dR, [2][64] (mean, 1/std) for the BatchNorm statistics."""
        if kind in (self.TT_ACT, self.TT_DZ, self.TT_DA):
            a = np.zeros((P, 64), dtype=np.uint16)
        elif kind == self.TT_Z:
            a = np.zeros((P, 64), dtype=np.float32)
        elif kind in (self.TT_R, self.TT_DR):
            a = np.zeros(P, dtype=np.float32)
        else:
            a = np.zeros((2, 64), dtype=np.float32)
        _check(lib().msf_cnn_train_tensor(self.handle, kind, layer, a.ctypes.data, a.nbytes))
        if a.dtype == np.uint16:
            return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return a.astype(np.float64)


def msf_training_batch(vol_stack, vol: msf_vol, B: int, H: int, W: int, sigma_lo: float, sigma_hi: float,
                       seed: int, noisy, clean, stream=None):
    _check(lib().msf_training_batch(_f32(vol_stack), ctypes.byref(vol), B, H, W, sigma_lo, sigma_hi,
                                    ctypes.c_uint64(seed & (2 ** 64 - 1)), _f32(noisy), _f32(clean),
                                    _stream(stream)))


def msf_denoise(cnn: Cnn, orient: int, vol: msf_vol, x, out, stream=None):
    _check(lib().msf_denoise(cnn.handle, orient, ctypes.byref(vol), _f32(x), _f32(out), _stream(stream)))


def msf_denoise_batch(cnns, orient: int, vols, xs, outs, stream=None):
    """H_{orient,t} of several problems (one handle per problem, same parameters)."""
    n = len(cnns)
    hc = (ctypes.c_void_p * n)(*[c.handle.value for c in cnns])
    hv = (msf_vol * n)(*vols)
    hi = (ctypes.c_void_p * n)(*[_f32(x) for x in xs])
    ho = (ctypes.c_void_p * n)(*[_f32(o) for o in outs])
    _check(lib().msf_denoise_batch(hc, n, orient, hv, hi, ho, _stream(stream)))


MSF_TILE_AUTO, MSF_TILE_16x8, MSF_TILE_PAIR = 0, 1, 2


def msf_cnn_set_tuning(cnn: Cnn, orient: int, vol: msf_vol, tile: int, chunk: int = 0):
    _check(lib().msf_cnn_set_tuning(cnn.handle, orient, ctypes.byref(vol), tile, chunk))


def msf_cnn_autotune(cnn: Cnn, vol: msf_vol, x, out, stream=None):
    """Times the conv launch choices on x; returns {orient: (tile, chunk)}."""
    ch = (ctypes.c_int * 6)()
    _check(lib().msf_cnn_autotune(cnn.handle, ctypes.byref(vol), _f32(x), _f32(out), _stream(stream), ch))
    return {o: (ch[2 * o], ch[2 * o + 1]) for o in range(3)}


def msf_train_step(cnn: Cnn, noisy, clean, lr: float, stream=None, want_loss: bool = True):
    B, _, H, W = noisy.shape
    loss = ctypes.c_float(0.0)
    _check(lib().msf_train_step(cnn.handle, _f32(noisy), _f32(clean), B, H, W, lr,
                                ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def pack_params(convs, bns, stats=None) -> np.ndarray:
    """Flat parameter layout of msf_cnn_set_params from per-layer arrays:
    W_l, b_l for l = 1..10, then gamma, beta, running mean, running var for 2..9."""
    parts = []
    for w, b in convs:
        parts += [np.asarray(w).ravel(), np.asarray(b).ravel()]
    for l, (g, be) in enumerate(bns):
        mean, var = (stats[l] if stats is not None else (np.zeros_like(g), np.ones_like(g)))
        parts += [np.asarray(g).ravel(), np.asarray(be).ravel(), np.asarray(mean).ravel(), np.asarray(var).ravel()]
    return np.concatenate(parts).astype(np.float32)


def unpack_params(flat: np.ndarray, channels=64, in_frames=5, layers=10):
    convs, bns, stats = [], [], []
    o = 0
    for l in range(layers):
        cin = in_frames if l == 0 else channels
        cout = 1 if l == layers - 1 else channels
        n = cout * cin * 9
        w = flat[o:o + n].reshape(cout, cin, 3, 3); o += n
        b = flat[o:o + cout]; o += cout
        convs.append((w.astype(np.float64), b.astype(np.float64)))
    for l in range(layers - 2):
        g = flat[o:o + channels]; o += channels
        be = flat[o:o + channels]; o += channels
        mean = flat[o:o + channels]; o += channels
        var = flat[o:o + channels]; o += channels
        bns.append((g.astype(np.float64), be.astype(np.float64)))
        stats.append((mean.astype(np.float64), var.astype(np.float64)))
    assert o == flat.size
    return convs, bns, stats


# ------------------------------------------------------------------ MACE


class Mace:
    """Owns an msf_mace handle over caller tensors W, X [K+1, nt, nz, ny, nx]."""

    def __init__(self, proj: Projector, W, X, y, lam, prior: int, mrf: msf_mrf | None = None,
                 cnn: Cnn | None = None, orient: int = 0):
        """K = W.shape[0] - 1 prior agents; with the CNN prior and K = 1 the
        single agent is the CNN of orientation `orient` (0 xy-t, 1 yz-t, 2 zx-t)."""
        K = W.shape[0] - 1
        self.desc = msf_mace_desc(proj.handle, prior, K, cnn.handle if cnn else None,
                                  mrf if mrf is not None else msf_mrf(2.0, 1.2, 1.0, 1.0, 0.5),
                                  _f32(W), _f32(X), _f32(y), _f32(lam), orient)
        self._keep = (proj, W, X, y, lam, cnn)
        h = ctypes.c_void_p()
        _check(lib().msf_mace_create(ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_mace_destroy(self.handle)
            self.handle = None

    __del__ = close


def mace_params(rho: float, sigma: float, mu, n_cg: int, n_sweeps: int = 0, use_graph: bool = False,
                n_icd: int = 0):
    return msf_mace_params(rho, sigma, (ctypes.c_double * 4)(*(list(mu) + [0.0] * (4 - len(mu)))), n_cg, n_sweeps,
                           1 if use_graph else 0, n_icd)


def msf_mace_step(m: Mace, rho: float, sigma: float, mu, n_cg: int, n_sweeps: int = 0, stream=None,
                  want_residual: bool = True, use_graph: bool = False, n_icd: int = 0):
    prm = mace_params(rho, sigma, mu, n_cg, n_sweeps, use_graph, n_icd)
    r = ctypes.c_double(0.0)
    _check(lib().msf_mace_step(m.handle, ctypes.byref(prm), ctypes.byref(r) if want_residual else None,
                               _stream(stream)))
    return r.value if want_residual else None


def msf_mace_set_counts(m: Mace, counts_host, I0: float, c: float, stream=None):
    """New photon counts for the problem from a host tensor (float32, contiguous;
    pinned memory keeps the copy asynchronous)."""
    import torch
    if counts_host.is_cuda or counts_host.dtype != torch.float32 or not counts_host.is_contiguous():
        raise ValueError("expected a contiguous float32 host tensor")
    _check(lib().msf_mace_set_counts(m.handle, counts_host.data_ptr(), I0, c, _stream(stream)))


def msf_mace_consensus(W, X, mu, rho: float, work, stream=None):
    """Consensus and Mann update of stacked states W, X [K1, ...] in place; the
    two FP64 sums of the consensus spread stay in work[MSF_CONSENSUS_SUMS:+2]
    (work: CUDA float64 tensor of MSF_CONSENSUS_WORK elements)."""
    import torch
    K1 = W.shape[0]
    if X.shape != W.shape:
        raise ValueError("W and X must have the same shape")
    if work.dtype != torch.float64 or work.numel() < MSF_CONSENSUS_WORK:
        raise ValueError(f"work must be a float64 tensor of at least {MSF_CONSENSUS_WORK} elements")
    m = (ctypes.c_double * 4)(*(list(mu) + [0.0] * (4 - len(mu))))
    _check(lib().msf_mace_consensus(_f32(W), _f32(X), K1, W[0].numel(), m, rho, _ptr(work), _stream(stream)))


class MaceBatch:
    """A queue of independent MACE problems advanced together (msf_mace_batch_*)."""

    def __init__(self, maces):
        arr = (ctypes.c_void_p * len(maces))(*[m.handle.value for m in maces])
        h = ctypes.c_void_p()
        _check(lib().msf_mace_batch_create(arr, len(maces), ctypes.byref(h)))
        self.handle = h
        self._keep = list(maces)

    def close(self):
        if getattr(self, "handle", None):
            lib().msf_mace_batch_destroy(self.handle)
            self.handle = None

    __del__ = close


def msf_mace_batch_step(b: MaceBatch, params, stream=None, want_residuals: bool = True):
    n = len(b._keep)
    arr = (msf_mace_params * n)(*params)
    res = (ctypes.c_double * n)()
    _check(lib().msf_mace_batch_step(b.handle, arr, res if want_residuals else None, _stream(stream)))
    return list(res) if want_residuals else None


def msf_projector_autotune(proj: Projector, stream=None):
    choice = (ctypes.c_int * 3)()
    _check(lib().msf_projector_autotune(proj.handle, _stream(stream), choice))
    return tuple(choice)


def msf_projector_set_tuning(proj: Projector, fwd_cols: int, fwd_rows: int, adj_zrun: int):
    _check(lib().msf_projector_set_tuning(proj.handle, fwd_cols, fwd_rows, adj_zrun))


# ------------------------------------------------------------------ phantoms


def msf_phantom_voxelize(vol: msf_vol, ell: np.ndarray, x, ss: int = 4, stream=None):
    e = np.ascontiguousarray(ell, dtype=np.float64)
    n_ell = e.shape[-2]
    _check(lib().msf_phantom_voxelize(ctypes.byref(vol), e.ctypes.data, n_ell, ss, _f32(x), _stream(stream)))


def msf_phantom_project(proj: Projector, ell: np.ndarray, y, stream=None):
    e = np.ascontiguousarray(ell, dtype=np.float64)
    _check(lib().msf_phantom_project(proj.handle, e.ctypes.data, e.shape[-2], _f32(y), _stream(stream)))


def msf_selftest_wait(limit_ns: int, stream=None) -> int:
    """Runs the bounded-wait self-test; returns the library status (4 = timeout, the expected outcome)."""
    return lib().msf_selftest_wait(ctypes.c_uint64(int(limit_ns)), _stream(stream))
