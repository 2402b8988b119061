"""Python binding of libbisp (include/bisp.h): argument marshalling only.

Every step of the estimator runs in the library's CUDA kernels.  Device inputs are
torch CUDA tensors (PyTorch supplies device memory and streams); host inputs are numpy
arrays.  If the compiled library is missing, importing this package builds it with nvcc;
if that fails, the import raises - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbisp.so")
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "bisp.h")

BISP_OK, BISP_EINVAL, BISP_ENOMEM, BISP_ECUDA, BISP_ESTATE, BISP_ETIMEOUT, BISP_EUNSUPPORTED = range(7)
STATUS_NAMES = ["BISP_OK", "BISP_EINVAL", "BISP_ENOMEM", "BISP_ECUDA", "BISP_ESTATE", "BISP_ETIMEOUT",
                "BISP_EUNSUPPORTED"]
LOS = {"global": 0, "local": 1}
MAS = {"NGP": 1, "CIC": 2, "TSC": 3, 1: 1, 2: 2, 3: 3}
DATA, RANDOMS = 0, 1
PRECISION = {"fp32": 0, "fp64": 1, 0: 0, 1: 1}
ESTIMATOR = {"bispectrum": 0, "threept": 1, 0: 0, 1: 1}


class BispError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("nmesh", C.c_int), ("box_len", C.c_double), ("k_edges", C.POINTER(C.c_double)),
                ("nbins", C.c_int), ("ells", C.POINTER(C.c_int)), ("n_mult", C.c_int), ("los", C.c_int),
                ("observer", C.c_double * 3), ("mas", C.c_int), ("interlace", C.c_int), ("fkp_P0", C.c_double),
                ("max_device_bytes", C.c_size_t), ("want_window", C.c_int), ("precision", C.c_int),
                ("estimator", C.c_int), ("diagonal_only", C.c_int), ("los_object", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("nmesh", C.c_int), ("nbins", C.c_int), ("n_mult", C.c_int), ("n_dchan", C.c_int),
                ("n_nchan", C.c_int), ("n_fcomp", C.c_int), ("alpha", C.c_double), ("norm_I", C.c_double),
                ("n_data", C.c_int64), ("n_randoms", C.c_int64), ("device_bytes", C.c_size_t),
                ("kernel_launches", C.c_int), ("ms_assign_data", C.c_double), ("ms_assign_randoms", C.c_double),
                ("ms_measure", C.c_double), ("ms_pair", C.c_double), ("pair_bytes", C.c_double),
                ("pair_launches", C.c_int), ("pair_kernel", C.c_int), ("zpass_groups", C.c_int)]


def _load(path=None, checked=False):
    path = path or _LIB_PATH
    if not os.path.exists(path):
        from . import build as _b
        path = _b.build(checked=checked)
    lib = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    lib.bisp_plan_create.argtypes = [C.POINTER(vp), C.POINTER(_Params), vp]
    lib.bisp_assign.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int64, C.c_int]
    lib.bisp_measure.argtypes = [vp, dp, dp, dp, dp, dp]
    lib.bisp_measure_batch.argtypes = [vp, vp, C.c_int]
    lib.bisp_plan_destroy.argtypes = [vp]
    lib.bisp_last_error.restype = C.c_char_p
    lib.bisp_plan_query.argtypes = [vp, C.POINTER(_Info)]
    lib.bisp_cell_order.argtypes = [C.c_int, C.c_double, C.c_int, vp, C.c_int64, vp, vp, vp]
    lib.bisp_debug_fetch.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, C.c_size_t]
    lib.bisp_check_word.argtypes = [C.POINTER(C.c_uint64), C.c_int]
    lib.bisp_cell_order_noalloc.argtypes = [C.c_int, C.c_double, C.c_int, vp, C.c_int64, vp, vp, vp]
    lib.bisp_covariance.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp]
    lib.bisp_covariance_factors.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
    lib.bisp_chi2.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp]
    ip = C.POINTER(C.c_int)
    lib.bisp_wigner9j.argtypes = [ip, dp]
    lib.bisp_masked_zeta.argtypes = [ip, C.c_int, dp, ip, C.c_int, dp, ip, C.c_int, dp, dp, C.c_int, C.c_int, dp, dp]
    lib.bisp_zeta_to_bk.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, dp, dp, C.c_int, dp, C.c_int, dp]
    lib.bisp_bk_to_zeta.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, dp, dp, C.c_int, dp, C.c_int, dp]
    lib.bisp_tree_multipoles.argtypes = [dp, dp, C.c_int, C.c_double, C.c_double, C.c_double, ip, C.c_int, dp,
                                         C.c_int, dp, C.c_int, C.c_int, dp]
    for f in ("bisp_plan_create", "bisp_assign", "bisp_measure", "bisp_measure_batch", "bisp_plan_destroy",
              "bisp_plan_query", "bisp_cell_order", "bisp_debug_fetch", "bisp_cell_order_noalloc",
              "bisp_covariance", "bisp_covariance_factors", "bisp_chi2", "bisp_wigner9j", "bisp_masked_zeta",
              "bisp_zeta_to_bk", "bisp_bk_to_zeta", "bisp_tree_multipoles", "bisp_check_word"):
        getattr(lib, f).restype = C.c_int
    return lib


_lib = None


def lib():
    """The loaded libbisp (built on first use)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def use_checked_library():
    """Switch this process to libbisp_checked.so (built on first use: the same kernels with device
    bounds checks, see bisp_check_word in include/bisp.h); returns the previous library handle,
    which use_library() restores."""
    global _lib
    prev = _lib
    _lib = _load(os.path.join(_HERE, "libbisp_checked.so"), checked=True)
    return prev


def use_library(handle):
    """Make a library handle returned by use_checked_library() the current one again."""
    global _lib
    _lib = handle


def check_word(reset=False):
    """The checked library's device check word (0: every check passed); BispError from the release
    library (BISP_EUNSUPPORTED)."""
    w = C.c_uint64(0)
    _check(lib().bisp_check_word(C.byref(w), 1 if reset else 0))
    return int(w.value)


def header_functions():
    """Names of the functions declared in include/bisp.h."""
    txt = open(_HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:bisp_status|const char\*)\s+(bisp_\w+)\s*\(", txt, re.M)))


def _check(st):
    if st != BISP_OK:
        raise BispError(st, lib().bisp_last_error().decode())


def _ptr(a):
    """(pointer, is_device) of a torch CUDA tensor or a numpy array (kept alive by caller)."""
    if a is None:
        return None, None
    if hasattr(a, "is_cuda") and a.is_cuda:
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr()), 1
    arr = np.ascontiguousarray(a)
    return C.c_void_p(arr.ctypes.data), 0


def _stream_handle(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Plan:
    """A measurement plan: mesh, bins, multipoles, line of sight, assignment scheme."""

    def __init__(self, nmesh, box_len, k_edges, ells, los="global", observer=(0.0, 0.0, 0.0), mas="TSC",
                 interlace=False, fkp_P0=0.0, want_window=False, max_device_bytes=0, stream=None,
                 precision="fp32", estimator="bispectrum", diagonal_only=False, los_object=3):
        """k_edges: k-bin edges [h/Mpc] for the bispectrum, r-bin edges [Mpc/h] for the
        three-point function (estimator="threept"; measure() then returns zeta as "B" and the
        window multipoles Q as "window").  los_object: 3 (default), 1 or 2, the object whose line
        of sight carries the y_L^{M*} weight (App. B)."""
        self._edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        self._ells = np.ascontiguousarray(np.asarray(ells, dtype=np.int32).reshape(-1))
        p = _Params()
        p.nmesh = int(nmesh)
        p.box_len = float(box_len)
        p.k_edges = self._edges.ctypes.data_as(C.POINTER(C.c_double))
        p.nbins = len(self._edges) - 1
        p.ells = self._ells.ctypes.data_as(C.POINTER(C.c_int))
        p.n_mult = len(self._ells) // 3
        p.los = LOS[los] if isinstance(los, str) else int(los)
        p.observer = (C.c_double * 3)(*[float(v) for v in observer])
        p.mas = MAS[mas]
        p.interlace = 1 if interlace else 0
        p.fkp_P0 = float(fkp_P0)
        p.max_device_bytes = int(max_device_bytes)
        p.want_window = 1 if want_window else 0
        # names map to the enums; integers go to the library as given (it validates them)
        p.precision = PRECISION[precision] if precision in PRECISION else int(precision)
        p.estimator = ESTIMATOR[estimator] if estimator in ESTIMATOR else int(estimator)
        p.diagonal_only = 1 if diagonal_only else 0
        p.los_object = int(los_object)
        self.nbins = p.nbins
        self.want_window = bool(want_window)
        self.n_mult = p.n_mult
        self.nmesh = p.nmesh
        self._h = C.c_void_p()
        _check(lib().bisp_plan_create(C.byref(self._h), C.byref(p), _stream_handle(stream)))

    def assign(self, which, xyz, w=None, nbar=None):
        """Assign a catalogue: xyz (n, 3) float32, optional w and nbar (n,) float32, either
        all torch CUDA tensors or all host arrays."""
        keep = []
        for a in (xyz, w, nbar):
            if a is not None and not (hasattr(a, "is_cuda") and a.is_cuda):
                a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
        px, dev = _ptr(keep[0])
        pw, _ = _ptr(keep[1])
        pn, _ = _ptr(keep[2])
        n = int(keep[0].shape[0]) if keep[0] is not None else 0
        _check(lib().bisp_assign(self._h, int(which), px, pw, pn, n, int(dev or 0)))

    def measure(self):
        """Dict of FP64 arrays [n_mult, nbins, nbins]: B, shot, window, window_shot; nmodes [nbins]."""
        shape = (self.n_mult, self.nbins, self.nbins)
        out = {k: np.zeros(shape) for k in ("B", "shot", "window", "window_shot")}
        out["nmodes"] = np.zeros(self.nbins)
        dp = C.POINTER(C.c_double)
        info = self.info()
        args = [out[k].ctypes.data_as(dp) for k in ("B", "shot")]
        if info["n_randoms"] > 0 and self.want_window:
            args += [out[k].ctypes.data_as(dp) for k in ("window", "window_shot")]
        else:
            args += [None, None]
            del out["window"], out["window_shot"]
        args.append(out["nmodes"].ctypes.data_as(dp))
        _check(lib().bisp_measure(self._h, *args))
        return out

    def _out_arrays(self):
        shape = (self.n_mult, self.nbins, self.nbins)
        out = {k: np.zeros(shape) for k in ("B", "shot")}
        if self.info()["n_randoms"] > 0 and self.want_window:
            out.update(window=np.zeros(shape), window_shot=np.zeros(shape))
        out["nmodes"] = np.zeros(self.nbins)
        return out

    def info(self):
        i = _Info()
        _check(lib().bisp_plan_query(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def fetch_spectrum(self, which, chan):
        """Deconvolved half spectrum of a channel: complex64 [N, N, N/2]."""
        N = self.nmesh
        a = np.empty((N, N, N // 2), dtype=np.complex64)
        _check(lib().bisp_debug_fetch(self._h, 0, int(which), int(chan), C.c_void_p(a.ctypes.data), a.nbytes))
        return a

    def fetch_mesh(self, which, chan):
        """Assigned real mesh of a channel (needs BISP_DEBUG=BISP_DEBUG_KEEP_MESH at plan creation)."""
        N = self.nmesh
        a = np.empty((N, N, N), dtype=np.float32)
        _check(lib().bisp_debug_fetch(self._h, 1, int(which), int(chan), C.c_void_p(a.ctypes.data), a.nbytes))
        return a

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().bisp_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cell_order(nmesh, box_len, mas, xyz, stream=None):
    """(keys, order) of a torch CUDA float32 (n, 3) tensor: stable order by home mesh node."""
    import torch
    assert xyz.is_cuda and xyz.dtype == torch.float32 and xyz.is_contiguous()
    n = xyz.shape[0]
    keys = torch.empty(n, dtype=torch.int32, device=xyz.device)
    order = torch.empty(n, dtype=torch.int32, device=xyz.device)
    s = _stream_handle(stream if stream is not None else torch.cuda.current_stream())
    _check(lib().bisp_cell_order(int(nmesh), float(box_len), MAS[mas], C.c_void_p(xyz.data_ptr()), n,
                                 C.c_void_p(keys.data_ptr()), C.c_void_p(order.data_ptr()), s))
    return keys, order


class _Outputs(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in ("B", "shot", "window", "window_shot", "nmodes")]


def measure_batch(plans):
    """bisp_measure_batch over a list of Plans: one output dict per plan (as Plan.measure)."""
    outs = [p._out_arrays() for p in plans]
    arr = (_Outputs * max(len(plans), 1))()
    dp = C.POINTER(C.c_double)
    for i, o in enumerate(outs):
        for k in ("B", "shot", "window", "window_shot", "nmodes"):
            setattr(arr[i], k, o[k].ctypes.data_as(dp) if k in o else None)
    handles = (C.c_void_p * max(len(plans), 1))(*[p._h.value for p in plans])
    _check(lib().bisp_measure_batch(handles, arr, len(plans)))
    return outs


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def covariance(X, n_par=None):
    """Covariance statistics of a batch of data vectors X [n_mock, n_bin] (Eq. Covariance,
    App. E): dict with mean, cov, corr, hartlap and, when n_par is given, percival_m."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    nm, nb = X.shape
    mean, cov, corr = np.zeros(nb), np.zeros((nb, nb)), np.zeros((nb, nb))
    _check(lib().bisp_covariance(_dp(X), nm, nb, _dp(mean), _dp(cov), _dp(corr)))
    h, m = C.c_double(), C.c_double()
    _check(lib().bisp_covariance_factors(nm, nb, int(n_par or 0), C.byref(h),
                                         C.byref(m) if n_par is not None else None))
    out = {"mean": mean, "cov": cov, "corr": corr, "hartlap": h.value}
    if n_par is not None:
        out["percival_m"] = m.value
    return out


def chi2(cov, n_mock, x_obs, x_theory):
    """(x_obs - x_theory)^T C_Hartlap^{-1} (x_obs - x_theory) (App. E)."""
    cov = np.ascontiguousarray(cov, dtype=np.float64)
    xo = np.ascontiguousarray(x_obs, dtype=np.float64)
    xt = np.ascontiguousarray(x_theory, dtype=np.float64)
    out = C.c_double()
    _check(lib().bisp_chi2(_dp(cov), cov.shape[0], int(n_mock), _dp(xo), _dp(xt), C.byref(out)))
    return out.value


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def wigner9j(j):
    """Wigner 9j symbol of nine integers (row-major)."""
    a = np.ascontiguousarray(j, dtype=np.int32).reshape(9)
    out = C.c_double()
    _check(lib().bisp_wigner9j(_ip(a), C.byref(out)))
    return out.value


def masked_zeta(theory, window, ells_out, r, w, ic=True):
    """Masked three-point multipoles (Eq. zetaMask) and the integral constraint (Eq. IC).
    theory, window: dicts (l1, l2, L) -> [nr, nr] arrays on the radii r with quadrature weights w.
    Returns ({l: [nr, nr]}, zeta_bar)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    nr = len(r)
    lt = list(theory)
    lq = list(window)
    et = np.ascontiguousarray(np.array(lt, dtype=np.int32).reshape(-1))
    eq = np.ascontiguousarray(np.array(lq, dtype=np.int32).reshape(-1))
    eo = np.ascontiguousarray(np.array(list(ells_out), dtype=np.int32).reshape(-1))
    zt = np.ascontiguousarray(np.stack([theory[e] for e in lt]), dtype=np.float64)
    qq = np.ascontiguousarray(np.stack([window[e] for e in lq]), dtype=np.float64)
    out = np.zeros((len(eo) // 3, nr, nr))
    zb = C.c_double()
    _check(lib().bisp_masked_zeta(_ip(et), len(lt), _dp(zt), _ip(eq), len(lq), _dp(qq), _ip(eo), len(eo) // 3,
                                  _dp(r), _dp(w), nr, 1 if ic else 0, _dp(out), C.byref(zb)))
    return {tuple(e): out[i] for i, e in enumerate(np.array(list(ells_out)).reshape(-1, 3).tolist())}, zb.value


def zeta_to_bk(l1, l2, r, w, zeta, k1, k2):
    """Hankel transform of zeta [nr, nr] to B [nk1, nk2] (Eq. masked_bispectrum)."""
    r, w, z, k1, k2 = (np.ascontiguousarray(a, dtype=np.float64) for a in (r, w, zeta, k1, k2))
    B = np.zeros((len(k1), len(k2)))
    _check(lib().bisp_zeta_to_bk(int(l1), int(l2), _dp(r), _dp(w), len(r), _dp(z), _dp(k1), len(k1), _dp(k2),
                                 len(k2), _dp(B)))
    return B


def bk_to_zeta(l1, l2, k, wk, B, r1, r2):
    """Hankel transform of B [nk, nk] to zeta [nr1, nr2] (Eq. HankelTransform)."""
    k, wk, B, r1, r2 = (np.ascontiguousarray(a, dtype=np.float64) for a in (k, wk, B, r1, r2))
    z = np.zeros((len(r1), len(r2)))
    _check(lib().bisp_bk_to_zeta(int(l1), int(l2), _dp(k), _dp(wk), len(k), _dp(B), _dp(r1), len(r1), _dp(r2),
                                 len(r2), _dp(z)))
    return z


def tree_multipoles(k_tab, p_tab, b1, b2, f, ells, k1, k2, n_mu=24):
    """Tree-level bispectrum multipoles (App. F) [n_mult, nk1, nk2] for a tabulated P(k)."""
    kt, pt, k1, k2 = (np.ascontiguousarray(a, dtype=np.float64) for a in (k_tab, p_tab, k1, k2))
    e = np.ascontiguousarray(np.array(list(ells), dtype=np.int32).reshape(-1))
    out = np.zeros((len(e) // 3, len(k1), len(k2)))
    _check(lib().bisp_tree_multipoles(_dp(kt), _dp(pt), len(kt), float(b1), float(b2), float(f), _ip(e), len(e) // 3,
                                      _dp(k1), len(k1), _dp(k2), len(k2), int(n_mu), _dp(out)))
    return out
