"""Python binding of the C ABI in include/fpca.h (argument marshalling only).

Every computation runs in libfpca.so's CUDA kernels; this module only turns
torch tensors (device memory, owned by the caller) into pointers and sizes.
It never falls back to a CPU path: if the library is missing or no sm_103
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpca.so")

# fpca_status
OK, E_INVALID_ARG, E_UNSUPPORTED, E_CUDA, E_OOM, E_TIMEOUT, E_NUMERIC = range(7)
# fpca_prec
F64, F32, BF16, F32C = 0, 1, 2, 4
# per-point status
PT_OK, PT_FALLBACK, PT_EMPTY = 0, 1, 2
DENSE, SPARSE = 0, 1
COV_RESIDUAL, COV_RAW = 0, 1

# the symbols include/fpca.h declares
SYMBOLS = (
    "fpca_create", "fpca_destroy", "fpca_set_stream", "fpca_last_error", "fpca_sync",
    "fpca_launch_count", "fpca_bin_mean", "fpca_smooth_mean", "fpca_bin_cov",
    "fpca_smooth_cov_project", "fpca_rproj_eig", "fpca_profile_enable", "fpca_profile_count",
    "fpca_profile_entry", "fpca_bin_mean_static", "fpca_bw_param_count", "fpca_bw_predict",
    "fpca_bw_train_step", "fpca_bw_features", "fpca_cov_factor_bytes", "fpca_bin_cov_factor",
    "fpca_smooth_cov_apply", "fpca_smooth_cov_tiles", "fpca_rproj_eig_factor", "fpca_sigma2",
    "fpca_smooth_cov_diag", "fpca_scores_pace", "fpca_scores_integral", "fpca_reconstruct",
    "fpca_mise", "fpca_bw_trust_region", "fpca_check_wait", "fpca_set_sweep_kernel",
    "fpca_set_cv_batch", "fpca_graph_begin", "fpca_graph_end", "fpca_graph_launch",
    "fpca_graph_launches", "fpca_graph_destroy",
    "fpca_bw_mlp_init", "fpca_bw_mlp_io", "fpca_smooth_mean_cv", "fpca_alu_probe",
)


class Graph:
    """An instantiated CUDA graph of library calls (fpca_graph_*)."""

    def __init__(self, lib, h):
        self.lib, self.h = lib, h

    @property
    def launches(self):
        return int(self.lib.fpca_graph_launches(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.fpca_graph_destroy(self.h)
            self.h = None


class FpcaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fpca status {status}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("m", ctypes.c_int * 3)]

    @classmethod
    def of(cls, m):
        g = cls()
        g.d = len(m)
        for k in range(3):
            g.m[k] = int(m[k]) if k < len(m) else 1
        return g


class Data(ctypes.Structure):
    _fields_ = [
        ("layout", ctypes.c_int),
        ("n", ctypes.c_int),
        ("y", ctypes.c_void_p),
        ("y_prec", ctypes.c_int),
        ("mask", ctypes.c_void_p),
        ("offs", ctypes.c_void_p),
        ("t", ctypes.c_void_p),
    ]


class TrOptions(ctypes.Structure):
    _fields_ = [
        ("delta0", ctypes.c_double),
        ("delta_min", ctypes.c_double),
        ("delta_max", ctypes.c_double),
        ("h_lo", ctypes.c_double),
        ("h_hi", ctypes.c_double),
        ("max_iter", ctypes.c_int),
    ]


class CovBins(ctypes.Structure):
    _fields_ = [
        ("nfold", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("cnt", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("q", ctypes.c_void_p),
        ("asym", ctypes.c_int),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load libfpca.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, dbl_p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.fpca_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    lib.fpca_destroy.argtypes = [vp]
    lib.fpca_destroy.restype = None
    lib.fpca_set_stream.argtypes = [vp, vp]
    lib.fpca_last_error.argtypes = [vp]
    lib.fpca_last_error.restype = ctypes.c_char_p
    lib.fpca_sync.argtypes = [vp]
    lib.fpca_launch_count.argtypes = [vp]
    lib.fpca_launch_count.restype = ctypes.c_uint64
    lib.fpca_check_wait.argtypes = [vp, i32]
    lib.fpca_set_sweep_kernel.argtypes = [vp, i32]
    lib.fpca_set_cv_batch.argtypes = [vp, i32]
    lib.fpca_graph_begin.argtypes = [vp]
    lib.fpca_graph_end.argtypes = [vp, ctypes.POINTER(vp)]
    lib.fpca_graph_launch.argtypes = [vp, vp]
    lib.fpca_graph_launches.argtypes = [vp]
    lib.fpca_graph_launches.restype = ctypes.c_uint64
    lib.fpca_graph_destroy.argtypes = [vp]
    lib.fpca_graph_destroy.restype = None
    lib.fpca_alu_probe.argtypes = [vp, i32, i32, i32, dbl_p]
    lib.fpca_bw_mlp_init.argtypes = [vp, ctypes.c_uint64, vp]
    lib.fpca_smooth_mean_cv.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, i32,
                                        dbl_p, i32, vp]
    lib.fpca_bw_mlp_io.argtypes = [vp, vp, vp, vp, ctypes.c_char_p, i32]
    lib.fpca_bin_mean.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, vp, vp, vp]
    lib.fpca_smooth_mean.argtypes = [vp, ctypes.POINTER(Grid), vp, vp, vp, dbl_p, vp, vp]
    lib.fpca_bin_cov.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, i32, i32, vp,
                                 i32, vp, vp, vp, vp]
    lib.fpca_smooth_cov_project.argtypes = [vp, ctypes.POINTER(Grid), ctypes.POINTER(CovBins),
                                            dbl_p, i32, i32, vp, vp, i32, vp, vp, vp, vp]
    lib.fpca_rproj_eig.argtypes = [vp, ctypes.POINTER(Grid), vp, i32, vp, vp, i32, i32, i32, i32,
                                   vp, vp, vp]
    lib.fpca_bw_features.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, vp, vp, vp,
                                     ctypes.POINTER(CovBins), vp]
    lib.fpca_bw_param_count.argtypes = []
    lib.fpca_bw_param_count.restype = ctypes.c_int64
    lib.fpca_bw_predict.argtypes = [vp, vp, vp, i32, vp]
    lib.fpca_bw_train_step.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, i32, ctypes.c_float,
                                       ctypes.c_float, vp, vp]
    lib.fpca_bin_mean_static.argtypes = [vp, i32, i32, vp, i32, vp, vp, vp, vp, vp]
    lib.fpca_cov_factor_bytes.argtypes = [ctypes.POINTER(Grid), i32]
    lib.fpca_cov_factor_bytes.restype = ctypes.c_size_t
    lib.fpca_bin_cov_factor.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, vp,
                                        ctypes.c_size_t]
    lib.fpca_smooth_cov_apply.argtypes = [vp, ctypes.POINTER(Grid), vp, i32, dbl_p, vp, i32, vp]
    lib.fpca_smooth_cov_tiles.argtypes = [vp, ctypes.POINTER(Grid), vp, i32, dbl_p, i32,
                                          ctypes.POINTER(ctypes.c_int32), vp]
    lib.fpca_rproj_eig_factor.argtypes = [vp, ctypes.POINTER(Grid), vp, i32, dbl_p, vp, i32, i32,
                                          i32, vp, vp, vp]
    lib.fpca_smooth_cov_diag.argtypes = [vp, ctypes.POINTER(Grid), vp, i32, dbl_p, vp]
    lib.fpca_scores_pace.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, vp, vp,
                                     i32, vp, vp]
    lib.fpca_scores_integral.argtypes = [vp, ctypes.POINTER(Data), ctypes.POINTER(Grid), vp, vp,
                                         i32, vp]
    lib.fpca_reconstruct.argtypes = [vp, ctypes.POINTER(Grid), vp, vp, i32, vp, i32, vp]
    lib.fpca_mise.argtypes = [vp, ctypes.POINTER(Grid), vp, vp, i32, i32, vp]
    lib.fpca_bw_trust_region.argtypes = [vp, ctypes.POINTER(Grid), ctypes.POINTER(CovBins), i32,
                                         dbl_p, ctypes.POINTER(TrOptions), dbl_p, dbl_p,
                                         ctypes.POINTER(ctypes.c_int), dbl_p, i32]
    lib.fpca_sigma2.argtypes = [vp, ctypes.POINTER(Grid), vp, vp, vp, dbl_p, vp, vp, i32,
                                ctypes.c_longlong, vp, vp, vp, vp]
    lib.fpca_profile_enable.argtypes = [vp, i32]
    lib.fpca_profile_count.argtypes = [vp]
    lib.fpca_profile_entry.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]
    for name in SYMBOLS:
        f = getattr(lib, name)
        if name not in ("fpca_destroy", "fpca_last_error", "fpca_launch_count",
                        "fpca_bw_param_count", "fpca_cov_factor_bytes", "fpca_graph_launches",
                        "fpca_graph_destroy"):
            f.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _doubles(vals):
    vals = [float(x) for x in vals]
    return (ctypes.c_double * len(vals))(*vals)


class Context:
    """An fpca_ctx bound to one CUDA device and a stream (torch stream or None)."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        st = self.lib.fpca_create(ctypes.byref(h), int(device), s)
        if st != OK:
            raise FpcaError(st, "fpca_create failed (no usable sm_103 device?)")
        self.h = h
        self.device = torch.device("cuda", device)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fpca_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise FpcaError(st, self.lib.fpca_last_error(self.h).decode())

    def set_stream(self, stream):
        self._check(self.lib.fpca_set_stream(self.h, None if stream is None else
                                             ctypes.c_void_p(stream.cuda_stream)))

    def sync(self):
        self._check(self.lib.fpca_sync(self.h))

    # ---- CUDA graphs of call sequences ----------------------------------------
    def graph_begin(self):
        """Start recording this context's calls (a created stream, timing off)."""
        self._check(self.lib.fpca_graph_begin(self.h))

    def graph_end(self):
        """Close the recording; returns a Graph (replay with graph_launch)."""
        h = ctypes.c_void_p()
        self._check(self.lib.fpca_graph_end(self.h, ctypes.byref(h)))
        return Graph(self.lib, h)

    def graph_launch(self, graph):
        self._check(self.lib.fpca_graph_launch(self.h, graph.h))

    def set_sweep_kernel(self, kernel):
        """0 automatic (timed once per grid and windows), 1 scalar, 2 packed pairs."""
        self._check(self.lib.fpca_set_sweep_kernel(self.h, int(kernel)))

    def set_cv_batch(self, batch):
        """K-fold CV grid schedule: True (one t-side launch for the whole grid),
        False (item by item) or "auto" (the default: timed once, faster kept)."""
        mode = 2 if batch == "auto" else (1 if batch else 0)
        self._check(self.lib.fpca_set_cv_batch(self.h, mode))

    def bw_mlp_init(self, params, seed):
        """He-normal initial network parameters from a counter-based generator."""
        self._check(self.lib.fpca_bw_mlp_init(self.h, int(seed), _ptr(params)))

    def bw_mlp_io(self, params, path, save, feat_mu=None, feat_sd=None):
        """Save (save=True) or load the network and its feature standardisation."""
        self._check(self.lib.fpca_bw_mlp_io(self.h, _ptr(params), _ptr(feat_mu), _ptr(feat_sd),
                                            str(path).encode(), int(bool(save))))

    def alu_probe(self, fp64, blocks, iters):
        """Queue the FMA-throughput probe; returns the flops it performs."""
        out = ctypes.c_double(0.0)
        self._check(self.lib.fpca_alu_probe(self.h, int(bool(fp64)), int(blocks), int(iters),
                                            ctypes.byref(out)))
        return out.value

    def check_wait(self, arrive):
        """Queue the bounded-wait self-check (fpca_check_wait); its outcome is
        reported by the next sync()."""
        self._check(self.lib.fpca_check_wait(self.h, int(bool(arrive))))

    @property
    def launches(self):
        return int(self.lib.fpca_launch_count(self.h))

    def profile(self, enable=True):
        """Turn per-kernel timing on or off (clears the totals)."""
        self._check(self.lib.fpca_profile_enable(self.h, int(bool(enable))))

    def profile_read(self):
        """{kernel name: (total ms, launches)} of the timed launches so far."""
        out = {}
        for i in range(self.lib.fpca_profile_count(self.h)):
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            cnt = ctypes.c_uint64()
            self._check(self.lib.fpca_profile_entry(self.h, i, ctypes.byref(name), ctypes.byref(ms),
                                                    ctypes.byref(cnt)))
            out[name.value.decode()] = (ms.value, int(cnt.value))
        return out

    # ---- bandwidth network ---------------------------------------------------
    def bw_param_count(self):
        return int(self.lib.fpca_bw_param_count())

    def bw_features(self, data, m, cnt, w, v, v2, ccnt, cw, cv, feat, nfold=0):
        bins = CovBins()
        bins.nfold = int(nfold)
        bins.prec = F64 if cw.dtype.itemsize == 8 else F32
        bins.cnt, bins.w, bins.v = ccnt.data_ptr(), cw.data_ptr(), cv.data_ptr()
        bins.q = None
        self._check(self.lib.fpca_bw_features(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                              _ptr(cnt), _ptr(w), _ptr(v), _ptr(v2),
                                              ctypes.byref(bins), _ptr(feat)))

    # ---- noise variance ------------------------------------------------------
    def sigma2(self, m, cnt, w, v2, h, mu, gdiag, gdiag_stride, sigma2_t, status=None,
               sigma2=None, domain=None):
        """Eq. (2.5)-(2.6); gdiag a device tensor whose element p * gdiag_stride is
        Gamma_hat(t_p, t_p) (e.g. a P x P surface with stride P + 1)."""
        gp = F64 if gdiag.dtype.itemsize == 8 else F32
        self._check(self.lib.fpca_sigma2(self.h, ctypes.byref(Grid.of(m)), _ptr(cnt), _ptr(w),
                                         _ptr(v2), _doubles(h), _ptr(mu), _ptr(gdiag), gp,
                                         int(gdiag_stride), _ptr(domain), _ptr(sigma2_t),
                                         _ptr(status), _ptr(sigma2)))

    # ---- scores and reconstruction -------------------------------------------
    def scores_pace(self, data, m, mu, evals, evecs, L, sigma2, scores):
        """Eq. (2.7); evecs P x k column-major (its first L columns are used);
        sigma2 a one-element device tensor of float64."""
        self._check(self.lib.fpca_scores_pace(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                              _ptr(mu), _ptr(evals), _ptr(evecs), int(L),
                                              _ptr(sigma2), _ptr(scores)))

    def scores_integral(self, data, m, mu, evecs, L, scores):
        self._check(self.lib.fpca_scores_integral(self.h, ctypes.byref(data),
                                                  ctypes.byref(Grid.of(m)), _ptr(mu), _ptr(evecs),
                                                  int(L), _ptr(scores)))

    def mise(self, m, xhat, x, n, out):
        """out: one-element float64 device tensor; x float64 or float32, n x P."""
        xp = F64 if x.dtype.itemsize == 8 else F32
        self._check(self.lib.fpca_mise(self.h, ctypes.byref(Grid.of(m)), _ptr(xhat), _ptr(x), xp,
                                       int(n), _ptr(out)))

    def reconstruct(self, m, mu, evecs, L, scores, n, xhat):
        self._check(self.lib.fpca_reconstruct(self.h, ctypes.byref(Grid.of(m)), _ptr(mu),
                                              _ptr(evecs), int(L), _ptr(scores), int(n),
                                              _ptr(xhat)))

    # ---- d = 3 fused smoother ------------------------------------------------
    def cov_factor_bytes(self, m, n):
        return int(self.lib.fpca_cov_factor_bytes(ctypes.byref(Grid.of(m)), int(n)))

    def bin_cov_factor(self, data, m, mu, factor):
        """factor: a uint8 device tensor of at least cov_factor_bytes(m, n) bytes."""
        self._check(self.lib.fpca_bin_cov_factor(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                                 _ptr(mu), _ptr(factor), int(factor.numel())))

    def smooth_cov_apply(self, m, factor, n, h, x, y):
        self._check(self.lib.fpca_smooth_cov_apply(self.h, ctypes.byref(Grid.of(m)), _ptr(factor),
                                                   int(n), _doubles(h), _ptr(x), int(x.shape[1]),
                                                   _ptr(y)))

    def smooth_cov_tiles(self, m, factor, n, h, tiles, out):
        """tiles: host int32 array (ntiles, 6) of s- and t-box corners."""
        import numpy as np
        tl = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1, 6))
        arr = (ctypes.c_int32 * tl.size)(*tl.ravel().tolist())
        self._check(self.lib.fpca_smooth_cov_tiles(self.h, ctypes.byref(Grid.of(m)), _ptr(factor),
                                                   int(n), _doubles(h), int(tl.shape[0]), arr,
                                                   _ptr(out)))

    def smooth_cov_diag(self, m, factor, n, h, diag):
        self._check(self.lib.fpca_smooth_cov_diag(self.h, ctypes.byref(Grid.of(m)), _ptr(factor),
                                                  int(n), _doubles(h), _ptr(diag)))

    def rproj_eig_factor(self, m, factor, n, h, omega, k, evals, evecs, fve=None, power_iters=0):
        self._check(self.lib.fpca_rproj_eig_factor(self.h, ctypes.byref(Grid.of(m)), _ptr(factor),
                                                   int(n), _doubles(h), _ptr(omega),
                                                   int(omega.shape[1]), int(k), int(power_iters),
                                                   _ptr(evals), _ptr(evecs), _ptr(fve)))

    def bw_predict(self, params, feat, out):
        self._check(self.lib.fpca_bw_predict(self.h, _ptr(params), _ptr(feat), int(feat.shape[0]),
                                             _ptr(out)))

    def bw_train_step(self, params, m, v, step, feat, target, tmask, lr=1e-3, wd=1e-4,
                      loss=None, grad=None):
        self._check(self.lib.fpca_bw_train_step(
            self.h, _ptr(params), _ptr(m), _ptr(v), int(step), _ptr(feat), _ptr(target),
            _ptr(tmask), int(feat.shape[0]), float(lr), float(wd), _ptr(loss), _ptr(grad)))

    # ---- data descriptors --------------------------------------------------
    @staticmethod
    def dense(y, mask=None):
        """Dense data descriptor; it holds references to ``y`` and ``mask``."""
        d = Data()
        d._keep = (y, mask)
        d.layout = DENSE
        d.n = int(y.shape[0])
        d.y = y.data_ptr()
        d.y_prec = F64 if y.dtype.itemsize == 8 else F32
        d.mask = None if mask is None else mask.data_ptr()
        return d

    @staticmethod
    def sparse(offs, t, y):
        """Sparse data descriptor; it holds references to its tensors."""
        d = Data()
        d._keep = (offs, t, y)
        d.layout = SPARSE
        d.n = int(offs.shape[0]) - 1
        d.y = y.data_ptr()
        d.y_prec = F64
        d.offs = offs.data_ptr()
        d.t = t.data_ptr()
        return d

    # ---- entry points --------------------------------------------------------
    def bin_mean(self, data, m, cnt, w, v, v2=None):
        self._check(self.lib.fpca_bin_mean(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                           _ptr(cnt), _ptr(w), _ptr(v), _ptr(v2)))

    def smooth_mean(self, m, cnt, w, v, h, mu, status=None):
        self._check(self.lib.fpca_smooth_mean(self.h, ctypes.byref(Grid.of(m)), _ptr(cnt), _ptr(w),
                                              _ptr(v), _doubles(h), _ptr(mu), _ptr(status)))

    def smooth_mean_cv(self, data, m, fold, nfold, hs, cv):
        """K-fold CV score of the mean smoother for each bandwidth vector in hs."""
        flat = [float(x) for hv in hs for x in (hv if hasattr(hv, "__len__") else [hv] * len(m))]
        self._check(self.lib.fpca_smooth_mean_cv(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                                 _ptr(fold), int(nfold), _doubles(flat), len(hs),
                                                 _ptr(cv)))

    def bin_cov(self, data, m, mu, prec, cnt, w, v, q=None, mode=COV_RESIDUAL, fold=None, nfold=0):
        self._check(self.lib.fpca_bin_cov(self.h, ctypes.byref(data), ctypes.byref(Grid.of(m)),
                                          _ptr(mu), int(prec), int(mode), _ptr(fold), int(nfold),
                                          _ptr(cnt), _ptr(w), _ptr(v), _ptr(q)))

    def smooth_cov_project(self, m, cnt, w, v, h, prec, q=None, nfold=0, mu_raw=None, omega=None,
                           gamma=None, status=None, y=None, cv=None, symmetric=True):
        """symmetric=False for bins that are not symmetric in (s, t) (fpca_bin_cov's are)."""
        if cnt.dtype.itemsize != 4 or cnt.dtype.is_floating_point:
            raise TypeError(f"cnt must hold int32 pair counts (got {cnt.dtype})")
        if w.dtype != v.dtype or (q is not None and q.dtype != w.dtype):
            raise TypeError("w, v (and q) must share one floating type")
        bins = CovBins()
        bins.asym = 0 if symmetric else 1
        bins.nfold = int(nfold)
        bins.prec = F64 if w.dtype.itemsize == 8 else F32
        bins.cnt, bins.w, bins.v = cnt.data_ptr(), w.data_ptr(), v.data_ptr()
        bins.q = None if q is None else q.data_ptr()
        hs = [x for row in h for x in row]
        nh = len(h)
        l = 0 if omega is None else int(omega.shape[1])
        self._check(self.lib.fpca_smooth_cov_project(
            self.h, ctypes.byref(Grid.of(m)), ctypes.byref(bins), _doubles(hs), nh, int(prec),
            _ptr(mu_raw), _ptr(omega), l, _ptr(gamma), _ptr(status), _ptr(y), _ptr(cv)))

    def bw_trust_region(self, m, cnt, w, v, q, nfold, prec, h0, options=None, trace_cap=256):
        """Section 3.3 trust-region search on the CV of the given fold bins.
        Returns (h_best, cv_best, trace) with trace a list of (h tuple, cv)."""
        bins = CovBins()
        bins.nfold = int(nfold)
        bins.prec = F64 if w.dtype.itemsize == 8 else F32
        bins.cnt, bins.w, bins.v, bins.q = cnt.data_ptr(), w.data_ptr(), v.data_ptr(), q.data_ptr()
        d = len(m)
        opt = None
        if options is not None:
            opt = TrOptions()
            base = dict(delta0=0.4, delta_min=0.01, delta_max=1.0, h_lo=0.02, h_hi=0.6, max_iter=20)
            base.update(options)
            for k, val in base.items():
                setattr(opt, k, val)
        hb = (ctypes.c_double * d)()
        cvb = ctypes.c_double()
        ne = ctypes.c_int()
        tr = (ctypes.c_double * (trace_cap * (d + 1)))()
        self._check(self.lib.fpca_bw_trust_region(
            self.h, ctypes.byref(Grid.of(m)), ctypes.byref(bins), int(prec), _doubles(h0),
            None if opt is None else ctypes.byref(opt), hb, ctypes.byref(cvb), ctypes.byref(ne),
            tr, int(trace_cap)))
        trace = [(tuple(tr[i * (d + 1):i * (d + 1) + d]), tr[i * (d + 1) + d])
                 for i in range(min(ne.value, trace_cap))]
        return tuple(hb), cvb.value, trace

    def rproj_eig(self, m, gamma, k, evals, evecs, fve=None, domain=None, omega=None,
                  power_iters=0, full=False):
        l = 0 if omega is None else int(omega.shape[1])
        gp = F64 if gamma.dtype.itemsize == 8 else F32
        self._check(self.lib.fpca_rproj_eig(self.h, ctypes.byref(Grid.of(m)), _ptr(gamma), gp,
                                            _ptr(domain), _ptr(omega), l, int(k),
                                            int(power_iters), int(bool(full)), _ptr(evals),
                                            _ptr(evecs), _ptr(fve)))
