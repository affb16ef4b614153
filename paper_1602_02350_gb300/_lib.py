"""ctypes binding of ``librs.so`` (the C ABI in include/rs.h).

Argument marshalling only: every step runs in the library's CUDA kernels.  Tensors
must be CUDA tensors (PyTorch supplies device memory and streams); unsigned index
data travels in int32 / int64 tensors holding the uint32 / uint64 bit patterns.
There is no CPU fallback: without the built library every call raises.
"""

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librs.so")

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ENONFINITE, RS_ETIMEOUT, RS_EDIVERGED, RS_ENOTCONVERGED, RS_EUNSUPPORTED = range(9)
RS_F64, RS_F32, RS_BF16, RS_FP8E4M3 = 0, 1, 2, 3
RS_SKETCH_GAUSSIAN, RS_SKETCH_COUNTSKETCH = 0, 1
RS_SAMPLE_IMPORTANCE, RS_SAMPLE_UNIFORM = 0, 1

_DT = {torch.float64: RS_F64, torch.float32: RS_F32, torch.bfloat16: RS_BF16, torch.float8_e4m3fn: RS_FP8E4M3}
_TORCH = {RS_F64: torch.float64, RS_F32: torch.float32, RS_BF16: torch.bfloat16}


class RsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rs status {code}: {msg}")
        self.code = code


class Matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("row_scale", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("d", ctypes.c_int64), ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SketchParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("s", ctypes.c_int64),
                ("q_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class SvrgParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("eta", ctypes.c_double), ("eta_mult", ctypes.c_double),
                ("m", ctypes.c_int64), ("epochs", ctypes.c_int32), ("epoch0", ctypes.c_int32),
                ("sampling", ctypes.c_int32), ("average", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("refine", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("step", ctypes.c_int32), ("reserved", ctypes.c_int32)]


MLP_IN, MLP_HIDDEN, MLP_OUT = 67, 128, 3
MLP_NPARAM = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_OUT * MLP_HIDDEN + MLP_OUT


class MlpNorm(ctypes.Structure):
    _fields_ = [("in_mean", ctypes.c_float * MLP_IN), ("in_std", ctypes.c_float * MLP_IN),
                ("out_mean", ctypes.c_float * MLP_OUT), ("out_std", ctypes.c_float * MLP_OUT)]


class Problem(ctypes.Structure):
    _fields_ = [("X", Matrix), ("y", ctypes.c_void_p), ("k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Chain(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("eta_mult", ctypes.c_double), ("m", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("w_out", ctypes.c_void_p), ("snapshots", ctypes.c_void_p)]


class BatchParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("sketch_kind", ctypes.c_int32), ("q_blocks", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("average", ctypes.c_int32),
                ("sketch_seed", ctypes.c_uint64)]


class CatalystParams(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("outer", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("chain_cluster", ctypes.c_int32), ("chain_threads", ctypes.c_int32), ("chain_stages", ctypes.c_int32),
                ("chain_ms", ctypes.c_float), ("fullgrad_stages", ctypes.c_int32), ("fullgrad_ms", ctypes.c_float),
                ("candidates", ctypes.c_int32), ("cached", ctypes.c_int32)]


class History(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int32), ("epochs_run", ctypes.c_int32), ("snapshots", ctypes.c_void_p),
                ("mu_norm2", ctypes.POINTER(ctypes.c_double)), ("epoch_ms", ctypes.POINTER(ctypes.c_float))]


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "rs_create": [ctypes.POINTER(_P), ctypes.c_int, _P],
    "rs_destroy": [_P],
    "rs_set_stream": [_P, _P],
    "rs_last_error": [],
    "rs_abi_version": [],
    "rs_launch_count": [_P],
    "rs_philox_words": [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, _P],
    "rs_gaussian": [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _P,
                    ctypes.c_int64],
    "rs_countsketch": [_P, ctypes.POINTER(Matrix), ctypes.c_uint64, ctypes.c_int64, _P, ctypes.c_int64, _P, _P],
    "rs_range_sketch": [_P, ctypes.POINTER(Matrix), ctypes.POINTER(SketchParams), _P],
    "rs_orthonormalize": [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _P],
    "rs_sym_eig": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P],
    "rs_ritz": [_P, ctypes.POINTER(Matrix), _P, ctypes.c_int64, _P, _P],
    "rs_sketch": [_P, ctypes.POINTER(Matrix), ctypes.POINTER(SketchParams), _P, _P],
    "rs_precondition": [_P, ctypes.POINTER(Matrix), _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(Matrix),
                        _P, ctypes.POINTER(ctypes.c_double)],
    "rs_map_output": [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, _P, _P],
    "rs_sampling_weights": [_P, _P, ctypes.c_int32, ctypes.c_int64, _P],
    "rs_sampling_table": [_P, _P, ctypes.c_int64, _P],
    "rs_index_stream": [_P, _P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                        ctypes.c_int32, ctypes.c_int32, _P, _P],
    "rs_full_gradient": [_P, ctypes.POINTER(Matrix), _P, ctypes.c_int64, ctypes.c_double, _P, _P],
    "rs_full_gradient_static": [_P, ctypes.POINTER(Matrix), _P, ctypes.c_int64, ctypes.c_double, _P, _P],
    "rs_svrg_epoch": [_P, ctypes.POINTER(Matrix), ctypes.c_int64, ctypes.c_double, _P, _P, ctypes.c_int64,
                      ctypes.c_double, _P, _P, ctypes.c_int32, _P],
    "rs_svrg_solve": [_P, ctypes.POINTER(Matrix), ctypes.POINTER(Matrix), _P, _P, _P, _P, ctypes.c_int64,
                      ctypes.POINTER(SvrgParams), _P, _P,
                      ctypes.POINTER(History), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
    "rs_solve": [_P, ctypes.POINTER(Matrix), _P, ctypes.POINTER(SketchParams), ctypes.POINTER(SvrgParams), _P,
                 ctypes.POINTER(History)],
    "rs_objective": [_P, ctypes.POINTER(Matrix), _P, ctypes.c_double, _P, _P, ctypes.POINTER(ctypes.c_double)],
    "rs_trace_c": [_P, ctypes.POINTER(Matrix), ctypes.POINTER(ctypes.c_double)],
    "rs_speedup_ratio": [_P, _P, ctypes.c_int64, ctypes.c_double, _P, _P],
    "rs_wait_probe": [_P, ctypes.c_int64, ctypes.c_int32],
    "rs_autotune": [_P, ctypes.POINTER(Matrix), ctypes.c_int64, ctypes.POINTER(TuneReport)],
    "rs_catalyst_solve": [_P, ctypes.POINTER(Matrix), ctypes.POINTER(Matrix), _P, _P, _P, _P, ctypes.c_int64,
                          ctypes.POINTER(SvrgParams), ctypes.POINTER(CatalystParams), _P, ctypes.POINTER(History),
                          ctypes.POINTER(ctypes.c_double)],
    "rs_solve_batched": [_P, ctypes.POINTER(Problem), ctypes.c_int32, ctypes.POINTER(Chain), ctypes.c_int32,
                         ctypes.POINTER(BatchParams), ctypes.POINTER(ctypes.c_float)],
    "rs_mlp_forward": [_P, _P, _P, ctypes.c_int64, _P],
    "rs_solve_proposed": [_P, ctypes.POINTER(Matrix), _P, ctypes.POINTER(SketchParams), ctypes.POINTER(SvrgParams),
                          _P, ctypes.POINTER(MlpNorm), ctypes.c_int32, _P, ctypes.POINTER(History),
                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
    "rs_mlp_train_step": [_P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(AdamParams), _P, _P],
    "rs_propose": [_P, _P, ctypes.POINTER(MlpNorm), ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int64,
                   ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
}
_RESTYPES = {"rs_last_error": ctypes.c_char_p, "rs_launch_count": ctypes.c_int64}


def lib():
    """Load librs.so (built in-tree by ``paper_1602_02350_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_1602_02350_gb300.build` "
                               "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, ctypes.c_int)
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != RS_OK:
        raise RsError(rc, lib().rs_last_error().decode(errors="replace"))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need_cuda(*ts):
    for t in ts:
        if t is not None and (not isinstance(t, torch.Tensor) or not t.is_cuda):
            raise TypeError("expected a CUDA tensor")


class Fp8Rows:
    """FP8-e4m3 rows with one float scale per row (value = code * scale): the component storage
    rs_precondition writes for z_dtype=torch.float8_e4m3fn."""

    def __init__(self, codes, scale):
        self.codes, self.scale = codes, scale
        self.shape = codes.shape
        self.dtype = codes.dtype

    def dequantize(self):
        return self.codes.float() * self.scale[:, None]


def matrix(t, row_scale=None):
    """rs_matrix descriptor of a row-major 2-D CUDA tensor (row stride = t.stride(0)), or of Fp8Rows."""
    if isinstance(t, Fp8Rows):
        return matrix(t.codes, row_scale=t.scale)
    _need_cuda(t)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("matrix: need a 2-D tensor with unit column stride")
    return Matrix(t.data_ptr(), None if row_scale is None else row_scale.data_ptr(), t.shape[0], t.shape[1],
                  t.stride(0), _DT[t.dtype], 0)


class Context:
    """An rs_ctx bound to a CUDA device and stream (default: the current torch stream)."""

    def __init__(self, device=0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("rs: no CUDA device (the library has no CPU fallback)")
        self.device = torch.device("cuda", device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        h = ctypes.c_void_p()
        _check(lib().rs_create(ctypes.byref(h), device, ctypes.c_void_p(s.cuda_stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().rs_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    @property
    def launches(self):
        return lib().rs_launch_count(self.h)

    def _empty(self, *shape, dtype):
        return torch.empty(*shape, dtype=dtype, device=self.device)


def _ctdt(t):
    return RS_F64 if t.dtype == torch.float64 else RS_F32


def _compute_dtype(X):
    return torch.float64 if X.dtype == torch.float64 else torch.float32


# ----------------------------------------------------------------------------- entry points

def rs_philox_words(ctx, seed, c2, c3, count):
    out = ctx._empty(count * 4, dtype=torch.int32)
    _check(lib().rs_philox_words(ctx.h, seed, c2, c3, count, _ptr(out)))
    return out


def rs_gaussian(ctx, seed, rows, cols, dtype=torch.float32, row0=0):
    out = ctx._empty(rows, cols, dtype=dtype)
    _check(lib().rs_gaussian(ctx.h, seed, row0, rows, cols, _DT[dtype], _ptr(out), cols))
    return out


def rs_countsketch(ctx, X, seed, s, with_hash=False):
    ct = _compute_dtype(X)
    SX = ctx._empty(s, X.shape[1], dtype=ct)
    bucket = ctx._empty(X.shape[0], dtype=torch.int32) if with_hash else None
    sign = ctx._empty(X.shape[0], dtype=ct) if with_hash else None
    M = matrix(X)
    _check(lib().rs_countsketch(ctx.h, ctypes.byref(M), seed, s, _ptr(SX), X.shape[1], _ptr(bucket), _ptr(sign)))
    return (SX, bucket, sign) if with_hash else SX


def _sketch_params(k, seed, kind, s, q):
    kind_i = RS_SKETCH_COUNTSKETCH if kind in ("countsketch", RS_SKETCH_COUNTSKETCH) else RS_SKETCH_GAUSSIAN
    return SketchParams(kind_i, k, s, q, 0, seed)


def rs_range_sketch(ctx, X, k, seed, kind="gaussian", s=0):
    Y = ctx._empty(X.shape[1], k, dtype=_compute_dtype(X))
    M = matrix(X)
    p = _sketch_params(k, seed, kind, s, 1)
    _check(lib().rs_range_sketch(ctx.h, ctypes.byref(M), ctypes.byref(p), _ptr(Y)))
    return Y


def rs_orthonormalize(ctx, Y):
    _need_cuda(Y)
    Y = Y.contiguous()
    Q = torch.empty_like(Y)
    _check(lib().rs_orthonormalize(ctx.h, _ptr(Y), Y.shape[0], Y.shape[1], _ctdt(Y), _ptr(Q)))
    return Q


def rs_sym_eig(ctx, G, prec=RS_F64):
    _need_cuda(G)
    G = G.to(torch.float64).contiguous()
    k = G.shape[0]
    ev = ctx._empty(k, dtype=torch.float64)
    W = ctx._empty(k, k, dtype=torch.float64)
    _check(lib().rs_sym_eig(ctx.h, _ptr(G), k, prec, _ptr(ev), _ptr(W)))
    return ev, W


def rs_ritz(ctx, X, Q):
    k = Q.shape[1]
    V = ctx._empty(X.shape[1], k, dtype=_compute_dtype(X))
    s2 = ctx._empty(k, dtype=torch.float64)
    M = matrix(X)
    _check(lib().rs_ritz(ctx.h, ctypes.byref(M), _ptr(Q.contiguous()), k, _ptr(V), _ptr(s2)))
    return V, s2


def rs_sketch(ctx, X, k, seed, kind="gaussian", s=0, q=1):
    V = ctx._empty(X.shape[1], k, dtype=_compute_dtype(X))
    s2 = ctx._empty(k, dtype=torch.float64)
    M = matrix(X)
    p = _sketch_params(k, seed, kind, s, q)
    _check(lib().rs_sketch(ctx.h, ctypes.byref(M), ctypes.byref(p), _ptr(V), _ptr(s2)))
    return V, s2


def _padded_ld(d, dtype):
    es = torch.empty((), dtype=dtype).element_size()
    return ((d * es + 15) // 16 * 16) // es


def rs_precondition(ctx, X, V, sigma2, lam, want_beta_hat=True, z_dtype=None):
    """Components Z ((n + d) x d, stored like X, or in z_dtype = torch.bfloat16 for float32 X, or
    z_dtype = torch.float8_e4m3fn: then Z is Fp8Rows (codes and per-row scales))."""
    n, d = X.shape
    zt = X.dtype if z_dtype is None else z_dtype
    ld = _padded_ld(d, zt)
    Zs = ctx._empty(n + d, ld, dtype=zt)
    Z = Zs[:, :d]
    if zt == torch.float8_e4m3fn:
        Z = Fp8Rows(Z, ctx._empty(n + d, dtype=torch.float32))
    beta = ctx._empty(n + d, dtype=_compute_dtype(X))
    MX, MZ = matrix(X), matrix(Z)
    bh = ctypes.c_double(0.0)
    _check(lib().rs_precondition(ctx.h, ctypes.byref(MX), _ptr(V.contiguous()), _ptr(sigma2), V.shape[1], lam,
                                 ctypes.byref(MZ), _ptr(beta), ctypes.byref(bh) if want_beta_hat else None))
    return Z, beta, bh.value


def rs_map_output(ctx, V, sigma2, lam, w_tilde):
    w = torch.empty_like(w_tilde)
    _check(lib().rs_map_output(ctx.h, _ptr(V.contiguous()), _ptr(sigma2), V.shape[0], V.shape[1], lam,
                               _ctdt(w_tilde), _ptr(w_tilde), _ptr(w)))
    return w


def rs_sampling_weights(ctx, beta):
    W = ctx._empty(beta.shape[0], dtype=torch.int32)
    _check(lib().rs_sampling_weights(ctx.h, _ptr(beta), _ctdt(beta), beta.shape[0], _ptr(W)))
    return W


def rs_sampling_table(ctx, W):
    cum = ctx._empty(W.shape[0], dtype=torch.int64)
    _check(lib().rs_sampling_table(ctx.h, _ptr(W), W.shape[0], _ptr(cum)))
    return cum


def rs_index_stream(ctx, W, cum, N, seed, epoch, m, t0=0, sampling=RS_SAMPLE_IMPORTANCE, dtype=torch.float32):
    idx = ctx._empty(m, dtype=torch.int32)
    inq = ctx._empty(m, dtype=dtype)
    _check(lib().rs_index_stream(ctx.h, _ptr(W), _ptr(cum), N, seed, epoch, t0, m, sampling, _DT[dtype], _ptr(idx),
                                 _ptr(inq)))
    return idx, inq


def rs_full_gradient(ctx, Z, y, n, lam, w):
    mu = ctx._empty(Z.shape[1], dtype=w.dtype)
    M = matrix(Z)
    _check(lib().rs_full_gradient(ctx.h, ctypes.byref(M), _ptr(y), n, lam, _ptr(w), _ptr(mu)))
    return mu


def rs_full_gradient_static(Z, y, n, lam, w, stream=None, out=None):
    """Allocation-free full gradient (no context; scratch is a fixed array in the library's device
    data).  ``out`` may be a preallocated CUDA tensor; the call itself allocates nothing on the
    device.  ``stream`` defaults to the current torch stream of Z's device."""
    _need_cuda(Z, y, w)
    mu = torch.empty(Z.shape[1], dtype=w.dtype, device=Z.device) if out is None else out
    s = stream if stream is not None else torch.cuda.current_stream(Z.device)
    M = matrix(Z)
    with torch.cuda.device(Z.device):
        _check(lib().rs_full_gradient_static(ctypes.c_void_p(s.cuda_stream), ctypes.byref(M), _ptr(y), n, lam, _ptr(w),
                                             _ptr(mu)))
    return mu


def rs_svrg_epoch(ctx, Z, n, lam, idx, inv_nq, eta, w_bar, mu, average=True):
    out = torch.empty_like(w_bar)
    M = matrix(Z)
    _check(lib().rs_svrg_epoch(ctx.h, ctypes.byref(M), n, lam, _ptr(idx), _ptr(inv_nq), idx.shape[0], eta,
                               _ptr(w_bar), _ptr(mu), 1 if average else 0, _ptr(out)))
    return out


def _svrg_params(lam, epochs, seed, eta=0.0, eta_mult=0.0, m=0, epoch0=0, sampling=RS_SAMPLE_IMPORTANCE, average=True,
                 refine=False):
    return SvrgParams(lam, eta, eta_mult, m, epochs, epoch0, sampling, 1 if average else 0, seed, 1 if refine else 0, 0)


def _history(ctx, epochs, d, dtype, snapshots):
    mu2 = (ctypes.c_double * max(1, epochs))()
    ems = (ctypes.c_float * max(1, epochs))()
    snaps = ctx._empty(max(1, epochs), d, dtype=dtype) if snapshots else None
    h = History(epochs, 0, None if snaps is None else snaps.data_ptr(),
                ctypes.cast(mu2, ctypes.POINTER(ctypes.c_double)), ctypes.cast(ems, ctypes.POINTER(ctypes.c_float)))
    return h, mu2, ems, snaps


def rs_svrg_solve(ctx, Z, y, V, sigma2, lam, epochs, seed, beta=None, w0=None, eta=0.0, eta_mult=0.0, m=0,
                  epoch0=0, sampling=RS_SAMPLE_IMPORTANCE, average=True, snapshots=False, X=None, refine=False):
    d = Z.shape[1]
    w = ctx._empty(d, dtype=V.dtype)
    p = _svrg_params(lam, epochs, seed, eta, eta_mult, m, epoch0, sampling, average, refine)
    MX = matrix(X) if X is not None else None
    h, mu2, ems, snaps = _history(ctx, epochs, d, V.dtype, snapshots)
    eu, mu_ = ctypes.c_double(0), ctypes.c_int64(0)
    M = matrix(Z)
    _check(lib().rs_svrg_solve(ctx.h, ctypes.byref(M), ctypes.byref(MX) if MX is not None else None, _ptr(y),
                               _ptr(beta), _ptr(V.contiguous()), _ptr(sigma2),
                               V.shape[1], ctypes.byref(p), _ptr(w0), _ptr(w), ctypes.byref(h), ctypes.byref(eu),
                               ctypes.byref(mu_)))
    info = {"eta": eu.value, "m": mu_.value, "mu_norm2": list(mu2)[:epochs], "epoch_ms": list(ems)[:epochs],
            "snapshots": snaps[:epochs] if snaps is not None else None}
    return w, info


def rs_catalyst_solve(ctx, Z, y, V, sigma2, lam, outer, epochs, seed, kappa=0.0, beta=None, eta_mult=1.0, m=0,
                      epoch0=0, sampling=RS_SAMPLE_IMPORTANCE, average=True, snapshots=False, X=None, refine=False):
    """Accelerated SVRG (Catalyst) on the components Z: ``outer`` proximal problems of ``epochs`` epochs
    each.  Returns (w, info) with info holding kappa, the outer iterates (snapshots) and their times."""
    d = Z.shape[1]
    w = ctx._empty(d, dtype=V.dtype)
    p = _svrg_params(lam, epochs, seed, 0.0, eta_mult, m, epoch0, sampling, average, refine)
    cp = CatalystParams(float(kappa), int(outer), 0)
    MX = matrix(X) if X is not None else None
    h, _, ems, snaps = _history(ctx, outer, d, V.dtype, snapshots)
    ku = ctypes.c_double(0)
    M = matrix(Z)
    _check(lib().rs_catalyst_solve(ctx.h, ctypes.byref(M), ctypes.byref(MX) if MX is not None else None, _ptr(y),
                                   _ptr(beta), _ptr(V.contiguous()), _ptr(sigma2), V.shape[1], ctypes.byref(p),
                                   ctypes.byref(cp), _ptr(w), ctypes.byref(h), ctypes.byref(ku)))
    info = {"kappa": ku.value, "epoch_ms": list(ems)[:outer], "snapshots": snaps[:outer] if snaps is not None else None}
    return w, info


def rs_solve(ctx, X, y, k, lam, epochs, sketch_seed, svrg_seed, kind="gaussian", s=0, q=1, eta=0.0, eta_mult=0.0,
             m=0, sampling=RS_SAMPLE_IMPORTANCE, average=True, snapshots=False, w_out=None, refine=None):
    """Alg. 3 end to end.  X / y may be CUDA tensors or (pinned) CPU tensors; w_out likewise."""
    d = X.shape[1]
    ct = torch.float64 if X.dtype == torch.float64 else torch.float32
    if w_out is None:
        w_out = ctx._empty(d, dtype=ct) if X.is_cuda else torch.empty(d, dtype=ct)
    M = Matrix(X.data_ptr(), None, X.shape[0], d, X.stride(0), _DT[X.dtype], 0)
    sp = _sketch_params(k, sketch_seed, kind, s, q)
    if refine is None:
        refine = X.dtype == torch.bfloat16
    p = _svrg_params(lam, epochs, svrg_seed, eta, eta_mult, m, 0, sampling, average, refine)
    h, mu2, ems, snaps = _history(ctx, epochs, d, ct, snapshots)
    _check(lib().rs_solve(ctx.h, ctypes.byref(M), _ptr(y), ctypes.byref(sp), ctypes.byref(p), _ptr(w_out),
                          ctypes.byref(h)))
    info = {"mu_norm2": list(mu2)[:epochs], "epoch_ms": list(ems)[:epochs],
            "snapshots": snaps[:epochs] if snaps is not None else None}
    return w_out, info


def rs_objective(ctx, X, y, lam, w, w_ref=None):
    out = (ctypes.c_double * 2)()
    M = matrix(X)
    _check(lib().rs_objective(ctx.h, ctypes.byref(M), _ptr(y), lam, _ptr(w), _ptr(w_ref),
                              ctypes.cast(out, ctypes.POINTER(ctypes.c_double))))
    return out[0], out[1]


def rs_trace_c(ctx, X):
    """tr(C) = ||X||_F^2 / n in double."""
    out = ctypes.c_double(0.0)
    M = matrix(X)
    _check(lib().rs_trace_c(ctx.h, ctypes.byref(M), ctypes.byref(out)))
    return out.value


def rs_autotune(ctx, Z, n):
    """Time the launch layouts of the inner loop and the full-gradient pass for components Z and keep
    the fastest in the context; returns the report as a dict."""
    r = TuneReport()
    M = matrix(Z)
    _check(lib().rs_autotune(ctx.h, ctypes.byref(M), n, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in TuneReport._fields_}


def rs_wait_probe(ctx, budget_cycles, complete):
    """Run one bounded device-side wait; raises RsError(RS_ETIMEOUT) when it gives up."""
    _check(lib().rs_wait_probe(ctx.h, int(budget_cycles), 1 if complete else 0))


def rs_speedup_ratio(ctx, sigma2, trace_c):
    """ratio(k) after Thm 1 for k = 1..len(sigma2) from sketched eigenvalues (CUDA float64, descending)
    and tr(C): returns (ratio, sqrt(ratio)) as CUDA float64 tensors."""
    _need_cuda(sigma2)
    s2 = sigma2.to(torch.float64).contiguous()
    K = s2.shape[0]
    r = ctx._empty(K, dtype=torch.float64)
    ra = ctx._empty(K, dtype=torch.float64)
    _check(lib().rs_speedup_ratio(ctx.h, _ptr(s2), K, float(trace_c), _ptr(r), _ptr(ra)))
    return r, ra


def rs_solve_batched(ctx, problems, chains, epochs, sketch_seed=0, kind="gaussian", q=1, refine=None, use_graph=True,
                     average=True, snapshots=False):
    """Solve many chains at once.

    problems: list of (X, y, k) with X a CUDA tensor (float32 or bfloat16, row stride padded to 16
    bytes), y float32 labels and k the sketch rank (0 = d / 16).
    chains: list of dicts with keys problem, lam, and optionally eta_mult, m, seed.
    Returns (list of w (float32, d), list of snapshot tensors or None, epoch_ms list)."""
    np_ = len(problems)
    P = (Problem * np_)()
    for i, (X, y, k) in enumerate(problems):
        _need_cuda(X, y)
        P[i] = Problem(matrix(X), y.data_ptr(), int(k), 0)
    nc = len(chains)
    C = (Chain * nc)()
    outs, snaps = [], []
    for i, ch in enumerate(chains):
        pi = int(ch["problem"])
        d = problems[pi][0].shape[1] if 0 <= pi < np_ else 1   # an invalid index is rejected by the library
        w = ctx._empty(d, dtype=torch.float32)
        sn = ctx._empty(epochs, d, dtype=torch.float32) if snapshots else None
        outs.append(w)
        snaps.append(sn)
        C[i] = Chain(int(ch["problem"]), 0, float(ch["lam"]), float(ch.get("eta_mult", 0.0)), int(ch.get("m", 0)),
                     int(ch.get("seed", 0)), w.data_ptr(), None if sn is None else sn.data_ptr())
    if refine is None:
        refine = problems[0][0].dtype == torch.bfloat16
    kind_i = RS_SKETCH_COUNTSKETCH if kind in ("countsketch", RS_SKETCH_COUNTSKETCH) else RS_SKETCH_GAUSSIAN
    bp = BatchParams(epochs, kind_i, q, 1 if refine else 0, 1 if use_graph else 0, 1 if average else 0, sketch_seed)
    ems = (ctypes.c_float * epochs)()
    _check(lib().rs_solve_batched(ctx.h, P, np_, C, nc, ctypes.byref(bp), ems))
    return outs, (snaps if snapshots else None), list(ems)


# ----------------------------------------------------------------------------- proposal network

def _f32(ctx, t):
    _need_cuda(t)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return t


def rs_mlp_forward(ctx, theta, X):
    """Network outputs (B x 3, float32) for the rows of X (B x 67)."""
    _f32(ctx, theta), _f32(ctx, X)
    out = ctx._empty(X.shape[0], MLP_OUT, dtype=torch.float32)
    _check(lib().rs_mlp_forward(ctx.h, _ptr(theta), _ptr(X), X.shape[0], _ptr(out)))
    return out


def rs_mlp_train_step(ctx, theta, adam_m, adam_v, X, T, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                      want_grad=False, loss_out=None):
    """One Adam step in place on theta / adam_m / adam_v.  Returns (gradient or None, loss tensor)."""
    for t in (theta, adam_m, adam_v, X, T):
        _f32(ctx, t)
    g = ctx._empty(MLP_NPARAM, dtype=torch.float32) if want_grad else None
    loss = loss_out if loss_out is not None else ctx._empty(1, dtype=torch.float32)
    p = AdamParams(lr, beta1, beta2, eps, step, 0)
    _check(lib().rs_mlp_train_step(ctx.h, _ptr(theta), _ptr(adam_m), _ptr(adam_v), _ptr(X), _ptr(T), X.shape[0],
                                   ctypes.byref(p), _ptr(g), _ptr(loss)))
    return g, loss


def mlp_norm(in_mean, in_std, out_mean, out_std):
    nm = MlpNorm()
    for j in range(MLP_IN):
        nm.in_mean[j], nm.in_std[j] = float(in_mean[j]), float(in_std[j])
    for j in range(MLP_OUT):
        nm.out_mean[j], nm.out_std[j] = float(out_mean[j]), float(out_std[j])
    return nm


def rs_propose(ctx, sigma2, lam, n, d, trace_c, theta=None, norm=None):
    """(k, eta_mult, m, used_fallback) for sketched eigenvalues sigma2 (64 values, descending)."""
    s = (ctypes.c_double * 64)(*[float(v) for v in list(sigma2)[:64]])
    if theta is not None:
        _f32(ctx, theta)
    k, em, m, fb = ctypes.c_int32(0), ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int32(0)
    _check(lib().rs_propose(ctx.h, _ptr(theta), ctypes.byref(norm) if norm is not None else None, s, lam, n, d,
                            trace_c, ctypes.byref(k), ctypes.byref(em), ctypes.byref(m), ctypes.byref(fb)))
    return k.value, em.value, m.value, bool(fb.value)


def rs_solve_proposed(ctx, X, y, lam, epochs, sketch_seed, svrg_seed, theta=None, norm=None, kind="gaussian", s=0,
                      q=1, z_dtype=None, sampling=RS_SAMPLE_IMPORTANCE, average=True, snapshots=False, w_out=None,
                      k_fixed=0):
    """Alg. 3 with proposed (k, eta, m), or with k_fixed > 64 the sketch rank fixed by the caller and
    only (eta, m) proposed.  X / y / w_out may be CUDA or (pinned) CPU tensors.
    Returns (w, info) with info holding k, eta_mult, m, fallback and the epoch history."""
    d = X.shape[1]
    ct = torch.float64 if X.dtype == torch.float64 else torch.float32
    if w_out is None:
        w_out = ctx._empty(d, dtype=ct) if X.is_cuda else torch.empty(d, dtype=ct)
    M = Matrix(X.data_ptr(), None, X.shape[0], d, X.stride(0), _DT[X.dtype], 0)
    sp = _sketch_params(max(64, int(k_fixed)), sketch_seed, kind, s, q)
    zt = _DT[z_dtype] if z_dtype is not None else _DT[X.dtype]
    p = _svrg_params(lam, epochs, svrg_seed, 0.0, 0.0, 0, 0, sampling, average, refine=zt != _DT[X.dtype] or
                     X.dtype == torch.bfloat16)
    h, mu2, ems, snaps = _history(ctx, epochs, d, ct, snapshots)
    if theta is not None:
        _need_cuda(theta)
    k, em, m, fb = ctypes.c_int32(0), ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int32(0)
    _check(lib().rs_solve_proposed(ctx.h, ctypes.byref(M), _ptr(y), ctypes.byref(sp), ctypes.byref(p), _ptr(theta),
                                   ctypes.byref(norm) if norm is not None else None, zt, _ptr(w_out), ctypes.byref(h),
                                   ctypes.byref(k), ctypes.byref(em), ctypes.byref(m), ctypes.byref(fb)))
    info = {"k": k.value, "eta_mult": em.value, "m": m.value, "fallback": bool(fb.value),
            "mu_norm2": list(mu2)[:epochs], "epoch_ms": list(ems)[:epochs],
            "snapshots": snaps[:epochs] if snaps is not None else None}
    return w_out, info
