"""ctypes binding of libsmap (include/smap.h): argument marshalling only.

Every function keeps the C name. Array arguments accept numpy arrays (host
memory, on_device = 0) or CUDA torch tensors (device memory, on_device = 1);
one call must not mix the two. All arithmetic happens in the CUDA library:
if it is not built this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# SMAP_LIBRARY may name another build of the library (the bounds-checked
# debug build, paper_2312_08684_gb300/_build_debug/libsmap_debug.so).
LIB_PATH = os.environ.get("SMAP_LIBRARY") or os.path.join(_PKG, "_build", "libsmap.so")

SMAP_OK, SMAP_E_INVAL, SMAP_E_NOMEM, SMAP_E_CUDA, SMAP_E_STATE, SMAP_E_TIMEOUT, \
    SMAP_E_NONFINITE, SMAP_E_UNSUPPORTED = range(8)
SMAP_MODEL_NGM1D, SMAP_MODEL_RANGE_CV2D, SMAP_MODEL_CLUTTER_CV2D, SMAP_MODEL_PLANAR_ARM, \
    SMAP_MODEL_LINEAR_GAUSS = 1, 2, 3, 4, 5
SMAP_BW_MEDIAN_ITER, SMAP_BW_MEDIAN_STEP, SMAP_BW_FIXED = 0, 1, 2
SMAP_PRIOR_MIXTURE, SMAP_PRIOR_MEANGRAD, SMAP_PRIOR_MAPCOND = 0, 1, 2

# Every symbol include/smap.h declares (the CPU tests check the library exports them).
EXPORTS = [
    "smap_create", "smap_destroy", "smap_dims", "smap_reset", "smap_set_particle_counts",
    "smap_step", "smap_map_sequence", "smap_run_batch", "smap_get_history",
    "smap_get_backpointers", "smap_get_scores", "smap_get_steps", "smap_viterbi",
    "smap_autotune", "smap_set_variant", "smap_num_variants", "smap_variant_info",
    "smap_get_variant", "smap_debug_svgd", "smap_debug_philox", "smap_debug_normals",
    "smap_kernel_launches", "smap_status_string", "smap_last_error", "smap_last_kernel_ms",
    "smap_viterbi_noalloc", "smap_debug_median_stats",
    "smap_proposal_create", "smap_proposal_destroy", "smap_proposal_dims", "smap_proposal_get_weights",
    "smap_proposal_set_weights", "smap_proposal_fit_normalization", "smap_proposal_forward",
    "smap_proposal_loss_grad", "smap_proposal_train", "smap_proposal_last_error", "smap_proposal_capture",
    "smap_set_proposal", "smap_pf_run_batch", "smap_debug_proposal_forward", "smap_debug_record_learned_init",
    "smap_state_size", "smap_save", "smap_load", "smap_debug_df", "smap_debug_bounds_probe",
    "smap_debug_recursion_stats",
]
MLP_IN_P, MLP_OUT_P, MLP_H = 32, 16, 256


class SmapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"smap status {status}: {msg}")
        self.status = status


class smap_config(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int),
        ("N", ctypes.c_int), ("L", ctypes.c_int), ("step", ctypes.c_double),
        ("bw_rule", ctypes.c_int), ("bw_value", ctypes.c_double), ("prior", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("batch", ctypes.c_int), ("max_T", ctypes.c_int),
        ("x0", ctypes.POINTER(ctypes.c_double)), ("stream", ctypes.c_void_p), ("kernel", ctypes.c_int),
    ]


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int


def load():
    """Loads libsmap.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsmap.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                           "or python paper_2312_08684_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    L.smap_create.argtypes = [ctypes.POINTER(smap_config), ctypes.POINTER(_VP)]
    L.smap_create.restype = st
    L.smap_destroy.argtypes = [_VP]
    L.smap_destroy.restype = None
    L.smap_dims.argtypes = [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.smap_reset.argtypes = [_VP, _VP]
    L.smap_set_particle_counts.argtypes = [_VP, _VP]
    L.smap_step.argtypes = [_VP, _VP, _VP, _I]
    L.smap_map_sequence.argtypes = [_VP, _VP, _VP, _I]
    L.smap_run_batch.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _I]
    L.smap_pf_run_batch.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _I]
    L.smap_get_history.argtypes = [_VP, _VP, _I]
    L.smap_get_backpointers.argtypes = [_VP, _VP, _I]
    L.smap_get_scores.argtypes = [_VP, _VP, _I]
    L.smap_get_steps.argtypes = [_VP, _VP]
    L.smap_viterbi.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I]
    L.smap_autotune.argtypes = [_VP, _VP, _I, _I, _I, ctypes.POINTER(_I), _VP, _I]
    L.smap_set_variant.argtypes = [_VP, _I]
    L.smap_num_variants.argtypes = []
    L.smap_variant_info.argtypes = [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.smap_get_variant.argtypes = [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.smap_debug_svgd.argtypes = [_VP, _I, _VP, _I, _VP, _VP, _I, _VP, _VP, _VP]
    u32 = ctypes.c_uint32
    L.smap_debug_philox.argtypes = [u32, u32, u32, u32, u32, u32, _I, _VP]
    L.smap_debug_normals.argtypes = [ctypes.c_uint64, u32, u32, u32, _I, _I, _VP]
    L.smap_last_kernel_ms.argtypes = [_VP, _VP, _VP]
    L.smap_debug_median_stats.argtypes = [_VP, _VP]
    L.smap_proposal_create.argtypes = [_I, ctypes.POINTER(ctypes.c_double), _I, ctypes.c_uint64, _VP,
                                       ctypes.POINTER(_VP)]
    L.smap_proposal_destroy.argtypes = [_VP]
    L.smap_proposal_destroy.restype = None
    L.smap_proposal_dims.argtypes = [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                     ctypes.POINTER(ctypes.c_long)]
    L.smap_proposal_get_weights.argtypes = [_VP, _VP, _VP]
    L.smap_proposal_set_weights.argtypes = [_VP, _VP, _VP]
    L.smap_proposal_fit_normalization.argtypes = [_VP, _VP, _VP, ctypes.c_long]
    L.smap_proposal_forward.argtypes = [_VP, _VP, ctypes.c_long, _VP]
    L.smap_proposal_loss_grad.argtypes = [_VP, _VP, _VP, ctypes.c_long, _VP, _VP]
    L.smap_proposal_train.argtypes = [_VP, _VP, _VP, ctypes.c_long, _I, _I, ctypes.c_double, ctypes.c_double,
                                      _VP]
    L.smap_proposal_last_error.argtypes = [_VP]
    L.smap_proposal_last_error.restype = ctypes.c_char_p
    L.smap_proposal_capture.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    L.smap_set_proposal.argtypes = [_VP, _VP, _I]
    L.smap_debug_proposal_forward.argtypes = [_VP, _VP, ctypes.c_long, _VP, ctypes.c_uint64, _I]
    L.smap_debug_record_learned_init.argtypes = [_VP, _VP]
    L.smap_state_size.argtypes = [_VP, ctypes.POINTER(ctypes.c_size_t)]
    L.smap_debug_df.argtypes = [_I, _VP, _I, _VP]
    L.smap_debug_recursion_stats.argtypes = [_VP, _VP]
    L.smap_debug_bounds_probe.argtypes = [_I, _I, _VP, _VP, _VP]
    L.smap_save.argtypes = [_VP, _VP, ctypes.c_size_t]
    L.smap_load.argtypes = [_VP, _VP, ctypes.c_size_t]
    L.smap_viterbi_noalloc.argtypes = [_I, ctypes.POINTER(ctypes.c_double), _I, _I, _I, _I,
                                       _VP, _VP, _VP, _VP, _VP, _VP]
    L.smap_kernel_launches.argtypes = []
    L.smap_kernel_launches.restype = ctypes.c_uint64
    L.smap_status_string.argtypes = [_I]
    L.smap_status_string.restype = ctypes.c_char_p
    L.smap_last_error.argtypes = [_VP]
    L.smap_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, dtype, writable=False):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
               np.uint16: torch.uint16 if hasattr(torch, "uint16") else torch.int16,
               np.uint8: torch.uint8}[dtype]
        if a.dtype != tdt and not (dtype == np.uint16 and a.dtype == torch.int16):
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags.c_contiguous:
        if writable:
            raise TypeError(f"output array must be C-contiguous {np.dtype(dtype)}")
        arr = np.ascontiguousarray(arr, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def _check(st, h=None):
    if st != SMAP_OK:
        L = load()
        msg = L.smap_last_error(h).decode() if h else L.smap_status_string(st).decode()
        raise SmapError(st, msg or L.smap_status_string(st).decode())


def _same_side(*flags):
    f = [x for x in flags if x is not None]
    if f and any(x != f[0] for x in f):
        raise ValueError("one call must not mix host arrays and device tensors")
    return f[0] if f else 0


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))


# ---------------------------------------------------------------- calls ----
def smap_create(model, params, N, L, step, bw_rule, bw_value, prior, seed, batch, max_T, x0,
                stream=None, kernel=0):
    lib = load()
    params = np.ascontiguousarray(params, dtype=np.float64).ravel()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    cfg = smap_config(int(model), params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(params),
                      int(N), int(L), float(step), int(bw_rule), float(bw_value), int(prior),
                      ctypes.c_uint64(int(seed)), int(batch), int(max_T),
                      x0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream), int(kernel))
    h = ctypes.c_void_p()
    st = lib.smap_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != SMAP_OK:
        raise SmapError(st, lib.smap_status_string(st).decode())
    return h


def smap_destroy(h):
    load().smap_destroy(h)


def smap_dims(h):
    d, dy = ctypes.c_int(), ctypes.c_int()
    _check(load().smap_dims(h, ctypes.byref(d), ctypes.byref(dy)), h)
    return d.value, dy.value


def smap_reset(h, x0=None):
    p, _, keep = _arg(x0, np.float64)
    _check(load().smap_reset(h, p), h)


def smap_set_particle_counts(h, N_per_seq=None):
    p, _, keep = _arg(N_per_seq, np.int32)
    _check(load().smap_set_particle_counts(h, p), h)


def smap_step(h, y, active=None):
    py, dev, k1 = _arg(y, np.float32)
    pa, _, k2 = _arg(None if active is None else np.asarray(active, np.uint8), np.uint8)
    _check(load().smap_step(h, py, pa, dev), h)


def smap_map_sequence(h, path=None, J=None):
    pp, d1, k1 = _arg(path, np.float32, True)
    pj, d2, k2 = _arg(J, np.float64, True)
    _check(load().smap_map_sequence(h, pp, pj, _same_side(d1, d2)), h)


def smap_run_batch(h, y_all, T_per_seq=None, N_per_seq=None, path=None, J=None):
    py, d0, k0 = _arg(y_all, np.float32)
    pt, _, k1 = _arg(None if T_per_seq is None else np.asarray(T_per_seq, np.int32), np.int32)
    pn, _, k2 = _arg(None if N_per_seq is None else np.asarray(N_per_seq, np.int32), np.int32)
    pp, d3, k3 = _arg(path, np.float32, True)
    pj, d4, k4 = _arg(J, np.float64, True)
    _check(load().smap_run_batch(h, py, pt, pn, pp, pj, _same_side(d0, d3, d4)), h)


def smap_pf_run_batch(h, y_all, T_per_seq=None, N_per_seq=None, path=None, J=None):
    py, d0, k0 = _arg(y_all, np.float32)
    pt, _, k1 = _arg(None if T_per_seq is None else np.asarray(T_per_seq, np.int32), np.int32)
    pn, _, k2 = _arg(None if N_per_seq is None else np.asarray(N_per_seq, np.int32), np.int32)
    pp, d3, k3 = _arg(path, np.float32, True)
    pj, d4, k4 = _arg(J, np.float64, True)
    _check(load().smap_pf_run_batch(h, py, pt, pn, pp, pj, _same_side(d0, d3, d4)), h)


def smap_get_history(h, out):
    p, dev, keep = _arg(out, np.float32, True)
    _check(load().smap_get_history(h, p, dev), h)


def smap_get_backpointers(h, out):
    p, dev, keep = _arg(out, np.uint16, True)
    _check(load().smap_get_backpointers(h, p, dev), h)


def smap_get_scores(h, out):
    p, dev, keep = _arg(out, np.float64, True)
    _check(load().smap_get_scores(h, p, dev), h)


def smap_get_steps(h, out):
    p, _, keep = _arg(out, np.int32, True)
    _check(load().smap_get_steps(h, p), h)


def smap_viterbi(h, hist, y_all, T_per_seq=None, N_per_seq=None, path=None, J=None, psi=None):
    ph, d0, k0 = _arg(hist, np.float32)
    py, d1, k1 = _arg(y_all, np.float32)
    pt, _, k2 = _arg(None if T_per_seq is None else np.asarray(T_per_seq, np.int32), np.int32)
    pn, _, k3 = _arg(None if N_per_seq is None else np.asarray(N_per_seq, np.int32), np.int32)
    pp, d4, k4 = _arg(path, np.float32, True)
    pj, d5, k5 = _arg(J, np.float64, True)
    ps, d6, k6 = _arg(psi, np.uint16, True)
    _check(load().smap_viterbi(h, ph, py, pt, pn, pp, pj, ps, _same_side(d0, d1, d4, d5, d6)), h)


def smap_viterbi_noalloc(model, params, x0, hist, y, path, J, stream=None):
    """The dynamic programme without device allocation. x0, hist, y, path, J
    must be CUDA tensors (shapes as in include/smap.h); asynchronous on stream."""
    params = np.ascontiguousarray(params, dtype=np.float64).ravel()
    B, T, N, _ = hist.shape
    ptrs = []
    for a, dt in ((x0, np.float64), (hist, np.float32), (y, np.float32), (path, np.float32),
                  (J, np.float64)):
        p, dev, _ = _arg(a, dt, True)
        if dev != 1:
            raise ValueError("smap_viterbi_noalloc takes device tensors only")
        ptrs.append(p)
    _check(load().smap_viterbi_noalloc(int(model), params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       len(params), int(B), int(N), int(T), *ptrs, _stream_ptr(stream)))


def smap_autotune(h, y_all, sample, steps):
    py, dev, keep = _arg(y_all, np.float32)
    n = smap_num_variants()
    ms = np.zeros(n, np.float32)
    chosen = ctypes.c_int()
    _check(load().smap_autotune(h, py, int(sample), int(steps), dev, ctypes.byref(chosen),
                                ctypes.c_void_p(ms.ctypes.data), n), h)
    return chosen.value, ms


def smap_set_variant(h, v):
    _check(load().smap_set_variant(h, int(v)), h)


def smap_num_variants():
    return int(load().smap_num_variants())


def smap_variant_info(v):
    """(particles per thread, block-size bound, threads per particle)."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().smap_variant_info(int(v), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def smap_get_variant(h):
    v, t, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().smap_get_variant(h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(g)), h)
    return v.value, t.value, g.value


def smap_debug_svgd(h, t, x_prev, x_init, y, n_iters, phi_prev=None):
    x_prev = np.ascontiguousarray(x_prev, np.float32)
    x_init = np.ascontiguousarray(x_init, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    ph = None if phi_prev is None else np.ascontiguousarray(phi_prev, np.float64)
    x_out = np.empty_like(x_init)
    h_out = np.empty((x_init.shape[0], max(int(n_iters), 1)), np.float32)
    _check(load().smap_debug_svgd(h, int(t), ctypes.c_void_p(x_prev.ctypes.data), int(x_prev.shape[1]),
                                  ctypes.c_void_p(x_init.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                  int(n_iters), ctypes.c_void_p(x_out.ctypes.data),
                                  ctypes.c_void_p(h_out.ctypes.data),
                                  None if ph is None else ctypes.c_void_p(ph.ctypes.data)), h)
    return x_out, h_out[:, : int(n_iters)]


def smap_debug_philox(c0, c1, c2, c3, key0, key1, n):
    out = np.empty((int(n), 4), np.uint32)
    _check(load().smap_debug_philox(c0, c1, c2, c3, key0, key1, int(n), ctypes.c_void_p(out.ctypes.data)))
    return out


def smap_debug_normals(seed, seq, t, i0, n, d):
    out = np.empty((int(n), int(d)), np.float32)
    _check(load().smap_debug_normals(ctypes.c_uint64(int(seed)), int(seq), int(t), int(i0), int(n),
                                     int(d), ctypes.c_void_p(out.ctypes.data)))
    return out


def smap_debug_bounds_probe(rows, index):
    """Debug build only: (value loaded, failed-check code, index) of one checked row load."""
    v = np.zeros(1, np.float32)
    c = np.zeros(2, np.int32)
    _check(load().smap_debug_bounds_probe(int(rows), int(index), ctypes.c_void_p(v.ctypes.data),
                                          ctypes.c_void_p(c.ctypes.data), ctypes.c_void_p(c[1:].ctypes.data)))
    return float(v[0]), int(c[0]), int(c[1])


def smap_debug_recursion_stats(h):
    """(particle-steps, near-ties, exact candidate scores) since the last read; reading resets them."""
    out = np.zeros(3, np.uint64)
    _check(load().smap_debug_recursion_stats(h, ctypes.c_void_p(out.ctypes.data)), h)
    return tuple(int(v) for v in out)


def smap_debug_df(fn, x):
    """Double-float exp (0), log (1) or sqrt (2) of float64 inputs, on the device."""
    x = np.ascontiguousarray(x, np.float64).ravel()
    out = np.empty_like(x)
    _check(load().smap_debug_df(int(fn), ctypes.c_void_p(x.ctypes.data), len(x), ctypes.c_void_p(out.ctypes.data)))
    return out


def smap_last_kernel_ms(h):
    """(step-kernel ms, whole batched device work ms) of the last smap_run_batch."""
    a = np.zeros(1, np.float32)
    b = np.zeros(1, np.float32)
    _check(load().smap_last_kernel_ms(h, ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data)), h)
    return float(a[0]), float(b[0])


def smap_debug_median_stats(h):
    """(bracket hits, histogram locates, radix fallbacks, refined locates) since the last reset,
    batched run or debug SVGD call."""
    out = np.zeros(4, np.int32)
    _check(load().smap_debug_median_stats(h, ctypes.c_void_p(out.ctypes.data)), h)
    return tuple(int(v) for v in out)


# ------------------------------------------------------------- proposal ----
def _pcheck(st, p):
    if st != SMAP_OK:
        L = load()
        raise SmapError(st, L.smap_proposal_last_error(p).decode() or L.smap_status_string(st).decode())


def _dev(a, dtype):
    p, dev, _ = _arg(a, dtype, True)
    if dev != 1:
        raise ValueError("this call takes CUDA tensors")
    return p


def smap_proposal_create(model, params, seed=1, stream=None):
    params = np.ascontiguousarray(params, dtype=np.float64).ravel()
    p = ctypes.c_void_p()
    st = load().smap_proposal_create(int(model), params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     len(params), ctypes.c_uint64(int(seed)), _stream_ptr(stream), ctypes.byref(p))
    if st != SMAP_OK:
        raise SmapError(st, load().smap_status_string(st).decode())
    return p


def smap_proposal_destroy(p):
    load().smap_proposal_destroy(p)


def smap_proposal_dims(p):
    a, b, c, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
    _pcheck(load().smap_proposal_dims(p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)), p)
    return a.value, b.value, c.value, n.value


def smap_proposal_get_weights(p):
    n = smap_proposal_dims(p)[3]
    theta = np.empty(n, np.float32)
    norm = np.empty(2 * MLP_IN_P + 2 * MLP_OUT_P, np.float32)
    _pcheck(load().smap_proposal_get_weights(p, ctypes.c_void_p(theta.ctypes.data), ctypes.c_void_p(norm.ctypes.data)), p)
    return theta, norm


def smap_proposal_set_weights(p, theta=None, norm=None):
    t = None if theta is None else np.ascontiguousarray(theta, np.float32)
    n = None if norm is None else np.ascontiguousarray(norm, np.float32)
    _pcheck(load().smap_proposal_set_weights(p, None if t is None else ctypes.c_void_p(t.ctypes.data),
                                             None if n is None else ctypes.c_void_p(n.ctypes.data)), p)


def smap_proposal_fit_normalization(p, feat, targ):
    _pcheck(load().smap_proposal_fit_normalization(p, _dev(feat, np.float32), _dev(targ, np.float32),
                                                   int(feat.shape[0])), p)


def smap_proposal_forward(p, feat, disp):
    _pcheck(load().smap_proposal_forward(p, _dev(feat, np.float32), int(feat.shape[0]), _dev(disp, np.float32)), p)


def smap_debug_proposal_forward(p, feat, disp, wait_ns, stall=0):
    _pcheck(load().smap_debug_proposal_forward(p, _dev(feat, np.float32), int(feat.shape[0]),
                                               _dev(disp, np.float32), int(wait_ns), int(stall)), p)


def smap_proposal_loss_grad(p, feat, targ):
    n = smap_proposal_dims(p)[3]
    g = np.empty(n, np.float32)
    loss = ctypes.c_double()
    _pcheck(load().smap_proposal_loss_grad(p, _dev(feat, np.float32), _dev(targ, np.float32), int(feat.shape[0]),
                                           ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)), p)
    return loss.value, g


def smap_proposal_train(p, feat, targ, steps, batch, lr, lr_final):
    curve = np.empty(max(int(steps), 1), np.float32)
    _pcheck(load().smap_proposal_train(p, _dev(feat, np.float32), _dev(targ, np.float32), int(feat.shape[0]),
                                       int(steps), int(batch), float(lr), float(lr_final),
                                       ctypes.c_void_p(curve.ctypes.data)), p)
    return curve[: int(steps)]


def smap_proposal_last_error(p):
    return load().smap_proposal_last_error(p).decode()


def smap_proposal_capture(p, h, feat, targ):
    rows = ctypes.c_long()
    _check(load().smap_proposal_capture(p, h, _dev(feat, np.float32), _dev(targ, np.float32), int(feat.shape[0]),
                                        ctypes.byref(rows)), h)
    return rows.value


def smap_set_proposal(h, p, L_learned):
    _check(load().smap_set_proposal(h, p, int(L_learned)), h)


def smap_debug_record_learned_init(h, xinit_all=None):
    """xinit_all: CUDA tensor [B][max_T][N][d] float32, or None to stop recording."""
    ptr = None if xinit_all is None else _dev(xinit_all, np.float32)
    _check(load().smap_debug_record_learned_init(h, ptr), h)


def smap_state_size(h):
    n = ctypes.c_size_t()
    _check(load().smap_state_size(h, ctypes.byref(n)), h)
    return int(n.value)


def smap_save(h):
    """The handle's online state as a host byte array (see include/smap.h)."""
    buf = np.empty(smap_state_size(h), np.uint8)
    _check(load().smap_save(h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes), h)
    return buf


def smap_load(h, buf):
    buf = np.ascontiguousarray(buf, np.uint8)
    _check(load().smap_load(h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes), h)


def smap_kernel_launches():
    return int(load().smap_kernel_launches())


def smap_status_string(s):
    return load().smap_status_string(int(s)).decode()


def smap_last_error(h):
    return load().smap_last_error(h).decode()
