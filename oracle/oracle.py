"""Python access to the FP64 CPU oracle (``smap_oracle.c``).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
module. The product path (``paper_2312_08684_gb300``) never does.

Every function here is argument marshalling over the C library; the arithmetic
is in ``smap_oracle.c`` (plain double loops following Algorithms 1 and 2 of the
paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smap_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None

MODEL_NGM1D, MODEL_RANGE_CV2D, MODEL_CLUTTER_CV2D, MODEL_PLANAR_ARM, MODEL_LINEAR_GAUSS = 1, 2, 3, 4, 5
BW_MEDIAN_ITER, BW_MEDIAN_STEP, BW_FIXED = 0, 1, 2
PRIOR_MIXTURE, PRIOR_MEANGRAD, PRIOR_MAPCOND = 0, 1, 2

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U32 = ctypes.POINTER(ctypes.c_uint32)


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int), ("dy", ctypes.c_int),
                ("q", ctypes.c_double * 16), ("p", ctypes.c_double * 128), ("np", ctypes.c_int)]


class _RunCfg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("params", _D), ("np", ctypes.c_int),
                ("N", ctypes.c_int), ("L", ctypes.c_int), ("eps", ctypes.c_double),
                ("bw_rule", ctypes.c_int), ("bw_value", ctypes.c_double),
                ("prior", ctypes.c_int), ("seed", ctypes.c_uint64), ("kernel", ctypes.c_int)]

# Stein kernels of the oracle (om_kernel): 0 RBF, 1 IMQ, 2 Matern 3/2
KERNEL_RBF, KERNEL_IMQ, KERNEL_MATERN32 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(_Model)
            L.om_setup.argtypes = [P, ctypes.c_int, _D, ctypes.c_int]
            L.om_transition.argtypes = [P, ctypes.c_int, _D, _D]
            L.om_loglik.argtypes = [P, ctypes.c_int, _D, _D]
            L.om_loglik.restype = ctypes.c_double
            L.om_grad_loglik.argtypes = [P, ctypes.c_int, _D, _D, _D]
            L.om_logtrans.argtypes = [P, _D, _D]
            L.om_logtrans.restype = ctypes.c_double
            L.om_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.om_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_int, _D]
            L.om_median_sqdist.argtypes = [_D, ctypes.c_int, ctypes.c_int]
            L.om_median_sqdist.restype = ctypes.c_double
            L.om_bandwidth.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.om_bandwidth.restype = ctypes.c_double
            L.om_grad_prior.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D]
            L.om_svgd_iteration.argtypes = [P, ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_int,
                                            _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int]
            L.om_svgd_iters.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        _D, _D, _D, ctypes.c_int, _D, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _D, ctypes.c_int]
            L.om_forward.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, ctypes.c_int,
                                     _I, _D]
            L.om_backtrack.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _I, _D,
                                       _D, _I]
            L.om_backtrack.restype = ctypes.c_double
            L.om_path_score.argtypes = [P, ctypes.c_int, _D, _D]
            L.om_path_score.restype = ctypes.c_double
            L.om_run_sequence.argtypes = [ctypes.POINTER(_RunCfg), ctypes.c_uint32, _D, ctypes.c_int,
                                          _D, _D, _I, _D, _D]
            L.om_viterbi_sets.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _D, _D, _D, _I, _D, _D, _D]
            L.om_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            L.om_uniform.restype = ctypes.c_double
            L.om_pf_sets.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint32, _D, _D, _D, _I]
            L.om_viterbi_margins.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _D, _D, _D, _D]
            L.om_mlp_nparams.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.om_mlp_nparams.restype = ctypes.c_long
            L.om_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_long, _D, _D]
            L.om_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_long, _D, _D, _D]
            L.om_mlp_loss_grad.restype = ctypes.c_double
            L.om_adam.argtypes = [ctypes.c_long, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double]
            L.om_proposal_features.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _D, _D]
            L.om_run_batch.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_uint64, ctypes.c_int, _I, _D, ctypes.c_int, _I, _D,
                                       _D, _D, ctypes.c_int, ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Model:
    """A scenario model as the oracle sees it (kind + parameter vector)."""

    def __init__(self, kind: int, params):
        self.kind = int(kind)
        self.params = _f64(params).ravel()
        self._m = _Model()
        rc = lib().om_setup(ctypes.byref(self._m), self.kind, _dp(self.params), len(self.params))
        if rc != 0:
            raise ValueError(f"oracle: bad model kind={kind} params={list(self.params)}")
        self.d = self._m.d
        self.dy = self._m.dy
        self.q = np.array(self._m.q[: self.d])

    @property
    def ref(self):
        return ctypes.byref(self._m)

    def transition(self, t, x):
        x = _f64(x); f = np.empty(self.d)
        lib().om_transition(self.ref, int(t), _dp(x), _dp(f))
        return f

    def loglik(self, t, z, x):
        z = _f64(z); x = _f64(x)
        return lib().om_loglik(self.ref, int(t), _dp(z), _dp(x))

    def grad_loglik(self, t, z, x):
        z = _f64(z); x = _f64(x); g = np.empty(self.d)
        lib().om_grad_loglik(self.ref, int(t), _dp(z), _dp(x), _dp(g))
        return g

    def logtrans(self, x, f):
        x = _f64(x); f = _f64(f)
        return lib().om_logtrans(self.ref, _dp(x), _dp(f))

    @staticmethod
    def _phi(phiprev, Np):
        """The previous step's scores phi_{t-1} (MAP-conditioned prior); None = zeros."""
        return _f64(np.zeros(Np) if phiprev is None else phiprev).reshape(Np)

    def grad_prior(self, prior, fprev, x, phiprev=None):
        fprev = _f64(fprev).reshape(-1, self.d); x = _f64(x); g = np.empty(self.d)
        ph = self._phi(phiprev, fprev.shape[0])
        lib().om_grad_prior(self.ref, int(prior), _dp(fprev), _dp(ph), fprev.shape[0], _dp(x), _dp(g))
        return g

    def svgd_iteration(self, prior, t, z, fprev, x, h, eps, kernel=KERNEL_RBF, phiprev=None):
        fprev = _f64(fprev).reshape(-1, self.d); x = _f64(x).reshape(-1, self.d).copy(); z = _f64(z)
        ph = self._phi(phiprev, fprev.shape[0])
        lib().om_svgd_iteration(self.ref, int(prior), int(t), _dp(z), _dp(fprev), _dp(ph), fprev.shape[0],
                                _dp(x), x.shape[0], float(h), float(eps), int(kernel))
        return x

    def svgd_iters(self, prior, bw_rule, bw_value, t, z, fprev, x, L, eps, kernel=KERNEL_RBF, phiprev=None):
        """L SVGD iterations from x (given f_t of the previous set and, for the
        MAP-conditioned prior, its scores phi_{t-1}). Returns (x, h[L])."""
        fprev = _f64(fprev).reshape(-1, self.d); x = _f64(x).reshape(-1, self.d).copy(); z = _f64(z)
        ph = self._phi(phiprev, fprev.shape[0])
        h = np.empty(max(int(L), 1))
        lib().om_svgd_iters(self.ref, int(prior), int(bw_rule), float(bw_value), int(t), _dp(z),
                            _dp(fprev), _dp(ph), fprev.shape[0], _dp(x), x.shape[0], int(L), float(eps), _dp(h),
                            int(kernel))
        return x, h[: int(L)]

    def forward(self, t, z, fprev, phi_prev, x):
        fprev = _f64(fprev).reshape(-1, self.d); x = _f64(x).reshape(-1, self.d); z = _f64(z)
        phi_prev = _f64(phi_prev)
        N = x.shape[0]
        psi = np.empty(N, dtype=np.int32); phi = np.empty(N)
        lib().om_forward(self.ref, int(t), _dp(z), _dp(fprev), fprev.shape[0], _dp(phi_prev),
                         _dp(x), N, _ip(psi), _dp(phi))
        return psi, phi

    def path_score(self, path, z):
        path = _f64(path).reshape(-1, self.d); z = _f64(z).reshape(-1, self.dy)
        return lib().om_path_score(self.ref, path.shape[0] - 1, _dp(path), _dp(z))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty(4, dtype=np.uint32)
    lib().om_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def normals(seed, seq, t, i, d):
    z = np.empty(d)
    lib().om_normals(ctypes.c_uint64(int(seed)), int(seq), int(t), int(i), int(d), _dp(z))
    return z


def median_sqdist(x):
    x = _f64(x)
    x = x.reshape(x.shape[0], -1)
    return lib().om_median_sqdist(_dp(x), x.shape[0], x.shape[1])


def bandwidth(x, scale=1.0):
    x = _f64(x)
    x = x.reshape(x.shape[0], -1)
    return lib().om_bandwidth(_dp(x), x.shape[0], x.shape[1], float(scale))


def backtrack(x0, hist, psi, phiT):
    hist = _f64(hist); T, N, d = hist.shape
    x0 = _f64(x0); psi = np.ascontiguousarray(np.asarray(psi, dtype=np.int32)); phiT = _f64(phiT)
    path = np.empty((T + 1, d)); idx = np.empty(T, dtype=np.int32)
    J = lib().om_backtrack(d, N, T, _dp(x0), _dp(hist), _ip(psi), _dp(phiT), _dp(path), _ip(idx))
    return path, idx, J


def run_sequence(kind, params, N, L, eps, bw_rule, bw_value, prior, seed, seq, x0, z, T=None,
                 kernel=KERNEL_RBF):
    """Algorithm 2 on one sequence. Returns dict(hist[T][N][d], psi[T][N], path[T+1][d], J)."""
    m = Model(kind, params)
    z = _f64(z).reshape(-1, m.dy)
    T = z.shape[0] if T is None else int(T)
    z = np.ascontiguousarray(z[:T])
    params = m.params
    cfg = _RunCfg(m.kind, _dp(params), len(params), int(N), int(L), float(eps), int(bw_rule),
                  float(bw_value), int(prior), ctypes.c_uint64(int(seed)), int(kernel))
    x0 = _f64(x0)
    hist = np.empty((T, int(N), m.d)); psi = np.empty((T, int(N)), dtype=np.int32)
    path = np.empty((T + 1, m.d)); J = ctypes.c_double()
    rc = lib().om_run_sequence(ctypes.byref(cfg), int(seq), _dp(x0), T, _dp(z), _dp(hist),
                               _ip(psi), _dp(path), ctypes.byref(J))
    if rc != 0:
        raise ValueError("oracle: run_sequence rejected its input")
    return {"hist": hist, "psi": psi, "path": path, "J": J.value}


def viterbi_sets(kind, params, x0, hist, z):
    """Forward recursion + backtracking over fixed particle sets hist[T][N][d]."""
    m = Model(kind, params)
    hist = _f64(hist); T, N, d = hist.shape
    z = _f64(z).reshape(-1, m.dy)[:T].copy()
    x0 = _f64(x0)
    psi = np.empty((T, N), dtype=np.int32); phiT = np.empty(N); path = np.empty((T + 1, d))
    J = ctypes.c_double()
    rc = lib().om_viterbi_sets(m.kind, _dp(m.params), len(m.params), N, T, _dp(x0), _dp(hist),
                               _dp(z), _ip(psi), _dp(phiT), _dp(path), ctypes.byref(J))
    if rc != 0:
        raise ValueError("oracle: viterbi_sets rejected its input")
    return {"psi": psi, "phiT": phiT, "path": path, "J": J.value}


def uniform(seed, seq, t, i):
    """U_i of the stratified resampling: (w0 + 1/2) / 2^32, Philox counter (i, t, seq, 256)."""
    return lib().om_uniform(ctypes.c_uint64(seed), seq, t, i)


def pf_sets(kind, params, N, seed, seq, x0, z):
    """Bootstrap particle filter with stratified resampling at every step (the
    supports of PF-MAP-Seq): hist [T][N][d] and ancestors [T][N]."""
    m = Model(kind, params)
    z = _f64(z).reshape(-1, m.dy).copy()
    T = z.shape[0]
    x0 = _f64(x0)
    hist = np.empty((T, N, m.d)); anc = np.empty((T, N), dtype=np.int32)
    rc = lib().om_pf_sets(m.kind, _dp(m.params), len(m.params), N, T, ctypes.c_uint64(seed), seq, _dp(x0),
                          _dp(z), _dp(hist), _ip(anc))
    if rc != 0:
        raise ValueError("oracle: pf_sets rejected its input")
    return hist, anc


def pf_map_sequence(kind, params, N, seed, seq, x0, z):
    """PF-MAP-Seq: the particle filter's sets, then the forward recursion and
    backtracking over them."""
    hist, anc = pf_sets(kind, params, N, seed, seq, x0, z)
    res = viterbi_sets(kind, params, x0, hist, z)
    res["hist"] = hist
    res["anc"] = anc
    return res


def viterbi_margins(kind, params, x0, hist, z):
    """Relative margin (best - second) / max(1, |best|) of every backpointer, [T][N]."""
    m = Model(kind, params)
    hist = _f64(hist); T, N, d = hist.shape
    z = _f64(z).reshape(-1, m.dy)[:T].copy()
    x0 = _f64(x0)
    out = np.empty((T, N))
    rc = lib().om_viterbi_margins(m.kind, _dp(m.params), len(m.params), N, T, _dp(x0), _dp(hist),
                                  _dp(z), _dp(out))
    if rc != 0:
        raise ValueError("oracle: viterbi_margins rejected its input")
    return out


def mlp_nparams(n_in, H, n_out):
    return int(lib().om_mlp_nparams(n_in, H, n_out))


def mlp_forward(n_in, H, n_out, W, X):
    """3-layer GELU perceptron, packed W = [W1, b1, W2, b2, W3, b3]."""
    W = _f64(W); X = _f64(X).reshape(-1, n_in)
    Y = np.empty((X.shape[0], n_out))
    lib().om_mlp_forward(n_in, H, n_out, _dp(W), X.shape[0], _dp(X), _dp(Y))
    return Y


def mlp_loss_grad(n_in, H, n_out, W, X, Tg):
    """(loss, gradient): mean squared error over rows and outputs."""
    W = _f64(W); X = _f64(X).reshape(-1, n_in); Tg = _f64(Tg).reshape(-1, n_out)
    G = np.empty_like(W)
    loss = lib().om_mlp_loss_grad(n_in, H, n_out, _dp(W), X.shape[0], _dp(X), _dp(Tg), _dp(G))
    return loss, G


def adam(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays."""
    for a in (theta, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().om_adam(len(theta), _dp(theta), _dp(g), _dp(m), _dp(v), int(t), float(lr), beta1, beta2, eps)


def proposal_features(kind, params, u, z):
    params = _f64(params); u = _f64(u); z = _f64(z)
    f = np.zeros(32)
    n = lib().om_proposal_features(int(kind), _dp(params), len(params), _dp(u), _dp(z), _dp(f))
    if n < 0:
        raise ValueError("oracle: bad model")
    return f[:n]


def run_batch(kind, params, N, L, eps, bw_rule, bw_value, prior, seed, seq_ids, x0, z, T,
              nthreads=None, kernel=KERNEL_RBF):
    """Algorithm 2 on many sequences over host threads. z is [B][maxT][dy]."""
    m = Model(kind, params)
    seq_ids = np.ascontiguousarray(np.asarray(seq_ids, dtype=np.int32))
    B = len(seq_ids)
    z = _f64(z).reshape(B, -1, m.dy)
    maxT = z.shape[1]
    T = np.ascontiguousarray(np.asarray(T, dtype=np.int32))
    x0 = _f64(x0).reshape(B, m.d)
    path = np.full((B, maxT + 1, m.d), np.nan); J = np.empty(B)
    nthreads = os.cpu_count() if nthreads is None else int(nthreads)
    rc = lib().om_run_batch(m.kind, _dp(m.params), len(m.params), int(N), int(L), float(eps),
                            int(bw_rule), float(bw_value), int(prior), ctypes.c_uint64(int(seed)),
                            B, _ip(seq_ids), _dp(x0), maxT, _ip(T), _dp(z), _dp(path), _dp(J),
                            nthreads, int(kernel))
    if rc != 0:
        raise ValueError("oracle: run_batch rejected its input")
    return {"path": path, "J": J, "threads": min(max(nthreads, 1), 256)}
