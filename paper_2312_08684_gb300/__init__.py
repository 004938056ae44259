"""GB300-native Stein-MAP-Seq (arXiv 2312.08684): MAP state-sequence estimation
by per-step Stein variational gradient descent over particle sets plus a
Viterbi max-plus recursion, on hand-written sm_103a CUDA behind a C ABI
(include/smap.h).

``_binding`` mirrors the C calls one to one; ``Estimator`` bundles a handle
with a workload description. Neither does any arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

from . import _binding as abi
from ._binding import SmapError, load  # noqa: F401


class Estimator:
    """One smap handle: B sequences, N particles, L SVGD iterations per step."""

    def __init__(self, kind, params, N, L, step, x0, max_T, bw_rule=0, bw_value=1.0, prior=0,
                 seed=1, stream=None, kernel=0):
        x0 = np.ascontiguousarray(x0, np.float64)
        self.B = int(x0.shape[0])
        self.N, self.L, self.max_T = int(N), int(L), int(max_T)
        self.h = abi.smap_create(kind, params, N, L, step, bw_rule, bw_value, prior, seed, self.B,
                                 max_T, x0, stream, kernel)
        self.d, self.dy = abi.smap_dims(self.h)

    @classmethod
    def from_workload(cls, wl, stream=None, **over):
        kw = dict(kind=wl.kind, params=wl.params, N=wl.N, L=wl.L, step=wl.step, x0=wl.x0,
                  max_T=wl.maxT, bw_rule=wl.bw_rule, bw_value=wl.bw_value, prior=wl.prior,
                  seed=wl.seed, stream=stream, kernel=wl.kernel)
        kw.update(over)
        return cls(**kw)

    def close(self):
        if getattr(self, "h", None) is not None:
            abi.smap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- calls (see include/smap.h) ---
    def run_batch(self, y_all, T=None, Nseq=None, path=None, J=None):
        if path is None:
            path = np.empty((self.B, self.max_T + 1, self.d), np.float32)
            J = np.empty(self.B, np.float64)
        abi.smap_run_batch(self.h, y_all, T, Nseq, path, J)
        return path, J

    def pf_run_batch(self, y_all, T=None, Nseq=None, path=None, J=None):
        """PF-MAP-Seq over the batch: bootstrap-filter supports, same recursion."""
        if path is None:
            path = np.empty((self.B, self.max_T + 1, self.d), np.float32)
            J = np.empty(self.B, np.float64)
        abi.smap_pf_run_batch(self.h, y_all, T, Nseq, path, J)
        return path, J

    def step(self, y, active=None):
        abi.smap_step(self.h, y, active)

    def map_sequence(self, path=None, J=None):
        if path is None:
            path = np.empty((self.B, self.max_T + 1, self.d), np.float32)
            J = np.empty(self.B, np.float64)
        abi.smap_map_sequence(self.h, path, J)
        return path, J

    def reset(self, x0=None):
        abi.smap_reset(self.h, x0)

    def set_particle_counts(self, Nseq):
        abi.smap_set_particle_counts(self.h, Nseq)

    def history(self):
        out = np.empty((self.B, self.max_T, self.N, self.d), np.float32)
        abi.smap_get_history(self.h, out)
        return out

    def backpointers(self):
        out = np.empty((self.B, self.max_T, self.N), np.uint16)
        abi.smap_get_backpointers(self.h, out)
        return out

    def scores(self):
        out = np.empty((self.B, self.N), np.float64)
        abi.smap_get_scores(self.h, out)
        return out

    def viterbi(self, hist, y_all, T=None, Nseq=None):
        path = np.empty((self.B, self.max_T + 1, self.d), np.float32)
        J = np.empty(self.B, np.float64)
        psi = np.empty((self.B, self.max_T, self.N), np.uint16)
        abi.smap_viterbi(self.h, hist, y_all, T, Nseq, path, J, psi)
        return path, J, psi

    def debug_svgd(self, t, x_prev, x_init, y, n_iters, phi_prev=None):
        return abi.smap_debug_svgd(self.h, t, x_prev, x_init, y, n_iters, phi_prev)

    def autotune(self, y_all, sample, steps):
        return abi.smap_autotune(self.h, y_all, sample, steps)

    def set_variant(self, v):
        abi.smap_set_variant(self.h, v)

    def variant(self):
        return abi.smap_get_variant(self.h)
