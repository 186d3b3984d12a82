"""Thin Python binding of libkcycle.so (the C ABI declared in include/kcycle.h).

Argument marshalling only: every step of the multigrid runs in the library's CUDA kernels.
Device arrays are torch CUDA tensors of dtype float64, shape (n, n), contiguous; torch is used
for device memory and streams only. The library must have been built (``build()`` in
``__graft_entry__`` or ``python -m paper_2010_00626_b300.build``); importing this module without
it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkcycle.so")

MG_OK, MG_NOT_CONVERGED = 0, 1
MG_KAPPA_W = 0x7FFFFFFF
CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy
MG_OPT_OMEGA, MG_OPT_COARSE_N, MG_OPT_LEVELS, MG_OPT_N, MG_OPT_LAUNCHES, MG_OPT_COARSE_N32 = 1, 2, 3, 4, 5, 6
MG_OPT_COARSE_OP, MG_OPT_STOP, MG_OPT_SMOOTHER, MG_OPT_COARSENING, MG_OPT_PRECOND = 7, 8, 9, 10, 11
MG_OPT_CONV_X, MG_OPT_CONV_Y, MG_OPT_FUSED_CALL, MG_OPT_TMA_PASSES, MG_OPT_CONDENSED_CHILDREN = 12, 13, 14, 15, 16
MG_OPT_TEST_STALL_COPY, MG_OPT_DEEP_CALLS, MG_OPT_TEST_STALL_BARRIER = 17, 18, 19
SMOOTHERS = {"jacobi": 0, "zebra": 1, "xzebra": 2}
COARSENINGS = {"full": 0, "y": 1}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libkcycle.so is not built ({LIB_PATH}); run python -m paper_2010_00626_b300.build")
_lib = ctypes.CDLL(LIB_PATH)

_h = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)

# every symbol declared in include/kcycle.h, with its signature
SIGNATURES = {
    "mg_setup": (_i, [_i, _d, _d, _i, _i, _i, ctypes.POINTER(_h)]),
    "mg_destroy": (_i, [_h]),
    "mg_set_option": (_i, [_h, _i, _d]),
    "mg_get_option": (_i, [_h, _i, _dp]),
    "mg_set_stream": (_i, [_h, _p]),
    "mg_kcycle": (_i, [_h, _p, _p, _i]),
    "mg_kcycle_adjoint": (_i, [_h, _p, _p, _i]),
    "mg_solve": (_i, [_h, _p, _p, _i, _d, _i, _ip, _dp, _dp]),
    "mg_solve_host": (_i, [_h, _p, _p, _i, _d, _i, _ip, _dp, _dp]),
    "mg_solve_adjoint": (_i, [_h, _p, _p, _i, _d, _i, _ip, _dp, _dp]),
    "mg_pcg": (_i, [_h, _p, _p, _i, _d, _i, _i, _ip, _dp, _dp]),
    "mg_pcg_mixed": (_i, [_h, _p, _p, _i, _d, _i, _i, _ip, _dp, _dp]),
    "mg_apply": (_i, [_h, _p, _p]),
    "mg_residual_norm": (_i, [_h, _p, _p, _dp]),
    "mg_param_grads": (_i, [_h, _p, _p, _dp, _dp]),
    "mg_stencils": (_i, [_h, _dp, _i, _ip]),
    "mg_counters": (_i, [_h, _i, _llp, _llp, _llp]),
    "mg_level_grid": (_i, [_h, _i, _i, _ip, _ip]),
    "mg_profile_cycle": (_i, [_h, _p, _p, _i, _i, _i, _dp, _ip, _ip, _ip]),
    "mg_residual_norm_noalloc": (_i, [_i, _d, _d, _p, _p, _p, _dp]),
    "mg_solve_mixed": (_i, [_h, _p, _p, _i, _d, _i, _ip, _dp, _dp]),
    "mg_kcycle_f32": (_i, [_h, _p, _p, _i]),
    "mg_batch_create": (_i, [_i, _ip, _dp, _dp, _ip, _i, _i, ctypes.POINTER(_h)]),
    "mg_batch_autotune": (_i, [_h, _i, _i, _ip]),
    "mg_batch_solve": (_i, [_h, ctypes.POINTER(_p), ctypes.POINTER(_p), _i, _d, _i, _i, _ip, _dp]),
    "mg_setup_batched": (_i, [_i, _ip, _dp, _dp, _i, _i, ctypes.POINTER(_h)]),
    "mg_solve_batched": (_i, [_h, ctypes.POINTER(_p), ctypes.POINTER(_p), _i, _d, _ip]),
    "mg_batch_set_option": (_i, [_h, _i, _d]),
    "mg_batch_instance": (_i, [_h, _i, ctypes.POINTER(_h)]),
    "mg_batch_size": (_i, [_h, _ip]),
    "mg_batch_destroy": (_i, [_h]),
    "mg_fp64_rate": (_i, [_dp]),
    "mg_status_string": (ctypes.c_char_p, [_i]),
    "mg_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class MultigridError(RuntimeError):
    pass


def fp64_rate():
    """Measured FP64 operations per second of the current device (mg_fp64_rate)."""
    out = ctypes.c_double()
    _check(_lib.mg_fp64_rate(ctypes.byref(out)), "mg_fp64_rate")
    return out.value


def _check(status: int, what: str) -> int:
    if status < 0:
        msg = _lib.mg_status_string(status).decode()
        detail = _lib.mg_last_error().decode()
        raise MultigridError(f"{what}: {msg} ({status}) {detail}")
    return status


def _dev(t, n, dtype="float64"):
    import torch
    want = getattr(torch, dtype)
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()
            and tuple(t.shape) == (n, n)):
        raise ValueError(f"expected a contiguous {dtype} CUDA tensor of shape ({n}, {n})")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, n, writable=False):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (n, n)):
        raise ValueError(f"expected a C-contiguous float64 array of shape ({n}, {n})")
    if writable and not a.flags.writeable:
        raise ValueError("array must be writable")
    return ctypes.c_void_p(a.ctypes.data)


class Multigrid:
    """One hierarchy for the Section 4 problem: ``mg_setup(n, eps, theta, levels, nu1, nu2)``."""

    def __init__(self, n, eps, theta, levels, nu1=2, nu2=2, omega=None, coarse_n=None, smoother="jacobi",
                 coarsening="full", convection=None, coarse_op=None):
        h = _h()
        _check(_lib.mg_setup(int(n), float(eps), float(theta), int(levels), int(nu1), int(nu2), ctypes.byref(h)),
               "mg_setup")
        self._h = h
        self.n, self.levels, self.eps, self.theta, self.nu1, self.nu2 = int(n), int(levels), eps, theta, nu1, nu2
        if omega is not None:
            self.set_option(MG_OPT_OMEGA, omega)
        if coarse_n is not None:
            self.set_option(MG_OPT_COARSE_N, coarse_n)
        if smoother not in SMOOTHERS or coarsening not in COARSENINGS:
            self.close()
            raise ValueError(f"smoother must be one of {sorted(SMOOTHERS)}, coarsening one of {sorted(COARSENINGS)}")
        if coarsening != "full":
            self.set_option(MG_OPT_COARSENING, COARSENINGS[coarsening])  # selects x-line zebra
        elif smoother != "jacobi":
            self.set_option(MG_OPT_SMOOTHER, SMOOTHERS[smoother])
        self.smoother, self.coarsening = smoother, coarsening
        if coarse_op is not None:
            self.set_option(MG_OPT_COARSE_OP, {"galerkin": 0, "rediscretized": 1}[coarse_op])
        if convection is not None:
            self.set_option(MG_OPT_CONV_X, convection[0])
            self.set_option(MG_OPT_CONV_Y, convection[1])

    @classmethod
    def _borrow(cls, handle, n, owner):
        """A Multigrid over a handle another object owns (a batch instance): close() releases nothing."""
        m = cls.__new__(cls)
        m._h, m._owner = handle, owner
        m.n = int(n)
        lv = ctypes.c_double()
        _check(_lib.mg_get_option(handle, MG_OPT_LEVELS, ctypes.byref(lv)), "mg_get_option")
        m.levels = int(lv.value)
        m.smoother, m.coarsening = None, "full"
        return m

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._h, self._owner = None, None
            return
        if getattr(self, "_h", None):
            _lib.mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------------- options / streams
    def set_option(self, key, value):
        _check(_lib.mg_set_option(self._h, int(key), float(value)), "mg_set_option")

    def get_option(self, key):
        out = _d()
        _check(_lib.mg_get_option(self._h, int(key), ctypes.byref(out)), "mg_get_option")
        return out.value

    def _stream(self):
        """Order the library's work on torch's current stream (the legacy default stream when
        torch reports handle 0, passed as cudaStreamLegacy)."""
        import torch
        s = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        _check(_lib.mg_set_stream(self._h, ctypes.c_void_p(s)), "mg_set_stream")

    # --------------------------------------------------------------------- cycles and solvers
    def kcycle(self, v, f, kappa):
        self._stream()
        _check(_lib.mg_kcycle(self._h, _dev(v, self.n), _dev(f, self.n), int(kappa)), "mg_kcycle")

    def kcycle_adjoint(self, v, f, kappa):
        self._stream()
        _check(_lib.mg_kcycle_adjoint(self._h, _dev(v, self.n), _dev(f, self.n), int(kappa)), "mg_kcycle_adjoint")

    def solve(self, v, f, kappa, tol, max_cycles, history=True, adjoint=False):
        """Returns (status, cycles, final_relres, history list); adjoint iterates the adjoint cycle."""
        self._stream()
        cyc, rel = _i(), _d()
        hist = np.zeros(max_cycles) if history else None
        fn = _lib.mg_solve_adjoint if adjoint else _lib.mg_solve
        st = _check(fn(self._h, _dev(v, self.n), _dev(f, self.n), int(kappa), float(tol), int(max_cycles),
                                  ctypes.byref(cyc), ctypes.byref(rel),
                                  hist.ctypes.data_as(_dp) if history else None), "mg_solve")
        return st, cyc.value, rel.value, (list(hist[:cyc.value]) if history else None)

    def solve_host(self, v, f, kappa, tol, max_cycles):
        """mg_solve_host on numpy arrays (v is updated in place). Returns (status, cycles, final_relres)."""
        cyc, rel = _i(), _d()
        st = _check(_lib.mg_solve_host(self._h, _host(v, self.n, True), _host(f, self.n), int(kappa), float(tol),
                                       int(max_cycles), ctypes.byref(cyc), ctypes.byref(rel), None),
                    "mg_solve_host")
        return st, cyc.value, rel.value

    def pcg(self, x, b, kappa, tol, max_iters, flexible=False, history=True, mixed=False):
        """MGCG (mixed: FP32 preconditioner cycles). Returns (status, iters, relres, history)."""
        self._stream()
        it, rel = _i(), _d()
        hist = np.zeros(max_iters) if history else None
        fn = _lib.mg_pcg_mixed if mixed else _lib.mg_pcg
        st = _check(fn(self._h, _dev(x, self.n), _dev(b, self.n), int(kappa), float(tol), int(max_iters),
                                int(bool(flexible)), ctypes.byref(it), ctypes.byref(rel),
                                hist.ctypes.data_as(_dp) if history else None), "mg_pcg")
        return st, it.value, rel.value, (list(hist[:it.value]) if history else None)

    def solve_mixed(self, x, f, kappa, tol, max_iters, history=True):
        """FP64 iterative refinement around FP32 kappa-cycles. Returns (status, iters, relres, history)."""
        self._stream()
        it, rel = _i(), _d()
        hist = np.zeros(max_iters) if history else None
        st = _check(_lib.mg_solve_mixed(self._h, _dev(x, self.n), _dev(f, self.n), int(kappa), float(tol),
                                        int(max_iters), ctypes.byref(it), ctypes.byref(rel),
                                        hist.ctypes.data_as(_dp) if history else None), "mg_solve_mixed")
        return st, it.value, rel.value, (list(hist[:it.value]) if history else None)

    def kcycle_f32(self, v, f, kappa):
        self._stream()
        _check(_lib.mg_kcycle_f32(self._h, _dev(v, self.n, "float32"), _dev(f, self.n, "float32"), int(kappa)),
               "mg_kcycle_f32")

    def apply(self, v, out):
        self._stream()
        _check(_lib.mg_apply(self._h, _dev(v, self.n), _dev(out, self.n)), "mg_apply")

    def residual_norm(self, v, f):
        self._stream()
        out = _d()
        _check(_lib.mg_residual_norm(self._h, _dev(v, self.n), _dev(f, self.n), ctypes.byref(out)),
               "mg_residual_norm")
        return out.value

    def param_grads(self, lam, u):
        self._stream()
        a, b = _d(), _d()
        _check(_lib.mg_param_grads(self._h, _dev(lam, self.n), _dev(u, self.n), ctypes.byref(a), ctypes.byref(b)),
               "mg_param_grads")
        return a.value, b.value

    def stencils(self):
        out = np.zeros(self.levels * 9)
        w = _i()
        _check(_lib.mg_stencils(self._h, out.ctypes.data_as(_dp), self.levels, ctypes.byref(w)), "mg_stencils")
        return out[: w.value * 9].reshape(w.value, 3, 3)

    def profile_cycle(self, v, f, kappa, with_norm=False, max_records=8192, fp32=False, graph=False):
        """Per-launch (ms, kind, level) of one cycle run launch by launch with CUDA events
        (fp32: the FP32 cycle of the mixed solve; graph: the launches and events replayed from a
        graph, as a solve runs them)."""
        self._stream()
        with_norm = int(bool(with_norm)) | (2 if fp32 else 0) | (4 if graph else 0)
        ms = np.zeros(max_records)
        kind = np.zeros(max_records, dtype=np.int32)
        level = np.zeros(max_records, dtype=np.int32)
        cnt = _i()
        _check(_lib.mg_profile_cycle(self._h, _dev(v, self.n), _dev(f, self.n), int(kappa), with_norm,
                                     max_records, ms.ctypes.data_as(_dp), kind.ctypes.data_as(_ip),
                                     level.ctypes.data_as(_ip), ctypes.byref(cnt)), "mg_profile_cycle")
        k = min(cnt.value, max_records)
        return ms[:k], kind[:k], level[:k]

    def level_grid(self, level, fp32=False):
        """(side of `level`, CTAs of one of its pass launches) in the FP64 or the FP32 cycle; 1 CTA
        for the levels inside the coarse-level kernel."""
        n, c = _i(), _i()
        _check(_lib.mg_level_grid(self._h, int(level), int(bool(fp32)), ctypes.byref(n), ctypes.byref(c)),
               "mg_level_grid")
        return n.value, c.value

    def counters(self, kappa):
        calls = (ctypes.c_longlong * self.levels)()
        lau, coarse = ctypes.c_longlong(), ctypes.c_longlong()
        _check(_lib.mg_counters(self._h, int(kappa), calls, ctypes.byref(lau), ctypes.byref(coarse)), "mg_counters")
        return list(calls), lau.value, coarse.value


class Batch:
    """Many independent instances solved by one graph launch (``mg_batch_*``)."""

    def __init__(self, ns, epss, thetas, nu1=2, nu2=2, levels=None, smoother="jacobi"):
        cnt = len(ns)
        h = _h()
        arr_i = (ctypes.c_int * cnt)(*[int(v) for v in ns])
        arr_e = (ctypes.c_double * cnt)(*[float(v) for v in epss])
        arr_t = (ctypes.c_double * cnt)(*[float(v) for v in thetas])
        arr_l = (ctypes.c_int * cnt)(*[int(v) for v in levels]) if levels is not None else None
        _check(_lib.mg_batch_create(cnt, arr_i, arr_e, arr_t, arr_l, int(nu1), int(nu2), ctypes.byref(h)),
               "mg_batch_create")
        self._h, self.ns = h, [int(v) for v in ns]
        if smoother not in SMOOTHERS:
            self.close()
            raise ValueError(f"smoother must be one of {sorted(SMOOTHERS)}")
        if smoother != "jacobi":
            self.set_option(MG_OPT_SMOOTHER, SMOOTHERS[smoother])

    def set_option(self, key, value):
        _check(_lib.mg_batch_set_option(self._h, int(key), float(value)), "mg_batch_set_option")

    def close(self):
        if getattr(self, "_h", None):
            _lib.mg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, kappa, mixed=False):
        """Returns {n: chosen coarse-kernel threshold}; shapes() gives every tuned option."""
        out = (ctypes.c_int * (2 * len(set(self.ns))))()
        _check(_lib.mg_batch_autotune(self._h, int(kappa), int(bool(mixed)), out), "mg_batch_autotune")
        return {out[2 * i]: out[2 * i + 1] for i in range(len(set(self.ns)))}

    def instance(self, index):
        """Instance `index` as a Multigrid that borrows the batch's handle (not destroyed by it)."""
        h = _h()
        _check(_lib.mg_batch_instance(self._h, int(index), ctypes.byref(h)), "mg_batch_instance")
        return Multigrid._borrow(h, self.ns[index], self)

    def shapes(self):
        """{n: {option: value}} of the first instance of each grid side (the autotuner sets every
        instance of a side alike)."""
        out = {}
        for i, n in enumerate(self.ns):
            if n in out:
                continue
            m = self.instance(i)
            out[n] = {"coarse_n": int(m.get_option(MG_OPT_COARSE_N)), "coarse_n32": int(m.get_option(MG_OPT_COARSE_N32)),
                      "fused_call": int(m.get_option(MG_OPT_FUSED_CALL)),
                      "condensed_children": int(m.get_option(MG_OPT_CONDENSED_CHILDREN)),
                      "tma_passes": int(m.get_option(MG_OPT_TMA_PASSES))}
        return out

    def solve(self, xs, fs, kappa, tol, max_iters, mixed=False):
        """xs, fs: lists of float64 CUDA tensors (n_i, n_i). Returns (status, iters list, relres list)."""
        import torch
        cnt = len(self.ns)
        px = (ctypes.c_void_p * cnt)(*[_dev(x, n).value for x, n in zip(xs, self.ns)])
        pf = (ctypes.c_void_p * cnt)(*[_dev(f, n).value for f, n in zip(fs, self.ns)])
        it = (ctypes.c_int * cnt)()
        rel = (ctypes.c_double * cnt)()
        torch.cuda.synchronize()
        st = _check(_lib.mg_batch_solve(self._h, px, pf, int(kappa), float(tol), int(max_iters), int(bool(mixed)),
                                        it, rel), "mg_batch_solve")
        return st, list(it), list(rel)
