"""ctypes binding of the FIRLS C ABI (``include/firls.h``).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library ``libfirls.so``.  PyTorch tensors provide device memory (their
``data_ptr()`` is passed through) and the CUDA stream.  There is no CPU
fallback: if the library is missing the import of a context raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfirls.so")

FIRLS_OK = 0
STATUS = {0: "FIRLS_OK", 1: "FIRLS_E_INVALID_ARG", 2: "FIRLS_E_SHAPE", 3: "FIRLS_E_GROUPMAP",
          4: "FIRLS_E_CUDA", 5: "FIRLS_E_NOMEM", 6: "FIRLS_E_BREAKDOWN", 7: "FIRLS_E_STATE",
          8: "FIRLS_E_DEVICE_TIMEOUT"}
PSI_HAAR, PSI_DB4, PSI_TV, PSI_TV_ANISO = 1, 2, 4, 8
PRECONDS = {"paper": 0, "jacobi": 1, "none": 2, "ilu0": 3}
REAL_X = 1

EXPORTED = ["firls_size_supported", "firls_create", "firls_set_operator", "firls_solve", "firls_solve_multi",
            "firls_last_error", "firls_destroy", "firls_apply_AHA", "firls_apply_Phi", "firls_apply_PhiT",
            "firls_apply_S_P", "firls_get_weights", "firls_get_precond", "firls_get_inverse_map",
            "firls_set_tuning", "firls_get_popcounts", "firls_set_wait_test", "firls_set_channels", "firls_dense_create",
            "firls_dense_set_matrix", "firls_dense_abar", "firls_dense_apply_AtA", "firls_dense_solve",
            "firls_dense_last_error", "firls_dense_destroy",
            "firls_set_timing", "firls_get_timing", "firls_apply_AHA_noalloc",
            "firls_cnn_create", "firls_cnn_set_params", "firls_cnn_get_params", "firls_cnn_get_grads",
            "firls_cnn_forward", "firls_cnn_train_step", "firls_cnn_destroy", "firls_objective",
            "firls_warm_start_guard", "firls_adjoint", "firls_data_consistency", "firls_autotune",
            "firls_get_tuning", "firls_slot_load", "firls_run", "firls_run_steps", "firls_slot_status",
            "firls_slot_retire", "firls_slot_move", "firls_set_active_slots",
            "firls_slot_get"]
KERNEL_CLASSES = ["row_fft", "col_fft_mask", "wavelet_S", "wavelet_Pinv", "row_ifft_combine", "ilu", "axpy",
                  "scalars", "weights", "other"]


class FirlsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class Params(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("pcg_tol", ctypes.c_float),
                ("outer_tol", ctypes.c_float), ("lambda_", ctypes.c_float), ("lambda_tv", ctypes.c_float),
                ("eps", ctypes.c_float), ("lambda_per_slice", ctypes.POINTER(ctypes.c_float)),
                ("lambda_tv_per_slice", ctypes.POINTER(ctypes.c_float)), ("outer_tol_kind", ctypes.c_int),
                ("precond", ctypes.c_int), ("outer_stall_tol", ctypes.c_float), ("pcg_tol_kind", ctypes.c_int),
                ("pcg_iters_late", ctypes.c_int), ("outer_late", ctypes.c_int), ("boundary_period", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("outer_done", ctypes.c_int), ("pcg_steps", ctypes.c_longlong), ("max_rel_change", ctypes.c_double),
                ("max_rel_residual", ctypes.c_double), ("n_breakdown", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libfirls.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FirlsError(4, f"{LIB_PATH} is missing; build it with paper_1411_5057_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    L.firls_size_supported.argtypes = [i32]
    L.firls_size_supported.restype = i32
    L.firls_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, u32, vp]
    L.firls_set_operator.argtypes = [vp, vp, u32, i32, vp, vp, i32, i32]
    L.firls_solve.argtypes = [vp, vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Stats)]
    L.firls_solve_multi.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(Params),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Stats)]
    L.firls_last_error.argtypes = [vp]
    L.firls_last_error.restype = ctypes.c_char_p
    L.firls_destroy.argtypes = [vp]
    L.firls_destroy.restype = None
    L.firls_apply_AHA.argtypes = [vp, vp, vp]
    L.firls_apply_Phi.argtypes = [vp, vp, vp]
    L.firls_apply_PhiT.argtypes = [vp, vp, vp]
    L.firls_apply_S_P.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, vp, vp]
    L.firls_get_weights.argtypes = [vp, vp, vp, vp]
    L.firls_get_precond.argtypes = [vp, vp, vp]
    L.firls_set_tuning.argtypes = [vp, i32, i32, i32]
    L.firls_get_inverse_map.argtypes = [vp, vp, vp]
    L.firls_get_popcounts.argtypes = [vp, vp]
    L.firls_set_wait_test.argtypes = [vp, i32]
    L.firls_set_channels.argtypes = [vp, i32]
    L.firls_apply_AHA_noalloc.argtypes = [i32, i32, vp, vp, vp, vp]
    L.firls_objective.argtypes = [vp, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(ctypes.c_double)]
    L.firls_adjoint.argtypes = [vp, vp, vp]
    L.firls_autotune.argtypes = [vp, ctypes.c_char_p]
    L.firls_slot_load.argtypes = [vp, i32, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.firls_run.argtypes = [vp, ctypes.POINTER(Params)]
    L.firls_run_steps.argtypes = [vp, ctypes.POINTER(Params), i32]
    L.firls_slot_status.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(i32)]
    L.firls_slot_retire.argtypes = [vp, i32]
    L.firls_slot_move.argtypes = [vp, i32, i32]
    L.firls_set_active_slots.argtypes = [vp, i32]
    L.firls_slot_get.argtypes = [vp, i32, vp]
    L.firls_get_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.firls_data_consistency.argtypes = [vp, vp, vp, vp]
    L.firls_warm_start_guard.argtypes = [vp, vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(ctypes.c_int)]
    fpp = ctypes.POINTER(ctypes.c_void_p)
    L.firls_cnn_create.argtypes = [ctypes.POINTER(vp), i32, i32, vp]
    L.firls_cnn_set_params.argtypes = [vp, fpp, fpp]
    L.firls_cnn_get_params.argtypes = [vp, fpp, fpp]
    L.firls_cnn_get_grads.argtypes = [vp, fpp, fpp]
    L.firls_cnn_forward.argtypes = [vp, vp, vp, vp]
    L.firls_cnn_train_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    L.firls_cnn_destroy.argtypes = [vp]
    L.firls_cnn_destroy.restype = None
    L.firls_set_timing.argtypes = [vp, i32]
    L.firls_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
    L.firls_dense_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, vp]
    L.firls_dense_set_matrix.argtypes = [vp, vp]
    L.firls_dense_abar.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.firls_dense_apply_AtA.argtypes = [vp, vp, vp]
    L.firls_dense_solve.argtypes = [vp, vp, ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Stats)]
    L.firls_dense_last_error.argtypes = [vp]
    L.firls_dense_last_error.restype = ctypes.c_char_p
    L.firls_dense_destroy.argtypes = [vp]
    _lib = L
    return L


def _need(t, numel, what, dtype=None):
    """Reject a CUDA tensor that does not hold `numel` contiguous elements
    (the library reads and writes exactly that many), or, with `dtype`, whose
    element type differs."""
    if t is None:
        return
    if not t.is_cuda or not t.is_contiguous() or t.numel() != numel:
        raise FirlsError(1, f"{what}: expected a contiguous CUDA tensor of {numel} elements, got "
                            f"{tuple(t.shape)} on {t.device}")
    if dtype is not None and t.dtype != dtype:
        raise FirlsError(1, f"{what}: expected {dtype}, got {t.dtype}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def size_supported(n: int) -> bool:
    return bool(lib().firls_size_supported(int(n)))


def make_params(outer, pcg, lam=0.0, lam_tv=0.0, pcg_tol=0.0, outer_tol=0.0, eps=0.0,
                lam_per_slice=None, lam_tv_per_slice=None, stop_on_distance=False, precond="paper",
                stall_tol=0.0, pcg_tol_rel=False, pcg_late=0, outer_late=0, boundary_period=1):
    """firls_params; precond is "paper", "jacobi" or "none" (FIRLS_PRECOND_*);
    pcg_tol_rel: pcg_tol is relative to each outer step's first residual;
    pcg_late > 0: outer steps from outer_late on run pcg_late PCG steps."""
    p = Params()
    p.pcg_iters_late, p.outer_late = int(pcg_late), int(outer_late)
    p.boundary_period = int(boundary_period)
    p.outer_stall_tol = float(stall_tol)
    p.pcg_tol_kind = 1 if pcg_tol_rel else 0
    p.outer_tol_kind = 1 if stop_on_distance else 0
    p.precond = PRECONDS[precond]
    p.outer_iters, p.pcg_iters = int(outer), int(pcg)
    p.pcg_tol, p.outer_tol = float(pcg_tol), float(outer_tol)
    p.lambda_, p.lambda_tv, p.eps = float(lam), float(lam_tv), float(eps)
    keep = []
    if lam_per_slice is not None:
        a = (ctypes.c_float * len(lam_per_slice))(*[float(v) for v in lam_per_slice])
        keep.append(a)
        p.lambda_per_slice = ctypes.cast(a, ctypes.POINTER(ctypes.c_float))
    if lam_tv_per_slice is not None:
        a = (ctypes.c_float * len(lam_tv_per_slice))(*[float(v) for v in lam_tv_per_slice])
        keep.append(a)
        p.lambda_tv_per_slice = ctypes.cast(a, ctypes.POINTER(ctypes.c_float))
    p._keep = keep
    return p


class DenseContext:
    """`problems` sparse-recovery problems with a dense M x N sensing matrix
    (own matrix per problem, or one shared), float32 device tensors."""

    def __init__(self, M, N, problems=1, shared=False, stream=None):
        import torch
        self.M, self.N, self.problems, self.shared = int(M), int(N), int(problems), bool(shared)
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib().firls_dense_create(ctypes.byref(h), self.M, self.N, self.problems, 1 if shared else 0,
                                      ctypes.c_void_p(self.stream.cuda_stream))
        if st != FIRLS_OK:
            raise FirlsError(st, f"firls_dense_create(M={M}, N={N}, problems={problems})")
        self.h = h

    def _check(self, st, what):
        if st != FIRLS_OK:
            msg = lib().firls_dense_last_error(self.h)
            raise FirlsError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().firls_dense_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_matrix(self, A):
        """A: float32 CUDA [problems, M, N] (or [M, N] when shared)."""
        _need(A, (1 if self.shared else self.problems) * self.M * self.N, "A", self._torch.float32)
        self._check(lib().firls_dense_set_matrix(self.h, _ptr(A)), "set_matrix")

    def abar(self):
        out = (ctypes.c_double * (1 if self.shared else self.problems))()
        self._check(lib().firls_dense_abar(self.h, out), "abar")
        return list(out)

    def apply_AtA(self, d, q):
        """q = A^T A d for every problem: float32 CUDA [problems, N] each."""
        f32 = self._torch.float32
        _need(d, self.problems * self.N, "d", f32)
        _need(q, self.problems * self.N, "q", f32)
        self._check(lib().firls_dense_apply_AtA(self.h, _ptr(d), _ptr(q)), "apply_AtA")

    def solve(self, b, params, x0=None, out=None, stats=False):
        torch = self._torch
        if out is None:
            out = torch.empty((self.problems, self.N), dtype=torch.float32, device=b.device)
        f32 = torch.float32
        _need(b, self.problems * self.M, "b", f32)
        _need(x0, self.problems * self.N, "x0", f32)
        _need(out, self.problems * self.N, "out", f32)
        s = Stats() if stats else None
        st = lib().firls_dense_solve(self.h, _ptr(b), ctypes.byref(params), _ptr(x0), _ptr(out),
                                     ctypes.byref(s) if s is not None else None)
        self._check(st, "dense_solve")
        return (out, s.as_dict()) if stats else out


class Context:
    """A batch of ``batch`` same-size slices (n x n) on the current device."""

    def __init__(self, n, batch=1, real=False, stream=None):
        import torch
        self.n, self.batch, self.real = int(n), int(batch), bool(real)
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib().firls_create(ctypes.byref(h), self.n, self.n, self.batch, REAL_X if real else 0,
                                ctypes.c_void_p(self.stream.cuda_stream))
        if st != FIRLS_OK:
            raise FirlsError(st, f"firls_create(n={n}, batch={batch})")
        self.h = h

    def _check(self, st, what):
        if st != FIRLS_OK:
            msg = lib().firls_last_error(self.h)
            raise FirlsError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().firls_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_operator(self, mask, psi, levels=0, groups=None, group_off=None, group_size=0):
        """mask: uint8 [batch, n, n] CUDA; groups: int32 CUDA ([G, g] or flat with group_off)."""
        _need(mask, self.batch * self.n * self.n, "mask")
        n_groups = 0
        if groups is not None:
            if group_off is not None:
                n_groups = group_off.numel() - 1
            else:
                n_groups, group_size = groups.shape
        self._check(lib().firls_set_operator(self.h, _ptr(mask), int(psi), int(levels), _ptr(groups),
                                             _ptr(group_off), int(n_groups), int(group_size)), "set_operator")

    def solve(self, b, params, x0=None, out=None, stats=False):
        torch = self._torch
        if out is None:
            out = torch.empty((self.batch, self.n, self.n), dtype=torch.complex64, device=b.device)
        nn = self.batch * self.n * self.n
        _need(b, nn, "b")
        _need(x0, nn, "x0")
        _need(out, nn, "out")
        s = Stats() if stats else None
        st = lib().firls_solve(self.h, _ptr(b), ctypes.byref(params), _ptr(x0), _ptr(out),
                               ctypes.byref(s) if s is not None else None)
        self._check(st, "solve")
        return (out, s.as_dict()) if stats else out

    def apply_AHA(self, d, q):
        self._check(lib().firls_apply_AHA(self.h, _ptr(d), _ptr(q)), "apply_AHA")

    def apply_Phi(self, x, c):
        self._check(lib().firls_apply_Phi(self.h, _ptr(x), _ptr(c)), "apply_Phi")

    def apply_PhiT(self, c, x):
        self._check(lib().firls_apply_PhiT(self.h, _ptr(c), _ptr(x)), "apply_PhiT")

    def apply_S_P(self, params, x, d, q, r, z):
        self._check(lib().firls_apply_S_P(self.h, ctypes.byref(params), _ptr(x), _ptr(d), _ptr(q), _ptr(r),
                                          _ptr(z)), "apply_S_P")

    # ---- continuous batching ----
    def slot_load(self, s, mask, b, lam, lam_tv, x0=None, eps=0.0):
        self._check(lib().firls_slot_load(self.h, int(s), _ptr(mask), _ptr(b), _ptr(x0), float(lam), float(lam_tv),
                                          float(eps)), "slot_load")

    def run(self, params):
        self._check(lib().firls_run(self.h, ctypes.byref(params)), "run")

    def run_steps(self, params, macro_steps):
        """Enqueue `macro_steps` macro steps (every slot advances on its own)."""
        self._check(lib().firls_run_steps(self.h, ctypes.byref(params), int(macro_steps)), "run_steps")

    def slot_status(self, with_pcg=False):
        """(done, outer steps, last relative change[, PCG steps]) per slot."""
        k = self.batch
        done, od, rc, pc = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_double * k)(), (ctypes.c_int * k)()
        self._check(lib().firls_slot_status(self.h, done, od, rc, pc), "slot_status")
        if with_pcg:
            return list(done), list(od), list(rc), list(pc)
        return list(done), list(od), list(rc)

    def slot_retire(self, s):
        self._check(lib().firls_slot_retire(self.h, int(s)), "slot_retire")

    def slot_move(self, src, dst):
        """Slot src continues in slot dst (src is retired)."""
        self._check(lib().firls_slot_move(self.h, int(src), int(dst)), "slot_move")

    def set_active_slots(self, k):
        """run / run_steps launch only slots [0, k) (0: all)."""
        self._check(lib().firls_set_active_slots(self.h, int(k)), "set_active_slots")

    def slot_get(self, s, out):
        self._check(lib().firls_slot_get(self.h, int(s), _ptr(out)), "slot_get")

    def autotune(self, cache_path=None):
        """Time the tile-shape choices on this context and keep the fastest."""
        self._check(lib().firls_autotune(self.h, cache_path.encode() if cache_path else None), "autotune")
        return self.tuning()

    def set_tuning(self, rows_per_cta=None, coarse_max=None, ilu_depth=None):
        """Set tile shapes (None keeps the current one, 0 the built-in default)."""
        cur = self.tuning()
        a = cur["rows_per_cta"] if rows_per_cta is None else rows_per_cta
        b = cur["coarse_max"] if coarse_max is None else coarse_max
        c = cur["ilu_depth"] if ilu_depth is None else ilu_depth
        self._check(lib().firls_set_tuning(self.h, a, b, c), "set_tuning")

    def set_channels(self, channels):
        """Multi-contrast images: every `channels` consecutive slices are the
        contrasts of one image (joint weights, one PCG on the stacked unknown)."""
        self._check(lib().firls_set_channels(self.h, int(channels)), "set_channels")

    def set_wait_test(self, enable=True):
        """Failure-detection test hook: the ILU kernel's bounded waits run out."""
        self._check(lib().firls_set_wait_test(self.h, 1 if enable else 0), "set_wait_test")

    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().firls_get_tuning(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "tuning")
        return {"rows_per_cta": a.value, "coarse_max": b.value, "ilu_depth": c.value}

    def adjoint(self, b, out=None):
        """A^H b (the zero-filled reconstruction)."""
        out = self._torch.empty((self.batch, self.n, self.n), dtype=self._torch.complex64,
                                device=b.device) if out is None else out
        self._check(lib().firls_adjoint(self.h, _ptr(b), _ptr(out)), "adjoint")
        return out

    def data_consistency(self, b, x, out=None):
        """F^H((1 - R) F x + R b)."""
        out = self._torch.empty_like(x) if out is None else out
        self._check(lib().firls_data_consistency(self.h, _ptr(b), _ptr(x), _ptr(out)), "data_consistency")
        return out

    def objective(self, b, params, x):
        """F_eps per slice (host list of floats)."""
        out = (ctypes.c_double * self.batch)()
        self._check(lib().firls_objective(self.h, _ptr(b), ctypes.byref(params), _ptr(x), out), "objective")
        return list(out)

    def warm_start_guard(self, b, params, x1, x0):
        """x0 = x1 where F_eps(x1) <= F_eps(A^H b), else A^H b; returns the per-slice choice."""
        ch = (ctypes.c_int * self.batch)()
        self._check(lib().firls_warm_start_guard(self.h, _ptr(b), ctypes.byref(params), _ptr(x1), _ptr(x0), ch),
                    "warm_start_guard")
        return [bool(v) for v in ch]

    def get_weights(self, w_wavelet=None, w_tv=None, w_tv2=None):
        self._check(lib().firls_get_weights(self.h, _ptr(w_wavelet), _ptr(w_tv), _ptr(w_tv2)), "get_weights")

    def get_precond(self, wavelet_diag=None, inv_a=None):
        self._check(lib().firls_get_precond(self.h, _ptr(wavelet_diag), _ptr(inv_a)), "get_precond")

    def get_inverse_map(self, offsets, ids):
        self._check(lib().firls_get_inverse_map(self.h, _ptr(offsets), _ptr(ids)), "get_inverse_map")

    def set_timing(self, enable=True):
        self._check(lib().firls_set_timing(self.h, 1 if enable else 0), "set_timing")

    def get_timing(self):
        """{class: (total ms, launches, applications)} over the macro steps of
        the last timed graph (for solve: one outer step)."""
        k = len(KERNEL_CLASSES)
        ms = (ctypes.c_double * k)()
        ln = (ctypes.c_int * k)()
        ap = (ctypes.c_int * k)()
        self._check(lib().firls_get_timing(self.h, ms, ln, ap), "get_timing")
        return {name: (ms[i], ln[i], ap[i]) for i, name in enumerate(KERNEL_CLASSES)}

    def get_popcounts(self, counts):
        self._check(lib().firls_get_popcounts(self.h, _ptr(counts)), "get_popcounts")


def solve_multi(ctxs, bs, params, outs, x0s=None, stats=False):
    """One call over contexts of different sizes: one CUDA graph per outer
    step; `params` is one Params per context (same schedule)."""
    k = len(ctxs)
    P = (Params * k)(*params)
    H = (ctypes.c_void_p * k)(*[c.h for c in ctxs])
    B = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
    O = (ctypes.c_void_p * k)(*[o.data_ptr() for o in outs])
    X = (ctypes.c_void_p * k)(*[x.data_ptr() for x in x0s]) if x0s is not None else None
    S = (Stats * k)() if stats else None
    st = lib().firls_solve_multi(H, k, B, P, X, O, S)
    if st != FIRLS_OK:
        raise FirlsError(st, "solve_multi: " + (lib().firls_last_error(ctxs[0].h) or b"").decode())
    return [s.as_dict() for s in S] if stats else None


CNN_CHANNELS = (3, 32, 32, 32, 32, 32, 2)


class Cnn:
    """The learned warm start: x1 = A^H b + CNN([Re A^H b, Im A^H b, mask])."""

    def __init__(self, n, batch, stream=None):
        import torch
        self._torch = torch
        self.n, self.batch = int(n), int(batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib().firls_cnn_create(ctypes.byref(h), self.n, self.batch, ctypes.c_void_p(self.stream.cuda_stream))
        if st != FIRLS_OK:
            raise FirlsError(st, f"firls_cnn_create(n={n}, batch={batch})")
        self.h = h

    def _arrays(self, arrs):
        import numpy as np
        keep = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
        ptrs = (ctypes.c_void_p * len(keep))(*[a.ctypes.data for a in keep])
        return keep, ptrs

    def set_params(self, params):
        """params: list of (w [3][3][cin][cout], b [cout]) float arrays."""
        kw, pw = self._arrays([w for w, _ in params])
        kb, pb = self._arrays([b for _, b in params])
        st = lib().firls_cnn_set_params(self.h, pw, pb)
        if st != FIRLS_OK:
            raise FirlsError(st, "firls_cnn_set_params")

    def _get(self, fn):
        import numpy as np
        ws = [np.zeros((3, 3, CNN_CHANNELS[l], CNN_CHANNELS[l + 1]), np.float32) for l in range(6)]
        bs = [np.zeros(CNN_CHANNELS[l + 1], np.float32) for l in range(6)]
        pw = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in ws])
        pb = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in bs])
        st = fn(self.h, pw, pb)
        if st != FIRLS_OK:
            raise FirlsError(st, "firls_cnn_get")
        return list(zip(ws, bs))

    def get_params(self):
        return self._get(lib().firls_cnn_get_params)

    def get_grads(self):
        return self._get(lib().firls_cnn_get_grads)

    def forward(self, atb, mask, out=None):
        out = self._torch.empty_like(atb) if out is None else out
        st = lib().firls_cnn_forward(self.h, _ptr(atb), _ptr(mask), _ptr(out))
        if st != FIRLS_OK:
            raise FirlsError(st, "firls_cnn_forward")
        return out

    def train_step(self, atb, mask, target, lr, out=None, want_loss=True):
        out = self._torch.empty_like(atb) if out is None else out
        loss = ctypes.c_double()
        st = lib().firls_cnn_train_step(self.h, _ptr(atb), _ptr(mask), _ptr(target), _ptr(out), ctypes.c_float(lr),
                                        ctypes.byref(loss) if want_loss else None)
        if st != FIRLS_OK:
            raise FirlsError(st, "firls_cnn_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "h", None):
            lib().firls_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bucket(batch, active):
    """Smallest slot count of the sequence batch, ceil(3/4 batch), ... that
    holds `active`."""
    k = batch
    while k > 1:
        nxt = max(1, min(k - 1, (3 * k + 3) // 4))
        if nxt < active:
            break
        k = nxt
    return k


def serve(ctx, masks, bs, lams, lam_tvs, params, outs, x0s=None, chunk=64, max_outer=400, stop_after=None,
          counters=None, pcg_steps=None, compact=True):
    """Continuous batching over a queue of slices with ctx.batch slots.

    masks/bs/outs: per-slice device tensors ([n][n]); lams/lam_tvs: floats;
    params: schedule (pcg_iters, tolerances; outer_iters ignored).  Every
    slot advances on its own; the slots are polled every `chunk` macro steps,
    and a slot is read out and refilled when its slice has converged
    (params.outer_tol) or reached max_outer outer steps.  With stop_after,
    returns once that many slices have completed and retires the slices still
    in flight (their entry in the result stays 0).  Returns the outer steps
    of every slice.  counters (a dict, optional) receives "runs" (calls of
    ctx.run_steps, each one graph of `chunk` macro steps), "loads",
    "retires" and "moves"; pcg_steps (a list of len(bs), optional) receives
    the PCG steps of every slice.  With compact, once the queue is empty and
    fewer slots than a smaller bucket holds still run, the running slices move to
    the lowest slots and only those are launched (buckets shrinking by 3/4);
    a slice's results do not depend on its slot.
    """
    cnt = counters if counters is not None else {}
    for k in ("runs", "loads", "retires", "moves"):
        cnt.setdefault(k, 0)
    ctx.set_active_slots(0)
    launched = ctx.batch
    q = len(bs)
    steps = [0] * q
    slot_of = [-1] * ctx.batch
    nxt = 0
    for s in range(ctx.batch):
        if nxt < q:
            ctx.slot_load(s, masks[nxt], bs[nxt], lams[nxt], lam_tvs[nxt], None if x0s is None else x0s[nxt])
            cnt["loads"] += 1
            slot_of[s] = nxt
            nxt += 1
        else:
            ctx.slot_retire(s)
            cnt["retires"] += 1
    run = Params.from_buffer_copy(params)
    run.outer_iters = 1
    active = sum(1 for v in slot_of if v >= 0)
    completed = 0
    try:
        while active:
            if stop_after is not None and completed >= stop_after:
                for s in range(ctx.batch):
                    if slot_of[s] >= 0:
                        ctx.slot_retire(s)
                        cnt["retires"] += 1
                        slot_of[s] = -1
                break
            ctx.run_steps(run, chunk)
            cnt["runs"] += 1
            done, od, _, pc = ctx.slot_status(with_pcg=True)
            for s in range(ctx.batch):
                i = slot_of[s]
                if i < 0 or not (done[s] or od[s] >= max_outer):
                    continue
                ctx.slot_get(s, outs[i])
                steps[i] = od[s]
                if pcg_steps is not None:
                    pcg_steps[i] = pc[s]
                completed += 1
                if nxt < q:
                    ctx.slot_load(s, masks[nxt], bs[nxt], lams[nxt], lam_tvs[nxt], None if x0s is None else x0s[nxt])
                    cnt["loads"] += 1
                    slot_of[s] = nxt
                    nxt += 1
                else:
                    ctx.slot_retire(s)
                    cnt["retires"] += 1
                    slot_of[s] = -1
                    active -= 1
            if compact and nxt >= q and active:
                k = _bucket(ctx.batch, active)
                if k < launched:
                    free = [t for t in range(k) if slot_of[t] < 0]
                    for src in range(k, launched):
                        if slot_of[src] >= 0:
                            dst = free.pop()
                            ctx.slot_move(src, dst)
                            cnt["moves"] += 1
                            slot_of[dst], slot_of[src] = slot_of[src], -1
                    launched = k
                    ctx.set_active_slots(k)
    finally:
        ctx.set_active_slots(0)
    return steps
