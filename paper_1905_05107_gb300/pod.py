"""ctypes binding of libpod_gb300.so (include/pod.h): argument marshalling
only.  Every step of the method runs in the library's CUDA kernels; there is
no CPU fallback, and every call raises if the library is missing.

Matrices follow the library's convention: A is m x n, column-major (each
snapshot contiguous).  From PyTorch, pass a CUDA tensor of shape (m, n) with
stride (1, lda), e.g. ``A_rowmajor_snapshots.t()`` or a tensor made from a
Fortran-ordered NumPy array.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpod_gb300.so")

POD_OK, POD_EINVAL, POD_ENOMEM, POD_ECUDA, POD_ERANK, POD_ETIMEOUT, POD_ENAN, POD_ESTATE, POD_EUNSUPPORTED = range(9)
POD_F32, POD_F64 = 0, 1
POD_L2N, POD_UNF, POD_ORT = 0, 1, 2
POD_ROW_L2N, POD_ROW_LS = 0, 1
POD_SUBSPACE, POD_MODES = 0, 1
POD_CORE_AUTO, POD_CORE_F32, POD_CORE_F64 = 0, 1, 2
POD_PREC_F32, POD_PREC_BF16, POD_PREC_BF16X3, POD_PREC_TF32X3 = 0, 1, 2, 3

EXPORTED = ["pod_init", "pod_iterate", "pod_modes", "pod_get_trace", "pod_replay_indices",
            "pod_backward", "pod_destroy", "pod_strerror", "pod_colnorms", "pod_sample",
            "pod_block_merge", "pod_reset", "pod_round_timings", "pod_counters", "pod_core_stats",
            "pod_sample_noalloc", "pod_last_rows", "pod_row_draws", "pod_wedin", "pod_atu", "pod_incremental", "pod_robust_rounds", "pod_set_wait_limit",
            "pod_refine_timings"]

ROUND_KERNELS = ["sample", "proj", "proj_sum", "cgs_gram", "cgs_sum", "chol1", "qr2_gram", "qr2_sum", "cgs_robust",
                 "chol1_robust", "qr2_robust", "core_svd", "update"]
ORT_KERNELS = ["ort_atu", "ort_values"]
ROW_KERNELS = ["rows_sample", "rows_gram", "rows_chol", "rows_core", "rows_block", "rows_setg"]


class PodParams(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
        ("k", ctypes.c_int32), ("c", ctypes.c_int32), ("w", ctypes.c_int32), ("r", ctypes.c_int32),
        ("rows", ctypes.c_int32), ("col_strategy", ctypes.c_int32), ("row_strategy", ctypes.c_int32),
        ("criterion", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
        ("refine", ctypes.c_int32), ("dtype", ctypes.c_int32), ("core", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("block_trunc", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("keep_tape", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class PodError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, strerror(status), status))


_LIB = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpod_gb300.so is not built; run "
                               "`python -m paper_1905_05107_gb300.build` (CUDA path required)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        L.pod_init.argtypes = [P(vp), P(PodParams), vp, vp]
        L.pod_iterate.argtypes = [vp, i32, P(i32), P(dbl), P(i32)]
        L.pod_modes.argtypes = [vp, vp, vp, vp]
        L.pod_get_trace.argtypes = [vp, i32, P(i32), P(i32), P(dbl)]
        L.pod_replay_indices.argtypes = [vp, P(i32), P(i32), i32]
        L.pod_backward.argtypes = [vp, vp, vp, vp, i32]
        L.pod_destroy.argtypes = [vp]
        L.pod_destroy.restype = None
        L.pod_strerror.argtypes = [ctypes.c_int]
        L.pod_strerror.restype = ctypes.c_char_p
        L.pod_colnorms.argtypes = [vp, i32, i64, i64, i64, vp, vp]
        L.pod_sample.argtypes = [vp, vp, i64, i32, u64, i32, i32, vp, vp, vp]
        L.pod_block_merge.argtypes = [i32, i64, vp, vp, i32, vp, i64, i32, i32, i32, vp, vp, P(i32), vp]
        L.pod_reset.argtypes = [vp, vp]
        L.pod_round_timings.argtypes = [vp, P(ctypes.c_float), i32, P(i32)]
        L.pod_counters.argtypes = [vp, P(i64), P(i32)]
        L.pod_core_stats.argtypes = [vp, P(i32), P(i64)]
        L.pod_sample_noalloc.argtypes = [vp, vp, i64, i32, u64, i32, i32, vp, vp, vp]
        L.pod_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
        L.pod_refine_timings.argtypes = [vp, P(ctypes.c_float), i32, P(i32)]
        for name in EXPORTED:
            if name not in ("pod_destroy", "pod_strerror"):
                getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def strerror(status: int) -> str:
    return lib().pod_strerror(status).decode()


def _check(status: int, where: str):
    if status != POD_OK:
        raise PodError(status, where)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return POD_F32
    if t.dtype == torch.float64:
        return POD_F64
    raise TypeError("A must be float32 or float64, got %s" % t.dtype)


def _check_colmajor(A):
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dim() != 2 or A.stride(0) != 1 or A.stride(1) < A.shape[0]:
        raise ValueError("A must be (m, n) column-major: stride (1, lda >= m); got stride %s" % (A.stride(),))


_STRATEGY = {"l2n": POD_L2N, "unf": POD_UNF, "ort": POD_ORT}
_CRITERION = {"subspace": POD_SUBSPACE, "modes": POD_MODES}
_CORE = {"auto": POD_CORE_AUTO, "f32": POD_CORE_F32, "f64": POD_CORE_F64}
_ROW_STRATEGY = {"l2n": POD_ROW_L2N, "ls": POD_ROW_LS}
_PRECISION = {"f32": POD_PREC_F32, "bf16": POD_PREC_BF16, "bf16x3": POD_PREC_BF16X3, "tf32x3": POD_PREC_TF32X3}


@dataclass
class PodResult:
    U: "object"            # (m, k) column-major tensor
    sigma: "object"        # (k,) float64 tensor
    V: Optional["object"]  # (n, k) column-major tensor or None
    iterations: int
    done: bool
    measure: float


class Context:
    """One POD problem on one CUDA device (pod_init ... pod_destroy)."""

    def __init__(self, A, k: int, c: int, r: int = 0, col_strategy: str = "unf",
                 criterion: str = "subspace", tol: float = 1e-8, max_iter: int = 0,
                 refine: bool = True, seed: int = 0x5107, core: str = "auto", rows: bool = False,
                 row_strategy: str = "l2n", w: int = 0, block_trunc: bool = False, precision: str = "auto",
                 keep_tape: bool = False, stream=None):
        import torch
        _check_colmajor(A)
        self.A = A                    # keeps the borrowed buffer alive
        self.m, self.n = int(A.shape[0]), int(A.shape[1])
        self.k = int(k)
        self.dtype = A.dtype
        self.refine = bool(refine)
        self.device = A.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(A.device)
        p = PodParams()
        p.m, p.n, p.lda = self.m, self.n, int(A.stride(1))
        p.k, p.c, p.w, p.r = int(k), int(c), int(w), int(r)
        p.rows = 1 if rows else 0
        p.col_strategy = _STRATEGY[col_strategy]
        p.row_strategy = _ROW_STRATEGY[row_strategy]
        p.criterion = _CRITERION[criterion]
        p.tol = float(tol)
        p.max_iter = int(max_iter)
        p.refine = 1 if refine else 0
        p.dtype = _dtype_code(A)
        p.core = _CORE[core]
        p.seed = int(seed) & ((1 << 64) - 1)
        p.block_trunc = 1 if block_trunc else 0
        if precision == "auto":
            # FP32 data: the A^T U contractions on tensor cores (split TF32)
            # wherever the layout allows it
            rr = int(r) if int(r) > 0 else int(k)
            ok = (A.dtype == torch.float32 and self.m % 4 == 0 and int(A.stride(1)) % 4 == 0 and rr <= 64
                  and A.data_ptr() % 16 == 0)
            precision = "tf32x3" if ok else "f32"
        p.precision = _PRECISION[precision]
        p.keep_tape = 1 if keep_tape else 0
        self.params = p
        self._h = ctypes.c_void_p()
        with torch.cuda.device(A.device):
            _check(lib().pod_init(ctypes.byref(self._h), ctypes.byref(p), _ptr(A), _stream(self.stream)),
                   "pod_init")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pod_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, max_steps: int = 1 << 30):
        done = ctypes.c_int32(0)
        meas = ctypes.c_double(0.0)
        steps = ctypes.c_int32(0)
        _check(lib().pod_iterate(self._h, int(max_steps), ctypes.byref(done), ctypes.byref(meas),
                                 ctypes.byref(steps)), "pod_iterate")
        return bool(done.value), float(meas.value), int(steps.value)

    def modes(self, with_v: bool = False):
        import torch
        U = torch.empty((self.k, self.m), dtype=self.dtype, device=self.device).t()
        sigma = torch.empty(self.k, dtype=torch.float64, device=self.device)
        V = torch.empty((self.k, self.n), dtype=self.dtype, device=self.device).t() if with_v else None
        _check(lib().pod_modes(self._h, _ptr(U), _ptr(sigma), _ptr(V) if V is not None else None),
               "pod_modes")
        return U, sigma, V

    def reset(self, A=None):
        """New problem of the same shape (keeps workspaces and the graph)."""
        if A is not None:
            _check_colmajor(A)
            if tuple(A.shape) != (self.m, self.n) or A.stride(1) != self.params.lda or A.dtype != self.dtype:
                raise ValueError("reset needs a matrix of the same shape, lda and dtype")
            self.A = A
        _check(lib().pod_reset(self._h, _ptr(A) if A is not None else None), "pod_reset")

    def round_timings(self):
        """Runs one round with CUDA events between kernels; returns {name: ms}."""
        buf = (ctypes.c_float * 32)()
        cnt = ctypes.c_int32(0)
        _check(lib().pod_round_timings(self._h, buf, 32, ctypes.byref(cnt)), "pod_round_timings")
        names = (["tape_u"] if self.params.keep_tape else []) + \
            (ORT_KERNELS if self.params.col_strategy == POD_ORT else []) + ROUND_KERNELS[:1] + \
            (ROW_KERNELS if self.params.rows else (ROW_KERNELS[1:] if self.params.block_trunc else [])) + \
            ROUND_KERNELS[1:]
        return dict(zip(names, [float(x) for x in buf[: cnt.value]]))

    def refine_timings(self):
        """Runs the closing refinement with CUDA events between kernels;
        returns {name: ms} (pod_refine_timings)."""
        buf = (ctypes.c_float * 16)()
        cnt = ctypes.c_int32(0)
        _check(lib().pod_refine_timings(self._h, buf, 16, ctypes.byref(cnt)), "pod_refine_timings")
        names = ["state0", "atu", "state1", "gram_y", "chol_y", "state2", "qr2_y", "svd_r", "state3", "update_u"]
        return dict(zip(names, [float(x) for x in buf[: cnt.value]]))

    def counters(self):
        launches = ctypes.c_int64(0)
        rounds = ctypes.c_int32(0)
        _check(lib().pod_counters(self._h, ctypes.byref(launches), ctypes.byref(rounds)), "pod_counters")
        return int(launches.value), int(rounds.value)

    def core_stats(self):
        """(Jacobi sweeps, clock cycles per phase) of the last core SVD."""
        sw = ctypes.c_int32(0)
        cyc = (ctypes.c_int64 * 6)()
        _check(lib().pod_core_stats(self._h, ctypes.byref(sw), cyc), "pod_core_stats")
        return int(sw.value), [int(x) for x in cyc]

    def trace(self, t: int):
        idx = (ctypes.c_int32 * self.params.c)()
        g = ctypes.c_int32(0)
        meas = ctypes.c_double(0.0)
        _check(lib().pod_get_trace(self._h, int(t), idx, ctypes.byref(g), ctypes.byref(meas)), "pod_get_trace")
        return np.array(idx[: g.value], dtype=np.int64), float(meas.value)

    def backward(self, dU, dsigma=None, accumulate: bool = False, dA=None):
        """dL/dA for the frozen draws of this run (pod_backward); needs
        keep_tape=True and modes() to have run.  dU: (m, k) like modes()'s U;
        dsigma: (k,) FP64 or None.  Returns dA (m, n), column-major, A's dtype."""
        import torch
        dU = dU.to(self.dtype)
        if dU.stride(0) != 1 or dU.stride(1) != self.m:
            dU = dU.t().contiguous().t()
        if dA is None:
            dA = torch.empty((self.n, self.m), dtype=self.dtype, device=self.device).t()
            accumulate = False
        ds = None
        if dsigma is not None:
            ds = dsigma.to(torch.float64).contiguous()
        _check(lib().pod_backward(self._h, _ptr(dU), _ptr(ds) if ds is not None else None, _ptr(dA),
                                  1 if accumulate else 0), "pod_backward")
        return dA

    def wedin(self):
        """Eq. 7 measure after pod_modes with refinement: dict with the bound,
        |R|_F, |S|_F and the estimated omega."""
        out = (ctypes.c_double * 4)()
        _check(lib().pod_wedin(self._h, out), "pod_wedin")
        return {"bound": out[0], "norm_R": out[1], "norm_S": out[2], "omega": out[3]}

    def set_wait_limit(self, polls: int):
        """Bound of the tensor-core kernels' pipeline waits (pod_set_wait_limit;
        0 = default)."""
        _check(lib().pod_set_wait_limit(self._h, int(polls)), "pod_set_wait_limit")

    def robust_rounds(self) -> int:
        """Rounds that needed the compensated-Gram rerun of the first CholeskyQR pass."""
        v = ctypes.c_int32(0)
        _check(lib().pod_robust_rounds(self._h, ctypes.byref(v)), "pod_robust_rounds")
        return int(v.value)

    def row_draws(self) -> int:
        """w, the row draws per ICRS iteration (0 without rows)."""
        w = ctypes.c_int32(0)
        _check(lib().pod_row_draws(self._h, ctypes.byref(w)), "pod_row_draws")
        return int(w.value)

    def last_rows(self):
        """(distinct rows ascending, their draw counts) of the latest ICRS round."""
        cap = max(1, self.row_draws())
        rows = (ctypes.c_int32 * cap)()
        cnt = (ctypes.c_int32 * cap)()
        h = ctypes.c_int32(0)
        _check(lib().pod_last_rows(self._h, rows, cnt, cap, ctypes.byref(h)), "pod_last_rows")
        return np.array(rows[: h.value], dtype=np.int64), np.array(cnt[: h.value], dtype=np.int64)

    def replay(self, index_sets: List[np.ndarray]):
        flat = np.concatenate([np.asarray(s, dtype=np.int32) for s in index_sets]) if index_sets else \
            np.zeros(0, dtype=np.int32)
        off = np.zeros(len(index_sets) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(s) for s in index_sets])
        flat = np.ascontiguousarray(flat, dtype=np.int32)
        _check(lib().pod_replay_indices(self._h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(index_sets)),
               "pod_replay_indices")


def pod(A, k: int, c: int, with_v: bool = False, **kw) -> PodResult:
    """Dominant k POD modes of the column-major CUDA tensor A (m x n)."""
    with Context(A, k, c, **kw) as ctx:
        done, meas, steps = ctx.iterate()
        U, sigma, V = ctx.modes(with_v=with_v)
        return PodResult(U=U, sigma=sigma, V=V, iterations=steps, done=done, measure=meas)


def colnorms(A, stream=None):
    import torch
    _check_colmajor(A)
    s = torch.empty(A.shape[1], dtype=torch.float64, device=A.device)
    _check(lib().pod_colnorms(_ptr(A), _dtype_code(A), A.shape[0], A.shape[1], A.stride(1), _ptr(s),
                              _stream(stream)), "pod_colnorms")
    return s


def incremental(A_host, k: int, c: int, blocks: int, r: int = 0, col_strategy: str = "unf",
                criterion: str = "subspace", tol: float = 1e-8, max_iter: int = 0, seed: int = 0x5107,
                core: str = "auto", rows: bool = False, row_strategy: str = "l2n", w: int = 0,
                precision: str = "f32", device=None, stream=None):
    """Algorithm 3 on a host matrix (pod_incremental): column blocks streamed
    to the device, ISMA per block, BLOCK MERGE.  A_host: CPU tensor (m, n),
    column-major (pinned for overlap).  Returns (U (m, k), sigma (k,)) on the
    device."""
    import torch
    if A_host.is_cuda or A_host.dim() != 2 or A_host.stride(0) != 1 or A_host.stride(1) < A_host.shape[0]:
        raise ValueError("A_host must be a (m, n) column-major CPU tensor")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    m, n = int(A_host.shape[0]), int(A_host.shape[1])
    p = PodParams()
    p.m, p.n, p.lda = m, n, int(A_host.stride(1))
    p.k, p.c, p.w, p.r = int(k), int(c), int(w), int(r)
    p.rows = 1 if rows else 0
    p.col_strategy = _STRATEGY[col_strategy]
    p.row_strategy = _ROW_STRATEGY[row_strategy]
    p.criterion = _CRITERION[criterion]
    p.tol = float(tol)
    p.max_iter = int(max_iter)
    p.refine = 0
    p.dtype = _dtype_code(A_host)
    p.core = _CORE[core]
    p.seed = int(seed) & ((1 << 64) - 1)
    p.precision = _PRECISION[precision]
    U = torch.empty((int(k), m), dtype=A_host.dtype, device=dev).t()
    sig = torch.empty(int(k), dtype=torch.float64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        _check(lib().pod_incremental(ctypes.byref(p), ctypes.c_void_p(A_host.data_ptr()), int(blocks), _ptr(U),
                                     _ptr(sig), _stream(st)), "pod_incremental")
    return U, sig


def atu(A, U, precision: str = "f32", stream=None):
    """Y = A^T U (FP64, n x r) through pod_atu."""
    import torch
    _check_colmajor(A)
    _check_colmajor(U)
    if U.stride(1) != A.shape[0] or U.dtype != A.dtype:
        raise ValueError("U must be m x r with leading dimension m and the dtype of A")
    n, r = int(A.shape[1]), int(U.shape[1])
    Y = torch.empty((r, n), dtype=torch.float64, device=A.device).t()
    st = stream if stream is not None else torch.cuda.current_stream(A.device)
    _check(lib().pod_atu(_ptr(A), _dtype_code(A), int(A.shape[0]), n, int(A.stride(1)), _ptr(U), r, _ptr(Y),
                         _PRECISION[precision], _stream(st)), "pod_atu")
    return Y


def sample(w, mask, c: int, seed: int, t: int, stream_id: int = 0, stream=None):
    """Draws from integer weights w (uint64 values in an int64 CUDA tensor);
    mask (uint8 CUDA tensor) is updated in place.  Returns sorted distinct
    indices (int32 CUDA tensor)."""
    import torch
    idx = torch.empty(c, dtype=torch.int32, device=w.device)
    g = torch.zeros(1, dtype=torch.int32, device=w.device)
    _check(lib().pod_sample(_ptr(w), _ptr(mask), w.shape[0], int(c), int(seed) & ((1 << 64) - 1), int(t),
                            int(stream_id), _ptr(idx), _ptr(g), _stream(stream)), "pod_sample")
    return idx[: int(g.item())]


def block_merge(U1, s1, C, r: int, core: str = "auto", stream=None):
    """Algorithm 2 with the new block given as its scaled factor C (m x g)."""
    import torch
    _check_colmajor(C)
    m, g = C.shape
    r1 = 0 if U1 is None else int(U1.shape[1])
    if r1:
        _check_colmajor(U1)
        assert U1.stride(1) == m
    U_out = torch.empty((max(r, 1), m), dtype=C.dtype, device=C.device).t()
    s_out = torch.empty(max(r, 1), dtype=torch.float64, device=C.device)
    rn = ctypes.c_int32(0)
    _check(lib().pod_block_merge(_dtype_code(C), m, _ptr(U1) if r1 else None, _ptr(s1) if r1 else None, r1,
                                 _ptr(C), C.stride(1), g, int(r), _CORE[core], _ptr(U_out), _ptr(s_out),
                                 ctypes.byref(rn), _stream(stream)), "pod_block_merge")
    return U_out[:, : rn.value], s_out[: rn.value]


def _autograd_function():
    import torch

    class PODFunction(torch.autograd.Function):
        """(U, sigma) = top-k POD modes of A by ISMA; backward through
        pod_backward with the forward's draws held fixed."""

        @staticmethod
        def forward(fctx, A, k, c, kwargs):
            ctx = Context(A, k, c, keep_tape=True, **kwargs)
            ctx.iterate()
            U, s, _ = ctx.modes()
            fctx.pod = ctx
            return U, s

        @staticmethod
        def backward(fctx, gU, gs):
            ctx = fctx.pod
            if gU is None:
                gU = torch.zeros((ctx.m, ctx.k), dtype=ctx.dtype, device=ctx.device)
            dA = ctx.backward(gU, gs)
            ctx.close()
            return dA, None, None, None

    return PODFunction


def pod_modes_autograd(A, k: int, c: int, **kw):
    """Differentiable (U, sigma) of A (torch.autograd)."""
    return _autograd_function().apply(A, k, c, kw)

