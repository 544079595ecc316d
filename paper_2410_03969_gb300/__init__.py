"""Python binding of the rpchol CUDA library (accelerated randomly pivoted
Cholesky, Epperly, Tropp, Webber, arXiv 2410.03969) for GB300 / sm_103a.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels behind the C ABI declared in ``include/rpchol.h``.  PyTorch,
when present, supplies device memory (its caching allocator) and the
current CUDA stream.  There is no CPU fallback: if the compiled library is
missing, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librpchol.so")

KERNELS = {"gaussian": 0, "laplace_l2": 1, "matern52": 2, "matern32": 3, "laplace_l1": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY",
          6: "ECANCELLED", 7: "ENUMERIC"}

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class RpcholOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("instance", ctypes.c_uint32), ("profile", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("dev_alloc", _ALLOC_FN), ("dev_free", _FREE_FN),
                ("alloc_user", ctypes.c_void_p)]


class RunStats(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("proposals", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("status", ctypes.c_int32), ("plain", ctypes.c_int32),
                ("residual_trace", ctypes.c_double), ("trace_error", ctypes.c_double),
                ("col_bytes", ctypes.c_double), ("col_flops", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 8), ("phase_launches", ctypes.c_int64 * 8),
                ("kernel_launches", ctypes.c_int64), ("mma_flops_tf32", ctypes.c_double),
                ("mma_flops_f16", ctypes.c_double)]

PHASES = ("propose", "H", "reject", "prep", "colstep", "round_end", "plain_gemv", "plain_finish")


class RpcholError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(code, code), msg))
        self.code = code


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("rpchol_version", ctypes.c_char_p, []),
    ("rpchol_last_error", ctypes.c_char_p, []),
    ("rpchol_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.POINTER(RpcholOpts), ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint64]),
    ("rpchol_run_plain", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64]),
    ("rpchol_run_block", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_uint64]),
    ("rpchol_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("rpchol_factor", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_copy_factor", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    ("rpchol_copy_factor_raw", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p]),
    ("rpchol_run_to_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p]),
    ("rpchol_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(RunStats)]),
    ("rpchol_destroy", None, [ctypes.c_void_p]),
    ("rpchol_save", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_size_t)]),
    ("rpchol_restore", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("rpchol_resume", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("rpchol_selftest_wait", ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]),
    ("rpchol_trace_error_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                  ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_int64, ctypes.c_void_p,
                                                  ctypes.c_void_p]),
    ("rpchol_lowmem_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_lowmem_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_uint64]),
    ("rpchol_lowmem_copy", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]),
    ("rpchol_lowmem_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("rpchol_rpqr_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_rpqr_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_uint64]),
    ("rpchol_rpqr_copy", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    ("rpchol_rpqr_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("rpchol_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_batch_run", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]),
    ("rpchol_batch_destroy", None, [ctypes.c_void_p]),
    ("rpchol_batch_set_mode", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("rpchol_batch_mode", ctypes.c_int32, [ctypes.c_void_p]),
    ("rpchol_context_bytes", ctypes.c_int64, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int32]),
    ("rpchol_server_create", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    ("rpchol_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_uint64)]),
    ("rpchol_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                          ctypes.c_void_p]),
    ("rpchol_server_copy_factor", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                                 ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_void_p]),
    ("rpchol_server_release", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("rpchol_server_destroy", None, [ctypes.c_void_p]),
]


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("rpchol CUDA library not built (%s missing); run "
                              "`python -m paper_2410_03969_gb300.build`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise RpcholError(code, where, lib().rpchol_last_error().decode())


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _current_stream():
    torch = _torch()
    if torch is not None and torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class _TorchAllocator:
    """Device memory from torch's caching allocator, handed to the library
    through the allocator callbacks of rpchol_opts."""

    def __init__(self):
        self.torch = _torch()
        dev = self.torch.cuda.current_device()

        def alloc(nbytes, stream, user):
            try:
                return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), dev,
                                                                   stream or 0))
            except Exception:  # out of memory -> NULL -> RPCHOL_ENOMEM
                return None

        def free(ptr, stream, user):
            if ptr:
                self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _ALLOC_FN(alloc)
        self.free = _FREE_FN(free)


class Factorizer:
    """One rpchol context: the points are copied to the device once, then
    ``run`` (accelerated RPCholesky), ``run_plain`` (simple RPCholesky) and
    ``run_block`` (block RPCholesky) factorise K(X, X) to rank k on the device."""

    def __init__(self, X, kernel: str, sigma: float, k_max: int, T_max: int = 256,
                 precision: str = "fp64", instance: int = 0, use_graph: bool = True,
                 torch_allocator: bool = True, stream=None, profile: bool = False):
        L = lib()
        self._ctx = ctypes.c_void_p()
        torch = _torch()
        on_device = 0
        keep = None
        if torch is not None and isinstance(X, torch.Tensor):
            if X.dtype not in (torch.float32, torch.float64):
                X = X.float()
            X = X.contiguous()
            on_device = 1 if X.is_cuda else 0
            ptr = X.data_ptr()
            dt = 0 if X.dtype == torch.float32 else 1
            N, d = X.shape
            keep = X
        else:
            Xn = np.ascontiguousarray(X)
            if Xn.dtype not in (np.float32, np.float64):
                Xn = Xn.astype(np.float32)
            ptr = Xn.ctypes.data
            dt = 0 if Xn.dtype == np.float32 else 1
            N, d = Xn.shape
            keep = Xn
        self.N, self.d = int(N), int(d)
        self.kernel, self.sigma = kernel, float(sigma)
        self.precision = precision
        self._alloc = None
        opts = RpcholOpts()
        opts.precision = PRECISIONS[precision]
        opts.use_graph = 1 if use_graph else 0
        opts.instance = int(instance)
        opts.profile = 1 if profile else 0
        opts.stream = stream if stream is not None else _current_stream()
        if torch_allocator and torch is not None and torch.cuda.is_available():
            self._alloc = _TorchAllocator()
            opts.dev_alloc = self._alloc.alloc
            opts.dev_free = self._alloc.free
        self._opts = opts
        _check(L.rpchol_create(KERNELS[kernel], float(sigma), ctypes.c_void_p(ptr), int(N),
                               int(d), dt, on_device, int(k_max), int(T_max), ctypes.byref(opts),
                               ctypes.byref(self._ctx)), "rpchol_create")
        del keep

    # -- runs -------------------------------------------------------------
    def run(self, k: int, T: int, seed: int):
        _check(lib().rpchol_run(self._ctx, int(k), int(T), int(seed) & (2**64 - 1)),
               "rpchol_run")
        return self

    def run_plain(self, k: int, seed: int):
        _check(lib().rpchol_run_plain(self._ctx, int(k), int(seed) & (2**64 - 1)),
               "rpchol_run_plain")
        return self

    def run_block(self, k: int, b: int, seed: int):
        _check(lib().rpchol_run_block(self._ctx, int(k), int(b), int(seed) & (2**64 - 1)),
               "rpchol_run_block")
        return self

    def save(self) -> bytes:
        """Checkpoint of the last run (host bytes)."""
        n = ctypes.c_size_t(0)
        _check(lib().rpchol_save(self._ctx, None, ctypes.byref(n)), "rpchol_save")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().rpchol_save(self._ctx, buf, ctypes.byref(n)), "rpchol_save")
        return buf.raw[:n.value]

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().rpchol_restore(self._ctx, buf, len(blob)), "rpchol_restore")
        return self

    def resume(self, k: int):
        _check(lib().rpchol_resume(self._ctx, int(k)), "rpchol_resume")
        return self

    def sync(self):
        _check(lib().rpchol_sync(self._ctx), "rpchol_sync")
        return self

    # -- results ----------------------------------------------------------
    def factor_view(self):
        """(F device pointer, ldF, dtype code, rank, pivots device pointer)."""
        F = ctypes.c_void_p()
        ld = ctypes.c_int64()
        dt = ctypes.c_int32()
        rank = ctypes.c_int64()
        piv = ctypes.c_void_p()
        _check(lib().rpchol_factor(self._ctx, ctypes.byref(F), ctypes.byref(ld), ctypes.byref(dt),
                                   ctypes.byref(rank), ctypes.byref(piv)), "rpchol_factor")
        return F.value, ld.value, dt.value, rank.value, piv.value

    def rank(self) -> int:
        return self.factor_view()[3]

    def copy_factor(self, F=True, pivots=True, d=True):
        """Host copies: F (N x rank, float64), pivots (int64), d (float64)."""
        rank = self.rank()
        Fh = np.zeros((self.N, max(rank, 1)), dtype=np.float64) if F else None
        Ph = np.zeros(max(rank, 1), dtype=np.int64) if pivots else None
        Dh = np.zeros(self.N, dtype=np.float64) if d else None
        _check(lib().rpchol_copy_factor(
            self._ctx, Fh.ctypes.data if F else None, max(rank, 1),
            Ph.ctypes.data if pivots else None, Dh.ctypes.data if d else None),
            "rpchol_copy_factor")
        out = {"rank": rank}
        if F:
            out["F"] = Fh[:, :rank]
        if pivots:
            out["S"] = Ph[:rank]
        if d:
            out["d"] = Dh
        return out

    def copy_factor_into(self, F_out_ptr: int, ld_out: int, piv_out_ptr: int | None = None):
        """Copy F (as float64) and the pivots to caller-provided memory (host
        or device pointers)."""
        _check(lib().rpchol_copy_factor(self._ctx, ctypes.c_void_p(F_out_ptr), int(ld_out),
                                        ctypes.c_void_p(piv_out_ptr) if piv_out_ptr else None,
                                        None), "rpchol_copy_factor")

    def copy_factor_raw(self, F_out_ptr: int, ld_out: int, piv_out_ptr: int | None = None):
        """Copy F in its stored dtype (float32 in mixed mode) and the pivots to
        caller memory (host or device pointers)."""
        _check(lib().rpchol_copy_factor_raw(self._ctx, ctypes.c_void_p(F_out_ptr), int(ld_out),
                                            ctypes.c_void_p(piv_out_ptr) if piv_out_ptr
                                            else None), "rpchol_copy_factor_raw")

    def run_to_host(self, k: int, T: int, seed: int, F_out_ptr: int, ld_out: int,
                    piv_out_ptr: int | None = None):
        """Accelerated RPCholesky with F streamed to caller memory (pinned host
        memory for full speed) round by round while the later rounds compute;
        synchronous, same results as run() followed by copy_factor_raw()."""
        _check(lib().rpchol_run_to_host(self._ctx, int(k), int(T), int(seed) & (2**64 - 1),
                                        ctypes.c_void_p(F_out_ptr), int(ld_out),
                                        ctypes.c_void_p(piv_out_ptr) if piv_out_ptr else None),
               "rpchol_run_to_host")
        return self

    def stats(self) -> dict:
        st = RunStats()
        _check(lib().rpchol_stats(self._ctx, ctypes.byref(st)), "rpchol_stats")
        out = {k: getattr(st, k) for k, _ in RunStats._fields_
               if k not in ("phase_ms", "phase_launches")}
        out["phase_ms"] = {PHASES[i]: st.phase_ms[i] for i in range(8)}
        out["phase_launches"] = {PHASES[i]: int(st.phase_launches[i]) for i in range(8)}
        return out

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().rpchol_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class LowMemFactorizer:
    """Algorithm 3 (low-memory accelerated RPCholesky, FP64): keeps the pivots
    and the Cholesky factor L of A(S,S), never an N x k factor."""

    def __init__(self, X, kernel: str, sigma: float, k_max: int, T_max: int = 256, stream=None):
        Xn = np.ascontiguousarray(X)
        if Xn.dtype not in (np.float32, np.float64):
            Xn = Xn.astype(np.float32)
        self.N, self.d = int(Xn.shape[0]), int(Xn.shape[1])
        self._ctx = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _check(lib().rpchol_lowmem_create(KERNELS[kernel], float(sigma),
                                          ctypes.c_void_p(Xn.ctypes.data), self.N, self.d,
                                          0 if Xn.dtype == np.float32 else 1, int(k_max),
                                          int(T_max), st, ctypes.byref(self._ctx)),
               "rpchol_lowmem_create")

    def run(self, k: int, T: int, seed: int):
        _check(lib().rpchol_lowmem_run(self._ctx, int(k), int(T), int(seed) & (2**64 - 1)),
               "rpchol_lowmem_run")
        return self

    def copy(self):
        """Host copies: L (rank x rank, lower triangular), S, d, rank, rounds."""
        rank, rounds = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().rpchol_lowmem_copy(self._ctx, None, 0, None, None, ctypes.byref(rank),
                                        ctypes.byref(rounds)), "rpchol_lowmem_copy")
        r = rank.value
        L = np.zeros((max(r, 1), max(r, 1)))
        S = np.zeros(max(r, 1), dtype=np.int64)
        dres = np.zeros(self.N)
        _check(lib().rpchol_lowmem_copy(self._ctx, L.ctypes.data, max(r, 1), S.ctypes.data,
                                        dres.ctypes.data, ctypes.byref(rank),
                                        ctypes.byref(rounds)), "rpchol_lowmem_copy")
        return {"L": L[:r, :r], "S": S[:r], "d": dres, "rank": r, "rounds": rounds.value}

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().rpchol_lowmem_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class RPQR:
    """Algorithm 5 (accelerated randomly pivoted QR, FP64) of a dense M x N
    matrix B: B ~ Q F^* with orthonormal Q (M x k) and F = B^* Q (N x k)."""

    def __init__(self, B, k_max: int, T_max: int = 256, stream=None):
        Bf = np.asfortranarray(np.asarray(B, dtype=np.float64))
        self.M, self.N = int(Bf.shape[0]), int(Bf.shape[1])
        self._ctx = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _check(lib().rpchol_rpqr_create(ctypes.c_void_p(Bf.ctypes.data), self.M, self.N, self.M,
                                        int(k_max), int(T_max), st, ctypes.byref(self._ctx)),
               "rpchol_rpqr_create")

    def run(self, k: int, T: int, seed: int):
        _check(lib().rpchol_rpqr_run(self._ctx, int(k), int(T), int(seed) & (2**64 - 1)),
               "rpchol_rpqr_run")
        return self

    def copy(self):
        """Host copies: Q (M x rank), F (N x rank), S, u, rank, rounds."""
        rank, rounds = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().rpchol_rpqr_copy(self._ctx, None, self.M, None, 1, None, None,
                                      ctypes.byref(rank), ctypes.byref(rounds)), "rpchol_rpqr_copy")
        r = rank.value
        Qt = np.zeros((max(r, 1), self.M))  # column-major Q: one row per column
        F = np.zeros((self.N, max(r, 1)))
        S = np.zeros(max(r, 1), dtype=np.int64)
        u = np.zeros(self.N)
        _check(lib().rpchol_rpqr_copy(self._ctx, Qt.ctypes.data, self.M, F.ctypes.data,
                                      max(r, 1), S.ctypes.data, u.ctypes.data,
                                      ctypes.byref(rank), ctypes.byref(rounds)),
               "rpchol_rpqr_copy")
        return {"Q": Qt[:r].T.copy(), "F": F[:, :r].copy(), "S": S[:r], "u": u, "rank": r,
                "rounds": rounds.value}

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().rpchol_rpqr_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


BATCH_GRAPH = 0
BATCH_ENGINE = 1


class Batch:
    """Several Factorizers run together in one launch; instance i uses block
    size T[i].  `mode` is the executor: BATCH_ENGINE (one persistent launch of
    clusters taking instances from a device queue; mixed precision with the
    tensor-core column step) or BATCH_GRAPH (one CUDA graph with a conditional
    round loop per instance).  Destroy (close) the batch before its
    factorizers."""

    def __init__(self, factorizers, T):
        self.members = list(factorizers)
        n = len(self.members)
        ctxs = (ctypes.c_void_p * n)(*[f._ctx.value for f in self.members])
        Ts = (ctypes.c_int32 * n)(*[int(t) for t in T])
        self._b = ctypes.c_void_p()
        _check(lib().rpchol_batch_create(ctxs, n, Ts, ctypes.byref(self._b)),
               "rpchol_batch_create")
        self.T = [int(t) for t in T]

    @property
    def mode(self):
        return int(lib().rpchol_batch_mode(self._b))

    @mode.setter
    def mode(self, m):
        _check(lib().rpchol_batch_set_mode(self._b, int(m)), "rpchol_batch_set_mode")

    def run(self, k, seeds, stream=None):
        n = len(self.members)
        ks = (ctypes.c_int64 * n)(*[int(v) for v in k])
        ss = (ctypes.c_uint64 * n)(*[int(v) & (2**64 - 1) for v in seeds])
        _check(lib().rpchol_batch_run(self._b, ks, ss,
                                      stream if stream is not None else _current_stream()),
               "rpchol_batch_run")
        return self

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            lib().rpchol_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sigma", ctypes.c_double), ("X", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("d", ctypes.c_int32), ("x_dtype", ctypes.c_int32),
                ("k", ctypes.c_int64), ("T", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class JobResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("rank", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("trace_error", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


JOB_STATES = ("waiting", "running", "finished", "failed")


def context_bytes(N: int, d: int, k_max: int, T_max: int, precision: str = "mixed") -> int:
    return int(lib().rpchol_context_bytes(int(N), int(d), int(k_max), int(T_max),
                                          PRECISIONS[precision]))


class Server:
    """Continuous-batching server (rpchol_server_*): jobs are admitted by
    device memory and slots as they free up and overlap on the GPU."""

    def __init__(self, mem_budget_bytes: int, max_slots: int):
        self._s = ctypes.c_void_p()
        _check(lib().rpchol_server_create(int(mem_budget_bytes), int(max_slots),
                                          ctypes.byref(self._s)), "rpchol_server_create")

    def submit(self, X, kernel: str, sigma: float, k: int, T: int = 0, seed: int = 0,
               precision: str = "mixed") -> int:
        Xn = np.ascontiguousarray(X)
        if Xn.dtype not in (np.float32, np.float64):
            Xn = Xn.astype(np.float32)
        job = Job(KERNELS[kernel], float(sigma), Xn.ctypes.data, Xn.shape[0], Xn.shape[1],
                  0 if Xn.dtype == np.float32 else 1, int(k), int(T), PRECISIONS[precision],
                  int(seed) & (2**64 - 1))
        t = ctypes.c_uint64()
        _check(lib().rpchol_server_submit(self._s, ctypes.byref(job), ctypes.byref(t)),
               "rpchol_server_submit")
        return int(t.value)

    def poll(self, ticket: int, wait_ms: int = 0) -> dict:
        r = JobResult()
        _check(lib().rpchol_server_poll(self._s, int(ticket), int(wait_ms), ctypes.byref(r)),
               "rpchol_server_poll")
        out = {k: getattr(r, k) for k, _ in JobResult._fields_}
        out["state"] = JOB_STATES[r.state]
        return out

    def copy_factor(self, ticket: int, N: int, rank: int, dtype=np.float32):
        F = np.zeros((N, max(rank, 1)), dtype=dtype)
        P = np.zeros(max(rank, 1), dtype=np.int64)
        _check(lib().rpchol_server_copy_factor(self._s, int(ticket), F.ctypes.data,
                                               max(rank, 1), P.ctypes.data),
               "rpchol_server_copy_factor")
        return F[:, :rank], P[:rank]

    def release(self, ticket: int):
        _check(lib().rpchol_server_release(self._s, int(ticket)), "rpchol_server_release")

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            lib().rpchol_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def version() -> str:
    return lib().rpchol_version().decode()
