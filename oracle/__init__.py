"""FP64 CPU oracle of simple and accelerated randomly pivoted Cholesky.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only users.  The product (the CUDA
library and its Python binding) never imports this package, and this
package never imports the product.  The arithmetic lives in plain C
(``rpchol_oracle.c``); this module compiles it with gcc and exposes it
through ctypes, with numpy arrays in and out.

Paper: Epperly, Tropp, Webber, arXiv 2410.03969.  Algorithm 6 (simple
RPCholesky), Algorithm 2 (accelerated RPCholesky) and Algorithm 1
(RejectionSampleSubmatrix); the readings taken where the paper is silent
are stated in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpchol_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNELS = {"gaussian": 0, "laplace_l2": 1, "matern52": 2, "matern32": 3, "laplace_l1": 4}

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_u53.restype = ctypes.c_double
        lib.orc_uniform_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, _f64p, _f64p]
        lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_phi.restype = ctypes.c_double
        lib.orc_kernel_entry.argtypes = [ctypes.c_int, ctypes.c_double, _f32p, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_int64]
        lib.orc_kernel_entry.restype = ctypes.c_double
        lib.orc_sample.argtypes = [_f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
        lib.orc_sample.restype = ctypes.c_int64
        lib.orc_weight_total.argtypes = [_f64p, ctypes.c_int64]
        lib.orc_weight_total.restype = ctypes.c_double
        lib.orc_reject_chol.argtypes = [_f64p, ctypes.c_int32, _f64p, _f64p, ctypes.c_int32,
                                        _i32p, _f64p, _i32p]
        lib.orc_rpc_plain.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_uint32, _f64p, _i64p, _f64p, _i64p]
        lib.orc_rpc_accel.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_int, _f64p, _i64p, _f64p, _f64p, _i64p, _i64p,
                                      _i32p, ctypes.c_int64]
        lib.orc_rpc_block.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, _f64p,
                                      _i64p, _f64p, _i64p, _i64p, _i32p, ctypes.c_int64]
        lib.orc_rpqr_accel.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, _f64p, _f64p, _i64p, _f64p, _i64p,
                                       _i64p]
        lib.orc_rpc_lowmem.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, _f64p,
                                       _i64p, _f64p, _i64p, _i64p]
        lib.orc_fixed_pivot_factor.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               _f64p, ctypes.c_int64, _i64p, ctypes.c_int64,
                                               _f64p, _f64p, _f64p]
        lib.orc_pivots_many.argtypes = [_f32p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p,
                                        ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_int64, _i64p, _i64p]
        lib.orc_accel_trace_many.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_int64, _f64p]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_has_openmp.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def set_threads(n: int) -> int:
    """Threads for the row loops (OpenMP); returns the count actually used."""
    return int(_load().orc_set_threads(int(n)))


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def u53(a: int, b: int) -> float:
    return float(_load().orc_u53(a, b))


def uniform_pair(seed: int, slot: int, rnd: int, inst: int = 0):
    up = ctypes.c_double()
    ua = ctypes.c_double()
    _load().orc_uniform_pair(seed, slot, rnd, inst, ctypes.byref(up), ctypes.byref(ua))
    return up.value, ua.value


def phi(kernel: str, sigma: float, r2: float) -> float:
    return float(_load().orc_phi(KERNELS[kernel], sigma, r2))


def kernel_matrix(X, kernel: str, sigma: float, rows=None, cols=None) -> np.ndarray:
    """Explicit kernel entries A(rows, cols) by the oracle's own evaluator."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, d = X.shape
    rows = np.arange(N) if rows is None else np.asarray(rows)
    cols = np.arange(N) if cols is None else np.asarray(cols)
    out = np.empty((len(rows), len(cols)))
    xp = _p(X, _f32p)
    kk = KERNELS[kernel]
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            out[a, b] = lib.orc_kernel_entry(kk, sigma, xp, d, int(i), int(j))
    return out


def sample(w, U: float, W: float | None = None) -> int:
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    if W is None:
        W = lib.orc_weight_total(_p(w, _f64p), len(w))
    return int(lib.orc_sample(_p(w, _f64p), len(w), W, U))


def reject_chol(H, u, uacc, max_accept=None):
    """Algorithm 1 on a b x b psd H.  Returns (accepted local indices, L)."""
    lib = _load()
    H = np.array(H, dtype=np.float64, order="C", copy=True)
    b = H.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    uacc = np.ascontiguousarray(uacc, dtype=np.float64)
    acc = np.zeros(b, dtype=np.int32)
    L = np.zeros((b, b))
    n = ctypes.c_int32()
    _check(lib.orc_reject_chol(_p(H, _f64p), b, _p(u, _f64p), _p(uacc, _f64p),
                               b if max_accept is None else int(max_accept),
                               _p(acc, _i32p), _p(L, _f64p), ctypes.byref(n)), "reject_chol")
    n = n.value
    return acc[:n].copy(), L[:n, :n].copy()


def _matrix_args(X=None, kernel="gaussian", sigma=1.0, A=None):
    if A is not None:
        A = np.ascontiguousarray(A, dtype=np.float64)
        return None, 0, 0, 1.0, A, A.shape[0]
    X = np.ascontiguousarray(X, dtype=np.float32)
    return X, X.shape[1], KERNELS[kernel], float(sigma), None, X.shape[0]


def rpc_plain(k, seed, X=None, kernel="gaussian", sigma=1.0, A=None, inst=0):
    """Algorithm 6.  Returns dict(F (N x rank), S, d, rank)."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    F = np.zeros((N, max(k, 1)))
    S = np.full(max(k, 1), -1, dtype=np.int64)
    dres = np.zeros(N)
    rank = ctypes.c_int64()
    _check(lib.orc_rpc_plain(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N, k, seed, inst,
                             _p(F, _f64p), _p(S, _i64p), _p(dres, _f64p), ctypes.byref(rank)),
           "rpc_plain")
    r = rank.value
    return {"F": F[:, :r].copy(), "S": S[:r].copy(), "d": dres, "rank": r}


def rpc_accel(k, T, seed, X=None, kernel="gaussian", sigma=1.0, A=None, inst=0, max_rounds=0,
              accept_rule=0):
    """Algorithm 2 with Algorithm 1.  Returns dict(F, S, d, dpre, rank, rounds, round_sizes)."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    F = np.zeros((N, max(k, 1)))
    S = np.full(max(k, 1), -1, dtype=np.int64)
    dres = np.zeros(N)
    dpre = np.zeros(N)
    rank = ctypes.c_int64()
    rounds = ctypes.c_int64()
    cap = 4 * k + 64 if max_rounds <= 0 else max_rounds
    sizes = np.zeros(cap, dtype=np.int32)
    _check(lib.orc_rpc_accel(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N, k, T, max_rounds, seed,
                             inst, accept_rule, _p(F, _f64p), _p(S, _i64p), _p(dres, _f64p),
                             _p(dpre, _f64p), ctypes.byref(rank), ctypes.byref(rounds),
                             _p(sizes, _i32p), cap), "rpc_accel")
    r = rank.value
    nr = rounds.value
    return {"F": F[:, :r].copy(), "S": S[:r].copy(), "d": dres, "dpre": dpre, "rank": r,
            "rounds": nr, "round_sizes": sizes[:min(nr, cap)].copy()}


def rpc_block(k, b, seed, X=None, kernel="gaussian", sigma=1.0, A=None, inst=0, max_rounds=0):
    """Algorithm 7 (block RPCholesky).  Returns dict(F, S, d, rank, rounds, round_sizes)."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    F = np.zeros((N, max(k, 1)))
    S = np.full(max(k, 1), -1, dtype=np.int64)
    dres = np.zeros(N)
    rank = ctypes.c_int64()
    rounds = ctypes.c_int64()
    cap = 4 * k + 64 if max_rounds <= 0 else max_rounds
    sizes = np.zeros(cap, dtype=np.int32)
    _check(lib.orc_rpc_block(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N, k, b, max_rounds, seed,
                             inst, _p(F, _f64p), _p(S, _i64p), _p(dres, _f64p),
                             ctypes.byref(rank), ctypes.byref(rounds), _p(sizes, _i32p), cap),
           "rpc_block")
    r = rank.value
    nr = rounds.value
    return {"F": F[:, :r].copy(), "S": S[:r].copy(), "d": dres, "rank": r, "rounds": nr,
            "round_sizes": sizes[:min(nr, cap)].copy()}


def rpqr_accel(B, k, T, seed, inst=0, max_rounds=0):
    """Algorithm 5 (accelerated randomly pivoted QR) of the dense M x N matrix B.
    Returns dict(Q (M x rank, orthonormal columns), F (N x rank, F = B^* Q), S, u
    (residual squared column norms), rank, rounds)."""
    lib = _load()
    B = np.asarray(B, dtype=np.float64)
    M, N = B.shape
    Bc = np.ascontiguousarray(B.T)  # column j of B contiguous
    Q = np.zeros((max(k, 1), M))
    F = np.zeros((N, max(k, 1)))
    S = np.full(max(k, 1), -1, dtype=np.int64)
    u = np.zeros(N)
    rank = ctypes.c_int64()
    rounds = ctypes.c_int64()
    _check(lib.orc_rpqr_accel(_p(Bc, _f64p), M, N, k, T, max_rounds, seed, inst, _p(Q, _f64p),
                              _p(F, _f64p), _p(S, _i64p), _p(u, _f64p), ctypes.byref(rank),
                              ctypes.byref(rounds)), "rpqr_accel")
    r = rank.value
    return {"Q": Q[:r].T.copy(), "F": F[:, :r].copy(), "S": S[:r].copy(), "u": u, "rank": r,
            "rounds": rounds.value}


def rpc_lowmem(k, T, seed, X=None, kernel="gaussian", sigma=1.0, A=None, inst=0, max_rounds=0):
    """Algorithm 3 (low-memory accelerated RPCholesky).  Returns dict(L (rank x rank, lower
    triangular, A(S,S) = L L^*), S, d, rank, rounds)."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    L = np.zeros((max(k, 1), max(k, 1)))
    S = np.full(max(k, 1), -1, dtype=np.int64)
    dres = np.zeros(N)
    rank = ctypes.c_int64()
    rounds = ctypes.c_int64()
    _check(lib.orc_rpc_lowmem(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N, k, T, max_rounds, seed,
                              inst, _p(L, _f64p), _p(S, _i64p), _p(dres, _f64p),
                              ctypes.byref(rank), ctypes.byref(rounds)), "rpc_lowmem")
    r = rank.value
    return {"L": L[:r, :r].copy(), "S": S[:r].copy(), "d": dres, "rank": r,
            "rounds": rounds.value}


def fixed_pivot_factor(S, X=None, kernel="gaussian", sigma=1.0, A=None):
    """Cholesky with the given pivot order.  Returns (F, d, tr(A - FF^*))."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    S = np.ascontiguousarray(S, dtype=np.int64)
    k = len(S)
    F = np.zeros((N, max(k, 1)))
    dres = np.zeros(N)
    te = ctypes.c_double()
    _check(lib.orc_fixed_pivot_factor(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N, _p(S, _i64p), k,
                                      _p(F, _f64p), _p(dres, _f64p), ctypes.byref(te)),
           "fixed_pivot_factor")
    return F[:, :k].copy(), dres, te.value


def pivots_many(algo, k, n, seed, T=1, X=None, kernel="gaussian", sigma=1.0, A=None, inst0=0):
    """First k pivots of n independent runs (algo 'plain' or 'accel')."""
    lib = _load()
    X, d, kk, sg, A, N = _matrix_args(X, kernel, sigma, A)
    S = np.full((n, k), -1, dtype=np.int64)
    ranks = np.zeros(n, dtype=np.int64)
    _check(lib.orc_pivots_many(_p(X, _f32p), d, kk, sg, _p(A, _f64p), N,
                               0 if algo == "plain" else 1, k, T, seed, inst0, n, _p(S, _i64p),
                               _p(ranks, _i64p)), "pivots_many")
    return S, ranks


def accel_trace_many(A, T, rounds, n, seed, inst0=0):
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros(n)
    _check(lib.orc_accel_trace_many(_p(A, _f64p), A.shape[0], T, rounds, seed, inst0, n,
                                    _p(out, _f64p)), "accel_trace_many")
    return out
