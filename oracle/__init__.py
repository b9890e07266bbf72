"""Plain CPU FP64 oracle for the KS-cutoff simulation of the discrete power law.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is the
independent checker of the CUDA library and shares no code with it: the C
source next to this file is compiled with gcc into ``_build/liboracle.so`` and
called through ctypes.  See ``oracle.c`` for the paper passages each function
follows and the parity status of each.  ``cutoff_lookup`` (plain Python) is
pinned by exactness at grid points, exact reproduction of functions bilinear
in (exponent, ln N), clamping at the grid's edges and single-row grids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOCONV = 0, 1, 2, 3
XCAP = 1 << 62

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.or_philox4x32_10.argtypes = [ctypes.POINTER(c.c_uint32), ctypes.POINTER(c.c_uint32),
                                         ctypes.POINTER(c.c_uint32)]
        lib.or_draw_m.restype = c.c_uint64
        lib.or_draw_m.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64]
        lib.or_hurwitz3.argtypes = [c.c_double, c.c_double, _f64p]
        lib.or_hurwitz.restype = c.c_double
        lib.or_hurwitz.argtypes = [c.c_double, c.c_double]
        lib.or_pmf.restype = c.c_double
        lib.or_pmf.argtypes = [c.c_double, c.c_uint64, c.c_uint64]
        lib.or_survival.restype = c.c_double
        lib.or_survival.argtypes = [c.c_double, c.c_double, c.c_uint64, c.c_uint64]
        lib.or_invert.restype = c.c_uint64
        lib.or_invert.argtypes = [c.c_double, c.c_double, c.c_uint64, c.c_uint64]
        lib.or_sample.argtypes = [c.c_double, c.c_uint64, c.c_uint64, c.c_uint32, c.c_uint32,
                                  c.c_uint32, c.c_int64, _u64p]
        lib.or_log_sum.restype = c.c_double
        lib.or_log_sum.argtypes = [_u64p, c.c_int64, c.c_uint64]
        lib.or_mle_from_logsum.argtypes = [c.c_double, c.c_int64, c.c_uint64, _f64p,
                                           ctypes.POINTER(c.c_int)]
        lib.or_mle.argtypes = [_u64p, c.c_int64, c.c_uint64, _f64p]
        lib.or_ks_brute.argtypes = [_u64p, c.c_int64, c.c_uint64, c.c_double, _f64p]
        lib.or_ks.argtypes = [_u64p, c.c_int64, c.c_uint64, c.c_double, _f64p]
        lib.or_replicate.argtypes = [c.c_double, c.c_uint64, c.c_int64, c.c_uint64, c.c_uint32,
                                     c.c_uint32, c.c_uint32, _f64p, _f64p]
        lib.or_cell.argtypes = [c.c_double, c.c_uint64, c.c_int64, c.c_uint64, c.c_uint32,
                                c.c_uint32, c.c_uint32, c.c_int64, c.c_int, _f64p, _f64p, _i64p]
        lib.or_quantile_index.restype = c.c_int64
        lib.or_quantile_index.argtypes = [c.c_int64, c.c_double]
        lib.or_quantiles.argtypes = [_f64p, c.c_int64, _f64p, c.c_int, _f64p]
        lib.or_fit.argtypes = [_i32p, c.c_int64, c.c_uint64, _f64p, _f64p]
        lib.or_bootstrap_pvalue.argtypes = [_i32p, c.c_int64, c.c_uint64, c.c_int64, c.c_uint64,
                                            c.c_uint32, c.c_int, _f64p, _f64p, _f64p, _f64p]
        lib.or_max_threads.restype = c.c_int
        lib.or_tz_survival_table.restype = c.c_double
        lib.or_tz_survival_table.argtypes = [c.c_double, c.c_int64, _f64p]
        lib.or_tz_invert.restype = c.c_int64
        lib.or_tz_invert.argtypes = [_f64p, c.c_int64, c.c_uint64]
        lib.or_tz_sample.argtypes = [c.c_double, c.c_int64, c.c_uint64, c.c_uint32, c.c_uint32,
                                     c.c_uint32, c.c_int64, _u64p]
        lib.or_tz_mle_from_logsum.argtypes = [c.c_double, c.c_int64, c.c_int64, _f64p]
        lib.or_tz_ks.argtypes = [_u64p, c.c_int64, c.c_int64, c.c_double, _f64p]
        lib.or_tz_replicate.argtypes = [c.c_double, c.c_int64, c.c_int64, c.c_uint64, c.c_uint32,
                                        c.c_uint32, c.c_uint32, _f64p, _f64p]
        lib.or_tz_cell.argtypes = [c.c_double, c.c_int64, c.c_int64, c.c_uint64, c.c_uint32,
                                   c.c_uint32, c.c_uint32, c.c_int64, c.c_int, _f64p, _f64p, _i64p]
        lib.or_draw_bits64.restype = c.c_uint64
        lib.or_draw_bits64.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64]
        lib.or_binom_pmf.restype = c.c_double
        lib.or_binom_pmf.argtypes = [c.c_int64, c.c_int64, c.c_double, c.c_double]
        lib.or_binomial.restype = c.c_int64
        lib.or_binomial.argtypes = [c.c_int64, c.c_uint64, c.c_uint64, c.c_double]
        lib.or_thresholds.argtypes = [c.c_double, c.c_uint64, c.c_int64, _u64p]
        lib.or_mn_sample.argtypes = [c.c_double, c.c_uint64, _u64p, c.c_uint64, c.c_uint32, c.c_uint32,
                                     c.c_uint32, c.c_int64, _u64p]
        lib.or_mn_cell.argtypes = [c.c_double, c.c_uint64, c.c_int64, c.c_uint64, c.c_uint32, c.c_uint32,
                                   c.c_uint32, c.c_int64, c.c_int, _f64p, _f64p, _i64p]
        lib.or_estimate_xmin.argtypes = [_u64p, c.c_int64, c.c_int64, c.c_int64, c.c_int, _u64p, _f64p, _f64p,
                                         _i64p, _i64p, _i64p]
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str, allow_nonconv: bool = False) -> int:
    if st == OK or (allow_nonconv and st == ENOCONV):
        return st
    raise OracleError(f"{what}: status {st}")


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def draw_m(seed: int, cell: int, rep: int, purpose: int, i: int) -> int:
    return int(_load().or_draw_m(seed, cell, rep, purpose, i))


def hurwitz3(s: float, a: float):
    out = np.zeros(3)
    _load().or_hurwitz3(float(s), float(a), _ptr(out, _f64p))
    return float(out[0]), float(out[1]), float(out[2])


def hurwitz(s: float, a: float) -> float:
    return float(_load().or_hurwitz(float(s), float(a)))


def pmf(alpha: float, xmin: int, k: int) -> float:
    return float(_load().or_pmf(alpha, xmin, k))


def survival(alpha: float, xmin: int, k: int, Z: float | None = None) -> float:
    if Z is None:
        Z = hurwitz(alpha, float(xmin))
    return float(_load().or_survival(alpha, Z, xmin, k))


def invert(alpha: float, xmin: int, m: int, Z: float | None = None) -> int:
    if Z is None:
        Z = hurwitz(alpha, float(xmin))
    return int(_load().or_invert(alpha, Z, xmin, m))


def sample(alpha: float, xmin: int, seed: int, cell: int, rep: int, purpose: int,
           n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _load().or_sample(alpha, xmin, seed, cell, rep, purpose, n, _ptr(out, _u64p))
    return out


def log_sum(x: np.ndarray, xmin: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    return float(_load().or_log_sum(_ptr(x, _u64p), x.size, xmin))


def mle_from_logsum(L: float, n: int, xmin: int):
    a = ctypes.c_double()
    it = ctypes.c_int()
    st = _load().or_mle_from_logsum(L, n, xmin, ctypes.byref(a), ctypes.byref(it))
    _check(st, "mle_from_logsum", allow_nonconv=True)
    return a.value, it.value, st


def mle(x: np.ndarray, xmin: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    a = ctypes.c_double()
    _check(_load().or_mle(_ptr(x, _u64p), x.size, xmin, ctypes.byref(a)), "mle", True)
    return a.value


def ks(x: np.ndarray, xmin: int, alpha: float, brute: bool = False) -> float:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    d = ctypes.c_double()
    fn = _load().or_ks_brute if brute else _load().or_ks
    _check(fn(_ptr(x, _u64p), x.size, xmin, alpha, ctypes.byref(d)), "ks")
    return d.value


def replicate(alpha: float, xmin: int, n: int, seed: int, cell: int, rep: int,
              purpose: int = 0):
    a = ctypes.c_double()
    d = ctypes.c_double()
    _check(_load().or_replicate(alpha, xmin, n, seed, cell, rep, purpose, ctypes.byref(a),
                                ctypes.byref(d)), "replicate", True)
    return a.value, d.value


def cell(alpha: float, xmin: int, n: int, R: int, seed: int, cell_id: int,
         purpose: int = 0, rep0: int = 0, threads: int = 0):
    """D and alpha-hat for replicates rep0..rep0+R-1 of one cell."""
    D = np.zeros(R)
    A = np.zeros(R)
    nc = ctypes.c_int64()
    _check(_load().or_cell(alpha, xmin, n, seed, cell_id, purpose, rep0, R, threads,
                           _ptr(D, _f64p), _ptr(A, _f64p), ctypes.byref(nc)), "cell")
    return D, A, int(nc.value)


def quantile_index(R: int, q: float) -> int:
    return int(_load().or_quantile_index(R, q))


def quantiles(D: np.ndarray, q) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.float64)
    qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    out = np.zeros(qa.size)
    _check(_load().or_quantiles(_ptr(D, _f64p), D.size, _ptr(qa, _f64p), qa.size,
                                _ptr(out, _f64p)), "quantiles")
    return out


def fit(data: np.ndarray, xmin: int):
    data = np.ascontiguousarray(data, dtype=np.int32)
    a = ctypes.c_double()
    d = ctypes.c_double()
    _check(_load().or_fit(_ptr(data, _i32p), data.size, xmin, ctypes.byref(a),
                          ctypes.byref(d)), "fit", True)
    return a.value, d.value


def bootstrap_pvalue(data: np.ndarray, xmin: int, B: int, seed: int, request_id: int,
                     threads: int = 0):
    data = np.ascontiguousarray(data, dtype=np.int32)
    a = ctypes.c_double()
    d = ctypes.c_double()
    p = ctypes.c_double()
    Db = np.zeros(B)
    _check(_load().or_bootstrap_pvalue(_ptr(data, _i32p), data.size, xmin, B, seed, request_id,
                                       threads, ctypes.byref(a), ctypes.byref(d),
                                       ctypes.byref(p), _ptr(Db, _f64p)), "bootstrap", True)
    return a.value, d.value, p.value, Db


def max_threads() -> int:
    return int(_load().or_max_threads())


# ---------------------------------------------------------------- truncated law
def tz_survival(gamma: float, K: int):
    """(Q[0..K], zeta_K): survival of the truncated law on 1..K."""
    Q = np.zeros(K + 1)
    z = _load().or_tz_survival_table(gamma, K, _ptr(Q, _f64p))
    return Q, float(z)


def tz_invert(Q: np.ndarray, K: int, m: int) -> int:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    return int(_load().or_tz_invert(_ptr(Q, _f64p), K, m))


def tz_sample(gamma: float, K: int, seed: int, cell: int, rep: int, purpose: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _load().or_tz_sample(gamma, K, seed, cell, rep, purpose, n, _ptr(out, _u64p))
    return out


def tz_mle(x: np.ndarray, K: int) -> float:
    g = ctypes.c_double()
    _check(_load().or_tz_mle_from_logsum(log_sum(x, 1), len(x), K, ctypes.byref(g)), "tz_mle")
    return g.value


def tz_mle_from_logsum(L: float, n: int, K: int) -> float:
    g = ctypes.c_double()
    _check(_load().or_tz_mle_from_logsum(L, n, K, ctypes.byref(g)), "tz_mle")
    return g.value


def tz_ks(x: np.ndarray, K: int, gamma: float) -> float:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    d = ctypes.c_double()
    _check(_load().or_tz_ks(_ptr(x, _u64p), x.size, K, gamma, ctypes.byref(d)), "tz_ks")
    return d.value


def tz_cell(gamma: float, K: int, n: int, R: int, seed: int, cell_id: int, purpose: int = 0,
            rep0: int = 0, threads: int = 0):
    """D and gamma-hat for replicates rep0..rep0+R-1 of one truncated cell."""
    D = np.zeros(R)
    A = np.zeros(R)
    nc = ctypes.c_int64()
    _check(_load().or_tz_cell(gamma, K, n, seed, cell_id, purpose, rep0, R, threads,
                              _ptr(D, _f64p), _ptr(A, _f64p), ctypes.byref(nc)), "tz_cell")
    return D, A, int(nc.value)


def cutoff_lookup(grid_alpha, grid_n, table: np.ndarray, alpha: float, n: int) -> np.ndarray:
    """Cutoffs at (alpha, n) from a table on the grid (grid_alpha[i], grid_n[k])
    (table[i, k, :]): bilinear in (alpha, ln n) between the four surrounding
    grid cells, clamped to the grid's edges (the reading of Section 3's use of
    the tables at a close value of the exponent)."""
    import math

    def bracket(g, v):
        if len(g) == 1:
            return 0, 0.0
        i = 0
        while i + 2 < len(g) and g[i + 1] <= v:
            i += 1
        t = (v - g[i]) / (g[i + 1] - g[i])
        return i, min(max(t, 0.0), 1.0)

    ia, wa = bracket([float(a) for a in grid_alpha], float(alpha))
    ln = [math.log(float(v)) for v in grid_n]
    k, wn = bracket(ln, math.log(float(n)))
    ia1 = ia + 1 if len(grid_alpha) > 1 else ia
    k1 = k + 1 if len(grid_n) > 1 else k
    out = np.zeros(table.shape[2])
    for j in range(table.shape[2]):
        v00, v10 = table[ia, k, j], table[ia1, k, j]
        v01, v11 = table[ia, k1, j], table[ia1, k1, j]
        out[j] = (1.0 - wa) * ((1.0 - wn) * v00 + wn * v01) + wa * ((1.0 - wn) * v10 + wn * v11)
    return out


def estimate_xmin(x: np.ndarray, max_candidates: int = 1000, min_tail: int = 10, threads: int = 0):
    """Lower end by KS minimisation over the smallest max_candidates distinct
    values: (best index or -1, xmin[], alpha_hat[], D[], n_tail[]) per candidate."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    xm = np.zeros(max_candidates, dtype=np.uint64)
    a = np.zeros(max_candidates)
    d = np.zeros(max_candidates)
    nt = np.zeros(max_candidates, dtype=np.int64)
    nc, best = ctypes.c_int64(), ctypes.c_int64()
    _check(_load().or_estimate_xmin(_ptr(x, _u64p), x.size, max_candidates, min_tail, threads, _ptr(xm, _u64p),
                                    _ptr(a, _f64p), _ptr(d, _f64p), _ptr(nt, _i64p), ctypes.byref(nc),
                                    ctypes.byref(best)), "estimate_xmin")
    m = nc.value
    return best.value, xm[:m], a[:m], d[:m], nt[:m]


MN_BINS = 2048
PURPOSE_MULTINOMIAL = 3


def draw_bits64(seed: int, cell: int, rep: int, purpose: int, i: int) -> int:
    return int(_load().or_draw_bits64(seed, cell, rep, purpose, i))


def binom_pmf(x: int, n: int, p: float, q: float | None = None) -> float:
    return float(_load().or_binom_pmf(x, n, p, 1.0 - p if q is None else q))


def binomial(n: int, num: int, den: int, u: float) -> int:
    """Bin(n, num/den) from one uniform u in (0, 1] (inversion along a fixed order)."""
    return int(_load().or_binomial(n, num, den, u))


def thresholds(alpha: float, xmin: int, length: int = MN_BINS) -> np.ndarray:
    T = np.zeros(length, dtype=np.uint64)
    _load().or_thresholds(alpha, xmin, length, _ptr(T, _u64p))
    return T


def mn_sample(alpha: float, xmin: int, seed: int, cell: int, rep: int, purpose: int, n: int,
              T: np.ndarray | None = None) -> np.ndarray:
    """One replicate of n values by the multinomial (conditional binomial) sampler."""
    T = thresholds(alpha, xmin) if T is None else np.ascontiguousarray(T, dtype=np.uint64)
    out = np.zeros(n, dtype=np.uint64)
    _load().or_mn_sample(alpha, xmin, _ptr(T, _u64p), seed, cell, rep, purpose, n, _ptr(out, _u64p))
    return out


def mn_cell(alpha: float, xmin: int, n: int, R: int, seed: int, cell_id: int, purpose: int = PURPOSE_MULTINOMIAL,
            rep0: int = 0, threads: int = 0):
    """D and alpha-hat for replicates rep0..rep0+R-1 drawn by the multinomial sampler."""
    D = np.zeros(R)
    A = np.zeros(R)
    nc = ctypes.c_int64()
    _check(_load().or_mn_cell(alpha, xmin, n, seed, cell_id, purpose, rep0, R, threads, _ptr(D, _f64p),
                              _ptr(A, _f64p), ctypes.byref(nc)), "mn_cell")
    return D, A, int(nc.value)
