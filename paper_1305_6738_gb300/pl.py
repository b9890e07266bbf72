"""ctypes binding of the C ABI in include/pl.h (argument marshalling only).

Every compute step runs in the CUDA library ``_build/libpl.so``; this module
only converts torch tensors / numpy arrays to pointers and status codes to
exceptions.  Importing it loads the library and raises ``ImportError`` if it
has not been built -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PL_LIB_PATH") or os.path.join(_HERE, "_build", "libpl.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)

PL_OK, PL_EINVAL, PL_ENOMEM, PL_ENOCONV, PL_ETIMEOUT, PL_ECUDA, PL_EBUSY = range(7)
PL_FP64, PL_FP32_BULK = 0, 1
_NAMES = {1: "PL_EINVAL", 2: "PL_ENOMEM", 3: "PL_ENOCONV", 4: "PL_ETIMEOUT", 5: "PL_ECUDA",
          6: "PL_EBUSY"}

EXPORTS = ["pl_create", "pl_destroy", "pl_last_error", "pl_sync", "pl_counters", "pl_probe_rates", "pl_set_tracing",
           "pl_trace", "pl_sample", "pl_fit_mle", "pl_ks_stat", "pl_ks_cutoffs",
           "pl_bootstrap_pvalue", "pl_fit_ks_noalloc", "pl_plan_cutoffs", "pl_plan_run",
           "pl_plan_destroy", "pl_autotune", "pl_set_split", "pl_autotune_cells", "pl_set_tuning", "pl_server_create", "pl_server_submit",
           "pl_server_poll", "pl_server_now", "pl_server_load", "pl_server_destroy",
           "pl_sample_truncated", "pl_ks_cutoffs_truncated", "pl_fit_ks_truncated", "pl_bespoke_cutoffs",
           "pl_bespoke_cutoffs_truncated", "pl_cutoff_lookup", "pl_estimate_xmin",
           "pl_ks_cutoffs_multinomial", "pl_bespoke_cutoffs_batch"]


class pl_cell(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("xmin", ctypes.c_uint64), ("n", ctypes.c_int64),
                ("replicates", ctypes.c_int64), ("cell_id", ctypes.c_uint64)]


class pl_tcell(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("K", ctypes.c_uint64), ("n", ctypes.c_int64),
                ("replicates", ctypes.c_int64), ("cell_id", ctypes.c_uint64)]


class pl_xmin_result(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_uint64), ("alpha_hat", ctypes.c_double), ("D", ctypes.c_double),
                ("n_tail", ctypes.c_int64), ("candidates", ctypes.c_int64)]


class pl_counter_info(ctypes.Structure):
    _fields_ = [("newton_capped", ctypes.c_uint64), ("tail_draws", ctypes.c_uint64),
                ("global_sorts", ctypes.c_uint64), ("fit_fallbacks", ctypes.c_uint64),
                ("resampled", ctypes.c_uint64)]


class pl_tuning(ctypes.Structure):
    _fields_ = [("split", ctypes.c_int64), ("item_reps", ctypes.c_int32), ("hist_shift", ctypes.c_int32),
                ("best_ms", ctypes.c_double)]


class pl_probe_info(ctypes.Structure):
    _fields_ = [("sm_clock_mhz", ctypes.c_double), ("mul_wide_per_sm_clk", ctypes.c_double),
                ("lop3_per_sm_clk", ctypes.c_double), ("dfma_per_sm_clk", ctypes.c_double),
                ("philox_words_per_s", ctypes.c_double), ("sms", ctypes.c_int32), ("pad", ctypes.c_int32)]


class pl_trace_info(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("law_ms", ctypes.c_float),
                ("replicate_ms", ctypes.c_float), ("select_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("sample_ms", ctypes.c_float),
                ("finish_ms", ctypes.c_float), ("waves", ctypes.c_uint32),
                ("draws", ctypes.c_uint64), ("sample_launches", ctypes.c_uint32)]


class pl_result(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n", ctypes.c_int64), ("alpha_hat", ctypes.c_double), ("D", ctypes.c_double),
                ("p", ctypes.c_double), ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


_vp = ctypes.c_void_p
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_lib.pl_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]
_lib.pl_create.restype = ctypes.c_int
_lib.pl_destroy.argtypes = [_vp]
_lib.pl_destroy.restype = None
_lib.pl_last_error.argtypes = [_vp]
_lib.pl_last_error.restype = ctypes.c_char_p
_lib.pl_sync.argtypes = [_vp, _vp]
_lib.pl_counters.argtypes = [_vp, _vp, ctypes.POINTER(pl_counter_info)]
_lib.pl_probe_rates.argtypes = [_vp, _vp, ctypes.POINTER(pl_probe_info)]
_lib.pl_set_tracing.argtypes = [_vp, ctypes.c_int]
_lib.pl_trace.argtypes = [_vp, _vp, ctypes.POINTER(pl_trace_info)]
_lib.pl_sample.argtypes = [_vp, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                           ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, _vp, _vp]
_lib.pl_fit_mle.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, _f64p, _vp]
_lib.pl_ks_stat.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                            _f64p, _vp]
_lib.pl_ks_cutoffs.argtypes = [_vp, ctypes.POINTER(pl_cell), ctypes.c_int, ctypes.c_uint64, _f64p,
                               ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.pl_bootstrap_pvalue.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64,
                                     ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _f64p, _f64p,
                                     _f64p, _vp]
_lib.pl_plan_cutoffs.argtypes = [_vp, ctypes.POINTER(pl_cell), ctypes.c_int, _f64p, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(_vp), _vp]
_lib.pl_plan_run.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _vp, _vp]
_lib.pl_autotune.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]
_lib.pl_set_split.argtypes = [_vp, ctypes.c_int64]
_lib.pl_autotune_cells.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                   ctypes.POINTER(pl_tuning), _vp]
_lib.pl_set_tuning.argtypes = [_vp, ctypes.POINTER(pl_tuning)]
_lib.pl_plan_destroy.argtypes = [_vp]
_lib.pl_plan_destroy.restype = None
_lib.pl_fit_ks_noalloc.argtypes = [_vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                   _vp, _vp]
_lib.pl_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_uint64, ctypes.c_int64]
_lib.pl_server_submit.argtypes = [_vp, ctypes.c_uint64, _vp, ctypes.c_int64, ctypes.c_uint64]
_lib.pl_server_poll.argtypes = [_vp, ctypes.POINTER(pl_result), ctypes.c_int, ctypes.c_double]
_lib.pl_server_poll.restype = ctypes.c_int
_lib.pl_server_now.argtypes = [_vp]
_lib.pl_server_now.restype = ctypes.c_double
_lib.pl_server_load.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_size_t), _u64p]
_lib.pl_server_destroy.argtypes = [_vp]
_lib.pl_sample_truncated.argtypes = [_vp, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, _vp, _vp]
_lib.pl_ks_cutoffs_truncated.argtypes = [_vp, ctypes.POINTER(pl_tcell), ctypes.c_int, ctypes.c_uint64, _f64p,
                                         ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.pl_fit_ks_truncated.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                     _f64p, _f64p, _vp]
_lib.pl_bespoke_cutoffs.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint64,
                                    ctypes.c_uint64, _f64p, ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p, _f64p,
                                    _vp]
_lib.pl_bespoke_cutoffs_truncated.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64,
                                              ctypes.c_uint64, ctypes.c_uint64, _f64p, ctypes.c_int, ctypes.c_int,
                                              _f64p, _f64p, _f64p, _f64p, _vp]
_lib.pl_cutoff_lookup.argtypes = [_vp, _f64p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, _vp,
                                  ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, _vp]
_lib.pl_estimate_xmin.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.POINTER(pl_xmin_result), _vp, _vp, _vp, _vp, _vp]
_lib.pl_ks_cutoffs_multinomial.argtypes = [_vp, ctypes.POINTER(pl_cell), ctypes.c_int, ctypes.c_uint64, _f64p,
                                           ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.pl_bespoke_cutoffs_batch.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _f64p,
                                          ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p, _f64p, _vp]
_lib.pl_server_destroy.restype = None
for _f in ["pl_sample_truncated", "pl_ks_cutoffs_truncated", "pl_fit_ks_truncated", "pl_bespoke_cutoffs",
           "pl_bespoke_cutoffs_truncated", "pl_cutoff_lookup", "pl_estimate_xmin", "pl_ks_cutoffs_multinomial", "pl_bespoke_cutoffs_batch", "pl_server_create", "pl_server_submit", "pl_server_load", "pl_autotune", "pl_set_split", "pl_autotune_cells", "pl_set_tuning", "pl_plan_cutoffs", "pl_plan_run", "pl_fit_ks_noalloc", "pl_sync", "pl_counters", "pl_probe_rates", "pl_set_tracing", "pl_trace", "pl_sample", "pl_fit_mle", "pl_ks_stat", "pl_ks_cutoffs",
           "pl_bootstrap_pvalue"]:
    getattr(_lib, _f).restype = ctypes.c_int


class PLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _data(x, what: str = "x"):
    """A data-set argument: a contiguous int32 tensor on a CUDA device (the
    entry points read it as int32[n] of device memory)."""
    if not (getattr(x, "is_cuda", False) and str(x.dtype) == "torch.int32" and x.is_contiguous()):
        raise ValueError(f"{what}: expected a contiguous torch.int32 CUDA tensor")
    return x


def _dev_f64(t, what: str, count: int):
    """A device output of `count` binary64 values."""
    if not (getattr(t, "is_cuda", False) and str(t.dtype) == "torch.float64" and t.is_contiguous()
            and t.numel() >= count):
        raise ValueError(f"{what}: expected a contiguous torch.float64 CUDA tensor of at least {count} elements")
    return t


def _ptr(t) -> int:
    """Device pointer of a torch tensor (or int passthrough)."""
    if isinstance(t, int):
        return t
    if t is None:
        return None
    return int(t.data_ptr())


@dataclass
class Cell:
    alpha: float
    xmin: int
    n: int
    replicates: int
    cell_id: int


@dataclass
class TCell:
    """A cell of the truncated law on 1..K (Tables 2-6)."""
    gamma: float
    K: int
    n: int
    replicates: int
    cell_id: int


class Context:
    """A library context on one CUDA device, with a workspace byte budget."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        h = _vp()
        st = _lib.pl_create(ctypes.byref(h), device, mem_budget_bytes)
        if st != PL_OK:
            raise PLError(st, "pl_create failed")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.pl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != PL_OK:
            raise PLError(st, _lib.pl_last_error(self._h).decode(errors="replace"))

    # ---- entry points (same names as the C ABI) --------------------------------
    def pl_sync(self, stream=None):
        self._check(_lib.pl_sync(self._h, _stream_ptr(stream)))

    def pl_counters(self, stream=None) -> dict:
        c = pl_counter_info()
        self._check(_lib.pl_counters(self._h, _stream_ptr(stream), ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in pl_counter_info._fields_}

    def pl_probe_rates(self, stream=None) -> dict:
        p = pl_probe_info()
        self._check(_lib.pl_probe_rates(self._h, _stream_ptr(stream), ctypes.byref(p)))
        return {k: getattr(p, k) for k, _ in pl_probe_info._fields_ if k != "pad"}

    def pl_set_tracing(self, on: bool = True):
        self._check(_lib.pl_set_tracing(self._h, 1 if on else 0))

    def pl_trace(self, stream=None) -> dict:
        t = pl_trace_info()
        self._check(_lib.pl_trace(self._h, _stream_ptr(stream), ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in pl_trace_info._fields_}

    def pl_sample(self, alpha: float, xmin: int, seed: int, cell_id: int, purpose: int, rep0: int,
                  nrep: int, n: int, out, stream=None):
        """out: torch.uint64 (or int64) device tensor of nrep*n elements."""
        assert out.numel() >= nrep * n and out.element_size() == 8
        self._check(_lib.pl_sample(self._h, alpha, xmin, seed, cell_id, purpose, rep0, nrep, n,
                                   _ptr(out), _stream_ptr(stream)))

    def pl_fit_mle(self, x, xmin: int, stream=None) -> float:
        """x: torch.int32 device tensor."""
        a = ctypes.c_double()
        self._check(_lib.pl_fit_mle(self._h, _ptr(_data(x)), x.numel(), xmin, ctypes.byref(a),
                                    _stream_ptr(stream)))
        return a.value

    def pl_ks_stat(self, x, xmin: int, alpha: float, prec: int = PL_FP64, stream=None) -> float:
        d = ctypes.c_double()
        self._check(_lib.pl_ks_stat(self._h, _ptr(_data(x)), x.numel(), xmin, alpha, prec, ctypes.byref(d),
                                    _stream_ptr(stream)))
        return d.value

    def pl_ks_cutoffs(self, cells, seed: int, q, prec: int = PL_FP64, cutoffs=None, D=None,
                      alpha_hat=None, stream=None):
        """cells: sequence of Cell (or objects with the same fields).  cutoffs: a
        device tensor (float64, len(cells)*len(q)) or None -> host numpy result.
        D / alpha_hat: optional device tensors receiving per-replicate values."""
        arr = (pl_cell * len(cells))(*[pl_cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id)
                                       for c in cells])
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        host = None
        if cutoffs is None:
            host = np.zeros(len(cells) * qa.size)
            out_ptr = host.ctypes.data
        elif isinstance(cutoffs, np.ndarray):
            host = cutoffs
            out_ptr = cutoffs.ctypes.data
        else:
            out_ptr = _ptr(cutoffs)
        self._check(_lib.pl_ks_cutoffs(self._h, arr, len(cells), seed,
                                       qa.ctypes.data_as(_f64p), qa.size, prec, out_ptr, _ptr(D),
                                       _ptr(alpha_hat), _stream_ptr(stream)))
        if host is not None:
            return host.reshape(len(cells), qa.size)
        return cutoffs

    def pl_sample_truncated(self, gamma: float, K: int, seed: int, cell_id: int, purpose: int, rep0: int,
                            nrep: int, n: int, out, stream=None):
        """out: 8-byte device tensor of nrep*n elements (values 1..K)."""
        assert out.numel() >= nrep * n and out.element_size() == 8
        self._check(_lib.pl_sample_truncated(self._h, gamma, K, seed, cell_id, purpose, rep0, nrep, n,
                                             _ptr(out), _stream_ptr(stream)))

    def pl_ks_cutoffs_truncated(self, cells, seed: int, q, prec: int = PL_FP64, cutoffs=None, D=None,
                                gamma_hat=None, stream=None):
        """As pl_ks_cutoffs for TCell cells; gamma_hat receives the per-replicate fits."""
        arr = (pl_tcell * len(cells))(*[pl_tcell(c.gamma, c.K, c.n, c.replicates, c.cell_id)
                                        for c in cells])
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        host = None
        if cutoffs is None:
            host = np.zeros(len(cells) * qa.size)
            out_ptr = host.ctypes.data
        elif isinstance(cutoffs, np.ndarray):
            host = cutoffs
            out_ptr = cutoffs.ctypes.data
        else:
            out_ptr = _ptr(cutoffs)
        self._check(_lib.pl_ks_cutoffs_truncated(self._h, arr, len(cells), seed,
                                                 qa.ctypes.data_as(_f64p), qa.size, prec, out_ptr, _ptr(D),
                                                 _ptr(gamma_hat), _stream_ptr(stream)))
        if host is not None:
            return host.reshape(len(cells), qa.size)
        return cutoffs

    def pl_fit_ks_truncated(self, x, K: int, gamma: float = float("nan"), prec: int = PL_FP64, stream=None):
        """x: torch.int32 device tensor (values 1..K).  Returns (gamma, D); gamma NaN fits it."""
        g, d = ctypes.c_double(), ctypes.c_double()
        self._check(_lib.pl_fit_ks_truncated(self._h, _ptr(_data(x)), x.numel(), K, gamma, prec, ctypes.byref(g),
                                             ctypes.byref(d), _stream_ptr(stream)))
        return g.value, d.value

    def pl_bespoke_cutoffs(self, x, xmin: int, R: int, seed: int, request_id: int, q, prec: int = PL_FP64,
                           stream=None):
        """Returns (alpha_hat, D, p, cutoffs[nq])."""
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        cut = np.zeros(qa.size)
        a, d, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(_lib.pl_bespoke_cutoffs(self._h, _ptr(_data(x)), x.numel(), xmin, R, seed, request_id,
                                            qa.ctypes.data_as(_f64p), qa.size, prec, ctypes.byref(a),
                                            ctypes.byref(d), ctypes.byref(p), cut.ctypes.data_as(_f64p),
                                            _stream_ptr(stream)))
        return a.value, d.value, p.value, cut

    def pl_bespoke_cutoffs_batch(self, xs, xmins, R: int, seed: int, request_ids, q, prec: int = PL_FP64,
                                 stream=None):
        """xs: torch.int32 device tensors.  Returns (alpha_hat[], D[], p[], cutoffs[nsets, nq])."""
        k = len(xs)
        ptrs = (ctypes.c_void_p * k)(*[_ptr(_data(x, "xs[]")) for x in xs])
        ns = (ctypes.c_int64 * k)(*[x.numel() for x in xs])
        xm = (ctypes.c_uint64 * k)(*[int(v) for v in xmins])
        rid = (ctypes.c_uint64 * k)(*[int(v) for v in request_ids])
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        a, d, p, cut = np.zeros(k), np.zeros(k), np.zeros(k), np.zeros(k * qa.size)
        self._check(_lib.pl_bespoke_cutoffs_batch(self._h, k, ptrs, ns, xm, R, seed, rid, qa.ctypes.data_as(_f64p),
                                                  qa.size, prec, a.ctypes.data_as(_f64p), d.ctypes.data_as(_f64p),
                                                  p.ctypes.data_as(_f64p), cut.ctypes.data_as(_f64p),
                                                  _stream_ptr(stream)))
        return a, d, p, cut.reshape(k, qa.size)

    def pl_bespoke_cutoffs_truncated(self, x, K: int, R: int, seed: int, request_id: int, q,
                                     prec: int = PL_FP64, stream=None):
        """Returns (gamma_hat, D, p, cutoffs[nq])."""
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        cut = np.zeros(qa.size)
        g, d, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(_lib.pl_bespoke_cutoffs_truncated(self._h, _ptr(_data(x)), x.numel(), K, R, seed, request_id,
                                                      qa.ctypes.data_as(_f64p), qa.size, prec, ctypes.byref(g),
                                                      ctypes.byref(d), ctypes.byref(p), cut.ctypes.data_as(_f64p),
                                                      _stream_ptr(stream)))
        return g.value, d.value, p.value, cut

    def pl_cutoff_lookup(self, grid_alpha, grid_n, table, nq: int, alpha, n, out, stream=None):
        """grid_alpha, grid_n: host sequences; table, alpha (float64), n (int64), out: device tensors."""
        ga = np.ascontiguousarray(np.asarray(grid_alpha, dtype=np.float64))
        gn = np.ascontiguousarray(np.asarray(grid_n, dtype=np.int64))
        self._check(_lib.pl_cutoff_lookup(self._h, ga.ctypes.data_as(_f64p), ga.size,
                                          gn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), gn.size, _ptr(table),
                                          nq, _ptr(alpha), _ptr(n), alpha.numel(), _ptr(out),
                                          _stream_ptr(stream)))
        return out

    def pl_estimate_xmin(self, x, max_candidates: int = 1000, min_tail: int = 10, cand_xmin=None,
                         cand_alpha=None, cand_D=None, cand_ntail=None, stream=None) -> dict:
        """x: torch.int32 device tensor.  Returns the pl_xmin_result fields; cand_* are
        optional device tensors (uint64/int64, float64, float64, int64) of max_candidates."""
        r = pl_xmin_result()
        self._check(_lib.pl_estimate_xmin(self._h, _ptr(_data(x)), x.numel(), max_candidates, min_tail, ctypes.byref(r),
                                          _ptr(cand_xmin), _ptr(cand_alpha), _ptr(cand_D), _ptr(cand_ntail),
                                          _stream_ptr(stream)))
        return {k: getattr(r, k) for k, _ in pl_xmin_result._fields_}

    def pl_ks_cutoffs_multinomial(self, cells, seed: int, q, prec: int = PL_FP64, cutoffs=None, D=None,
                                  alpha_hat=None, stream=None):
        """As pl_ks_cutoffs, with the multinomial histogram sampler (stream tag 3)."""
        arr = (pl_cell * len(cells))(*[pl_cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id) for c in cells])
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        host = None
        if cutoffs is None:
            host = np.zeros(len(cells) * qa.size)
            out_ptr = host.ctypes.data
        elif isinstance(cutoffs, np.ndarray):
            host = cutoffs
            out_ptr = cutoffs.ctypes.data
        else:
            out_ptr = _ptr(cutoffs)
        self._check(_lib.pl_ks_cutoffs_multinomial(self._h, arr, len(cells), seed, qa.ctypes.data_as(_f64p),
                                                   qa.size, prec, out_ptr, _ptr(D), _ptr(alpha_hat),
                                                   _stream_ptr(stream)))
        if host is not None:
            return host.reshape(len(cells), qa.size)
        return cutoffs

    def pl_autotune(self, stream=None) -> int:
        v = ctypes.c_int64()
        self._check(_lib.pl_autotune(self._h, _stream_ptr(stream), ctypes.byref(v)))
        return v.value

    def pl_set_split(self, split: int):
        self._check(_lib.pl_set_split(self._h, split))

    def pl_autotune_cells(self, cells, prec: int = PL_FP32_BULK, sample_replicates: int = 500,
                          stream=None) -> dict:
        arr = (pl_cell * len(cells))(*[pl_cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id)
                                       for c in cells])
        t = pl_tuning()
        self._check(_lib.pl_autotune_cells(self._h, arr, len(cells), prec, sample_replicates, ctypes.byref(t),
                                           _stream_ptr(stream)))
        return {k: getattr(t, k) for k, _ in pl_tuning._fields_}

    def pl_set_tuning(self, split: int, item_reps: int = 0, hist_shift: int = 0):
        t = pl_tuning(split, item_reps, hist_shift, 0.0)
        self._check(_lib.pl_set_tuning(self._h, ctypes.byref(t)))

    def pl_plan_cutoffs(self, cells, q, prec: int = PL_FP64, stream=None) -> "Plan":
        arr = (pl_cell * len(cells))(*[pl_cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id)
                                       for c in cells])
        qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        h = _vp()
        self._check(_lib.pl_plan_cutoffs(self._h, arr, len(cells), qa.ctypes.data_as(_f64p), qa.size,
                                         prec, ctypes.byref(h), _stream_ptr(stream)))
        return Plan(self, h)

    def pl_bootstrap_pvalue(self, x, xmin: int, B: int, seed: int, request_id: int,
                            prec: int = PL_FP64, stream=None):
        a, d, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(_lib.pl_bootstrap_pvalue(self._h, _ptr(_data(x)), x.numel(), xmin, B, seed, request_id,
                                             prec, ctypes.byref(a), ctypes.byref(d), ctypes.byref(p),
                                             _stream_ptr(stream)))
        return a.value, d.value, p.value


class Plan:
    """A planned cutoff computation (pl_plan_cutoffs); run() only enqueues kernels."""

    def __init__(self, ctx: Context, h):
        self._ctx = ctx
        self._h = h

    def run(self, seed: int, cutoffs, D=None, alpha_hat=None, stream=None):
        self._ctx._check(_lib.pl_plan_run(self._h, seed, _ptr(cutoffs), _ptr(D), _ptr(alpha_hat),
                                          _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.pl_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pl_fit_ks_noalloc(x, xmin: int, alpha: float, out, prec: int = PL_FP64, stream=None):
    """Fit (alpha NaN) or evaluate D at alpha for one data set, with the library's
    fixed scratch instead of a context (no device allocation by the library).
    x: int32 device tensor (n <= 262144); out: float64 device tensor of 3 elements
    receiving (alpha, D, zeta(alpha, xmin)) in stream order."""
    _data(x)
    _dev_f64(out, "out", 3)
    st = _lib.pl_fit_ks_noalloc(_ptr(x), x.numel(), xmin, alpha, prec, _ptr(out), _stream_ptr(stream))
    if st != PL_OK:
        raise PLError(st, "pl_fit_ks_noalloc failed")


class Server:
    """Continuous-batching engine of bootstrap fit requests (pl_server_*)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, workers: int = 4,
                 prec: int = PL_FP32_BULK, seed: int = 1, B: int = 2500):
        h = _vp()
        st = _lib.pl_server_create(ctypes.byref(h), device, mem_budget_bytes, workers, prec, seed, B)
        if st != PL_OK:
            raise PLError(st, "pl_server_create failed")
        self._h = h

    def pl_server_submit(self, request_id: int, x: np.ndarray, xmin: int = 1):
        """x: host int32 array (copied by the call)."""
        xa = np.ascontiguousarray(x, dtype=np.int32)
        st = _lib.pl_server_submit(self._h, request_id, xa.ctypes.data, xa.size, xmin)
        if st != PL_OK:
            raise PLError(st, "pl_server_submit failed")

    def pl_server_poll(self, max_results: int = 256, wait_s: float = 0.0) -> list[dict]:
        buf = (pl_result * max_results)()
        k = _lib.pl_server_poll(self._h, buf, max_results, wait_s)
        return [{f: getattr(buf[i], f) for f, _ in pl_result._fields_ if f != "pad"} for i in range(k)]

    def pl_server_now(self) -> float:
        return _lib.pl_server_now(self._h)

    def pl_server_load(self) -> tuple[int, int, int, int]:
        """(queued, running, reserved bytes, kernels launched by finished requests)"""
        q, r, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_uint64()
        _lib.pl_server_load(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b), ctypes.byref(k))
        return q.value, r.value, b.value, k.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.pl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
