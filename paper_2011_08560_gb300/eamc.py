"""Thin ctypes binding of libeamc.so (include/eamc.h).

Argument marshalling only: every step of the Monte Carlo path runs in the CUDA library.
The functions keep the C names; ``Context`` wraps one ``ea_ctx``.  PyTorch is used only to
hand over the current CUDA stream.  There is no CPU fallback: importing this module on a
machine where the library cannot be loaded raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from .build import LIB

EA_OK, EA_EINVAL, EA_ENOMEM, EA_ECUDA, EA_ETIMEOUT, EA_ESTATE = 0, -1, -2, -3, -4, -5
EA_ALWAYS = 0xFFFFFFFF
EA_FLAT, EA_POWERLAW, EA_ONE_OVER_K, EA_CANON = 0, 1, 2, 3
EA_REC_PLAIN, EA_REC_BERG = 0, 1
EA_ORDER_LEX, EA_ORDER_COLOUR = 0, 1


class EamcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"eamc error {code}: {msg}")
        self.code = code


class ea_rt_stats(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("n_rt", ctypes.c_int32),
                ("t_first", ctypes.c_int64), ("t_last", ctypes.c_int64),
                ("e_min", ctypes.c_int32), ("e_g", ctypes.c_int32),
                ("requeue", ctypes.c_int32), ("pad", ctypes.c_int32)]


RT_DTYPE = np.dtype([(f, np.int64 if t is ctypes.c_int64 else np.int32) for f, t in ea_rt_stats._fields_])
assert RT_DTYPE.itemsize == ctypes.sizeof(ea_rt_stats)


class ea_chain_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("L", ctypes.c_int32), ("b_top", ctypes.c_int32),
                ("parity", ctypes.c_int32), ("rid", ctypes.c_uint32),
                ("stream", ctypes.c_uint32), ("E", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("t", ctypes.c_uint64)]


class ea_pt_stats(ctypes.Structure):
    _fields_ = [("n_rt", ctypes.c_int32), ("phase", ctypes.c_int32),
                ("t_first", ctypes.c_int64), ("t_last", ctypes.c_int64),
                ("e_min", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ea_srv_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_L", ctypes.c_int32), ("Ls", ctypes.c_int32 * 16),
                ("mem_budget", ctypes.c_size_t), ("base_sweeps", ctypes.c_int32),
                ("poll_ticks", ctypes.c_int32), ("max_ahead", ctypes.c_int32), ("sweep_order", ctypes.c_int32)]


class ea_job(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("rid", ctypes.c_uint32), ("stream", ctypes.c_uint32),
                ("kind", ctypes.c_int32), ("recursion", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("pole", ctypes.c_double),
                ("rt_target", ctypes.c_int32), ("iter_steps", ctypes.c_int32),
                ("ticks_per_step", ctypes.c_int32), ("max_prod_ticks", ctypes.c_int32),
                ("max_requeues", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ea_srv_result(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("L", ctypes.c_int32),
                ("rid", ctypes.c_uint32), ("rt_target", ctypes.c_int32), ("n_rt", ctypes.c_int32),
                ("requeues", ctypes.c_int32), ("t_first", ctypes.c_int64), ("t_last", ctypes.c_int64),
                ("e_g", ctypes.c_int32), ("e_min", ctypes.c_int32), ("sweeps", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ea_srv_counters(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_uint64), ("ticks_read", ctypes.c_uint64), ("attempts", ctypes.c_uint64),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("done", ctypes.c_uint64), ("censored", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64), ("round_trips", ctypes.c_uint64),
                ("mem_used", ctypes.c_size_t), ("seconds", ctypes.c_double)]


EA_JOB_DONE, EA_JOB_CENSORED, EA_JOB_FAILED = 1, 2, 3

P = ctypes.c_void_p
_i, _u32, _u64, _f64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double

# name -> (restype, argtypes); the same names as include/eamc.h
SIGNATURES = {
    "ea_last_error": (ctypes.c_char_p, []),
    "ea_create": (_i, [ctypes.POINTER(P), _i, P, _u64]),
    "ea_destroy": (None, [P]),
    "ea_init_disorder": (_i, [P, _i, _i, _i, _u32, _u32, P, P, ctypes.POINTER(_i)]),
    "ea_num_chains": (_i, [P]),
    "ea_describe": (_i, [P, _i, _i, P]),
    "muca_set_ensemble": (_i, [P, _i, _i, _i, _f64, _f64, _f64]),
    "muca_set_weights": (_i, [P, _i, _i, P, _i]),
    "muca_get_weights": (_i, [P, _i, _i, P, _i]),
    "muca_set_thresholds": (_i, [P, _i, _i, P, _i]),
    "muca_get_thresholds": (_i, [P, _i, _i, P, _i]),
    "muca_set_eg": (_i, [P, _i, _i, P]),
    "muca_run_sweeps": (_i, [P, _u64, _i]),
    "muca_update_weights": (_i, [P]),
    "muca_set_recursion": (_i, [P, _i, _i, _i]),
    "muca_get_recursion_state": (_i, [P, _i, _i, P, _i]),
    "muca_build_ensemble": (_i, [P, _i, _i, _i, _f64, _f64, _f64]),
    "get_histograms": (_i, [P, _i, _i, P, _i, _i]),
    "get_roundtrips": (_i, [P, _i, _i, P, _i]),
    "get_state": (_i, [P, _i, _i, P, _i, P, P]),
    "ea_synchronize": (_i, [P]),
    "ea_check": (_i, [P]),
    "ea_snapshot_size": (_i, [P, P]),
    "ea_snapshot_save": (_i, [P, P, ctypes.c_size_t]),
    "ea_snapshot_load": (_i, [P, P, ctypes.c_size_t]),
    "muca_set_launch": (_i, [P, _i, _u64, _i]),
    "ea_reset_chains": (_i, [P, P, _i, P, P]),
    "muca_set_sweep_multiplier": (_i, [P, _i, _i]),
    "muca_set_tile_width": (_i, [P, _i, _i]),
    "muca_set_sweep_order": (_i, [P, _i, _i]),
    "muca_get_tile_width": (_i, [_i, _i, _i, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i)]),
    "muca_get_tile_width_colour": (_i, [_i, _i, _i, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i)]),
    "muca_update_weights_subset": (_i, [P, P, _i]),
    "muca_copy_weights": (_i, [P, P, P, _i]),
    "ea_graph_capture": (_i, [P, _i, _u64, _i, _i]),
    "ea_graph_launch": (_i, [P, _i]),
    "ea_graph_release": (_i, [P]),
    "muca_run_sweeps_noalloc": (_i, [_i, _i, _i, _u64, P, P, P, P, P, P, P, _u64, _u64, P]),
    "ea_srv_create": (_i, [ctypes.POINTER(P), _i, P, _u64, ctypes.POINTER(ea_srv_config)]),
    "ea_srv_destroy": (None, [P]),
    "ea_srv_submit": (_i, [P, ctypes.POINTER(ea_job), ctypes.POINTER(_u64)]),
    "ea_srv_cancel": (_i, [P, _u64]),
    "ea_srv_step": (_i, [P, _i]),
    "ea_srv_poll": (_i, [P, P, _i, ctypes.POINTER(_i), _i]),
    "ea_srv_stats": (_i, [P, ctypes.POINTER(ea_srv_counters)]),
    "ea_srv_context": (_i, [P, ctypes.POINTER(P)]),
    "ea_srv_tile_bytes": (ctypes.c_size_t, [_i, _i]),
    "pt_init": (_i, [P, _i, _i, _i, _u32, _i, P, P]),
    "pt_set_rt_bounds": (_i, [P, P, P]),
    "pt_run": (_i, [P, _u64, _i]),
    "pt_get_state": (_i, [P, P, P, P, P]),
    "pt_get_roundtrips": (_i, [P, P, _i]),
    "pt_get_swap_counts": (_i, [P, P]),
    "pt_set_betas": (_i, [P, P]),
    "pt_get_betas": (_i, [P, P]),
    "pt_get_exchange_counts": (_i, [P, P, P]),
    "pt_adapt": (_i, [P, ctypes.c_double]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libeamc.so (built in-tree by __graft_entry__.build()); raises if missing."""
    global _lib
    if _lib is None:
        if not Path(LIB).exists():
            raise ImportError(f"{LIB} is missing: build it with __graft_entry__.build()")
        _lib = ctypes.CDLL(str(LIB))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def tile_width_info(dim: int, L: int, width: int, order: int = 0):
    """(dynamic shared memory per sweep block, thresholds in shared memory?) for tiles of this
    (dim, L, width) in sweep order `order`, or None when that width is not available."""
    smem, in_smem = ctypes.c_size_t(0), ctypes.c_int(0)
    fn = lib().muca_get_tile_width_colour if order == 1 else lib().muca_get_tile_width
    if fn(dim, L, width, ctypes.byref(smem), ctypes.byref(in_smem)) != EA_OK:
        return None
    return smem.value, bool(in_smem.value)


def narrow_widths(dim: int, L: int, order: int = 0) -> list:
    """The tile widths below 32 available at (dim, L) in sweep order `order`, narrowest first."""
    return [w for w in (4, 8, 16) if tile_width_info(dim, L, w, order)]


def narrow_width(dim: int, L: int, order: int = 0) -> int:
    """The narrowest tile width available at (dim, L) in sweep order `order` (32 when there is
    no narrow one)."""
    ws = narrow_widths(dim, L, order)
    return ws[0] if ws else 32


def check(rc: int) -> int:
    if rc != EA_OK:
        raise EamcError(rc, lib().ea_last_error().decode())
    return rc


def _out(out, shape, dtype):
    """A caller's output buffer after checking it, or a new zeroed one."""
    if out is None:
        return np.zeros(shape, dtype=dtype)
    if out.shape != tuple(shape) or out.dtype != np.dtype(dtype) or not out.flags["C_CONTIGUOUS"]:
        raise ValueError(f"output buffer must be C-contiguous {np.dtype(dtype)} of shape {tuple(shape)}")
    return out


def _p(a: np.ndarray):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "buffers must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """One ea_ctx: a batch of MUCA chains resident on a CUDA device."""

    def __init__(self, seed: int, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        check(lib().ea_create(ctypes.byref(self._h), device, st, seed))
        self.seed = seed

    def close(self):
        if self._h:
            lib().ea_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # a1
    def init_disorder(self, dim: int, L: int, n: int, rid0: int = 0, stream: int = 0,
                      couplings: np.ndarray | None = None, spins: np.ndarray | None = None) -> int:
        first = ctypes.c_int(-1)
        J = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
        S = None if spins is None else np.ascontiguousarray(spins, dtype=np.int8)
        check(lib().ea_init_disorder(self._h, dim, L, n, rid0, stream, _p(J), _p(S),
                                     ctypes.byref(first)))
        return first.value

    def num_chains(self) -> int:
        return lib().ea_num_chains(self._h)

    def describe(self, chain0: int = 0, n: int | None = None):
        n = self.num_chains() - chain0 if n is None else n
        out = (ea_chain_desc * n)()
        check(lib().ea_describe(self._h, chain0, n, out))
        return [{f: getattr(d, f) for f, _ in ea_chain_desc._fields_} for d in out]

    # a5
    def set_ensemble(self, chain0: int, n: int, kind: int, alpha: float = -3.6,
                     pole: float = 96.0, beta: float = 1.0):
        check(lib().muca_set_ensemble(self._h, chain0, n, kind, alpha, pole, beta))

    def build_ensemble(self, chain0: int, n: int, kind: int, alpha: float = -3.6,
                       pole: float = 96.0, beta: float = 1.0):
        check(lib().muca_build_ensemble(self._h, chain0, n, kind, alpha, pole, beta))

    def _rows(self, chain0, n):
        return max(d["b_top"] for d in self.describe(chain0, n)) + 1

    def set_weights(self, chain0: int, lnW: np.ndarray):
        lnW = np.ascontiguousarray(np.atleast_2d(lnW), dtype=np.float64)
        check(lib().muca_set_weights(self._h, chain0, lnW.shape[0], _p(lnW), lnW.shape[1]))

    def get_weights(self, chain0: int = 0, n: int | None = None, rows: int | None = None, out=None):
        """ln W rows; `out` (float64 [n, rows], e.g. in pinned memory) is filled when given."""
        n = self.num_chains() - chain0 if n is None else n
        rows = self._rows(chain0, n) if rows is None else rows
        out = _out(out, (n, rows), np.float64)
        check(lib().muca_get_weights(self._h, chain0, n, _p(out), rows))
        return out

    def set_thresholds(self, chain0: int, thr: np.ndarray):
        thr = np.ascontiguousarray(np.atleast_2d(thr), dtype=np.uint32)
        check(lib().muca_set_thresholds(self._h, chain0, thr.shape[0], _p(thr), thr.shape[1]))

    def get_thresholds(self, chain0: int = 0, n: int | None = None, rows: int | None = None):
        n = self.num_chains() - chain0 if n is None else n
        rows = self._rows(chain0, n) if rows is None else rows
        out = np.zeros((n, rows * 8), dtype=np.uint32)
        check(lib().muca_get_thresholds(self._h, chain0, n, _p(out), rows * 8))
        return out

    def set_eg(self, chain0: int, n: int, e_g: np.ndarray | None = None):
        arr = None if e_g is None else np.ascontiguousarray(e_g, dtype=np.int32)
        check(lib().muca_set_eg(self._h, chain0, n, _p(arr)))

    # a2 + a3
    def run_sweeps(self, n_sweeps: int, count_roundtrips: bool = False):
        check(lib().muca_run_sweeps(self._h, n_sweeps, int(count_roundtrips)))

    # a4
    def update_weights(self):
        check(lib().muca_update_weights(self._h))

    # f1
    def set_recursion(self, chain0: int, n: int, mode: int):
        check(lib().muca_set_recursion(self._h, chain0, n, mode))

    def recursion_state(self, chain0: int = 0, n: int | None = None, rows: int | None = None):
        """Berg accumulators as float64 [n, rows, 2] = (D, G) per bin."""
        n = self.num_chains() - chain0 if n is None else n
        rows = self._rows(chain0, n) if rows is None else rows
        out = np.zeros((n, rows, 2), dtype=np.float64)
        check(lib().muca_get_recursion_state(self._h, chain0, n, _p(out), 2 * rows))
        return out

    def histograms(self, chain0: int = 0, n: int | None = None, reset: bool = False,
                   rows: int | None = None, out=None):
        n = self.num_chains() - chain0 if n is None else n
        rows = self._rows(chain0, n) if rows is None else rows
        out = _out(out, (n, rows), np.uint32)
        check(lib().get_histograms(self._h, chain0, n, _p(out), rows, int(reset)))
        return out

    def roundtrips(self, chain0: int = 0, n: int | None = None, reset: bool = False):
        return [{f: r[f].item() for f in RT_DTYPE.names if f != "pad"}
                for r in self.roundtrips_array(chain0, n, reset)]

    def roundtrips_array(self, chain0: int = 0, n: int | None = None, reset: bool = False, out=None):
        """Round-trip records as a numpy structured array (fields of ea_rt_stats)."""
        n = self.num_chains() - chain0 if n is None else n
        out = _out(out, (n,), RT_DTYPE)
        check(lib().get_roundtrips(self._h, chain0, n, _p(out), int(reset)))
        return out

    def state(self, chain0: int = 0, n: int | None = None, spins: bool = True):
        n = self.num_chains() - chain0 if n is None else n
        descs = self.describe(chain0, n)
        V = max(d["L"] ** d["dim"] for d in descs)
        S = np.zeros((n, V), dtype=np.int8) if spins else None
        E = np.zeros(n, dtype=np.int32)
        t = np.zeros(n, dtype=np.uint64)
        check(lib().get_state(self._h, chain0, n, _p(S), V, _p(E), _p(t)))
        return S, E, t

    def check(self):
        """Raises EamcError if a sweep broke an invariant since the last check."""
        check(lib().ea_check(self._h))

    def synchronize(self):
        check(lib().ea_synchronize(self._h))

    # checkpoint / resume
    def snapshot(self) -> bytes:
        n = ctypes.c_size_t(0)
        check(lib().ea_snapshot_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(lib().ea_snapshot_save(self._h, buf, n.value))
        return buf.raw

    def restore(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        check(lib().ea_snapshot_load(self._h, buf, len(data)))

    # a9: serving support
    def reset_chains(self, chains, rids, streams):
        c = np.ascontiguousarray(chains, dtype=np.int32)
        r = np.ascontiguousarray(rids, dtype=np.uint32)
        s = np.ascontiguousarray(streams, dtype=np.uint32)
        check(lib().ea_reset_chains(self._h, _p(c), c.shape[0], _p(r), _p(s)))

    def set_sweep_order(self, order: int, chains_per_cta: int = 0):
        """EA_ORDER_LEX or EA_ORDER_COLOUR for every chain of the context (see the header)."""
        check(lib().muca_set_sweep_order(self._h, order, chains_per_cta))

    def set_tile_width(self, L: int, width: int):
        """Chains per tile (32, or 16 for L = 7, 8 in 3D) for chains of size L added
        afterwards."""
        check(lib().muca_set_tile_width(self._h, L, width))

    def set_sweep_multiplier(self, L: int, multiplier: int):
        check(lib().muca_set_sweep_multiplier(self._h, L, multiplier))

    def copy_weights(self, src, dst):
        a = np.ascontiguousarray(src, dtype=np.int32)
        b = np.ascontiguousarray(dst, dtype=np.int32)
        assert a.shape == b.shape
        check(lib().muca_copy_weights(self._h, _p(a), _p(b), a.shape[0]))

    def update_weights_subset(self, chains):
        c = np.ascontiguousarray(chains, dtype=np.int32)
        check(lib().muca_update_weights_subset(self._h, _p(c), c.shape[0]))

    # a8: launch configuration and the captured iteration graph
    def set_launch(self, persistent: bool = False, sweeps_per_launch: int = 0,
                   blocks_per_sm: int = 0):
        check(lib().muca_set_launch(self._h, int(persistent), sweeps_per_launch, blocks_per_sm))

    def graph_capture(self, n_iter: int, sweeps_per_iter: int, count_roundtrips: bool = False,
                      update_weights: bool = True):
        check(lib().ea_graph_capture(self._h, n_iter, sweeps_per_iter, int(count_roundtrips),
                                     int(update_weights)))

    def graph_launch(self, replays: int = 1):
        check(lib().ea_graph_launch(self._h, replays))

    def graph_release(self):
        check(lib().ea_graph_release(self._h))

    # a6 + a7: parallel tempering
    def pt_init(self, dim: int, L: int, n_real: int, betas, rid0: int = 0,
                couplings: np.ndarray | None = None):
        b = np.ascontiguousarray(betas, dtype=np.float64)
        J = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
        check(lib().pt_init(self._h, dim, L, n_real, rid0, b.shape[0], _p(b), _p(J)))
        self._pt = (dim, L, n_real, b.shape[0])

    def pt_set_rt_bounds(self, e_g, e_hot):
        eg = np.ascontiguousarray(e_g, dtype=np.int32)
        eh = np.ascontiguousarray(e_hot, dtype=np.int32)
        check(lib().pt_set_rt_bounds(self._h, _p(eg), _p(eh)))

    def pt_run(self, n_sweeps: int, count_roundtrips: bool = False):
        check(lib().pt_run(self._h, n_sweeps, int(count_roundtrips)))

    def pt_state(self, spins: bool = True):
        dim, L, n, M = self._pt
        V = L ** dim
        S = np.zeros((n, M, V), dtype=np.int8) if spins else None
        E = np.zeros((n, M), dtype=np.int32)
        lab = np.zeros((n, M), dtype=np.int32)
        t = ctypes.c_uint64(0)
        check(lib().pt_get_state(self._h, _p(S), _p(E), _p(lab), ctypes.byref(t)))
        return S, E, lab, t.value

    def pt_roundtrips(self, reset: bool = False):
        dim, L, n, M = self._pt
        out = (ea_pt_stats * (n * M))()
        check(lib().pt_get_roundtrips(self._h, out, int(reset)))
        return [[{f: getattr(out[r * M + l], f) for f, _ in ea_pt_stats._fields_ if f != "pad"}
                 for l in range(M)] for r in range(n)]

    def pt_swap_counts(self):
        M = self._pt[3]
        out = np.zeros(M - 1, dtype=np.uint64)
        check(lib().pt_get_swap_counts(self._h, _p(out)))
        return out

    # f2: per-realization temperatures and the constant-exchange-rate adaptation
    def pt_set_betas(self, betas):
        dim, L, n, M = self._pt
        b = np.ascontiguousarray(betas, dtype=np.float64)
        assert b.shape == (n, M)
        check(lib().pt_set_betas(self._h, _p(b)))

    def pt_betas(self):
        dim, L, n, M = self._pt
        out = np.zeros((n, M), dtype=np.float64)
        check(lib().pt_get_betas(self._h, _p(out)))
        return out

    def pt_exchange_counts(self):
        dim, L, n, M = self._pt
        acc = np.zeros((n, M - 1), dtype=np.uint32)
        att = np.zeros(M - 1, dtype=np.uint64)
        check(lib().pt_get_exchange_counts(self._h, _p(acc), _p(att)))
        return acc, att

    def pt_adapt(self, eta: float = 0.5):
        check(lib().pt_adapt(self._h, eta))
