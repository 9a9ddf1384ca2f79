"""CPU oracle for generalized-ensemble Monte Carlo on the 3D (and 2D) +-J EA spin glass.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs import this package.  It shares no code with the
CUDA library in ``paper_2011_08560_gb300``: the arithmetic lives in ``eamc_oracle.c``
(plain C, one chain at a time, spins as +-1 integers) and this module only marshals numpy
arrays into it.

What each function follows (Mueller, Schnabel, Janke, arXiv:2011.08560):
  energy / disorder .......... Sec. II, Eq. "hamiltonian"; 3V couplings +-1 with p = 1/2
  muca_sweeps ................ Sec. II, Eq. "muca" (generalized Metropolis, sequential; sites
                               lexicographic or colour class by colour class)
  quantize ................... Eq. "muca": P_acc = min(1, W(E_new)/W(E_old)) as a u32 threshold
  ln_profile ................. Eq. "power_law" (normalised to 1 at E = 0)
  update_weights ............. Sec. II, the iterative weight procedure (W <- W P_SH / H)
  update_weights_berg ........ Sec. II / Janke 2003: Berg's accumulated error-weighted recursion
  build_weights .............. Eq. "muca-weights", nonflat weight, Eq. "1/k", canonical
  pt_tables / pt_sweeps ...... Sec. II, parallel tempering and Eq. "temperatureexchange"
  pt_colour .................. sweep order of PT (checkerboard for even L, 3 colours for odd L)
  pt_adapt ................... Sec. II, PT: constant exchange rates by moving the temperatures
  round trips ................ Sec. III (top -> E_g -> top, times in sweeps)
  dos_bruteforce ............. exact g(E) by enumeration (used to pin the chain)

Parity pins live in ``tests/test_oracle_*.py``.  Two things have no pin ("parity unpinned"):
absolute round-trip times, and agreement with the authors' own weight recursion.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "eamc_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libeamc_oracle.so"

ALWAYS = 0xFFFFFFFF
FLAT, POWERLAW, ONE_OVER_K, CANON = 0, 1, 2, 3


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no GPU, no CUDA)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"libeamc_oracle.{os.getpid()}.so"
        # -ffp-contract=off: every expression is evaluated as written (no fused multiply-add),
        # so the oracle gives the same numbers on x86-64 and on AArch64
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(_SRC),
                               "-o", str(tmp), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class RT(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("n_rt", ctypes.c_int32),
                ("t_first", ctypes.c_int64), ("t_last", ctypes.c_int64),
                ("e_min", ctypes.c_int32), ("e_g", ctypes.c_int32),
                ("requeue", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        P = ctypes.c_void_p
        i32, u32, u64, f64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        sig = {
            "or_philox4x32_10": (None, [P, P, P]),
            "or_volume": (i32, [i32, i32]),
            "or_nbonds": (i32, [i32, i32]),
            "or_make_disorder": (None, [i32, i32, u64, u32, P]),
            "or_make_spins": (None, [i32, i32, u64, u32, u32, P]),
            "or_energy": (i32, [i32, i32, P, P]),
            "or_parity": (i32, [i32, i32, P]),
            "or_bin_of_energy": (i32, [i32, i32, i32]),
            "or_energy_of_bin": (i32, [i32, i32, i32, i32]),
            "or_btop": (i32, [i32, i32, i32]),
            "or_descend": (i32, [i32, i32, P, P, i32, P]),
            "or_muca_sweeps": (i32, [i32, i32, u64, u32, u32, P, P, P, u64, u64, P, i32, P,
                                     P, i32, P, P]),
            "or_rt_replay": (None, [P, P, i32, i32, i32, P]),
            "or_muca_sweeps_order": (i32, [i32, i32, u64, u32, u32, P, P, P, u64, u64, P, i32, P,
                                           P, i32, P, P, i32]),
            "or_quantize": (None, [i32, i32, P, P]),
            "or_ln_profile": (f64, [i32, f64, f64, i32, i32]),
            "or_update_weights": (None, [i32, i32, i32, i32, i32, f64, f64, i32, P, P]),
            "or_update_weights_berg": (None, [i32, i32, i32, i32, i32, f64, f64, i32, P, P, P, P]),
            "or_build_weights": (None, [i32, i32, i32, i32, i32, f64, f64, f64, i32, P, P]),
            "or_pt_tables": (None, [i32, i32, P, i32, P, P]),
            "or_pt_colours": (i32, [i32]),
            "or_pt_colour": (i32, [i32, i32, i32]),
            "or_pt_adapt": (None, [i32, P, P, P, f64]),
            "or_pt_sweeps": (i32, [i32, i32, u64, u32, i32, P, P, P, P, u64, u64, P, P, i32,
                                   P, i32, i32, i32, P, P]),
            "or_dos_bruteforce": (i32, [i32, i32, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def volume(dim: int, L: int) -> int:
    return lib().or_volume(dim, L)


def nbonds(dim: int, L: int) -> int:
    return lib().or_nbonds(dim, L)


def make_disorder(dim: int, L: int, seed: int, rid: int) -> np.ndarray:
    J = np.zeros(nbonds(dim, L), dtype=np.int8)
    lib().or_make_disorder(dim, L, seed, rid, _p(J))
    return J


def make_spins(dim: int, L: int, seed: int, rid: int, stream: int = 0) -> np.ndarray:
    S = np.zeros(volume(dim, L), dtype=np.int8)
    lib().or_make_spins(dim, L, seed, rid, stream, _p(S))
    return S


def energy(dim: int, L: int, J: np.ndarray, S: np.ndarray) -> int:
    return lib().or_energy(dim, L, _p(J), _p(S))


def parity(dim: int, L: int, J: np.ndarray) -> int:
    return lib().or_parity(dim, L, _p(J))


def bin_of_energy(dim: int, L: int, E: int) -> int:
    return lib().or_bin_of_energy(dim, L, E)


def energy_of_bin(dim: int, L: int, par: int, b: int) -> int:
    return lib().or_energy_of_bin(dim, L, par, b)


def btop(dim: int, L: int, par: int) -> int:
    return lib().or_btop(dim, L, par)


def descend(dim: int, L: int, J: np.ndarray, S: np.ndarray, e_top: int) -> int:
    E = np.array([energy(dim, L, J, S)], dtype=np.int32)
    rc = lib().or_descend(dim, L, _p(J), _p(S), e_top, _p(E))
    if rc != 0:
        raise RuntimeError("descent stuck in a local minimum above E_top")
    return int(E[0])


def quantize(dim: int, lnW: np.ndarray) -> np.ndarray:
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    b_top = lnW.shape[0] - 1
    thr = np.zeros((b_top + 1) * 8, dtype=np.uint32)
    lib().or_quantize(dim, b_top, _p(lnW), _p(thr))
    return thr


def ln_profile(kind: int, alpha: float, pole: float, e_g: int, E: int) -> float:
    return lib().or_ln_profile(kind, alpha, pole, e_g, E)


def update_weights(dim, L, par, kind, alpha, pole, e_g, lnW, hist) -> np.ndarray:
    lnW = np.ascontiguousarray(lnW, dtype=np.float64).copy()
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    lib().or_update_weights(dim, L, par, lnW.shape[0] - 1, kind, alpha, pole, e_g, _p(lnW),
                            _p(hist))
    return lnW


def berg_state(n_bins: int) -> np.ndarray:
    """Accumulators of the Berg recursion: row 0 = D (weighted mean of the ln Omega
    differences of neighbouring bins), row 1 = G (sum of their weights); both start at 0."""
    return np.zeros((2, n_bins), dtype=np.float64)


def update_weights_berg(dim, L, par, kind, alpha, pole, e_g, lnW, hist, acc) -> np.ndarray:
    """One step of the accumulated recursion; `acc` (from berg_state) is updated in place."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64).copy()
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    assert acc.dtype == np.float64 and acc.flags.c_contiguous and acc.shape == (2, lnW.shape[0])
    lib().or_update_weights_berg(dim, L, par, lnW.shape[0] - 1, kind, alpha, pole, e_g, _p(lnW),
                                 _p(hist), _p(acc[0]), _p(acc[1]))
    return lnW


def build_weights(dim, L, par, kind, alpha, pole, beta, e_g, lnOmega) -> np.ndarray:
    lnOmega = np.ascontiguousarray(lnOmega, dtype=np.float64)
    lnW = np.zeros_like(lnOmega)
    lib().or_build_weights(dim, L, par, lnW.shape[0] - 1, kind, alpha, pole, beta, e_g,
                           _p(lnOmega), _p(lnW))
    return lnW


def rt_replay(energies, times, e_top: int, e_bottom: int, rt: RT | None = None) -> RT:
    """Runs the oracle's round-trip check (Sec. III) once per element of `energies`, observed
    at sweep indices `times`, starting from `rt` (default: a fresh record, phase 0)."""
    E = np.ascontiguousarray(energies, dtype=np.int32)
    t = np.ascontiguousarray(times, dtype=np.int64)
    assert E.shape == t.shape and E.ndim == 1
    if rt is None:
        rt = RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=0, e_g=e_bottom, requeue=0, pad=0)
    lib().or_rt_replay(_p(E), _p(t), E.shape[0], e_top, e_bottom, ctypes.byref(rt))
    return rt


def dos_bruteforce(dim: int, L: int, J: np.ndarray) -> np.ndarray:
    g = np.zeros(nbonds(dim, L) + 1, dtype=np.uint64)
    if lib().or_dos_bruteforce(dim, L, _p(J), _p(g)) != 0:
        raise ValueError("lattice too large to enumerate")
    return g


# ------------------------------------------------------------------------- one MUCA chain
class Chain:
    """One MUCA chain (one realization, one RNG stream) advanced by the C oracle."""

    def __init__(self, dim: int, L: int, seed: int, rid: int, stream: int = 0,
                 J: np.ndarray | None = None, S: np.ndarray | None = None,
                 descend_to_top: bool = True, order: int = 0):
        """order: 0 lexicographic sweeps, 1 colour class by colour class (or_muca_sweeps_order)."""
        self.dim, self.L, self.seed, self.rid, self.stream = dim, L, seed, rid, stream
        self.order = order
        self.V, self.nb = volume(dim, L), nbonds(dim, L)
        self.J = make_disorder(dim, L, seed, rid) if J is None else np.ascontiguousarray(J, np.int8)
        self.S = make_spins(dim, L, seed, rid, stream) if S is None else np.ascontiguousarray(S, np.int8).copy()
        self.parity = parity(dim, L, self.J)
        self.b_top = btop(dim, L, self.parity)
        self.e_top = energy_of_bin(dim, L, self.parity, self.b_top)
        self.E = energy(dim, L, self.J, self.S)
        if descend_to_top:
            self.E = descend(dim, L, self.J, self.S, self.e_top)
        self.t = 0
        self.hist = np.zeros(self.b_top + 1, dtype=np.uint32)
        self.rt = RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=self.E, e_g=-(1 << 30),
                     requeue=0, pad=0)

    def sweeps(self, n: int, thr: np.ndarray, count_rt: bool = False, trace: bool = False,
               attempt_trace: bool = False):
        """n sweeps; returns the energy after each sweep (trace=True), the energy after each
        attempt as an (n, V) array (attempt_trace=True), both as a tuple, or None."""
        thr = np.ascontiguousarray(thr, dtype=np.uint32)
        assert thr.shape[0] >= (self.b_top + 1) * 8
        E = np.array([self.E], dtype=np.int32)
        tr = np.zeros(n, dtype=np.int32) if trace else None
        at = np.zeros((n, self.V), dtype=np.int32) if attempt_trace else None
        lib().or_muca_sweeps_order(self.dim, self.L, self.seed, self.rid, self.stream, _p(self.J),
                                   _p(self.S), _p(E), self.t, n, _p(thr), self.b_top, _p(self.hist),
                                   ctypes.byref(self.rt), int(count_rt),
                                   _p(tr) if trace else None, _p(at) if attempt_trace else None,
                                   self.order)
        self.E = int(E[0])
        self.t += n
        if trace and attempt_trace:
            return tr, at
        return at if attempt_trace else tr


# ------------------------------------------------------------------------- PT
def pt_tables(dim: int, betas, dmax: int):
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    M = betas.shape[0]
    thr_k = np.zeros(M * 8, dtype=np.uint32)
    thr_pair = np.zeros(max(M - 1, 1) * (dmax + 1), dtype=np.uint32)
    lib().or_pt_tables(dim, M, _p(betas), dmax, _p(thr_k), _p(thr_pair))
    return thr_k, thr_pair


def pt_colour(dim: int, L: int, i: int) -> int:
    return lib().or_pt_colour(dim, L, i)


def pt_colours(L: int) -> int:
    return lib().or_pt_colours(L)


def pt_attempts(M: int, t0: int, t1: int) -> np.ndarray:
    """Exchange attempts of each pair (k, k+1) in sweeps t0..t1-1 (pair k is tried when
    t = k mod 2)."""
    n = t1 - t0
    out = np.zeros(max(M - 1, 1), dtype=np.uint64)
    for k in range(M - 1):
        first = t0 + ((k - t0) % 2)          # first t >= t0 with t = k (mod 2)
        out[k] = 0 if first >= t1 else (t1 - 1 - first) // 2 + 1
    return out


def pt_adapt(betas, n_acc, n_att, eta: float) -> np.ndarray:
    b = np.ascontiguousarray(betas, dtype=np.float64).copy()
    acc = np.ascontiguousarray(n_acc, dtype=np.uint64)
    att = np.ascontiguousarray(n_att, dtype=np.uint64)
    lib().or_pt_adapt(b.shape[0], _p(b), _p(acc), _p(att), eta)
    return b


class PTRealization:
    """M replicas of one realization under parallel tempering, advanced by the oracle."""

    def __init__(self, dim: int, L: int, seed: int, rid: int, betas,
                 J: np.ndarray | None = None):
        self.dim, self.L, self.seed, self.rid = dim, L, seed, rid
        self.V, self.nb = volume(dim, L), nbonds(dim, L)
        self.betas = np.ascontiguousarray(betas, dtype=np.float64)
        self.M = self.betas.shape[0]
        self.J = make_disorder(dim, L, seed, rid) if J is None else np.ascontiguousarray(J, np.int8)
        self.S = np.concatenate([make_spins(dim, L, seed, rid, stream=k) for k in range(self.M)])
        self.E = np.array([energy(dim, L, self.J, self.S[k * self.V:(k + 1) * self.V])
                           for k in range(self.M)], dtype=np.int32)
        self.label = np.arange(self.M, dtype=np.int32)
        self.dmax = self.nb // 2
        self.thr_k, self.thr_pair = pt_tables(dim, self.betas, self.dmax)
        self.t = 0
        self.rt = (RT * self.M)()
        for k in range(self.M):
            self.rt[k].t_first = -1
            self.rt[k].t_last = -1
            self.rt[k].e_min = int(self.E[k])
        self.swap_acc = np.zeros(max(self.M - 1, 1), dtype=np.uint64)
        self._win_t, self._win_acc = 0, self.swap_acc.copy()

    def set_betas(self, betas):
        self.betas = np.ascontiguousarray(betas, dtype=np.float64)
        self.thr_k, self.thr_pair = pt_tables(self.dim, self.betas, self.dmax)

    def window_rates(self):
        """(accepted, attempted) exchanges per pair since the last adapt()."""
        return self.swap_acc - self._win_acc, pt_attempts(self.M, self._win_t, self.t)

    def adapt(self, eta: float):
        acc, att = self.window_rates()
        self.set_betas(pt_adapt(self.betas, acc, att, eta))
        self._win_t, self._win_acc = self.t, self.swap_acc.copy()

    def sweeps(self, n: int, count_rt: bool = False, e_g: int = 0, e_hot: int = 0,
               label_trace: bool = False):
        """n PT sweeps; with label_trace=True returns the (n, M) energies of each replica
        label after every sweep's exchanges."""
        lt = np.zeros((n, self.M), dtype=np.int32) if label_trace else None
        rc = lib().or_pt_sweeps(self.dim, self.L, self.seed, self.rid, self.M, _p(self.J),
                                _p(self.S), _p(self.E), _p(self.label), self.t, n,
                                _p(self.thr_k), _p(self.thr_pair), self.dmax, self.rt,
                                int(count_rt), e_g, e_hot, _p(self.swap_acc),
                                _p(lt) if label_trace else None)
        if rc != 0:
            raise ValueError("or_pt_sweeps failed")
        self.t += n
        return lt
