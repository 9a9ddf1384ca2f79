"""muca_run_sweeps_noalloc, the entry point for callers that cannot allocate device memory,
gives exactly what the context path (ea_init_disorder / muca_set_thresholds /
muca_run_sweeps) gives, on two calls in a row that continue one trajectory.

This file is collected last so that a stop at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 77


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("L,n", [(6, 40), (7, 9)])
def test_noalloc_matches_context_path(eamc, orc, L, n):
    import torch
    dim = 3
    V = L ** dim
    rng = np.random.default_rng(L)
    J = np.stack([orc.make_disorder(dim, L, 123, 900 + k) for k in range(n)]).astype(np.int8)
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=900, stream=3, couplings=J)
    # weights with structure -> thresholds from the library's own quantisation
    rows = max(d["b_top"] for d in ctx.describe()) + 1
    lnW = np.cumsum(rng.normal(0.2, 0.3, size=(n, rows))[:, ::-1], axis=1)[:, ::-1].copy()
    lnW -= lnW[:, -1:]
    ctx.set_weights(0, lnW)
    thr = ctx.get_thresholds(rows=rows)
    S0, E0, _ = ctx.state()
    dev = torch.device("cuda:0")
    B = ((dim * V) // 2 >> 1) + 1
    assert rows == B or rows == B - 1
    thr_full = np.zeros((n, B * 8), np.uint32)
    thr_full[:, :thr.shape[1]] = thr
    t_rid = torch.tensor(np.arange(900, 900 + n, dtype=np.uint32).view(np.int32), device=dev)
    t_stream = torch.full((n,), 3, dtype=torch.int32, device=dev)
    t_J = torch.tensor(J, device=dev)
    t_S = torch.tensor(S0[:, :V].copy(), device=dev)
    t_E = torch.zeros(n, dtype=torch.int32, device=dev)
    t_thr = torch.tensor(thr_full.view(np.int32), device=dev)
    t_hist = torch.zeros((n, B), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = 0
    for sweeps in (37, 25):                       # two calls in a row
        rc = eamc.lib().muca_run_sweeps_noalloc(
            dim, L, n, SEED, _ptr(t_rid), _ptr(t_stream), _ptr(t_J), _ptr(t_S), _ptr(t_E),
            _ptr(t_thr), _ptr(t_hist), t0, sweeps, None)
        assert rc == 0, eamc.lib().ea_last_error()
        ctx.run_sweeps(sweeps)
        t0 += sweeps
        S, E, t = ctx.state()
        H = ctx.histograms(rows=B)
        assert np.array_equal(t_S.cpu().numpy(), S[:, :V])
        assert np.array_equal(t_E.cpu().numpy(), E)
        assert np.array_equal(t_hist.cpu().numpy().view(np.uint32), H)
        assert (t == t0).all()


def test_noalloc_rejects_oversize(eamc):
    """256 chains of L=12 do not fit the static scratch array: a clear error, nothing runs."""
    import torch
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda:0")
    p = _ptr(dummy)
    rc = eamc.lib().muca_run_sweeps_noalloc(3, 12, 256, 1, p, p, p, p, p, p, p, 0, 1, None)
    assert rc == eamc.EA_EINVAL
    assert b"scratch" in eamc.lib().ea_last_error()
    assert (dummy == 0).all()
