"""muca_run_sweeps_noalloc, the entry point for callers that cannot allocate device memory
(code inside another framework's memory pool or under a fixed device-memory budget, plugins
that may only touch the buffers they are handed), gives exactly what the context path
(ea_init_disorder / muca_set_thresholds / muca_run_sweeps) gives, on two calls in a row that
continue one trajectory, and allocates nothing while doing so.

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


class Case:
    """n chains of L^3 set up identically in a context and as caller-owned device buffers."""

    def __init__(self, eamc, orc, L, n, rid0=900, walls=True):
        import torch
        dim = self.dim = 3
        self.L, self.n, self.V = L, n, L ** dim
        self.B = ((dim * self.V) // 2 >> 1) + 1
        rng = np.random.default_rng(L + 17 * n)
        J = np.stack([orc.make_disorder(dim, L, 123, rid0 + k) for k in range(n)]).astype(np.int8)
        self.ctx = eamc.Context(seed=SEED)
        self.ctx.init_disorder(dim, L, n, rid0=rid0, stream=3, couplings=J)
        rows = max(d["b_top"] for d in self.ctx.describe()) + 1
        # weights with structure -> thresholds from the library's own quantisation
        lnW = np.cumsum(rng.normal(0.2, 0.3, size=(n, rows))[:, ::-1], axis=1)[:, ::-1].copy()
        lnW -= lnW[:, -1:]
        self.ctx.set_weights(0, lnW)
        thr = self.ctx.get_thresholds(rows=rows)
        thr_full = np.zeros((n, self.B * 8), np.uint32)
        thr_full[:, :thr.shape[1]] = thr
        if not walls:
            # a table without walls: every move "always" where the library wrote 0 for a move
            # out of the range (both paths must reject those moves anyway)
            thr_full[thr_full == 0] = 0xFFFFFFFF
            self.ctx.set_thresholds(0, thr_full[:, :rows * 8].copy())
        S0, _, _ = self.ctx.state()
        dev = torch.device("cuda:0")
        self.t_rid = torch.tensor(np.arange(rid0, rid0 + n, dtype=np.uint32).view(np.int32), device=dev)
        self.t_stream = torch.full((n,), 3, dtype=torch.int32, device=dev)
        self.t_J = torch.tensor(J, device=dev)
        self.t_S = torch.tensor(S0[:, :self.V].copy(), device=dev)
        self.t_E = torch.zeros(n, dtype=torch.int32, device=dev)
        self.t_thr = torch.tensor(thr_full.view(np.int32), device=dev)
        self.t_hist = torch.zeros((n, self.B), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()

    def call(self, eamc, t0, sweeps):
        return eamc.lib().muca_run_sweeps_noalloc(
            self.dim, self.L, self.n, SEED, _ptr(self.t_rid), _ptr(self.t_stream), _ptr(self.t_J),
            _ptr(self.t_S), _ptr(self.t_E), _ptr(self.t_thr), _ptr(self.t_hist), t0, sweeps, None)

    def check_equal(self, t0):
        S, E, t = self.ctx.state()
        H = self.ctx.histograms(rows=self.B)
        assert np.array_equal(self.t_S.cpu().numpy(), S[:, :self.V])
        assert np.array_equal(self.t_E.cpu().numpy(), E)
        assert np.array_equal(self.t_hist.cpu().numpy().view(np.uint32), H)
        assert (t == t0).all()


@pytest.mark.parametrize("L,n,walls", [(6, 40, True), (7, 9, True), (5, 33, False)])
def test_noalloc_matches_context_path(eamc, orc, L, n, walls):
    c = Case(eamc, orc, L, n, walls=walls)
    t0 = 0
    for sweeps in (37, 25):                       # two calls in a row
        rc = c.call(eamc, t0, sweeps)
        assert rc == 0, eamc.lib().ea_last_error()
        c.ctx.run_sweeps(sweeps)
        t0 += sweeps
        c.check_equal(t0)
    assert c.ctx.check() is None                  # the context's chains stayed in range
    c.ctx.close()


def test_noalloc_allocates_nothing(eamc, orc):
    """After a first call, further calls leave the device's free memory unchanged."""
    import torch
    c = Case(eamc, orc, 6, 64)
    assert c.call(eamc, 0, 10) == 0, eamc.lib().ea_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(3):
        assert c.call(eamc, 10 + 10 * k, 10) == 0, eamc.lib().ea_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    c.ctx.close()


def test_noalloc_refused_chain_writes_nothing(eamc, orc):
    """One chain above E_top among valid ones: EA_EINVAL, no sweep runs and no output buffer
    changes, so the corrected call then continues from the same t0 exactly as the context."""
    import torch
    c = Case(eamc, orc, 6, 40)
    good_S = c.t_S.clone()
    bad = c.t_S.clone()
    # chain 17 starts from a configuration above E_top: greedy ascent (flip while E rises)
    J17 = c.t_J[17].cpu().numpy()
    S = np.ones(c.V, np.int8)
    E = orc.energy(3, 6, J17, S)
    while E <= 0:
        for i in range(c.V):
            S[i] = -S[i]
            e = orc.energy(3, 6, J17, S)
            if e > E:
                E = e
            else:
                S[i] = -S[i]
    bad[17] = torch.from_numpy(S).to(bad.device)
    c.t_S.copy_(bad)
    c.t_E.fill_(12345)
    c.t_hist.fill_(7)
    rc = c.call(eamc, 0, 20)
    assert rc == eamc.EA_EINVAL
    assert b"E_top" in eamc.lib().ea_last_error()
    assert (c.t_E == 12345).all() and (c.t_hist == 7).all()
    assert (c.t_S == bad).all()
    # fixed input, same t0: identical to the context path
    c.t_S.copy_(good_S)
    c.t_E.zero_()
    c.t_hist.zero_()
    assert c.call(eamc, 0, 20) == 0, eamc.lib().ea_last_error()
    c.ctx.run_sweeps(20)
    c.check_equal(20)
    c.ctx.close()


def test_noalloc_rejects_oversize(eamc):
    """256 chains of L=12 do not fit the static scratch array: a clear error, nothing runs."""
    import torch
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda:0")
    p = _ptr(dummy)
    rc = eamc.lib().muca_run_sweeps_noalloc(3, 12, 256, 1, p, p, p, p, p, p, p, 0, 1, None)
    assert rc == eamc.EA_EINVAL
    assert b"scratch" in eamc.lib().ea_last_error()
    assert (dummy == 0).all()
    # a sweep range that would wrap the 32-bit sweep counter is refused as well
    rc = eamc.lib().muca_run_sweeps_noalloc(3, 4, 1, 1, p, p, p, p, p, p, p, (1 << 64) - 8, 16, None)
    assert rc == eamc.EA_EINVAL
    assert (dummy == 0).all()
