"""Batching around the sweep (GPU): one-launch setup of problems of uneven n,
concurrent applications as one CUDA graph, graph replay, the chunk-length
autotuner and its cache, and bounded-wait failure reporting.

The batched setup runs the same per-item code as the single-problem setup,
and the graphs replay the same kernels, so their results must be bit-identical
to the direct path; the direct path itself is held to the oracle.
"""
import os

import numpy as np
import pytest

from oracle import sweep2d as S
from paper_1007_4291_gb300 import build as B
from paper_1007_4291_gb300 import hs
from paper_1007_4291_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_PML = 20.0
C_MOVING = None      # library default: the moving PMLs take the boundary C (Eq. helma reuses sigma_2)
BP = 6


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    B.build()
    return hs.load()


def opts(**kw):
    base = dict(alpha=2.0, pml_C=C_PML, layers_per_step=3, chunk=8, max_nrhs=4)
    base.update(kw)
    return hs.hs_default_options(**base)


def omega_of(n):
    return 2 * np.pi * (n + 1) / 16.0


def relerr(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def apply_direct(plan, r, nrhs):
    z = torch.empty_like(r)
    hs.hs_apply(plan, r, z, nrhs, hs.HS_C64)
    torch.cuda.synchronize()
    assert hs.hs_last_device_status(plan) == hs.HS_OK
    return z


NS = [31, 45, 63, 47]   # uneven sizes in one batch


def test_batched_setup_matches_single_setup_and_oracle():
    cs = [I.random_velocity(n, 100 + k) for k, n in enumerate(NS)]
    plans = hs.hs_setup_batched([c.ravel() for c in cs], [omega_of(n) for n in NS], NS, 2, BP, BP, opts())
    singles = [hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(graphs=0)) for c, n in zip(cs, NS)]
    try:
        for k, n in enumerate(NS):
            r = I.random_rhs(n, 2, 7 + k)
            rg = torch.from_numpy(r).to("cuda").to(torch.complex64)
            zb = apply_direct(plans[k], rg, 2).cpu().numpy()
            zs = apply_direct(singles[k], rg, 2).cpu().numpy()
            assert np.array_equal(zb, zs), n          # same per-item arithmetic
            st = S.setup(cs[k], omega_of(n), BP, BP, 3, 2.0, C_PML, Cm=C_MOVING)
            ref = S.apply(st, r.astype(np.complex64).astype(np.complex128))
            assert relerr(zb.astype(np.complex128), ref) <= 1e-4, n
    finally:
        for p in plans + singles:
            hs.hs_destroy(p)


def test_batched_setup_with_options_per_problem():
    """Problems of different sizes reserve their own RHS capacity and chunk
    length in one batched setup; each plan equals its own single setup."""
    ns = [31, 63]
    cs = [I.random_velocity(n, 300 + k) for k, n in enumerate(ns)]
    ol = [opts(max_nrhs=2, chunk=8, graphs=0), opts(max_nrhs=6, chunk=0, graphs=0)]
    plans = hs.hs_setup_batched([c.ravel() for c in cs], [omega_of(n) for n in ns], ns, 2, BP, BP, ol)
    singles = [hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, o) for c, n, o in zip(cs, ns, ol)]
    try:
        nr = [2, 6]
        rs = [torch.from_numpy(I.random_rhs(n, q, 60 + k)).to("cuda").to(torch.complex64)
              for k, (n, q) in enumerate(zip(ns, nr))]
        zs = [torch.empty_like(r) for r in rs]
        hs.hs_apply_batched(plans, rs, zs, nr, hs.HS_C64)
        torch.cuda.synchronize()
        for k in range(2):
            assert hs.hs_last_device_status(plans[k]) == hs.HS_OK
            assert torch.equal(zs[k], apply_direct(singles[k], rs[k], nr[k])), k
        r3 = torch.zeros(3, 31, 31, dtype=torch.complex64, device="cuda")
        with pytest.raises(hs.HsError):          # beyond the first problem's own capacity
            hs.hs_apply(plans[0], r3, torch.empty_like(r3), 3, hs.HS_C64)
    finally:
        for p in plans + singles:
            hs.hs_destroy(p)


@pytest.mark.parametrize("sep", [1, 2, 4])
def test_separator_grouping_option_gives_the_same_result(sep):
    """Any fixed number of RHS per separator-solve CTA (the autotuner's
    second knob) computes the same arithmetic per RHS: bit-identical to the
    automatic choice."""
    n = 63
    c = I.random_velocity(n, 14)
    pa = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=7, graphs=0))
    pf = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=7, sep_rhs_per_cta=sep))
    try:
        r = torch.from_numpy(I.random_rhs(n, 7, 15)).to("cuda").to(torch.complex64)   # 7: a ragged last group
        assert torch.equal(apply_direct(pa, r, 7), apply_direct(pf, r, 7))
    finally:
        hs.hs_destroy(pa)
        hs.hs_destroy(pf)


@pytest.mark.parametrize("nrhs", [100, 160])     # two and four RHS per separator-solve CTA
def test_many_rhs_match_the_same_rhs_in_slices(nrhs):
    """The separator solve groups more RHS per CTA when the RHS of both
    fronts outnumber the SMs; each RHS's arithmetic is unchanged, so the
    result equals the applications of 50-RHS slices (one RHS per CTA)."""
    n = 63
    c = I.random_velocity(n, 11)
    p = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=nrhs, graphs=0))
    try:
        r = torch.from_numpy(I.random_rhs(n, nrhs, 13)).to("cuda").to(torch.complex64)
        z = apply_direct(p, r, nrhs)
        for q0 in range(0, nrhs, 50):
            q1 = min(nrhs, q0 + 50)
            assert torch.equal(z[q0:q1], apply_direct(p, r[q0:q1].contiguous(), q1 - q0)), q0
    finally:
        hs.hs_destroy(p)


def test_graph_replay_is_bit_identical_to_direct_launches():
    n = 63
    c = I.random_velocity(n, 3)
    pg = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(graphs=1))
    pd = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(graphs=0))
    try:
        for seed in (1, 2, 3):       # capture on the first call, replay after; new data each time
            r = torch.from_numpy(I.random_rhs(n, 3, seed)).to("cuda").to(torch.complex64)
            assert torch.equal(apply_direct(pg, r, 3), apply_direct(pd, r, 3))
        r = torch.from_numpy(I.random_rhs(n, 1, 9)).to("cuda").to(torch.complex64)   # another nrhs
        assert torch.equal(apply_direct(pg, r, 1), apply_direct(pd, r, 1))
    finally:
        hs.hs_destroy(pg)
        hs.hs_destroy(pd)


def test_apply_batched_matches_per_problem_applies():
    cs = [I.random_velocity(n, 200 + k) for k, n in enumerate(NS)]
    plans = hs.hs_setup_batched([c.ravel() for c in cs], [omega_of(n) for n in NS], NS, 2, BP, BP,
                                opts(graphs=0))
    try:
        nr = [1, 3, 2, 4]
        for call in range(3):        # capture, then two replays with fresh inputs
            rs = [torch.from_numpy(I.random_rhs(n, q, 50 + 10 * call + k)).to("cuda").to(torch.complex64)
                  for k, (n, q) in enumerate(zip(NS, nr))]
            zs = [torch.empty_like(r) for r in rs]
            hs.hs_apply_batched(plans, rs, zs, nr, hs.HS_C64)
            torch.cuda.synchronize()
            for k in range(len(NS)):
                assert hs.hs_last_device_status(plans[k]) == hs.HS_OK
                assert torch.equal(zs[k], apply_direct(plans[k], rs[k], nr[k])), (call, k)
    finally:
        for p in plans:
            hs.hs_destroy(p)


def test_apply_batched_rejects_repeated_plan_and_bad_nrhs():
    n = 31
    p = hs.hs_setup(I.constant_velocity(n).ravel(), omega_of(n), n, 2, BP, BP, opts())
    try:
        r = torch.zeros(4 * n * n, dtype=torch.complex64, device="cuda")
        with pytest.raises(hs.HsError):
            hs.hs_apply_batched([p, p], [r, r], [r, r], [1, 1], hs.HS_C64)
        with pytest.raises(hs.HsError):
            hs.hs_apply_batched([p], [r], [r], [5], hs.HS_C64)
    finally:
        hs.hs_destroy(p)


def test_autotune_writes_cache_that_setup_reads(tmp_path):
    n = 95
    c = I.random_velocity(n, 5)
    cache = str(tmp_path / "tune.txt")
    o = opts(max_nrhs=2, chunk=0, tune_cache=cache)
    best, ms, sep = hs.hs_autotune(c.ravel(), omega_of(n), n, 2, BP, BP, 2, opt=o)
    assert best >= 2 and ms > 0 and sep in (1, 2, 4)
    line = open(cache).read().strip().splitlines()[-1]
    assert ("n=%d" % n) in line and ("chunk=%d" % best) in line and ("sep=%d" % sep) in line
    # a setup with chunk = 0 and the cache gives the same operator as chunk = best
    pt = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=2, chunk=0, tune_cache=cache))
    pe = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=2, chunk=best, sep_rhs_per_cta=sep))
    try:
        r = torch.from_numpy(I.random_rhs(n, 2, 4)).to("cuda").to(torch.complex64)
        assert torch.equal(apply_direct(pt, r, 2), apply_direct(pe, r, 2))
    finally:
        hs.hs_destroy(pt)
        hs.hs_destroy(pe)
    os.remove(cache)


@pytest.mark.parametrize("prec", [hs.HS_C64, hs.HS_C128])
def test_non_finite_pivot_is_reported_as_breakdown(prec):
    """omega = 1e160 overflows omega^2/c^2 in both factor precisions: every
    diagonal block has a non-finite pivot, the setup reports HS_EBREAKDOWN
    (no plan is returned), and the next setup still runs."""
    n = 31
    c = I.constant_velocity(n)
    with pytest.raises(hs.HsError) as err:
        hs.hs_setup(c.ravel(), 1e160, n, 2, BP, BP, opts(factor_prec=prec))
    assert err.value.code == hs.HS_EBREAKDOWN
    good = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(factor_prec=prec))
    try:
        r = torch.from_numpy(I.random_rhs(n, 2, 5)).to("cuda").to(torch.complex64)
        apply_direct(good, r, 2)
    finally:
        hs.hs_destroy(good)


def test_expired_device_wait_is_reported_and_context_stays_usable():
    """A plan whose device waits may take one clock cycle: the first
    shared-memory copy cannot land in time, every CTA gives up together,
    drains its copies in flight, records HS_ETIMEOUT and exits; the host
    reads the status, and the next plan still runs."""
    n = 63
    c = I.random_velocity(n, 8)
    bad = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(spin_budget=1, graphs=0))
    try:
        r = torch.from_numpy(I.random_rhs(n, 2, 1)).to("cuda").to(torch.complex64)
        z = torch.empty_like(r)
        hs.hs_apply(bad, r, z, 2, hs.HS_C64)
        assert hs.hs_sync(bad) == hs.HS_ETIMEOUT
    finally:
        hs.hs_destroy(bad)
    good = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts())
    try:
        r = I.random_rhs(n, 2, 1)
        z = apply_direct(good, torch.from_numpy(r).to("cuda").to(torch.complex64), 2).cpu().numpy()
        ref = S.apply(S.setup(c, omega_of(n), BP, BP, 3, 2.0, C_PML, Cm=C_MOVING),
                      r.astype(np.complex64).astype(np.complex128))
        assert relerr(z.astype(np.complex128), ref) <= 1e-4
    finally:
        hs.hs_destroy(good)


def test_async_setup_orders_every_later_call():
    """async_setup = 1: hs_setup returns once the factorisation is queued on
    its stream.  An application issued at once on another stream, a solve
    and the status read order themselves after it: the application equals the
    synchronously set up plan's bit for bit, and the solve converges."""
    n, R = 127, 4
    c = I.random_velocity(n, 11)
    s_setup, s_use = torch.cuda.Stream(), torch.cuda.Stream()
    sync_plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=R, graphs=0))
    async_plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=R, graphs=0, async_setup=1),
                             stream=s_setup)
    try:
        r = torch.from_numpy(I.random_rhs(n, R, 12)).to("cuda").to(torch.complex64)
        torch.cuda.synchronize()
        z_async, z_sync = torch.empty_like(r), torch.empty_like(r)
        hs.hs_apply(async_plan, r, z_async, R, hs.HS_C64, stream=s_use)
        hs.hs_apply(sync_plan, r, z_sync, R, hs.HS_C64)
        torch.cuda.synchronize()
        assert hs.hs_last_device_status(async_plan) == hs.HS_OK
        assert torch.equal(z_async, z_sync)
        f = torch.from_numpy(I.point_sources(n, R, 13, BP)).to("cuda")
        u = torch.zeros_like(f)
        torch.cuda.synchronize()     # f and u were made on the default stream
        code, info = hs.hs_solve(async_plan, f, u, R, 1e-6, 100, stream=s_use)
        assert code == hs.HS_OK and info["max_relres"] <= 1e-6
        assert hs.hs_sync(async_plan, s_use) == hs.HS_OK
    finally:
        hs.hs_destroy(async_plan)
        hs.hs_destroy(sync_plan)


def test_plan_memory_is_reused_and_released():
    """Plans draw their buffers from a pool that keeps freed memory: a plan
    set up after another was destroyed (warm pool), and one set up after
    hs_release_workspace returned the pool's memory, give the same result."""
    n, R = 95, 3
    c = I.random_velocity(n, 14)
    r = torch.from_numpy(I.random_rhs(n, R, 15)).to("cuda").to(torch.complex64)
    outs = []
    for release in (False, False, True):
        if release:
            assert hs.hs_release_workspace() == hs.HS_OK
        p = hs.hs_setup(c.ravel(), omega_of(n), n, 2, BP, BP, opts(max_nrhs=R, graphs=0))
        try:
            outs.append(apply_direct(p, r, R).clone())
        finally:
            hs.hs_destroy(p)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
