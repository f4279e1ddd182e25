"""Row-slab domain decomposition (paper_1904_04048_gb300/slab.py) on CPU.

* The plan: the owned rows partition the grid, every message a slab sends
  lands in the halo rows of its neighbour that hold the same grid rows, and
  slabs thinner than the halo are refused.
* Stepping: slabs advanced by the FP64 oracle with halo exchange every T
  levels (Eq. A2 reads only the R-neighbourhood of a node) reproduce the
  undivided oracle run bit for bit, and the combined norms equal the
  undivided norms; in one process (all slabs) and over world-size 2 and 3
  gloo process groups (one slab per rank)."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from conftest import ROOT
from paper_1904_04048_gb300 import slab
from slab_oracle import OracleSolver

RADIUS = {5: 1, 9: 1, 13: 2}


@pytest.mark.parametrize("periodic", [False, True], ids=["zero", "periodic"])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("R,T", [(1, 1), (1, 6), (2, 4), (2, 3)])
@pytest.mark.parametrize("ny", [56, 57, 100])
def test_plan_partitions_rows_and_pairs_messages(periodic, world, R, T, ny):
    nx = 9
    if ny // world < R * T and world > 1:
        with pytest.raises(ValueError):
            slab.plan_slabs(nx, ny, world, 0, R, T, periodic)
        return
    plans = [slab.plan_slabs(nx, ny, world, r, R, T, periodic) for r in range(world)]
    owned = np.concatenate([np.arange(p.r0, p.r1) for p in plans])
    assert np.array_equal(owned, np.arange(ny))
    assert max(p.own for p in plans) - min(p.own for p in plans) <= 1
    for p in plans:
        g = p.global_rows()
        lo, hi = p.owned_local
        assert np.array_equal(g[lo:hi], np.arange(p.r0, p.r1))
        if not periodic:  # no halo beyond the grid's zero boundary
            assert g.min() >= 0 and g.max() < ny
        # every send has the matching receive on the peer, in the same order
        for peer, tag, j0 in p.sends():
            q = plans[peer]
            matches = [j for (src, t, j) in q.recvs() if src == p.rank and t == tag]
            assert len(matches) == 1, (p.rank, peer, tag)
            j1 = matches[0]
            assert np.array_equal(p.global_rows()[j0:j0 + p.H], q.global_rows()[j1:j1 + p.H])
        # halo rows are exactly the rows the receives fill
        filled = sorted(r for (_, _, j) in p.recvs() for r in range(j, j + p.H))
        assert filled == list(range(0, p.lo_halo)) + list(range(hi, p.ny_local))


def _runs(orc, scheme, nx, ny, world, T, periodic, u0, v0, lam, tau, h):
    bc = orc.BC_PERIODIC if periodic else orc.BC_ZERO
    runs = []
    for r in range(world):
        plan = slab.plan_slabs(nx, ny, world, r, RADIUS[scheme], T, periodic)
        runs.append(slab.SlabRun(plan, OracleSolver(orc, scheme, nx, plan.ny_local, lam, tau, bc, h)))
    return runs


def _ic(nx, ny, periodic, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 / nx
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    k1, k2 = 2 * math.pi * 2, 2 * math.pi * 1
    u0 = np.cos(k1 * x[None, :] + k2 * y[:, None]) + 0.05 * rng.standard_normal((ny, nx))
    v0 = 0.3 * rng.standard_normal((ny, nx))
    if not periodic:
        u0[:3] = u0[-3:] = 0.0
    return u0, v0, h, (k1, k2)


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("periodic", [False, True], ids=["zero", "periodic"])
@pytest.mark.parametrize("world,T", [(2, 4), (3, 2), (4, 3)])
def test_local_slabs_equal_undivided_oracle_bitwise(orc, scheme, periodic, world, T):
    nx, ny, n_t = 23, 61, 27
    u0, v0, h, kk = _ic(nx, ny, periodic, seed=scheme + world)
    lam = 0.6
    tau = lam * h
    bc = orc.BC_PERIODIC if periodic else orc.BC_ZERO
    rp, rc, _ = orc.run(scheme, u0, v0, lam, tau, n_t, bc=bc)
    runs = _runs(orc, scheme, nx, ny, world, T, periodic, u0, v0, lam, tau, h)
    ex = slab.LocalExchange()
    slab.first_step(runs, ex, [slab.extended_rows(r.plan, u0) for r in runs],
                    [slab.extended_rows(r.plan, v0) for r in runs])
    slab.step_n(runs, ex, n_t - 1)
    got_c = np.concatenate([r.solver.cur[slice(*r.plan.owned_local)] for r in runs])
    got_p = np.concatenate([r.solver.prev[slice(*r.plan.owned_local)] for r in runs])
    assert np.array_equal(got_c, rc) and np.array_equal(got_p, rp)
    l2, linf = slab.error_vs_exact(runs, ex, kk)
    whole = OracleSolver(orc, scheme, nx, ny, lam, tau, bc, h)
    whole.prev, whole.cur, whole.k = rp, rc, n_t
    s = whole.error_sums(kk, 0, ny, 0)
    assert abs(l2 - math.sqrt(s[0] / s[1])) <= 1e-13 * l2 and linf == s[2] / s[3]


def test_thin_slabs_are_refused():
    with pytest.raises(ValueError):
        slab.plan_slabs(64, 20, 3, 0, 2, 4, True)   # 6-row slabs, 8 halo rows
    p = slab.plan_slabs(64, 24, 3, 1, 2, 4, True)   # exactly 8 rows each
    assert p.own == 8 and p.ny_local == 24


def test_shard_splits_independent_work():
    items = list(range(17))
    parts = [slab.shard(items, r, 4) for r in range(4)]
    assert sorted(sum(parts, [])) == items and all(abs(len(a) - len(b)) <= 1 for a in parts for b in parts)


# -------------------------------------------------------------- gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, scheme, periodic, T, q):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import oracle
    from paper_1904_04048_gb300 import slab as sl
    from slab_oracle import OracleSolver as OS
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, n_t = 19, 53, 23
        u0, v0, h, kk = _ic(nx, ny, periodic, seed=7)
        lam = 0.6
        tau = lam * h
        bc = oracle.BC_PERIODIC if periodic else oracle.BC_ZERO
        plan = sl.plan_slabs(nx, ny, world, rank, RADIUS[scheme], T, periodic)
        run = sl.SlabRun(plan, OS(oracle, scheme, nx, plan.ny_local, lam, tau, bc, h))
        ex = sl.DistExchange()
        sl.first_step([run], ex, [sl.extended_rows(plan, u0)], [sl.extended_rows(plan, v0)])
        sl.step_n([run], ex, n_t - 1)
        l2, linf = sl.error_vs_exact([run], ex, kk)
        lo, hi = plan.owned_local
        q.put((rank, plan.r0, run.solver.prev[lo:hi].copy(), run.solver.cur[lo:hi].copy(), l2, linf))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("scheme,periodic,T", [(13, True, 4), (9, False, 6), (5, True, 3)])
def test_gloo_ranks_equal_undivided_oracle_bitwise(orc, world, scheme, periodic, T):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, scheme, periodic, T, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=180) for _ in range(world)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nx, ny, n_t = 19, 53, 23
    u0, v0, h, kk = _ic(nx, ny, periodic, seed=7)
    lam = 0.6
    bc = orc.BC_PERIODIC if periodic else orc.BC_ZERO
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, n_t, bc=bc)
    got_p = np.concatenate([o[2] for o in out])
    got_c = np.concatenate([o[3] for o in out])
    assert np.array_equal(got_c, rc) and np.array_equal(got_p, rp)
    whole = OracleSolver(orc, scheme, nx, ny, lam, lam * h, bc, h)
    whole.prev, whole.cur, whole.k = rp, rc, n_t
    s = whole.error_sums(kk, 0, ny, 0)
    for o in out:  # every rank holds the same combined norms
        assert abs(o[4] - math.sqrt(s[0] / s[1])) <= 1e-13 * o[4] and o[5] == s[2] / s[3]
