"""Host logic of the source-sharded trace on CPU: the longest-processing-time partition of
art_partition_sources, and the all-reduce of per-rank outputs on two gloo ranks whose
fields come from the FP64 oracle (Sec. 2.1: the field of several sources is the sum over the
rays of every source)."""
import itertools
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1711_06277_gb300 import _lib as C
from paper_1711_06277_gb300 import shard, synth


def _brute_force_makespan(work, nranks):
    best = np.inf
    for assign in itertools.product(range(nranks), repeat=len(work)):
        load = np.zeros(nranks)
        np.add.at(load, list(assign), work)
        best = min(best, load.max())
    return best


@pytest.mark.parametrize("seed", range(6))
def test_partition_assigns_every_source_once_within_lpt_bound(seed):
    rng = np.random.default_rng(seed)
    n, nranks = 9, 3
    work = rng.pareto(1.5, n) + 0.01
    rank, load = shard.partition(work, nranks)
    assert rank.shape == (n,) and set(np.unique(rank)) <= set(range(nranks))
    np.testing.assert_allclose(np.bincount(rank, weights=work, minlength=nranks), load, rtol=1e-12)
    assert load.sum() == pytest.approx(work.sum(), rel=1e-12)
    opt = _brute_force_makespan(work, nranks)
    # Graham's bound for longest processing time first: at most (4/3 - 1/(3m)) of the optimum
    assert load.max() <= (4 / 3 - 1 / (3 * nranks)) * opt * (1 + 1e-12)


def test_partition_large_balance_and_determinism():
    work = synth.power_law_luminosities(1024, seed=5) * 1e9 + 1e5
    for nranks in (2, 4, 8):
        rank, load = shard.partition(work, nranks)
        # list-scheduling bound: the largest load exceeds the mean by at most one item
        assert load.max() <= work.sum() / nranks + work.max() * (1 + 1e-12)
        rank2, _ = shard.partition(work.copy(), nranks)
        assert np.array_equal(rank, rank2)
    # equal estimates are dealt round-robin in index order
    rank, load = shard.partition(np.ones(8), 4)
    assert rank.tolist() == [0, 1, 2, 3, 0, 1, 2, 3] and load.tolist() == [2, 2, 2, 2]
    # one rank takes everything; an empty source list is valid
    assert shard.partition(work[:5], 1)[0].tolist() == [0] * 5
    assert len(shard.partition([], 3)[0]) == 0
    # more ranks than sources: each source alone on a rank, the other ranks empty
    rank, load = shard.partition([3.0, 1.0], 4)
    assert sorted(rank.tolist()) == [0, 1] and sorted(load.tolist()) == [0.0, 0.0, 1.0, 3.0]


def test_partition_rejects_bad_input():
    import ctypes
    L = C.lib()
    w = (ctypes.c_double * 2)(1.0, -1.0)
    r = (ctypes.c_int * 2)()
    assert L.art_partition_sources(2, w, 2, r, None) == C.ART_EINVAL
    w = (ctypes.c_double * 2)(1.0, float("nan"))
    assert L.art_partition_sources(2, w, 2, r, None) == C.ART_EINVAL
    w = (ctypes.c_double * 2)(1.0, 2.0)
    assert L.art_partition_sources(2, w, 0, r, None) == C.ART_EINVAL
    assert L.art_partition_sources(-1, w, 2, r, None) == C.ART_EINVAL
    assert L.art_partition_sources(2, w, 2, r, None) == C.ART_OK


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


N = 16


def _problem():
    rho = synth.lognormal_field(N, 1.5, seed=21)
    pos = synth.uniform_positions(5, seed=21)
    L = synth.power_law_luminosities(5, seed=21)
    return rho, pos, L


def _oracle(rho, pos, L):
    return O.trace(O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / N, sigma_H=8.0, level0=2,
                             tau_max=30.0), nthreads=1)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rho, pos, L = _problem()
    # work per source: the oracle's own crossing count of that source alone
    work = np.array([_oracle(rho, pos[s:s + 1], L[s:s + 1]).crossings for s in range(len(L))],
                    dtype=np.float64)
    owner, _ = shard.partition(work, world)
    mine = np.flatnonzero(owner == rank)
    buf = torch.zeros((4, N, N, N), dtype=torch.float64)
    stats = None
    if len(mine):
        r = _oracle(rho, pos[mine], L[mine])
        # each rank's retired-ray weights add up for its own l_max (Sec. 2.2 destroy counter)
        assert r.destroy == r.destroy_expected
        buf[0] = torch.from_numpy(r.gamma)
        buf[1:4] = torch.from_numpy(r.force)
        stats = {"crossings": r.crossings, "rays_total": r.rays, "destroy": r.destroy,
                 "L_in": r.L_in, "L_absorbed": r.absorbed, "L_escaped": r.escaped,
                 "L_dropped": r.dropped}
    shard.reduce_fields(buf)
    tallies = shard.reduce_tallies(stats, "cpu")
    out[rank] = (buf.numpy().copy(), tallies, mine.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_sum_equals_full_trace():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    rho, pos, L = _problem()
    full = _oracle(rho, pos, L)
    # every source traced by exactly one rank, both ranks busy
    owned = sorted(res[0][2] + res[1][2])
    assert owned == list(range(len(L))) and res[0][2] and res[1][2]
    for rank in (0, 1):
        buf, tallies, _ = res[rank]
        np.testing.assert_allclose(buf[0], full.gamma, rtol=1e-12, atol=1e-14 * full.gamma.max())
        np.testing.assert_allclose(buf[1:4], full.force, rtol=1e-12,
                                   atol=1e-14 * np.abs(full.force).max())
        assert tallies["crossings"] == full.crossings
        assert tallies["rays_total"] == full.rays
        assert tallies["L_escaped"] == pytest.approx(full.escaped, rel=1e-12)
        assert tallies["L_in"] == pytest.approx(full.L_in, rel=1e-12)


def test_reduce_without_process_group_is_identity():
    t = torch.arange(6, dtype=torch.float32)
    assert torch.equal(shard.reduce_fields(t.clone()), t)
    tal = shard.reduce_tallies(None, "cpu")
    assert all(v == 0 for v in tal.values())
