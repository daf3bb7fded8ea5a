"""The N > 1 paths on CPU ranks (gloo, world size 2).

Every box here has one GPU, so the multi-rank logic runs as CPU processes:

* replicas (what ``bench.py --gpus N`` runs): each rank times its own step;
  the job's time is the slowest rank's, taken with one all-reduce, and the
  job's throughput counts every rank's keys over that time;
* the level exchange of a monolithic multi-GPU build: each rank fills its
  shard of F_d (Algorithm 2), the fills are gathered, and merging them in
  rank order gives the fill of the whole level -- the same arrays on every
  rank, equal to a single-process fill and to the build's A_0.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1702_03154_gb300 import inputs
        res = {}
        # replicas: slowest rank's time, whole-job throughput
        ms = 10.0 + 5.0 * rank
        res["max_ms"] = bench.max_over_ranks(ms, world, "cpu")
        res["value"] = bench.job_value(10**8, world, res["max_ms"])
        # monolithic level exchange: shard, fill, gather, merge
        keys = inputs.splitmix64_keys(20000, 142)
        o = oracle.build(keys, gamma=2.0, levels=25, seed=9)
        n0, m0, off0, s0 = o.level_info(0)
        A, C = oracle.fill_level(keys[rank::world], s0, m0)
        As = [torch.empty(m0, dtype=torch.uint8) for _ in range(world)]
        Cs = [torch.empty(m0, dtype=torch.uint8) for _ in range(world)]
        dist.all_gather(As, torch.from_numpy(A))
        dist.all_gather(Cs, torch.from_numpy(C))
        mA, mC = As[0].numpy(), Cs[0].numpy()
        for r in range(1, world):
            mA, mC = oracle.merge_fill(mA, mC, As[r].numpy(), Cs[r].numpy())
        wA, wC = oracle.fill_level(keys, s0, m0)
        bits = np.unpackbits(o.level_bits_words(0).view(np.uint8), bitorder="little")[:m0]
        res["merge_ok"] = bool(np.array_equal(mA, wA) and np.array_equal(mC, wC)
                               and np.array_equal(mA, bits))
        # every rank ends with the same arrays
        h = torch.tensor([int(mA.sum()), int(mC.sum())], dtype=torch.int64)
        hs = [torch.empty(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(hs, h)
        res["same_on_all"] = all(torch.equal(x, hs[0]) for x in hs)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, res = q.get(timeout=240)
        got[r] = res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r]["max_ms"] == 15.0
        assert got[r]["value"] == pytest.approx(2 * 10**8 / 0.015 / 1e6)
        assert got[r]["merge_ok"] and got[r]["same_on_all"]


# ------------------------------------------- one part per rank (Sec. 4.3)
# DistributedMPHF's exchange and offset logic on gloo ranks.  Its device
# steps (route, build, lookup, offset, scatter back) are stood in for by the
# oracle on the CPU, so the global indices must equal the oracle's
# partitioned mode over the union of every rank's keys, with K = world size.
class _OracleOps:
    def __init__(self):
        self.device = torch.device("cpu")

    def empty(self, n):
        return torch.empty(int(n), dtype=torch.int64)

    def route(self, keys, K, part_seed, with_src):
        import oracle
        k = keys.numpy().view(np.uint64)
        p = oracle.parts(k, K, part_seed)
        order = np.argsort(p, kind="stable")
        off = np.zeros(K + 1, dtype=np.uint64)
        np.cumsum(np.bincount(p.astype(np.int64), minlength=K).astype(np.uint64), out=off[1:])
        src = torch.from_numpy(order.astype(np.int64)) if with_src else None
        return torch.from_numpy(k[order].view(np.int64).copy()), src, off

    def build(self, keys, gamma, levels, seed):
        import oracle
        return oracle.build(keys.numpy().view(np.uint64), gamma=gamma, levels=levels, seed=seed)

    def lookup(self, f, keys):
        return torch.from_numpy(f.lookup(keys.numpy().view(np.uint64)).view(np.int64).copy())

    def add_offset(self, vals, offset):
        v = vals.numpy().view(np.uint64)
        hit = v != np.uint64((1 << 64) - 1)
        v[hit] += np.uint64(offset)
        return vals

    def unroute(self, vals, src):
        out = torch.empty_like(vals)
        out[src] = vals
        return out


def _part_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1702_03154_gb300 import inputs
        from paper_1702_03154_gb300.distributed import DistributedMPHF
        all_keys = inputs.splitmix64_keys(30011, 160)
        mine = all_keys[rank::world]                       # this rank's share
        d = DistributedMPHF(torch.from_numpy(mine.view(np.int64).copy()), part_seed=21,
                            gamma=2.0, levels=25, seed=4, ops=_OracleOps())
        P = oracle.PartitionedOracle(all_keys, world, 21, gamma=2.0, levels=25, seed=4)
        res = {"offsets": bool(np.array_equal(d.offsets, P.offsets)), "N": d.N}
        # queries: another share of the members plus non-members, of a
        # different size on each rank
        q = np.concatenate([all_keys[(rank + 1) % world::world][: 5000 + 777 * rank],
                            inputs.splitmix64_keys(300 + rank, 161 + rank)])
        got = d.lookup(torch.from_numpy(q.view(np.int64).copy())).numpy().view(np.uint64)
        res["lookup"] = bool(np.array_equal(got, P.lookup(q)))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_one_part_per_gloo_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_part_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, res = q.get(timeout=240)
        got[r] = res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r] == {"offsets": True, "N": 30011, "lookup": True}, got[r]
