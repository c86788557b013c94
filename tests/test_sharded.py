"""Multi-GPU form on CPU ranks (gloo, world size 2): the state shards of an
anneal, each run with its global state offset, reproduce one anneal of all
states; the ranks agree on the best state (lowest energy, ties to the lowest
global index); and a rank that dies before the exchange makes the other
rank's exchange fail with an error instead of hanging.  The per-shard
annealer is the oracle, so these tests need no GPU."""
import datetime
import multiprocessing as mp
import socket

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_2407_19987_gb300.sharded import local_best, shard_range


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    inst = W.tiny_dense(1)
    return inst, W.geometric_betas(5.0, 0.05, 40), 11, 77


def _rank_main(rank, world, port, q, fail_rank):
    import torch.distributed as dist

    from paper_2407_19987_gb300.sharded import anneal_sharded
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=5))
        inst, betas, B, seed = _case()

        def oracle_shard(lo, hi):
            if rank == fail_rank:
                raise RuntimeError("injected failure")
            r = O.anneal(inst, seed, hi - lo, betas, state0=lo)
            return W.pack_bits(r["bestX"]).view(np.int32), r["bestE"]

        out = anneal_sharded(inst, seed, B, betas, anneal_fn=oracle_shard)
        q.put((rank, "ok", out["range"], out["bestX"], out["bestE"], out["best_E"], out["best_index"],
               out["best_X"]))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which decides
        q.put((rank, "error", repr(e)))


def _run(world, fail_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in ps:
        p.start()
    res = {}
    try:
        for _ in range(world):
            item = q.get(timeout=timeout)
            res[item[0]] = item
    finally:
        for p in ps:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
                p.join()
    return res


def test_shard_range_covers_states_evenly():
    for B in (0, 1, 5, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            rs = [shard_range(B, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == B
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def test_local_best_takes_lowest_index_on_ties():
    assert local_best(np.array([3.0, -1.0, -1.0, 2.0]), 10) == (-1.0, 11, 1)
    assert local_best(np.zeros(0), 5)[1] == -1


def test_sharded_anneal_equals_single_anneal():
    inst, betas, B, seed = _case()
    res = _run(2)
    assert all(v[1] == "ok" for v in res.values()), res
    ref = O.anneal(inst, seed, B, betas)
    bx = np.concatenate([res[r][3] for r in range(2)])
    be = np.concatenate([res[r][4] for r in range(2)])
    assert [res[r][2] for r in range(2)] == [(0, 6), (6, 11)]
    np.testing.assert_array_equal(W.unpack_bits(bx.view(np.uint32), inst.N), ref["bestX"])
    np.testing.assert_array_equal(be, ref["bestE"])
    k = int(np.argmin(ref["bestE"]))
    for r in range(2):
        assert res[r][5] == ref["bestE"][k] and res[r][6] == k
        np.testing.assert_array_equal(W.unpack_bits(res[r][7][None, :], inst.N)[0], ref["bestX"][k])


def test_rank_failure_ends_the_exchange_with_an_error():
    res = _run(2, fail_rank=1, timeout=120)
    assert res[1][1] == "error" and "injected failure" in res[1][2]
    assert res[0][1] == "error"          # the survivor's collective failed instead of hanging
