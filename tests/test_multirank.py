"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) check that the
shards are disjoint slices of the single-rank workload, that the reported time is the
slowest rank's, and that the whole-job rate counts every rank's series."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2604_00048_b300 import synth

        per = 24
        rc = synth.Recipe(**{**synth.RECIPES["hetero_tile"].__dict__, "T": 40, "n_bands": 2})
        s0 = bench.rank_series0(rank, per)
        mine = synth.generate_tile(rc, per, series0=s0)["x"]
        ms = 10.0 + 5.0 * rank  # rank 1 is slower
        slow = bench.max_over_ranks(ms, "cpu")
        rate = bench.aggregate_rate(per, world, 3, slow)
        q.put((rank, s0, mine.numpy(), slow, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import bench  # noqa: F401  (importable without a GPU)
    from paper_2604_00048_b300 import synth

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, s0, x, slow, rate = q.get(timeout=120)
        res[r] = (s0, x, slow, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rc = synth.Recipe(**{**synth.RECIPES["hetero_tile"].__dict__, "T": 40, "n_bands": 2})
    full = synth.generate_tile(rc, 48)["x"].numpy()
    assert res[0][0] == 0 and res[1][0] == 24
    assert (res[0][1] == full[:, :, :24]).all() and (res[1][1] == full[:, :, 24:]).all()
    for r in range(world):
        assert res[r][2] == 15.0                      # the slowest rank's time on every rank
        assert abs(res[r][3] - 48 * 3 / 0.015) < 1e-6  # all series over that time
