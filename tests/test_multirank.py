"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2).

Frames are independent, so ranks decode disjoint frame sets and the only
cross-rank step is the timing reduction (max over ranks).  No GPU is used.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        code = synth.make_code("0.1", 4)
        K = 3
        fr = synth.make_frames(code, K, 0.161, first=bench.frame_offset(rank, K))
        # each rank reports a different step time; the job time is the slowest
        t = bench.max_over_ranks(1.0 + rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, fr.llr[:, :8].tolist())
        out[rank] = (t, gathered, bench.job_mbit_per_s(world, K, code.n, t))
    finally:
        dist.destroy_process_group()


def test_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    times = [res[r][0] for r in range(world)]
    assert times == [2.0, 2.0]                     # max over ranks on every rank
    shards = res[0][1]
    a, b = np.array(shards[0]), np.array(shards[1])
    assert a.shape == b.shape and not np.array_equal(a, b)   # disjoint frame sets
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert res[0][2] == pytest.approx(world * 3 * 320 / 2.0 / 1e6)
    assert bench.frame_offset(1, 128) == 128


def test_single_process_max_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_mbit_per_s(1, 128, 10**6, 0.128) == pytest.approx(1000.0)


def _decode_worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        code = synth.make_code("0.1", 8)
        K = 3
        fr = synth.make_frames(code, K, 0.3, first=bench.frame_offset(rank, K))
        hard, post, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 4)
        gathered = [None] * world
        dist.all_gather_object(gathered, (hard.tolist(), ok.tolist()))
        out[rank] = gathered
    finally:
        dist.destroy_process_group()


def test_sharded_decode_equals_one_process_decoding_every_frame():
    # frames are independent: the ranks' shards, concatenated in rank order,
    # decode exactly as one process decoding all of them
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_decode_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    import synth
    code = synth.make_code("0.1", 8)
    fr = synth.make_frames(code, world * 3, 0.3)
    hard, _, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 4)
    for r in range(world):
        got_hard = np.concatenate([np.array(res[r][k][0]) for k in range(world)])
        got_ok = np.concatenate([np.array(res[r][k][1]) for k in range(world)])
        np.testing.assert_array_equal(got_hard, hard)
        np.testing.assert_array_equal(got_ok, ok)
