"""The N > 1 path on CPU: two gloo ranks shard the Monte-Carlo frames by frame id (disjoint
ranges, counter-based channel) and merge only their integer counters (sum) and durations
(max), with the FP64 oracle standing in for the GPU decoder.  The merged counts must equal
one process decoding the union of the ranges.  For data-parallel training of the learned
min-sum, the ranks' gradients on their own frames, averaged by the all-reduce, must equal
one process's gradient on the union of the frames."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

FRAMES, STEPS, SEED, EBN0, ITERS = 6, 2, 5, 1.5, 10


def _code():
    shifts = synth.qc_shifts(3, 6, 16, seed=1)
    rp, col = oracle.csr_rows(oracle.qc_parity_check(shifts, 16))
    return rp, col, 6 * 16


def _counts(first):
    rp, col, N = _code()
    mu = oracle.channel_awgn(SEED, first, FRAMES, N, oracle.sigma_from_ebn0(EBN0, 0.5))
    _, hard, iters, ok = oracle.sp_decode(rp, col, N, mu, ITERS, early_stop=True, nthreads=1)
    errs = hard.sum(axis=1)
    return {"frames": FRAMES, "frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()),
            "iters_sum": int(np.asarray(iters).sum()), "undetected": int(((errs > 0) & (ok == 1)).sum())}


def _worker(rank, world, port, q):
    from paper_1204_0334_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        firsts = [shard.first_frame(rank, s, FRAMES) for s in range(STEPS)]
        tot = shard.merge_counts([_counts(f) for f in firsts], dist)
        slowest = shard.max_over_ranks(float(rank + 1), dist)
        q.put((rank, firsts, tot, slowest))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_shard_frames_and_merge_counters():
    from paper_1204_0334_gb300 import shard

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    ranges = [(f, f + FRAMES) for _, firsts, _, _ in got for f in firsts]
    ranges.sort()
    assert all(a[1] <= b[0] for a, b in zip(ranges, ranges[1:])), "frame ranges overlap"
    assert got[0][2] == got[1][2], "ranks disagree on the merged counters"
    assert got[0][3] == got[1][3] == float(world)  # the job's duration is the slowest rank's
    want = {k: 0 for k in shard.COUNTERS}
    for f0, _ in ranges:
        for k, v in _counts(f0).items():
            want[k] += v
    assert got[0][2] == want
    assert want["frames"] == world * STEPS * FRAMES and want["frame_errors"] > 0


def test_rank_ranges_are_disjoint_and_bounded():
    from paper_1204_0334_gb300 import shard

    a = shard.first_frame(0, 5, 1 << 17)
    b = shard.first_frame(1, -3, 1 << 17)
    assert a + (1 << 17) <= b
    with pytest.raises(ValueError):
        shard.first_frame(0, 1 << 30, 1 << 17)


def _noms_setup():
    shifts = synth.qc_shifts(3, 6, 8, seed=5)
    H = oracle.qc_parity_check(shifts, 8)
    rp, col = oracle.csr_rows(H)
    cb = oracle.circulant_index(rp, col, 8, 6)
    rng = np.random.default_rng(3)
    T = 3
    params = np.stack([rng.uniform(0.6, 1.0, (T, 18)), rng.uniform(0.0, 0.4, (T, 18))], axis=-1)
    return rp, col, cb, 48, T, params


def _noms_frames(first, n):
    return oracle.channel_awgn(21, first, n, 48, oracle.sigma_from_ebn0(1.0, 0.5))


NOMS_FRAMES = (5, 3)  # uneven shards: the average must weight by frame counts


def _noms_worker(rank, world, port, q):
    from paper_1204_0334_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rp, col, cb, N, T, params = _noms_setup()
        n = NOMS_FRAMES[rank]
        mu = _noms_frames(rank * 100, n)
        _, _, g = oracle.noms(rp, col, cb, N, mu, T, params, want_grad=True)
        avg = shard.average_gradient(torch.from_numpy(g), n, dist)
        q.put((rank, avg.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_average_noms_gradient_over_all_frames():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_noms_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rp, col, cb, N, T, params = _noms_setup()
    union = np.concatenate([_noms_frames(r * 100, NOMS_FRAMES[r]) for r in range(world)])
    _, _, want = oracle.noms(rp, col, cb, N, union, T, params, want_grad=True)
    assert np.abs(want).max() > 0
    for _, g in got:
        assert np.allclose(g, want, rtol=1e-12, atol=1e-15 * np.abs(want).max())
    assert np.array_equal(got[0][1], got[1][1])  # every rank steps with the same gradient
