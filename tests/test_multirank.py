"""The multi-GPU exchange on CPU ranks (gloo, world size 2): shards of one
stream, sketched separately with their global indices, all-reduced, equal the
sketch of the whole stream - and so give the same top-k."""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1711_00975_gb300.distributed import allreduce_counters, shard_range

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N, BOX, ROWS, LOG2W, K, RATE = 300_000, 20.0, 5, 14, 200, 0.5


def _params():
    return oracle.Params(ROWS, LOG2W, BOX, 0.1, hash_seed=9, sample_seed=4)


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = synth.BoxSpec(n=N, box=BOX, n_halo=40, seed=2)
    box = synth.HaloBox(spec)
    lo, cnt = shard_range(N, rank, world)
    xyz = box.generate(lo, cnt)
    p = _params()
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz, g0=lo, rate=RATE)
    t = torch.from_numpy(C.copy())
    allreduce_counters(t)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_the_stream():
    for n, w in [(10, 3), (7, 7), (1_000_003, 4), (0, 2)]:
        spans = [shard_range(n, r, w) for r in range(w)]
        assert spans[0][0] == 0 and sum(c for _, c in spans) == n
        assert all(spans[i][0] + spans[i][1] == spans[i + 1][0] for i in range(w - 1))
    with pytest.raises(ValueError):
        shard_range(10, 3, 3)


def test_two_ranks_sum_to_the_whole_stream(tmp_path):
    port = 29500 + os.getpid() % 2000
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    spec = synth.BoxSpec(n=N, box=BOX, n_halo=40, seed=2)
    xyz = synth.HaloBox(spec).generate()
    p = _params()
    whole = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=RATE)
    for r in range(2):
        merged = np.load(tmp_path / f"rank{r}.npy")
        assert np.array_equal(merged, whole)
    wk, we = oracle.topk_full(whole, p, K, nthreads=2)
    mk, me = oracle.topk_full(np.load(tmp_path / "rank0.npy"), p, K, nthreads=2)
    assert np.array_equal(wk, mk) and np.array_equal(we, me)
