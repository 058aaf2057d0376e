"""Several ranks through the library: each rank sketches its shard of one
stream (seeked to the shard's global index, so the sampling is unchanged),
the counters are summed with the process group's all-reduce (Sec. 5: the
sketches can be summed), and the root's full search runs on the sum.  Two
gloo ranks share cuda:0 here (no kernel waits on another rank's); the sum must
equal the oracle's sketch of the whole stream bit for bit and the root's top-k
the oracle's full search."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu

N, BOX, ROWS, LOG2W, K = 4_000_000, 50.0, 5, 20, 500


def _spec():
    return synth.BoxSpec(n=N, box=BOX, n_halo=4000, seed=12)


def _worker(rank, world, port, out_dir, rate):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1711_00975_gb300 import halosketch as hs
    from paper_1711_00975_gb300.distributed import ShardedSketch
    sk = hs.Sketch(ROWS, LOG2W, BOX, 0.1, hash_seed=9, sample_seed=4)
    sh = ShardedSketch(sk, N, rank, world)
    xyz = synth.HaloBox(_spec()).generate(sh.lo, sh.count)
    for _ in range(2):                      # a second pass: reset and seek hold
        sh.reset()
        sh.update(torch.from_numpy(xyz).cuda(), rate)
        res = sh.topk(K)
    np.save(os.path.join(out_dir, f"counters{rank}.npy"), sk.counters())
    if res is not None:
        np.save(os.path.join(out_dir, "keys.npy"), res[0])
        np.save(os.path.join(out_dir, "est.npy"), res[1])
    st = sk.stats()
    np.save(os.path.join(out_dir, f"launches{rank}.npy"),
            np.array([st["update_launches"], st["flush_launches"]]))
    sk.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("rate", [1.0, 0.3])
def test_two_ranks_through_the_library(tmp_path, rate):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    port = 29500 + (os.getpid() + int(rate * 10)) % 2000
    mp.spawn(_worker, args=(2, port, str(tmp_path), rate), nprocs=2, join=True)
    xyz = synth.HaloBox(_spec()).generate()
    p = oracle.Params(ROWS, LOG2W, BOX, 0.1, 9, 4)
    whole = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=rate,
                                 nthreads=oracle.default_threads())
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"counters{r}.npy"), whole)
        upd, flushes = np.load(tmp_path / f"launches{r}.npy")
        assert upd >= 2 and flushes >= 2          # the binned update ran on every rank
    wk, we = oracle.topk_full(whole, p, K, nthreads=oracle.default_threads())
    assert np.array_equal(np.load(tmp_path / "keys.npy"), wk)
    assert np.array_equal(np.load(tmp_path / "est.npy"), we)
