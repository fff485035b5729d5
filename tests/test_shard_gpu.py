"""One instance sharded by chromosome rows, each rank's rows on the GPU (qieo_create_row_block,
qieo_rows_observe, qieo_rows_rotate through the C ABI), the exchange over torch.distributed
(gloo) ranks: the gathered state, every generation's elite and the best record equal the
unsharded oracle bit for bit.

The ranks are separate processes that share the one GPU. Their kernels never wait on one
another: each generation's exchange (an all-reduce of the packed key and a broadcast of
the elite's alleles) goes through the host, between launches."""
import os
import socket

import numpy as np
import pytest

from paper_2609_30862_gb300 import shard as S
from paper_2609_30862_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out_path):
    import torch
    import torch.distributed as dist
    from paper_2609_30862_gb300 import qieo as Q
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        Q.load(build_if_missing=False)
        prob, np_, chunks, seed, inst, D, lam, rule, flags = case
        r0, r1 = S.row_range(np_, world, rank)
        with Q.Instance(prob, r1 - r0, seed=seed, inst=inst, D=D, lam=lam, rule=rule,
                        flags=flags, row0=r0) as blk:
            ex = S.EliteExchange(np_, prob.ng, problem=prob, lam=lam)
            he, hf, best, t0 = [], [], (None, -1, -1, None), 0
            for g in chunks:                      # runs continue from the generation reached
                e, f, b = S.run_sharded_blocks(g, blk.rows_observe, lambda c: blk.allele_row(c - r0),
                                               blk.rows_rotate, ex, t0=t0)
                he.append(e)
                hf.append(f)
                if best[1] < 0 or b[0] > best[0]:
                    best = b
                t0 += g
            k, t = blk.state()
            fit = blk.fitness()
        blocks = [None] * world
        dist.all_gather_object(blocks, (k, fit, t))
        if rank == 0:
            np.savez(out_path, k=np.concatenate([b[0] for b in blocks], axis=0),
                     f=np.concatenate([b[1] for b in blocks]), t=np.array([b[2] for b in blocks]),
                     he=np.concatenate(he), hf=np.concatenate(hf),
                     best=np.array(best[:3], dtype=np.int64), best_x=best[3])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,np_,ng,rule,chunks,flags", [
    (2, 64, 3000, 0, [25], 0),
    (2, 33, 1000, 1, [10, 15], 0),           # ragged split, rule R2, a run continued
    (3, 40, 5000, 0, [30], 0x100),           # byte state
])
def test_sharded_rows_on_gpu_equal_unsharded(tmp_path, world, np_, ng, rule, chunks, flags):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2609_30862_gb300 import qieo as Q
    Q.load()                                  # build once before the ranks start
    prob = W.knapsack(ng, 40 + world)
    seed, inst, D, lam = 11, 3, 100, 1
    case = (prob, np_, chunks, seed, inst, D, lam, rule, flags)
    out = str(tmp_path / "sharded.npz")
    mp.spawn(_rank_main, args=(world, _free_port(), case, out), nprocs=world, join=True)
    got = np.load(out)
    gens = sum(chunks)
    st = O.run(prob, np_, gens, seed=seed, inst=inst, D=D, lam=lam, rule=rule)
    assert np.array_equal(got["k"], st.k)
    assert np.array_equal(got["f"], st.f)
    assert list(got["t"]) == [gens] * world
    assert np.array_equal(got["he"], st.hist_e)
    assert np.array_equal(got["hf"], st.hist_f)
    assert tuple(int(v) for v in got["best"]) == tuple(int(v) for v in st.best)
    assert np.array_equal(got["best_x"], st.best_x)


def test_row_block_rejects_misuse():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30862_gb300 import qieo as Q
    Q.load()
    prob = W.knapsack(100, 2)
    with Q.Instance(prob, 10, row0=20) as blk:
        with pytest.raises(Q.QieoError):
            blk.run(1)                          # row blocks advance by observe + rotate
        with pytest.raises(Q.QieoError):
            blk.rows_rotate(np.zeros(100, dtype=np.uint8))   # nothing observed yet
        f, c = blk.rows_observe(0)
        assert 20 <= c < 30
        with pytest.raises(Q.QieoError):
            blk.rows_rotate(np.full(100, 2, dtype=np.uint8))  # not an allele
        with pytest.raises(Q.QieoError):
            Q.qieo_create_batch([blk.h])
    with pytest.raises(Q.QieoError):
        Q.Instance(prob, 10, row0=-1)
    with pytest.raises(Q.QieoError):
        Q.Instance(prob, 10, row0=0, elite_on_host=1)
