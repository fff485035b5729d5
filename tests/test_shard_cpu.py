"""One instance sharded by chromosome rows over CPU ranks (torch.distributed, gloo).

The exchange per generation is an all-reduce MAX of a packed (fitness, -index) key and a
broadcast of the elite's alleles from the rank that owns it. Each rank computes its rows
with the oracle's row-block functions; the gathered result must equal the unsharded oracle
bit for bit (state, per-generation elites, best record), for even and ragged splits and for
both key forms (packed 64-bit and the two-reduction form for wide fitness)."""
import os
import socket

import numpy as np
import pytest

from paper_2609_30862_gb300 import shard as S
from paper_2609_30862_gb300 import workload as W


def test_packed_key_orders_by_fitness_then_lowest_index():
    rng = np.random.default_rng(5)
    f = rng.integers(-2**31, 2**31, 400)
    f[::3] = 7                                     # many ties
    c = rng.integers(0, 2**32, 400)
    keys = [S.pack_key(int(a), int(b)) for a, b in zip(f, c)]
    for i in range(0, 400, 7):
        for j in range(0, 400, 11):
            want = (f[i], -int(c[i])) > (f[j], -int(c[j]))
            assert (keys[i] > keys[j]) == want
    for a, b, k in zip(f, c, keys):
        assert S.unpack_key(k) == (int(a), int(b))
        assert -2**63 <= k < 2**63
    with pytest.raises(ValueError):
        S.pack_key(2**31, 0)
    with pytest.raises(ValueError):
        S.pack_key(0, -1)


def test_key_form_follows_the_problem_bounds():
    """The key form is a function of the problem alone, so every rank picks the same one."""
    assert not S.key_is_wide([10] * 100, [15] * 100)
    assert S.key_is_wide([1] * 4, [2**30] * 4)                   # sum |v| beyond 2^31 - 1
    assert S.key_is_wide([2**29] * 4, [1] * 4, lam=2)             # lam sum w beyond 2^31
    assert not S.key_is_wide([2**29] * 4, [1] * 4, lam=1)         # exactly 2^31: fits
    assert S.key_is_wide([1], [-(2**31)])                         # |v| counts


@pytest.mark.parametrize("np_,world", [(10, 2), (11, 3), (3, 4), (1024, 8)])
def test_row_ranges_cover_the_population(np_, world):
    seen = []
    for r in range(world):
        r0, r1 = S.row_range(np_, world, r)
        assert r1 - r0 in (np_ // world, np_ // world + 1)
        seen.extend(range(r0, r1))
        for c in range(r0, r1):
            assert S.owner_of(c, np_, world) == r
    assert seen == list(range(np_))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out_path):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob, np_, gens, seed, inst, D, lam, rule, wide = case
        ng = prob.ng
        r0, r1 = S.row_range(np_, world, rank)
        k = np.zeros((r1 - r0, ng), dtype=np.int16)
        last = {}

        def observe_rows(t):
            x, f = O.rows_observe(prob, k, t, r0, seed=seed, inst=inst, D=D, lam=lam)
            last["x"] = x
            return f, x

        def rotate_rows(x_e):
            O.rows_rotate(k, last["x"], x_e, D=D, rule=rule)

        ex = S.EliteExchange(np_, ng, problem=prob, lam=lam)
        assert ex.wide == wide
        he, hf, best = S.run_sharded(np_, ng, gens, observe_rows, rotate_rows, ex, r0)
        blocks = [None] * world
        dist.all_gather_object(blocks, k)
        if rank == 0:
            np.savez(out_path, k=np.concatenate(blocks, axis=0), he=he, hf=hf,
                     best=np.array(best[:3], dtype=np.int64), best_x=best[3])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,np_,wide,rule", [(2, 24, False, 0), (3, 25, False, 1),
                                                  (2, 9, True, 0)])
def test_sharded_run_equals_unsharded(tmp_path, world, np_, wide, rule):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    O.build()
    if wide:   # values beyond 2^31 in total: fitness needs the two-reduction form
        rng = np.random.default_rng(3)
        w = rng.integers(1, 11, 120).astype(np.int32)
        v = rng.integers(2**27, 2**28, 120).astype(np.int32)
        prob = W.custom_problem(w, v, int(w.sum()) // 2)
    else:
        prob = W.knapsack(333, 21)
    gens, seed, inst, D, lam = 40, 9, 4, 100, 1
    case = (prob, np_, gens, seed, inst, D, lam, rule, wide)
    out = str(tmp_path / "sharded.npz")
    mp.spawn(_rank_main, args=(world, _free_port(), case, out), nprocs=world, join=True)
    got = np.load(out)
    st = O.run(prob, np_, gens, seed=seed, inst=inst, D=D, lam=lam, rule=rule)
    assert np.array_equal(got["k"], st.k)
    assert np.array_equal(got["he"], st.hist_e)
    assert np.array_equal(got["hf"], st.hist_f)
    assert tuple(int(v) for v in got["best"]) == tuple(int(v) for v in st.best)
    assert np.array_equal(got["best_x"], st.best_x)
    if wide:
        assert int(np.max(np.abs(st.hist_f))) > 2**31
