"""The solve server (continuous batching): results equal the same solve run alone, requests
arriving while others run are admitted as memory frees up, oversized requests are refused,
queued requests can be cancelled."""
import time

import numpy as np
import pytest

from paper_2609_30862_gb300 import qieo as Q
from paper_2609_30862_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Q.load()


def alone(prob, np_, gens, seed, inst, rule=0):
    with Q.Instance(prob, np_, seed=seed, inst=inst, rule=rule) as I:
        I.run(gens)
        return I.best()


def test_server_results_equal_alone_in_the_mix():
    specs = W.batch_manifest(40, first_seed=300)
    with Q.Server(gens_per_step=7) as srv:
        ids = []
        for i, sp in enumerate(specs):
            prob = W.knapsack(sp.ng, sp.seed)
            gens = 20 + (i % 3) * 9
            ids.append((srv.submit(prob, sp.np_, gens, seed=sp.seed, inst=sp.seed, rule=i % 2),
                        prob, sp, gens, i % 2))
            if i % 10 == 9:
                time.sleep(0.003)          # later requests arrive while earlier ones run
        for rid, prob, sp, gens, rule in ids:
            res, bits = srv.poll(rid, wait_ms=60000)
            assert res.state == Q.QIEO_SOLVE_DONE, res.status
            b_bits, bf, bg, bc = alone(prob, sp.np_, gens, sp.seed, sp.seed, rule)
            assert (res.fitness, res.generation, res.chromosome) == (bf, bg, bc)
            assert np.array_equal(bits, b_bits)
            assert res.submit_s <= res.admit_s <= res.done_s


def test_server_admits_by_memory_and_matches_oracle():
    """An arena that holds about two of these solves: the rest wait for memory."""
    from oracle import oracle as O
    prob = W.knapsack(3000, 5)
    with Q.Server(memory_bytes=6 << 20, gens_per_step=5) as srv:
        ids = [srv.submit(prob, 300, 12, seed=s, inst=s) for s in range(6)]
        for s, rid in enumerate(ids):
            res, bits = srv.poll(rid, wait_ms=60000)
            assert res.state == Q.QIEO_SOLVE_DONE
            st = O.run(prob, 300, 12, seed=s, inst=s)
            assert (res.fitness, res.generation, res.chromosome) == tuple(int(v) for v in st.best)
            assert np.array_equal(bits, st.best_x)
        admits = sorted(srv.poll(r)[0].admit_s for r in ids)
        dones = sorted(srv.poll(r)[0].done_s for r in ids)
        assert admits[-1] >= dones[0]          # the last admission waited for a finish


def test_server_refuses_solves_larger_than_the_arena():
    with Q.Server(memory_bytes=1 << 20) as srv:
        with pytest.raises(Q.QieoError) as e:
            srv.submit(W.knapsack(20000, 1), 512, 10)
        assert e.value.status == Q.QIEO_ERR_OOM


def test_server_cancel_queued_only():
    prob = W.knapsack(3000, 6)
    with Q.Server(memory_bytes=4 << 20, gens_per_step=50) as srv:
        first = srv.submit(prob, 300, 400, seed=1)
        queued = [srv.submit(prob, 300, 10, seed=s) for s in range(2, 6)]
        srv.cancel(queued[-1])
        assert srv.poll(queued[-1])[0].state == Q.QIEO_SOLVE_CANCELLED
        res = srv.poll(first, wait_ms=0)[0]
        if res.state == Q.QIEO_SOLVE_RUNNING:
            with pytest.raises(Q.QieoError) as e:
                srv.cancel(first)
            assert e.value.status == Q.QIEO_ERR_BUSY
        for rid in [first] + queued[:-1]:
            assert srv.poll(rid, wait_ms=60000)[0].state == Q.QIEO_SOLVE_DONE


def test_server_counts_steps_and_launches():
    """The server's counters agree with what it was asked to do: every request admitted and
    completed, at least one step per gens_per_step generations, and per step one batched
    launch per generation plus the final rotation (one group here: narrow items, R1)."""
    srv = Q.Server(gens_per_step=10)
    probs = [W.knapsack(200 + 37 * i, 300 + i) for i in range(6)]
    ids = [srv.submit(p, 40, 30, seed=3, inst=i) for i, p in enumerate(probs)]
    for rid in ids:
        res, _ = srv.poll(rid, wait_ms=60000)
        assert res.state == Q.QIEO_SOLVE_DONE
    st = srv.stats()
    srv.close()
    assert st["submitted"] == st["admitted"] == st["completed"] == 6
    assert st["queued"] == 0 and st["active"] == 0 and 1 <= st["max_active"] <= 6
    assert st["steps"] >= 3
    assert st["kernel_launches"] >= 6 + st["steps"] * 2


def test_server_convergence_stop():
    """Requests with QIEO_FLAG_CONVERGE leave as soon as they converged; each result equals
    the oracle's run with the same stop, and a request without the flag runs its cap."""
    from oracle import oracle as O
    srv = Q.Server(gens_per_step=10)
    cases = [(200, 30, 3), (120, 17, 8), (60, 5, 2), (300, 40, 11)]
    ids = [srv.submit(W.knapsack(ng, s), np_, 400, seed=s, flags=Q.QIEO_FLAG_CONVERGE)
           for ng, np_, s in cases]
    plain = srv.submit(W.knapsack(90, 5), 16, 60, seed=5)
    for rid, (ng, np_, s) in zip(ids, cases):
        res, bits = srv.poll(rid, wait_ms=60000)
        ref = O.run(W.knapsack(ng, s), np_, 400, seed=s, window=20)
        assert res.state == Q.QIEO_SOLVE_DONE and res.converged == 1
        assert res.generations_run == int(ref.t[0]) < 400
        assert (res.fitness, res.generation, res.chromosome) == tuple(int(v) for v in ref.best)
        assert np.array_equal(bits, ref.best_x)
    res, _ = srv.poll(plain, wait_ms=60000)
    assert res.state == Q.QIEO_SOLVE_DONE and res.converged == 0 and res.generations_run == 60
    srv.close()
