"""Batched runs (many instances in one launch per generation) and the autotuner, bit for bit
against the CPU oracle run on each instance alone."""
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


def check_against_oracle(inst, prob, np_, gens, seed, iid, D=100, lam=1, rule=0):
    from oracle import oracle as O
    st = O.run(prob, np_, gens, seed=seed, inst=iid, D=D, lam=lam, rule=rule)
    k, t = inst.state()
    assert t == gens
    assert np.array_equal(k, st.k)
    e, f = inst.history(0, gens)
    assert np.array_equal(e, st.hist_e) and np.array_equal(f, st.hist_f)
    assert np.array_equal(inst.fitness(), st.f)
    assert np.array_equal(inst.alleles(), st.x)
    bits, bf, bg, bc = inst.best()
    assert (bf, bg, bc) == tuple(int(v) for v in st.best)
    assert np.array_equal(bits, st.best_x)


SPECS = [  # (ng, np, rule, D, lam, wide items)
    (5, 7, 0, 100, 1, False), (50, 32, 0, 100, 1, False), (100, 64, 1, 100, 1, False),
    (257, 9, 0, 100, 1, False), (1000, 40, 1, 100, 1, False), (2048, 33, 0, 100, 1, False),
    (2055, 20, 0, 12, 1, False), (4099, 11, 1, 100, 3, False), (700, 50, 0, 100, 1, True),
    (31, 128, 0, 100, 1, False), (6000, 17, 0, 100, 1, False), (90, 256, 1, 100, 1, False),
]


def make(spec, i):
    ng, np_, rule, D, lam, wide = spec
    if wide:
        rng = np.random.default_rng(i)
        prob = W.custom_problem(rng.integers(0, 5000, ng), rng.integers(0, 5000, ng), 5000 * ng // 4)
    else:
        prob = W.knapsack(ng, 100 + i)
    inst = Q.Instance(prob, np_, seed=i + 1, inst=i, D=D, lam=lam, rule=rule)
    return prob, inst


def test_batch_matches_each_instance_alone():
    made = [make(s, i) for i, s in enumerate(SPECS)]
    with Q.Batch([m[1] for m in made]) as b:
        for g in (5, 5, 3, 5):          # repeated lengths replay a captured graph
            b.run(g)
    for i, (s, (prob, inst)) in enumerate(zip(SPECS, made)):
        check_against_oracle(inst, prob, s[1], 18, i + 1, i, s[3], s[4], s[2])
        inst.close()


def test_batch_per_generation_form():
    """A member with QIEO_FLAG_PER_GENERATION makes the batch run one launch per generation
    (graph replay for repeated lengths) instead of one persistent launch; same results."""
    made = []
    for i, s_ in enumerate(SPECS[:7]):
        ng, np_, rule, D, lam, wide = s_
        prob = W.knapsack(ng, 100 + i) if not wide else make(s_, i)[0]
        inst = Q.Instance(prob, np_, seed=i + 1, inst=i, D=D, lam=lam, rule=rule,
                          flags=Q.QIEO_FLAG_PER_GENERATION if i == 3 else 0)
        made.append((prob, inst))
    with Q.Batch([m[1] for m in made]) as b:
        for g in (6, 6, 4):
            b.run(g)
    for i, (s_, (prob, inst)) in enumerate(zip(SPECS[:7], made)):
        check_against_oracle(inst, prob, s_[1], 16, i + 1, i, s_[3], s_[4], s_[2])
        inst.close()


def test_batch_and_single_runs_interleave():
    """Members keep their own generation counters: single runs and batch runs mix."""
    made = [make(s, i) for i, s in enumerate(SPECS[:6])]
    made[0][1].run(3)
    made[3][1].run(1)
    with Q.Batch([m[1] for m in made]) as b:
        b.run(4)
        made[2][1].run(2)
        b.run(4)
    for i, (s, (prob, inst)) in enumerate(zip(SPECS[:6], made)):
        k, t = inst.state()
        gens = 8 + (3 if i == 0 else 1 if i == 3 else 2 if i == 2 else 0)
        check_against_oracle(inst, prob, s[1], gens, i + 1, i, s[3], s[4], s[2])
        inst.close()


def test_batch_sample_of_the_batched_workload():
    """The first 24 instances of the 256-instance manifest (Ng log-uniform in [50, 20000],
    Np in {32..512}, seeds 1..24), 12 generations."""
    specs = W.batch_manifest(256)[:24]
    insts = []
    for sp in specs:
        prob = W.knapsack(sp.ng, sp.seed)
        insts.append((prob, sp, Q.Instance(prob, sp.np_, seed=sp.seed, inst=sp.seed)))
    with Q.Batch([x[2] for x in insts]) as b:
        b.run(12)
    for prob, sp, inst in insts:
        check_against_oracle(inst, prob, sp.np_, 12, sp.seed, sp.seed)
        inst.close()


def test_autotune_keeps_results_and_is_remembered():
    prob = W.knapsack(300, 21)
    with Q.Instance(prob, 48, seed=21) as inst:
        shape = inst.autotune(4)
        assert shape.lanes_per_row in (1, 2, 4, 8, 16, 32)
        k, t = inst.state()
        assert t == 0 and not k.any()
        inst.run(25)
        check_against_oracle(inst, prob, 48, 25, 21, 0)
    with Q.Instance(prob, 48, seed=22) as other:      # same (ng, np, D, rule, items) key
        s2 = other.shape()
        assert (s2.lanes_per_row, s2.warps_per_row) == (shape.lanes_per_row, shape.warps_per_row)


def test_batch_rejects_bad_members():
    prob = W.knapsack(50, 1)
    with Q.Instance(prob, 8) as a, Q.Instance(prob, 8, elite_on_host=1) as h:
        with pytest.raises(Q.QieoError):
            Q.qieo_create_batch([a.h, a.h])
        with pytest.raises(Q.QieoError):
            Q.qieo_create_batch([a.h, h.h])


def test_batch_with_converging_members():
    """Members with QIEO_FLAG_CONVERGE stop at the oracle's stopping generation inside the
    batched runs (some inside a run, one on a run's last generation) while the others keep
    going; every member equals its own oracle run."""
    from oracle import oracle as O
    cases = [(200, 30, 3), (120, 17, 8), (60, 5, 2), (60, 8, 2), (300, 40, 11)]
    made = []
    for ng, np_, seed in cases:
        prob = W.knapsack(ng, seed)
        ref = O.run(prob, np_, 300, seed=seed, window=20)
        made.append((prob, np_, seed, ref, Q.Instance(prob, np_, seed=seed, flags=Q.QIEO_FLAG_CONVERGE)))
    plain_prob = W.knapsack(500, 77)
    plain = Q.Instance(plain_prob, 24, seed=77)
    first = int(made[2][3].t[0])           # one member stops exactly at the end of run 1
    with Q.Batch([m[4] for m in made] + [plain]) as b:
        b.run(first)
        for g in (25, 25, 25, 25, 25, 25, 25, 25, 25, 25):
            b.run(g)
    total = first + 250
    for prob, np_, seed, ref, inst in made:
        k, t = inst.state()
        assert ref.stopped and t == int(ref.t[0]) <= total
        assert np.array_equal(k, ref.k)
        e, f = inst.history(0, t)
        assert np.array_equal(e, ref.hist_e) and np.array_equal(f, ref.hist_f)
        bits, bf, bg, bc = inst.best()
        assert (bf, bg, bc) == tuple(int(v) for v in ref.best)
        assert inst.convergence()[0]
        inst.close()
    check_against_oracle(plain, plain_prob, 24, total, 77, 0)
    plain.close()


def test_one_call_batched_run():
    """qieo_run_batch equals a kept batch (and each member's oracle run)."""
    made = [make(s, i) for i, s in enumerate(SPECS[:5])]
    Q.qieo_run_batch([m[1] for m in made], 9)
    Q.qieo_run_batch([m[1] for m in made], 4)
    for i, (s, (prob, inst)) in enumerate(zip(SPECS[:5], made)):
        check_against_oracle(inst, prob, s[1], 13, i + 1, i, s[3], s[4], s[2])
        inst.close()


def test_batch_from_saturated_states():
    """Batched members that start fully saturated (fixed-allele passes from the first
    generation, rows that disagree with the elite drawing again), against the oracle run
    on each alone."""
    from saturated import load_state, saturated_start
    from oracle import oracle as O
    specs = [(3001, 83, 0), (1500, 40, 1), (5000, 64, 0)]
    made = []
    for i, (ng, np_, rule) in enumerate(specs):
        prob = W.knapsack(ng, 50 + i)
        k0 = saturated_start(ng, np_, 60 + i, n_odd=5, flips=30)
        inst = Q.Instance(prob, np_, seed=i + 3, rule=rule)
        load_state(inst, k0)
        made.append((prob, k0, inst))
    with Q.Batch([m[2] for m in made]) as b:
        for g in (30, 30, 11):
            b.run(g)
    for i, ((ng, np_, rule), (prob, k0, inst)) in enumerate(zip(specs, made)):
        st = O.State(np_, ng)
        st.k[:] = k0
        O.run(prob, np_, 71, seed=i + 3, rule=rule, state=st)
        k, t = inst.state()
        assert t == 71
        assert np.array_equal(k, st.k)
        e, f = inst.history(0, 71)
        assert np.array_equal(e, st.hist_e) and np.array_equal(f, st.hist_f)
        assert np.array_equal(inst.alleles(), st.x)
        bits, bf, bg, bc = inst.best()
        assert (bf, bg, bc) == tuple(int(v) for v in st.best)
        inst.close()


def test_persistent_batch_wait_that_runs_out_is_reported():
    """In the persistent form a segment of a member's next generation waits, bounded, for
    that member's previous generation. With a 1 ns bound the waits of that member run out:
    the run still ends (no trap, no hang), the member reports QIEO_ERR_TIMEOUT, the other
    members are unaffected, and after qieo_reset the member runs correctly again."""
    probs = [W.knapsack(3000, 41), W.knapsack(2500, 42)]
    a = Q.Instance(probs[0], 120, seed=41)
    b = Q.Instance(probs[1], 90, seed=42)
    try:
        a.set_wait_timeout(1)
        with Q.Batch([a, b]) as bt:
            bt.run(6)
        with pytest.raises(Q.QieoError) as e:
            a.synchronize()
        assert e.value.status == Q.QIEO_ERR_TIMEOUT
        check_against_oracle(b, probs[1], 90, 6, 42, 0)
        a.set_wait_timeout(10 * 10**9)
        a.reset()
        with Q.Batch([a]) as bt:
            bt.run(6)
        check_against_oracle(a, probs[0], 120, 6, 41, 0)
    finally:
        a.close()
        b.close()
