"""The fixed-vector words and the sparse form of a generation, bit for bit against the CPU
oracle.

An instance that keeps the words (the one-launch-per-generation deferred form: rule R1,
items in [0, 255], 16-bit state, the default tile) records for every 8-gene vector whether
all its qubits sit at a bound, and a generation in which most vectors are fixed processes
in full only the vectors that are not, or that the previous elite turns away from their
bound. The cases cover ragged tiles and row groups, splits of a run (the first generation
of a run does not rotate), segments from 8 to 256 rows, starts from saturated states, the
switch between the dense and the sparse form, and every way the state changes outside the
kernels that keep the words (batches, checkpoints, a new launch shape).
"""
import numpy as np
import pytest

from paper_2609_30862_gb300 import qieo as Q
from paper_2609_30862_gb300 import workload as W
from saturated import load_state, saturated_start

pytestmark = pytest.mark.gpu

PG = Q.QIEO_FLAG_PER_GENERATION          # one launch per generation at any size
SPARSE = PG | Q.QIEO_FLAG_SPARSE_ALWAYS


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Q.load()


def check(I, st, gens):
    k, t = I.state()
    assert t == gens == int(st.t[0])
    assert np.array_equal(k, st.k), "angle indices differ"
    e, f = I.history(0, gens)
    assert np.array_equal(e, st.hist_e), "elite indices differ"
    assert np.array_equal(f, st.hist_f), "elite fitness differs"
    assert np.array_equal(I.fitness(), st.f), "fitness differs"
    assert np.array_equal(I.alleles(), st.x), "alleles differ"
    bits, bf, bg, bc = I.best()
    assert (bf, bg, bc) == tuple(int(v) for v in st.best)
    assert np.array_equal(bits, st.best_x)


def run_both(prob, np_, chunks, seed, flags, shape=None, k0=None, fixed_words=1, rule=0):
    from oracle import oracle as O
    gens = int(sum(chunks))
    st = O.State(np_, prob.ng)
    if k0 is not None:
        st.k[:] = k0
    O.run(prob, np_, gens, seed=seed, state=st, rule=rule)
    with Q.Instance(prob, np_, seed=seed, flags=flags, rule=rule) as I:
        if shape is not None:
            I.set_shape(*shape)
        assert I.shape().fixed_words == fixed_words
        if k0 is not None:
            load_state(I, k0)
        for g in chunks:
            I.run(g)
        check(I, st, gens)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("flags", [SPARSE, PG])
@pytest.mark.parametrize("ng,np_,seed", [(4696, 70, 61), (2100, 19, 62), (1500, 8, 63)])
def test_natural_collapse(flags, ng, np_, seed, rule):
    """Spread generations, the collapse, and the saturated tail, in runs of several lengths:
    three tiles with a ragged last one (4,696 genes), a ragged last group of 8 rows (70 and
    19 rows), one tile and one row group (1,500 x 8). SPARSE_ALWAYS takes the sparse form
    from the first generation, the default once half of the vectors is fixed; rules R1 and
    R2 (which rotates only the qubits whose allele differed from the elite's)."""
    run_both(W.knapsack(ng, seed), np_, [1, 60, 139, 50], seed, flags, rule=rule)


@pytest.mark.parametrize("flags", [SPARSE, PG])
@pytest.mark.parametrize("shape", [(32, 8, 1), (32, 8, 2), (32, 8, 5), (32, 8, 0)])
def test_segment_lengths(flags, shape):
    """Grids of 1, 2, 5 and the default number of blocks: segments of up to 256 rows (cut
    at multiples of 8), 600 rows in two tiles of which the second holds 7 vectors."""
    run_both(W.knapsack(2100, 64), 600, [30, 90], 64, flags, shape=shape)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("flags", [SPARSE, PG])
def test_from_saturated_states(flags, rule):
    """Every qubit at a bound from the start: rows share one pattern except 9 with 40 genes
    flipped, so the elite's column disagreements make whole columns unstable. The state is
    placed through a checkpoint, which clears the words."""
    k0 = saturated_start(3001, 83, 71 + rule, n_odd=9, flips=40)
    run_both(W.knapsack(3001, 71), 83, [1, 2, 37, 25], 71, flags, k0=k0, rule=rule)


def test_fixed_words_kept_where_the_form_allows():
    prob = W.knapsack(3001, 2)
    cases = [
        (PG, 0, 1),
        (PG | Q.QIEO_FLAG_NO_FIXED_WORDS, 0, 0),
        (PG, 1, 1),                                   # rule R2
        (PG | Q.QIEO_FLAG_STATE_I8, 0, 0),
        (PG | Q.QIEO_FLAG_FORCE_WIDE, 0, 0),
        (PG | Q.QIEO_FLAG_SIXTEEN, 0, 0),
        (PG | Q.QIEO_FLAG_CONVERGE, 0, 0),
        (0, 0, 0),                                    # resident form at this size
        (Q.QIEO_FLAG_STREAMED, 0, 0),                 # cooperative at this size
    ]
    for flags, rule, want in cases:
        with Q.Instance(prob, 64, rule=rule, flags=flags) as I:
            assert I.shape().fixed_words == want, (flags, rule)
    with Q.Instance(prob, 64, flags=PG, row0=0) as I:      # a row block of a sharded population
        assert I.shape().fixed_words == 0
    with Q.Instance(prob, 64, flags=PG) as I:
        I.set_shape(32, 4, 0)                         # another tile: no words
        assert I.shape().fixed_words == 0
        I.set_shape(32, 8, 0)
        assert I.shape().fixed_words == 1


def test_shape_changes_keep_results():
    """Words dropped and taken up again when the launch shape changes between runs."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(3001, 72), 96, 72
    st = O.run(prob, np_, 160, seed=seed)
    with Q.Instance(prob, np_, seed=seed, flags=SPARSE) as I:
        I.run(70)
        I.set_shape(32, 4, 0)
        I.run(30)
        I.set_shape(32, 8, 3)
        I.run(60)
        check(I, st, 160)


def test_batch_between_single_runs():
    """A batched run (whose kernels keep no words) between single runs of the same
    instances."""
    from oracle import oracle as O
    probs = [W.knapsack(2500, 80 + i) for i in range(3)]
    insts = [Q.Instance(p, 72, seed=80 + i, flags=SPARSE) for i, p in enumerate(probs)]
    try:
        for I in insts:
            I.run(90)
        with Q.Batch(insts) as b:
            b.run(25)
        for I in insts:
            I.run(45)
        for i, (I, p) in enumerate(zip(insts, probs)):
            check(I, O.run(p, 72, 160, seed=80 + i), 160)
    finally:
        for I in insts:
            I.close()


def test_checkpoint_round_trip_mid_collapse():
    """Save in the middle of the collapse, load into a fresh instance (its words cleared),
    continue: equal to the unbroken oracle run."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(3001, 90), 88, 90
    st = O.run(prob, np_, 200, seed=seed)
    with Q.Instance(prob, np_, seed=seed, flags=SPARSE) as a:
        a.run(110)
        blob = a.save()
    with Q.Instance(prob, np_, seed=seed, flags=SPARSE) as b:
        b.run(7)                                      # words of another state, then replaced
        b.load(blob)
        b.run(90)
        check(b, st, 200)


def test_drawn_vectors_equal_the_oracle_count_of_unstable_vectors():
    """In a sparse generation exactly the unstable vectors draw: the others have every qubit
    at a bound on the side of the previous elite's allele. Counted here from the oracle's
    states (the state observed in generation t - 1 and the elite alleles of t - 1) for every
    generation of one run but its first (dense) one."""
    from oracle import oracle as O
    prob, np_, seed, G = W.knapsack(3000, 95), 72, 95, 160      # 3000 genes: no padding
    K, nv = 25, 3000 // 8
    want = []                                       # drawn vectors of generations 1 .. G-1
    st = O.State(np_, prob.ng)
    for t in range(G - 1):
        k_obs = st.k.copy()                         # the state generation t observes
        O.run(prob, np_, 1, seed=seed, state=st)    # generation t (and its CIP)
        xe = st.x[int(st.hist_e[-1])].astype(np.int16).reshape(nv, 8)
        at = (np.abs(k_obs) == K).reshape(np_, nv, 8)
        side = (k_obs > 0).astype(np.int16).reshape(np_, nv, 8)
        stable = (at & (side == xe[None])).all(axis=2)   # stable in generation t + 1
        want.append(np_ * nv - int(stable.sum()))
    O.run(prob, np_, 1, seed=seed, state=st)
    with Q.Instance(prob, np_, seed=seed, flags=SPARSE) as I:
        I.run(G)
        got = I.drawn_vectors(0, G)
        check(I, st, G)
    assert got[0] == np_ * nv                       # generation 0: nothing is fixed
    assert list(got[1:]) == want
    assert min(want) < np_ * nv // 10               # the run reaches the collapsed phase
    with Q.Instance(prob, np_, seed=seed, flags=PG | Q.QIEO_FLAG_NO_FIXED_WORDS) as I:
        I.run(2)
        with pytest.raises(Q.QieoError):
            I.drawn_vectors(0, 2)


@pytest.mark.parametrize("D", [4, 12, 40, 1000])
def test_other_rotation_steps(D):
    """Other rotation steps π/D change K, the bound offsets 0 and 8K and the threshold table
    whose zero low words mark a fixed vector; D = 4 (K = 1) saturates after one step."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(2600, 100 + D), 40, 100 + D
    gens = 140 if D < 1000 else 60
    st = O.run(prob, np_, gens, seed=seed, D=D)
    for flags in (SPARSE, PG):
        with Q.Instance(prob, np_, seed=seed, D=D, flags=flags) as I:
            assert I.shape().fixed_words == 1
            I.run(gens // 3)
            I.run(gens - gens // 3)
            check(I, st, gens)


def test_item_sums_at_the_form_limit():
    """The form needs the sums of all weights and of all values below 2^25 (the biased row
    changes of a sparse generation stay below 2^26): 131,584 weights of 255 (512 below 2^25)
    keep the words and the run equals the oracle; 131,600 (at or above 2^25) do not."""
    from oracle import oracle as O
    limit = 1 << 25
    ng = 131_584
    below = W.custom_problem(np.full(ng, 255, dtype=np.int32), np.full(ng, 7, dtype=np.int32), 255 * ng // 2)
    assert 255 * ng < limit
    with Q.Instance(below, 24, seed=5, flags=SPARSE) as I:
        assert I.shape().fixed_words == 1
        I.run(80)
        check(I, O.run(below, 24, 80, seed=5, kind="omp"), 80)
    ng = 131_600
    at = W.custom_problem(np.full(ng, 255, dtype=np.int32), np.full(ng, 7, dtype=np.int32), 255 * ng // 2)
    assert 255 * ng >= limit
    with Q.Instance(at, 4, seed=5, flags=PG) as I:
        assert I.shape().fixed_words == 0
