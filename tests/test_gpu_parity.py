"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is element by element: angle indices, alleles, fitness, elite index and
fitness per generation, the best record and the threshold table must be identical (all
are integers; the method has no floating point after the table).
"""
import numpy as np
import pytest

from paper_2609_30862_gb300 import qieo as Q
from paper_2609_30862_gb300 import workload as W
from saturated import load_state, saturated_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Q.load()


def compare(prob, np_, chunks, seed=1, inst=0, D=100, lam=1, rule=0, flags=0, host=0,
            shape=None, kind="serial", oracle_mod=None, check_alleles=True):
    from oracle import oracle as O
    gens = int(sum(chunks))
    st = O.run(prob, np_, gens, seed=seed, inst=inst, D=D, lam=lam, rule=rule, kind=kind)
    with Q.Instance(prob, np_, seed=seed, inst=inst, D=D, lam=lam, rule=rule,
                    elite_on_host=host, flags=flags) as I:
        if shape is not None:
            I.set_shape(*shape)
        for g in chunks:
            I.run(g)
        k, t = I.state()
        assert t == gens == int(st.t[0])
        assert np.array_equal(k, st.k), "angle indices differ"
        e, f = I.history(0, gens)
        assert np.array_equal(e, st.hist_e), "elite indices differ"
        assert np.array_equal(f, st.hist_f), "elite fitness differs"
        assert np.array_equal(I.fitness(), st.f), "fitness differs"
        if check_alleles:
            assert np.array_equal(I.alleles(), st.x), "alleles differ"
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in st.best)
        assert np.array_equal(bits, st.best_x)
        return I.shape()


def test_threshold_table_matches_oracle():
    from oracle import oracle as O
    for D in (4, 12, 100, 1000, 4000):
        with Q.Instance(W.knapsack(8, 1), 1, D=D) as I:
            assert np.array_equal(I.thresholds(), O.threshold_table(D)), D


def test_device_philox_known_answers():
    """The device Philox4x32-10 on the published known-answer vectors (tests/golden)."""
    from test_oracle_pins import read_philox_kat
    rows = read_philox_kat()
    ck = np.array([c + k for c, k, _ in rows], dtype=np.uint32)
    out = Q.qieo_philox(ck)
    for (c, k, want), got in zip(rows, out):
        assert [int(x) for x in got] == want


def test_device_philox_matches_oracle():
    from oracle import oracle as O
    rng = np.random.default_rng(7)
    ck = rng.integers(0, 2**32, size=(4096, 6), dtype=np.uint64).astype(np.uint32)
    ck[0] = 0
    ck[1] = 0xFFFFFFFF
    out = Q.qieo_philox(ck)
    for row, got in zip(ck[:512], out[:512]):
        assert np.array_equal(got, O.philox4x32_10(row[:4], row[4:]))


@pytest.mark.parametrize("flags", [0, Q.QIEO_FLAG_STREAMED, Q.QIEO_FLAG_PER_GENERATION])
def test_c1_full_run(flags):
    """Ng = 100, Np = 64, 500 generations, Philox seed 1: the small named workload, as one
    cooperative launch with the state resident in shared memory (the default at this
    size), as one cooperative launch streaming the state, and as one launch per
    generation."""
    c = W.WORKLOADS["c1"]
    shape = compare(W.knapsack(c["ng"], c["item_seed"]), c["np"], [c["gens"]], seed=c["seed"],
                    inst=c["inst"], flags=flags)
    assert shape.persistent == (0 if flags == Q.QIEO_FLAG_PER_GENERATION else 1)
    assert shape.resident == (1 if flags == 0 else 0)


def test_c1_rule_r2():
    c = W.WORKLOADS["c1"]
    compare(W.knapsack(c["ng"], c["item_seed"]), c["np"], [300], seed=3, rule=1)


@pytest.mark.parametrize("flags", [Q.QIEO_FLAG_NO_GRAPH, Q.QIEO_FLAG_FORCE_WIDE,
                                   Q.QIEO_FLAG_SYNC_RUN | Q.QIEO_FLAG_TIME_KERNELS,
                                   Q.QIEO_FLAG_COOPERATIVE | Q.QIEO_FLAG_FORCE_WIDE,
                                   Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_NO_GRAPH,
                                   Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_FORCE_WIDE,
                                   Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_SYNC_RUN |
                                   Q.QIEO_FLAG_TIME_KERNELS])
def test_flags_do_not_change_results(flags):
    compare(W.knapsack(700, 5), 48, [60], seed=5, rule=0, flags=flags)


@pytest.mark.parametrize("rule", [0, 1])
def test_cooperative_launch(rule):
    """One cooperative launch per run (grid barrier between generations) gives the same
    results as one launch per generation."""
    compare(W.knapsack(2500, 15), 60, [7, 7, 7, 4], seed=15, rule=rule,
            flags=Q.QIEO_FLAG_COOPERATIVE)
    compare(W.knapsack(2500, 15), 60, [7, 7], seed=15, rule=rule,
            flags=Q.QIEO_FLAG_COOPERATIVE | Q.QIEO_FLAG_REGISTER_PREFETCH)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("flags,shape", [(0, None), (Q.QIEO_FLAG_FORCE_WIDE, None), (0, (32, 2, 0)),
                                         (0, (4, 1, 7)), (0, (32, 8, 40)), (0, (1, 1, 64)),
                                         (Q.QIEO_FLAG_TIME_GENERATIONS, None)])
def test_resident_form(rule, flags, shape):
    """The state kept in shared memory for a whole run (one cooperative launch): across run
    boundaries, with wide item sums, with several rows per pass, shares that span two tiles,
    one lane per row tile (256 rows per pass), and with per-generation device timestamps."""
    prob = W.knapsack(5000, 17)
    got = compare(prob, 90, [9, 9, 5], seed=17, rule=rule, flags=flags, shape=shape)
    assert got.resident == 1 and got.persistent == 1


def test_resident_form_wide_items_and_large_lambda():
    rng = np.random.default_rng(4)
    prob = W.custom_problem(rng.integers(0, 3000, 900), rng.integers(0, 3000, 900), 3000 * 900 // 3)
    got = compare(prob, 70, [13, 7], seed=4, lam=7, rule=1)
    assert got.resident == 1 and got.narrow == 0


@pytest.mark.parametrize("rule", [0, 1])
def test_host_determine_elite_variant(rule):
    compare(W.knapsack(500, 2), 40, [25, 15], seed=2, rule=rule, host=1)


@pytest.mark.parametrize("flags", [0, Q.QIEO_FLAG_PER_GENERATION])
def test_split_runs(flags):
    compare(W.knapsack(333, 8), 37, [1, 10, 29, 7], seed=8, rule=1, flags=flags)


@pytest.mark.parametrize("rule", [0, 1])
def test_repeated_run_length_uses_graph(rule):
    """The second and later runs of the same length replay a captured CUDA graph (one launch
    per generation)."""
    compare(W.knapsack(1200, 6), 50, [6, 6, 6, 6, 3, 6], seed=6, rule=rule,
            flags=Q.QIEO_FLAG_PER_GENERATION)


@pytest.mark.parametrize("ng", [1, 7, 8, 9, 31, 33, 127, 255, 257, 2048, 2055, 4099])
@pytest.mark.parametrize("np_", [1, 3, 19])
def test_ragged_sizes(ng, np_):
    """Ragged gene and chromosome counts, through the default (cooperative at these sizes)
    and the one-launch-per-generation forms."""
    compare(W.knapsack(ng, ng + np_), np_, [12], seed=ng, inst=np_, rule=(ng + np_) % 2)
    compare(W.knapsack(ng, ng + np_), np_, [5, 7], seed=ng, inst=np_, rule=(ng + np_) % 2,
            flags=Q.QIEO_FLAG_PER_GENERATION)


@pytest.mark.parametrize("shape", [(32, 8, 0), (32, 8, 1), (32, 8, 7), (32, 4, 3), (32, 2, 50),
                                   (32, 1, 0), (16, 1, 9), (8, 1, 0), (4, 1, 33), (2, 1, 0),
                                   (1, 1, 5), (1, 1, 0), (32, 8, 100000)])
def test_launch_shape_independence(shape):
    """Results do not depend on the block shape: integer sums are exact and every draw is
    keyed by (gene, chromosome, generation), not by thread."""
    compare(W.knapsack(1500, 4), 70, [15], seed=4, shape=shape)


@pytest.mark.parametrize("rule", [0, 1])
def test_async_ring_and_register_streaming_agree(rule):
    """The state streams through the per-thread cp.async ring by default and through
    register prefetch with QIEO_FLAG_REGISTER_PREFETCH. Both equal the oracle (also across
    run boundaries and with one launch per generation)."""
    prob = W.knapsack(5000, 17)
    compare(prob, 90, [9, 9, 5], seed=17, rule=rule)
    compare(prob, 90, [9, 9, 5], seed=17, rule=rule, flags=Q.QIEO_FLAG_REGISTER_PREFETCH)
    compare(prob, 90, [6, 4], seed=17, rule=rule, flags=Q.QIEO_FLAG_COOPERATIVE)


def test_long_shares_split_into_segments():
    """Two blocks over 6000 rows x 2 tiles: each block's share crosses a tile boundary and
    exceeds the 1536 tile-rows its shared memory sums at once. With fixed-vector words the
    queue's segments are at most 256 rows."""
    prob = W.knapsack(2050, 18)
    shape = compare(prob, 6000, [2, 1], seed=18, shape=(32, 8, 2), flags=Q.QIEO_FLAG_NO_FIXED_WORDS)
    assert shape.tiles == 2 and shape.rows_per_cta == 1536 and shape.fixed_words == 0
    compare(prob, 6000, [2, 1], seed=18, shape=(32, 8, 2), flags=Q.QIEO_FLAG_REGISTER_PREFETCH)
    shape = compare(prob, 6000, [2, 1], seed=18, shape=(32, 8, 2))
    assert shape.tiles == 2 and shape.rows_per_cta == 256 and shape.fixed_words == 1


def test_wide_items_and_penalty():
    """Weights/values outside the 16-bit packed range, negative values, lambda > 1."""
    rng = np.random.default_rng(11)
    w = rng.integers(0, 2**31 - 1, 300).astype(np.int32)
    v = rng.integers(-2**31, 2**31 - 1, 300).astype(np.int32)
    prob = W.custom_problem(w, v, int(w.astype(np.int64).sum() // 3))
    shape = compare(prob, 24, [20], seed=9, lam=7)
    assert shape.narrow == 0
    prob2 = W.custom_problem(rng.integers(0, 1000, 900), rng.integers(0, 1000, 900), 20000)
    compare(prob2, 33, [20], seed=10, lam=3, rule=1)


def test_scan_mode_elite():
    """lambda * sum(w) beyond the 40-bit elite key: the elite comes from a lowest-index
    argmax over the fitness array instead of the key."""
    prob = W.knapsack(300, 13)
    compare(prob, 45, [25], seed=13, lam=2**30)


def test_many_tiles_packed_and_wide_sums():
    """One lane per row tile. 263 tiles per row fit the 12-bit tile count of the packed row
    word; 4,100 tiles do not, so the 64-bit row sums are used."""
    prob = W.knapsack(2100, 14)
    shape = compare(prob, 12, [8], seed=14, shape=(1, 1, 0))
    assert shape.tiles == 263 and shape.narrow == 1
    prob = W.knapsack(32800, 15)
    shape = compare(prob, 12, [3], seed=15, shape=(1, 1, 0))
    assert shape.tiles == 4100 and shape.narrow == 0


@pytest.mark.parametrize("ng,narrow", [(263000, 1), (263200, 0)])
def test_packed_row_sum_limit(ng, narrow):
    """Items of 255 everywhere: total weight just below 2^26 keeps the packed row word,
    just above it switches to the 64-bit row sums. Both match the oracle."""
    w = np.full(ng, 255, dtype=np.int32)
    prob = W.custom_problem(w, w.copy(), int(w.sum()) // 2)
    shape = compare(prob, 4, [3], seed=16)
    assert shape.narrow == narrow


def test_narrow_boundary_items():
    """Largest items the packed 16-bit path accepts (255) and zero items."""
    ng = 4096
    w = np.full(ng, 255, dtype=np.int32)
    v = np.full(ng, 255, dtype=np.int32)
    w[::7] = 0
    prob = W.custom_problem(w, v, int(w.sum()) // 2)
    shape = compare(prob, 9, [10], seed=12)
    assert shape.narrow == 1


@pytest.mark.parametrize("D", [4, 12, 1000])
def test_other_rotation_steps(D):
    compare(W.knapsack(150, 3), 20, [80], seed=3, D=D, rule=D % 8 // 4)


def test_degenerate_capacity():
    """W = 0: every non-empty pack is infeasible; all-zero weights: every pack fits."""
    compare(W.custom_problem([1, 2, 3, 4, 5], [1, 1, 1, 1, 1], 0), 6, [30], seed=1)
    compare(W.custom_problem([0] * 20, list(range(20)), 0), 6, [30], seed=1)


def test_reset_and_zero_generations():
    prob = W.knapsack(100, 1)
    with Q.Instance(prob, 16) as I:
        I.run(0)
        bits, f, g, c = I.best()
        assert (f, g, c) == (0, -1, -1)
        k, t = I.state()
        assert t == 0 and not k.any()
        I.run(17)
        I.reset()
        k, t = I.state()
        assert t == 0 and not k.any()
        assert I.best()[2] == -1
    compare(prob, 16, [17], seed=1)


@pytest.mark.parametrize("flags", [0, Q.QIEO_FLAG_STREAMED])
def test_c2_full_size(flags):
    """Ng = 10,000, Np = 1,024, 1,000 generations: bit-exact against the OpenMP build of
    the oracle (identical to the serial one by construction and by test), with the state
    resident in shared memory (the default: 20 MB fits the SMs' shared memory) and
    streamed from device memory every generation."""
    c = W.WORKLOADS["c2"]
    shape = compare(W.knapsack(c["ng"], c["item_seed"]), c["np"], [c["gens"]], seed=c["seed"],
                    inst=c["inst"], kind="omp", flags=flags)
    assert shape.resident == (1 if flags == 0 else 0)


def test_c3_full_run_properties():
    """All 200 generations of c3 as the benchmark runs them, checked by what holds at any
    size (the element-by-element oracle comparison of the same run is test_c3_full_run in
    test_gpu_fullsize.py): the best record is the first generation of largest elite fitness
    in the history, its alleles evaluate to its fitness by eq. (1) (recomputed on the host),
    every elite index is a chromosome, every angle index lies in [-K, K], and the allele
    planes of the last generation evaluate to the reported fitness of every chromosome."""
    c = W.WORKLOADS["c3"]
    prob = W.knapsack(c["ng"], c["item_seed"])
    with Q.Instance(prob, c["np"], seed=c["seed"], inst=c["inst"]) as I:
        I.run(c["gens"])
        e, f = I.history(0, c["gens"])
        bits, bf, bg, bc = I.best()
        assert bf == int(f.max()) and bg == int(np.argmax(f)) and bc == int(e[bg])
        assert np.all((e >= 0) & (e < c["np"]))
        w = prob.weights.astype(np.int64)
        v = prob.values.astype(np.int64)
        sw, sv = int(bits.astype(np.int64) @ w), int(bits.astype(np.int64) @ v)
        assert bf == (sv if sw <= prob.capacity else -(sw - prob.capacity))
        x = I.alleles()
        fit = I.fitness()
        for row in range(0, c["np"], 257):      # a sample of rows: eq. (1) from the alleles
            swr, svr = int(x[row].astype(np.int64) @ w), int(x[row].astype(np.int64) @ v)
            assert fit[row] == (svr if swr <= prob.capacity else -(swr - prob.capacity))
        k, t = I.state()
        assert t == c["gens"] and int(k.min()) >= -25 and int(k.max()) <= 25


def test_barrier_wait_timeout_is_reported():
    """A grid-barrier wait that runs out ends the run with QIEO_ERR_TIMEOUT (no trap, no
    hang); after qieo_reset the instance runs correctly again."""
    from oracle import oracle as O
    prob = W.knapsack(6000, 16)
    with Q.Instance(prob, 300, seed=16, flags=Q.QIEO_FLAG_COOPERATIVE) as I:
        assert I.shape().grid_ctas > 1
        I.set_wait_timeout(1)
        I.run(5)
        with pytest.raises(Q.QieoError) as e:
            I.synchronize()
        assert e.value.status == Q.QIEO_ERR_TIMEOUT
        I.set_wait_timeout(10 * 10**9)
        I.reset()
        I.run(5)
        k, t = I.state()
        ref = O.run(prob, 300, 5, seed=16)
        assert t == 5 and np.array_equal(k, ref.k)


@pytest.mark.parametrize("rule", [0, 1])
def test_unfused_four_launch_form(rule):
    """QIEO_FLAG_UNFUSED runs CIP, QIP, Evaluation and DetermineElite as four launches per
    generation; results equal the oracle (ragged ng, split runs), and with kernel timing
    every step's time is accounted for every generation."""
    prob = W.knapsack(1003, 31)
    compare(prob, 37, [6, 5], seed=31, rule=rule, flags=Q.QIEO_FLAG_UNFUSED)
    with Q.Instance(prob, 37, seed=31, rule=rule,
                    flags=Q.QIEO_FLAG_UNFUSED | Q.QIEO_FLAG_TIME_KERNELS) as I:
        I.run(8)
        I.run(4)
        ms, gens = I.phase_times()
        assert gens == 12
        assert all(v > 0 for v in ms.values()), ms


def test_host_elite_phase_time():
    prob = W.knapsack(500, 32)
    compare(prob, 20, [5], seed=32, host=1, flags=Q.QIEO_FLAG_TIME_KERNELS)
    with Q.Instance(prob, 20, seed=32, elite_on_host=1, flags=Q.QIEO_FLAG_TIME_KERNELS) as I:
        I.run(6)
        ms, gens = I.phase_times()
        assert gens == 6 and ms["determine_elite"] > 0 and ms["qip"] == 0


def _first_stable(hist_f, window=20):
    for t in range(window - 1, len(hist_f)):
        if np.all(hist_f[t - window + 1:t + 1] == hist_f[t]):
            return t
    return None


@pytest.mark.parametrize("where", ["inside", "boundary", "first", "no_graph"])
def test_convergence_stop_matches_oracle(where):
    """QIEO_FLAG_CONVERGE: the run stops at the generation the oracle's convergence test
    picks, whether that falls inside a run, on a run's last generation, or in the first
    run; runs after the stop change nothing."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(200, 3), 30, 3
    ref = O.run(prob, np_, 400, seed=seed, window=20)
    tc = int(ref.t[0]) - 1
    assert ref.stopped and tc == _first_stable(O.run(prob, np_, 400, seed=seed).hist_f)
    chunks = {"inside": [tc - 5, 50, 50], "boundary": [tc + 1, 30], "first": [400, 10],
              "no_graph": [7] * 40}[where]
    flags = Q.QIEO_FLAG_CONVERGE | (Q.QIEO_FLAG_NO_GRAPH if where == "no_graph" else 0)
    with Q.Instance(prob, np_, seed=seed, flags=flags) as I:
        for g in chunks:
            I.run(g)
        k, t = I.state()
        assert t == tc + 1
        assert np.array_equal(k, ref.k)
        e, f = I.history(0, t)
        assert np.array_equal(e, ref.hist_e) and np.array_equal(f, ref.hist_f)
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in ref.best)
        assert np.array_equal(bits, ref.best_x)
        assert I.convergence() == (True, 20)


def test_convergence_flag_off_runs_every_generation():
    from oracle import oracle as O
    prob = W.knapsack(200, 3)
    compare(prob, 30, [150], seed=3)
    with Q.Instance(prob, 30, seed=3, flags=Q.QIEO_FLAG_CONVERGE) as I:
        I.run(10)
        stopped, stable = I.convergence()
        ref = O.run(prob, 30, 10, seed=3, window=20)
        assert not stopped and stable == int(ref.conv[0])


@pytest.mark.parametrize("rule,D,ng", [(0, 100, 1003), (1, 100, 777), (0, 120, 64), (0, 4, 33)])
def test_byte_state_equals_oracle(rule, D, ng):
    """QIEO_FLAG_STATE_I8 stores every angle index in one byte: the same trajectory as the
    16-bit state (oracle), across split runs, ragged sizes and other rotation steps."""
    prob = W.knapsack(ng, 40 + D)
    compare(prob, 29, [7, 6, 7], seed=40, rule=rule, D=D, flags=Q.QIEO_FLAG_STATE_I8)


def test_byte_state_with_convergence_and_saturation():
    """Byte state through the saturated phase (fixed-allele passes) and the convergence stop."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(200, 3), 30, 3
    compare(prob, np_, [150, 60], seed=seed, flags=Q.QIEO_FLAG_STATE_I8)
    ref = O.run(prob, np_, 400, seed=seed, window=20)
    with Q.Instance(prob, np_, seed=seed, flags=Q.QIEO_FLAG_STATE_I8 | Q.QIEO_FLAG_CONVERGE) as I:
        I.run(400)
        k, t = I.state()
        assert t == int(ref.t[0]) and np.array_equal(k, ref.k)
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in ref.best)


def test_byte_state_needs_packed_item_sums():
    w = np.full(40, 300, dtype=np.int32)
    prob = W.custom_problem(w, w.copy(), 3000)
    with pytest.raises(Q.QieoError) as e:
        Q.Instance(prob, 8, flags=Q.QIEO_FLAG_STATE_I8)
    assert e.value.status == Q.QIEO_ERR_INVALID and "STATE_I8" in str(e.value)


@pytest.mark.parametrize("flags", [0, Q.QIEO_FLAG_PER_GENERATION, Q.QIEO_FLAG_STATE_I8,
                                   Q.QIEO_FLAG_CONVERGE])
def test_checkpoint_resume_is_bit_exact(flags):
    """Save after 30 generations, load into a fresh instance of the same problem and run up
    to 120 more: the state, the whole elite history, the best record and the convergence
    stop (here at generation 106) equal one uninterrupted run (and the oracle)."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(200, 3), 30, 3
    window = 20 if flags == Q.QIEO_FLAG_CONVERGE else 0
    ref = O.run(prob, np_, 150, seed=seed, window=window)
    with Q.Instance(prob, np_, seed=seed, flags=flags) as a:
        a.run(30)
        blob = a.save()
    with Q.Instance(prob, np_, seed=seed, flags=flags) as b:
        b.run(3)                                   # overwritten by the load
        b.load(blob)
        assert b.state()[1] == 30
        b.run(120)
        k, t = b.state()
        assert t == int(ref.t[0]) and np.array_equal(k, ref.k)
        e, f = b.history(0, t)
        assert np.array_equal(e, ref.hist_e) and np.array_equal(f, ref.hist_f)
        bits, bf, bg, bc = b.best()
        assert (bf, bg, bc) == tuple(int(v) for v in ref.best)
        assert np.array_equal(bits, ref.best_x)


def test_checkpoint_rejects_another_problem():
    with Q.Instance(W.knapsack(200, 3), 30, seed=3) as a:
        a.run(5)
        blob = a.save()
    with Q.Instance(W.knapsack(200, 3), 30, seed=4) as b:   # other Philox seed
        with pytest.raises(Q.QieoError) as e:
            b.load(blob)
        assert e.value.status == Q.QIEO_ERR_INVALID
        with pytest.raises(Q.QieoError):
            b.load(blob[:100])


def compare_from(prob, k0, chunks, seed=1, rule=0, flags=0, shape=None, D=100):
    from oracle import oracle as O
    np_, ng = k0.shape
    gens = int(sum(chunks))
    st = O.State(np_, ng)
    st.k[:] = k0
    O.run(prob, np_, gens, seed=seed, D=D, rule=rule, state=st)
    with Q.Instance(prob, np_, seed=seed, D=D, rule=rule, flags=flags) as I:
        if shape is not None:
            I.set_shape(*shape)
        load_state(I, k0, D, byte_state=bool(flags & Q.QIEO_FLAG_STATE_I8))
        for g in chunks:
            I.run(g)
        k, t = I.state()
        assert t == gens
        assert np.array_equal(k, st.k), "angle indices differ"
        e, f = I.history(0, gens)
        assert np.array_equal(e, st.hist_e) and np.array_equal(f, st.hist_f)
        assert np.array_equal(I.fitness(), st.f)
        assert np.array_equal(I.alleles(), st.x)
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in st.best)
        assert np.array_equal(bits, st.best_x)


@pytest.mark.parametrize("flags,shape", [
    (0, None),                                              # cooperative at this size
    (Q.QIEO_FLAG_PER_GENERATION, None),
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_FORCE_WIDE, None),
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_STATE_I8, None),
    (Q.QIEO_FLAG_PER_GENERATION, (32, 2)),                  # four rows per pass
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_NO_GRAPH, (32, 8, 37)),   # odd grid
])
@pytest.mark.parametrize("rule", [0, 1])
def test_fixed_allele_passes_from_a_saturated_state(flags, shape, rule):
    """Every qubit starts at a bound, so passes are fixed-allele passes from the first
    generation on, except where a row disagrees with the elite: those rows rotate away from
    the bound, draw again, and come back. Runs split into several lengths, through each
    launch form, sum form, state width and tile shape."""
    k0 = saturated_start(3001, 83, 31 + rule, n_odd=9, flips=40)
    compare_from(W.knapsack(3001, 31), k0, [1, 2, 37, 25], seed=31, rule=rule, flags=flags,
                 shape=shape)


def test_fixed_allele_passes_through_natural_saturation():
    """A population that saturates on its own within a run: spread generations, the
    fixed-allele passes once qubits reach the bounds, and later elite changes."""
    compare(W.knapsack(4000, 41), 128, [180, 220], seed=41, rule=0,
            flags=Q.QIEO_FLAG_PER_GENERATION)
    compare(W.knapsack(4000, 42), 96, [400], seed=42, rule=1)


@pytest.mark.parametrize("flags,shape", [
    (0, (32, 8, 3)),                                        # cooperative, 134 rows per block
    (Q.QIEO_FLAG_PER_GENERATION, (32, 8, 3)),
    (Q.QIEO_FLAG_PER_GENERATION, (32, 2, 5)),               # four rows per pass, 6 tiles
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_FORCE_WIDE, (32, 8, 2)),
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_STATE_I8, (32, 4, 4)),
    (Q.QIEO_FLAG_PER_GENERATION | Q.QIEO_FLAG_NO_GRAPH, (32, 8, 1)),   # one block, whole queue
])
@pytest.mark.parametrize("rule", [0, 1])
def test_segment_queue(flags, shape, rule):
    """Grids small enough that each block's share is at least 64 tile-rows, so the deferred
    forms take their segments from the guided queue (large segments first, 4-row ones
    last) instead of equal static shares."""
    compare(W.knapsack(3001, 51), 200, [1, 30, 45], seed=51, rule=rule, flags=flags, shape=shape)
    k0 = saturated_start(3001, 200, 52 + rule, n_odd=11, flips=60)
    compare_from(W.knapsack(3001, 52), k0, [2, 40], seed=52, rule=rule, flags=flags, shape=shape)


def test_segment_queue_with_convergence_stop():
    """The convergence stop through queued per-generation launches (the stopping launch
    applies the last CIP alone; later launches do nothing)."""
    from oracle import oracle as O
    prob, np_, seed = W.knapsack(1200, 7), 256, 7
    ref = O.run(prob, np_, 600, seed=seed, window=20)
    assert ref.stopped
    tc = int(ref.t[0]) - 1
    with Q.Instance(prob, np_, seed=seed, flags=Q.QIEO_FLAG_CONVERGE) as I:
        I.set_shape(32, 8, 2)            # 1 tile x 256 rows: 128 rows per block
        for g in (tc - 7, 40, 40):
            I.run(g)
        k, t = I.state()
        assert t == tc + 1
        assert np.array_equal(k, ref.k)
        e, f = I.history(0, t)
        assert np.array_equal(e, ref.hist_e) and np.array_equal(f, ref.hist_f)
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in ref.best)


@pytest.mark.parametrize("ng,np_", [(1, 3), (9, 5), (16, 7), (17, 33), (4095, 9), (4096, 12), (4097, 40),
                                    (9001, 64), (2000, 700)])
def test_sixteen_genes_per_pass(ng, np_):
    """QIEO_FLAG_SIXTEEN (two 8-gene vectors per thread and pass) equals the oracle: ragged
    gene counts (odd vector counts leave a thread one active vector, short rows leave
    threads none), static shares and split runs."""
    prob = W.knapsack(ng, ng + 3 * np_)
    flags = Q.QIEO_FLAG_SIXTEEN | Q.QIEO_FLAG_PER_GENERATION
    compare(prob, np_, [7, 6], seed=ng, inst=np_, flags=flags)


def test_sixteen_genes_per_pass_queued():
    """The queued form: 9,000 genes (three 512-vector tiles per row) x 7,000 rows give each
    of the 304 blocks a share of at least 64 tile-rows, so the blocks take segments from the
    queue."""
    prob = W.knapsack(9000, 77)
    shape = compare(prob, 7000, [12, 8], seed=77, inst=2, kind="omp",
                    flags=Q.QIEO_FLAG_SIXTEEN | Q.QIEO_FLAG_PER_GENERATION)
    assert shape.persistent == 0


def test_sixteen_genes_per_pass_from_saturated_state():
    prob = W.knapsack(5000, 64)
    k0 = saturated_start(5000, 256, 65, n_odd=9, flips=40)
    from oracle import oracle as O
    st = O.State(256, 5000)
    st.k[:] = k0
    O.run(prob, 256, 30, seed=5, state=st)
    with Q.Instance(prob, 256, seed=5, flags=Q.QIEO_FLAG_SIXTEEN | Q.QIEO_FLAG_PER_GENERATION) as I:
        load_state(I, k0)
        I.run(30)
        k, t = I.state()
        assert t == 30 and np.array_equal(k, st.k)
        e, f = I.history(0, 30)
        assert np.array_equal(e, st.hist_e) and np.array_equal(f, st.hist_f)
        assert np.array_equal(I.alleles(), st.x)
        bits, bf, bg, bc = I.best()
        assert (bf, bg, bc) == tuple(int(v) for v in st.best)
