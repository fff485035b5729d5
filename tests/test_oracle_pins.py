"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test ties one part of the oracle to the paper or to mathematics that the oracle's
code does not share: an independent Philox implementation, a 60-digit evaluation of the
threshold table, a dynamic-programming knapsack optimum and the closed-form cases of
eq. (1), binomial frequencies of the observation, the amplitude (rotation-matrix) form of
the loop against the angle-index form, and the loop's fixed points at the bounds (qubits at
theta = 0 or pi/2 on the elite's side).
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2609_30862_gb300 import workload as W


# --------------------------------------------------------------------------- Philox

_TORCH_PHILOX_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
    uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen/core/PhiloxRNGEngine.h")) else None


def test_philox_matches_pytorch_header(oracle_mod):
    """Philox4x32-10 (Salmon et al. 2011) against PyTorch's own engine, which keys with
    the 64-bit seed and counts (offset, subsequence) in the same four words."""
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("PyTorch headers or g++ unavailable")
    rng = np.random.default_rng(2609)
    cases = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64)
    cases[0] = 0
    cases[1] = 2**32 - 1
    cases[2, :4] = [5, 17, 3, 0]          # the shape of a QIEO counter: (j/4, c, t, 0)
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        with open(src, "w") as fh:
            fh.write(_TORCH_PHILOX_PROG)
        try:
            subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", inc,
                                   "-I", os.path.join(inc, "torch/csrc/api/include"),
                                   src, "-o", exe], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            pytest.skip("PyTorch Philox header does not compile standalone here")
        inp = "\n".join(" ".join(str(int(x)) for x in row) for row in cases) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()],
                   dtype=np.uint64)
    for row, want in zip(cases, ref):
        got = oracle_mod.philox4x32_10(row[:4], row[4:])
        assert [int(x) for x in got] == [int(x) for x in want], row


def read_philox_kat():
    """The published Philox4x32-10 known-answer vectors (tests/golden)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    """The three known-answer vectors published with Philox4x32-10."""
    rows = read_philox_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert [int(x) for x in oracle_mod.philox4x32_10(ctr, key)] == want


def test_philox_uniform_bytes(oracle_mod):
    """Chi-square on the bytes of 16k Philox words: no bias at the 1e-6 level."""
    out = np.concatenate([oracle_mod.philox4x32_10([i, 7, 3, 0], [1, 0]) for i in range(4096)])
    counts = np.bincount(out.view(np.uint8), minlength=256)
    exp = counts.sum() / 256.0
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 255 degrees of freedom: mean 255, sd ~22.6; 6 sd band.
    assert 255 - 6 * 22.6 < chi2 < 255 + 6 * 22.6


# --------------------------------------------------------------------------- table

@pytest.mark.parametrize("D", [4, 8, 12, 20, 100, 200, 1000, 4000])
def test_threshold_table_exact(oracle_mod, D):
    """T[n] = round(sin^2(n pi / D) 2^32) exactly (60-digit evaluation), with the
    closed-form end points T[0] = 0, T[K] = 2^31, T[2K] = 2^32 and symmetry."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    T = oracle_mod.threshold_table(D)
    K = D // 4
    assert T.shape == (2 * K + 1,)
    assert int(T[0]) == 0 and int(T[K]) == 2**31 and int(T[2 * K]) == 2**32
    for n in range(2 * K + 1):
        exact = mp.sin(n * mp.pi / D) ** 2 * 2**32
        want = int(mp.floor(exact + mp.mpf(1) / 2))
        assert abs(exact - mp.floor(exact) - mp.mpf(1) / 2) > mp.mpf(10) ** -20
        assert int(T[n]) == want, (D, n)
        assert int(T[n]) + int(T[2 * K - n]) == 2**32
    assert np.all(np.diff(T.astype(np.int64)) > 0)


def test_table_rejects_bad_D(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.threshold_table(10)


# --------------------------------------------------------------------------- eq. (1)

def _dp_knapsack(w, v, W_):
    """Textbook 0/1 knapsack dynamic program over capacity (max value, weight <= W)."""
    best = np.zeros(W_ + 1, dtype=np.int64)
    for wi, vi in zip(w, v):
        if wi <= W_:
            best[wi:] = np.maximum(best[wi:], best[:W_ + 1 - wi] + vi)
    return int(best[W_])


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_equals_dp_optimum(oracle_mod, seed):
    """Maximum of eq. (1) over all subsets = the DP optimum: every feasible subset has
    f >= 0 and every infeasible one f < 0, so the maximiser is a feasible optimum."""
    rng = np.random.default_rng(seed)
    ng = int(rng.integers(1, 17))
    w = rng.integers(1, 30, ng).astype(np.int32)
    v = rng.integers(0, 40, ng).astype(np.int32)
    cap = int(rng.integers(0, w.sum() + 1))
    best, x = oracle_mod.bruteforce(w, v, cap, 3)
    assert best == _dp_knapsack(w, v, cap)
    assert int((w.astype(np.int64) * x).sum()) <= cap


def test_fitness_closed_forms(oracle_mod):
    w = np.array([4, 7, 1, 9], dtype=np.int32)
    v = np.array([10, 3, 8, 20], dtype=np.int32)
    cap = 11
    assert oracle_mod.fitness([0, 0, 0, 0], w, v, cap) == 0                  # empty pack
    assert oracle_mod.fitness([1, 1, 0, 0], w, v, cap) == 13                 # sum w = 11 = W: feasible
    assert oracle_mod.fitness([1, 1, 1, 0], w, v, cap, 1) == -1              # sum w = 12 > W
    assert oracle_mod.fitness([1, 1, 1, 1], w, v, cap, 1) == -(21 - 11)
    assert oracle_mod.fitness([1, 1, 1, 1], w, v, cap, 5) == -5 * (21 - 11)  # linear in lambda
    for j in range(4):
        e = np.zeros(4, dtype=np.uint8)
        e[j] = 1
        want = int(v[j]) if w[j] <= cap else -(int(w[j]) - cap)
        assert oracle_mod.fitness(e, w, v, cap) == want


def test_determine_elite_lowest_index(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = rng.integers(-3, 3, int(rng.integers(1, 40))).astype(np.int64)
        assert oracle_mod.determine_elite(f) == int(np.argmax(f))   # argmax: first maximum


# --------------------------------------------------------------------------- observation

@pytest.mark.parametrize("n", [0, 1, 7, 13, 25, 37, 49, 50])
def test_observation_frequency(oracle_mod, n):
    """With every qubit at angle index n, P(x = 1) = sin^2(n pi / D) (5 sigma band);
    the end points are deterministic."""
    D, K = 100, 25
    prob = W.knapsack(500, 4)
    st = oracle_mod.State(200, 500)
    st.k[:] = n - K
    st = oracle_mod.run(prob, 200, 1, seed=9, state=st)
    p = math.sin(n * math.pi / D) ** 2
    m = st.x.size
    mean = st.x.mean()
    if n in (0, 2 * K):
        assert mean == (1.0 if n == 2 * K else 0.0)
    else:
        assert abs(mean - p) < 5 * math.sqrt(p * (1 - p) / m)


# --------------------------------------------------------------------------- loop

def _amplitude_angle_index(alpha, beta, D):
    theta = np.arctan2(beta, alpha)
    k = (theta - math.pi / 4) / (math.pi / D)
    return np.rint(k).astype(np.int64), np.abs(k - np.rint(k)) * (math.pi / D)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("D,ng,np_,gens,seed", [(100, 60, 24, 150, 1), (12, 30, 16, 80, 2),
                                                (4, 20, 8, 40, 3), (100, 100, 64, 60, 5)])
def test_angle_index_form_equals_amplitude_form(oracle_mod, rule, D, ng, np_, gens, seed):
    """The integer angle-index loop and the rotation-matrix loop in (alpha, beta) give the
    same alleles, fitness, elites and best record; the angle index tracks
    atan2(beta, alpha) and the amplitudes stay normalised."""
    prob = W.knapsack(ng, seed)
    a = oracle_mod.run(prob, np_, gens, seed=seed, inst=7, D=D, rule=rule)
    b = oracle_mod.run_fp64(prob, np_, gens, seed=seed, inst=7, D=D, rule=rule)
    assert b["near_ties"] == 0
    assert np.array_equal(a.x, b["x"]) and np.array_equal(a.f, b["f"])
    assert np.array_equal(a.hist_e, b["hist_e"]) and np.array_equal(a.hist_f, b["hist_f"])
    assert np.array_equal(a.best, b["best"]) and np.array_equal(a.best_x, b["best_x"])
    k, err = _amplitude_angle_index(b["alpha"], b["beta"], D)
    assert np.array_equal(k, a.k.astype(np.int64))
    assert err.max() < 1e-12 * (gens + 1)
    assert b["max_norm_err"] < 1e-12
    assert a.k.min() >= -(D // 4) and a.k.max() <= D // 4


def test_elite_and_best_record(oracle_mod):
    prob = W.knapsack(80, 11)
    st = oracle_mod.run(prob, 32, 120, seed=11)
    # the best-so-far is the first generation elite of maximal fitness
    g = int(np.argmax(st.hist_f))
    assert st.best[0] == st.hist_f.max() and st.best[1] == g
    assert st.best[2] == st.hist_e[g]
    assert oracle_mod.fitness(st.best_x, prob.weights, prob.values, prob.capacity) == st.best[0]
    # the last generation's elite is the lowest-index maximum of its fitness array
    assert st.hist_e[-1] == int(np.argmax(st.f)) and st.hist_f[-1] == st.f.max()
    # fitness of every chromosome of the last generation agrees with eq. (1)
    for c in range(32):
        assert st.f[c] == oracle_mod.fitness(st.x[c], prob.weights, prob.values, prob.capacity)


def test_ties_pick_lowest_index(oracle_mod):
    """With two items there are at most four distinct strings, so many chromosomes tie
    for the maximum in every generation; the elite must be the first of them."""
    prob = W.custom_problem([3, 4], [5, 6], 5)
    st = oracle_mod.State(16, 2)
    for _ in range(30):
        st = oracle_mod.run(prob, 16, 1, seed=5, state=st)
        assert st.hist_e[-1] == int(np.argmax(st.f))
        assert (st.f == st.f.max()).sum() >= 1


def test_split_runs_equal_one_run(oracle_mod):
    """run(a) then run(b) equals run(a + b): the random stream is keyed by the absolute
    generation and the last CIP of a run is not repeated."""
    prob = W.knapsack(70, 2)
    one = oracle_mod.run(prob, 20, 90, seed=3, rule=1)
    two = oracle_mod.run(prob, 20, 35, seed=3, rule=1)
    two = oracle_mod.run(prob, 20, 55, seed=3, rule=1, state=two)
    for name in ("k", "t", "best", "best_x", "x", "f", "hist_e", "hist_f"):
        assert np.array_equal(getattr(one, name), getattr(two, name)), name


def test_best_bounded_by_optimum(oracle_mod):
    """QIEO is a heuristic: its best is never above the exact optimum (reaching it is
    reported, not required)."""
    for seed in range(4):
        prob = W.knapsack(18, 40 + seed)
        opt, _ = oracle_mod.bruteforce(prob.weights, prob.values, prob.capacity)
        st = oracle_mod.run(prob, 32, 200, seed=seed)
        assert st.best[0] <= opt
        assert st.best[0] >= 0


def test_openmp_build_identical(oracle_mod):
    prob = W.knapsack(300, 6)
    a = oracle_mod.run(prob, 96, 40, seed=2)
    b = oracle_mod.run(prob, 96, 40, seed=2, kind="omp", threads=4)
    for name in ("k", "t", "best", "best_x", "x", "f", "hist_e", "hist_f"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name


def test_rejects_invalid(oracle_mod):
    prob = W.knapsack(10, 1)
    with pytest.raises(ValueError):
        oracle_mod.run(prob, 4, 1, D=30)
    with pytest.raises(ValueError):
        oracle_mod.run(prob, 4, 1, lam=0)
    with pytest.raises(ValueError):
        oracle_mod.run(prob, 0, 1)


def _first_converged(hist_f, window):
    """First generation t whose last `window` elite fitness values (t-window+1 .. t) are all
    equal, found from the history of a run without the stop (the definition itself)."""
    for t in range(window - 1, len(hist_f)):
        if np.all(hist_f[t - window + 1:t + 1] == hist_f[t]):
            return t
    return None


@pytest.mark.parametrize("ng,np_,seed,rule", [(200, 30, 3, 0), (120, 17, 8, 0), (60, 5, 2, 0)])
def test_convergence_stop_matches_its_definition(oracle_mod, ng, np_, seed, rule):
    """Sec. IV: stop once the elite fitness has been stable for 20 generations. The
    stopping generation equals the first one that the definition picks out of an
    unstopped run's history, the stopped state equals that run cut after it (its CIP
    included), split runs stop at the same place, and a stopped instance stays put."""
    O = oracle_mod
    prob = W.knapsack(ng, seed)
    full = O.run(prob, np_, 400, seed=seed, rule=rule)
    tc = _first_converged(full.hist_f, 20)
    assert tc is not None
    stopped = O.run(prob, np_, 400, seed=seed, rule=rule, window=20)
    assert int(stopped.t[0]) == tc + 1 and stopped.stopped
    cut = O.run(prob, np_, tc + 1, seed=seed, rule=rule)
    assert np.array_equal(stopped.k, cut.k)
    assert np.array_equal(stopped.hist_e, cut.hist_e) and np.array_equal(stopped.hist_f, cut.hist_f)
    assert np.array_equal(stopped.best, cut.best)
    split = O.State(np_, ng)
    for g in (7, 13, 50, 400):
        split = O.run(prob, np_, g, seed=seed, rule=rule, state=split, window=20)
    assert int(split.t[0]) == tc + 1 and np.array_equal(split.k, stopped.k)
    again = O.run(prob, np_, 10, seed=seed, rule=rule, state=stopped.copy(), window=20)
    assert int(again.t[0]) == tc + 1 and np.array_equal(again.k, stopped.k)


def test_convergence_window_one_and_cap(oracle_mod):
    """Window 1 stops after the first generation; a cap below the stopping generation runs
    exactly the cap; rule R2 keeps the population diverse, and where the definition finds
    no stable window the run goes to its cap."""
    O = oracle_mod
    prob = W.knapsack(100, 4)
    one = O.run(prob, 12, 50, seed=4, window=1)
    assert int(one.t[0]) == 1
    capped = O.run(prob, 12, 5, seed=4, window=20)
    assert int(capped.t[0]) == 5 and not capped.stopped
    prob = W.knapsack(120, 8)
    full = O.run(prob, 17, 150, seed=8, rule=1)
    assert _first_converged(full.hist_f, 20) is None
    r2 = O.run(prob, 17, 150, seed=8, rule=1, window=20)
    assert int(r2.t[0]) == 150 and not r2.stopped and np.array_equal(r2.k, full.k)


@pytest.mark.parametrize("rule,D,start", [(0, 100, "fresh"), (0, 12, "fresh"), (1, 100, "saturated"),
                                          (0, 100, "saturated")])
def test_qubits_at_a_bound_on_the_elite_side_stay_put(oracle_mod, rule, D, start):
    """What lets a generation skip most of its work once the population has collapsed: a
    qubit at theta = 0 or pi/2 (angle index -K or K) observes its side whatever the draw
    (T[0] = 0, T[2K] = 2^32), and CIP leaves it when that side is the elite's allele (R1
    rotates toward the elite's allele and it already sits at that bound; R2 rotates only the
    qubits whose allele differs from the elite's). So an 8-gene vector whose qubits all sit at
    the bound on the side of generation t's elite keeps its angle indices through CIP(t), and
    generation t + 1 observes exactly the elite's alleles there. Checked vector by vector on
    every generation of runs from the initial state (R1 collapses them) and from saturated
    states (rows sharing one pattern but for a few; R2 keeps a fresh population spread), with
    the checked vectors a majority by the end."""
    from saturated import saturated_start
    O = oracle_mod
    ng, np_, seed, G = 2400, 48, 40 + rule + D, (150 if start == "fresh" else 40)
    K, nv = D // 4, ng // 8
    prob = W.knapsack(ng, seed)
    st = O.State(np_, ng)
    if start == "saturated":
        st.k[:] = saturated_start(ng, np_, seed, n_odd=6, flips=30, D=D)
    checked, last_frac = 0, 0.0
    for t in range(G - 1):
        k_obs = st.k.copy()                              # observed by generation t
        O.run(prob, np_, 1, seed=seed, rule=rule, D=D, state=st)   # generation t and CIP(t)
        xe = st.x[int(st.hist_e[-1])].astype(np.int16).reshape(nv, 8)
        at = (np.abs(k_obs.astype(np.int32)) == K).reshape(np_, nv, 8)
        side = (k_obs > 0).astype(np.int16).reshape(np_, nv, 8)
        stable = (at & (side == xe[None])).all(axis=2)    # [np_, nv]
        k_next = st.k.reshape(np_, nv, 8)
        assert np.array_equal(k_next[stable], k_obs.reshape(np_, nv, 8)[stable]), t
        nxt = O.run(prob, np_, 1, seed=seed, rule=rule, D=D, state=st.copy())   # generation t + 1
        x_next = nxt.x.reshape(np_, nv, 8)
        want = np.broadcast_to(xe[None], (np_, nv, 8)).astype(np.uint8)
        assert np.array_equal(x_next[stable], want[stable]), t
        checked += int(stable.sum())
        last_frac = float(stable.mean())
    assert last_frac > 0.5 and checked > 0
