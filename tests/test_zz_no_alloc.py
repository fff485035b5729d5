"""qieo_generation_noalloc: a generation for callers that cannot allocate device memory.

The entry point takes the caller's device buffers and keeps its own working memory in a
fixed device array, so it never calls cudaMalloc. These tests call it through the C ABI
on device buffers made by the test, several times in a row, and compare every output with
what the allocating instance API produces for the same generations, and, in one case,
directly with the CPU oracle. All results are exact integers, so the tolerance is zero.
"""
import numpy as np
import pytest

from paper_2609_30862_gb300 import qieo as Q
from paper_2609_30862_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Q.load()
    return torch


def _params(np_, seed, inst, rule, D=100, lam=1, stream=None):
    p = Q.qieo_default_params()
    p.np, p.seed, p.instance_id, p.rotate_rule = np_, seed, inst, rule
    p.dtheta_den, p.penalty_lambda = D, lam
    p.stream = stream
    return p


@pytest.mark.parametrize("ng,np_,rule,D,lam,gens", [(1000, 48, 0, 100, 1, 2), (333, 17, 1, 12, 3, 2),
                                                    (7, 5, 0, 4, 1, 2), (64, 1000, 0, 4, 1, 6),
                                                    (40, 700, 1, 4, 1, 6)])
def test_noalloc_matches_instance_two_calls(torch_cuda, ng, np_, rule, D, lam, gens):
    """Consecutive calls against the instance path. The populations of 700 and 1,000
    chromosomes make each thread of the last block's argmax stride over several
    chromosomes, and D = 4 (K = 1) saturates the angles within the first generations, so
    that many chromosomes tie on fitness and the lowest-index rule decides."""
    torch = torch_cuda
    prob = W.knapsack(ng, ng + np_)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d_w = torch.from_numpy(prob.weights).to(dev)
    d_v = torch.from_numpy(prob.values).to(dev)
    d_k = torch.zeros((np_, ng), dtype=torch.int16, device=dev)
    d_x = torch.zeros((np_, ng), dtype=torch.uint8, device=dev)
    d_f = torch.zeros(np_, dtype=torch.int64, device=dev)
    d_e = torch.full((1,), -1, dtype=torch.int32, device=dev)
    params = _params(np_, 5, 9, rule, D, lam, stream.cuda_stream)
    with Q.Instance(prob, np_, seed=5, inst=9, D=D, lam=lam, rule=rule,
                    stream=stream.cuda_stream) as inst:
        for t in range(gens):
            Q.qieo_generation_noalloc(d_w.data_ptr(), d_v.data_ptr(), ng, prob.capacity, params, t,
                                      d_k.data_ptr(), d_x.data_ptr(), d_f.data_ptr(),
                                      d_e.data_ptr())
            inst.run(1)
            torch.cuda.synchronize()
            k_ref, t_ref = inst.state()
            e_ref, _ = inst.history(t, 1)
            assert t_ref == t + 1
            assert np.array_equal(d_k.cpu().numpy(), k_ref), "angle indices differ"
            assert np.array_equal(d_x.cpu().numpy(), inst.alleles()), "alleles differ"
            assert np.array_equal(d_f.cpu().numpy(), inst.fitness()), "fitness differs"
            assert int(d_e.cpu()[0]) == int(e_ref[0]), "elite differs"


def test_noalloc_rejects_population_beyond_static_array(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    d = torch.zeros(16, dtype=torch.int32, device=dev)
    params = _params(Q.QIEO_NOALLOC_MAX_NP + 1, 1, 0, 0)
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_generation_noalloc(d.data_ptr(), d.data_ptr(), 8, 10, params, 0, d.data_ptr(),
                                  d.data_ptr(), d.data_ptr(), d.data_ptr())
    assert e.value.status == Q.QIEO_ERR_INVALID
    assert str(Q.QIEO_NOALLOC_MAX_NP) in str(e.value)


def _buffers(torch, prob, np_, k0=None):
    dev = torch.device("cuda", 0)
    ng = prob.weights.shape[0]
    d_w = torch.from_numpy(prob.weights).to(dev)
    d_v = torch.from_numpy(prob.values).to(dev)
    d_k = (torch.from_numpy(k0).to(dev) if k0 is not None
           else torch.zeros((np_, ng), dtype=torch.int16, device=dev))
    d_x = torch.zeros((np_, ng), dtype=torch.uint8, device=dev)
    d_f = torch.zeros(np_, dtype=torch.int64, device=dev)
    d_e = torch.full((1,), -1, dtype=torch.int32, device=dev)
    return d_w, d_v, d_k, d_x, d_f, d_e


def test_noalloc_matches_oracle_directly(torch_cuda):
    """Five consecutive calls against the CPU oracle, generation by generation: angle
    indices after the rotation, alleles, fitness and the elite."""
    from oracle import oracle as O
    torch = torch_cuda
    prob = W.knapsack(500, 31)
    np_, rule = 90, 0
    d_w, d_v, d_k, d_x, d_f, d_e = _buffers(torch, prob, np_)
    stream = torch.cuda.current_stream()
    params = _params(np_, 3, 4, rule, 100, 1, stream.cuda_stream)
    st = None
    for t in range(5):
        Q.qieo_generation_noalloc(d_w.data_ptr(), d_v.data_ptr(), 500, prob.capacity, params, t,
                                  d_k.data_ptr(), d_x.data_ptr(), d_f.data_ptr(), d_e.data_ptr())
        st = O.run(prob, np_, 1, seed=3, inst=4, rule=rule, state=st)
        torch.cuda.synchronize()
        assert np.array_equal(d_k.cpu().numpy(), st.k), t
        assert np.array_equal(d_x.cpu().numpy(), st.x), t
        assert np.array_equal(d_f.cpu().numpy(), st.f), t
        assert int(d_e.cpu()[0]) == int(st.hist_e[-1]), t


def test_noalloc_out_of_range_angles(torch_cuda):
    """Angle indices outside [-K, K] (invalid input) are observed as the nearest bound, and
    a rotation step is taken only where it lands inside [-K, K]: the outputs equal those of
    the same call on the clamped indices, except that the out-of-range indices themselves
    stay where they are unless their step brings them back into range."""
    torch = torch_cuda
    K = 25
    prob = W.knapsack(96, 8)
    np_ = 40
    rng = np.random.default_rng(5)
    k_bad = rng.integers(-K, K + 1, size=(np_, 96)).astype(np.int16)
    k_bad[::3, ::5] = K + 3
    k_bad[1::3, 2::7] = -K - 4
    k_bad[2, 1] = K + 1
    k_clamped = np.clip(k_bad, -K, K).astype(np.int16)
    stream = torch.cuda.current_stream()
    params = _params(np_, 9, 1, 0, 100, 1, stream.cuda_stream)
    outs = []
    for k0 in (k_bad, k_clamped):
        d_w, d_v, d_k, d_x, d_f, d_e = _buffers(torch, prob, np_, k0)
        Q.qieo_generation_noalloc(d_w.data_ptr(), d_v.data_ptr(), 96, prob.capacity, params, 0,
                                  d_k.data_ptr(), d_x.data_ptr(), d_f.data_ptr(), d_e.data_ptr())
        torch.cuda.synchronize()
        outs.append((d_k.cpu().numpy(), d_x.cpu().numpy(), d_f.cpu().numpy(), int(d_e.cpu()[0])))
    (kb, xb, fb, eb), (kc, xc, fc, ec) = outs
    assert np.array_equal(xb, xc) and np.array_equal(fb, fc) and eb == ec
    inside = (k_bad >= -K) & (k_bad <= K)
    assert np.array_equal(kb[inside], kc[inside])
    step = np.where(xc[ec] == 1, 1, -1)[None, :].repeat(np_, axis=0)
    moved = k_bad + step
    expect = np.where((moved >= -K) & (moved <= K), moved, k_bad)
    assert np.array_equal(kb[~inside], expect[~inside])
    assert kb[2, 1] in (K, K + 1)
