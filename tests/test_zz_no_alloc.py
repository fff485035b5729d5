"""qieo_generation_noalloc: a generation for callers that cannot allocate device memory.

The entry point takes the caller's device buffers and keeps its own working memory in a
fixed device array, so it never calls cudaMalloc. These tests call it through the C ABI
on device buffers made by the test, twice in a row (generations 0 and 1), and compare
every output with what the allocating instance API produces for the same generations.
All results are exact integers, so the tolerance is zero.
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


@pytest.mark.parametrize("ng,np_,rule,D,lam", [(1000, 48, 0, 100, 1), (333, 17, 1, 12, 3),
                                               (7, 5, 0, 4, 1)])
def test_noalloc_matches_instance_two_calls(torch_cuda, ng, np_, rule, D, lam):
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
        for t in range(2):
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
