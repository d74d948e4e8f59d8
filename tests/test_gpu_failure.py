"""Failure detection on the GPU without faulting it.

Every device-side wait of the library is bounded (the kernels' waits for their staged bulk copies
and the envy contraction's waits for its tensor-core work). Here the bound is forced to zero polls
(fr_config.max_wait_polls = -1, a wait that nothing can satisfy in time): each kernel must report
FR_ETIMEOUT through its status word, drain its own copies in flight and stop, and the context must
stay usable -- after restoring the default bound and resetting the optimiser state, the same steps
reproduce a fresh context's results exactly. FR_ENUMERIC is exercised with a relevance value that
leaves an item's impact below the FP32 range (the FP64 oracle's impact stays positive).
"""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu
ETIMEOUT, ENUMERIC = 5, 4


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def make(U, I, K, seed=3, **kw):
    g = fr.FairRank(U, I, K, **kw)
    g.set_relevance(synth.relevance_lowrank(U, I, seed=seed).astype(np.float32))
    g.set_exposure(synth.dcg_exposure(K))
    return g


def expect_status(status, fn, *args):
    with pytest.raises(fr.FairRankError) as ei:
        fn(*args)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


@pytest.mark.parametrize("U,I,K", [
    (64, 300, 10),    # free costs, register sweep (tile staged one consumer ahead)
    (64, 1000, 10),   # free costs, 11-column tile sweep (late wait in the update mode)
    (40, 900, 20),    # free costs, 21-column tile sweep
])
def test_free_cost_wait_expiry_reports_timeout_and_context_recovers(torch, U, I, K):
    ref = make(U, I, K).step(3)
    g = make(U, I, K, max_wait_polls=-1)
    msg = expect_status(ETIMEOUT, g.step, 2)  # the first solve's tile wait
    assert "wait" in msg
    g.set_wait_limit(0)
    g.reset()
    np.testing.assert_array_equal(g.step(3), ref)
    # the fused gradient + Sinkhorn kernel's wait (after a healthy first solve)
    g.reset()
    g.step(1)
    g.set_wait_limit(-1)
    expect_status(ETIMEOUT, g.step, 1)
    g.set_wait_limit(0)
    g.reset()
    np.testing.assert_array_equal(g.step(3), ref)
    g.close()


@pytest.mark.parametrize("grad_mode", [fr.GRAD_IMPLICIT, fr.GRAD_UNROLLED])
def test_per_item_wait_expiry_in_sweep_and_gradient_kernels(torch, grad_mode):
    U, I, K = 48, 500, 10
    kw = dict(param=fr.PARAM_ITEM, grad_mode=grad_mode, sinkhorn_iters=20)
    ref = make(U, I, K, **kw).step(2)
    g = make(U, I, K, max_wait_polls=-1, **kw)
    expect_status(ETIMEOUT, g.impacts)  # the Sinkhorn kernel's relevance-row wait
    g.set_wait_limit(0)
    g.reset()
    g.impacts()
    g.set_wait_limit(-1)
    expect_status(ETIMEOUT, g.grad)  # the gradient (implicit or adjoint) kernel's wait
    g.set_wait_limit(0)
    g.reset()
    np.testing.assert_array_equal(g.step(2), ref)
    g.close()


def test_envy_contraction_wait_expiry(torch):
    U, I, K = 200, 300, 10
    g = make(U, I, K)
    g.step(2)
    ok = g.metrics()
    g.set_wait_limit(-1)
    msg = expect_status(ETIMEOUT, g.metrics)  # the tensor-core commit waits
    assert "envy" in msg
    g.set_wait_limit(0)
    again = g.metrics()
    assert again == ok
    g.close()


def test_batched_markets_wait_expiry(torch):
    sizes = [(120, 200, 5), (90, 150, 10), (60, 300, 20)]
    b = fr.FairRankBatch(sizes, max_wait_polls=-1, sinkhorn_iters=10)
    for j, (U, I, K) in enumerate(sizes):
        b.set_relevance(j, synth.relevance_lowrank(U, I, seed=j).astype(np.float32))
        b.set_exposure(j, synth.dcg_exposure(K))
    expect_status(ETIMEOUT, b.step, 1)
    b.close()


def test_wait_limit_argument_checks(torch):
    g = make(8, 20, 5)
    expect_status(1, g.set_wait_limit, -2)
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(8, 20, 5, max_wait_polls=-3)
    assert ei.value.status == 1
    g.close()


@pytest.mark.parametrize("param", [fr.PARAM_FULL_C, fr.PARAM_ITEM])
def test_impact_below_fp32_range_reports_numeric_error(torch, param):
    """Item 5's only positive relevance is the smallest FP32 subnormal: its impact, r times an
    exposure-weighted probability below one half, rounds to zero in FP32, so F = sum log Imp is not
    finite and the library reports FR_ENUMERIC. In FP64 the same impact is positive."""
    U, I, K = 16, 40, 5
    r = synth.relevance_uniform(U, I, 4).astype(np.float32) + np.float32(0.05)
    r[:, 5] = 0.0
    r[3, 5] = np.float32(1e-45)
    assert r[3, 5] > 0
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, param=param)
    g.set_relevance(r)
    g.set_exposure(e)
    msg = expect_status(ENUMERIC, g.impacts)
    assert "impact" in msg
    o = oracle.Oracle(U, I, K, param=param)
    o.set_relevance(r.astype(np.float64))
    o.set_exposure(e)
    imp, _, F = o.impacts()
    assert imp[5] > 0 and np.isfinite(F)
    g.close()


def test_allocation_failure_reports_enomem_and_frees_what_it_took(torch):
    """A context larger than the GPU (free costs for 3 million consumers x 1024 items x 21 columns:
    C and each Adam moment 258 GB) fails with FR_ENOMEM instead of faulting, gives back every block
    it had allocated, and the device stays usable for the next context."""
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    msg = expect_status(2, fr.FairRank, 3_000_000, 1024, 20)  # FR_ENOMEM
    assert "cudaMalloc" in msg or "memory" in msg
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    g = make(8, 100, 10)
    F = g.step(2)
    assert np.isfinite(F).all()
    g.close()
