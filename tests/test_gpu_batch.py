"""GPU parity of the batched-market path (fr_batch_*): every market of a batch against its own
single-market context on the same GPU and against the FP64 oracle; autotuner choices; BF16 storage;
a sample of the batching workload's market-size distribution (|U| ~ U[100, 4000], |I| ~ U[100, 2000],
K in {5, 10, 20})."""
import numpy as np
import pytest

import oracle
from gpu_util import NSW_RTOL, X_ATOL, rel, require_gpu
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu

# Batch against single-market contexts: two FP32 paths that differ only in the order of the
# cross-CTA partial sums, each within NSW_RTOL of the FP64 oracle, so within 2 NSW_RTOL of each
# other. theta after Adam steps: Adam divides each coordinate's step by its own gradient scale, so
# the summation-order noise of coordinates with small gradients reaches theta almost undamped.
PAIR_RTOL = 2 * NSW_RTOL
THETA_ATOL = 3e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


# (U, I, K): exact 21 / 11 / 6-column kernels, padded 8 / 16 / 32 buckets, |I| == K, two markets
# sharing a bucket, 3000 items (16 rows per thread candidates), a single consumer
SIZES = [(13, 300, 20), (40, 129, 10), (7, 77, 5), (9, 50, 3), (5, 200, 12), (4, 20, 20),
         (21, 310, 20), (3, 3000, 20), (1, 64, 5), (30, 1000, 10), (6, 40, 30)]


def relevance(j, U, I):
    return synth.relevance_lowrank(U, I, seed=100 + j).astype(np.float32)


def single(U, I, K, r, **kw):
    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, **kw)
    g.set_relevance(r)
    g.set_exposure(synth.dcg_exposure(K))
    return g


def make_batch(sizes, rs, **kw):
    b = fr.FairRankBatch(sizes, **kw)
    for j, ((U, I, K), r) in enumerate(zip(sizes, rs)):
        b.set_relevance(j, r)
        b.set_exposure(j, synth.dcg_exposure(K))
    return b


def test_batch_matches_single_contexts_and_oracle():
    L, steps = 20, 11  # one captured chunk of 8 steps plus 3 direct steps
    rs = [relevance(j, U, I) for j, (U, I, K) in enumerate(SIZES)]
    b = make_batch(SIZES, rs, sinkhorn_iters=L)
    F = b.step(steps)
    assert F.shape == (steps, len(SIZES))
    for j, ((U, I, K), r) in enumerate(zip(SIZES, rs)):
        g = single(U, I, K, r, sinkhorn_iters=L)
        Fs = g.step(steps)
        np.testing.assert_allclose(F[:, j], Fs, rtol=PAIR_RTOL)
        np.testing.assert_allclose(b.policy(j), g.policy(), atol=X_ATOL)
        np.testing.assert_allclose(b.theta(j), g.get_state()[0], atol=THETA_ATOL, rtol=1e-5)
        if U * I <= 20000:
            o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=L)
            o.set_relevance(r.astype(np.float64))
            o.set_exposure(synth.dcg_exposure(K))
            Fo, _ = o.step(steps)
            np.testing.assert_allclose(F[:, j], Fo, rtol=NSW_RTOL)
            imp, util, Fj = b.impacts(j)
            oimp, outil, oF = o.impacts()
            np.testing.assert_allclose(imp, oimp, rtol=1e-6)
            assert rel(util, outil) < 1e-6 and rel(Fj, oF) < NSW_RTOL


def test_autotune_choices_and_state_preserved():
    sizes = SIZES[:6]
    rs = [relevance(j, U, I) for j, (U, I, K) in enumerate(sizes)]
    b = make_batch(sizes, rs, sinkhorn_iters=15)
    F1 = b.step(3)
    tun = b.tuning()
    assert len(tun) >= 5 and sum(t["markets"] for t in tun) == len(sizes)
    for t in tun:
        assert t["rows_per_thread"] in (8, 16, 24) and t["consumers_per_chunk"] in (4, 16)
        assert t["threads"] % 32 == 0 and t["threads"] * t["rows_per_thread"] >= t["max_items"]
    imp_before = [b.impacts(j)[0] for j in range(len(sizes))]
    b.autotune()  # retuning keeps theta and the warm start
    for j in range(len(sizes)):
        np.testing.assert_allclose(b.impacts(j)[0], imp_before[j], rtol=1e-6)
    F2 = b.step(2)
    c = make_batch(sizes, rs, sinkhorn_iters=15)
    Fc = c.step(5)
    np.testing.assert_allclose(np.vstack([F1, F2]), Fc, rtol=PAIR_RTOL)


def test_batch_bf16_matches_single_bf16():
    sizes = [(11, 500, 20), (8, 90, 5), (6, 1500, 10)]
    bits = [synth.to_bf16_bits(relevance(j, U, I)) for j, (U, I, K) in enumerate(sizes)]
    b = make_batch(sizes, bits, rel_dtype=fr.BF16, sinkhorn_iters=20)
    F = b.step(4)
    for j, ((U, I, K), r) in enumerate(zip(sizes, bits)):
        g = single(U, I, K, r, rel_dtype=fr.BF16, sinkhorn_iters=20)
        np.testing.assert_allclose(F[:, j], g.step(4), rtol=PAIR_RTOL)


def test_batching_workload_size_sample():
    """24 markets drawn from the batching workload's size distribution, 2 steps, every market
    against its single-market context; the two smallest, the median and the largest one also
    against the oracle."""
    ms = synth.markets(24, seed=3)
    sizes = [(m.n_users, m.n_items, m.n_slots) for m in ms]
    rs = [synth.relevance_lowrank_fast(m.n_users, m.n_items, seed=m.seed) for m in ms]
    b = make_batch(sizes, rs, sinkhorn_iters=50)
    F = b.step(2)
    for j, ((U, I, K), r) in enumerate(zip(sizes, rs)):
        np.testing.assert_allclose(F[:, j], single(U, I, K, r).step(2), rtol=PAIR_RTOL)
    order = np.argsort([U * I for U, I, K in sizes])
    # the two smallest, the median and the largest market
    for j in list(order[:2]) + [order[len(order) // 2], order[-1]]:
        U, I, K = sizes[j]
        o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=50)
        o.set_relevance(rs[j].astype(np.float64))
        o.set_exposure(synth.dcg_exposure(K))
        np.testing.assert_allclose(F[:, j], o.step(2)[0], rtol=NSW_RTOL)


@pytest.mark.parametrize("param,sizes", [
    # per-item markets at the batched limit (8 rows per thread, 512 threads): 4096 items
    (fr.PARAM_ITEM, [(2, 4096, 20), (2, 4096, 10), (2, 4096, 5), (2, 4096, 30)]),
    # free-cost markets at their variants' limits
    (fr.PARAM_FULL_C, [(2, 4096, 10), (2, 2048, 20), (2, 2048, 5)]),
])
def test_batch_largest_markets_match_single_contexts(param, sizes):
    L, steps = 10, 3
    rs = [relevance(40 + j, U, I) for j, (U, I, K) in enumerate(sizes)]
    b = make_batch(sizes, rs, param=param, sinkhorn_iters=L)
    F = b.step(steps)
    for j, ((U, I, K), r) in enumerate(zip(sizes, rs)):
        g = fr.FairRank(U, I, K, param=param, sinkhorn_iters=L)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        np.testing.assert_allclose(F[:, j], g.step(steps), rtol=PAIR_RTOL)
        g.close()
    b.close()
    with pytest.raises(fr.FairRankError) as ex:
        fr.FairRankBatch([(2, 4097, 20)])
    assert ex.value.status == 7


def test_batch_rejections():
    with pytest.raises(fr.FairRankError) as ex:
        fr.FairRankBatch([(3, 5000, 10)])
    assert ex.value.status == 7
    with pytest.raises(fr.FairRankError) as ex:
        fr.FairRankBatch([(3, 50, 10), (3, 50, 10)], grad_mode=fr.GRAD_UNROLLED)
    assert ex.value.status == 7
    b = fr.FairRankBatch([(3, 50, 10), (4, 60, 5)])
    with pytest.raises(fr.FairRankError) as ex:
        b.step(1)  # relevance and exposure not set
    assert ex.value.status == 6
    with pytest.raises(fr.FairRankError):
        b.set_exposure(2, synth.dcg_exposure(5))


# ---- free-cost markets (the paper's Problem (8)) -----------------------------------------------
# (U, I, K): 21-column tile sweep (two markets sharing a stride-512 bucket), 11 columns in registers
# and in the stride-1024 tile, padded 8 / 16 / 32 buckets, |I| == K, the exact 50-column kernel,
# a single consumer
SIZES_P1 = [(13, 300, 20), (21, 310, 20), (40, 129, 10), (30, 1000, 10), (7, 77, 5), (5, 200, 12),
            (4, 20, 20), (6, 40, 30), (4, 50, 49), (1, 64, 5)]


def single_p1(U, I, K, r, **kw):
    g = fr.FairRank(U, I, K, param=fr.PARAM_FULL_C, **kw)
    g.set_relevance(r)
    g.set_exposure(synth.dcg_exposure(K))
    return g


@pytest.mark.parametrize("opt", [fr.ADAM, fr.SGD])
def test_free_cost_batch_matches_single_contexts_and_oracle(opt):
    """Every free-cost market of one batch (kernel variants on concurrent launches, chunked
    consumers with their own partial rows, one graph chunk of 8 steps plus direct steps) against its
    own single-market context on the GPU and, where the oracle is quick, the FP64 oracle: F after
    every step; with SGD also the policies and impacts (Adam renormalises every cell's step by its
    own gradient scale, so the two paths' different FP32 summation orders reach the policy of
    near-stationary cells almost undamped; F is the contract there)."""
    L, steps = 20, 11
    kw = dict(sinkhorn_iters=L, optimizer=opt, lr=0.1 if opt == fr.ADAM else 0.5)
    rs = [relevance(j, U, I) for j, (U, I, K) in enumerate(SIZES_P1)]
    b = make_batch(SIZES_P1, rs, param=fr.PARAM_FULL_C, **kw)
    F = b.step(steps)
    assert F.shape == (steps, len(SIZES_P1))
    for j, ((U, I, K), r) in enumerate(zip(SIZES_P1, rs)):
        g = single_p1(U, I, K, r, **kw)
        Fs = g.step(steps)
        np.testing.assert_allclose(F[:, j], Fs, rtol=PAIR_RTOL)
        if opt == fr.SGD:
            np.testing.assert_allclose(b.policy(j), g.policy(), atol=X_ATOL)
            imp_b, _, F_b = b.impacts(j)
            imp_s, _, F_s = g.impacts()
            np.testing.assert_allclose(imp_b, imp_s, rtol=PAIR_RTOL)
        # |U| = 1: the uniform policy is optimal and the gradient is at rounding level, which Adam
        # turns into lr-sized steps in either precision, so FP32 and FP64 walk apart there
        if U * I <= 20000 and (U > 1 or opt == fr.SGD):
            o = oracle.Oracle(U, I, K, param=oracle.PARAM_FULL_C, iters=L, optimizer=opt,
                              lr=kw["lr"])
            o.set_relevance(r.astype(np.float64))
            o.set_exposure(synth.dcg_exposure(K))
            Fo, _ = o.step(steps)
            np.testing.assert_allclose(F[:, j], Fo, rtol=NSW_RTOL)
            if opt == fr.SGD:
                np.testing.assert_allclose(b.policy(j), o.policy(), atol=X_ATOL)
        g.close()
    with pytest.raises(fr.FairRankError):
        b.theta(0)
    b.close()


def test_free_cost_batch_autotune_and_reset():
    sizes = [(60, 300, 10), (45, 900, 10), (30, 200, 20)]
    rs = [relevance(10 + j, U, I) for j, (U, I, K) in enumerate(sizes)]
    b = make_batch(sizes, rs, param=fr.PARAM_FULL_C, sinkhorn_iters=15)
    b.autotune()
    for row in b.tuning():
        assert row["consumers_per_chunk"] in (4, 16)
    F1 = b.step(9)
    b.reset()
    F2 = b.step(9)
    np.testing.assert_array_equal(F1, F2)  # deterministic, and reset restores C = 0
    b.close()
