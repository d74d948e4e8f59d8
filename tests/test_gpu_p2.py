"""GPU parity of the per-item parametrisation c_uik = -r(u,i) e_k exp(theta_i) against the FP64
oracle, through the C-ABI: FP32 and BF16 relevance (the oracle gets the same BF16-rounded values),
exact and padded column counts, 8 / 16 / 20 / 24 rows per thread."""
import numpy as np
import pytest

import oracle
from gpu_util import NSW_RTOL, X_ATOL, rel, require_gpu
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def pair_item(U, I, K, r, bf16=False, **kw):
    e = synth.dcg_exposure(K)
    if bf16:
        bits = synth.to_bf16_bits(np.asarray(r, dtype=np.float32))
        r_gpu, r_or = bits, synth.bf16_bits_to_f64(bits)
    else:
        r_gpu = np.ascontiguousarray(r, dtype=np.float32)
        r_or = r_gpu.astype(np.float64)
    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, rel_dtype=fr.BF16 if bf16 else fr.F32, **kw)
    g.set_relevance(r_gpu)
    g.set_exposure(e)
    okw = {k: v for k, v in kw.items() if k in ("epsilon", "warm_start", "optimizer", "lr")}
    if "sinkhorn_iters" in kw:
        okw["iters"] = kw["sinkhorn_iters"]
    o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, **okw)
    o.set_relevance(r_or)
    o.set_exposure(e)
    return g, o


def seeded(U, I, K, seed):
    m = oracle.num_cols(I, K)
    th = synth.random_state(I, seed, 0.4).astype(np.float32)
    m1 = synth.random_state(I, seed, 0.01, 1).astype(np.float32)
    m2 = np.abs(synth.random_state(I, seed, 1e-4, 2)).astype(np.float32)
    gg = synth.random_state(U * m, seed, 0.5, 3).reshape(U, m).astype(np.float32)
    return th, m1, m2, gg


@pytest.mark.parametrize("U,I,K,L,bf16", [
    (9, 300, 20, 50, False),    # 21 columns, 8 rows/thread
    (5, 2000, 20, 30, True),    # 21 columns, 16 rows/thread, BF16 relevance
    (3, 9000, 20, 20, False),   # 21 columns, 20 rows/thread
    (2, 10500, 20, 15, False),  # 21 columns, 24 rows/thread
    (7, 129, 10, 40, False),    # 11 columns, ragged
    (6, 77, 5, 50, True),       # 6 columns
    (4, 50, 3, 30, False),      # generic 8-column bucket
    (4, 200, 12, 30, False),    # generic 16-column bucket
    (3, 20, 20, 25, False),     # |I| == K: no dummy column, generic 32-column bucket
    (1, 60, 5, 40, False),      # one consumer
    (4, 40, 1, 30, False),      # one slot: two columns
])
def test_item_param_one_step_from_seeded_state(U, I, K, L, bf16):
    r = synth.relevance_lowrank(U, I, seed=I + K)
    g, o = pair_item(U, I, K, r, bf16=bf16, sinkhorn_iters=L)
    th, m1, m2, gg = seeded(U, I, K, seed=I)
    g.set_state(th, m1, m2, gg, t=2)
    o.set_state(th.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                gg.astype(np.float64), 2)
    imp, _, F = g.impacts()
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    dth, dr = g.grad(want_dr=True)
    oth, odr = o.grad(want_dr=True)
    assert np.linalg.norm(dth - oth) <= 1e-5 * np.linalg.norm(oth)
    assert np.linalg.norm(dr - odr) <= 1e-5 * np.linalg.norm(odr)
    Fg = g.step(1)
    Fo, _ = o.step(1)
    assert rel(Fg[0], Fo[0]) < NSW_RTOL
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    pg, _, _, _, tg = g.get_state()
    po, _, _, _, to = o.get_state()
    assert tg == to == 3
    np.testing.assert_allclose(pg, po, atol=2e-6, rtol=1e-5)


# The largest shape of each per-item variant: 24 rows per thread and 512 threads give 12288 items
# for 6, 11 and 21 columns with BF16 relevance; with FP32 relevance the gradient kernel's shared
# arrays (20 bytes per item) fill the 227 KB first; the generic buckets take 8 rows per thread.
@pytest.mark.parametrize("I,K,bf16", [
    (12288, 20, True), (12288, 10, True), (12288, 5, True),
    (11088, 20, False), (11352, 10, False), (11400, 5, False),
    (4096, 3, False), (4096, 30, False),
])
def test_largest_shape_of_each_per_item_variant(I, K, bf16):
    U, L = 2, 10
    r = synth.relevance_lowrank_fast(U, I, seed=I + K)
    g, o = pair_item(U, I, K, r, bf16=bf16, sinkhorn_iters=L)
    th = synth.random_state(I, I, 0.4).astype(np.float32)
    g.set_state(param=th)
    o.set_state(param=th.astype(np.float64))
    imp, _, F = g.impacts()
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    dth = g.grad()
    oth = o.grad()
    assert np.linalg.norm(dth - oth) <= 1e-5 * np.linalg.norm(oth)
    Fg = g.step(1)
    Fo, _ = o.step(1)
    assert rel(Fg[0], Fo[0]) < NSW_RTOL
    g.close()


@pytest.mark.parametrize("I,K,bf16", [(12289, 20, True), (11096, 20, False), (11360, 10, False),
                                      (11408, 5, False), (4097, 3, False)])
def test_per_item_shapes_past_the_limits_are_rejected(I, K, bf16):
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(2, I, K, param=fr.PARAM_ITEM, rel_dtype=fr.BF16 if bf16 else fr.F32)
    assert ei.value.status == 7  # FR_EUNSUPPORTED


def test_item_param_trajectory():
    U, I, K = 40, 500, 10
    r = synth.relevance_lowrank(U, I, seed=3)
    g, o = pair_item(U, I, K, r)
    F = g.step(40)
    Fo, _ = o.step(40)
    np.testing.assert_allclose(F, Fo, rtol=NSW_RTOL)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)


def test_item_param_sgd_ascent_and_solve():
    U, I, K = 10, 120, 5
    r = synth.relevance_lowrank(U, I, seed=8)
    g, o = pair_item(U, I, K, r, optimizer=fr.SGD, lr=0.5)
    F = g.step(20)
    Fo, _ = o.step(20)
    np.testing.assert_allclose(F, Fo, rtol=NSW_RTOL)
    assert np.all(np.diff(F) > -1e-6 * np.abs(F[1:]))
    g2, o2 = pair_item(U, I, K, r)
    _, gn = o2.step(30)
    thr = float(gn[20]) * 1.0000001
    o3 = pair_item(U, I, K, r)[1]
    assert g2.solve(thr, 30)[0] == o3.solve(thr, 30)[0]


def test_item_param_state_round_trip_and_reset():
    U, I, K = 3, 41, 4
    g, _ = pair_item(U, I, K, synth.relevance_uniform(U, I, 1))
    th, m1, m2, gg = seeded(U, I, K, seed=5)
    g.set_state(th, m1, m2, gg, t=7)
    p, a, b, q, t = g.get_state()
    np.testing.assert_array_equal(p, th)
    np.testing.assert_array_equal(a, m1)
    np.testing.assert_array_equal(b, m2)
    np.testing.assert_allclose(q, gg, rtol=1e-6)
    assert t == 7
    g.reset()
    p, a, b, q, t = g.get_state()
    assert not p.any() and not a.any() and t == 0


def test_bf16_precision_scale_sample():
    """|I| = 10^4, K = 20, BF16 relevance (rank-32 sigmoid, 5% boosted items): per-consumer
    policies of sampled consumers and F of the sub-market against the oracle on the same
    BF16-rounded relevance."""
    U, I, K = 16, 10000, 20
    r = synth.relevance_lowrank_fast(U, I, seed=0, boost_frac=0.05)
    g, o = pair_item(U, I, K, r, bf16=True, sinkhorn_iters=50)
    th = synth.random_state(I, 11, 0.3).astype(np.float32)
    g.set_state(param=th)
    o.set_state(param=th.astype(np.float64))
    _, _, F = g.impacts()
    _, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    for u in (0, 9, 15):
        np.testing.assert_allclose(g.policy(u, 1), o.policy(u, 1), atol=X_ATOL)


def test_two_live_contexts_sharing_a_kernel():
    """Two contexts whose shapes select the same kernel with different shared-memory sizes: the
    larger one still launches after the smaller one was created (the limit is per kernel)."""
    ra = synth.relevance_lowrank(4, 1000, seed=1).astype(np.float32)
    rb = synth.relevance_lowrank(4, 300, seed=2).astype(np.float32)
    a, oa = pair_item(4, 1000, 20, ra, sinkhorn_iters=20)
    b, _ = pair_item(4, 300, 20, rb, sinkhorn_iters=20)
    b.step(1)
    Fa = a.step(2)
    np.testing.assert_allclose(Fa, oa.step(2)[0], rtol=NSW_RTOL)


def test_precision_workload_full_size_sampled_parity():
    """The precision workload at its full size: |U| = 200000, |I| = 10^4, K = 20, L = 50, BF16
    relevance (rank-32 sigmoid, 5% boosted items), two ascent steps from theta = 0 in the launch
    configuration the benchmark's comparison uses. The oracle then solves a seeded sample of 64
    consumers at the GPU's final theta from the GPU's warm start of the last solve, on the same
    BF16-rounded relevance: the sampled policies (max-abs 1e-5), the sample's impacts formed from
    the GPU policies (1e-5 relative) and the sample's NSW (1e-6 relative)."""
    U, I, K, L, blk, n_sample = 200000, 10000, 20, 50, 20000, 64
    rb = np.empty((U, I), dtype=np.uint16)
    for u0 in range(0, U, blk):
        rb[u0:u0 + blk] = synth.to_bf16_bits(
            synth.relevance_lowrank_fast(U, I, seed=0, boost_frac=0.05, row0=u0, rows=blk))
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, rel_dtype=fr.BF16)
    g.set_relevance(rb)
    g.set_exposure(e)
    g.step(1, trace=False)
    _, _, _, g0, _ = g.get_state()  # warm start of the last solve
    F = g.step(1)
    theta = g.get_state()[0]
    assert np.isfinite(F).all()
    sample = np.sort(np.random.default_rng(7).choice(U, n_sample, replace=False))
    X = np.stack([g.policy(int(u), 1)[0] for u in sample]).astype(np.float64)
    g.close()
    r_s = synth.bf16_bits_to_f64(rb[sample])
    del rb
    o = oracle.Oracle(n_sample, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=True)
    o.set_relevance(r_s)
    o.set_exposure(e)
    o.set_state(param=theta.astype(np.float64), g=g0[sample].astype(np.float64))
    imp_o, _, F_o = o.impacts()
    assert np.max(np.abs(X - o.policy())) <= X_ATOL
    e_pad = np.r_[e, np.zeros(fr.num_cols(I, K) - K)]
    imp_g = (r_s * (X @ e_pad)).sum(axis=0)
    assert np.max(np.abs(imp_g - imp_o) / imp_o) <= 1e-5
    assert rel(float(np.sum(np.log(imp_g))), F_o) <= NSW_RTOL
