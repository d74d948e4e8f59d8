"""GPU parity of the free-cost path (Problem (8)) against the FP64 oracle, through the C-ABI.

Tolerances: F (Eq. 5) within 1e-6 relative, policy X within 1e-5 max-abs, impacts within 1e-6
relative, gradients within 1e-5 relative L2 (FP32 kernels against the FP64 oracle on identical
seeded inputs)."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import NSW_RTOL, X_ATOL, pair, rel, require_gpu, seeded_state
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_initial_sweep_is_the_uniform_policy():
    U, I, K = 6, 23, 5
    r = synth.relevance_uniform(U, I, 3)
    g, o = pair(U, I, K, r)
    imp, util, F = g.impacts()
    oimp, outil, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    X = g.policy()
    b = np.r_[np.ones(K), I - K] / I
    np.testing.assert_allclose(X, np.broadcast_to(b, X.shape), atol=1e-6)


@pytest.mark.parametrize("U,I,K,eps,L,warm", [
    (50, 50, 50, 1.0, 50, 1),     # square doubly-stochastic (no dummy column)
    (7, 37, 10, 1.0, 50, 1),      # ragged item count, dummy column
    (3, 129, 10, 0.7, 20, 1),     # several warps per consumer, eps != 1
    (5, 11, 10, 1.0, 30, 0),      # dummy mass 1, cold start
    (2, 300, 3, 1.3, 1, 1),       # generic column bucket, L = 1
    (3, 64, 25, 1.0, 30, 1),      # generic 32-column bucket
    (4, 64, 20, 1.0, 40, 1),      # 21 columns (tile sweep, 512-float stride), one warp
    (4, 300, 20, 1.0, 30, 1),     # 21 columns, 512-float stride, several warps
    (3, 900, 20, 0.8, 20, 1),     # 21 columns, 1024-float stride, eps != 1
    (2, 1999, 20, 1.0, 10, 1),    # 21 columns, 2048-float stride, ragged item count
    # L = 1 runs only the last iteration's instantiation, L = 2 one of each
    (3, 200, 10, 1.0, 1, 1),      # 11 columns, register sweep
    (3, 701, 10, 0.9, 2, 0),      # 11 columns, register sweep, cold start
    (3, 1000, 10, 1.0, 1, 1),     # 11 columns, tile sweep
    (2, 1030, 10, 0.9, 2, 1),     # 11 columns, tile sweep, 2048-float stride
    (2, 700, 20, 1.0, 1, 1),      # 21 columns, tile sweep
    (1, 30, 5, 1.0, 50, 1),       # one consumer: one CTA, no cross-CTA partials
    (4, 40, 1, 1.0, 30, 1),       # one slot: two columns (the slot and the dummy)
])
def test_one_step_from_seeded_state(U, I, K, eps, L, warm):
    one_step_parity(U, I, K, eps, L, warm)


def one_step_parity(U, I, K, eps, L, warm):
    r = synth.relevance_lowrank(U, I, seed=U + I)
    g, o = pair(U, I, K, r, epsilon=eps, sinkhorn_iters=L, warm_start=warm)
    C, m1, m2, gg = seeded_state(U, I, K, seed=I)
    g.set_state(C, m1, m2, gg, t=3)
    o.set_state(C.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                gg.astype(np.float64), 3)
    # solve at the seeded state: F, impacts, policy, gradient
    imp, _, F = g.impacts()
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    dg = g.grad()
    do = o.grad()
    assert np.linalg.norm(dg - do) <= 1e-5 * np.linalg.norm(do)
    # one ascent step
    Fg = g.step(1)
    Fo, _ = o.step(1)
    assert rel(Fg[0], Fo[0]) < NSW_RTOL
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    pg, m1g, m2g, ggg, tg = g.get_state()
    po, m1o, m2o, ggo, to = o.get_state()
    assert tg == to == 4
    np.testing.assert_allclose(pg.reshape(-1), po, atol=2e-5, rtol=1e-5)


# The largest shape of each free-cost variant (threads: one per R items, at most 512 per CTA;
# shared memory: at most 227 KB per CTA, which the 32- and 64-column buckets reach first, since
# they also hold the policy in shared memory for the Gram block), and the first shape past it.
@pytest.mark.parametrize("I,K", [
    (4096, 10),   # 11 columns, tile sweep at a 4096-float stride, 512 threads
    (2048, 20),   # 21 columns, tile sweep at a 2048-float stride, 256 threads
    (2048, 5),    # 8-column bucket, 512 threads
    (2048, 15),   # 16-column bucket, 512 threads
    (1024, 19),   # 32-column bucket, 512 threads
    (776, 31),    # 32 columns: 776 items fill the shared memory
    (512, 40),    # 64-column bucket, 512 threads
    (320, 63),    # 64 columns: 320 items fill the shared memory
])
def test_largest_shape_of_each_free_cost_variant(I, K):
    one_step_parity(2, I, K, 1.0, 10, 1)


@pytest.mark.parametrize("I,K", [(4097, 10), (2049, 20), (2049, 5), (1025, 19), (777, 31),
                                 (513, 40), (321, 63)])
def test_free_cost_shapes_past_the_limits_are_rejected(I, K):
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(2, I, K)
    assert ei.value.status == 7  # FR_EUNSUPPORTED, with the limit in the message


def test_parity50_trajectory_against_golden():
    """|U| = |I| = 50, square, r ~ U(0,1) seed 0, 100 Adam steps x 50 Sinkhorn iterations."""
    gold = json.load(open(os.path.join(GOLDEN, "parity50.json")))
    U, I, K = gold["n_users"], gold["n_items"], gold["n_slots"]
    r = synth.workload_relevance("parity50")
    g, _ = pair(U, I, K, r, lr=gold["lr"])
    _, _, F0 = g.impacts()
    assert rel(F0, gold["F0"]) < NSW_RTOL
    F = g.step(gold["steps"])
    Fo = np.array(gold["F"])
    errs = np.abs(F - Fo) / np.abs(Fo)
    assert errs[:10].max() < NSW_RTOL
    assert errs.max() < NSW_RTOL, f"max rel F error {errs.max():.2e} at step {errs.argmax()}"
    imp, _, _ = g.impacts()
    np.testing.assert_allclose(imp, gold["imp_final"], rtol=1e-5)


def test_plain2000x1000_trajectory_against_golden():
    """The benchmarked workload in full: 2000 consumers x 1000 items, K = 10 (11 columns),
    low-rank-sigmoid relevance (seed 0), 500 Adam steps x 50 Sinkhorn iterations. F after every
    step against the FP64 oracle's stored trajectory (1e-6 relative), the final impacts at 1e-5
    relative, as for the 100-step square workload."""
    gold = json.load(open(os.path.join(GOLDEN, "plain2000x1000.json")))
    U, I, K = gold["n_users"], gold["n_items"], gold["n_slots"]
    r = synth.workload_relevance("plain2000x1000")
    g = fr.FairRank(U, I, K, lr=gold["lr"], sinkhorn_iters=gold["iters"])
    g.set_relevance(np.ascontiguousarray(r, dtype=np.float32))
    g.set_exposure(synth.dcg_exposure(K))
    _, _, F0 = g.impacts()
    assert rel(F0, gold["F0"]) < NSW_RTOL
    F = g.step(gold["steps"])
    Fo = np.array(gold["F"])
    errs = np.abs(F - Fo) / np.abs(Fo)
    assert errs.max() < NSW_RTOL, f"max rel F error {errs.max():.2e} at step {errs.argmax()}"
    imp, _, _ = g.impacts()
    np.testing.assert_allclose(imp, gold["imp_final"], rtol=1e-5)
    assert g.log_form_solves() == 0
    g.close()


def test_sgd_trajectory_policy_parity():
    U, I, K = 9, 40, 6
    r = synth.relevance_lowrank(U, I, seed=5)
    g, o = pair(U, I, K, r, optimizer=fr.SGD, lr=0.5)
    F = g.step(30)
    Fo, _ = o.step(30)
    np.testing.assert_allclose(F, Fo, rtol=NSW_RTOL)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    assert np.all(np.diff(F) > -1e-6 * np.abs(F[1:]))  # monotone ascent at small steps


def test_multiple_calls_equal_one_call_and_are_deterministic():
    U, I, K = 8, 30, 4
    r = synth.relevance_uniform(U, I, 11)
    g1, _ = pair(U, I, K, r)
    a = np.concatenate([g1.step(5), g1.step(20), g1.step(1)])
    g2, _ = pair(U, I, K, r)
    b = g2.step(26)
    np.testing.assert_array_equal(a, b)
    g2.reset()
    np.testing.assert_array_equal(g2.step(26), b)


def test_solve_stops_like_the_oracle():
    U, I, K = 6, 20, 3
    r = synth.relevance_lowrank(U, I, seed=2)
    g, o = pair(U, I, K, r)
    _, gn = o.step(60)
    thr = float(gn[40]) * 1.0000001
    o2 = pair(U, I, K, r)[1]
    n_o, F_o = o2.solve(thr, 60)
    n_g, F_g = g.solve(thr, 60)
    assert n_g == n_o
    assert rel(F_g, F_o) < NSW_RTOL


def test_single_consumer_uniform_policy_is_optimal_and_solve_stops_at_once():
    """|U| = 1 from C = 0: the uniform policy (x_ik = b_k / |I|) is optimal, so the gradient
    vanishes up to rounding and Algorithm 1's stop test ends the solve after its first step, on the
    GPU as in the oracle; SGD keeps the policy uniform and F at the closed form
    sum_i log(r_i sum_k e_k / |I|)."""
    U, I, K = 1, 30, 5
    r = synth.relevance_lowrank(U, I, seed=12)
    g, o = pair(U, I, K, r, optimizer=fr.SGD, lr=0.5)
    e = synth.dcg_exposure(K)
    r64 = np.asarray(r, dtype=np.float32).astype(np.float64)[0]
    F_unif = float(np.sum(np.log(r64 * e.sum() / I)))
    t = 1e-4
    n_g, F_g = g.solve(t, 20)
    n_o, F_o = o.solve(t, 20)
    assert n_g == n_o == 1
    _, gn = g.trace()
    assert gn.size == 1 and gn[0] <= 1e-5
    assert rel(F_g, F_unif) < 1e-7 and rel(F_o, F_unif) < 1e-12
    b = np.r_[np.ones(K), I - K] / I
    np.testing.assert_allclose(g.policy()[0], np.broadcast_to(b, (I, K + 1)), atol=1e-6)


@pytest.mark.parametrize("param", [fr.PARAM_FULL_C, fr.PARAM_ITEM])
def test_single_item_single_slot(param):
    """|I| = K = 1: one column, no dummy, so every policy is x = 1 whatever the costs; F is
    log(sum_u r_u e_1) at every step and the gradient is zero up to FP32 rounding."""
    U, I, K = 3, 1, 1
    r = np.array([[0.3], [0.9], [0.55]], dtype=np.float32)
    kw = {} if param == fr.PARAM_FULL_C else {"param": fr.PARAM_ITEM}
    g, o = pair(U, I, K, r, sinkhorn_iters=10, **kw)
    F_exact = float(np.log(r.astype(np.float64).sum()))  # e_1 = 1 / log2(2) = 1
    imp, _, F = g.impacts()
    assert rel(F, F_exact) < 1e-7 and rel(o.impacts()[2], F_exact) < 1e-14
    np.testing.assert_allclose(imp, [r.astype(np.float64).sum()], rtol=1e-7)
    np.testing.assert_allclose(g.policy(), np.ones((U, 1, 1)), atol=1e-7)
    dg = g.grad()
    assert np.max(np.abs(dg)) <= 1e-6
    Fs = g.step(3)
    Fo, _ = o.step(3)
    np.testing.assert_allclose(Fs, F_exact, rtol=1e-7)
    np.testing.assert_allclose(Fo, F_exact, rtol=1e-14)
    np.testing.assert_allclose(g.policy(), np.ones((U, 1, 1)), atol=1e-7)
    g.close()


@pytest.mark.parametrize("param", [fr.PARAM_FULL_C, fr.PARAM_ITEM])
def test_trace_reports_each_steps_objective_and_gradient_norm(param):
    """fr_trace after fr_step: F after each step equals the trace fr_step returned, and the FP64
    gradient norm of each step (the quantity Algorithm 1's stop test compares with t) matches the
    oracle's; after fr_solve the record covers exactly the steps the solve ran."""
    U, I, K = 9, 40, 5
    r = synth.relevance_lowrank(U, I, seed=4)
    kw = {} if param == fr.PARAM_FULL_C else {"param": fr.PARAM_ITEM}
    g, o = pair(U, I, K, r, **kw)
    F = g.step(15)
    Ft, gn = g.trace()
    np.testing.assert_array_equal(Ft, F)
    Fo, gno = o.step(15)
    np.testing.assert_allclose(gn, gno, rtol=1e-5)
    thr = float(gno[-1]) * 0.999
    n, Fs = g.solve(thr, 4)
    no, Fso = o.solve(thr, 4)
    Ft2, gn2 = g.trace()
    assert n == no and Ft2.size == n and gn2.size == n and Ft2[-1] == Fs
    assert rel(Fs, Fso) < NSW_RTOL
    assert np.all(gn2[:-1] > thr) and (n == 4 or gn2[-1] <= thr)
    g.close()


def test_error_statuses():
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(4, 5, 2, param=fr.PARAM_ITEM, grad_mode=7)
    g = fr.FairRank(4, 6, 2)
    with pytest.raises(fr.FairRankError) as ei:
        g.step(1)
    assert ei.value.status == 6  # FR_ESTATE
    bad = np.ones((4, 6), np.float32)
    bad[2, 3] = -1
    with pytest.raises(fr.FairRankError) as ei:
        g.set_relevance(bad)
    assert ei.value.status == 1
    zero_item = np.ones((4, 6), np.float32)
    zero_item[:, 5] = 0
    with pytest.raises(fr.FairRankError):
        g.set_relevance(zero_item)
    with pytest.raises(fr.FairRankError):
        g.set_exposure([1.0, 0.0])
    with pytest.raises(fr.FairRankError):
        g.policy(3, 2)
    g.set_relevance(np.ones((4, 6), np.float32))
    g.set_exposure([1.0, 0.5])
    g.step(2)
    assert g.launch_count() > 0


def test_state_round_trip():
    U, I, K = 3, 17, 4
    g, _ = pair(U, I, K, synth.relevance_uniform(U, I, 1))
    C, m1, m2, gg = seeded_state(U, I, K, seed=9)
    g.set_state(C, m1, m2, gg, t=12)
    p, a, b, q, t = g.get_state()
    np.testing.assert_array_equal(p, C)
    np.testing.assert_array_equal(a, m1)
    np.testing.assert_array_equal(b, m2)
    np.testing.assert_allclose(q, gg, rtol=1e-6)
    assert t == 12


def test_full_size_plain_workload_sampled_parity():
    """2000 x 1000, K = 10 (the benchmarked shape): per-consumer Sinkhorn parity on sampled
    consumers at a seeded state, and F / impacts of the whole market after the solve and after
    one ascent step against the oracle."""
    U, I, K = 2000, 1000, 10
    r = synth.relevance_lowrank(U, I, seed=0)
    g, o = pair(U, I, K, r)
    C, m1, m2, gg = seeded_state(U, I, K, seed=77, scale=0.5)
    g.set_state(C, m1, m2, gg, t=0)
    o.set_state(C.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                gg.astype(np.float64), 0)
    b, _ = oracle.marginals(I, K, synth.dcg_exposure(K))
    for u in (0, 1, 777, 1999):
        X = g.policy(u, 1)[0]
        xo, _, _ = oracle.sinkhorn(C[u].astype(np.float64), b, 1.0, 50, gg[u].astype(np.float64))
        np.testing.assert_allclose(X, xo, atol=X_ATOL)
        np.testing.assert_allclose(X.sum(1), 1.0, atol=1e-5)
    imp, _, F = g.impacts()
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    Fg = g.step(1)
    Fo, _ = o.step(1)
    assert rel(Fg[0], Fo[0]) < NSW_RTOL
    x0 = g.policy(1234, 1)[0]
    np.testing.assert_allclose(x0, o.policy(1234, 1)[0], atol=X_ATOL)
    # warm-started solves keep the tile sweep's exponential form throughout
    assert g.kernel_variant()["tile_stride"] > 0 and g.log_form_solves() == 0


def _rows_leaving_range(C, b, eps, L):
    """How often a row's sum S_i of the fused log2-domain iteration (row shifts fixed at a cold
    start) leaves [2^-64, 2^64] during an L-iteration solve, and the largest drift |g'_k - g'_k(0)|
    of a column potential, in FP64: the inputs below must reach the exact re-shift branch of the
    sweeps, and (drift beyond 30 log2 units) the tile sweep's switch to its log form."""
    cp = C / (eps * np.log(2.0))
    g = np.zeros(C.shape[1])
    ct = cp + (g - cp).max(1)[:, None]
    n, drift = 0, 0.0
    for _ in range(L):
        drift = max(drift, float(np.abs(g).max()))
        p = np.exp2(g - ct)
        S = p.sum(1)
        bad = (S < 2.0 ** -64) | (S > 2.0 ** 64)
        if bad.any():
            n += int(bad.sum())
            ct[bad] += (g - ct).max(1)[bad, None]
            p = np.exp2(g - ct)
            S = p.sum(1)
        g -= np.log2((p / S[:, None]).sum(0) / b)
    return n, drift


@pytest.mark.parametrize("I,K,scale", [
    (40, 10, 5.0),    # register sweep, 11 columns
    (40, 5, 5.0),     # register sweep, 8-column bucket
    (1030, 10, 1.5),  # tile sweep (more than 1024 items, 11 columns)
    (300, 20, 2.0),   # tile sweep, 21 columns
])
def test_rows_leaving_the_exponent_range_are_reshifted(I, K, scale):
    """eps = 0.1 and N(0, scale^2) costs from a cold start: potentials drift far enough during the
    solve that some rows' sums leave the exponent range fixed by their initial shift, so the sweep
    must re-shift them exactly; the solve still matches the oracle. (Wider cost spreads at 1030
    items leave some items with impacts below FP32's normal range, which the library reports as
    FR_ENUMERIC; the spreads here keep every impact above 1e-26.)

    Exponents reach E = max|c| / (eps ln 2) ~ 100-300 log2 units here. A term's exponent
    g'_k - c~_ik is the difference of two FP32 numbers of magnitude up to E, each rounded (up to
    E 2^-24 apiece), and g'_k also carries the rounding of the last column update, so the term is
    off by up to ~3 E 2^-24 ln 2 relative; impacts (sums of such terms) and the policy are
    compared at 4 E 2^-24 (~2.3e-5 at 1030 items, where 1.0e-5 was measured on the deepest
    tails), F (a sum of logs over items, where these errors average) at the usual 1e-6."""
    U, L, eps = 4, 50, 0.1
    r = synth.relevance_lowrank(U, I, seed=4)
    g, o = pair(U, I, K, r, epsilon=eps, sinkhorn_iters=L, warm_start=0)
    C, m1, m2, gg = seeded_state(U, I, K, seed=21, scale=scale)
    b, _ = oracle.marginals(I, K, synth.dcg_exposure(K))
    ranges = [_rows_leaving_range(C[u].astype(np.float64), b, eps, L) for u in range(U)]
    assert sum(n for n, _ in ranges) > 0
    assert min(d for _, d in ranges) > 60.0  # every consumer drifts well past 30 log2 units
    g.set_state(C, m1, m2, gg, t=0)
    o.set_state(C.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                gg.astype(np.float64), 0)
    tol = 4.0 * float(np.abs(C).max()) / (eps * np.log(2.0)) * 2.0 ** -24
    imp, _, F = g.impacts()
    # every consumer's solve leaves the sweep's exponential form (tile sweep, and the register
    # sweep of at most 11 columns) for the log form
    assert g.log_form_solves() == U
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=tol)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=max(X_ATOL, tol))


@pytest.mark.parametrize("U,I,K", [
    (1300, 1001, 10),  # register sweep
    (1300, 1201, 10),  # tile sweep
    (400, 1999, 20),   # tile sweep, 21 columns (one CTA per SM)
])
def test_several_consumers_per_cta_ragged_items(U, I, K):
    """A ragged item count (padding rows up to the next multiple of 8 in every tile) and more
    consumers than resident CTAs, so each CTA stages and solves several in turn and accumulates
    their impacts: whole-market F, impacts and gradient after the solve, F over two ascent steps,
    and the policies of consumers solved after the first by their CTA."""
    r = synth.relevance_lowrank(U, I, seed=8)
    g, o = pair(U, I, K, r)
    C, m1, m2, gg = seeded_state(U, I, K, seed=31, scale=0.5)
    g.set_state(C, m1, m2, gg, t=0)
    o.set_state(C.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                gg.astype(np.float64), 0)
    imp, _, F = g.impacts()
    oimp, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    np.testing.assert_allclose(imp, oimp, rtol=1e-6)
    dg, do = g.grad(), o.grad()
    assert np.linalg.norm(dg - do) <= 1e-5 * np.linalg.norm(do)
    Fg = g.step(2)
    Fo, _ = o.step(2)
    np.testing.assert_allclose(Fg, Fo, rtol=NSW_RTOL)
    for u in (3, U // 2 + 1, U - 1):
        np.testing.assert_allclose(g.policy(u, 1)[0], o.policy(u, 1)[0], atol=X_ATOL)


def test_differentiation_size_free_costs_sampled_parity():
    """|U| = 20000, |I| = 2000, K = 20 (21 columns), L = 100 under free costs (the tile sweep at a
    2048-float stride, one CTA per SM, about 130 consumers per CTA; C and the Adam moments 3.4 GB
    each): at a seeded state (C ~ N(0, 0.25), zero moments and potentials) the policies of sampled
    consumers against the oracle's Sinkhorn on their cost tiles, rows summing to one, and one
    ascent step raising F. (The full market is too large for the FP64 oracle in a test.)"""
    U, I, K, L = 20000, 2000, 20, 100
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, sinkhorn_iters=L)
    g.set_relevance(synth.relevance_lowrank_fast(U, I, seed=7))
    g.set_exposure(e)
    m = oracle.num_cols(I, K)
    C = (np.random.default_rng(41).standard_normal((U, I, m), dtype=np.float32) * 0.5)
    zeros = np.zeros((U, I, m), np.float32)
    g.set_state(C, zeros, zeros, np.zeros((U, m), np.float32), t=0)
    imp, _, F0 = g.impacts()
    assert np.isfinite(F0) and np.all(imp > 0)
    b, _ = oracle.marginals(I, K, e)
    for u in (0, 1, 9876, 19999):
        X = g.policy(u, 1)[0]
        xo, _, _ = oracle.sinkhorn(C[u].astype(np.float64), b, 1.0, L, np.zeros(m))
        np.testing.assert_allclose(X, xo, atol=X_ATOL)
        np.testing.assert_allclose(X.sum(1), 1.0, atol=1e-5)
    F = g.step(1)
    assert F[0] > F0


@pytest.mark.parametrize("I,K,expect", [
    (1000, 10, (11, 8, True, 128, 1024)),   # tile sweep (the benchmarked shape)
    (500, 10, (11, 4, True, 128, 0)),       # register sweep
    (2000, 20, (21, 8, True, 256, 2048)),   # 21-column tile sweep
    (300, 3, (8, 4, False, 96, 0)),         # padded 8-column bucket
])
def test_kernel_variant_reports_the_selected_sweep(I, K, expect):
    g = fr.FairRank(3, I, K)
    v = g.kernel_variant()
    got = (v["n_cols_kernel"], v["rows_per_thread"], v["exact"], v["threads"], v["tile_stride"])
    assert got == expect
    assert 1 <= v["grid"] <= 3
    p = fr.FairRank(3, I, K, param=fr.PARAM_ITEM).kernel_variant()
    assert p["tile_stride"] == 0 and p["threads"] % 32 == 0
