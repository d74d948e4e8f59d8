"""GPU parity of the unrolled gradient (adjoint kernel with checkpointed column potentials) of the
per-item parametrisation, through the C-ABI and through torch.autograd: against the FP64 oracle's
reverse sweep over the same L iterations, against central finite differences (h = 1e-3) of the
oracle's L-iteration map, and at the differentiation workload's full size (|U| = 20000, |I| = 2000,
m = 20, L = 100, checkpoints every 10) on a 64-consumer subset plus an identity that holds at any
size."""
import numpy as np
import pytest

import oracle
from gpu_util import NSW_RTOL, X_ATOL, rel, require_gpu
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5  # relative L2 error of dL/dtheta and dL/dr against the FP64 oracle


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def pair_unrolled(U, I, K, r, L, ce, bf16=False, warm=True):
    e = synth.dcg_exposure(K)
    if bf16:
        bits = synth.to_bf16_bits(np.asarray(r, dtype=np.float32))
        r_gpu, r_or = bits, synth.bf16_bits_to_f64(bits)
    else:
        r_gpu = np.ascontiguousarray(r, dtype=np.float32)
        r_or = r_gpu.astype(np.float64)
    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, rel_dtype=fr.BF16 if bf16 else fr.F32,
                    sinkhorn_iters=L, grad_mode=fr.GRAD_UNROLLED, ckpt_every=ce,
                    warm_start=int(warm))
    g.set_relevance(r_gpu)
    g.set_exposure(e)
    o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=warm,
                      grad_mode=oracle.GRAD_UNROLLED)
    o.set_relevance(r_or)
    o.set_exposure(e)
    return g, o


def l2rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("U,I,K,L,ce,bf16", [
    (9, 300, 20, 30, 10, False),    # 21 columns, 8 rows/thread, whole segments
    (5, 2000, 20, 25, 7, False),    # 21 columns, 256 threads, ragged last segment
    (3, 3000, 20, 12, 5, True),     # 21 columns, 16 rows/thread, BF16 relevance
    (3, 5000, 10, 12, 4, False),    # 11 columns, 24 rows/thread
    (7, 129, 10, 40, 10, False),    # 11 columns, ragged rows
    (6, 77, 5, 33, 10, True),       # 6 columns
    (4, 50, 3, 30, 7, False),       # padded 8-column bucket
    (4, 200, 12, 30, 10, False),    # padded 16-column bucket
    (3, 20, 20, 25, 25, False),     # |I| == K (no dummy column), padded 32-column bucket
    (4, 60, 5, 1, 10, False),       # L = 1: the output layer only
    (4, 60, 5, 9, 1, False),        # a checkpoint at every iteration
    # the largest shapes (at most 256 threads): 24 rows per thread for 6, 11 and 21 columns,
    # 8 rows for the padded buckets
    (2, 6144, 20, 10, 5, False),    # 21 columns
    (2, 6144, 10, 8, 4, True),      # 11 columns, BF16 relevance
    (2, 6144, 5, 8, 3, False),      # 6 columns
    (2, 2048, 3, 10, 5, False),     # padded 8-column bucket
    (2, 2048, 30, 6, 3, False),     # padded 32-column bucket
])
def test_unrolled_grad_matches_oracle(U, I, K, L, ce, bf16):
    r = synth.relevance_lowrank(U, I, seed=I + K + L)
    g, o = pair_unrolled(U, I, K, r, L, ce, bf16=bf16)
    m = oracle.num_cols(I, K)
    th = synth.random_state(I, I + 1, 0.4).astype(np.float32)
    gg = synth.random_state(U * m, I + 1, 0.5, 3).reshape(U, m).astype(np.float32)
    g.set_state(param=th, g=gg)
    o.set_state(param=th.astype(np.float64), g=gg.astype(np.float64))
    _, _, F = g.impacts()
    _, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    dth, dr = g.grad(want_dr=True)
    oth, odr = o.grad(want_dr=True)
    assert l2rel(dth, oth) <= GRAD_RTOL
    assert l2rel(dr, odr) <= GRAD_RTOL
    # an explicit omega (dL/dImp of another objective)
    om = (0.5 + synth.uniform(I, 77, I)).astype(np.float32)
    dth2 = g.grad(omega=om)
    oth2 = o.grad(omega=om.astype(np.float64))
    assert l2rel(dth2, oth2) <= GRAD_RTOL


def test_unrolled_ascent_trajectory_matches_oracle():
    """Adam steps driven by the unrolled gradient (a new checkpoint set every sweep)."""
    U, I, K = 12, 400, 10
    r = synth.relevance_lowrank(U, I, seed=21)
    g, o = pair_unrolled(U, I, K, r, L=20, ce=6)
    F = g.step(15)
    Fo, _ = o.step(15)
    np.testing.assert_allclose(F, Fo, rtol=NSW_RTOL)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    pg = g.get_state()[0]
    po = o.get_state()[0]
    # Adam divides each coordinate's step by its own gradient scale, so the FP32 gradient error of
    # coordinates with small gradients reaches theta almost undamped: a few 1e-6 after 15 steps
    np.testing.assert_allclose(pg, po, atol=1e-5, rtol=1e-5)


def test_unrolled_grad_against_central_differences():
    """dF/dtheta and dF/dr of the GPU adjoint against central differences (h = 1e-3) of F computed
    by the FP64 oracle's L-iteration map from a cold start (the map the reverse sweep
    differentiates)."""
    U, I, K, L, h = 6, 40, 5, 20, 1e-3
    r = synth.relevance_lowrank(U, I, seed=4)
    e = synth.dcg_exposure(K)
    th = synth.random_state(I, 3, 0.4).astype(np.float32).astype(np.float64)
    r32 = r.astype(np.float32).astype(np.float64)

    def F_oracle(theta, rr):
        o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=False)
        o.set_relevance(rr)
        o.set_exposure(e)
        o.set_state(param=theta)
        return o.impacts()[2]

    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, warm_start=0,
                    grad_mode=fr.GRAD_UNROLLED, ckpt_every=6)
    g.set_relevance(r32.astype(np.float32))
    g.set_exposure(e)
    g.set_state(param=th.astype(np.float32))
    dth, dr = g.grad(want_dr=True)
    fd = np.array([(F_oracle(th + h * np.eye(I)[i], r32) - F_oracle(th - h * np.eye(I)[i], r32))
                   / (2 * h) for i in range(I)])
    assert l2rel(dth, fd) <= 2e-5
    for (u, i) in [(0, 0), (2, 7), (5, 39), (3, 20)]:
        d = np.zeros_like(r32)
        d[u, i] = h
        f = (F_oracle(th, r32 + d) - F_oracle(th, r32 - d)) / (2 * h)
        assert abs(dr[u, i] - f) <= 2e-5 * max(abs(f), 1.0)


def test_autograd_function_matches_library_and_oracle():
    import torch

    from paper_2406_10262_gb300.autograd import SinkhornImpact
    U, I, K, L = 8, 150, 10, 30
    r = synth.relevance_lowrank(U, I, seed=9).astype(np.float32)
    th0 = synth.random_state(I, 9, 0.3).astype(np.float32)
    g, o = pair_unrolled(U, I, K, r, L=L, ce=10, warm=False)
    theta = torch.tensor(th0, device="cuda", requires_grad=True)
    rt = torch.tensor(r, device="cuda", requires_grad=True)
    imp = SinkhornImpact.apply(theta, rt, g)
    loss = torch.log(imp).sum()  # F of Eq. 5
    loss.backward()
    o.set_state(param=th0.astype(np.float64))
    oimp, _, oF = o.impacts()
    assert rel(loss.item(), oF) < NSW_RTOL
    np.testing.assert_allclose(imp.detach().cpu().numpy(), oimp, rtol=1e-6)
    oth, odr = o.grad(want_dr=True)
    assert l2rel(theta.grad.cpu().numpy(), oth) <= GRAD_RTOL
    assert l2rel(rt.grad.cpu().numpy(), odr) <= GRAD_RTOL
    # a second objective through the same function: sum_i Imp_i^2 / 2 (omega = Imp)
    theta.grad = None
    imp = SinkhornImpact.apply(theta, rt.detach(), g)
    (0.5 * (imp ** 2).sum()).backward()
    oth2 = o.grad(omega=oimp)
    assert l2rel(theta.grad.cpu().numpy(), oth2) <= GRAD_RTOL


def test_autograd_rejects_stale_backward():
    import torch

    from paper_2406_10262_gb300.autograd import SinkhornImpact
    U, I, K = 3, 30, 4
    r = synth.relevance_uniform(U, I, 2).astype(np.float32)
    g, _ = pair_unrolled(U, I, K, r, L=5, ce=2)
    theta = torch.zeros(I, device="cuda", requires_grad=True)
    rt = torch.tensor(r, device="cuda")
    a = SinkhornImpact.apply(theta, rt, g).sum()
    SinkhornImpact.apply(theta + 0.1, rt, g)
    with pytest.raises(RuntimeError):
        a.backward()


def test_unrolled_config_rejections():
    with pytest.raises(fr.FairRankError) as ex:  # beyond the free-cost adjoint's 1024 items
        fr.FairRank(4, 1100, 5, param=fr.PARAM_FULL_C, grad_mode=fr.GRAD_UNROLLED)
    assert ex.value.status == 7
    with pytest.raises(fr.FairRankError) as ex:
        fr.FairRank(4, 30, 5, param=fr.PARAM_ITEM, grad_mode=fr.GRAD_UNROLLED, ckpt_every=0)
    assert ex.value.status == 1
    with pytest.raises(fr.FairRankError) as ex:  # beyond the adjoint's 6144 items
        fr.FairRank(2, 7000, 20, param=fr.PARAM_ITEM, grad_mode=fr.GRAD_UNROLLED)
    assert ex.value.status == 7


def test_differentiation_workload_full_size():
    """|U| = 20000, |I| = 2000, m = 20, L = 100, checkpoints every 10, FP32, cold start, seeded theta
    and omega. (a) dL/dr of 64 sampled consumers and dL/dtheta of the 64-consumer sub-market against
    the FP64 oracle; (b) at full size, dL/dtheta_i = sum_u r(u,i) dL/dr(u,i) - omega_i Imp_i (from
    dL/dr = omega v - w rho and dL/dtheta = -sum_u r w rho)."""
    U, I, K, L, ce = 20000, 2000, 20, 100, 10
    r = synth.relevance_lowrank_fast(U, I, seed=7)
    e = synth.dcg_exposure(K)
    th = synth.random_state(I, 17, 0.3).astype(np.float32)
    om = (0.5 + synth.uniform(18, 77, I)).astype(np.float32)
    kw = dict(param=fr.PARAM_ITEM, sinkhorn_iters=L, warm_start=0, grad_mode=fr.GRAD_UNROLLED,
              ckpt_every=ce)
    g = fr.FairRank(U, I, K, **kw)
    g.set_relevance(r)
    g.set_exposure(e)
    g.set_state(param=th)
    imp, _, _ = g.impacts()
    dth, dr = g.grad(omega=om, want_dr=True)
    lhs = np.einsum("ui,ui->i", r.astype(np.float64), dr.astype(np.float64))
    assert l2rel(dth, lhs - om.astype(np.float64) * imp) <= 1e-5
    del g
    sub = np.sort(np.random.default_rng(5).choice(U, 64, replace=False))
    rs = np.ascontiguousarray(r[sub])
    o = oracle.Oracle(64, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=False,
                      grad_mode=oracle.GRAD_UNROLLED)
    o.set_relevance(rs.astype(np.float64))
    o.set_exposure(e)
    o.set_state(param=th.astype(np.float64))
    oth, odr = o.grad(omega=om.astype(np.float64), want_dr=True)
    assert l2rel(dr[sub], odr) <= GRAD_RTOL
    gs = fr.FairRank(64, I, K, **kw)
    gs.set_relevance(rs)
    gs.set_exposure(e)
    gs.set_state(param=th)
    assert l2rel(gs.grad(omega=om), oth) <= GRAD_RTOL


# ---- free costs (the paper's Problem (8)): dL/dc for every cell ---------------------------------
def pair_unrolled_p1(U, I, K, r, L, ce, warm=True, **kw):
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, param=fr.PARAM_FULL_C, sinkhorn_iters=L, grad_mode=fr.GRAD_UNROLLED,
                    ckpt_every=ce, warm_start=int(warm), **kw)
    g.set_relevance(np.ascontiguousarray(r, dtype=np.float32))
    g.set_exposure(e)
    okw = {k: v for k, v in kw.items() if k in ("optimizer", "lr", "epsilon")}
    o = oracle.Oracle(U, I, K, param=oracle.PARAM_FULL_C, iters=L, warm_start=warm,
                      grad_mode=oracle.GRAD_UNROLLED, **okw)
    o.set_relevance(np.asarray(r, dtype=np.float32).astype(np.float64))
    o.set_exposure(e)
    return g, o


@pytest.mark.parametrize("U,I,K,L,ce", [
    (6, 40, 10, 20, 5),      # 11 columns
    (5, 1000, 10, 12, 5),    # 11 columns, 256 threads, ragged last segment
    (4, 300, 20, 15, 4),     # 21 columns
    (3, 500, 20, 6, 2),      # 21 columns at the row limit (2 rows per thread)
    (4, 30, 5, 17, 6),       # padded 8-column bucket
    (3, 100, 13, 9, 3),      # padded 16-column bucket
    (3, 60, 25, 8, 8),       # padded 32-column bucket
    (3, 24, 24, 10, 4),      # |I| == K (no dummy column)
    (4, 50, 5, 1, 10),       # L = 1: the output layer only
    (4, 50, 5, 7, 1),        # a checkpoint at every iteration: the sweep's records, no re-runs
    (5, 1000, 10, 12, 1),    # the same, recorded by the 11-column tile sweep
    (4, 300, 20, 15, 1),     # the same, 21 columns
    # the largest shapes (at most 256 threads): 4 rows per thread up to 16 columns, 2 above
    (2, 1024, 10, 10, 5),    # 11 columns
    (2, 1024, 7, 8, 4),      # padded 8-column bucket, 8 columns
    (2, 1024, 15, 8, 4),     # padded 16-column bucket, 16 columns
    (2, 512, 20, 8, 4),      # 21 columns
    (2, 512, 31, 6, 3),      # padded 32-column bucket, 32 columns
])
def test_free_cost_unrolled_grad_matches_oracle(U, I, K, L, ce):
    """dL/dC of every cell and dL/dr from the adjoint kernel against the oracle's reverse sweep of
    the same L iterations from the same warm start, for F and for an explicit omega."""
    from gpu_util import seeded_state
    r = synth.relevance_lowrank(U, I, seed=I + K + L)
    g, o = pair_unrolled_p1(U, I, K, r, L, ce)
    C, _, _, gg = seeded_state(U, I, K, seed=I + L, scale=0.6)
    g.set_state(param=C, g=gg)
    o.set_state(param=C.astype(np.float64), g=gg.astype(np.float64))
    _, _, F = g.impacts()
    _, _, oF = o.impacts()
    assert rel(F, oF) < NSW_RTOL
    dC, dr = g.grad(want_dr=True)
    oC, odr = o.grad(want_dr=True)
    assert l2rel(dC, oC) <= GRAD_RTOL
    assert l2rel(dr, odr) <= GRAD_RTOL
    om = (0.5 + synth.uniform(I, 78, I)).astype(np.float32)
    dC2 = g.grad(omega=om)
    oC2 = o.grad(omega=om.astype(np.float64))
    assert l2rel(dC2, oC2) <= GRAD_RTOL
    # gauge invariance of the L-iteration map: every row of dL/dC_u sums to zero
    assert np.abs(dC.sum(axis=2)).max() <= 1e-5 * np.abs(dC).max()
    g.close()


@pytest.mark.parametrize("opt,ce", [(fr.ADAM, 6), (fr.SGD, 6), (fr.ADAM, 1)])
def test_free_cost_unrolled_trajectory_matches_oracle(opt, ce):
    """Ascent steps driven by the adjoint (optimiser applied in the adjoint kernel, then the
    Sinkhorn kernel on the new costs): F after every step against the oracle's trajectory; with a
    checkpoint every iteration the adjoint reverses the sweep's own records."""
    U, I, K, L = 8, 60, 10, 20
    r = synth.relevance_lowrank(U, I, seed=31)
    lr = 0.1 if opt == fr.ADAM else 0.5
    g, o = pair_unrolled_p1(U, I, K, r, L, ce, optimizer=opt, lr=lr)
    F = g.step(12)
    Fo, _ = o.step(12)
    np.testing.assert_allclose(F, Fo, rtol=NSW_RTOL)
    np.testing.assert_allclose(g.policy(), o.policy(), atol=X_ATOL)
    done, Fs = g.solve(0.0, 3)  # the device-side loop with the adjoint in its body
    ds, Fso = o.solve(0.0, 3)
    assert done == ds == 3 and rel(Fs, Fso) < NSW_RTOL
    g.close()


def test_free_cost_unrolled_limits():
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(4, 2000, 10, param=fr.PARAM_FULL_C, grad_mode=fr.GRAD_UNROLLED)
    assert ei.value.status == 7 and "n_items" in str(ei.value)


@pytest.mark.parametrize("I,K,param", [
    (1025, 10, fr.PARAM_FULL_C), (513, 20, fr.PARAM_FULL_C), (1025, 15, fr.PARAM_FULL_C),
    (513, 31, fr.PARAM_FULL_C), (6145, 20, fr.PARAM_ITEM), (2049, 3, fr.PARAM_ITEM),
])
def test_unrolled_shapes_past_the_limits_are_rejected(I, K, param):
    with pytest.raises(fr.FairRankError) as ei:
        fr.FairRank(2, I, K, param=param, grad_mode=fr.GRAD_UNROLLED, ckpt_every=5)
    assert ei.value.status == 7  # FR_EUNSUPPORTED
