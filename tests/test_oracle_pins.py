"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Every check compares the oracle with something other than itself: closed forms, Theorem 1,
the characterisation of the entropic-OT optimum, finite differences, torch autograd and
torch.optim in float64, and brute-force enumeration of permutation mixtures.
"""
import numpy as np
import pytest
import torch

import oracle
from bruteforce import nsw_bruteforce
from paper_2406_10262_gb300 import synth


def rng(seed):
    return np.random.default_rng(seed)


def feasible_policy(I, K, seed, delta=0.05):
    """Random strictly positive X satisfying Eqs. (1)-(3): a mixture of random assignments of K
    items to the K slots (the rest to the dummy) plus delta of the uniform policy."""
    g = rng(seed)
    m = oracle.num_cols(I, K)
    X = np.zeros((I, m))
    w = g.dirichlet(np.ones(6))
    for wt in w:
        perm = g.permutation(I)
        A = np.zeros((I, m))
        for k in range(K):
            A[perm[k], k] = 1.0
        if m > K:
            A[perm[K:], K] = 1.0
        X += wt * A
    b, _ = oracle.marginals(I, K, np.ones(K))
    return (1 - delta) * X + delta * b[None, :] / I


# ---- Sec. 2 ------------------------------------------------------------------------------
def test_marginals_closed_form():
    b, e = oracle.marginals(7, 3, [1.0, 0.5, 0.25])
    assert oracle.num_cols(7, 3) == 4
    np.testing.assert_array_equal(b, [1, 1, 1, 4])  # dummy slot absorbs |I| - K items
    np.testing.assert_array_equal(e, [1.0, 0.5, 0.25, 0.0])
    b, e = oracle.marginals(4, 4, [1, 2, 3, 4])
    assert oracle.num_cols(4, 4) == 4 and np.all(b == 1.0)


# ---- Problem (7): Sinkhorn --------------------------------------------------------------
@pytest.mark.parametrize("I,K", [(6, 6), (9, 4)])
def test_zero_cost_gives_uniform_policy(I, K):
    b, _ = oracle.marginals(I, K, np.ones(K))
    m = len(b)
    x1, _, _ = oracle.sinkhorn(np.zeros((I, m)), b, 0.7, 1)
    np.testing.assert_allclose(x1, 1.0 / m, rtol=0, atol=1e-15)
    for L in (2, 5, 30):
        x, _, _ = oracle.sinkhorn(np.zeros((I, m)), b, 0.7, L)
        np.testing.assert_allclose(x, np.broadcast_to(b / I, (I, m)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("I,K,eps", [(5, 5, 1.0), (8, 3, 0.3), (12, 4, 2.0)])
def test_theorem1_round_trip(I, K, eps):
    """Theorem 1: C = -eps log X makes X the Sinkhorn solution; from g = 0 one iteration gives
    f = g = 0 and returns X."""
    X = feasible_policy(I, K, seed=I + K)
    b, _ = oracle.marginals(I, K, np.ones(K))
    C = -eps * np.log(X)
    x, g, gp = oracle.sinkhorn(C, b, eps, 1)
    np.testing.assert_allclose(x, X, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g, 0.0, atol=1e-13)
    x5, _, _ = oracle.sinkhorn(C, b, eps, 5)
    np.testing.assert_allclose(x5, X, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("I,K,eps", [(7, 3, 0.5), (6, 6, 1.0)])
def test_converged_sinkhorn_is_the_entropic_ot_optimum(I, K, eps):
    """The optimum of Problem (7) is the unique matrix with the prescribed marginals whose
    log x + c/eps is additively separable (KKT); check both properties at convergence."""
    g = rng(11)
    b, _ = oracle.marginals(I, K, np.ones(K))
    C = g.normal(size=(I, len(b)))
    x, _, _ = oracle.sinkhorn(C, b, eps, 3000)
    np.testing.assert_allclose(x.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(x.sum(0), b, atol=1e-10)
    Z = np.log(x) + C / eps
    D = Z - Z.mean(1, keepdims=True) - Z.mean(0, keepdims=True) + Z.mean()
    assert np.abs(D).max() < 1e-12


def test_gauge_invariance():
    g = rng(3)
    I, K, eps = 9, 4, 0.8
    b, _ = oracle.marginals(I, K, np.ones(K))
    C = g.normal(size=(I, len(b)))
    kappa = g.normal(size=(I, 1)) * 3
    tau = g.normal(size=(1, len(b))) * 3
    x, _, _ = oracle.sinkhorn(C, b, eps, 7)
    xr, _, _ = oracle.sinkhorn(C + kappa, b, eps, 7)  # row shifts are absorbed by f exactly
    np.testing.assert_allclose(xr, x, rtol=1e-12, atol=1e-15)
    xc, _, _ = oracle.sinkhorn(C + kappa + tau, b, eps, 3000)
    x_inf, _, _ = oracle.sinkhorn(C, b, eps, 3000)
    np.testing.assert_allclose(xc, x_inf, rtol=1e-10, atol=1e-13)


def test_column_residual_decreases_geometrically():
    g = rng(5)
    I, K, eps = 20, 5, 0.5
    b, _ = oracle.marginals(I, K, np.ones(K))
    C = g.normal(size=(I, len(b)))
    res = []
    for L in (5, 10, 20, 40):
        x, _, _ = oracle.sinkhorn(C, b, eps, L)
        np.testing.assert_allclose(x.sum(1), 1.0, atol=1e-14)  # Eq. (1) exact after row update
        res.append(np.abs(x.sum(0) - b).max())
    assert res[0] > res[1] > res[2] > res[3]
    assert res[3] < 1e-3 * res[0] or res[3] < 1e-13


# ---- gradients ----------------------------------------------------------------------------
def F_of_C(C, r, e_pad, b, eps, L, g0=None):
    """F(X*(C)) of Eq. (5) for all consumers, X* from the oracle's Sinkhorn."""
    U, I, m = C.shape
    imp = np.zeros(I)
    for u in range(U):
        x, _, _ = oracle.sinkhorn(C[u], b, eps, L, None if g0 is None else g0[u])
        imp += r[u] * (x @ e_pad)
    return np.sum(np.log(imp)), imp


def small_problem(U=2, I=5, K=2, seed=0, eps=1.0):
    r = synth.relevance_uniform(U, I, seed) + 0.05
    e_in = synth.dcg_exposure(K)
    b, e_pad = oracle.marginals(I, K, e_in)
    C = rng(seed + 100).normal(size=(U, I, len(b))) * 0.7
    return r, e_in, b, e_pad, C


def test_implicit_gradient_matches_finite_differences_at_convergence():
    r, e_in, b, e_pad, C = small_problem(U=2, I=5, K=2)
    eps, L = 0.9, 2500
    F0, imp = F_of_C(C, r, e_pad, b, eps, L)
    dC = np.zeros_like(C)
    for u in range(C.shape[0]):
        x, _, _ = oracle.sinkhorn(C[u], b, eps, L)
        gx = (r[u] / imp)[:, None] * e_pad[None, :]
        dC[u] = oracle.implicit_grad(x, gx, eps)
    h = 1e-5
    g = rng(9)
    for _ in range(12):
        j = tuple(g.integers(0, s) for s in C.shape)
        Cp, Cm = C.copy(), C.copy()
        Cp[j] += h
        Cm[j] -= h
        fd = (F_of_C(Cp, r, e_pad, b, eps, L)[0] - F_of_C(Cm, r, e_pad, b, eps, L)[0]) / (2 * h)
        assert abs(fd - dC[j]) < 1e-7 + 1e-6 * abs(fd), (j, fd, dC[j])
    # gauge invariance of X*(C): no component along row or column shifts
    np.testing.assert_allclose(dC.sum(axis=2), 0.0, atol=1e-14)
    np.testing.assert_allclose(dC.sum(axis=1), 0.0, atol=1e-14)


def torch_sinkhorn_x(c, b, eps, L, g0):
    """Independent torch restatement of L log-domain iterations (for autograd)."""
    g = g0
    logb = torch.log(b)
    for l in range(L):
        gl = g
        f = -eps * torch.logsumexp((g[None, :] - c) / eps, dim=1)
        g = eps * logb - eps * torch.logsumexp((f[:, None] - c) / eps, dim=0)
    return torch.softmax((gl[None, :] - c) / eps, dim=1)


@pytest.mark.parametrize("I,K,L,eps", [(5, 2, 1, 1.0), (6, 3, 7, 0.6), (4, 4, 12, 1.3)])
def test_unrolled_gradient_matches_torch_autograd(I, K, L, eps):
    g = rng(I * 10 + L)
    b, e_pad = oracle.marginals(I, K, synth.dcg_exposure(K))
    m = len(b)
    C = g.normal(size=(I, m))
    g0 = g.normal(size=m) * 0.3
    gx = g.uniform(0.1, 1.0, size=(I, m))
    dc = oracle.unrolled_grad(C, b, eps, L, g0, gx)
    ct = torch.tensor(C, dtype=torch.float64, requires_grad=True)
    x = torch_sinkhorn_x(ct, torch.tensor(b), eps, L, torch.tensor(g0))
    (x * torch.tensor(gx)).sum().backward()
    np.testing.assert_allclose(dc, ct.grad.numpy(), rtol=1e-10, atol=1e-12)
    xo, _, _ = oracle.sinkhorn(C, b, eps, L, g0)
    np.testing.assert_allclose(xo, x.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_unrolled_gradient_matches_finite_differences_of_L_step_map():
    r, e_in, b, e_pad, C = small_problem(U=2, I=6, K=3, seed=4)
    eps, L = 1.0, 10
    g0 = rng(1).normal(size=(2, len(b))) * 0.2
    F0, imp = F_of_C(C, r, e_pad, b, eps, L, g0)
    dC = np.stack([oracle.unrolled_grad(C[u], b, eps, L, g0[u], (r[u] / imp)[:, None] * e_pad[None, :])
                   for u in range(2)])
    h = 1e-5
    g = rng(2)
    for _ in range(10):
        j = tuple(g.integers(0, s) for s in C.shape)
        Cp, Cm = C.copy(), C.copy()
        Cp[j] += h
        Cm[j] -= h
        fd = (F_of_C(Cp, r, e_pad, b, eps, L, g0)[0] - F_of_C(Cm, r, e_pad, b, eps, L, g0)[0]) / (2 * h)
        assert abs(fd - dC[j]) < 1e-8 + 1e-6 * abs(fd)


def test_implicit_and_unrolled_agree_in_the_limit():
    r, e_in, b, e_pad, C = small_problem(U=1, I=6, K=2, seed=8)
    eps = 1.0
    x_inf, g_inf, _ = oracle.sinkhorn(C[0], b, eps, 4000)
    gx = rng(3).uniform(size=x_inf.shape)
    d_imp = oracle.implicit_grad(x_inf, gx, eps)
    d_unr = oracle.unrolled_grad(C[0], b, eps, 400, np.zeros(len(b)), gx)
    np.testing.assert_allclose(d_unr, d_imp, atol=1e-9)


# ---- optimiser ----------------------------------------------------------------------------
def test_adam_matches_torch_maximize():
    g = rng(21)
    p0 = g.normal(size=40)
    grads = [g.normal(size=40) * s for s in (1.0, 1e-3, 5.0, 0.2, 1e-6)]
    p, m1, m2 = p0.copy(), np.zeros(40), np.zeros(40)
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=0.07, betas=(0.85, 0.995), eps=1e-8, maximize=True,
                           foreach=False)
    for t, gr in enumerate(grads, start=1):
        oracle.adam(p, m1, m2, gr, t, 0.07, 0.85, 0.995, 1e-8)
        pt.grad = torch.tensor(gr)
        opt.step()
        np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-13, atol=1e-15)
    ps = p0.copy()
    oracle.sgd(ps, grads[0], 0.3)
    pt2 = torch.tensor(p0, requires_grad=True)
    o2 = torch.optim.SGD([pt2], lr=0.3, maximize=True)
    pt2.grad = torch.tensor(grads[0])
    o2.step()
    np.testing.assert_allclose(ps, pt2.detach().numpy(), rtol=1e-15)


# ---- Eqs. (4)-(5), Algorithm 1 ------------------------------------------------------------
def engine(U, I, K, r, **kw):
    o = oracle.Oracle(U, I, K, **kw)
    o.set_relevance(r)
    o.set_exposure(synth.dcg_exposure(K))
    return o


@pytest.mark.parametrize("U,I,K", [(7, 9, 3), (5, 5, 5)])
def test_uniform_policy_F_closed_form(U, I, K):
    r = synth.relevance_uniform(U, I, 1)
    o = engine(U, I, K, r)
    imp, util, F = o.impacts()
    e = synth.dcg_exposure(K)
    imp_unif = r.sum(0) * e.sum() / I  # x_uik = b_k/|I| and b_k = 1 on real slots
    np.testing.assert_allclose(imp, imp_unif, rtol=1e-13)
    np.testing.assert_allclose(F, np.log(imp_unif).sum(), rtol=1e-13)
    np.testing.assert_allclose(util, imp_unif.sum() / U, rtol=1e-13)


@pytest.mark.parametrize("kind", ["single", "separable"])
def test_uniform_policy_is_stationary_when_optimal(kind):
    """|U| = 1 or r(u,i) = a_u s_i: F is symmetric under item permutations and concave, so the
    uniform policy (C = 0) is optimal and the gradient vanishes."""
    I, K = 8, 3
    if kind == "single":
        U, r = 1, synth.relevance_uniform(1, I, 2) + 0.1
    else:
        U = 4
        g = rng(4)
        r = np.outer(g.uniform(0.2, 1, U), g.uniform(0.2, 1, I))
    o = engine(U, I, K, r, optimizer=oracle.SGD, lr=0.1)
    d = o.grad()
    assert np.abs(d).max() < 1e-13
    F, _ = o.step(3)  # SGD: Adam would normalise the rounding-level gradient into O(lr) steps
    _, _, F0 = engine(U, I, K, r).impacts()
    np.testing.assert_allclose(F, F0, rtol=1e-12)


@pytest.mark.parametrize("U,I,seed", [(2, 3, 1), (3, 3, 2), (2, 4, 3), (3, 4, 4), (1, 4, 5)])
def test_algorithm1_reaches_bruteforce_optimum(U, I, seed):
    r = synth.relevance_uniform(U, I, seed)
    e = synth.dcg_exposure(I)
    bf = nsw_bruteforce(r, e)
    assert bf["gap"] < 1e-10
    o = engine(U, I, I, r, lr=0.1, iters=50)
    F, _ = o.step(2000)
    gap, res = o.certificate()
    assert F[-1] <= bf["F"] + 1e-9  # X stays feasible, so F cannot beat F*
    assert bf["F"] - F[-1] < 1e-4 * (1 + abs(bf["F"]))
    assert gap >= bf["F"] - F[-1] - 1e-6  # Frank-Wolfe bound (X feasible up to `res`)
    imp, _, _ = o.impacts()
    np.testing.assert_allclose(imp, bf["imp"], rtol=2e-3)  # Imp* is unique


def test_nsw_is_concave_in_the_policies():
    """Eq. (5) with Eq. (4): F is a sum of logarithms of impacts linear in the policies, so
    F((X + Y) / 2) >= (F(X) + F(Y)) / 2 for feasible X, Y, strictly when the impacts differ. The
    oracle's F of chosen policies comes from Theorem 1's costs C_u = -eps log X_u, from which one
    Sinkhorn iteration from g = 0 returns X_u (checked)."""
    U, I, K = 3, 7, 3
    r = synth.relevance_uniform(U, I, 5)

    def F_of(Xs):
        o = oracle.Oracle(U, I, K, iters=1, warm_start=False)
        o.set_relevance(r)
        o.set_exposure(synth.dcg_exposure(K))
        o.set_state(param=np.stack([-np.log(X) for X in Xs]))
        np.testing.assert_allclose(o.policy(), np.stack(Xs), rtol=1e-12, atol=1e-15)
        return o.impacts()[2]

    for seed in range(6):
        Xs = [feasible_policy(I, K, seed=100 * seed + u) for u in range(U)]
        Ys = [feasible_policy(I, K, seed=100 * seed + 50 + u) for u in range(U)]
        Ms = [(x + y) / 2 for x, y in zip(Xs, Ys)]
        fx, fy, fm = F_of(Xs), F_of(Ys), F_of(Ms)
        assert fm > (fx + fy) / 2 + 1e-9
        assert F_of(Xs) == fx  # deterministic


def test_certificate_bounds_gap_for_random_feasible_policies():
    U, I = 3, 4
    r = synth.relevance_uniform(U, I, 7)
    e = synth.dcg_exposure(I)
    Fstar = nsw_bruteforce(r, e)["F"]
    for s in range(5):
        X = np.stack([feasible_policy(I, I, seed=50 + 3 * s + u, delta=0.2) for u in range(U)])
        o = engine(U, I, I, r, iters=1, warm_start=False)
        o.set_state(param=-np.log(X))  # Theorem 1: the policy is X itself
        np.testing.assert_allclose(o.policy(), X, rtol=1e-12)
        gap, res = o.certificate()
        _, _, F = o.impacts()
        assert res < 1e-12
        assert gap >= Fstar - F - 1e-12 and Fstar - F > 0


def test_small_step_sgd_ascent_is_monotone():
    U, I, K = 6, 10, 3
    r = synth.relevance_lowrank(U, I, seed=3)
    o = engine(U, I, K, r, optimizer=oracle.SGD, lr=0.05, iters=200, warm_start=True)
    F, _ = o.step(40)
    assert np.all(np.diff(F) > -1e-12)
    assert F[-1] > F[0]


def test_metrics_match_definition_by_item_swap():
    """Sec. 4.1 metrics recomputed by literally handing item j's rankings to item i."""
    U, I, K = 4, 6, 2
    r = synth.relevance_uniform(U, I, 9)
    e = synth.dcg_exposure(K)
    o = engine(U, I, K, r)
    o.step(15)
    X = o.policy()
    imp, _, _ = o.impacts()
    met = o.metrics()

    def impact_of_item(i, Xslice):
        return sum(r[u, i] * sum(e[k] * Xslice[u, k] for k in range(K)) for u in range(U))

    envy = []
    for i in range(I):
        own = impact_of_item(i, X[:, i, :])
        envy.append(max(impact_of_item(i, X[:, j, :]) - own for j in range(I)))
    np.testing.assert_allclose(met["mean_envy"], np.mean(envy), rtol=1e-12)
    unif = np.array([impact_of_item(i, np.tile(np.r_[np.ones(K), I - K] / I, (U, 1))) for i in range(I)])
    assert met["better_pct"] == pytest.approx(100.0 * np.mean(imp > 1.1 * unif))
    assert met["worse_pct"] == pytest.approx(100.0 * np.mean(imp < 0.9 * unif))
    assert met["utility"] == pytest.approx(imp.sum() / U, rel=1e-14)
    # at the uniform policy every item holds the same rankings: no envy, nobody better/worse off
    m0 = engine(U, I, K, r).metrics()
    assert abs(m0["mean_envy"]) < 1e-14 and m0["better_pct"] == 0 and m0["worse_pct"] == 0


def test_metrics_at_optimum_match_bruteforce_optimum():
    U, I = 2, 3
    r = synth.relevance_uniform(U, I, 1)
    e = synth.dcg_exposure(I)
    bf = nsw_bruteforce(r, e)
    o = engine(U, I, I, r)
    o.step(2000)
    V = np.einsum("uik,k->ui", bf["X"], e)
    E = r.T @ V
    envy_bf = (E - np.diag(E)[:, None]).max(axis=1).mean()
    assert o.metrics()["mean_envy"] == pytest.approx(envy_bf, abs=5e-4)


# ---- per-item parametrisation -------------------------------------------------------------
def test_item_parametrisation_cost_and_gradients():
    U, I, K = 3, 7, 3
    r = synth.relevance_uniform(U, I, 12) + 0.05
    e = synth.dcg_exposure(K)
    theta = rng(6).normal(size=I) * 0.5
    b, e_pad = oracle.marginals(I, K, e)
    c = oracle.cost_item(r[0], e_pad, theta)
    np.testing.assert_allclose(c, -r[0][:, None] * e_pad[None, :] * np.exp(theta)[:, None], rtol=1e-15)

    def F_theta(th, rr, L, warm_g=None):
        imp = np.zeros(I)
        for u in range(U):
            cu = -rr[u][:, None] * e_pad[None, :] * np.exp(th)[:, None]
            x, _, _ = oracle.sinkhorn(cu, b, 1.0, L, None if warm_g is None else warm_g[u])
            imp += rr[u] * (x @ e_pad)
        return np.log(imp).sum()

    for mode, L in ((oracle.GRAD_UNROLLED, 9), (oracle.GRAD_IMPLICIT, 3000)):
        o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=False, grad_mode=mode)
        o.set_relevance(r)
        o.set_exposure(e)
        o.set_state(param=theta)
        dth, dr = o.grad(want_dr=True)
        h = 1e-5
        for i in range(I):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += h
            tm[i] -= h
            fd = (F_theta(tp, r, L) - F_theta(tm, r, L)) / (2 * h)
            assert abs(fd - dth[i]) < 1e-7 + 1e-6 * abs(fd)
        for (u, i) in [(0, 0), (1, 3), (2, 6)]:
            rp, rm = r.copy(), r.copy()
            rp[u, i] += h
            rm[u, i] -= h
            fd = (F_theta(theta, rp, L) - F_theta(theta, rm, L)) / (2 * h)
            assert abs(fd - dr[u, i]) < 1e-7 + 1e-6 * abs(fd)


# ---- Algorithm 1's threshold loop -----------------------------------------------------------
@pytest.mark.parametrize("kind", ["single", "separable"])
def test_solve_stops_after_one_step_when_uniform_policy_is_optimal(kind):
    """|U| = 1 or separable r: the uniform policy (C = 0) is optimal, so the gradient of the first
    step is at rounding level and Algorithm 1 with t = 1e-12 stops after exactly one step, with F
    equal to the uniform policy's closed form."""
    I, K = 8, 3
    if kind == "single":
        U, r = 1, synth.relevance_uniform(1, I, 2) + 0.1
    else:
        U = 4
        g = rng(4)
        r = np.outer(g.uniform(0.2, 1, U), g.uniform(0.2, 1, I))
    e = synth.dcg_exposure(K)
    F_unif = np.log(r.sum(0) * e.sum() / I).sum()
    for opt in (oracle.SGD, oracle.ADAM):
        o = engine(U, I, K, r, optimizer=opt, lr=0.1)
        done, F = o.solve(1e-12, 50)
        assert done == 1
        np.testing.assert_allclose(F, F_unif, rtol=1e-12)


def test_solve_with_zero_threshold_runs_every_step():
    """A non-separable market has a nonzero gradient at every iterate, so t = 0 never stops the
    loop early: max_steps steps run (and max_steps = 0 runs none)."""
    U, I, K = 3, 6, 2
    r = synth.relevance_uniform(U, I, 6) + 0.05
    o = engine(U, I, K, r)
    done, F = o.solve(0.0, 17)
    assert done == 17
    _, gn = engine(U, I, K, r).step(17)
    assert np.all(gn > 0)
    o0 = engine(U, I, K, r)
    done0, F0 = o0.solve(0.0, 0)
    assert done0 == 0
    np.testing.assert_allclose(F0, engine(U, I, K, r).impacts()[2], rtol=0)


def test_step_trace_reports_the_norm_of_the_gradient_it_ascends():
    """The norm tested by Algorithm 1's stop rule is ||dF/dC||_2 of the step's own gradient: each
    entry of the step trace equals the norm of orc_grad (pinned by finite differences) taken at
    the state before that step."""
    U, I, K = 3, 5, 2
    r = synth.relevance_uniform(U, I, 8) + 0.05
    o = engine(U, I, K, r)
    for _ in range(4):
        d = o.grad()
        _, gn = o.step(1)
        np.testing.assert_allclose(gn[0], np.linalg.norm(d), rtol=1e-12)


@pytest.mark.parametrize("U,I,seed", [(2, 3, 1), (3, 4, 4)])
def test_solve_stops_at_the_first_step_below_threshold(U, I, seed):
    """On brute-force instances (where the step trajectory reaches F*, pinned above): for a
    threshold strictly between the gradient norm of step j and the smallest norm of the earlier
    steps, solve(t) runs exactly j steps (1-based) and returns the F the step trajectory has
    after step j. A stop tested before the update, or on the next step's norm, fails this."""
    r = synth.relevance_uniform(U, I, seed)
    bf = nsw_bruteforce(r, synth.dcg_exposure(I))
    F_tr, gn = engine(U, I, I, r, lr=0.1, iters=50).step(400)
    assert bf["F"] - F_tr[-1] < 1e-3 * (1 + abs(bf["F"]))
    running_min = np.minimum.accumulate(gn)
    records = [j for j in range(1, len(gn)) if gn[j] < running_min[j - 1]]
    picks = sorted({records[0], records[len(records) // 2], records[-1]})
    for j in picks:
        t = 0.5 * (gn[j] + running_min[j - 1])
        assert gn[j] <= t < running_min[j - 1]
        done, F = engine(U, I, I, r, lr=0.1, iters=50).solve(t, 400)
        assert done == j + 1
        assert F == F_tr[j]


# ---- gradient of a weighted impact sum (the backward of Imp) --------------------------------
def imp_of(param_kind, P, r, e_pad, b, eps, L):
    """Imp (Eq. 4) for all consumers from cold-started Sinkhorn solves of the oracle, for free
    costs C [U, I, m] or per-item variables theta [I]."""
    U, I = r.shape
    imp = np.zeros(I)
    for u in range(U):
        if param_kind == "C":
            cu = P[u]
        else:
            cu = -r[u][:, None] * e_pad[None, :] * np.exp(P)[:, None]
        x, _, _ = oracle.sinkhorn(cu, b, eps, L)
        imp += r[u] * (x @ e_pad)
    return imp


@pytest.mark.parametrize("param_kind", ["C", "theta"])
@pytest.mark.parametrize("mode,L", [(oracle.GRAD_IMPLICIT, 3000), (oracle.GRAD_UNROLLED, 9)])
def test_omega_weighted_gradient_matches_finite_differences(param_kind, mode, L):
    """orc_grad with an explicit omega is the gradient of L = sum_i omega_i Imp_i (not of F):
    central differences of that sum for a random omega, in the parameters and in r."""
    U, I, K = 3, 6, 2
    eps = 1.0 if param_kind == "theta" else 0.8
    r = synth.relevance_uniform(U, I, 31) + 0.05
    e = synth.dcg_exposure(K)
    b, e_pad = oracle.marginals(I, K, e)
    g = rng(77)
    omega = g.uniform(-1.0, 2.0, size=I)
    if param_kind == "C":
        P = g.normal(size=(U, I, len(b))) * 0.6
        o = oracle.Oracle(U, I, K, param=oracle.PARAM_FULL_C, epsilon=eps, iters=L,
                          warm_start=False, grad_mode=mode)
    else:
        P = g.normal(size=I) * 0.5
        o = oracle.Oracle(U, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=False,
                          grad_mode=mode)
    o.set_relevance(r)
    o.set_exposure(e)
    o.set_state(param=P)
    dP, dr = o.grad(omega=omega, want_dr=True)
    dP_F = o.grad()
    assert np.abs(dP - dP_F).max() > 1e-3  # omega is not 1/Imp: the two gradients differ
    Lw = lambda PP, rr: omega @ imp_of(param_kind, PP, rr, e_pad, b, eps, L)
    h = 1e-5
    coords = [tuple(g.integers(0, s) for s in P.shape) for _ in range(8)]
    for j in coords:
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += h
        Pm[j] -= h
        fd = (Lw(Pp, r) - Lw(Pm, r)) / (2 * h)
        assert abs(fd - dP[j]) < 1e-7 + 1e-6 * abs(fd), (j, fd, dP[j])
    for (u, i) in [(0, 0), (1, 3), (2, 5)]:
        rp, rm = r.copy(), r.copy()
        rp[u, i] += h
        rm[u, i] -= h
        fd = (Lw(P, rp) - Lw(P, rm)) / (2 * h)
        assert abs(fd - dr[u, i]) < 1e-7 + 1e-6 * abs(fd), ((u, i), fd, dr[u, i])
