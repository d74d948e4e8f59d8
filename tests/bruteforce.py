"""Brute-force NSW optimum for tiny square instances (|I| = K <= 4, |U| <= 3).

By Birkhoff-von Neumann every doubly-stochastic X_u is a mixture of permutation matrices, so
Problem (6) becomes a maximisation of F over mixture weights lambda_u on the simplex of the |I|!
permutations of each consumer. F is concave in lambda; we maximise it by pairwise Frank-Wolfe with
an exact enumeration LMO and exact line search, and stop when the Frank-Wolfe gap (an upper bound
on F* - F) is below `tol`. Independent of the oracle: numpy only.
"""
from __future__ import annotations

import itertools

import numpy as np


def nsw_bruteforce(r: np.ndarray, e: np.ndarray, tol: float = 1e-12, max_iter: int = 200000):
    r = np.asarray(r, dtype=np.float64)
    U, I = r.shape
    K = len(e)
    assert I == K, "square instances only"
    perms = list(itertools.permutations(range(I)))
    P = len(perms)
    # A[u, p, i] = impact on item i of consumer u ranking by permutation p (item i -> slot p[i])
    A = np.zeros((U, P, I))
    for p, pi in enumerate(perms):
        for i in range(I):
            A[:, p, i] = r[:, i] * e[pi[i]]
    lam = np.full((U, P), 1.0 / P)

    def imp_of(l):
        return np.einsum("up,upi->i", l, A)

    gap = np.inf
    for it in range(max_iter):
        imp = imp_of(lam)
        g = np.einsum("upi,i->up", A, 1.0 / imp)  # dF/dlambda
        gap = float(np.sum(g.max(axis=1) - np.sum(lam * g, axis=1)))
        if gap < tol:
            break
        u = it % U
        s = int(np.argmax(g[u]))
        active = np.where(lam[u] > 0)[0]
        a = int(active[np.argmin(g[u, active])])
        if s == a:
            continue
        d = A[u, s] - A[u, a]
        gmax = lam[u, a]
        # exact line search of the concave phi(t) = sum log(imp + t d) on [0, gmax]
        dphi = lambda t: float(np.sum(d / (imp + t * d)))
        if dphi(gmax) >= 0:
            t = gmax
        else:
            lo, hi = 0.0, gmax
            for _ in range(100):
                mid = 0.5 * (lo + hi)
                if dphi(mid) > 0:
                    lo = mid
                else:
                    hi = mid
            t = 0.5 * (lo + hi)
        lam[u, s] += t
        lam[u, a] -= t
        if lam[u, a] < 1e-300:
            lam[u, a] = 0.0
    imp = imp_of(lam)
    X = np.zeros((U, I, K))
    for p, pi in enumerate(perms):
        for i in range(I):
            X[:, i, pi[i]] += lam[:, p]
    return dict(F=float(np.sum(np.log(imp))), imp=imp, X=X, gap=gap, lam=lam)
