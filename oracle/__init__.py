"""FP64 CPU oracle for NSW fair ranking via gradient ascent over Sinkhorn (arXiv 2406.10262).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the CPU-baseline leg of
bench.py use it to produce expected values. The CUDA library never imports or links it, and it
imports nothing from the CUDA side; both consume inputs from `paper_2406_10262_gb300.synth`.

The arithmetic lives in fr_oracle.c (plain double-precision loops, see its header for the passage
each function restates and how each is pinned). This module is a ctypes loader plus numpy
marshalling.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from ._build import build_oracle

PARAM_FULL_C, PARAM_ITEM = 0, 1
GRAD_IMPLICIT, GRAD_UNROLLED = 0, 1
ADAM, SGD = 0, 1

_dp = ct.POINTER(ct.c_double)
_lib = None


class Config(ct.Structure):
    _fields_ = [
        ("n_users", ct.c_int32), ("n_items", ct.c_int32), ("n_slots", ct.c_int32),
        ("param", ct.c_int32), ("epsilon", ct.c_double), ("sinkhorn_iters", ct.c_int32),
        ("warm_start", ct.c_int32), ("grad_mode", ct.c_int32), ("optimizer", ct.c_int32),
        ("lr", ct.c_double), ("beta1", ct.c_double), ("beta2", ct.c_double),
        ("adam_eps", ct.c_double), ("n_threads", ct.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(build_oracle())
        i32, i64, d = ct.c_int32, ct.c_int64, ct.c_double
        vp = ct.c_void_p
        sig = {
            "orc_num_cols": (i32, [i32, i32]),
            "orc_marginals": (None, [i32, i32, _dp, _dp, _dp]),
            "orc_sinkhorn": (None, [i32, i32, _dp, _dp, d, i32, _dp, _dp, _dp]),
            "orc_cost_item": (None, [i32, i32, _dp, _dp, _dp, _dp]),
            "orc_implicit_grad": (None, [i32, i32, _dp, _dp, d, _dp]),
            "orc_unrolled_grad": (None, [i32, i32, _dp, _dp, d, i32, _dp, _dp, _dp]),
            "orc_adam": (None, [i64, _dp, _dp, _dp, _dp, i64, d, d, d, d]),
            "orc_sgd": (None, [i64, _dp, _dp, d]),
            "orc_create": (vp, [ct.POINTER(Config)]),
            "orc_destroy": (None, [vp]),
            "orc_set_relevance": (i32, [vp, _dp]),
            "orc_set_exposure": (i32, [vp, _dp, i32]),
            "orc_set_state": (i32, [vp, _dp, _dp, _dp, _dp, i64]),
            "orc_get_state": (i32, [vp, _dp, _dp, _dp, _dp, ct.POINTER(i64)]),
            "orc_step": (i32, [vp, i32, _dp, _dp]),
            "orc_solve": (i32, [vp, d, i32, ct.POINTER(i32), _dp]),
            "orc_impacts": (i32, [vp, _dp, _dp, _dp]),
            "orc_policy": (i32, [vp, i32, i32, _dp]),
            "orc_grad": (i32, [vp, _dp, _dp, _dp]),
            "orc_metrics": (i32, [vp, _dp, _dp, _dp, _dp]),
            "orc_certificate": (i32, [vp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- stateless building blocks ------------------------------------------------------------
def num_cols(I: int, K: int) -> int:
    return lib().orc_num_cols(I, K)


def marginals(I: int, K: int, e_in):
    m = num_cols(I, K)
    b, e = np.zeros(m), np.zeros(m)
    lib().orc_marginals(I, K, _p(_f64(e_in)), _p(b), _p(e))
    return b, e


def sinkhorn(c, b, eps: float, L: int, g0=None):
    """One consumer. Returns (x, g_L, g_{L-1})."""
    c = _f64(c)
    I, m = c.shape
    g = np.zeros(m) if g0 is None else _f64(g0).copy()
    x = np.zeros((I, m))
    gp = np.zeros(m)
    lib().orc_sinkhorn(I, m, _p(c), _p(_f64(b)), eps, L, _p(g), _p(x), _p(gp))
    return x, g, gp


def cost_item(r_u, e, theta):
    r_u, e, theta = _f64(r_u), _f64(e), _f64(theta)
    c = np.zeros((r_u.shape[0], e.shape[0]))
    lib().orc_cost_item(r_u.shape[0], e.shape[0], _p(r_u), _p(e), _p(theta), _p(c))
    return c


def implicit_grad(x, gx, eps: float):
    x, gx = _f64(x), _f64(gx)
    dc = np.zeros_like(x)
    lib().orc_implicit_grad(x.shape[0], x.shape[1], _p(x), _p(gx), eps, _p(dc))
    return dc


def unrolled_grad(c, b, eps: float, L: int, g0, gx):
    c, gx = _f64(c), _f64(gx)
    dc = np.zeros_like(c)
    lib().orc_unrolled_grad(c.shape[0], c.shape[1], _p(c), _p(_f64(b)), eps, L, _p(_f64(g0)),
                            _p(gx), _p(dc))
    return dc


def adam(p, m1, m2, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on p, m1, m2 (float64 contiguous)."""
    lib().orc_adam(p.size, _p(p), _p(m1), _p(m2), _p(_f64(grad)), t, lr, beta1, beta2, eps)


def sgd(p, grad, lr):
    lib().orc_sgd(p.size, _p(p), _p(_f64(grad)), lr)


# ---- engine ---------------------------------------------------------------------------------
class Oracle:
    """Algorithm 1 with state, mirroring the fr_* C-ABI of the CUDA library."""

    def __init__(self, n_users, n_items, n_slots, param=PARAM_FULL_C, epsilon=1.0, iters=50,
                 warm_start=True, grad_mode=GRAD_IMPLICIT, optimizer=ADAM, lr=None, beta1=0.9,
                 beta2=0.999, adam_eps=1e-8, threads=None):
        if lr is None:
            lr = 0.1 if param == PARAM_FULL_C else 0.05
        if threads is None:
            threads = os.cpu_count() or 1
        self.cfg = Config(n_users, n_items, n_slots, param, epsilon, iters, int(warm_start),
                          grad_mode, optimizer, lr, beta1, beta2, adam_eps, threads)
        self.U, self.I, self.K = n_users, n_items, n_slots
        self.m = num_cols(n_items, n_slots)
        self.param = param
        self.h = lib().orc_create(ct.byref(self.cfg))
        if not self.h:
            raise ValueError("invalid oracle configuration")

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self.h = None

    @property
    def nparam(self):
        return self.I if self.param == PARAM_ITEM else self.U * self.I * self.m

    def set_relevance(self, r):
        r = _f64(r)
        assert r.shape == (self.U, self.I)
        if lib().orc_set_relevance(self.h, _p(r)):
            raise ValueError("invalid relevance")

    def set_exposure(self, e):
        e = _f64(e)
        if lib().orc_set_exposure(self.h, _p(e), e.shape[0]):
            raise ValueError("invalid exposure")

    def set_state(self, param=None, m1=None, m2=None, g=None, t=0):
        conv = lambda a: None if a is None else _f64(a).reshape(-1)
        if lib().orc_set_state(self.h, _p(conv(param)), _p(conv(m1)), _p(conv(m2)), _p(conv(g)), t):
            raise ValueError("invalid state")

    def get_state(self):
        p, m1, m2 = np.zeros(self.nparam), np.zeros(self.nparam), np.zeros(self.nparam)
        g = np.zeros(self.U * self.m)
        t = ct.c_int64()
        lib().orc_get_state(self.h, _p(p), _p(m1), _p(m2), _p(g), ct.byref(t))
        return p, m1, m2, g.reshape(self.U, self.m), t.value

    def step(self, n):
        F = np.zeros(max(n, 1))
        gn = np.zeros(max(n, 1))
        if lib().orc_step(self.h, n, _p(F), _p(gn)):
            raise RuntimeError("orc_step failed")
        return F[:n], gn[:n]

    def solve(self, t, max_steps):
        done = ct.c_int32()
        F = ct.c_double()
        if lib().orc_solve(self.h, t, max_steps, ct.byref(done), ct.byref(F)):
            raise RuntimeError("orc_solve failed")
        return done.value, F.value

    def impacts(self):
        imp = np.zeros(self.I)
        util, F = ct.c_double(), ct.c_double()
        if lib().orc_impacts(self.h, _p(imp), ct.byref(util), ct.byref(F)):
            raise RuntimeError("orc_impacts failed")
        return imp, util.value, F.value

    def policy(self, u0=0, n_u=None):
        n_u = self.U - u0 if n_u is None else n_u
        x = np.zeros((n_u, self.I, self.m))
        if lib().orc_policy(self.h, u0, n_u, _p(x)):
            raise RuntimeError("orc_policy failed")
        return x

    def grad(self, omega=None, want_dr=False):
        dp = np.zeros(self.nparam)
        dr = np.zeros((self.U, self.I)) if want_dr else None
        om = None if omega is None else _f64(omega)
        if lib().orc_grad(self.h, _p(om), _p(dp), _p(dr)):
            raise RuntimeError("orc_grad failed")
        if self.param == PARAM_FULL_C:
            dp = dp.reshape(self.U, self.I, self.m)
        return (dp, dr) if want_dr else dp

    def metrics(self):
        vals = [ct.c_double() for _ in range(4)]
        if lib().orc_metrics(self.h, *[ct.byref(v) for v in vals]):
            raise RuntimeError("orc_metrics failed")
        return dict(zip(["utility", "mean_envy", "better_pct", "worse_pct"], [v.value for v in vals]))

    def certificate(self):
        gap, res = ct.c_double(), ct.c_double()
        if lib().orc_certificate(self.h, ct.byref(gap), ct.byref(res)):
            raise RuntimeError("orc_certificate failed")
        return gap.value, res.value
