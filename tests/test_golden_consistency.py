"""The stored expected values under tests/golden/ are the current oracle's: parity50 regenerated in
full by its own script, and the first steps of plain2000x1000 (whose full 500-step run takes tens of
minutes) recomputed. A change to the oracle's arithmetic that is not followed by regenerating the
files fails here instead of silently moving the GPU tests' reference."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402
import oracle  # noqa: E402
from paper_2406_10262_gb300 import synth  # noqa: E402

RTOL = 1e-12  # the oracle is deterministic; this leaves room for another libm's last bit


def stored(name):
    return json.load(open(os.path.join(HERE, "golden", f"{name}.json")))


def test_parity50_golden_is_the_oracles_output():
    g = stored("parity50")
    out = make_golden.run("parity50")
    for key in ("n_users", "n_items", "n_slots", "iters", "steps", "lr", "epsilon"):
        assert out[key] == g[key], key
    np.testing.assert_allclose(out["F0"], g["F0"], rtol=RTOL)
    np.testing.assert_allclose(out["F"], g["F"], rtol=RTOL)
    np.testing.assert_allclose(out["grad_norm"], g["grad_norm"], rtol=RTOL)
    np.testing.assert_allclose(out["imp_final"], g["imp_final"], rtol=RTOL)


def test_plain2000x1000_golden_starts_like_the_oracle():
    g = stored("plain2000x1000")
    w = synth.WORKLOADS["plain2000x1000"]
    assert (g["n_users"], g["n_items"], g["n_slots"], g["iters"]) == \
        (w["n_users"], w["n_items"], w["n_slots"], w["iters"])
    o = oracle.Oracle(w["n_users"], w["n_items"], w["n_slots"], iters=w["iters"], **make_golden.HYPER)
    o.set_relevance(synth.workload_relevance("plain2000x1000", seed=0))
    o.set_exposure(synth.dcg_exposure(w["n_slots"]))
    _, _, F0 = o.impacts()
    F, gn = o.step(2)
    np.testing.assert_allclose(F0, g["F0"], rtol=RTOL)
    np.testing.assert_allclose(F, g["F"][:2], rtol=RTOL)
    np.testing.assert_allclose(gn, g["grad_norm"][:2], rtol=RTOL)


def test_oracle_results_do_not_depend_on_its_thread_count():
    """The stored trajectories are written on one machine and used on another with a different
    core count: F, the gradient norms and the gradient must be bit-identical for any number of
    OpenMP threads (every reduction over consumers runs in a fixed order)."""
    U, I, K = 37, 60, 5
    r = synth.relevance_lowrank(U, I, seed=9)
    for param in (oracle.PARAM_FULL_C, oracle.PARAM_ITEM):
        runs = []
        for threads in (1, 3, 8):
            o = oracle.Oracle(U, I, K, param=param, iters=20, threads=threads)
            o.set_relevance(r)
            o.set_exposure(synth.dcg_exposure(K))
            F, gn = o.step(5)
            runs.append((F, gn, np.asarray(o.grad()).ravel()))
        for F, gn, g in runs[1:]:
            np.testing.assert_array_equal(F, runs[0][0])
            np.testing.assert_array_equal(gn, runs[0][1])
            np.testing.assert_array_equal(g, runs[0][2])
