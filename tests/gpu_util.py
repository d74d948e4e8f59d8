"""Shared helpers of the GPU tests: building the library and running the oracle beside it."""
import numpy as np
import pytest

import oracle
from paper_2406_10262_gb300 import build as frbuild
from paper_2406_10262_gb300 import fairrank as fr
from paper_2406_10262_gb300 import synth

# Tolerances of the FP32 path against the FP64 oracle (NSW relative, policy max-abs)
NSW_RTOL = 1e-6
X_ATOL = 1e-5


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    frbuild.build()
    return torch


def pair(U, I, K, r, seed_state=None, **kw):
    """A GPU problem and an oracle problem with the same inputs and configuration."""
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, **kw)
    g.set_relevance(np.ascontiguousarray(r, dtype=np.float32))
    g.set_exposure(e)
    okw = {k: v for k, v in kw.items() if k in ("epsilon", "warm_start", "optimizer", "lr", "beta1", "beta2", "adam_eps", "param")}
    if "sinkhorn_iters" in kw:
        okw["iters"] = kw["sinkhorn_iters"]
    o = oracle.Oracle(U, I, K, **okw)
    o.set_relevance(np.asarray(r, dtype=np.float32).astype(np.float64))  # same FP32 values
    o.set_exposure(e)
    return g, o


def seeded_state(U, I, K, seed, scale=1.0):
    m = oracle.num_cols(I, K)
    C = synth.random_state(U * I * m, seed, scale).reshape(U, I, m).astype(np.float32)
    m1 = (synth.random_state(U * I * m, seed, 0.01, 1)).reshape(U, I, m).astype(np.float32)
    m2 = np.abs(synth.random_state(U * I * m, seed, 1e-4, 2)).reshape(U, I, m).astype(np.float32)
    g = synth.random_state(U * m, seed, 0.5, 3).reshape(U, m).astype(np.float32)
    return C, m1, m2, g


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
