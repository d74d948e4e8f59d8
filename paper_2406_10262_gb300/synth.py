"""Seeded synthetic inputs for the fair-ranking workloads (numpy only).

This module generates problem data -- relevance matrices r(u,i), exposure curves e(k), market
shapes and initial optimiser states -- and nothing else: it holds none of the ranking method's
arithmetic, so both the CUDA path and the FP64 oracle can consume its output.

Randomness is counter based: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) evaluated at counters 1..n of a stream whose base is derived
from (seed, stream id). Uniforms are the top 53 bits scaled by 2^-53; normals use Box-Muller.
Every tensor draws from its own stream id, so shapes can change without reshuffling others.

The paper evaluates on the synthetic generator of Saito & Joachims and on the Delicious dataset
(Sec. 4.1); neither is available here, so the workloads below stand in for them with seeded data
of the stated shapes and value distributions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids
S_REL, S_P, S_Q, S_BIAS, S_BOOST, S_MARKET, S_STATE = 1, 2, 3, 4, 5, 6, 7


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n SplitMix64 outputs of stream (seed, stream), counters offset+1 .. offset+n."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed * 0x100000001B3 + stream * 0xD1B54A32D192ED03) & (2**64 - 1)],
                             dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(base + ctr * _GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) doubles: (x >> 11) * 2^-53."""
    return (splitmix64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def normal(seed: int, stream: int, n: int, std: float = 1.0, mean: float = 0.0) -> np.ndarray:
    """N(mean, std^2) doubles by Box-Muller on pairs of uniforms of one stream."""
    h = (n + 1) // 2
    u = uniform(seed, stream, 2 * h)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
    return mean + std * z[:n]


def dcg_exposure(K: int) -> np.ndarray:
    """e(k) = 1 / log2(k + 1) for slots k = 1..K (the position-based exposure of the workloads)."""
    return 1.0 / np.log2(np.arange(2, K + 2, dtype=np.float64))


def relevance_uniform(U: int, I: int, seed: int = 0) -> np.ndarray:
    """r(u,i) ~ Uniform(0,1), float64, shape (U, I)."""
    return uniform(seed, S_REL, U * I).reshape(U, I)


def relevance_lowrank(U: int, I: int, seed: int = 0, dim: int = 32, boost_frac: float = 0.0,
                      boost: float = 10.0, dtype=np.float64, row0: int = 0, rows: int | None = None):
    """r(u,i) = sigmoid(p_u . q_i + b_i): p, q ~ N(0, std 1/sqrt(dim)) of dimension dim and an item
    bias b_i ~ N(-1, 1) (long-tailed popularity). A seeded boost_frac of the items get their odds
    multiplied by `boost` (b_i += log(boost)). Rows row0 .. row0+rows of the (U, I) matrix.

    The dot products are accumulated one dimension at a time with elementwise float64 numpy
    operations so that the values do not depend on the BLAS of the machine."""
    rows = U - row0 if rows is None else rows
    std = 1.0 / math.sqrt(dim)
    q = normal(seed, S_Q, I * dim, std=std).reshape(I, dim)
    b = normal(seed, S_BIAS, I, std=1.0, mean=-1.0)
    if boost_frac > 0.0:
        nb = int(round(boost_frac * I))
        order = np.argsort(uniform(seed, S_BOOST, I), kind="stable")
        b[order[:nb]] += math.log(boost)
    # the consumer factors of all U rows, then the block: `normal` pairs its Box-Muller draws
    # according to the count requested, so drawing only row0 + rows rows would give other values
    # (and blocks that repeat rows of other blocks)
    p = normal(seed, S_P, U * dim, std=std).reshape(U, dim)[row0:row0 + rows]
    z = np.broadcast_to(b, (rows, I)).copy()
    for d in range(dim):
        z += p[:, d:d + 1] * q[None, :, d]
    r = 1.0 / (1.0 + np.exp(-z))
    return r.astype(dtype)


def relevance_lowrank_fast(U: int, I: int, seed: int = 0, dim: int = 32, boost_frac: float = 0.0,
                           boost: float = 10.0, row0: int = 0, rows: int | None = None):
    """Same distribution as relevance_lowrank, float32 through a BLAS matmul: for matrices too
    large for the elementwise path. Values may differ across machines, and a row block from the
    same rows of the whole matrix, in the last bits (the matmul's blocking), so both sides of any
    comparison must consume the same array."""
    rows = U - row0 if rows is None else rows
    std = 1.0 / math.sqrt(dim)
    q = normal(seed, S_Q, I * dim, std=std).reshape(I, dim).astype(np.float32)
    b = normal(seed, S_BIAS, I, std=1.0, mean=-1.0)
    if boost_frac > 0.0:
        nb = int(round(boost_frac * I))
        order = np.argsort(uniform(seed, S_BOOST, I), kind="stable")
        b[order[:nb]] += math.log(boost)
    p = normal(seed, S_P, U * dim, std=std).reshape(U, dim)[row0:row0 + rows]  # as above
    z = p.astype(np.float32) @ q.T
    z += b.astype(np.float32)[None, :]
    np.negative(z, out=z)
    np.exp(z, out=z)
    z += np.float32(1.0)
    np.reciprocal(z, out=z)
    return z


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (b >> np.uint32(16)) & np.uint32(1)
    rounded = (b + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


@dataclass
class Market:
    n_users: int
    n_items: int
    n_slots: int
    seed: int


def markets(n_markets: int, seed: int = 0, users=(100, 4000), items=(100, 2000),
            slots=(5, 10, 20)) -> list[Market]:
    """Independent markets with |U| ~ U[users], |I| ~ U[items] (integers, inclusive) and K drawn
    uniformly from `slots`; each market's relevance uses its own seed."""
    u = uniform(seed, S_MARKET, 3 * n_markets).reshape(n_markets, 3)
    out = []
    for j in range(n_markets):
        nu = users[0] + int(u[j, 0] * (users[1] - users[0] + 1))
        ni = items[0] + int(u[j, 1] * (items[1] - items[0] + 1))
        k = slots[int(u[j, 2] * len(slots))]
        out.append(Market(nu, max(ni, k), k, seed * 1000003 + j + 1))
    return out


def random_state(n: int, seed: int, scale: float = 1.0, stream_off: int = 0) -> np.ndarray:
    """Seeded N(0, scale^2) values for optimiser states (costs, moments, potentials)."""
    return normal(seed, S_STATE + 16 * stream_off, n, std=scale)


# ---- the named workloads -------------------------------------------------------------------
WORKLOADS = {
    # 50 consumers x 50 items, 50 slots (square doubly-stochastic X_u), r ~ U(0,1), seed 0
    "parity50": dict(n_users=50, n_items=50, n_slots=50, gen="uniform", steps=100, iters=50),
    # 2000 consumers x 1000 items, 10 slots + dummy, low-rank sigmoid relevance, 500 steps
    "plain2000x1000": dict(n_users=2000, n_items=1000, n_slots=10, gen="lowrank", steps=500,
                           iters=50),
}


def workload_relevance(name: str, seed: int = 0) -> np.ndarray:
    w = WORKLOADS[name]
    if w["gen"] == "uniform":
        return relevance_uniform(w["n_users"], w["n_items"], seed)
    return relevance_lowrank(w["n_users"], w["n_items"], seed)
