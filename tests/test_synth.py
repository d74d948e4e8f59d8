"""The seeded input generators against definitions outside this code: SplitMix64's published first
outputs, the 53-bit uniform construction, Box-Muller moments, the exposure curve, the relevance
recipe (sigmoid of a rank-32 product plus an item bias; boosted items' odds exactly 10x) and
BF16 rounding against torch's round-to-nearest-even conversion."""
import math

import numpy as np
import torch

from paper_2406_10262_gb300 import synth

# SplitMix64 (Steele, Lea & Flood 2014) from state 0: its first three outputs, as printed by the
# reference implementation
SPLITMIX64_STATE0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_matches_the_published_sequence():
    # seed 0, stream 0 derive base state 0 (the mixer maps 0 to 0)
    assert [int(x) for x in synth.splitmix64(0, 0, 3)] == SPLITMIX64_STATE0
    # counters offset + 1 .. offset + n continue the same sequence
    assert [int(x) for x in synth.splitmix64(0, 0, 2, offset=1)] == SPLITMIX64_STATE0[1:]


def test_uniforms_are_the_top_53_bits():
    u = synth.uniform(0, 0, 3)
    np.testing.assert_array_equal(u, [(x >> 11) * 2.0**-53 for x in SPLITMIX64_STATE0])
    big = synth.uniform(3, 9, 200000)
    assert big.min() >= 0.0 and big.max() < 1.0
    assert abs(big.mean() - 0.5) < 3e-3 and abs(big.var() - 1 / 12) < 2e-3


def test_box_muller_normals_have_the_stated_moments():
    z = synth.normal(4, 2, 400001, std=2.0, mean=-1.0)
    assert z.size == 400001
    assert abs(z.mean() + 1.0) < 0.02 and abs(z.std() - 2.0) < 0.02
    # fourth standardised moment of a normal: 3
    k = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(k - 3.0) < 0.05


def test_dcg_exposure():
    e = synth.dcg_exposure(7)
    np.testing.assert_allclose(e, [1.0 / math.log2(k + 1) for k in range(1, 8)], rtol=1e-15)
    assert e[0] == 1.0 and e[2] == 0.5 and np.all(np.diff(e) < 0)


def test_lowrank_relevance_recipe_and_boost():
    U, I = 40, 200
    r = synth.relevance_lowrank(U, I, seed=3)
    assert r.shape == (U, I) and np.all((r > 0) & (r < 1))
    rb = synth.relevance_lowrank(U, I, seed=3, boost_frac=0.05)
    odds = (rb / (1 - rb)) / (r / (1 - r))
    boosted = np.all(np.abs(odds - 10.0) < 1e-9, axis=0)
    same = np.all(np.abs(odds - 1.0) < 1e-12, axis=0)
    assert boosted.sum() == round(0.05 * I) and np.all(boosted | same)
    # long-tailed popularity: the logit's item bias has mean -1 and unit spread, the rank-32 part a
    # spread of 1/sqrt(32) (p, q of std 1/sqrt(32))
    z = np.log(r / (1 - r))
    assert abs(z.mean() + 1.0) < 0.2 and 0.8 < z.mean(axis=0).std() < 1.2
    assert 0.1 < (z - z.mean(axis=0)).std() < 0.3
    # row blocks are slices of the whole matrix
    np.testing.assert_array_equal(synth.relevance_lowrank(U, I, seed=3, row0=10, rows=7), r[10:17])


def test_row_blocks_assemble_the_whole_matrix_without_repeated_rows():
    """The large workloads are generated in row blocks: concatenated blocks must be the whole
    matrix (the matmul path: up to its last bits) with every consumer's row distinct."""
    U, I, blk = 80, 50, 20
    for f, rtol in ((synth.relevance_lowrank, 0.0), (synth.relevance_lowrank_fast, 2e-6)):
        rows = np.concatenate([f(U, I, seed=0, boost_frac=0.05, row0=u0, rows=blk)
                               for u0 in range(0, U, blk)])
        full = f(U, I, seed=0, boost_frac=0.05)
        np.testing.assert_allclose(rows, full, rtol=rtol, atol=0)
        assert len(np.unique(rows, axis=0)) == U


def test_fast_lowrank_relevance_matches_the_elementwise_one():
    U, I = 30, 500
    np.testing.assert_allclose(synth.relevance_lowrank_fast(U, I, seed=5, boost_frac=0.05),
                               synth.relevance_lowrank(U, I, seed=5, boost_frac=0.05), rtol=2e-6)


def test_bf16_rounding_is_round_to_nearest_even():
    g = np.random.default_rng(0)
    x = np.concatenate([g.normal(size=5000), g.uniform(0, 1, 5000),
                        # exact ties between two bfloat16 values: odd and even lower neighbours
                        np.array([1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, 0.5 + 2.0**-9])]).astype(np.float32)
    ours = synth.to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    np.testing.assert_array_equal(synth.bf16_bits_to_f64(ours),
                                  torch.from_numpy(x).to(torch.bfloat16).double().numpy())


def test_batching_markets_follow_the_stated_distribution():
    """|U| ~ U[100, 4000], |I| ~ U[100, 2000] (inclusive integers), K uniform over {5, 10, 20},
    each market with its own relevance seed; reproducible."""
    ms = synth.markets(3000, seed=0)
    U = np.array([m.n_users for m in ms])
    I = np.array([m.n_items for m in ms])
    K = np.array([m.n_slots for m in ms])
    assert U.min() >= 100 and U.max() <= 4000 and I.min() >= 100 and I.max() <= 2000
    assert abs(U.mean() - 2050) < 60 and abs(I.mean() - 1050) < 30
    assert set(K) == {5, 10, 20} and all(abs((K == k).mean() - 1 / 3) < 0.04 for k in (5, 10, 20))
    assert len({m.seed for m in ms}) == len(ms) and np.all(I >= K)
    assert [(m.n_users, m.n_items, m.n_slots, m.seed) for m in synth.markets(5, seed=0)] == \
        [(m.n_users, m.n_items, m.n_slots, m.seed) for m in ms[:5]]
