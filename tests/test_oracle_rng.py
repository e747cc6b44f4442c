"""Pins for the oracle's counter-based generator (oracle/rng.py).

Philox4x64-10 is checked against numpy's own Philox bit generator (a library
implementation of the same published function), and the normal transform by
its moments and a Kolmogorov-Smirnov test.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import rng


def test_scalar_matches_numpy_philox():
    r = np.random.default_rng(1)
    for _ in range(20):
        key = [int(v) for v in r.integers(0, 2**63, size=2)]
        ctr = [int(v) for v in r.integers(0, 2**63, size=4)]
        # numpy increments the counter before producing a block
        prev = list(ctr)
        prev[0] = (prev[0] - 1) % (1 << 64)
        bg = np.random.Philox(key=key, counter=prev)
        assert tuple(int(v) for v in bg.random_raw(4)) == rng.philox4x64_scalar(ctr, key)


def test_vectorised_matches_scalar():
    r = np.random.default_rng(2)
    c = r.integers(0, 2**63, size=(4, 64), dtype=np.uint64)
    c[0, :5] = np.uint64(2**64 - 1)  # exercise wrap-around of the high words
    key = (0xFFFFFFFFFFFFFFFF, 12345)
    out = rng.philox4x64(c[0], c[1], c[2], c[3], *key)
    for j in range(64):
        ref = rng.philox4x64_scalar([int(c[i, j]) for i in range(4)], key)
        assert tuple(int(out[i][j]) for i in range(4)) == ref


def test_normals_moments_and_ks():
    z = rng.normals(7, rng.TAG_PRIOR_DW, 4, np.arange(50000, dtype=np.uint64), np.uint64(3), np.uint64(0)).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # odd counts keep the leading normals of the block
    z3 = rng.normals(7, rng.TAG_PRIOR_DW, 3, np.uint64(5), np.uint64(3), np.uint64(0))
    z4 = rng.normals(7, rng.TAG_PRIOR_DW, 4, np.uint64(5), np.uint64(3), np.uint64(0))
    assert np.array_equal(z3, z4[:3])


def test_uniforms():
    u = rng.uniform_open0(3, rng.TAG_PCN_ACCEPT, np.arange(100000, dtype=np.uint64), np.uint64(9))
    assert u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    v = rng.u53_int(3, rng.TAG_RESAMPLE, 11)
    assert 0 <= v < 2**53


def test_streams_are_distinct():
    a = rng.window_increments(0, rng.TAG_PRIOR_DW, 4, 5, 8, 0.025, 0)
    b = rng.window_increments(0, rng.TAG_PCN, 4, 5, 8, 0.025, 0)
    c = rng.window_increments(0, rng.TAG_PRIOR_DW, 4, 5, 8, 0.025, 1)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # a particle's draws do not depend on how many particles are drawn
    d = rng.window_increments(0, rng.TAG_PRIOR_DW, 2, 5, 8, 0.025, 0, particle0=2)
    assert np.array_equal(a[2:], d)


# Known-answer vectors published with Philox4x32-10 (Salmon et al., SC'11, and the
# Random123 distribution that accompanies it): (counter, key) -> output, 32-bit words.
PHILOX4X32_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX4X32_KAT)
def test_philox4x32_known_answers(ctr, key, out):
    assert rng.philox4x32_scalar(ctr, key) == out
    v = rng.philox4x32(*(np.array([c], dtype=np.uint64) for c in ctr), *key)
    assert tuple(int(w[0]) for w in v) == out


def test_philox4x32_vectorised_matches_scalar():
    r = np.random.default_rng(5)
    c = r.integers(0, 2**32, size=(4, 64), dtype=np.uint64)
    c[0, :3] = np.uint64(2**32 - 1)
    key = (0xFFFFFFFF, 0x1234ABCD)
    out = rng.philox4x32(c[0], c[1], c[2], c[3], *key)
    for j in range(64):
        ref = rng.philox4x32_scalar([int(c[i, j]) for i in range(4)], key)
        assert tuple(int(out[i][j]) for i in range(4)) == ref


def test_key32_separates_seeds_and_tags():
    keys = {rng.key32(s, t) for s in (0, 1, 2, 3, 2**32, 2**40 + 5) for t in range(1, 11)}
    assert len(keys) == 6 * 10


def test_normals32_moments_and_ks():
    z = rng.normals32(7, rng.TAG_PCN, 4, np.arange(50000, dtype=np.uint64), np.uint64(3), np.uint64(0)).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # a prefix of a longer draw is the shorter draw, and the two generators differ
    a = rng.normals32(7, rng.TAG_PCN, 6, np.uint64(2), np.uint64(1), np.uint64(4))
    b = rng.normals32(7, rng.TAG_PCN, 8, np.uint64(2), np.uint64(1), np.uint64(4))
    assert np.array_equal(a, b[:6])
    c = rng.normals(7, rng.TAG_PCN, 8, np.uint64(2), np.uint64(1), np.uint64(4))
    assert not np.allclose(b, c)


def test_window_increments32_layout():
    d = rng.window_increments(3, rng.TAG_PCN, 2, 3, 8, 0.25, 5, particle0=4, gen=rng.GEN32)
    assert d.shape == (2, 3, 8)
    ref = 0.5 * rng.normals32(3, rng.TAG_PCN, 8, np.uint64(2), np.uint64(5), np.uint64(5))
    assert np.array_equal(d[1, 2], ref)
