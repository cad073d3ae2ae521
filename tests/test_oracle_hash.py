"""Pins for the oracle's counter-based hash (jitter of Sec. 3.2, noise lattice).

The hash is the published single-state PCG hash (Jarzynski & Olano, JCGT 2020:
one 32-bit PCG LCG step, then the RXS-M-XS output permutation).  It is pinned
by inverting it exactly with the published constants (a dropped term, a wrong
shift or a wrong constant breaks the round trip), by uniformity and by
avalanche statistics.
"""
import numpy as np
import pytest

M32 = 0xFFFFFFFF
LCG_MUL, LCG_INC, RXS_MUL = 747796405, 2891336453, 277803737


def _inverse_pcg(h: int) -> int:
    word = h ^ (h >> 22)                                 # undo (w >> 22) ^ w
    x = (word * pow(RXS_MUL, -1, 1 << 32)) & M32          # undo the odd multiply
    rot = (x >> 28) + 4                                   # top 4 bits unchanged by the xorshift
    state = x
    s = x >> rot
    while s:
        state ^= s
        s >>= rot
    return ((state - LCG_INC) * pow(LCG_MUL, -1, 1 << 32)) & M32


def test_pcg_inverts_exactly(oracle):
    rng = np.random.default_rng(11)
    vals = [0, 1, 2, 0xFFFFFFFF, 0x80000000] + [int(v) for v in rng.integers(0, 1 << 32, 2000)]
    for v in vals:
        assert _inverse_pcg(oracle.pcg(v)) == v


def test_hash4_nesting(oracle):
    # h(a,b,c,d) = pcg(a ^ pcg(b ^ pcg(c ^ pcg(d))))
    rng = np.random.default_rng(12)
    for a, b, c, d in rng.integers(0, 1 << 32, (200, 4)):
        a, b, c, d = int(a), int(b), int(c), int(d)
        h = oracle.hash4(a, b, c, d)
        # peel one level with the exact inverse
        inner = _inverse_pcg(h) ^ a
        assert inner == oracle.pcg(b ^ oracle.pcg(c ^ oracle.pcg(d)))


def test_batch_matches_scalar(oracle):
    rng = np.random.default_rng(13)
    keys = rng.integers(0, 1 << 32, (500, 4), dtype=np.uint64).astype(np.uint32)
    out = oracle.hash4_batch(keys)
    for k, h in zip(keys[:50], out[:50]):
        assert oracle.hash4(*[int(v) for v in k]) == int(h)


def test_unit_uniform_chi2(oracle):
    n = 1 << 20
    i = np.arange(n, dtype=np.uint32)
    keys = np.stack([i & 1023, i >> 10, np.full(n, 7, np.uint32), np.full(n, 0x4A17 ^ 3, np.uint32)],
                    axis=1)
    u = (oracle.hash4_batch(keys) >> 8).astype(np.float64) / 16777216.0
    assert u.min() >= 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120.0  # 63 dof: p ~ 1e-5 tail


def test_avalanche(oracle):
    rng = np.random.default_rng(14)
    base = rng.integers(0, 1 << 32, 400)
    flips = []
    for v in base:
        h0 = oracle.pcg(int(v))
        for bit in range(32):
            flips.append(bin(h0 ^ oracle.pcg(int(v) ^ (1 << bit))).count("1"))
    assert 15.0 < np.mean(flips) < 17.0


def test_unit_is_top_24_bits(oracle):
    for h in (0, 255, 256, 0xFFFFFFFF, 0x12345678):
        assert oracle.unit(h) == (h >> 8) / 16777216.0


def test_jitter_range_and_frame_dependence(oracle):
    us = [oracle.jitter(3, 10, 20, f) for f in range(64)]
    assert all(0.0 <= u < 1.0 for u in us)
    assert len(set(us)) == 64
    assert oracle.jitter(3, 10, 20, 5) == oracle.unit(oracle.hash4(10, 20, 5, 3 ^ 0x4A17))
