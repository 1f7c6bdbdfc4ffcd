"""Pins for the oracle's Morton keys, sort order and level chop (Sect. 3.1)."""
import numpy as np
import pytest

import oracle

B = 21
CMAX = (1 << B) - 1


def decode(keys):
    keys = np.asarray(keys, np.uint64)
    c = np.zeros((keys.size, 3), np.int64)
    for k in range(B):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            c[:, a] |= ((keys >> np.uint64(3 * k + sh)) & np.uint64(1)).astype(np.int64) << k
    return c


def test_octants_2x2x2():
    # one point per octant of a cube: the top key digit is 4x + 2y + z
    pts = []
    for x in (0, 1):
        for y in (0, 1):
            for z in (0, 1):
                pts.append([0.25 + 0.5 * x, 0.25 + 0.5 * y, 0.25 + 0.5 * z, 1.0])
    pos = np.array(pts, np.float32)
    keys = oracle.morton_keys(pos)
    top = (keys >> np.uint64(60)).astype(int)
    assert list(top) == [4 * x + 2 * y + z for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    # corners quantise to 0 and to the clamped maximum on every axis
    c = decode(keys)
    assert set(np.unique(c)) == {0, CMAX}


def test_exact_cell_roundtrip():
    rng = np.random.default_rng(7)
    n = 2000
    c = rng.integers(0, CMAX, size=(n, 3))
    # (c + 1/2) / 2^21 is exact in float32; two corner points pin lo = 0, size = 1
    x = (c + 0.5) / float(1 << B)
    pos = np.zeros((n + 2, 4), np.float32)
    pos[:n, :3] = x
    pos[n, :3] = 0.0
    pos[n + 1, :3] = 1.0
    keys = oracle.morton_keys(pos)
    assert np.array_equal(decode(keys[:n]), c)
    assert np.array_equal(decode(keys[n:]), [[0, 0, 0], [CMAX, CMAX, CMAX]])


def test_sort_matches_library_and_is_stable():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 50, size=5000).astype(np.uint64) << np.uint64(40)
    order = oracle.sort_order(keys)
    ref = np.lexsort((np.arange(keys.size), keys))
    assert np.array_equal(order, ref)


def test_zorder_of_grid():
    # Z-order on a 4x4x4 grid equals ordering by interleaved digits
    g = np.arange(4)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    cell = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = np.zeros((64, 4), np.float32)
    pos[:, :3] = (cell + 0.5) / 4.0
    pos = np.concatenate([pos, [[0, 0, 0, 0], [1, 1, 1, 0]]]).astype(np.float32)
    keys = oracle.morton_keys(pos)[:64]
    digits = [(4 * (cell[:, 0] >> l & 1) + 2 * (cell[:, 1] >> l & 1) + (cell[:, 2] >> l & 1))
              for l in (1, 0)]
    ref = np.lexsort((digits[1], digits[0]))
    assert np.array_equal(np.argsort(keys, kind="stable"), ref)


def _runs(sk, lo, hi, shift):
    out, p = [], lo
    while p < hi:
        q = p + 1
        while q < hi and (int(sk[q]) >> shift) == (int(sk[p]) >> shift):
            q += 1
        out.append((p, q - p))
        p = q
    return out


def _recursive_leaves(sk, T):
    leaves = []
    def rec(lo, hi, L):
        if hi - lo <= T or L == 21:
            leaves.append((L, lo, hi - lo))
            return
        for p, c in _runs(sk, lo, hi, 63 - 3 * (L + 1)):
            rec(p, p + c, L + 1)
    if len(sk):
        rec(0, len(sk), 0)
    return sorted(leaves)


@pytest.mark.parametrize("n,T,spread", [(1, 8, 60), (9, 8, 60), (3000, 8, 63), (3000, 16, 63),
                                        (2000, 8, 12), (500, 4, 3)])
def test_chop_invariants(n, T, spread):
    rng = np.random.default_rng(n + T)
    keys = np.sort(rng.integers(0, 1 << spread, size=n, dtype=np.int64).astype(np.uint64))
    ch = oracle.chop(keys, T)
    # level-major order, first-particle order within a level
    assert np.all(np.diff(ch.level) >= 0)
    for L in np.unique(ch.level):
        sel = ch.level == L
        assert np.all(np.diff(ch.first[sel]) > 0)
    for i in range(ch.level.size):
        L, f, c = int(ch.level[i]), int(ch.first[i]), int(ch.count[i])
        sh = 63 - 3 * L
        pref = {int(k) >> sh for k in keys[f:f + c]} if L > 0 else {0}
        assert len(pref) == 1
        if c > T and L < 21:
            kids = range(ch.child_first[i], ch.child_first[i] + ch.nchild[i])
            assert sum(ch.count[k] for k in kids) == c
            assert ch.first[ch.child_first[i]] == f
            # siblings are maximal runs: neighbours differ in their prefix
            for a, b in zip(kids, list(kids)[1:]):
                assert int(keys[ch.first[b]]) >> (sh - 3) != int(keys[ch.first[a]]) >> (sh - 3)
        else:
            assert ch.nchild[i] == 0
    leaves = sorted((int(ch.level[i]), int(ch.first[i]), int(ch.count[i]))
                    for i in range(ch.level.size) if ch.nchild[i] == 0)
    assert leaves == _recursive_leaves(keys, T)
    assert sum(c for _, _, c in leaves) == n
