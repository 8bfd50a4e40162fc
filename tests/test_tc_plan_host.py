"""Host-only checks of the box plans the tensor-core tile passes use to move a tile of 12
index bits by cp.async.bulk.tensor (qc_tc_box_plan, qc_tc_block_plan; no GPU needed).

A plan groups the state's index bits into at most 5 dimensions of consecutive bits
(dimension 0 = bits 0..3); a dimension that is not one run of tile bits is copied one
element at a time and its tile bits become box coordinates (at most 2: the tile is 1, 2
or 4 boxes).  The kernel relies on one property: the box layout puts local index u of
the tile at the state address whose bit local_bits[i] is bit i of u.  These tests check
that property on seeded random tiles, check by brute force over every grouping that the
plan uses the fewest coordinate bits, and pin the block layouts the GPU tests use."""
import itertools

import numpy as np
import pytest

M, L, MAXC = 12, 4, 2


def _plan(n, bits):
    import paper_2503_03016_gb300 as P
    try:
        return P.qc_tc_box_plan(n, bits)
    except P.QCError as e:
        assert e.status == 4  # QC_ERR_UNSUPPORTED
        return None


def _runs(n, tile):
    out, b = [], L
    while b < n:
        t = b in tile
        a = b
        while b < n and (b in tile) == t:
            b += 1
        out.append((a, b - a, t))
    return out


def _min_coord_bits(n, tile):
    """Fewest tile bits left in dimensions not copied whole, over every grouping of the
    runs above bit 3 into at most 4 consecutive groups (brute force)."""
    runs = _runs(n, tile)
    R = len(runs)
    best = None
    for g in range(1, 5):
        for cuts in itertools.combinations(range(1, R), g - 1):
            bounds = (0,) + cuts + (R,)
            cost = 0
            for i, j in zip(bounds[:-1], bounds[1:]):
                if j - i > 1:
                    cost += sum(ln for (_, ln, t) in runs[i:j] if t)
            best = cost if best is None else min(best, cost)
    return best


def _check_layout(n, tile, local, dims, coords):
    assert sorted(local) == sorted(tile)
    assert local[:L] == list(range(L))
    assert len(coords) <= MAXC
    # the dimensions cover bits 0 .. n-1 once, in order; padding dimensions are empty
    nxt = 0
    for (a, ln, whole) in dims:
        if ln == 0:
            continue
        assert a == nxt
        nxt = a + ln
        if whole:
            assert all(b in tile for b in range(a, a + ln)) and ln <= 8
    assert nxt == n
    for (d, off) in coords:
        a, ln, whole = dims[d]
        assert not whole and 0 <= off < ln and (a + off) in tile
    # local index u -> state address, through the boxes and through local_bits
    nc = len(coords)
    rng = np.random.default_rng(n)
    for u in [0, (1 << M) - 1] + [int(v) for v in rng.integers(0, 1 << M, 200)]:
        e, j = u & ((1 << (M - nc)) - 1), u >> (M - nc)
        addr, shift = 0, 0
        for (a, ln, whole) in dims:
            if ln and whole:
                addr |= ((e >> shift) & ((1 << ln) - 1)) << a
                shift += ln
        assert shift == M - nc
        for q, (d, off) in enumerate(coords):
            if (j >> q) & 1:
                addr |= 1 << (dims[d][0] + off)
        want = sum(1 << local[i] for i in range(M) if (u >> i) & 1)
        assert addr == want, (u, addr, want)


def test_box_plans_map_local_bits_and_use_fewest_coordinates():
    rng = np.random.default_rng(2026)
    seen = {None: 0, 0: 0, 1: 0, 2: 0}
    for _ in range(400):
        n = int(rng.integers(12, 35))
        tile = set(range(L)) | set(int(v) for v in rng.choice(np.arange(L, n), M - L, replace=False))
        order = [int(v) for v in rng.permutation(sorted(tile))]
        plan = _plan(n, order)
        best = _min_coord_bits(n, tile)
        if plan is None:
            assert best > MAXC, (n, sorted(tile), best)
            seen[None] += 1
            continue
        local, dims, coords = plan
        assert len(coords) == best, (n, sorted(tile), coords, best)
        _check_layout(n, tile, local, dims, coords)
        seen[len(coords)] += 1
    # the sample reaches every outcome
    assert all(v > 0 for v in seen.values()), seen


def test_box_plan_rejects_invalid_tiles():
    import paper_2503_03016_gb300 as P
    with pytest.raises(P.QCError):
        P.qc_tc_box_plan(20, list(range(11)) + [3])  # a repeated bit
    with pytest.raises(P.QCError):
        P.qc_tc_box_plan(20, list(range(11)) + [20])  # a bit beyond n


def test_block_plans_contain_the_block_and_map_local_bits():
    import paper_2503_03016_gb300 as P
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = int(rng.integers(12, 33))
        k = int(rng.integers(1, 6))
        qs = [int(v) for v in rng.choice(n, k, replace=False)]
        try:
            local, dims, coords = P.qc_tc_block_plan(n, qs)
        except P.QCError as e:
            assert e.status == 4
            continue
        tile = set(local)
        assert set(range(L)) <= tile and {n - 1 - q for q in qs} <= tile
        _check_layout(n, tile, local, dims, coords)


def test_block_plan_layouts_pinned():
    """The layouts the block benchmark and the GPU block tests use: a block on index
    bits 10..14 of 28 qubits is one box; the spread block (index bits 24, 18, 13, 7, 1)
    takes two coordinate bits; index bits 6, 9, 12, 15, 19 of 22 qubits have no plan
    (the gathering block kernel takes them); the 20-qubit layouts are one box or two."""
    import paper_2503_03016_gb300 as P
    n = 28
    _, _, coords = P.qc_tc_block_plan(n, [n - 1 - b for b in range(10, 15)])
    assert coords == []
    _, _, coords = P.qc_tc_block_plan(n, [3, 9, 14, 20, 26])
    assert len(coords) == 2
    with pytest.raises(P.QCError):
        P.qc_tc_block_plan(22, [22 - 1 - b for b in (6, 9, 12, 15, 19)])
    # the 20-qubit layouts of the GPU block tests: one box, then two boxes
    for bits, nc in (((9, 10, 11, 12), 0), ((9, 10, 11, 12, 13), 0), ((2, 7, 12, 17), 1), ((1, 6, 11, 15, 18), 1)):
        _, _, coords = P.qc_tc_block_plan(20, [20 - 1 - b for b in bits])
        assert len(coords) == nc, (bits, coords)
