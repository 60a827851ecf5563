"""Pins for the oracle's clutter-resistant distance and ranking (CPU only).

Listing 1 / Eq. distanceFunctionExpression: for every row r in [0,N) and column c in [1,N),
with needle delta a = n[r][c] - n[r][c-1] and haystack delta b = h[r][c] - h[r][c-1], add
(a - b)^2 where a != 0.  Ranking (Section 4.1, tie rule of Section 4.2): the rank of the true
match is the number of haystack images with a strictly smaller distance.
"""
import numpy as np
import pytest

import synth


def img(rows):
    return np.array(rows, dtype=np.uint16)


def test_hand_computed_distance(oracle_mod):
    # needle deltas: row0 (c=1..3) = (+2, 0, -1), row1 = (0, +3, 0)
    n = img([[1, 3, 3, 2], [5, 5, 8, 8], [0, 0, 0, 0], [7, 7, 7, 7]])
    # haystack deltas: row0 = (+1, +4, -1), row1 = (+2, +1, -3), rows 2,3 arbitrary
    h = img([[0, 1, 5, 4], [2, 4, 5, 2], [9, 0, 9, 0], [1, 2, 3, 4]])
    # needle-nonzero positions only: row0 c1: (2-1)^2 = 1; row0 c3: (-1-(-1))^2 = 0;
    # row1 c2: (3-1)^2 = 4  -> total 5 (haystack changes elsewhere are ignored)
    assert oracle_mod.crss(n, h) == 5
    # the reverse direction uses the other image's non-zero deltas:
    # h as needle: row0 c1 (1-2)^2=1, c2 (4-0)^2=16, c3 (-1+1)^2=0; row1 c1 (2-0)^2=4,
    # c2 (1-3)^2=4, c3 (-3-0)^2=9; row2 c1..3 deltas (-9,+9,-9) vs 0: 243; row3 (1,1,1) vs 0: 3
    assert oracle_mod.crss(h, n) == 1 + 16 + 0 + 4 + 4 + 9 + 243 + 3


def test_first_column_and_last_row_are_in_range(oracle_mod):
    N = 6
    n = np.zeros((N, N), np.uint16)
    h = np.zeros((N, N), np.uint16)
    n[N - 1, 1:] = 4           # only change: last row, column 1 (delta +4)
    assert oracle_mod.crss(n, h) == 16
    n2 = np.zeros((N, N), np.uint16)
    n2[0, 0] = 3               # column 0 alone is never a position; it changes delta at c=1
    assert oracle_mod.crss(n2, h) == 9
    n3 = np.zeros((N, N), np.uint16)
    n3[2, N - 1] = 1           # last column
    assert oracle_mod.crss(n3, h) == 1


def test_self_distance_zero_and_nonnegative(oracle_mod):
    rng = np.random.default_rng(0)
    ims = synth.images.rici_like_images(rng, 20, 16)
    for a in ims[:5]:
        assert oracle_mod.crss(a, a) == 0
    r = oracle_mod.crss_search(ims, ims, return_distances=True)
    assert (r["distances"] >= 0).all() and (np.diag(r["distances"]) == 0).all()
    assert not np.array_equal(r["distances"], r["distances"].T)  # asymmetric


def test_constant_rows_needle_scores_zero(oracle_mod):
    rng = np.random.default_rng(1)
    needle = np.repeat(rng.integers(0, 100, size=(16, 1)), 16, axis=1).astype(np.uint16)
    for h in synth.images.rici_like_images(rng, 10, 16):
        assert oracle_mod.crss(needle, h) == 0


def test_row_constant_clutter_is_ignored(oracle_mod):
    """Fig. intersectioncounts: a constant added to a whole row leaves every delta unchanged."""
    rng = np.random.default_rng(2)
    ims = synth.images.rici_like_images(rng, 10, 32)
    for a, b in zip(ims[:5], ims[5:]):
        shifted = b.astype(np.int64) + rng.integers(0, 50, size=(32, 1))
        assert oracle_mod.crss(a, shifted.astype(np.uint16)) == oracle_mod.crss(a, b)


def test_clutter_plateau_changes_only_its_edges(oracle_mod):
    # needle row: count steps from 0 to 2 between the 3rd and 4th circle
    n = img([[0, 0, 0, 2, 2, 2, 2, 2]] * 8)
    # clutter adds 2 crossings to circles 1..5: deltas +2 at c=1 and -2 at c=6, edge intact
    h = img([[0, 2, 2, 4, 4, 4, 2, 2]] * 8)
    assert oracle_mod.crss(n, h) == 0
    # the edge moved by one circle: needle delta +2 at c=3 now meets 0 -> 4 per row
    h2 = img([[0, 0, 0, 0, 2, 2, 2, 2]] * 8)
    assert oracle_mod.crss(n, h2) == 4 * 8


def test_extreme_values_use_64_bit(oracle_mod):
    N = 64
    n = np.zeros((N, N), np.uint16)
    h = np.zeros((N, N), np.uint16)
    n[:, 1::2] = 65535      # needle deltas alternate +65535 / -65535 from c=1
    h[:, 0::2] = 65535      # haystack deltas alternate -65535 / +65535
    # every position has |a - b| = 131070 and a != 0: 64 rows x 63 columns
    assert oracle_mod.crss(n, h) == 64 * 63 * 131070 ** 2


def test_rank_matches_sorted_position_and_tie_rule(oracle_mod):
    rng = np.random.default_rng(4)
    hay = synth.images.rici_like_images(rng, 300, 16)
    q = 40
    match = rng.choice(300, q, replace=False)
    needles = hay[match].copy()
    hay = synth.images.add_plateaus(rng, hay, 0.5, 0.2, heights=1)
    # plant exact duplicates of some true matches (ties must not cost rank)
    for k in range(0, q, 4):
        hay[k] = hay[match[k]]
    r = oracle_mod.crss_search(needles, hay, true_match=match, return_distances=True)
    D = r["distances"]
    for i in range(q):
        order = np.argsort(D[i], kind="stable")
        ds = D[i][order]
        # first position in ascending order holding the true distance = the best rank
        first = int(np.searchsorted(ds, D[i, match[i]], side="left"))
        assert r["rank"][i] == first
        assert r["true_distance"][i] == D[i, match[i]]
        assert r["top1"][i] == order[0] and D[i, order[0]] == ds[0]
    dup = [k for k in range(0, q, 4) if k != match[k]]
    assert all(r["top1"][k] <= min(k, match[k]) for k in dup if r["rank"][k] == 0)


def test_self_search_ranks_zero_tiny_scene(oracle_mod):
    s = synth.tiny_scene()
    ims = oracle_mod.rici_fp64(s.vertices, s.normals, s.triangles, np.arange(s.num_vertices), 0.3, 32)
    r = oracle_mod.crss_search(ims, ims)
    assert (r["rank"] == 0).all() and (r["true_distance"] == 0).all()
