"""CPU models of two device algorithms of the labelling kernels, checked under
arbitrary interleavings of the warp's lanes (the GPU parity tests fix the
kernels' results; these fix the arguments that make them hold under any
schedule).

1. The tile union-find over runs: lane r owns row r's runs (ids r*32 + j).
   Each run of row r > 0 takes as parent the first run of row r-1 that it
   touches; pointer jumping (parent := grandparent, rounds separated by
   barriers, until no parent changes) makes every parent a tree root; the
   remaining touching pairs join their trees (union by smaller root, the
   compare-and-min of the kernel); a last find per run flattens. Within a
   round the lanes' loads and stores are interleaved at random, so a load may
   see another lane's store of the same round. The result must be the tile's
   4- or 8-connected components, each run's slot holding the component's
   smallest run id.
2. The warp-wide segment search: the lanes read 32 evenly spaced entries of
   the remaining range of a nondecreasing prefix table and vote; the answer
   is the last segment whose start is <= g (empty segments skipped).
"""
from __future__ import annotations

import bisect

import numpy as np
import pytest
from scipy import ndimage

from paper_1607_00908_gb300 import inputs as I

TW, TH = 64, 32


def runs_of(row):
    """(start, length) of the runs of a boolean row, left to right."""
    out, c = [], 0
    while c < len(row):
        if row[c]:
            s = c
            while c < len(row) and row[c]:
                c += 1
            out.append((s, c - s))
        else:
            c += 1
    return out


def touching_pairs(runs, runs_up, conn8):
    """(j, ju) pairs in the order the kernel enumerates them."""
    pairs = []
    if not conn8:
        # one pair per segment of (row AND row above), in column order
        cover = {}
        for j, (s, n) in enumerate(runs):
            for c in range(s, s + n):
                cover[c] = j
        cover_up = {}
        for ju, (s, n) in enumerate(runs_up):
            for c in range(s, s + n):
                cover_up[c] = ju
        last = None
        for c in range(TW):
            if c in cover and c in cover_up:
                p = (cover[c], cover_up[c])
                if p != last:
                    pairs.append(p)
                last = p
            else:
                last = None
    else:
        # each run above, widened by one column on each side, meets runs below
        for ju, (su, nu) in enumerate(runs_up):
            lo, hi = su - 1, su + nu   # inclusive widened range
            for j, (s, n) in enumerate(runs):
                if s <= hi and s + n - 1 >= lo:
                    pairs.append((j, ju))
    return pairs


def model_tile_uf(mask, conn8, rng):
    """Run the kernel's union-find on one tile with random lane interleaving;
    returns ({run id: root id}, runs per row, jumping rounds)."""
    rows = [runs_of(mask[r]) for r in range(TH)]
    par = {}
    for r in range(TH):
        for j in range(len(rows[r])):
            par[r * 32 + j] = r * 32 + j
    linked = {r: [] for r in range(TH)}
    more = {r: False for r in range(TH)}
    pairs = {r: (touching_pairs(rows[r], rows[r - 1], conn8) if r > 0 else []) for r in range(TH)}
    for r in range(1, TH):
        seen = set()
        for j, ju in pairs[r]:
            if j in seen:
                more[r] = True
            else:
                seen.add(j)
                linked[r].append(j)
                par[r * 32 + j] = (r - 1) * 32 + ju
    # pointer jumping: each lane's per-run steps (load p, load pp, store) are
    # interleaved at random with the other lanes' within a round
    rounds = 0
    while True:
        rounds += 1
        assert rounds <= 40, "jumping did not settle"
        progs = []
        for r in range(TH):
            ops = []
            for j in linked[r]:
                ops.append(r * 32 + j)
            if ops:
                progs.append([r, ops, 0, None, None])   # lane, runs, next run, p, pp
        changed = False
        while progs:
            k = int(rng.integers(len(progs)))
            lane = progs[k]
            x = lane[1][lane[2]]
            if lane[3] is None:
                lane[3] = par[x]                  # load p
            elif lane[4] is None:
                lane[4] = par[lane[3]]            # load pp (may see this round's stores)
            else:
                if lane[4] != lane[3]:
                    par[x] = lane[4]              # store
                    changed = True
                lane[2] += 1
                lane[3] = lane[4] = None
                if lane[2] == len(lane[1]):
                    progs.pop(k)
        if not changed:
            break
    for x in par:                                 # every parent is now a tree root
        assert par[par[x]] == par[x]

    def find(x):
        while par[x] != x:
            x = par[x]
        return x

    # remaining pairs: union by smaller root (compare-and-min), lanes in random order
    order = [r for r in range(TH) if more[r]]
    rng.shuffle(order)
    for r in order:
        seen = set()
        for j, ju in pairs[r]:
            if j in seen:
                a, b = find(r * 32 + j), find((r - 1) * 32 + ju)
                while a != b:
                    lo_, hi_ = min(a, b), max(a, b)
                    if par[hi_] == hi_:
                        par[hi_] = lo_
                        break
                    a, b = find(hi_), lo_
            seen.add(j)
    return {x: find(x) for x in par}, rows, rounds


def check_tile(mask, conn8, rng):
    roots, rows, rounds = model_tile_uf(mask, conn8, rng)
    lab, _ = ndimage.label(mask, structure=np.ones((3, 3)) if conn8 else None)
    # same partition as the reference labelling, root = smallest run id
    comp_of_run = {}
    for r in range(TH):
        for j, (s, _) in enumerate(rows[r]):
            comp_of_run[r * 32 + j] = lab[r, s]
    by_comp = {}
    for x, c in comp_of_run.items():
        by_comp.setdefault(c, []).append(x)
    for c, xs in by_comp.items():
        assert {roots[x] for x in xs} == {min(xs)}, (c, xs[:5])
    assert len({roots[x] for x in roots}) == len(by_comp)
    return rounds


@pytest.mark.parametrize("conn8", [False, True])
def test_tile_union_find_model_matches_labels_under_random_schedules(conn8):
    rng = np.random.default_rng(7)
    fields = []
    for k in range(6):
        F = I.smoothed_noise(TH, TW, float(rng.uniform(1.0, 5.0)), seed=k)
        fields.append(F > float(rng.uniform(-0.5, 0.8)))
    fields.append(rng.random((TH, TW)) < 0.5)
    fields.append((np.indices((TH, TW)).sum(0) % 2) == 0)                  # checkerboard
    fields.append(np.tile(np.arange(TW) % 3 == 0, (TH, 1)))                  # 31-deep chains
    comb = np.zeros((TH, TW), bool)
    comb[:, ::4] = True
    comb[TH - 1, :] = True                                                   # teeth joined at the bottom only
    fields.append(comb)
    spiral = np.zeros((TH, TW), bool)
    spiral[1, 1:63] = spiral[1:31, 62] = spiral[30, 1:63] = spiral[3:31, 1] = True
    spiral[3, 1:60] = spiral[3:28, 59] = spiral[27, 4:60] = True
    fields.append(spiral)
    worst = 0
    for mask in fields:
        for _ in range(3):                                                   # three schedules each
            worst = max(worst, check_tile(mask, conn8, rng))
    assert worst <= 7   # log2(32) rounds plus the round that sees no change


def test_warp_segment_search_model():
    """The 32-ary search returns bisect's answer on tables with empty segments."""
    rng = np.random.default_rng(3)

    def warp_seg(pre, n_act, g):
        lo, n = 0, n_act + 1
        while True:
            s = (n + 31) // 32
            votes = [lane * s < n and pre[lo + lane * s] <= g for lane in range(32)]
            k = sum(votes) - 1
            assert votes == [True] * (k + 1) + [False] * (31 - k)   # a prefix of the lanes
            if s == 1:
                return lo + k
            lo += k * s
            n = min(s, n - k * s)

    for n_act in (1, 2, 31, 32, 33, 64, 100, 1023, 1024, 1025, 5000):
        sizes = rng.integers(0, 4, size=n_act)
        sizes[rng.integers(n_act)] += 1                                      # at least one item
        pre = np.concatenate([[0], np.cumsum(sizes)]).tolist()
        for g in range(pre[-1]):
            assert warp_seg(pre, n_act, g) == bisect.bisect_right(pre, g) - 1
