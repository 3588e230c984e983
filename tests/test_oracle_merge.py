"""Pins of the H_1 merge of Sec. III in the oracle's windows.

H_1 = the window columns that reach past the window's last block, seen on
the window's rows.  merge_h1 = 1 merges the H_1 columns with equal
restrictions (the window's parity-check problem keeps the same distinct
columns); merge_h1 = 2 replaces H_1 by one column per detector of the last
block (an identity matrix).  A merged column's probability is that of an odd
number of its independent members firing, pinned here by enumerating every
subset of the members.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import oracle_dem
from paper_2403_18901_gb300.workloads import preset


def _cols(win):
    return [tuple(win["col_rows"][win["col_ptr"][c]:win["col_ptr"][c + 1]]) for c in range(win["n_cols"])]


def _odd_probability(ps):
    """P(an odd number fire) by enumerating all subsets (independent events)."""
    tot = 0.0
    for bits in itertools.product((0, 1), repeat=len(ps)):
        if sum(bits) % 2:
            tot += math.prod(p if b else 1.0 - p for p, b in zip(ps, bits))
    return tot


def _llr32(p):
    return np.float32(math.log((1.0 - p) / p))


def _h1(o, win):
    hi = (win["r0"] + win["n_blocks"]) * o.w
    return [c for c in range(win["n_cols"])
            if o.col_dets[o.col_ptr[win["gcols"][c] + 1] - 1] >= hi]


@pytest.mark.parametrize("k", [0, 1, 5])
def test_equal_restrictions_merge(k):
    o = oracle_dem("144", 0.003, 12)
    base = o.window(3, 1, k)
    m = o.window(3, 1, k, merge=1)
    h1 = _h1(o, base)
    cb, cm = _cols(base), _cols(m)
    # the committed prefix and every column outside H_1 are untouched
    nonh1 = [c for c in range(base["n_cols"]) if c not in set(h1)]
    assert m["n_commit"] == base["n_commit"] and (m["commit"][:m["n_commit"]] == 1).all()
    keep = [c for c in range(m["n_cols"]) if m["gcols"][c] in set(base["gcols"][nonh1])]
    assert [cm[c] for c in keep] == [cb[c] for c in nonh1]
    assert (m["llr"][keep] == base["llr"][nonh1]).all()
    # the distinct columns of the window are the same set; H_1's equal
    # restrictions collapse (504 -> 288 for [[144]]: 72 of weight one = I_w)
    assert set(cm) == set(cb) and len(set(cb)) == len(cm)
    classes = {}
    for c in h1:
        classes.setdefault(cb[c], []).append(c)
    assert len(h1) == 7 * o.w and len(classes) == 4 * o.w
    w1 = [r for r in classes if len(r) == 1]
    last0 = (base["n_blocks"] - 1) * o.w
    assert sorted(r[0] for r in w1) == list(range(last0, last0 + o.w))
    # each merged column: the class's first member's place, odd-count probability
    for rows, members in classes.items():
        c = cm.index(rows)
        assert m["gcols"][c] == base["gcols"][members[0]]
        want = _odd_probability([o.col_p[base["gcols"][x]] for x in members])
        got = m["llr"][c]
        assert abs(int(got.view(np.int32)) - int(_llr32(want).view(np.int32))) <= 1, (rows, got, want)


def test_identity_merge():
    o = oracle_dem("144", 0.003, 12)
    base = o.window(3, 1, 2)
    m = o.window(3, 1, 2, merge=2)
    h1 = _h1(o, base)
    last0 = (base["n_blocks"] - 1) * o.w
    cb, cm = _cols(base), _cols(m)
    assert m["n_cols"] == base["n_cols"] - len(h1) + o.w
    ident = cm[-o.w:]
    assert ident == [(last0 + t,) for t in range(o.w)]
    for t in range(o.w):
        members = [c for c in h1 if last0 + t in cb[c]]
        want = _odd_probability([o.col_p[base["gcols"][x]] for x in members])
        got = m["llr"][m["n_cols"] - o.w + t]
        assert abs(int(got.view(np.int32)) - int(_llr32(want).view(np.int32))) <= 1


def test_last_window_and_w_equal_f_unchanged():
    o = oracle_dem("72", 0.003, 6)
    nwin = o.n_windows(3, 1)
    a, b = o.window(3, 1, nwin - 1), o.window(3, 1, nwin - 1, merge=1)
    assert (a["gcols"] == b["gcols"]).all() and (a["llr"] == b["llr"]).all()
    a, b = o.window(2, 2, 0), o.window(2, 2, 0, merge=2)
    assert (a["gcols"] == b["gcols"]).all()


@pytest.mark.parametrize("merge", [1, 2])
def test_merged_windows_decode(merge):
    """Whole memory experiments run with either merge; the exact merge keeps
    the equation every window solves, so every residue-free shot stays
    residue free with it on a zero-noise syndrome."""
    o = oracle_dem("72", 0.003, 6)
    params = preset("configured", k_guess=3, merge_h1=merge)
    det, obs = o.sample(72_510, 0, 40)
    fail, pred, _ = o.run_shots(params, det, obs, threads=8)
    assert fail.shape == (40,) and (fail <= 3).all()
    zero = np.zeros_like(det)
    f0, p0, _ = o.run_shots(params, zero, np.zeros_like(obs))
    assert not f0.any() and not p0.any()
