"""Pins of the oracle's full decision tree of Fig. 2 (main branch, 2^k
guessing tree, side branches split off the main branch at D_split = k ..
side_max, Alg. 2).

* Path counts and depth limits: the caption of Fig. 2 and the thread counts of
  the appendix (15 threads = 1 main + 14 tree branches two per thread + 7 side
  branches for N <= 144; 32 threads = 1 + 30/2 + 16 for N = 288).
* A side branch repeats the main branch decision for decision until its split
  depth, where it selects the same VN and takes the other value (Alg. 2: only
  D = D_split is contrary), and stops D_split + 10 steps deep at most.
* Adding side branches leaves the main branch and the tree branches 2..2^k-1
  unchanged.
"""
import ctypes as C

import numpy as np
import pytest

from conftest import oracle_dem
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset


def _paths(params):
    P = O.make_params(params)
    return O.lib().qdo_n_paths(C.byref(P)), O.lib().qdo_path_dmax_all(C.byref(P))


def test_path_counts_match_the_papers_thread_counts():
    p144 = preset("paper", k_guess=4)
    nb, dmx = _paths(p144)
    # 1 main + 14 tree + 7 side (D_split 4..10; D_split 4 is id 1)
    assert nb == 22 and dmx == 25
    threads = 1 + (nb - 1 - 7) // 2 + 7
    assert threads == 15
    p288 = preset("paper", 5, d_max_main=40, d_max_other=25, side_max=20, n_pre=16)
    nb, dmx = _paths(p288)
    assert nb == 47 and dmx == 40  # 1 + 30 + 16; side D_max up to 20 + 20
    assert 1 + (nb - 1 - 16) // 2 + 16 == 32
    assert _paths(preset("configured", k_guess=4)) == (16, 25)  # the configured 2^k tree


def _window_syndromes(o, params, k, n, seed):
    win = o.window(params["W"], params["F"], k)
    det, _ = o.sample(seed, 0, n)
    idx = np.arange(o.n_det)
    bits = ((det[:, idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)
    r0 = win["r0"] * o.w
    return [bits[s, r0:r0 + win["n_rows"]] for s in range(n)]


@pytest.mark.parametrize("key,R,k,p", [("72", 6, 3, 0.004), ("144", 12, 4, 0.004)])
def test_side_branches_follow_the_main_branch_until_their_split(key, R, k, p):
    o = oracle_dem(key, p, R)
    params = preset("paper", k_guess=k, p=p)
    plain = dict(params, side_max=0)
    nt = 1 << k
    extra = params["d_max_other"] - k
    seen_split = 0
    for s in _window_syndromes(o, params, 1, 40, seed=777 + k):
        _, info, tr = o.decode_window(params, 1, s, trace=True)
        if info["prebp_converged"]:
            continue
        _, info0, tr0 = o.decode_window(plain, 1, s, trace=True)
        assert (tr["short_cols"] == tr0["short_cols"]).all()
        main = tr["steps"][0]
        # the main branch and tree branches 2..2^k-1 are unchanged by the side branches
        for b in [0] + list(range(2, nt)):
            assert tr["branches"][b] == tr0["branches"][b]
            assert tr["steps"][b] == tr0["steps"][b]
        sides = [(1, k)] + [(nt + i, k + 1 + i) for i in range(params["side_max"] - k)]
        assert len(tr["branches"]) == nt + params["side_max"] - k
        for b, split in sides:
            st = tr["steps"][b]
            depth = tr["branches"][b][1]
            assert depth <= split + extra
            m_depth = tr["branches"][0][1]
            for D in range(1, min(split, depth + 1)):
                assert st[D - 1] == main[D - 1], (b, D)
            if depth >= split and main[split - 1][0] >= 0 and st[split - 1][0] >= 0:
                assert st[split - 1][0] == main[split - 1][0]        # same VN
                assert st[split - 1][1] == 1 - main[split - 1][1]    # the other value
                seen_split += 1
            if m_depth < split:  # the main branch ended first: the side branch is the main branch
                assert tr["branches"][b] == tr["branches"][0]
    assert seen_split > 0, "no side branch reached its split; pick another seed"


@pytest.mark.parametrize("key,R,k,p", [("72", 6, 3, 0.004), ("144", 12, 4, 0.004)])
def test_message_restart_at_splits(key, R, k, p):
    """reinit_on_split (the appendix's snapshot implementation): only the
    paths that continue from another path's status -- side branches at their
    split, odd tree ids at D = k -- change, and only after that decimation."""
    o = oracle_dem(key, p, R)
    params = preset("paper", k_guess=k, p=p)
    re_params = dict(params, reinit_on_split=1)
    nt = 1 << k
    restarts = {1: k}
    restarts.update({nt + i: k + 1 + i for i in range(params["side_max"] - k)})
    restarts.update({b: k for b in range(3, nt, 2)})
    changed = 0
    for s in _window_syndromes(o, params, 1, 40, seed=991 + k):
        _, info, tr = o.decode_window(params, 1, s, trace=True)
        if info["prebp_converged"]:
            continue
        _, _, tr1 = o.decode_window(re_params, 1, s, trace=True)
        for b in range(len(tr["branches"])):
            if b not in restarts:
                assert tr1["branches"][b] == tr["branches"][b] and tr1["steps"][b] == tr["steps"][b], b
                continue
            D = restarts[b]
            assert tr1["steps"][b][:D] == tr["steps"][b][:D], b  # identical through the split decimation
            changed += tr1["steps"][b][D:] != tr["steps"][b][D:]
    assert changed > 0, "no restart changed a path; pick another seed"


def test_message_restart_without_splits_changes_nothing():
    o = oracle_dem("72", 0.004, 6)
    params = preset("paper", k_guess=0, p=0.004, side_max=0)
    for s in _window_syndromes(o, params, 1, 10, seed=5):
        a = o.decode_window(params, 1, s, trace=True)
        b = o.decode_window(dict(params, reinit_on_split=1), 1, s, trace=True)
        assert (a[0] == b[0]).all() and a[2]["branches"] == b[2]["branches"]
