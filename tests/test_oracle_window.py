"""Pins of the oracle's sampler, sliding-window driver (Sec. III, Eq. (8)-(12))
and decision tree (Alg. 2, Fig. 2)."""
import math

import numpy as np
import pytest

from conftest import oracle_dem, read_golden
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset


def test_philox_known_answers():
    for r in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def _bits(det, n_det):
    idx = np.arange(n_det)
    return ((det[:, idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)


def test_sampler_detector_marginals_closed_form():
    """A detector is the XOR of independent column flips, so
    P(det_j = 1) = (1 - prod_{c ni j} (1 - 2 p_c)) / 2."""
    dem = oracle_dem("72", 0.003, 6)
    n = 40000
    det, obs = dem.sample(seed=7, shot_offset=0, n_shots=n)
    emp = _bits(det, dem.n_det).mean(0)
    prod = np.ones(dem.n_det)
    for c in range(dem.n_cols):
        for d in dem.col_dets[dem.col_ptr[c]:dem.col_ptr[c + 1]]:
            prod[d] *= 1 - 2 * dem.col_p[c]
    want = (1 - prod) / 2
    sd = np.sqrt(want * (1 - want) / n)
    assert np.all(np.abs(emp - want) < 5 * sd + 1e-4)
    # shots are a function of (seed, global shot index): offsets compose
    d2, o2 = dem.sample(seed=7, shot_offset=100, n_shots=50)
    assert (d2 == det[100:150]).all() and (o2 == obs[100:150]).all()


@pytest.mark.parametrize("key,R,W,F", [("72", 6, 3, 1), ("144", 12, 3, 1), ("72", 6, 4, 2),
                                       ("72", 6, 7, 1)])
def test_windows_partition_the_columns(key, R, W, F):
    """Each detector-bearing column is committed by exactly one window, and a
    window's columns are the un-committed ones touching its rows (Eq. (8))."""
    dem = oracle_dem(key, 0.003, R)
    w = dem.w
    nw = dem.n_windows(W, F)
    B = R + 1
    assert nw == (1 if W >= B else math.ceil((B - W) / F) + 1)
    committed = np.zeros(dem.n_cols, np.int32)
    for k in range(nw):
        win = dem.window(W, F, k)
        r0, nb = win["r0"], win["n_blocks"]
        assert win["n_rows"] == nb * w
        for i, c in enumerate(win["gcols"]):
            dets = dem.col_dets[dem.col_ptr[c]:dem.col_ptr[c + 1]]
            assert r0 * w <= dets[0] < (r0 + nb) * w
            assert committed[c] == 0
            if win["commit"][i]:
                committed[c] += 1
    assert (committed == 1).all()
    if (key, W) == ("144", 3):
        # first window 29w columns (H0' is 2w), later ones 30w
        assert dem.window(W, F, 0)["n_cols"] == 29 * w
        assert dem.window(W, F, 1)["n_cols"] == 30 * w


def _global_correction(dem, P, corr_words):
    nw = dem.n_windows(P["W"], P["F"])
    e = np.zeros(dem.n_cols, np.uint8)
    for k in range(nw):
        win = dem.window(P["W"], P["F"], k)
        for i, c in enumerate(win["gcols"]):
            if win["commit"][i] and (corr_words[k, i >> 5] >> np.uint32(i & 31)) & 1:
                e[c] = 1
    return e


@pytest.mark.parametrize("preset_name", ["paper", "configured"])
def test_commit_residue_iff_global_equation(preset_name):
    """All partial equations Eq. (9) hold iff the overall equation Eq. (10)
    holds; the observable prediction is L e (Eq. (12))."""
    dem = oracle_dem("72", 0.003, 6)
    P = preset(preset_name, k_guess=3)
    det, obs = dem.sample(seed=11, shot_offset=0, n_shots=120)
    fail, pred, corr = dem.run_shots(P, det, obs, threads=O.default_threads(), want_corr=True)
    s = _bits(det, dem.n_det)
    for sh in range(len(fail)):
        e = _global_correction(dem, P, corr[sh])
        synd = np.zeros(dem.n_det, np.uint8)
        om = 0
        for c in np.nonzero(e)[0]:
            synd[dem.col_dets[dem.col_ptr[c]:dem.col_ptr[c + 1]]] ^= 1
            om ^= int(dem.col_obs[c])
        residue_ok = (synd == s[sh]).all()
        assert residue_ok == (not (fail[sh] & 1))
        assert om == pred[sh]
        assert bool(fail[sh] & 2) == (om != obs[sh])


def test_zero_syndrome_window():
    dem = oracle_dem("72", 0.003, 6)
    P = preset("configured", k_guess=3)
    win = dem.window(3, 1, 1)
    corr, info, _ = dem.decode_window(P, 1, np.zeros(win["n_rows"], np.uint8))
    assert info["prebp_converged"] and info["prebp_iters"] == 1 and corr.sum() == 0


def _gdg_window(dem, P, seed, want_depth):
    det, _ = dem.sample(seed=seed, shot_offset=0, n_shots=200)
    s = _bits(det, dem.n_det)
    win = dem.window(P["W"], P["F"], 1)
    r0 = win["r0"] * dem.w
    for sh in range(200):
        corr, info, tr = dem.decode_window(P, 1, s[sh, r0:r0 + win["n_rows"]], trace=True)
        if info["prebp_converged"]:
            continue
        br = tr["branches"]
        if all(b[1] >= want_depth for b in br):
            return tr
    return None


def test_decision_tree_msb_first():
    """Alg. 2 line "b = the D-th bit of id": read most significant first, id 1
    is contrary to the favoured value only at depth k (the first side branch
    of Fig. 2), id 2^(k-1) only at depth 1."""
    dem = oracle_dem("72", 0.003, 6)
    k = 3
    P = preset("configured", k_guess=k)
    tr = _gdg_window(dem, P, seed=3, want_depth=k + 1)
    assert tr is not None
    st = tr["steps"]
    # ids 0 and 1: same decisions before depth k, same VN at depth k, opposite values
    for D in range(1, k):
        assert st[0][D - 1] == st[1][D - 1]
    assert st[0][k - 1][0] == st[1][k - 1][0]
    assert st[0][k - 1][1] == 1 - st[1][k - 1][1]
    # id 2^(k-1) differs from id 0 already at depth 1
    h = 1 << (k - 1)
    assert st[0][0][0] == st[h][0][0] and st[0][0][1] == 1 - st[h][0][1]


def _wilson_hi(k, n, z=1.96):
    ph = k / n
    return (ph + z * z / (2 * n) + z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n))) / (1 + z * z / n)


def test_main_branch_error_suppression():
    """Sec. IV-B: the main branch alone, limited to 25 steps, as the inner
    window decoder for N = 144 gives a logical error rate per round below the
    physical rate.  p = 0.002 (low-error mode, Fig. 3 caption), R = 12,
    paper preset, k = 0; per-round rate p_L = 1 - (1 - P_L)^(1/R)
    (appendix "Stim circuit implementation"), 95% Wilson upper bound."""
    dem = oracle_dem("144", 0.002, 12)
    P = preset("paper", k_guess=0, p=0.002, side_max=0)  # the main branch alone
    n = 1500
    det, obs = dem.sample(seed=144_002, shot_offset=0, n_shots=n)
    fail, _, _ = dem.run_shots(P, det, obs, threads=O.default_threads())
    k = int((fail > 0).sum())
    p_round_hi = 1 - (1 - _wilson_hi(k, n)) ** (1 / 12)
    assert p_round_hi < 0.002, (k, n, p_round_hi)


def test_guessing_tree_beats_main_branch():
    """Sec. IV-B: the guessing tree improves on the main branch alone."""
    dem = oracle_dem("144", 0.003, 12)
    n = 600
    det, obs = dem.sample(seed=144_003, shot_offset=0, n_shots=n)
    f0, _, _ = dem.run_shots(preset("paper", k_guess=0, side_max=0), det, obs, threads=O.default_threads())
    f4, _, _ = dem.run_shots(preset("paper", k_guess=4), det, obs, threads=O.default_threads())
    assert int((f4 > 0).sum()) < int((f0 > 0).sum())
