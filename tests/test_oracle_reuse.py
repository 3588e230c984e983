"""Pins of the message reuse between windows (Sec. VI names it as future
work: reuse the BP messages of the branch with the minimum path metric to
initialise the next window).  The oracle's reading: the next window's pre-BP
starts the first VN->CN messages of a shared column from the output path's
final posterior (+-clip for a column it decimated), other columns from the
prior.
"""
import numpy as np

from conftest import oracle_dem
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset


def _synd(o, det_row, win):
    rows = np.arange(win["r0"] * o.w, win["r0"] * o.w + win["n_rows"])
    return ((det_row[rows >> 5] >> (rows & 31)) & 1).astype(np.uint8)


def test_kept_values():
    """What a window keeps: the pre-BP's own posterior when it converges (the
    posteriors of plain min-sum BP on the window, run independently here);
    otherwise the output path's posterior on the columns GDG held, +-clip
    where it decimated, consistent with the correction (Eq. (4)), and
    nothing elsewhere."""
    o = oracle_dem("72", 0.003, 6)
    P = preset("configured", k_guess=3, reuse_msgs=1)
    win = o.window(3, 1, 1)
    det, _ = o.sample(72_300, 0, 60)
    seen = {True: 0, False: 0}
    for s in range(det.shape[0]):
        synd = _synd(o, det[s], win)
        corr, info, keep = o.decode_window_reuse(P, 1, synd)
        seen[info["prebp_converged"]] += 1
        if info["prebp_converged"]:
            it, e, post = O.bp_run(win["n_rows"], win["col_ptr"], win["col_rows"], win["llr"], synd,
                                   alpha=P["alpha"], clip=P["clip"], max_iter=P["n_pre"])
            assert it > 0 and (keep == post).all() and (e == corr).all()
        else:
            held = ~np.isnan(keep)
            assert held.sum() == info["n_short"]
            assert ((keep[held] <= 0) == (corr[held] == 1)).all()
            assert not corr[~held].any()
            big = np.abs(keep[held]) == P["clip"]
            assert big.any()
    assert seen[True] > 0 and seen[False] > 0


def test_priors_as_kept_values_change_nothing():
    """Starting every message from the prior, given explicitly, is the plain
    pre-BP (Sec. II-A initialisation)."""
    o = oracle_dem("72", 0.003, 6)
    P = preset("configured", k_guess=3)
    win = o.window(3, 1, 2)
    det, _ = o.sample(72_301, 0, 40)
    for s in range(det.shape[0]):
        synd = _synd(o, det[s], win)
        c0, i0, k0 = o.decode_window_reuse(P, 2, synd)
        c1, i1, k1 = o.decode_window_reuse(P, 2, synd, init=win["llr"].copy())
        c2, i2, k2 = o.decode_window_reuse(P, 2, synd, init=np.full(win["n_cols"], np.nan, np.float32))
        assert (c0 == c1).all() and (c0 == c2).all() and i0 == i1 == i2
        assert np.array_equal(k0, k1, equal_nan=True) and np.array_equal(k0, k2, equal_nan=True)


def test_reuse_runs_whole_experiments():
    o = oracle_dem("72", 0.003, 6)
    det, obs = o.sample(72_302, 0, 64)
    f0, p0, c0 = o.run_shots(preset("configured", k_guess=3), det, obs, threads=8, want_corr=True)
    f1, p1, c1 = o.run_shots(preset("configured", k_guess=3, reuse_msgs=1), det, obs, threads=8, want_corr=True)
    assert (c0[:, 0] == c1[:, 0]).all()  # the first window has nothing to reuse
    assert (c0 != c1).any()              # later windows start differently
    zero = np.zeros_like(det)
    fz, pz, _ = o.run_shots(preset("configured", k_guess=3, reuse_msgs=1), zero, np.zeros_like(obs))
    assert not fz.any() and not pz.any()
