"""Pins of the second reading of "100 initial BP iterations": the initial BP
run as the first decimation step of GDG on the whole window (n_pre = 0, no
shortening, iters_first = 100), instead of a pre-BP whose only outputs are
the ranking and an early exit.

Every decision path starts from the priors (Sec. II-A) and decides nothing
before its first SELECT-VN, so all paths run the same first step, which is
plain min-sum BP (Eq. (1)-(4), early stop) on the window: where that BP
converges within the first step, every path converges with its estimate and
the window returns it (path 0 wins the tie of equal metrics, Alg. 2); where
it does not, path 0 runs at least the whole first step.
"""
import numpy as np

from conftest import oracle_dem
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset


def _window_synd(o, det, win):
    rows = np.arange(win["r0"] * o.w, win["r0"] * o.w + win["n_rows"])
    return ((det[rows >> 5] >> (rows & 31)) & 1).astype(np.uint8)


def test_first_step_is_plain_bp_on_the_window():
    o = oracle_dem("72", 0.003, 6)
    P1 = preset("configured", k_guess=2, n_pre=0, shorten=0, iters_first=100, d_max_main=3, d_max_other=3,
                peel_at_init=0)
    win = o.window(3, 1, 0)
    det, _ = o.sample(72_100, 0, 60)
    n_conv = n_open = 0
    for s in range(det.shape[0]):
        synd = _window_synd(o, det[s], win)
        if not synd.any():
            continue
        it, e_bp, _ = O.bp_run(win["n_rows"], win["col_ptr"], win["col_rows"], win["llr"], synd,
                               alpha=P1["alpha"], clip=P1["clip"], max_iter=100)
        corr, info, tr = o.decode_window(P1, 0, synd, trace=True)
        assert not info["prebp_converged"] and info["n_short"] == win["n_cols"]
        b0 = tr["branches"][0]
        if it > 0:  # BP converged at iteration it
            n_conv += 1
            assert info["winner"] == 0 and b0[0] == 0 and b0[1] == 1 and b0[2] == it
            assert all(b == b0 for b in tr["branches"])
            assert (corr == e_bp).all()
        else:
            n_open += 1
            assert b0[2] >= 100
    assert n_conv > 10 and n_open > 0


def test_iters_first_equal_to_iters_per_step_changes_nothing():
    o = oracle_dem("72", 0.003, 6)
    base = preset("configured", k_guess=2)
    det, obs = o.sample(72_101, 0, 24)
    f0, p0, c0 = o.run_shots(base, det, obs, want_corr=True)
    f1, p1, c1 = o.run_shots(dict(base, iters_first=base["iters_per_step"]), det, obs, want_corr=True)
    assert (f0 == f1).all() and (p0 == p1).all() and (c0 == c1).all()
