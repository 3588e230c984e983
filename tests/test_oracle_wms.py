"""Pins of the oracle's learned weighted min-sum reference (FP64): its
gradient against central finite differences at generic points, and the
model with every weight equal to alpha against the plain min-sum of the C
oracle (Eq. (1)-(3))."""
import numpy as np
import pytest

from conftest import oracle_dem
from oracle import oracle as O
from oracle import wms_ref


def _loopy(rng, n, m, wc=3):
    H = np.zeros((m, n), np.uint8)
    for i in range(n):
        H[rng.choice(m, wc, replace=False), i] = 1
    cols = [np.nonzero(H[:, i])[0] for i in range(n)]
    ptr = np.cumsum([0] + [len(c) for c in cols])
    return H, ptr, np.concatenate(cols)


@pytest.mark.parametrize("seed", range(4))
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    n, m, T = 16, 8, 5
    H, ptr, rows = _loopy(rng, n, m)
    llr = rng.uniform(1.0, 6.0, n)
    e = (rng.random(n) < 0.2).astype(np.int64)
    s = (H.astype(np.int64) @ e) % 2
    if not s.any():
        s[0] = 1
    g = wms_ref.Graph(m, ptr, rows, llr)
    w = rng.uniform(0.5, 1.2, size=(T, g.ne))
    L, gw = wms_ref.loss_and_grad(g, w, s)
    assert abs(L - wms_ref.forward(g, w, s)) < 1e-12
    h = 1e-6
    idx = [(t, k) for t in range(T) for k in range(g.ne)]
    pick = rng.choice(len(idx), 30, replace=False)
    for q in pick:
        t, k = idx[q]
        wp, wm = w.copy(), w.copy()
        wp[t, k] += h
        wm[t, k] -= h
        fd = (wms_ref.forward(g, wp, s) - wms_ref.forward(g, wm, s)) / (2 * h)
        assert abs(fd - gw[t, k]) <= 1e-6 + 1e-4 * abs(fd), (t, k, fd, gw[t, k])


def test_alpha_weights_reduce_to_plain_minsum():
    d = oracle_dem("72", 0.003, 6)
    win = d.window(3, 1, 1)
    det, _ = d.sample(5, 0, 3)
    idx = np.arange(d.n_det)
    bits = ((det[:, idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)
    g = wms_ref.Graph(win["n_rows"], win["col_ptr"], win["col_rows"], win["llr"])
    T, alpha = 6, 0.625
    for sh in range(3):
        s = bits[sh, win["r0"] * d.w: win["r0"] * d.w + win["n_rows"]]
        post64 = wms_ref.posteriors(g, np.full((T, g.ne), alpha), s)
        _, _, post32 = O.bp_run(win["n_rows"], win["col_ptr"], win["col_rows"], win["llr"], s,
                                alpha=alpha, max_iter=T, early_stop=False)
        assert np.allclose(post64, post32, rtol=1e-5, atol=1e-4)
