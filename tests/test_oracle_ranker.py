"""Pins of the oracle's decimation ranker (no counterpart in the paper; it
replaces the argmin of Alg. 1): closed-form scores of hand-built networks,
the parameter grids, an independent FP64 model (and its gradient against
finite differences), and the candidate records the oracle writes at each
selection step checked against the window matrix and the decision trace."""
import numpy as np
import pytest

from conftest import oracle_dem
from oracle import oracle as O
from oracle import ranker_ref
from paper_2403_18901_gb300.workloads import preset


def _params(W1=None, b1=None, W2=None, b2=0.0):
    p = np.zeros(641, np.float32)
    if W1 is not None:
        p[:512] = np.asarray(W1, np.float32).reshape(-1)
    if b1 is not None:
        p[512:576] = b1
    if W2 is not None:
        p[576:640] = W2
    p[640] = b2
    return p


def _grid_x(rng, n):
    x = np.zeros((n, 8), np.float32)
    x[:, :5] = rng.integers(-127, 128, (n, 5)) * 0.5
    x[:, 5] = rng.integers(0, 128, n)
    x[:, 6] = rng.integers(1, 12, n)
    x[:, 7] = rng.integers(0, 4, n)
    return x


def test_closed_form_scores():
    rng = np.random.default_rng(3)
    x = _grid_x(rng, 200)
    # constant network: the score is b2 as given (b2 is not rounded)
    s = O.ranker_score(_params(b2=0.3), x)
    assert (s == np.float32(0.3)).all()
    # units 0..7 copy relu(x_k), units 8..15 relu(-x_k): sum of relu = sum relu(x)
    W1 = np.zeros((64, 8))
    W1[np.arange(8), np.arange(8)] = 1.0
    W1[8 + np.arange(8), np.arange(8)] = -1.0
    W2 = np.zeros(64)
    W2[:8] = 1.0
    assert (O.ranker_score(_params(W1, None, W2), x) == np.maximum(x, 0).sum(1)).all()
    W2[8:16] = -1.0  # relu(x) - relu(-x) = x
    assert (O.ranker_score(_params(W1, None, W2), x) == x.sum(1)).all()
    # a negative pre-activation and an exact zero give h = 0
    W1b = np.zeros((64, 8))
    W1b[0, 0] = 1.0
    W2b = np.zeros(64)
    W2b[0] = 1.0
    xz = np.zeros((3, 8), np.float32)
    xz[:, 0] = [-3.0, 0.0, 2.5]
    assert list(O.ranker_score(_params(W1b, None, W2b), xz)) == [0.0, 0.0, 2.5]


@pytest.mark.parametrize("raw,expect", [
    (2.0 ** -7, 0.0),             # half a grid step rounds to even (0)
    (3 * 2.0 ** -7, 2.0 ** -5),   # 1.5 steps round to even (2 steps)
    (5.0, 2.0), (-7.0, -2.0),     # clamped to [-2, 2]
    (0.40, 26 / 64),              # 25.6 steps -> 26
])
def test_weight_grid(raw, expect):
    W1 = np.zeros((64, 8))
    W1[0, 0] = raw
    W2 = np.zeros(64)
    W2[0] = 1.0
    x = np.zeros((1, 8), np.float32)
    x[0, 0] = 1.0
    assert O.ranker_score(_params(W1, None, W2), x)[0] == np.float32(max(expect, 0.0))
    # the same rounding on the second layer
    W1[0, 0] = 1.0
    W2[0] = raw
    assert O.ranker_score(_params(W1, None, W2), x)[0] == np.float32(expect)


def test_bias_grid():
    W2 = np.zeros(64)
    W2[0] = 1.0
    x = np.zeros((1, 8), np.float32)
    for raw, expect in [(2.0 ** -8, 0.0), (3 * 2.0 ** -8, 2.0 ** -6), (300.0, 300.0), (1000.0, 512.0)]:
        b1 = np.zeros(64)
        b1[0] = raw
        assert O.ranker_score(_params(None, b1, W2), x)[0] == np.float32(expect)


def test_fp64_model_matches_oracle_scores():
    rng = np.random.default_rng(11)
    for _ in range(5):
        p = rng.normal(0, 0.7, 641).astype(np.float32)
        p[512:576] = rng.normal(0, 3, 64)
        x = _grid_x(rng, 500)
        s32 = O.ranker_score(p, x).astype(np.float64)
        s64 = ranker_ref.forward(p, x, quant=True)
        assert np.allclose(s32, s64, rtol=1e-5, atol=1e-4 * np.abs(s64).max())


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 0.5, 641)
    x = rng.normal(0, 2.0, (64, 8))
    y = (rng.random(64) < 0.3).astype(np.float64)
    g, _ = ranker_ref.grad(p, x, y, pos_weight=3.0)
    h = 1e-6
    for i in rng.choice(641, 80, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (ranker_ref.loss(pp, x, y, 3.0).sum() - ranker_ref.loss(pm, x, y, 3.0).sum()) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


# ---- candidate records of the decoder ----
def _window_samples(o, params, k, n, seed):
    win = o.window(params["W"], params["F"], k)
    rng = np.random.default_rng(seed)
    p = o.col_p[win["gcols"]]
    out = []
    for _ in range(n):
        e = (rng.random(win["n_cols"]) < p).astype(np.uint8)
        s = np.zeros(win["n_rows"], np.uint8)
        for c in np.nonzero(e)[0]:
            s[win["col_rows"][win["col_ptr"][c]:win["col_ptr"][c + 1]]] ^= 1
        out.append((e, s))
    return win, out


def _gdg_windows(ranker=None, n=40, want=6):
    o = oracle_dem("72", 0.003, 6)
    params = preset("configured", k_guess=3, p=0.003)
    win, samples = _window_samples(o, params, 1, n, seed=17)
    res = []
    for e, s in samples:
        dump = np.zeros(20000, O.RANK_REC)
        _, info, tr = o.decode_window(params, 1, s, trace=True, ranker=ranker, dump=dump)
        if info["prebp_converged"]:
            continue
        assert info["n_dump"] <= dump.shape[0]
        res.append((e, s, info, tr, dump[:info["n_dump"]]))
        if len(res) == want:
            break
    assert res, "no window reached GDG"
    return o, params, win, res


def _groups(recs):
    out = {}
    for i, d in enumerate(recs["depth"]):
        out.setdefault(int(d), []).append(i)
    return out


def test_records_match_window_and_trace():
    o, params, win, res = _gdg_windows()
    deg = np.diff(win["col_ptr"])
    rpb = win["n_rows"] // win["n_blocks"]
    for e, s, info, tr, recs in res:
        assert (recs["path"] == 0).all()
        x = recs["x"]
        w = recs["wcol"]
        assert (x[:, 6] == deg[w]).all() and (x[:, 6] >= 3).all()
        first = win["col_rows"][win["col_ptr"][w]]
        assert (x[:, 7] == np.minimum(first // rpb, 255)).all()
        assert (x[:, 5] == np.round(x[:, 5])).all() and (x[:, 5] <= x[:, 6]).all() and (x[:, 5] >= 0).all()
        # L/4 and the mean of the four posteriors agree up to the two roundings
        assert (np.abs(x[:, 0] - x[:, 1:5].mean(1)) <= 0.5 + 1e-6).all()
        # L <= -1 forces f = 1 and L >= 1 forces f = 0
        f = recs["flags"] & 1
        assert (f[x[:, 0] <= -0.5] == 1).all() and (f[x[:, 0] >= 0.5] == 0).all()
        steps = tr["steps"][0]
        for D, idx in _groups(recs).items():
            assert len(set(w[idx])) == len(idx)
            sel = [i for i in idx if recs["flags"][i] & 2]
            assert len(sel) == 1
            g, value = steps[D - 1][0], steps[D - 1][1]
            assert tr["short_cols"][g] == w[sel[0]]
            assert value == (recs["flags"][sel[0]] & 1)  # path 0 keeps f


def _sel_per_group(recs):
    return {D: [i for i in idx if recs["flags"][i] & 2][0] for D, idx in _groups(recs).items()}


def test_constant_ranker_selects_lowest_column():
    _, _, _, res = _gdg_windows(ranker=_params(b2=1.0))
    for *_, recs in res:
        for D, idx in _groups(recs).items():
            assert _sel_per_group(recs)[D] == idx[0]  # records come in short-column order


def test_degree_ranker_selects_first_highest_degree():
    W1 = np.zeros((64, 8))
    W1[0, 6] = 1.0
    W2 = np.zeros(64)
    W2[0] = 1.0
    _, _, _, res = _gdg_windows(ranker=_params(W1, None, W2))
    for *_, recs in res:
        for D, idx in _groups(recs).items():
            d = recs["x"][idx, 6]
            assert _sel_per_group(recs)[D] == idx[int(np.argmax(d))]


def test_history_ranker_selects_first_smallest_sum():
    # score = relu(-x0) - relu(x0) = -x0: the smallest L/4 on the 1/2 grid
    W1 = np.zeros((64, 8))
    W1[0, 0], W1[1, 0] = -1.0, 1.0
    W2 = np.zeros(64)
    W2[0], W2[1] = 1.0, -1.0
    _, _, _, res = _gdg_windows(ranker=_params(W1, None, W2))
    for *_, recs in res:
        for D, idx in _groups(recs).items():
            assert _sel_per_group(recs)[D] == idx[int(np.argmin(recs["x"][idx, 0]))]
