"""Pins of the oracle's min-sum BP (Eq. (1)-(4)) and GDG (Alg. 1-3)."""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset


def _csc(H):
    cols = [np.nonzero(H[:, i])[0] for i in range(H.shape[1])]
    ptr = np.cumsum([0] + [len(c) for c in cols]).astype(np.int32)
    rows = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return ptr, rows


def test_single_check_node_hand_computed():
    H = np.ones((1, 3), np.uint8)
    ptr, rows = _csc(H)
    llr = np.array([2.0, -1.0, 3.0], np.float32)
    for r in read_golden("single_cn_minsum.txt"):
        alpha, s = float(r[0]), int(r[1])
        want = np.array([float(x) for x in r[2:5]], np.float32)
        _, _, post = O.bp_run(1, ptr, rows, llr, np.array([s], np.uint8), alpha=alpha,
                              max_iter=1, early_stop=False)
        assert (post == want).all(), (r, post)


def _random_tree(rng, n_vn, n_cn):
    """Random bipartite tree on n_vn VNs and n_cn CNs (every node connected)."""
    nodes = [("v", i) for i in range(n_vn)] + [("c", j) for j in range(n_cn)]
    while True:
        H = np.zeros((n_cn, n_vn), np.uint8)
        order = list(rng.permutation(len(nodes)))
        placed = [nodes[order[0]]]
        ok = True
        for idx in order[1:]:
            node = nodes[idx]
            opp = [p for p in placed if p[0] != node[0]]
            if not opp:
                ok = False
                break
            p = opp[rng.integers(len(opp))]
            v, c = (node[1], p[1]) if node[0] == "v" else (p[1], node[1])
            H[c, v] = 1
            placed.append(node)
        if ok:
            return H


def _min_marginals(H, llr, s):
    n = H.shape[1]
    best = {0: np.full(n, np.inf), 1: np.full(n, np.inf)}
    for bits in itertools.product([0, 1], repeat=n):
        e = np.array(bits, np.uint8)
        if ((H.astype(np.int64) @ e) % 2 != s).any():
            continue
        cost = float(np.dot(llr.astype(np.float64), e))
        for i in range(n):
            v = bits[i]
            if cost < best[v][i]:
                best[v][i] = cost
    return best


@pytest.mark.parametrize("seed", range(12))
def test_minsum_on_trees_gives_exact_min_marginals(seed):
    """On a tree-shaped Tanner graph min-sum with alpha = 1 computes
    Lambda_i^(t) = min{PM : e_i = 1} - min{PM : e_i = 0} once t exceeds the
    diameter (brute force over all 2^n patterns)."""
    rng = np.random.default_rng(seed)
    n_vn, n_cn = int(rng.integers(6, 13)), int(rng.integers(2, 6))
    H = _random_tree(rng, n_vn, n_cn)
    llr = rng.uniform(0.5, 5.0, n_vn).astype(np.float32)
    e_true = (rng.random(n_vn) < 0.3).astype(np.uint8)
    s = ((H.astype(np.int64) @ e_true) % 2).astype(np.uint8)
    ptr, rows = _csc(H)
    _, e, post = O.bp_run(n_cn, ptr, rows, llr, s, alpha=1.0, clip=1e6, max_iter=4 * (n_vn + n_cn),
                          early_stop=False)
    mm = _min_marginals(H, llr, s)
    for i in range(n_vn):
        if np.isfinite(mm[0][i]) and np.isfinite(mm[1][i]):
            assert abs(post[i] - (mm[1][i] - mm[0][i])) < 1e-3 * (1 + abs(post[i]))
    # and the hard decision is a minimum-PM solution when it is unique
    diff = mm[1] - mm[0]
    if np.all(np.isfinite(diff)) and np.all(np.abs(diff) > 1e-3):
        assert (((H.astype(np.int64) @ e) % 2) == s).all()
        assert abs(np.dot(llr.astype(np.float64), e) - mm[0].min()) < 1e-4


def test_syndrome_sign_symmetry():
    """Eq. (1): flipping the syndrome of a check negates all of its messages,
    so on a single check the posteriors move symmetrically."""
    H = np.ones((1, 4), np.uint8)
    ptr, rows = _csc(H)
    llr = np.array([1.5, 2.5, 0.75, 4.0], np.float32)
    _, _, p0 = O.bp_run(1, ptr, rows, llr, np.array([0], np.uint8), max_iter=1, early_stop=False)
    _, _, p1 = O.bp_run(1, ptr, rows, llr, np.array([1], np.uint8), max_iter=1, early_stop=False)
    assert np.allclose((p0 - llr), -(p1 - llr))


def _loopy(rng, n, m, wc=3):
    H = np.zeros((m, n), np.uint8)
    for i in range(n):
        H[rng.choice(m, wc, replace=False), i] = 1
    return H


@pytest.mark.parametrize("seed", range(10))
def test_gdg_on_tiny_loopy_graphs(seed):
    """GDG's output, when a path converges, satisfies H e = s and its path
    metric Eq. (5) is no smaller than the brute-force minimum."""
    rng = np.random.default_rng(100 + seed)
    n, m = 14, 7
    H = _loopy(rng, n, m)
    llr = rng.uniform(1.0, 6.0, n).astype(np.float32)
    e_true = (rng.random(n) < 0.2).astype(np.uint8)
    s = ((H.astype(np.int64) @ e_true) % 2).astype(np.uint8)
    ptr, rows = _csc(H)
    P = preset("paper", k_guess=2, iters_per_step=3)
    best, e, br = O.gdg_graph(P, m, ptr, rows, llr, s)
    mm = _min_marginals(H, llr, s)
    pm_min = min(mm[0].min(), mm[1].min())
    if best >= 0:
        assert (((H.astype(np.int64) @ e) % 2) == s).all()
        pm = float(np.dot(llr.astype(np.float64), e))
        assert pm >= pm_min - 1e-9
        assert abs(br[best][3] - pm) < 1e-9
        # min over converged paths, lowest id on ties
        conv = [(b[3], i) for i, b in enumerate(br) if b[0] == 0]
        assert min(conv)[1] == best


def test_zero_syndrome_converges_at_once():
    rng = np.random.default_rng(5)
    H = _loopy(rng, 20, 10)
    ptr, rows = _csc(H)
    llr = rng.uniform(1, 6, 20).astype(np.float32)
    it, e, _ = O.bp_run(10, ptr, rows, llr, np.zeros(10, np.uint8))
    assert it == 1 and e.sum() == 0
