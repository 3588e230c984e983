"""Pins of the oracle's BB code construction (appendix "Single shot syndrome
noise" worked example, code parameters of Fig. 3)."""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from gf2 import nullspace, rank
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import CODES


def _golden288():
    g = {r[0]: [int(x) for x in r[1:]] for r in read_golden("bb288_syndrome_code.txt")}
    return g


def test_first_columns_match_worked_example():
    g = _golden288()
    HX, _ = O.code_matrices(CODES["288"])
    w = 144
    A, B = HX[:, :w], HX[:, w:]
    assert sorted(np.nonzero(A[:, 0])[0].tolist()) == sorted(g["b1"])
    assert sorted(np.nonzero(B[:, 0])[0].tolist()) == sorted(g["b2"])


@pytest.mark.parametrize("key", ["72", "90", "108", "144", "288"])
def test_css_commutation_and_k(key):
    nk = {r[0]: (int(r[1]), int(r[2])) for r in read_golden("codes_nk.txt")}
    HX, HZ = O.code_matrices(CODES[key])
    n, k = nk[key]
    assert HX.shape == (n // 2, n)
    assert not ((HX.astype(np.int64) @ HZ.T.astype(np.int64)) % 2).any()
    # independent rank (tests/gf2.py), not the oracle's routine
    assert n - rank(HX) - rank(HZ) == k
    assert O.gf2_rank(HX) == rank(HX)
    # every column weight 3, every row weight 6
    assert (HX.sum(0) == 3).all() and (HX.sum(1) == 6).all()
    assert (HZ.sum(0) == 3).all() and (HZ.sum(1) == 6).all()


@pytest.mark.parametrize("key", ["72", "144", "288"])
def test_logical_z_basis(key):
    HX, HZ = O.code_matrices(CODES[key])
    LZ = O.logical_z(CODES[key])
    assert LZ.shape[0] == CODES[key]["k"]
    assert not ((HX.astype(np.int64) @ LZ.T.astype(np.int64)) % 2).any()
    assert rank(np.vstack([HZ, LZ])) == rank(HZ) + LZ.shape[0]


def _pair_count_in_span(M):
    """Number of weight-2 vectors in the column span of M: e_i + e_j lies in it
    iff columns i and j of a parity check of the span coincide."""
    K = nullspace(M.T)  # rows y with y^T M = 0
    cols = [tuple(K[:, i]) for i in range(M.shape[0])]
    from collections import Counter
    c = Counter(cols)
    return sum(v * (v - 1) // 2 for v in c.values()), cols


def test_216_weight_two_syndrome_codewords():
    g = _golden288()
    HX, _ = O.code_matrices(CODES["288"])
    n2, cols = _pair_count_in_span(HX)
    assert n2 == g["weight2_codewords"][0]
    # distance of the syndrome code of H_X is 2, of A and of B alone 3
    w = 144
    for M, key in [(HX[:, :w], "dist_A"), (HX[:, w:], "dist_B")]:
        n2m, colsm = _pair_count_in_span(M)
        assert n2m == 0 and all(any(c) for c in colsm)  # no weight 1 or 2
        # some weight-3 vector: any single column of M has weight 3
        assert int(M[:, 0].sum()) == g[key][0]
    assert g["dist_HX"][0] == 2 and n2 > 0


def test_lower_bound_coefficients():
    """864 = C(3,2)*288 and 2592 = C(3,2)*C(3,1)*2*144: count configurations on
    the oracle's [[288]] code directly."""
    g = _golden288()
    HX, _ = O.code_matrices(CODES["288"])
    n = HX.shape[1]
    # (a) weight-two syndrome errors on two of the three CNs of one data VN
    count_a = sum(len(list(itertools.combinations(np.nonzero(HX[:, i])[0], 2))) for i in range(n))
    assert count_a == g["coef_ps2"][0]
    # (b) three VNs whose columns sum to a weight-three vector of the form
    # b^2 shifted (b_1^2 or b_2^2): for each column c of A (resp. B), the
    # three columns c * monomial of the polynomial itself
    w = 144
    A, B = HX[:, :w], HX[:, w:]
    cnt = 0
    for M in (A, B):
        for c in range(w):
            col = M[:, c]
            # M @ col = the product of the generator with this column
            prod = (M.astype(np.int64) @ col.astype(np.int64)) % 2
            if prod.sum() == 3:
                cnt += 1
    assert 3 * 3 * 2 * cnt // 2 == g["coef_pdps2"][0]
