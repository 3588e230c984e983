"""Pins of the oracle's code-capacity models (appendix "Data qubit noise":
BSC(p_d) on the data qubits decoded with H_X; appendix "Single shot syndrome
noise": [H_X | I] with a virtual column per check).

* Structure stated in the appendix: for [[288,12,18]], 288 original VNs of
  degree three and 144 virtual VNs of degree one; 12 logical operators in the
  kernel of H_Z, independent of the row span of H_X.
* Every single data-qubit error is decoded (distance 18).
* The failure mechanism behind the appendix's lower bound 864 p_s^2: a
  weight-two syndrome error on two of the three checks of an original VN is
  explained more cheaply (p_s < p_d) by that VN plus the third check, so the
  data estimate has the wrong syndrome and the shot fails.
* The measured failure rate is not below the bound p_L(p_d) + 864 p_s^2 +
  2592 p_d p_s^2.
"""
import math

import numpy as np

from gf2 import rank
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import CAPACITY, CODES

MAIN = dict(CAPACITY, k_guess=0, side_max=0)  # the main branch alone (fast)


def _wilson_hi(k, n, z=1.96):
    ph = k / n
    return (ph + z * z / (2 * n) + z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n))) / (1 + z * z / n)


def test_structure_of_the_single_shot_matrix():
    code = CODES["288"]
    o = O.OracleDEM(code, 0.04, 0, capacity=(0.04, 1e-3))
    HX, HZ = O.code_matrices(code)
    w, n = HX.shape
    assert o.n_det == 2 * w and o.K == 12 and o.n_blocks == 2
    win = o.window(1, 1, 0)
    deg = np.diff(win["col_ptr"])
    assert win["n_rows"] == 144 and (deg == 3).sum() == 288 and (deg == 1).sum() == 144 and len(deg) == 432
    assert win["n_commit"] == 432
    assert o.window(1, 1, 1)["n_cols"] == 0  # the noiseless block only checks the residue
    LX = O.logical_x(code)
    assert LX.shape[0] == 12
    assert not ((HZ.astype(np.int64) @ LX.T.astype(np.int64)) % 2).any()
    assert rank(np.vstack([HX, LX])) == rank(HX) + 12
    # data columns carry exactly the logical bits of their qubit, virtual ones none
    for c in range(o.n_cols):
        dets, obs = o.column(c)
        if len(dets) == 1:
            assert obs == 0 and o.col_p[c] == 1e-3
        else:
            i = [q for q in range(n) if tuple(np.nonzero(HX[:, q])[0]) == tuple(d for d in dets if d < w)]
            assert len(i) == 1 and dets[3:] == tuple(d + w for d in dets[:3])
            assert obs == sum(int(LX[k, i[0]]) << k for k in range(12))


def _syndrome_bits(o, cols):
    s = np.zeros(o.n_det, np.uint8)
    for c in cols:
        for d in o.column(c)[0]:
            s[d] ^= 1
    return s


def _decode(o, params, s, obs_true=0):
    """Decode one shot given its detector bits; returns (failure flags, predicted observables)."""
    words = np.zeros((1, o.det_words), np.uint32)
    for d in np.nonzero(s)[0]:
        words[0, d >> 5] |= np.uint32(1) << np.uint32(d & 31)
    obs = np.full(1, obs_true, np.uint32)
    f, pred, _ = o.run_shots(params, words, obs, threads=1)
    return int(f[0]), int(pred[0])


def test_single_data_errors_are_decoded():
    code = CODES["288"]
    o = O.OracleDEM(code, 0.02, 0, capacity=(0.02, 0.0))
    data_cols = [c for c in range(o.n_cols)]
    assert len(data_cols) == 288
    for c in data_cols:
        f, pred = _decode(o, MAIN, _syndrome_bits(o, [c]), int(o.col_obs[c]))
        assert f == 0 and pred == o.col_obs[c], c


def test_weight_two_syndrome_error_fails():
    code = CODES["288"]
    o = O.OracleDEM(code, 0.03, 0, capacity=(0.03, 0.003))
    w = o.w
    virt = {o.column(c)[0][0]: c for c in range(o.n_cols) if len(o.column(c)[0]) == 1}
    data = [c for c in range(o.n_cols) if len(o.column(c)[0]) == 6]
    rng = np.random.default_rng(3)
    for c in rng.choice(data, 12, replace=False):
        checks = o.column(c)[0][:3]
        for a in range(3):
            for b in range(a + 1, 3):
                s = _syndrome_bits(o, [virt[checks[a]], virt[checks[b]]])
                assert not s[w:].any()
                f, _ = _decode(o, MAIN, s)
                assert f & 1, (c, checks[a], checks[b])  # wrong data syndrome: Eq. (11) residue


def test_failure_rate_respects_the_lower_bound():
    pd, ps = 0.02, 0.01
    o = O.OracleDEM(CODES["288"], pd, 0, capacity=(pd, ps))
    n = 600
    det, obs = o.sample(11, 0, n)
    f, _, _ = o.run_shots(MAIN, det, obs, threads=O.default_threads())
    k = int((f > 0).sum())
    bound = 864 * ps * ps + 2592 * pd * ps * ps
    assert _wilson_hi(k, n) >= bound, (k, n, bound)
