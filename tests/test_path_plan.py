"""Host-side checks of shot mode's decision-path plan (qd_path_plan): which
paths may resume from which snapshot.  A snapshot node of depth D joins paths
whose decisions at depths 1..D-1 agree; by Alg. 2 and Fig. 2 (ids MSB-first
over the k guessing depths, side branches contrary only at their split, the
main branch's Alg. 3 thresholds, message restarts) such paths are in the same
state after the BP of step D.  Checked against the decision rules stated
here, and against the oracle's own per-path decision records."""
import numpy as np
import pytest

from conftest import oracle_dem
from paper_2403_18901_gb300 import build as qbuild
from paper_2403_18901_gb300 import qdec
from paper_2403_18901_gb300.workloads import CAPACITY, preset


@pytest.fixture(scope="module", autouse=True)
def _lib():
    qbuild.build()
    qdec.lib()


def _split(P, i):
    k = P["k_guess"]
    if P["side_max"] <= 0:
        return 0
    if i >= 1 << k:
        return k + 1 + (i - (1 << k))
    return k if (i == 1 and k >= 1) else 0


def _dmax(P, i):
    s = _split(P, i)
    return P["d_max_main"] if i == 0 else (s + P["d_max_other"] - P["k_guess"] if s else P["d_max_other"])


def _decision(P, i, d):
    """(contrary guess value, main-branch thresholds, message restart) of path i at depth d."""
    k, s = P["k_guess"], _split(P, i)
    contrary = (d == s) if s else (d <= k and (i >> (k - d)) & 1 == 1)
    main = (not P["low_error_mode"]) and (i == 0 or (s and d <= s))
    restart = P["reinit_on_split"] and ((d == s) if s else (i % 2 == 1 and d == k))
    return (bool(contrary), bool(main), bool(restart))


PLANS = [("configured k3 p3e-3", preset("configured", 3, p=0.003)),
         ("configured k4 p3e-3", preset("configured", 4, p=0.003)),
         ("configured k4 p2e-3", preset("configured", 4, p=0.002)),
         ("configured k5 p3e-3", preset("configured", 5, p=0.003)),
         ("paper k4", preset("paper", 4, p=0.003)),
         ("paper k4 reinit", preset("paper", 4, p=0.004, reinit_on_split=1)),
         ("capacity", dict(CAPACITY))]


@pytest.mark.parametrize("name,P", PLANS, ids=[p[0] for p in PLANS])
@pytest.mark.parametrize("wave", [8, 6])
def test_plan_structure(name, P, wave):
    pl = qdec.path_plan(P, wave)
    nb = pl["nb"]
    assert nb == (1 << P["k_guess"]) + max(0, P["side_max"] - P["k_guess"])
    if nb <= wave:
        assert pl["n_nodes"] == -1  # every path has its own warp: nothing to plan
        return
    order, chain, fnode, fdep = pl["order"], pl["chain"], pl["fnode"], pl["fdep"]
    assert sorted(order.tolist()) == list(range(nb))
    assert order[0] == max(range(nb), key=lambda i: (_dmax(P, i), -i))  # the longest path first
    pos = {int(p): n for n, p in enumerate(order)}
    members = {}
    for p in range(nb):
        for D in range(1, _dmax(P, p) + 1):
            n = int(chain[p, D - 1])
            if n >= 0:
                members.setdefault(n, []).append((p, D))
        for D in range(_dmax(P, p) + 1, pl["dmx"] + 1):
            assert chain[p, D - 1] == -1
    assert len(members) == pl["n_nodes"]
    for n, ms in members.items():
        depths = {D for _, D in ms}
        assert len(depths) == 1 and len(ms) >= 2, (n, ms)
        D = depths.pop()
        ref = [_decision(P, ms[0][0], d) for d in range(1, D)]
        for p, _ in ms[1:]:
            assert [_decision(P, p, d) for d in range(1, D)] == ref, (n, p)
    for p in range(nb):
        if pos[p] < wave:
            assert fnode[p] == -1
        elif fnode[p] >= 0:
            D = int(fdep[p])
            assert chain[p, D - 1] == fnode[p]
            assert any(pos[q] < pos[p] for q, _ in members[int(fnode[p])])


def test_plan_matches_the_oracles_decision_records():
    """Paths joined at a node of depth D make identical decisions (selected
    VN, value, aggressive and peeled counts) at every depth before D in the
    oracle, which runs every path from the root."""
    P = preset("configured", 4, p=0.003)
    pl = qdec.path_plan(P, 8)
    o = oracle_dem("72", 0.003, 6)
    win = o.window(3, 1, 1)
    det, _ = o.sample(72_777, 0, 40)
    rows = np.arange(win["r0"] * o.w, win["r0"] * o.w + win["n_rows"])
    checked = 0
    for s in range(det.shape[0]):
        synd = ((det[s][rows >> 5] >> (rows & 31)) & 1).astype(np.uint8)
        _, info, tr = o.decode_window(P, 1, synd, trace=True)
        if info["prebp_converged"]:
            continue
        for p in range(pl["nb"]):
            for D in range(1, _dmax(P, p) + 1):
                n = int(pl["chain"][p, D - 1])
                if n < 0:
                    continue
                for q in range(p):
                    if pl["chain"][q, D - 1] == n:
                        assert tr["steps"][p][:D - 1] == tr["steps"][q][:D - 1], (s, p, q, D)
                        checked += 1
    assert checked > 0
