"""Pins of the oracle's SELECT-VN (Alg. 1) and AGG-DEC (Alg. 3).

Each case is a hand-built history / graph whose answer follows from the two
algorithms as printed: Alg. 3's thresholds P_A = -3 (main branch) / 0,
P_B = -12 (main) / -10, P_B = -16 at depth 1 on every branch, P_C = 30 for
D <= 4, P_D = 3 with at least three unsatisfied neighbour checks, every
comparison strict and over all four history entries; Alg. 1's candidates
(active, degree >= 3), the priority of an all-non-positive history
(Lambda_hist <= 0, decimated to 1), otherwise the smallest history sum with
f = sign(L_min) read through Eq. (4) (f = 1 iff L_min <= 0), strict '<' in
index order (ties to the lowest index).

The expected values are written by hand from those rules.  The mutation test
rebuilds the oracle with one plausible misreading planted at a time (on the
CPU) and requires the pins to catch every one.
"""
import ctypes as C
import os
import shutil

import numpy as np
import pytest

from oracle import build as obuild
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import preset

AGG = preset("configured", 4)  # aggressive mode (p > 0.002)
LOW = dict(AGG, low_error_mode=1)

# 6 checks x 6 VNs: VN0..3 of degree 3, VN4 of degree 2, VN5 of degree 1
H6 = np.zeros((6, 6), np.uint8)
for v, rows in enumerate([(0, 1, 2), (1, 2, 3), (3, 4, 5), (0, 4, 5), (0, 3), (5,)]):
    H6[list(rows), v] = 1


def _hist(*rows):
    """rows: one 4-entry history per VN (oldest first) -> [4][nc]."""
    return np.array(rows, np.float32).T.copy()


def _pos(n=6, v=2.0):
    return [[v] * 4 for _ in range(n)]


# (description, args of agg_dec, expected) -- Alg. 3
AGG_CASES = [
    ("main D=2, all four < -3, sum -16 < -12 -> 1", ([-4] * 4, 2, 1, 0), 1),
    ("main D=2, all four == -3 (strict) -> -1", ([-3] * 4, 2, 1, 0), -1),
    ("main D=2, one entry positive: not ALL < P_A -> -1", ([-20, -20, -20, 1], 2, 1, 0), -1),
    ("other D=2, all four < 0, sum -11 < -10 -> 1", ([-2.75] * 4, 2, 0, 0), 1),
    ("main D=2, -2.75 not < P_A(main) = -3 -> -1", ([-2.75] * 4, 2, 1, 0), -1),
    ("other D=2, sum -9.5 not < -10 -> -1", ([-1, -1, -1, -6.5], 2, 0, 0), -1),
    ("other D=2, sum -11 < -10 -> 1", ([-1, -1, -1, -8], 2, 0, 0), 1),
    ("other D=2, an entry equal to P_A(other) = 0 -> -1", ([0, -4, -4, -4], 2, 0, 0), -1),
    ("other D=1: P_B = -16, sum -14 -> -1", ([-3.5] * 4, 1, 0, 0), -1),
    ("other D=1: sum -18 < -16 -> 1", ([-4.5] * 4, 1, 0, 0), 1),
    ("main D=1: P_B = -16, sum -14 -> -1", ([-3.5] * 4, 1, 1, 0), -1),
    ("main D=2: sum -14 < -12 -> 1", ([-3.5] * 4, 2, 1, 0), 1),
    ("D=4, all four > 30 -> 0", ([31] * 4, 4, 0, 0), 0),
    ("D=4 main, all four > 30 -> 0", ([31] * 4, 4, 1, 0), 0),
    ("D=5, all four > 30 but D > 4, no unsatisfied checks -> -1", ([31] * 4, 5, 0, 0), -1),
    ("D=2, one entry 10: not ALL > 30, no unsatisfied -> -1", ([40, 40, 40, 10], 2, 0, 0), -1),
    ("D=2, all four == 30 (strict), no unsatisfied -> -1", ([30] * 4, 2, 0, 0), -1),
    ("D=9, all > 3 and exactly 3 unsatisfied -> 0", ([5] * 4, 9, 0, 3), 0),
    ("D=9 main, all > 3 and exactly 3 unsatisfied -> 0", ([5] * 4, 9, 1, 3), 0),
    ("D=9, all > 3 but only 2 unsatisfied -> -1", ([5] * 4, 9, 0, 2), -1),
    ("D=9, one entry 2: not ALL > 3 -> -1", ([5, 5, 5, 2], 9, 0, 5), -1),
    ("D=9, all four == 3 (strict) -> -1", ([3] * 4, 9, 0, 5), -1),
    ("D=5, all > 30 and 3 unsatisfied -> 0 (second clause)", ([31] * 4, 5, 0, 3), 0),
]


def _select_cases():
    """(description, params, hist, status, synd, D, main, expected (g, f, n_agg), checks)."""
    act = np.full(6, -1, np.int8)
    z = np.zeros(6, np.uint8)
    cases = []
    h = _pos()
    h[0] = [-1] * 4           # all non-positive, L = -4
    h[1] = [-10, -10, 5, 4]   # smaller L = -11, not all non-positive
    cases.append(("all-non-positive history beats a smaller L_min", LOW, h, act, z, 3, 1, (0, 1, 0)))
    h = _pos()
    h[1] = [-2] * 4
    h[2] = [-2] * 4
    cases.append(("tie among all-non-positive histories -> lowest index", LOW, h, act, z, 3, 1, (1, 1, 0)))
    h = _pos(v=3.0)
    h[1] = [-1, 2, -1, 2]
    h[3] = [2, -1, 2, -1]
    h[2] = [1.5] * 4
    cases.append(("tie of L_min = 2 -> lowest index, f = 0", LOW, h, act, z, 3, 1, (1, 0, 0)))
    h = _pos()
    h[0] = [1, -1, 0.5, -0.5]  # L = 0 exactly, one entry positive
    cases.append(("L_min = 0 -> f = 1 (Eq. (4): e = 1 iff LLR <= 0)", LOW, h, act, z, 3, 1, (0, 1, 0)))
    h = _pos()
    h[2] = [0.25] * 4
    cases.append(("all positive -> smallest sum, f = 0", LOW, h, act, z, 3, 1, (2, 0, 0)))
    h = _pos()
    h[4] = [-20] * 4
    h[5] = [-20] * 4
    h[3] = [1] * 4
    cases.append(("degree-2 and degree-1 VNs never selected", LOW, h, act, z, 3, 1, (3, 0, 0)))
    h = _pos()
    h[0] = [-20] * 4
    st = act.copy()
    st[0] = 1
    cases.append(("decimated VN never selected", LOW, h, st, z, 3, 1, (1, 0, 0)))
    h = _pos()
    h[0] = [0, -1, -1, -1]      # all <= 0 with a zero entry
    h[1] = [-10, -10, 1, 1]     # L = -18
    cases.append(("history with a zero entry still counts as non-positive", LOW, h, act, z, 3, 1, (0, 1, 0)))
    h = _pos()
    st = act.copy()
    st[:4] = 0
    cases.append(("no candidate -> g = -1", LOW, h, st, z, 3, 1, (-1, 0, 0)))
    # aggressive mode (Alg. 3 inside Alg. 1)
    h = _pos()
    h[0] = [-4] * 4   # main D=2: decided 1, leaves the selection
    h[1] = [-1] * 4   # not below P_A(main) = -3: stays a candidate
    cases.append(("aggressive 1 on the main branch, then the all-non-positive candidate", AGG, h, act, z, 2,
                  1, (1, 1, 1), {"status0": 1, "synd": [1, 1, 1, 0, 0, 0]}))
    h = _pos()
    h[0] = [-2.75] * 4
    cases.append(("main branch keeps -2.75 as a candidate", AGG, h, act, z, 2, 1, (0, 1, 0), {"status0": -1}))
    cases.append(("other branch decides -2.75 (sum -11) aggressively", AGG, h, act, z, 2, 0, (1, 0, 1),
                  {"status0": 1}))
    h = _pos()
    h[0] = [5] * 4
    s = np.array([1, 1, 1, 0, 0, 0], np.uint8)
    cases.append(("three unsatisfied neighbours -> aggressive 0", AGG, h, act, s, 9, 1, (1, 0, 1),
                  {"status0": 0, "synd": [1, 1, 1, 0, 0, 0]}))
    s = np.array([1, 1, 0, 0, 0, 0], np.uint8)
    cases.append(("two unsatisfied neighbours -> stays a candidate", AGG, h, act, s, 9, 1, (1, 0, 0),
                  {"status0": -1}))
    h = _pos()
    h[0] = [5] * 4
    h[1] = [-1] * 4  # e_1 = 1 flips rows 1, 2, 3
    s = np.array([1, 0, 0, 1, 0, 0], np.uint8)
    cases.append(("unsatisfied counted under the current decisions e, not s' alone", AGG, h, act, s, 9, 1,
                  (1, 1, 1), {"status0": 0}))
    out = []
    for c in cases:
        extra = c[8] if len(c) > 8 else {}
        out.append(c[:8] + (extra,))
    return out


SELECT_CASES = _select_cases()


def pin_failures(lib_=None):
    """Every pin that the oracle library handle lib_ (default: the oracle)
    gets wrong, as a list of descriptions."""
    bad = []
    for desc, (h, D, main, nus), want in AGG_CASES:
        got = O.agg_dec(AGG, h, D, main, nus, lib_=lib_)
        if got != want:
            bad.append(f"AGG-DEC {desc}: got {got}")
    for desc, P, h, st, sp, D, main, want, extra in SELECT_CASES:
        g, f, nagg, st2, sp2 = O.select_vn(P, H6, _hist(*h), st, sp, D, main, lib_=lib_)
        got = (g, f if g >= 0 else 0, nagg)
        if got != want:
            bad.append(f"SELECT-VN {desc}: got {got}, want {want}")
            continue
        if "status0" in extra and int(st2[0]) != extra["status0"]:
            bad.append(f"SELECT-VN {desc}: status[0] = {int(st2[0])}")
        if "synd" in extra and list(sp2) != extra["synd"]:
            bad.append(f"SELECT-VN {desc}: s' = {list(sp2)}")
    return bad


def test_thresholds_are_the_papers():
    """Alg. 3's constants as printed, and the low-error switch of Fig. 3's caption."""
    p = preset("configured", 4, p=0.003)
    assert (p["pa_main"], p["pa_other"], p["pb_main"], p["pb_other"], p["pb_d1"]) == (-3, 0, -12, -10, -16)
    assert (p["pc"], p["pd"], p["pc_max_depth"], p["n_unsat_min"]) == (30, 3, 4, 3)
    assert p["low_error_mode"] == 0 and preset("configured", 4, p=0.002)["low_error_mode"] == 1
    assert preset("paper", 4)["pa_main"] == -3


def test_select_and_agg_pins():
    bad = pin_failures()
    assert not bad, "\n".join(bad)


# One plausible misreading of Alg. 1 / Alg. 3 per entry: (name, text in
# oracle/gdg.c, replacement).  Each must be caught by the pins above.
MUTATIONS = [
    ("f = [L_min < 0]", "*f_out = (gmin != -1 && Lmin <= 0.0f) ? 1 : 0;",
     "*f_out = (gmin != -1 && Lmin < 0.0f) ? 1 : 0;"),
    ("no all-non-positive priority", "} else if (gt != -1) {", "} else if (0 && gt != -1) {"),
    ("any (not all) below P_A", "if (h[0] < PA && h[1] < PA && h[2] < PA && h[3] < PA && L < PB) return 1;",
     "if ((h[0] < PA || h[1] < PA || h[2] < PA || h[3] < PA) && L < PB) return 1;"),
    ("any (not all) above P_C", "int allc = h[0] > P->pc && h[1] > P->pc && h[2] > P->pc && h[3] > P->pc;",
     "int allc = h[0] > P->pc || h[1] > P->pc || h[2] > P->pc || h[3] > P->pc;"),
    ("any (not all) above P_D", "int alld = h[0] > P->pd && h[1] > P->pd && h[2] > P->pd && h[3] > P->pd;",
     "int alld = h[0] > P->pd || h[1] > P->pd || h[2] > P->pd || h[3] > P->pd;"),
    ("P_B = -16 at D = 1 on the main branch only", "if (D == 1) PB = P->pb_d1;",
     "if (D == 1 && main_branch) PB = P->pb_d1;"),
    ("P_A main / other swapped", "float PA = main_branch ? P->pa_main : P->pa_other;",
     "float PA = main_branch ? P->pa_other : P->pa_main;"),
    ("P_B main / other swapped", "float PB = main_branch ? P->pb_main : P->pb_other;",
     "float PB = main_branch ? P->pb_other : P->pb_main;"),
    ("more than (not at least) 3 unsatisfied", "n_unsat >= P->n_unsat_min", "n_unsat > P->n_unsat_min"),
    ("P_C test for D < 4", "D <= P->pc_max_depth", "D < P->pc_max_depth"),
    ("P_C test at every depth", "(allc && D <= P->pc_max_depth)", "(allc)"),
    ("degree-2 VNs allowed", "if (g->vdeg[i] <= 2) continue;", "if (g->vdeg[i] < 2) continue;"),
    ("ties to the highest index", "if (L < Lmin) {", "if (L <= Lmin) {"),
    ("all-negative test strict (< 0)",
     "h[0] <= 0.0f && h[1] <= 0.0f && h[2] <= 0.0f && h[3] <= 0.0f && L < Lt",
     "h[0] < 0.0f && h[1] < 0.0f && h[2] < 0.0f && h[3] < 0.0f && L < Lt"),
    ("unsatisfied counted from s' alone", "if (s->status[i] == -1) par ^= hard(s, i);", "if (0) par ^= hard(s, i);"),
    ("aggressive decision not applied", "decimate(g, s, i, b);\n        (*n_agg)++;",
     "(*n_agg)++;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = os.path.dirname(obuild.__file__)
    for f in obuild.SOURCES + ["qdo.h"]:
        shutil.copy(os.path.join(src, f), tmp_path / f)
    text = (tmp_path / "gdg.c").read_text()
    assert text.count(old) == 1, f"mutation site not unique in gdg.c: {old!r}"
    (tmp_path / "gdg.c").write_text(text.replace(old, new))
    out = str(tmp_path / f"liboracle_mut.so")
    obuild.compile_lib(str(tmp_path), out)
    L = O.declare_select(C.CDLL(out))
    assert pin_failures(L), f"no pin catches: {name}"
