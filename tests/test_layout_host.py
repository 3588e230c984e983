"""Host checks of definitions the kernels share with the host, built with g++
from gdg_kernel.cuh: the shared-memory layout (make_layout gives 16-byte
aligned, non-overlapping regions that fit, for the windows of every code and
window shape the tests and the bench decode; tests/layout_check.cpp states
the invariants) and the decision-path schedule (path_at, path_split,
path_reinit, path_dmax against the oracle's tree; tests/tree_check.cpp)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_18901_gb300.workloads import CODES

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("layout") / "layout_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-o", exe, os.path.join(HERE, "layout_check.cpp")],
                   check=True, capture_output=True)
    return exe


def _windows(key, rounds, W, F, capacity=None):
    if capacity is None:
        d = O.OracleDEM(CODES[key], 0.003, rounds)
    else:
        d = O.OracleDEM(CODES[key], capacity[0], 0, capacity=capacity)
    for k in range(d.n_windows(W, F)):
        w = d.window(W, F, k)
        if w["n_cols"] == 0:
            continue
        nr, nc, ne = w["n_rows"], w["n_cols"], w["n_edges"]
        ns = 2 * nr if (capacity is None and nc > 2 * nr) else nc
        deg = np.sort(np.diff(w["col_ptr"]))[::-1]
        yield nr, nc, ne, ns, int(deg[:ns].sum())


CASES = [("72", 6, 3, 1, None, 16), ("90", 10, 3, 1, None, 16), ("108", 10, 4, 1, None, 16),
         ("144", 12, 3, 1, None, 22), ("144", 6, 5, 2, None, 22), ("288", 3, 3, 1, None, 47),
         ("288", 4, 4, 1, None, 47), ("288", 0, 1, 1, (0.04, 0.001), 47), ("144", 0, 1, 1, (0.06, 0.0), 47)]


@pytest.mark.parametrize("key,rounds,W,F,capacity,nb", CASES)
def test_layouts_are_aligned_disjoint_and_fit(checker, key, rounds, W, F, capacity, nb):
    seen = set()
    for dims in _windows(key, rounds, W, F, capacity):
        if dims in seen:
            continue
        seen.add(dims)
        for nslots in (1, 3, 8):
            for stage in (0, 1):
                for ranker in (0, 1):
                    args = [str(x) for x in (*dims, nb, nslots, stage, ranker)]
                    r = subprocess.run([checker] + args, capture_output=True, text=True)
                    assert r.returncode == 0 and r.stdout.strip() == "ok", (args, r.stdout)


# ---- the decision-path schedule (path_split, path_reinit, path_at, path_dmax) ----

@pytest.fixture(scope="module")
def tree_checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("tree") / "tree_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-o", exe, os.path.join(HERE, "tree_check.cpp")],
                   check=True, capture_output=True)
    return exe


def _oracle_paths(params):
    import ctypes as C
    P = O.make_params(params, None, None)
    return O.lib().qdo_n_paths(C.byref(P)), O.lib().qdo_path_dmax_all(C.byref(P))


TREES = [("configured", dict(k_guess=k)) for k in range(1, 6)] + [
    ("paper", dict(k_guess=3)), ("paper", dict(k_guess=4)), ("paper", dict(k_guess=4, reinit_on_split=1)),
    ("paper", dict(k_guess=5, d_max_main=40, d_max_other=25, side_max=20, n_pre=16)),
    ("configured", dict(k_guess=4, reinit_on_split=1)), ("capacity", dict())]


@pytest.mark.parametrize("pname,over", TREES)
def test_path_schedule_matches_the_oracle_tree(tree_checker, pname, over):
    """The kernels' queue visits every path once, main branch first; path
    counts and the deepest D_max equal the oracle's; splits and message
    restarts follow the Fig. 2 reading (id 1 splits at depth k, ids 2^k..
    at k + 1 .. side_max; restarts at a side branch's split and at depth k
    for odd tree ids)."""
    from paper_2403_18901_gb300.workloads import CAPACITY, preset
    params = dict(CAPACITY, **over) if pname == "capacity" else preset(pname, **over)
    nb, dmax_all = _oracle_paths(params)
    k, side, reinit = params["k_guess"], params["side_max"], int(params["reinit_on_split"])
    args = [str(x) for x in (k, side, reinit, nb, params["d_max_main"], params["d_max_other"])]
    r = subprocess.run([tree_checker] + args, capture_output=True, text=True, check=True)
    rows = [tuple(int(v) for v in line.split()) for line in r.stdout.strip().splitlines()]
    ids = [row[1] for row in rows]
    assert sorted(ids) == list(range(nb)) and ids[0] == 0
    assert max(row[4] for row in rows) == dmax_all
    nt = 1 << k
    for _, pid, split, rst, dmax in rows:
        if pid >= nt:
            assert split == k + 1 + (pid - nt) and split <= side
        else:
            assert split == (k if (side > 0 and pid == 1) else 0)
        want_rst = (split if split else (k if pid % 2 == 1 else 0)) if reinit else 0
        assert rst == want_rst
        assert dmax == (params["d_max_main"] if pid == 0 else
                        (split + params["d_max_other"] - k if split else params["d_max_other"]))
