"""Host check of the decoder's shared-memory layout: make_layout (the one
definition shared by the host plan and the kernels) gives 16-byte aligned,
non-overlapping regions that fit, for the windows of every code and window
shape the tests and the bench decode (tests/layout_check.cpp states the
invariants)."""
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
