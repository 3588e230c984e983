"""Host-side checks of libqdec (no GPU needed): the library loads, exports
every entry point include/qdec.h declares, and its detector error model --
built by a backward sensitivity sweep -- equals the oracle's, which simulates
every fault directly (Sec. II-B)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, oracle_dem
from paper_2403_18901_gb300 import build as qbuild
from paper_2403_18901_gb300 import qdec
from paper_2403_18901_gb300.workloads import CODES


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qdec.lib()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "qdec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qd_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    syms = _declared_symbols()
    assert len(syms) >= 19
    raw = ctypes.CDLL(qdec.LIB_PATH)
    for s in syms:
        assert hasattr(raw, s), s
    assert set(syms) == set(qdec._SIGS), "binding and header disagree"


def test_invalid_arguments_are_rejected(lib):
    with pytest.raises(qdec.QdError) as e:
        qdec.Dem(dict(CODES["72"]), 0.7, 6)
    assert e.value.code == qdec.QD_EINVAL
    with pytest.raises(qdec.QdError):
        qdec.Dem(dict(CODES["72"]), 0.003, 0)


@pytest.mark.parametrize("key,R,p", [("72", 6, 0.003), ("144", 12, 0.003), ("90", 4, 0.002),
                                     ("108", 3, 0.004), ("288", 3, 0.002)])
def test_dem_equals_oracle(lib, key, R, p):
    d = qdec.Dem(CODES[key], p, R)
    o = oracle_dem(key, p, R)
    c = d.columns()
    assert d.n_cols == o.n_cols and d.n_det == o.n_det and d.K == o.K
    assert (c["col_ptr"] == o.col_ptr).all()
    assert (c["col_dets"] == o.col_dets[:len(c["col_dets"])]).all()
    assert (c["obs"] == o.col_obs).all()
    assert (c["prob"] == o.col_p).all()  # bit-identical doubles
    assert (c["llr"] == o.col_llr).all()


@pytest.mark.parametrize("key,pd,ps", [("288", 0.04, 1e-3), ("144", 0.02, 0.0), ("72", 0.05, 0.01)])
def test_code_capacity_dem_equals_oracle(lib, key, pd, ps):
    from oracle import oracle as O
    d = qdec.Dem(CODES[key], 0, 0, capacity=(pd, ps))
    o = O.OracleDEM(CODES[key], pd, 0, capacity=(pd, ps))
    c = d.columns()
    assert d.n_cols == o.n_cols and d.n_det == o.n_det and d.K == o.K and d.n_blocks == o.n_blocks
    assert (c["col_ptr"] == o.col_ptr).all()
    assert (c["col_dets"] == o.col_dets[:len(c["col_dets"])]).all()
    assert (c["obs"] == o.col_obs).all()
    assert (c["prob"] == o.col_p).all()
    assert (c["llr"] == o.col_llr).all()


def test_every_single_fault_is_a_dem_column(lib):
    """Fault by fault: the direct Pauli-frame simulation of every single fault
    (oracle) lands on a column of the library's merged DEM."""
    d = qdec.Dem(CODES["72"], 0.003, 3)
    o = oracle_dem("72", 0.003, 3)
    c = d.columns()
    cols = set()
    for i in range(d.n_cols):
        cols.add((tuple(c["col_dets"][c["col_ptr"][i]:c["col_ptr"][i + 1]].tolist()), int(c["obs"][i])))
    n = 0
    for loc in range(o.n_fault_locations()):
        _, _, info = o.fault_effect(loc, 1)
        for pat in range(1, info[1] + 1):
            dets, obs, _ = o.fault_effect(loc, pat)
            if dets or obs:
                assert (dets, obs) in cols
                n += 1
    assert n > 1000


def test_parameter_validation_without_a_gpu(lib):
    """Checks that fail before any device call, so they run on the host."""
    from paper_2403_18901_gb300.workloads import preset
    d = qdec.Dem(CODES["72"], 0.003, 6)
    bad = [dict(preset("paper", k_guess=4), side_max=2),          # side branches start at k
           dict(preset("configured", k_guess=3), F=4),            # F > W
           dict(preset("configured", k_guess=3), iters_per_step=0),
           dict(preset("configured", k_guess=3), alpha=0.0),
           dict(preset("configured", k_guess=3), d_max_other=1),  # d_max_other < k
           dict(preset("configured", k_guess=3), fallback=3),     # no such output rule
           dict(preset("configured", k_guess=3), merge_h1=-1)]
    for params in bad:
        with pytest.raises(qdec.QdError) as e:
            qdec.Decoder(d, params, max_shots=4)
        assert e.value.code == qdec.QD_EINVAL, params
    with pytest.raises(qdec.QdError) as e:
        qdec.Dem(CODES["288"], 0, 0, capacity=(0.6, 0.0))
    assert e.value.code == qdec.QD_EINVAL
    with pytest.raises(qdec.QdError) as e:
        qdec.Dem(CODES["288"], 0, 0, capacity=(0.04, -1e-3))
    assert e.value.code == qdec.QD_EINVAL
    # a prior outside (2^-15, 16) would make Eq. (5) inexact
    with pytest.raises(qdec.QdError) as e:
        qdec.Dem(CODES["288"], 0, 0, capacity=(0.04, 1e-9))
    assert e.value.code == qdec.QD_EUNSUPPORTED
    h = ctypes.c_void_p()
    assert lib.qd_batch_create((ctypes.c_void_p * 1)(), 0, ctypes.byref(h)) == qdec.QD_EINVAL
    assert lib.qd_ranker_eval(None, None, None, 0, 0, 1.0, 1.0, None, None, None, None) == qdec.QD_EINVAL


@pytest.mark.parametrize("key,R,W,F,merge", [("144", 12, 3, 1, 0), ("144", 12, 3, 1, 1), ("144", 12, 3, 1, 2),
                                              ("72", 6, 5, 2, 1), ("72", 6, 3, 1, 2), ("288", 3, 3, 1, 1)])
def test_windows_equal_the_oracle(lib, key, R, W, F, merge):
    """The decoder's windows (Eq. (8)), with and without the H_1 merge of
    Sec. III, equal the oracle's: columns, rows, commit prefix and the priors
    GDG uses, bit for bit."""
    p = 0.003
    d = qdec.Dem(CODES[key], p, R)
    o = oracle_dem(key, p, R)
    import numpy as np
    for k in range(o.n_windows(W, F)):
        g, w = d.window(W, F, k, merge), o.window(W, F, k, merge)
        for f in ("r0", "n_blocks", "n_rows", "n_cols", "n_edges", "n_commit"):
            assert g[f] == w[f], (k, f)
        assert (g["gcols"] == w["gcols"]).all() and (g["col_ptr"] == w["col_ptr"]).all()
        assert (g["col_rows"] == w["col_rows"]).all()
        assert (g["llr"].view(np.int32) == w["llr"].view(np.int32)).all(), k
