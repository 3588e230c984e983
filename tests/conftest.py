import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


_DEMS = {}


def oracle_dem(code_key, p, rounds):
    """Session-cached oracle DEM."""
    from oracle import oracle as O
    from paper_2403_18901_gb300.workloads import CODES
    key = (code_key, p, rounds)
    if key not in _DEMS:
        _DEMS[key] = O.OracleDEM(CODES[code_key], p, rounds)
    return _DEMS[key]
