"""Pins of the oracle's circuit and detector error model (Sec. II-B, Fig. 1,
appendix "Stim circuit implementation").

The determinism check propagates Z operators BACKWARD through the circuit
(Heisenberg picture), independently of the oracle's forward X-frame
simulation that builds the DEM."""
from collections import Counter

import numpy as np
import pytest

from conftest import oracle_dem
from oracle import oracle as O
from paper_2403_18901_gb300.workloads import CODES

OP_CNOT, OP_MZ, OP_RZ, OP_RX, OP_MRX, OP_NOISE = range(6)


def _measured_operators(dem):
    """For each Z measurement, push Z on the measured qubit backward to the
    start of the circuit.  Z on a qubit prepared in |+> (RX / MRX) means the
    outcome is random.  Returns, for every measurement, the Z support on the
    data qubits at the moment of the previous Z-ancilla reset, and a flag
    telling whether any X-ancilla preparation was hit."""
    ops = dem.circuit_ops()
    w = dem.w
    res = []
    meas_idx = [k for k in range(len(ops)) if ops[k, 0] == OP_MZ]
    for k in meas_idx:
        z = np.zeros(4 * w, np.uint8)
        z[ops[k, 1]] = 1
        random_hit = False
        support = None
        for q in range(k - 1, -1, -1):
            t, a, b, _ = ops[q]
            if t == OP_CNOT:
                z[a] ^= z[b]  # Z on target -> Z on control and target
            elif t in (OP_RX, OP_MRX):
                if z[a]:
                    random_hit = True
                    z[a] = 0
            elif t == OP_RZ:
                if a == ops[k, 1] and support is None:
                    support = z[w:3 * w].copy()
                z[a] = 0
            elif t == OP_MZ:
                pass
        res.append((support, random_hit))
    return res


@pytest.mark.parametrize("key,R", [("72", 3), ("144", 2), ("90", 2)])
def test_z_checks_measured_deterministically(key, R):
    dem = oracle_dem(key, 0.003, R)
    _, HZ = O.code_matrices(CODES[key])
    res = _measured_operators(dem)
    w = dem.w
    assert len(res) == R * w
    for m, (support, hit) in enumerate(res):
        assert not hit, f"measurement {m} depends on an X-basis preparation"
        # the measured operator is row (m mod w) of H_Z
        assert support is not None
        assert (support == HZ[m % w]).all()


@pytest.mark.parametrize("key,R", [("72", 6), ("144", 4), ("90", 3), ("108", 3)])
def test_dem_block_shapes(key, R):
    """H0' has 2w columns, every later H0 has 3w (Fig. 1 caption, appendix
    "Stim circuit implementation"); no column touches more than two
    consecutive blocks (Sec. II-B).  READING: the two-round columns number 7w
    per round (w measurement faults, 2 x 2w data faults between a data qubit's
    Z-check CNOTs, 2w X-ancilla hook faults partly seen in the same round),
    where the Fig. 1 caption states 9w."""
    dem = oracle_dem(key, 0.003, R)
    w = dem.w
    c = Counter()
    for col in range(dem.n_cols):
        dets, obs = dem.column(col)
        assert len(dets) > 0  # no undetectable logical fault at this distance
        b0, b1 = dets[0] // w, dets[-1] // w
        assert b1 - b0 <= 1
        c[(b0, b1 - b0)] += 1
    assert c[(0, 0)] == 2 * w
    for b in range(1, R + 1):
        assert c[(b, 0)] == 3 * w
    for b in range(R):
        assert c[(b, 1)] == 7 * w
    assert dem.n_cols == 2 * w + 10 * w * R
    assert dem.noiseless_detectors().sum() == 0


def test_measurement_faults_are_degree_two():
    """A flipped Z measurement in round r triggers the detectors of its check
    in blocks r-1 and r only (Sec. II-B)."""
    dem = oracle_dem("72", 0.003, 6)
    ops = dem.circuit_ops()
    w = dem.w
    locs = [k for k in range(len(ops)) if ops[k, 0] == OP_NOISE]
    loc_of = {op_index: i for i, op_index in enumerate(locs)}
    n = 0
    for k in range(len(ops) - 1):
        if ops[k, 0] == OP_NOISE and ops[k + 1, 0] == OP_MZ:
            rec = ops[k + 1, 3]
            r, i = rec // w, rec % w
            dets, obs, _ = dem.fault_effect(loc_of[k], 1)
            assert dets == (r * w + i, (r + 1) * w + i)
            assert obs == 0
            n += 1
    assert n == 6 * w


def test_h0prime_is_data_faults_before_all_cnots():
    """The 2w columns of H0' come from single faults on L or R data before all
    CNOTs of the first round (appendix "Stim circuit implementation")."""
    dem = oracle_dem("72", 0.003, 6)
    ops = dem.circuit_ops()
    w = dem.w
    locs = [k for k in range(len(ops)) if ops[k, 0] == OP_NOISE]
    first_cnot = min(k for k in range(len(ops)) if ops[k, 0] == OP_CNOT)
    data_cols = set()
    for i, k in enumerate(locs):
        if k < first_cnot and w <= ops[k, 1] < 3 * w:
            data_cols.add(dem.fault_effect(i, 1)[:2])
    h0p = set()
    for col in range(dem.n_cols):
        dets, obs = dem.column(col)
        if dets[-1] < w:
            h0p.add((dets, obs))
    assert data_cols == h0p and len(h0p) == 2 * w


def test_hook_faults_fill_h0():
    """The extra w columns of a later H0 come from faults on the X-check
    ancillas just before the round-6 CNOTs; each becomes two faults on L data
    that the current round's Z checks cannot see (appendix "Stim circuit
    implementation")."""
    dem = oracle_dem("72", 0.003, 6)
    ops = dem.circuit_ops()
    w = dem.w
    locs = [k for k in range(len(ops)) if ops[k, 0] == OP_NOISE]
    # round 2 spans the second block of 8 layers; find the X-ancilla CNOTs onto
    # L data that are the first of the two L-targets after the R-targets
    cnot_idx = [k for k in range(len(ops)) if ops[k, 0] == OP_CNOT and ops[k, 1] < w]
    per_round = len(cnot_idx) // 6
    r2 = cnot_idx[per_round * 1:per_round * 2]
    layer5 = r2[3 * w:4 * w]  # fourth X layer of the round: last R target (layer 5)
    hook = set()
    for k in layer5:
        noise = k + 1
        assert ops[noise, 0] == OP_NOISE
        dets, obs, info = dem.fault_effect(locs.index(noise), 1)  # X on control after layer 5
        hook.add((dets, obs))
        assert len({d // w for d in dets}) == 1
    blk = 2  # the faults after round 2 show up in block 2 only
    h0 = set()
    for col in range(dem.n_cols):
        dets, obs = dem.column(col)
        if dets[0] // w == blk and dets[-1] // w == blk:
            h0.add((dets, obs))
    assert len(hook) == w and hook <= h0
    assert len(h0 - hook) == 2 * w


def test_columns_canonical_and_priors():
    dem = oracle_dem("72", 0.003, 6)
    keys = [dem.column(c) for c in range(dem.n_cols)]
    assert keys == sorted(keys)
    assert len(set(keys)) == len(keys)
    lam = np.log((1 - dem.col_p) / dem.col_p).astype(np.float32)
    assert (lam == dem.col_llr).all()
    # Eq. (5) exactness requires positive priors well inside (2^-15, 16)
    assert dem.col_llr.min() > 2.0 ** -15 and dem.col_llr.max() < 16
