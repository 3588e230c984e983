"""The allocation-free decode + commit entry point (qd_decode_commit_static).

Callers that cannot call cudaMalloc while decoding -- a real-time loop that
cannot afford the stall of an allocation, or a framework that owns all device
memory -- decode and commit a window with scratch that lives in a fixed array
inside libqdec.  This test drives that entry point through the C ABI and checks,
bit for bit (the tolerance of every decoder test here), that it gives the same
committed syndromes, observable predictions and residue flags as the
two-call path qd_decode_windows + qd_commit_and_slide, over two complete
passes in a row (the array keeps the previous call's contents).  The file
sorts last so that a run stopping at the first failure has already run every
other test.
"""
import numpy as np
import pytest

from paper_2403_18901_gb300 import build as qbuild
from paper_2403_18901_gb300 import qdec
from paper_2403_18901_gb300.workloads import CODES, preset

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qbuild.build()
    qdec.lib()


def _run(dec, det0, n, use_static):
    det = det0.clone()
    pred = torch.zeros(n, dtype=torch.int32, device="cuda")
    resid = torch.zeros(n, dtype=torch.int32, device="cuda")
    corr = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
    for k in range(dec.n_windows):
        if use_static:
            dec.decode_commit_static(k, det, n, pred, resid)
        else:
            dec.decode_window(k, det, n, corr)
            dec.commit(k, corr, n, det, pred, resid)
    torch.cuda.synchronize()
    return det.cpu().numpy(), pred.cpu().numpy(), resid.cpu().numpy()


# (code, rounds, k, shots, launch mode): 0 = automatic (throughput shape at
# these batch sizes), 2 = one CTA per decision path, 3 = path state in global
# memory (the decoder's own union regions)
CASES = [("144", 12, 4, 600, 0), ("72", 6, 3, 513, 0), ("144", 12, 4, 24, 2), ("72", 6, 3, 300, 3)]


@pytest.mark.parametrize("key,R,k,n,mode", CASES)
def test_static_scratch_matches_two_call_path(key, R, k, n, mode):
    dem = qdec.Dem(CODES[key], 0.003, R)
    dec = qdec.Decoder(dem, preset("configured", k_guess=k), max_shots=n)
    dec.set_launch(mode)
    for seed in (11, 12):  # two calls in a row on different inputs
        det0, _ = dem.sample(seed=seed, shot_offset=0, n_shots=n)
        dec.reset_counters()
        ref = _run(dec, det0, n, use_static=False)
        c_ref = dec.counters()
        dec.reset_counters()
        got = _run(dec, det0, n, use_static=True)
        c_got = dec.counters()
        for a, b in zip(ref, got):
            assert (a == b).all()
        # the same work, counted in the decoder's counters by both paths
        assert list(c_ref) == list(c_got) and c_got[1] > 0 and c_got[4] == 0
    # and the same input twice through the static path
    again = _run(dec, det0, n, use_static=True)
    for a, b in zip(got, again):
        assert (a == b).all()


def test_static_scratch_allocates_nothing():
    dem = qdec.Dem(CODES["72"], 0.003, 6)
    n = 256
    dec = qdec.Decoder(dem, preset("configured", k_guess=3), max_shots=n)
    det0, _ = dem.sample(seed=21, shot_offset=0, n_shots=n)
    det = det0.clone()
    pred = torch.zeros(n, dtype=torch.int32, device="cuda")
    resid = torch.zeros(n, dtype=torch.int32, device="cuda")
    # warm-up: the array's address is looked up once, and every kernel of the
    # loop below (the copy included) is loaded before memory is measured
    det.copy_(det0)
    for k in range(dec.n_windows):
        dec.decode_commit_static(k, det, n, pred, resid)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        det.copy_(det0)
        for k in range(dec.n_windows):
            dec.decode_commit_static(k, det, n, pred, resid)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_static_scratch_rejects_oversized_batches():
    dem = qdec.Dem(CODES["144"], 0.003, 12)
    big = 40000
    dec = qdec.Decoder(dem, preset("configured", k_guess=4), max_shots=big)
    det = torch.zeros((big, dem.det_words), dtype=torch.int32, device="cuda")
    pred = torch.zeros(big, dtype=torch.int32, device="cuda")
    resid = torch.zeros(big, dtype=torch.int32, device="cuda")
    with pytest.raises(qdec.QdError) as e:
        dec.decode_commit_static(0, det, big, pred, resid)
    assert e.value.code == qdec.QD_EINVAL
    assert "static scratch" in str(e.value) and "30839" in str(e.value)
