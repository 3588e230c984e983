"""GPU tests of batched window steps (qd_batch_*): several decoders -- codes
of different sizes and window sizes W = 2, 3, 4 -- advance one window step
per launch pair.  The batch must reproduce, bit for bit, the per-decoder
path (itself bit-exact to the oracle) for every CTA shape, under CUDA-graph
replay, and after the autotuner has picked shapes; two members are also
compared with the oracle directly."""
import numpy as np
import pytest

from conftest import oracle_dem
from paper_2403_18901_gb300 import build as qbuild
from paper_2403_18901_gb300 import qdec
from paper_2403_18901_gb300.workloads import CODES, preset

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = 0.004
MEMBERS = [("72", 6, 2, 96), ("72", 6, 3, 80), ("90", 6, 4, 64), ("108", 6, 3, 48), ("72", 6, 4, 40)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qbuild.build()
    qdec.lib()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def setup():
    mem = []
    for i, (key, R, W, n) in enumerate(MEMBERS):
        d = qdec.Dem(CODES[key], P, R)
        params = preset("configured", k_guess=3, p=P, W=W)
        dec = qdec.Decoder(d, params, max_shots=n)
        det, obs = d.sample(seed=900 + i, shot_offset=0, n_shots=n)
        mem.append(dict(key=key, R=R, W=W, n=n, dem=d, params=params, dec=dec, det=det, obs=obs))
    return mem


def _reference(m):
    """Per-decoder window loop: qd_decode_windows + qd_commit_and_slide."""
    dec, n = m["dec"], m["n"]
    det = m["det"].clone()
    corr = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
    pred = torch.zeros(n, dtype=torch.int32, device="cuda")
    resid = torch.zeros(n, dtype=torch.int32, device="cuda")
    for k in range(dec.n_windows):
        dec.decode_window(k, det, n, corr)
        dec.commit(k, corr, n, det, pred, resid)
    torch.cuda.synchronize()
    return _u32(det), _u32(pred), _u32(resid)


def _fresh(mem):
    det = [m["det"].clone() for m in mem]
    pred = [torch.zeros(m["n"], dtype=torch.int32, device="cuda") for m in mem]
    resid = [torch.zeros(m["n"], dtype=torch.int32, device="cuda") for m in mem]
    return det, pred, resid


def _check(mem, det, pred, resid):
    torch.cuda.synchronize()
    for i, m in enumerate(mem):
        rd, rp, rr = m.setdefault("ref", _reference(m))
        assert (_u32(det[i]) == rd).all(), f"member {i}: committed syndromes differ"
        assert (_u32(pred[i]) == rp).all(), f"member {i}: observable predictions differ"
        assert (_u32(resid[i]) == rr).all(), f"member {i}: residue flags differ"


def test_batch_equals_per_decoder(setup):
    b = qdec.Batch([m["dec"] for m in setup])
    assert b.n_steps == max(m["dec"].n_windows for m in setup)
    det, pred, resid = _fresh(setup)
    n = [m["n"] for m in setup]
    for j in range(b.n_steps):
        b.step(j, det, n, pred, resid)
    _check(setup, det, pred, resid)


@pytest.mark.parametrize("warps,ctas", [(1, 2), (3, 1), (5, 2), (8, 2), (8, 1)])
def test_every_shape_is_bit_exact(setup, warps, ctas):
    b = qdec.Batch([m["dec"] for m in setup])
    for j in range(b.n_steps):
        b.set_shape(j, warps, ctas)
        assert b.info(j)["warps"] == warps
    det, pred, resid = _fresh(setup)
    n = [m["n"] for m in setup]
    for j in range(b.n_steps):
        b.step(j, det, n, pred, resid)
    _check(setup, det, pred, resid)


def test_graph_replay_and_autotune(setup):
    b = qdec.Batch([m["dec"] for m in setup])
    n = [m["n"] for m in setup]
    det0 = [m["det"].clone() for m in setup]
    for j in range(b.n_steps):
        ms = b.autotune(j, det0, n, reps=2)
        assert ms > 0 and 4 <= b.info(j)["warps"] <= 8
    det, pred, resid = _fresh(setup)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm the launch path before capture
        for j in range(b.n_steps):
            b.step(j, det, n, pred, resid, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for j in range(b.n_steps):
            b.step(j, det, n, pred, resid, stream=s)
    for rep in range(2):
        for i, m in enumerate(setup):
            det[i].copy_(m["det"])
            pred[i].zero_()
            resid[i].zero_()
        g.replay()
        _check(setup, det, pred, resid)


def test_members_match_oracle(setup):
    for i in (0, 2):  # [[72]] with W = 2, [[90]] with W = 4
        m = setup[i]
        o = oracle_dem(m["key"], P, m["R"])
        det0, obs0 = o.sample(900 + i, 0, m["n"])
        assert (_u32(m["det"]) == det0).all()
        ofail, opred, _ = o.run_shots(m["params"], det0, obs0, threads=8)
        b = qdec.Batch([m["dec"]])
        det, pred, resid = _fresh([m])
        for j in range(b.n_steps):
            b.step(j, det, [m["n"]], pred, resid)
        torch.cuda.synchronize()
        assert (_u32(pred[0]) == opred).all()
        fail = (_u32(resid[0]) & 1) | ((_u32(pred[0]) != obs0) << 1)
        assert (fail == ofail).all()


def test_output_rules_in_a_batch():
    """Members with different output rules for windows without a converged
    path (0 path 0, 1 fewest unsatisfied checks, 2 committed checks first)
    in one batch: each member equals its own per-decoder path, and a rule-2
    member equals the oracle."""
    mem = []
    for i, (key, R, W, n) in enumerate(MEMBERS):
        d = qdec.Dem(CODES[key], P, R)
        params = preset("configured", k_guess=3, p=P, W=W, fallback=i % 3)
        dec = qdec.Decoder(d, params, max_shots=n)
        det, obs = d.sample(seed=950 + i, shot_offset=0, n_shots=n)
        mem.append(dict(key=key, R=R, W=W, n=n, dem=d, params=params, dec=dec, det=det, obs=obs))
    b = qdec.Batch([m["dec"] for m in mem])
    det, pred, resid = _fresh(mem)
    n = [m["n"] for m in mem]
    for j in range(b.n_steps):
        b.step(j, det, n, pred, resid)
    _check(mem, det, pred, resid)
    m = mem[2]  # [[90]], W = 4, rule 2
    assert m["params"]["fallback"] == 2
    o = oracle_dem(m["key"], P, m["R"])
    det0, obs0 = o.sample(952, 0, m["n"])
    ofail, opred, _ = o.run_shots(m["params"], det0, obs0, threads=8)
    assert (_u32(pred[2]) == opred).all()
    fail = (_u32(resid[2]) & 1) | ((_u32(pred[2]) != obs0) << 1)
    assert (fail == ofail).all()
