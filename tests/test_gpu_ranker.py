"""GPU tests of the learned decimation ranker (the stand-in for the argmin of
Alg. 1; no counterpart in the paper).

* Decoding with a ranker is bit-exact to the oracle (both launch shapes,
  corrections, decision logs, final statuses): the tensor-core layer 1 is
  exact by the parameter grids and layer 2 runs in one fixed FP32 order.
* The candidate records the decode kernel writes equal the oracle's.
* Window-local samples: the detector placement and fault bits agree with
  the window matrix and with qd_wms_sample.
* The training kernel's gradient matches the FP64 reference; on grid-rounded
  parameters it runs on the tensor cores and its scores equal the oracle's
  bit for bit.
* A ranker trained on the decoder's own records gives fewer logical
  failures than Alg. 1 on the same held-out memory shots.
"""
import numpy as np
import pytest

from conftest import oracle_dem
from oracle import oracle as O
from oracle import ranker_ref
from paper_2403_18901_gb300 import build as qbuild
from paper_2403_18901_gb300 import qdec
from paper_2403_18901_gb300 import ranker as rk
from paper_2403_18901_gb300.workloads import CODES, preset

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qbuild.build()
    qdec.lib()


def _random_ranker(seed, coarse=False):
    rng = np.random.default_rng(seed)
    p = np.zeros(641, np.float32)
    if coarse:  # few distinct scores: many ties
        p[:512] = rng.integers(-1, 2, 512) * (rng.random(512) < 0.1)
        p[576:640] = rng.integers(-1, 2, 64)
    else:
        p[:512] = rng.normal(0, 0.6, 512)
        p[512:576] = rng.normal(0, 4, 64)
        p[576:640] = rng.normal(0, 0.5, 64)
    p[640] = 0.125
    return p


@pytest.mark.parametrize("key,R,k_guess,mode,seed,coarse", [
    ("72", 6, 3, 1, 11, False), ("72", 6, 3, 2, 12, True),
    ("144", 12, 4, 1, 13, False), ("144", 12, 4, 2, 14, False),
])
def test_ranker_decode_bit_exact(key, R, k_guess, mode, seed, coarse):
    from test_gpu_parity import _pipeline
    params = preset("configured", k_guess=k_guess, p=0.004)
    n = 96 if key == "72" else 48
    _pipeline(key, R, 0.004, params, n, seed, trace_windows=(0, 1, 2), mode=mode,
              ranker=_random_ranker(seed, coarse))


@pytest.mark.parametrize("mode", [1, 2])
def test_ranker_bb288_bit_exact(mode):
    """[[288,12,18]] with (3,1) windows and the decoder of p = 0.002
    (low-error mode; D_max 40 on the main path, 20 steps after the last
    guess), the ranker choosing the decimated VN in both launch shapes, on
    shots at p = 0.003 (so that most windows run GDG): corrections, decision
    logs and final statuses equal the oracle's."""
    from test_gpu_parity import _pipeline
    params = preset("configured", k_guess=4, p=0.002, d_max_main=40, d_max_other=24)
    assert params["low_error_mode"]
    _pipeline("288", 3, 0.003, params, 24 if mode == 1 else 8, 288_21, trace_windows=(0, 1), mode=mode,
              ranker=_random_ranker(288))


def test_ranker_low_error_mode_bit_exact():
    from test_gpu_parity import _pipeline
    params = preset("configured", k_guess=3, p=0.002)
    assert params["low_error_mode"]
    _pipeline("72", 6, 0.004, params, 96, 21, trace_windows=(1,), mode=1, ranker=_random_ranker(21))


def _bits(words, n):
    idx = np.arange(n)
    return ((words[..., idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)


def _window_setup(key="72", R=6, p=0.004, k=1):
    o = oracle_dem(key, p, R)
    d = qdec.Dem(CODES[key], p, R)
    params = preset("configured", k_guess=3 if key == "72" else 4, p=p)
    dec = qdec.Decoder(d, params, max_shots=1024)
    return o, d, params, dec


def test_window_sample_consistent():
    from paper_2403_18901_gb300.learn import Wms
    o, d, params, dec = _window_setup()
    k, n = 1, 300
    win = o.window(params["W"], params["F"], k)
    det = torch.zeros((n, d.det_words), dtype=torch.int32, device="cuda")
    fault = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
    dec.window_sample(k, 99, 1000, n, det, fault)
    wms = Wms(dec, k, 1, 1)
    synd = wms.sample(99, 1000, n)
    torch.cuda.synchronize()
    db = _bits(det.cpu().numpy().view(np.uint32), o.n_det)
    fb = _bits(fault.cpu().numpy().view(np.uint32), win["n_cols"])
    sb = _bits(synd.cpu().numpy().view(np.uint32), win["n_rows"])
    r0 = win["r0"] * o.w
    assert not db[:, :r0].any() and not db[:, r0 + win["n_rows"]:].any()
    assert (db[:, r0:r0 + win["n_rows"]] == sb).all()
    for s in range(n):
        acc = np.zeros(win["n_rows"], np.uint8)
        for c in np.nonzero(fb[s])[0]:
            acc[win["col_rows"][win["col_ptr"][c]:win["col_ptr"][c + 1]]] ^= 1
        assert (acc == sb[s]).all()
    assert fb.sum() > 0


@pytest.mark.parametrize("use_ranker", [False, True])
def test_dump_matches_oracle(use_ranker):
    o, d, params, dec = _window_setup()
    k, n = 1, 160
    ranker = _random_ranker(5) if use_ranker else None
    if ranker is not None:
        dec.set_ranker(ranker)
    recs, labels, total = rk.collect(dec, k, 7, 0, n, 1 << 18)
    assert total == recs.shape[0] and total > 0
    g = recs.cpu().numpy().view(O.RANK_REC).reshape(-1)
    # regenerate the same samples on the host side of the test
    det = torch.zeros((n, d.det_words), dtype=torch.int32, device="cuda")
    fault = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
    dec.window_sample(k, 7, 0, n, det, fault)
    win = o.window(params["W"], params["F"], k)
    r0 = win["r0"] * o.w
    db = _bits(det.cpu().numpy().view(np.uint32), o.n_det)
    fb = _bits(fault.cpu().numpy().view(np.uint32), win["n_cols"])
    want = []
    for s in range(n):
        dump = np.zeros(50000, O.RANK_REC)
        _, info, _ = o.decode_window(params, k, db[s, r0:r0 + win["n_rows"]], ranker=ranker, dump=dump)
        r = dump[:info["n_dump"]].copy()
        r["shot"] = s
        want.append(r)
    want = np.concatenate(want)
    assert want.shape[0] == g.shape[0]
    order = lambda a: np.lexsort((a["wcol"], a["depth"], a["shot"]))
    a, b = g[order(g)], want[order(want)]
    for f in ("shot", "wcol", "depth", "path", "flags"):
        assert (a[f] == b[f]).all(), f
    assert (a["x"] == b["x"]).all()
    lab = labels.cpu().numpy()[order(g)]
    assert (lab == fb[a["shot"], a["wcol"]]).all()


def test_training_gradient_matches_fp64():
    rng = np.random.default_rng(3)
    n = 3000
    recs = np.zeros(n, O.RANK_REC)
    recs["x"][:, :5] = rng.integers(-40, 41, (n, 5)) * 0.5
    recs["x"][:, 5] = rng.integers(0, 8, n)
    recs["x"][:, 6] = rng.integers(3, 7, n)
    recs["x"][:, 7] = rng.integers(0, 3, n)
    y = (rng.random(n) < 0.2).astype(np.uint8)
    p = rng.normal(0, 0.3, 641).astype(np.float32)
    rt = torch.from_numpy(recs.view(np.uint8).reshape(n, 48)).cuda()
    yt = torch.from_numpy(y).cuda()
    pt = torch.from_numpy(p).cuda()
    for quant in (False, True):
        gg, loss = rk.grad(pt, rt, yt, quantize=quant, pos_weight=4.0, scale=1.0)
        g64, l64 = ranker_ref.grad(p.astype(np.float64), recs["x"], y, pos_weight=4.0, quant=quant)
        assert np.allclose(loss.cpu().numpy(), l64, rtol=1e-4, atol=1e-5)
        assert np.abs(gg.cpu().numpy() - g64).max() <= 1e-3 * np.abs(g64).max()
        sc, _ = rk.evaluate(pt, rt, None, quantize=quant)
        s64 = ranker_ref.forward(p, recs["x"], quant=quant)
        assert np.allclose(sc.cpu().numpy(), s64, rtol=1e-5, atol=1e-4)
    # the tensor-core training kernel scores grid-rounded parameters exactly
    # as the oracle (and the decoder) do: exact layer 1, layer 2 in the same
    # fixed FP32 order
    sc, _ = rk.evaluate(pt, rt, None, quantize=True)
    so = O.ranker_score(p, recs["x"])
    assert (sc.cpu().numpy() == so).all()


def test_trained_ranker_lowers_logical_failures():
    """What the trained ranker gains over Alg. 1: fewer logical failures on
    the same held-out [[144,12,12]] memory shots (W=3, p=0.003, 12 rounds)."""
    d = qdec.Dem(CODES["144"], 0.003, 12)
    params = preset("configured", k_guess=4, p=0.003)
    n = 16384
    dec = qdec.Decoder(d, params, max_shots=n)
    p, info = rk.train(dec, 1, steps=300, shots_per_round=4096, rounds=4, cap=1 << 24, batch=65536,
                       lr=1e-2, seed=404)
    det, obs = d.sample(seed=777, shot_offset=0, n_shots=n)

    def failures():
        pr = torch.zeros(n, dtype=torch.int32, device="cuda")
        fl = torch.zeros(n, dtype=torch.int32, device="cuda")
        nf = torch.zeros(1, dtype=torch.int64, device="cuda")
        dec.decode_all(det.clone(), obs, n, pr, fl, nf)
        return int(nf.item())

    plain = failures()
    dec.set_ranker(p.cpu().numpy())
    ranked = failures()
    dec.set_ranker(None)
    assert failures() == plain  # removing the ranker restores Alg. 1
    assert ranked < plain, (ranked, plain, info)
