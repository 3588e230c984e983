"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Plain GDG is bit-exact by construction (FP32 with fixed per-node summation
order, no FMA, lexicographic argmin ties, one fixed peeling order, exact
FP64 path metrics), so every comparison below is exact: sampled shots,
per-window corrections, winning path, per-path status / depth / iterations /
path metric, the per-step decision log (selected VN, value, aggressive and
peeled counts), every path's final VN status, the ranked short columns, the
observable predictions and the failure flags.
"""
import numpy as np
import pytest

from conftest import oracle_dem
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


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _bits(words, n):
    idx = np.arange(n)
    return ((words[..., idx // 32] >> (idx % 32).astype(np.uint32)) & 1).astype(np.uint8)


def _apply_commit(det_row, o, win, corr_bits):
    """Test-side commit (Eq. (10)) with the oracle's DEM columns."""
    for i in np.nonzero(corr_bits[:win["n_commit"]])[0]:
        c = win["gcols"][i]
        for d in o.col_dets[o.col_ptr[c]:o.col_ptr[c + 1]]:
            det_row[d >> 5] ^= np.uint32(1) << np.uint32(d & 31)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("key,R,n,off", [("72", 6, 3000, 0), ("144", 12, 700, 12345)])
def test_sampler_bit_exact(key, R, n, off):
    d = qdec.Dem(CODES[key], 0.003, R)
    o = oracle_dem(key, 0.003, R)
    det, obs = d.sample(seed=2024, shot_offset=off, n_shots=n)
    torch.cuda.synchronize()
    od, oo = o.sample(2024, off, n)
    assert (_u32(det) == od).all()
    assert (_u32(obs) == oo).all()


def _pipeline(key, R, p, params, n, seed, trace_windows=(), mode=0, weights=None, ranker=None, capacity=None):
    """Run both implementations window by window on the same oracle-sampled
    shots; compare everything.  mode: launch shape (0 automatic, 1 one warp per
    decision path, 2 one CTA per decision path).  Returns (oracle fail, gpu fail)."""
    if capacity is None:
        o = oracle_dem(key, p, R)
    else:
        from oracle import oracle as O
        o = O.OracleDEM(CODES[key], capacity[0], 0, capacity=capacity)
    d = qdec.Dem(CODES[key], p, R, capacity=capacity)
    dec = qdec.Decoder(d, params, max_shots=n)
    dec.set_launch(mode)
    if weights is not None:
        for k, w in weights.items():
            dec.set_weights(k, torch.from_numpy(w).cuda())
    if ranker is not None:
        dec.set_ranker(ranker)
    det0, obs0 = o.sample(seed, 0, n)
    ofail, opred, ocorr = o.run_shots(params, det0, obs0, threads=8, want_corr=True, weights=weights,
                                       ranker=ranker)
    det = _to_dev(det0)
    obs = _to_dev(obs0)
    corr = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    pred = torch.zeros(n, dtype=torch.int32, device="cuda")
    resid = torch.zeros(n, dtype=torch.int32, device="cuda")
    fail = torch.zeros(n, dtype=torch.int32, device="cuda")
    host_det = det0.copy()
    n_gdg = 0
    for k in range(dec.n_windows):
        win = dec.window_info(k)
        owin = o.window(params["W"], params["F"], k, params.get("merge_h1", 0))
        assert (win["gcols"] == owin["gcols"]).all()
        assert win["n_commit"] == owin["n_commit"]
        tr = None
        if k in trace_windows:
            tr = torch.zeros((n, dec.trace_bytes), dtype=torch.uint8, device="cuda")
        dec.decode_window(k, det, n, corr, status, tr)
        g = _u32(corr)
        cw_o = ocorr.shape[2]
        if tr is not None:
            trn = tr.cpu().numpy()
            st = status.cpu().numpy()
            s_all = _bits(host_det, o.n_det)
            for sh in range(n):
                synd = s_all[sh, win["r0"] * o.w: win["r0"] * o.w + win["n_rows"]]
                oc, oinfo, otr = o.decode_window(params, k, synd, trace=True, weights=weights, ranker=ranker)
                gt = dec.parse_trace(trn[sh])
                assert gt["head"][0] == int(oinfo["prebp_converged"])
                assert gt["head"][3] == oinfo["prebp_iters"]
                if oinfo["prebp_converged"]:
                    assert st[sh] == -1
                    continue
                n_gdg += 1
                ns = oinfo["n_short"]
                assert gt["head"][1] == oinfo["winner"] and gt["head"][2] == ns
                assert st[sh] == (oinfo["winner"] if oinfo["winner"] >= 0 else -2)
                assert (gt["short_cols"][:ns] == otr["short_cols"]).all()
                for b, ob in enumerate(otr["branches"]):
                    gb = gt["branches"][b]
                    assert (gb["status"], gb["depth"], gb["iters"]) == ob[:3], (sh, b)
                    assert gb["pm"] == ob[3] or (np.isinf(gb["pm"]) and np.isinf(ob[3]))
                    ost = otr["steps"][b]
                    for D, rec in enumerate(ost):
                        grec = gt["steps"][b][D]
                        assert (grec["g"], grec["value"], grec["n_agg"], grec["n_peel"]) == rec, (sh, b, D)
                    assert (gt["final_status"][b][:ns] == otr["final_status"][b]).all(), (sh, b)
        assert (g[:, :cw_o] == ocorr[:, k, :]).all(), f"window {k}: corrections differ"
        dec.commit(k, corr, n, det, pred, resid)
        gbits = _bits(g, win["n_cols"])
        for sh in range(n):
            _apply_commit(host_det[sh], o, owin, gbits[sh])
    torch.cuda.synchronize()
    if trace_windows:
        assert n_gdg > 0, "no traced window ran GDG; pick another seed"
    assert (_u32(det) == host_det).all(), "committed syndromes differ"
    qdec._check(qdec.lib().qd_evaluate(qdec._ptr(pred), qdec._ptr(obs), qdec._ptr(resid), n,
                                       qdec._ptr(fail), None, qdec._stream(None)))
    gfail = _u32(fail)
    assert (_u32(pred) == opred).all()
    assert (gfail == ofail).all()
    assert dec.counters()[4] == 0  # every bulk (TMA) staging copy completed
    return ofail, gfail


@pytest.mark.parametrize("pname", ["configured", "paper"])
def test_bb72_pipeline_bit_exact(pname):
    params = preset(pname, k_guess=3)
    _pipeline("72", 6, 0.003, params, n=400, seed=72_003, trace_windows=(0, 2, 4))


def test_bb72_low_error_mode_and_k0():
    params = preset("paper", k_guess=0, p=0.002)
    assert params["low_error_mode"] == 1
    _pipeline("72", 6, 0.002, params, n=300, seed=72_002, trace_windows=(1,))
    params = preset("configured", k_guess=2, low_error_mode=1, peel_at_init=0)
    _pipeline("72", 6, 0.003, params, n=200, seed=72_004, trace_windows=(3,))


def test_bb144_pipeline_bit_exact():
    params = preset("configured", k_guess=4)
    _pipeline("144", 12, 0.003, params, n=150, seed=144_003, trace_windows=(0, 5, 10), mode=1)


@pytest.mark.parametrize("key,R,k,pname,n", [("144", 12, 4, "configured", 40), ("72", 6, 3, "paper", 64),
                                             ("144", 12, 5, "paper", 24)])
def test_path_per_cta_launch_bit_exact(key, R, k, pname, n):
    """The latency launch (one CTA per decision path, last CTA decides)."""
    _pipeline(key, R, 0.003, preset(pname, k_guess=k), n=n, seed=5150 + n,
              trace_windows=(0, 1, 2, 3), mode=2)


@pytest.mark.parametrize("key,R,pname,k,cluster,cps", [("144", 12, "configured", 4, 8, 16),
                                                       ("72", 6, "paper", 3, 8, 16),
                                                       ("72", 6, "configured", 1, 2, 2)])
def test_path_launch_splits_the_prebp_over_a_cluster(key, R, pname, k, cluster, cps):
    """Path mode runs each shot's pre-BP on a cluster of CTAs (the paths,
    rounded up to whole clusters); the parity tests above run this launch."""
    d = qdec.Dem(CODES[key], 0.003, R)
    dec = qdec.Decoder(d, preset(pname, k_guess=k), max_shots=4)
    info = dec.launch_info(1)
    assert info["path_cluster"] == cluster and info["path_ctas_per_shot"] == cps


def test_bb144_paper_preset_k5_bit_exact():
    params = preset("paper", k_guess=5)
    _pipeline("144", 12, 0.004, params, n=60, seed=144_004, trace_windows=tuple(range(11)))


def test_other_window_shapes():
    # (4,2) windows on [[90]] and a single global window on [[72]]
    _pipeline("90", 4, 0.003, preset("paper", k_guess=2, W=4, F=2), n=60, seed=90_003,
              trace_windows=(0,))
    _pipeline("72", 3, 0.003, preset("paper", k_guess=1, W=4, F=1), n=60, seed=72_005,
              trace_windows=(0,))


def test_host_buffer_path_equals_device_path():
    params = preset("configured", k_guess=3)
    o = oracle_dem("72", 0.003, 6)
    d = qdec.Dem(CODES["72"], 0.003, 6)
    n = 257  # ragged batch
    dec = qdec.Decoder(d, params, max_shots=512)
    det0, obs0 = o.sample(99, 0, n)
    ofail, opred, _ = o.run_shots(params, det0, obs0, threads=8)
    pred, fail, nf = dec.decode_host(det0, obs0)
    assert (pred == opred).all() and (fail == ofail).all()
    assert nf == int((ofail > 0).sum())
    # device path with the library's own scratch
    det = _to_dev(det0)
    obs = _to_dev(obs0)
    pr = torch.zeros(n, dtype=torch.int32, device="cuda")
    fl = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    dec.decode_all(det, obs, n, pr, fl, cnt)
    torch.cuda.synchronize()
    assert (_u32(pr) == opred).all() and (_u32(fl) == ofail).all()
    assert int(cnt.item()) == nf


def test_edge_cases():
    params = preset("configured", k_guess=3)
    d = qdec.Dem(CODES["72"], 0.003, 6)
    dec = qdec.Decoder(d, params, max_shots=64)
    # empty batch is a no-op
    pred, fail, nf = dec.decode_host(np.zeros((0, d.det_words), np.uint32), np.zeros(0, np.uint32))
    assert len(pred) == 0 and nf == 0
    # all-zero syndromes: zero corrections, no failures
    det = np.zeros((64, d.det_words), np.uint32)
    pred, fail, nf = dec.decode_host(det, np.zeros(64, np.uint32))
    assert (pred == 0).all() and (fail == 0).all() and nf == 0
    # one shot
    o = oracle_dem("72", 0.003, 6)
    det1, obs1 = o.sample(5, 7, 1)
    ofail, opred, _ = o.run_shots(params, det1, obs1)
    pred, fail, _ = dec.decode_host(det1, obs1)
    assert (pred == opred).all() and (fail == ofail).all()
    # batch above max_shots is refused
    with pytest.raises(qdec.QdError) as e:
        dec.decode_host(np.zeros((65, d.det_words), np.uint32), np.zeros(65, np.uint32))
    assert e.value.code == qdec.QD_EINVAL
    # unsupported parameters are refused at create time
    with pytest.raises(qdec.QdError) as e:
        qdec.Decoder(d, dict(params, iters_per_step=3), 8)
    assert e.value.code == qdec.QD_EUNSUPPORTED


def test_repeatable():
    """Same inputs twice -> identical outputs (no races in the peel / argmin)."""
    params = preset("configured", k_guess=4)
    o = oracle_dem("144", 0.003, 12)
    d = qdec.Dem(CODES["144"], 0.003, 12)
    dec = qdec.Decoder(d, params, max_shots=300)
    det0, obs0 = o.sample(31337, 0, 300)
    a = dec.decode_host(det0, obs0)
    b = dec.decode_host(det0, obs0)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


@pytest.mark.parametrize("mode", [1, 2])
def test_learned_weights_bit_exact(mode):
    """Weighted min-sum (per-edge, per-iteration weights in place of alpha) in
    the pre-BP and in every decision path, both launch shapes."""
    o = oracle_dem("72", 0.003, 6)
    params = preset("configured", k_guess=3)
    rng = np.random.default_rng(123)
    T = 7  # iterations past T reuse row T, exercised by the 100-iteration pre-BP
    weights = {}
    for k in range(o.n_windows(3, 1)):
        ne = o.window(3, 1, k)["n_edges"]
        weights[k] = rng.uniform(0.45, 0.9, size=(T, ne)).astype(np.float32)
    _pipeline("72", 6, 0.003, params, n=64 if mode == 2 else 200, seed=4242,
              trace_windows=(0, 1, 2, 3, 4), mode=mode, weights=weights)


@pytest.mark.parametrize("mode", [1, 2])
def test_bb288_bit_exact(mode):
    """[[288,12,18]]: the shortened window (864 columns) leaves room for fewer
    decision-path slots per CTA; both launch shapes stay bit-exact."""
    params = preset("configured", k_guess=4, p=0.002)
    _pipeline("288", 3, 0.002, params, n=40, seed=288_002, trace_windows=(0, 1), mode=mode)


@pytest.mark.parametrize("mode", [1, 2])
def test_full_decision_tree_bit_exact(mode):
    """The decision tree of Fig. 2 with its side branches (D_split = 4..10,
    22 paths), paper preset, both launch shapes, every path's log compared."""
    params = preset("paper", k_guess=4, p=0.004)
    assert params["side_max"] == 10
    _pipeline("144", 12, 0.004, params, n=48 if mode == 1 else 24, seed=144_444, trace_windows=(1, 6, 10),
              mode=mode)


def test_bb288_paper_tree_bit_exact():
    """[[288,12,18]] with its Sec. IV-C tree: D_max 40, tree depth 5, side
    branches up to D_split = 20, 20 steps after a split (47 paths)."""
    params = preset("paper", 5, p=0.002, d_max_main=40, d_max_other=25, side_max=20, n_pre=16)
    _pipeline("288", 3, 0.003, params, n=16, seed=288_003, trace_windows=(0, 1), mode=1)


@pytest.mark.parametrize("key,pd,ps,mode", [("288", 0.04, 1e-3, 1), ("288", 0.05, 3e-3, 2), ("144", 0.06, 0.0, 1)])
def test_code_capacity_bit_exact(key, pd, ps, mode):
    """Appendix workloads: BSC(p_d) decoded with H_X, and [H_X | I] with
    syndrome noise; one window over the whole matrix (plus the residue-only
    window of the single-shot model), GDG with the appendix's tree (D_max 40,
    depth-5 guessing tree, side branches to D_split 20, 47 paths)."""
    from paper_2403_18901_gb300.workloads import CAPACITY
    _pipeline(key, 0, pd, dict(CAPACITY), n=64 if mode == 1 else 24, seed=288_100, trace_windows=(0,), mode=mode,
              capacity=(pd, ps))


# a [[18,4]] bivariate-bicycle code (l = m = 3, A = 1 + y + y^2, B = 1 + y + x):
# windows of 18 / 27 columns and 9 / 18 checks
TINY18 = dict(name="[[18,4]]", n=18, k=4, l=3, m=3, A=[(0, 0), (0, 1), (0, 2)], B=[(0, 0), (0, 1), (1, 0)])


@pytest.mark.parametrize("ps,mode", [(0.0, 1), (0.02, 2), (0.0, 2)])
def test_tiny_windows_bit_exact(monkeypatch, ps, mode):
    """Windows of fewer than 256 columns (the small network of the ranking
    sort) and fewer checks than a warp round, in both launch shapes; path
    mode runs 6 paths on two clusters of 4 CTAs, two of them idle."""
    from paper_2403_18901_gb300.workloads import CAPACITY
    monkeypatch.setitem(CODES, "tiny18", TINY18)
    params = dict(CAPACITY, k_guess=2, side_max=4, d_max_main=12, d_max_other=8)
    if mode == 2:
        d = qdec.Dem(TINY18, 0.05, 0, capacity=(0.05, ps))
        info = qdec.Decoder(d, params, max_shots=4).launch_info(0)
        assert info["path_cluster"] == 4 and info["path_ctas_per_shot"] == 8
    _pipeline("tiny18", 0, 0.05, params, n=200 if mode == 1 else 40, seed=18_004, trace_windows=(0,), mode=mode,
              capacity=(0.05, ps))


def test_bb72_2000_shots_bit_exact():
    """[[72,12,6]], 6 rounds, p = 0.003, 2000 seeded shots (seed 72003):
    corrections of every window, committed syndromes, predictions and failures."""
    from paper_2403_18901_gb300.workloads import WORKLOADS
    w = WORKLOADS["bb72_r6_p3e-3"]
    _pipeline(w["code"], w["rounds"], w["p"], preset("configured", k_guess=w["k_guess"], p=w["p"]), n=w["shots"],
              seed=w["seed"])


@pytest.mark.parametrize("p,seed", [(0.002, 144_002), (0.003, 144_003)])
def test_bb144_2000_shot_subset_bit_exact(p, seed):
    """[[144,12,12]], 12 rounds, k = 4: the 2000-shot subset of the LER sweep,
    every window's corrections, committed syndromes, predictions, failures."""
    _pipeline("144", 12, p, preset("configured", k_guess=4, p=p), n=2000, seed=seed, mode=1)


def test_other_window_shapes_of_the_paper():
    """Sec. IV-C: (5,2) windows for [[144,12,12]] and (4,1) windows for
    [[288,12,18]] with the paper's decision tree for that code."""
    _pipeline("144", 6, 0.003, preset("paper", k_guess=4, W=5, F=2), n=40, seed=144_052, trace_windows=(0, 1),
              mode=1)
    p288 = preset("paper", 5, p=0.002, d_max_main=40, d_max_other=25, side_max=20, n_pre=16, W=4, F=1)
    _pipeline("288", 4, 0.003, p288, n=12, seed=288_041, trace_windows=(0, 1), mode=1)


@pytest.mark.parametrize("mode", [1, 2])
def test_message_restart_at_splits_bit_exact(mode):
    """reinit_on_split: side branches and odd tree ids restart their messages
    where they split off (the appendix's snapshot implementation)."""
    params = preset("paper", k_guess=4, p=0.004, reinit_on_split=1)
    _pipeline("144", 12, 0.004, params, n=40 if mode == 1 else 20, seed=144_555, trace_windows=(1, 5), mode=mode)


def test_message_restart_with_learned_weights_bit_exact():
    """The learned weights' iteration count restarts with the messages."""
    params = preset("configured", k_guess=3, p=0.003, reinit_on_split=1)
    o = oracle_dem("72", 0.003, 6)
    rng = np.random.default_rng(9)
    weights = {k: rng.uniform(0.45, 0.9, size=(25, o.window(3, 1, k)["n_edges"])).astype(np.float32)
               for k in range(o.n_windows(3, 1))}
    _pipeline("72", 6, 0.003, params, n=120, seed=7272, trace_windows=(0, 2), mode=1, weights=weights)



def test_path_state_in_global_memory_bit_exact():
    """Launch mode 3: the pre-BP scratch and the decision-path states of every
    CTA in global memory (the shape of windows too large for shared memory)."""
    _pipeline("144", 12, 0.003, preset("configured", k_guess=4, p=0.003), n=120, seed=144_333,
              trace_windows=(0, 5), mode=3)
    _pipeline("72", 6, 0.004, preset("paper", k_guess=3, p=0.004), n=120, seed=72_333, trace_windows=(1,), mode=3)


def test_window_too_large_for_shared_memory_bit_exact():
    """[[288,12,18]] with (6,1) windows: the pre-BP scratch of a 6-round window
    (8.6k columns) exceeds shared memory, so the decoder streams every CTA's
    union region through global memory on its own."""
    params = preset("configured", k_guess=2, p=0.002, W=6, F=1, d_max_main=12)
    _pipeline("288", 6, 0.002, params, n=8, seed=288_006, trace_windows=(0,), mode=1)


@pytest.mark.parametrize("key,R,n,mode,tw", [("72", 6, 60, 1, (0, 2)), ("144", 12, 16, 1, (1,)),
                                             ("144", 12, 8, 2, (0,))])
def test_initial_bp_as_first_step_bit_exact(key, R, n, mode, tw):
    """The second reading of "100 initial BP iterations": no pre-BP, no
    shortening, GDG on the whole window with a first step of 100 iterations.
    The [[144]] whole-window path states do not fit shared memory in the
    throughput shape, so they run in global memory."""
    params = preset("configured", k_guess=4 if key == "144" else 3, p=0.003, n_pre=0, shorten=0, iters_first=100)
    _pipeline(key, R, 0.003, params, n=n, seed=int(key) * 1000 + 7, trace_windows=tw, mode=mode)


@pytest.mark.parametrize("pname,p,n,mode", [("configured", 0.003, 400, 2), ("configured", 0.002, 300, 2),
                                            ("paper", 0.004, 300, 2), ("configured", 0.003, 300, 1)])
def test_shared_prefixes_change_nothing(pname, p, n, mode):
    """Shot mode resumes decision paths from snapshots of the prefixes they
    share with paths queued before them (mode 1), and parks and resumes
    paths at step boundaries to balance the warps (mode 2).  Every output -- corrections,
    statuses, the whole per-shot trace (every path's status, depth,
    iterations, metric, step log and final statuses) -- and the per-path work
    count equal those of every path run from the root; only the executed
    work drops."""
    d = qdec.Dem(CODES["144"], p, 12)
    runs = []
    for fork in (mode, 0):
        dec = qdec.Decoder(d, preset(pname, k_guess=4, p=p), max_shots=n)
        dec.set_launch(1)
        dec.set_fork(fork)
        det, _ = d.sample(seed=144_777, shot_offset=0, n_shots=n)
        corr = torch.zeros((n, dec.corr_words), dtype=torch.int32, device="cuda")
        status = torch.zeros(n, dtype=torch.int32, device="cuda")
        pred = torch.zeros(n, dtype=torch.int32, device="cuda")
        resid = torch.zeros(n, dtype=torch.int32, device="cuda")
        out = []
        for k in range(dec.n_windows):
            tr = torch.zeros((n, dec.trace_bytes), dtype=torch.uint8, device="cuda")
            dec.decode_window(k, det, n, corr, status, tr)
            out.append((corr.cpu().numpy().copy(), status.cpu().numpy().copy(), tr.cpu().numpy()))
            dec.commit(k, corr, n, det, pred, resid)
        torch.cuda.synchronize()
        runs.append((out, det.cpu().numpy(), pred.cpu().numpy(), resid.cpu().numpy(), dec.counters_ex()))
    (a, da, pa, ra, ca), (b, db, pb, rb, cb) = runs
    for k, (x, y) in enumerate(zip(a, b)):
        for u, v in zip(x, y):
            assert (u == v).all(), f"window {k} differs"
    assert (da == db).all() and (pa == pb).all() and (ra == rb).all()
    assert list(ca[:5]) == list(cb[:5]) and ca[4] == 0
    assert cb[5] == cb[1]  # from the root: executed = counted
    assert ca[5] < ca[1], "no decision path resumed from a shared prefix"


@pytest.mark.parametrize("merge,pname,mode,n", [(1, "configured", 1, 80), (2, "configured", 1, 80),
                                                (1, "paper", 2, 16), (2, "paper", 1, 60)])
def test_h1_merge_bit_exact(merge, pname, mode, n):
    """The H_1 merge of Sec. III (1: equal restrictions, 2: identity with the
    XOR priors): the GPU host builds the same merged windows as the oracle
    (columns, priors) and decodes them identically."""
    params = preset(pname, k_guess=4, p=0.003, merge_h1=merge)
    _pipeline("144", 12, 0.003, params, n=n, seed=144_900 + 10 * merge + mode, trace_windows=(1, 4), mode=mode)


@pytest.mark.parametrize("pname,mode,n", [("configured", 1, 120), ("configured", 2, 16), ("paper", 1, 120),
                                          ("configured", 3, 60)])
def test_message_reuse_bit_exact(pname, mode, n):
    """Message reuse between windows (Sec. VI): each window's pre-BP starts
    from what the previous window's output path kept; every window's
    corrections, the committed syndromes and the outcomes equal the oracle's,
    in the throughput shape, the path-per-CTA shape and with the path states
    in global memory."""
    params = preset(pname, k_guess=4, p=0.003, reuse_msgs=1)
    _pipeline("144", 12, 0.003, params, n=n, seed=144_610 + mode, mode=mode)


@pytest.mark.parametrize("fb,mode,reuse,n", [(0, 1, 0, 120), (2, 0, 0, 200), (1, 1, 0, 120), (2, 1, 0, 120), (2, 2, 0, 16),
                                             (2, 3, 0, 60), (2, 1, 1, 120), (2, 2, 1, 16)])
def test_fallback_bit_exact(fb, mode, reuse, n):
    """The output of a window without a converged path under the fallback
    rules (fewest unsatisfied checks; committed checks first): every window's
    corrections, the committed syndromes and the outcomes equal the oracle's,
    in every launch shape, with message reuse following the chosen path."""
    params = preset("configured", k_guess=4, p=0.003, fallback=fb, reuse_msgs=reuse)
    tw = (1, 4) if (mode, reuse) == (1, 0) else ()
    _pipeline("144", 12, 0.003, params, n=n, seed=144_740 + 10 * fb + mode + 100 * reuse, trace_windows=tw, mode=mode)
