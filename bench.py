"""Benchmark: sliding-window GDG decoding of [[144,12,12]] BB-code memory
experiments (12 noisy rounds, (3,1) windows, p = 0.003, 2^4 guessing paths)
on the GPU, through the libqdec C ABI.

One step = one complete sliding-window pass (decode + commit of all 11
windows, then the success test) over a batch of shots already resident in HBM.
Metric: windows/s (shots x windows per shot / step time).  Also reported:
the same metric end to end through qd_decode_shots_host (host buffers, copies
inside the timed region), per-window latency p50/p99 with one shot per window
step, the roofline fraction of the decode kernel and the CPU oracle's
throughput on this machine's cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank decodes its own shots (replicas, no collective on the
data path); rank 0 prints the JSON line with the max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

CODE_KEY, ROUNDS, P_PHYS, K_GUESS = "144", 12, 0.003, 4
METRIC = "[[144,12,12]] W=3 windows/s"
OPS_PER_EDGE_ITER = 10  # FP32/ALU operations of Eq. (1)-(3) per edge and iteration
BYTES_PER_EDGE_ITER = 16  # explicit-message shared-memory bytes per edge and iteration (4 B x 2 read + 2 written)
# DRAM bytes (read + write) of one decode_shot_kernel launch of the default
# workload, keyed by (preset, shots per launch, output rule), from one ncu
# capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum;
# see profiles/decode_shot_kernel_bb144_w3_p3e-3_configured.md).  Reported
# only for that workload; per launch, like "achieved".
TRAFFIC_PER_LAUNCH = {("configured", 20000, 2): 6414336 + 3036823040}
# Unit utilisation of the same kernel from one ncu --set full capture of a
# 4000-shot launch of this workload (same profile file): the shared-memory
# data pipe (l1tex__data_pipe_lsu_wavefronts_mem_shared, % of peak) and the
# ALU pipe (sm__pipe_alu_cycles_active, % of peak), as fractions.  What bounds
# the kernel in hardware terms; the algorithmic fractions above count only
# the method's arithmetic and message bytes.
PIPES_PER_LAUNCH = {("configured", 2): {"shared_data_pipe": 0.695, "alu_pipe": 0.574}}


FALLBACK_NAMES = {0: "path 0's estimate", 1: "fewest unsatisfied checks",
                  2: "fewest unsatisfied committed checks, then all"}


def workload_name(preset_name, fallback=0):
    return (f"[[144,12,12]] BB memory, {ROUNDS} rounds, (3,1) windows, p={P_PHYS}, "
            f"GDG 2^{K_GUESS} paths, preset={preset_name}, "
            f"no converged path -> {FALLBACK_NAMES[fallback]}")


def with_fallback(preset, fallback):
    """The workloads' preset() with the output rule for windows without a
    converged path set to `fallback` unless a caller overrides it."""
    def p(name, k_guess, p=None, **over):
        return preset(name, k_guess, p, **dict({"fallback": fallback}, **over))
    return p


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdg", choices=["gdg", "reference"])
    ap.add_argument("--shots", type=int, default=20000, help="shots per step per GPU")
    ap.add_argument("--preset", default="configured", choices=["configured", "paper"])
    ap.add_argument("--fallback", type=int, default=2, choices=[0, 1, 2],
                    help="output of a window without a converged decision path: 0 path 0's estimate, "
                         "1 fewest unsatisfied checks, 2 fewest unsatisfied committed checks, then all")
    ap.add_argument("--latency-shots", type=int, default=1000,
                    help="shots of the latency measurements (x windows per shot >= 1e4 windows)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--seed", type=int, default=144_003)
    ap.add_argument("--train-steps", type=int, default=245,
                    help="Adam steps per window type for the learned weights (0: skip); "
                         "245 x 4096 = 1.0e6 samples per window type")
    ap.add_argument("--train-batch", type=int, default=4096)
    ap.add_argument("--ranker-steps", type=int, default=1500,
                    help="Adam steps of the decimation ranker (0: skip)")
    ap.add_argument("--paper-shots", type=int, default=20000,
                    help="shots of the paper-preset (Fig. 2 tree) measurement (0: skip)")
    ap.add_argument("--sweep-shots", type=int, default=100000,
                    help="shots per physical error rate of the [[144]] LER sweep (0: skip)")
    ap.add_argument("--capacity-shots", type=int, default=20000,
                    help="shots of each appendix code-capacity measurement (0: skip)")
    ap.add_argument("--batch-shots", type=int, default=30000,
                    help="shots per code of the batched uneven workload (0: skip)")
    ap.add_argument("--ranker-shots", type=int, default=4096,
                    help="window samples per collection round for the ranker (4 rounds)")
    ap.add_argument("--r288-shots", type=int, default=50000,
                    help="[[288,12,18]] shots of the ranker-vs-Alg. 1 measurement (0: skip)")
    ap.add_argument("--r288-latency-shots", type=int, default=200)
    ap.add_argument("--reading-shots", type=int, default=2000,
                    help="shots of the second reading of the configured pre-BP (0: skip the readings section)")
    ap.add_argument("--shape-shots", type=int, default=5000,
                    help="shots of each other window shape of Sec. IV-C (0: skip)")
    return ap.parse_args()


def wilson(k, n, z=1.96):
    if n == 0:
        return (0.0, 1.0)
    ph = k / n
    c = (ph + z * z / (2 * n)) / (1 + z * z / n)
    h = z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / (1 + z * z / n)
    return (max(0.0, c - h), min(1.0, c + h))


def per_round(P, R=ROUNDS):
    return 1.0 - (1.0 - P) ** (1.0 / R)


def ler_entry(f, n, R=ROUNDS):
    lo, hi = wilson(f, n)
    return {"failures": int(f), "shots": int(n), "p_L": per_round(f / n, R) if n else None,
            "wilson95": [per_round(lo, R), per_round(hi, R)]}


def decode_pass(torch, dec, dem, seed, n_total, batch, offset=0):
    """Whole sliding-window passes over n_total fresh shots in batches (one
    warm-up batch first); returns (GPU seconds of the decode passes,
    failures, failures of Eq. (11) alone, GDG windows)."""
    pred = torch.empty(batch, dtype=torch.int32, device="cuda")
    fail = torch.empty(batch, dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int64, device="cuda")
    det, obs = dem.sample(seed, offset, min(batch, n_total))
    dec.decode_all(det, obs, det.shape[0], pred, fail, nf)  # warm-up
    nf.zero_()
    dec.reset_counters()
    t, done, resid_only = 0.0, 0, 0
    while done < n_total:
        n = min(batch, n_total - done)
        det, obs = dem.sample(seed, offset + done, n)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dec.decode_all(det, obs, n, pred, fail, nf)
        e1.record()
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1000.0
        resid_only += int((fail[:n] == 1).sum().item())
        done += n
    return t, int(nf.item()), resid_only, int(dec.counters()[3])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
def cpu_oracle_rate(params, seconds, seed):
    """The CPU oracle as it stands on all host cores, on a bounded sample of
    the same workload; returns (windows/s, cores, shots, seconds)."""
    from oracle import oracle as O
    from paper_2403_18901_gb300.workloads import CODES
    cores = O.default_threads()
    dem = O.OracleDEM(CODES[CODE_KEY], P_PHYS, ROUNDS)
    nwin = dem.n_windows(params["W"], params["F"])
    chunk = 4 * cores
    shots = 0
    t0 = time.perf_counter()
    off = 0
    while True:
        det, obs = dem.sample(seed + 7, off, chunk)
        dem.run_shots(params, det, obs, threads=cores)
        off += chunk
        shots += chunk
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return shots * nwin / el, cores, shots, el


def run_reference(args):
    """--impl reference: the CPU oracle, timed as it stands on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2403_18901_gb300.workloads import preset
    params = with_fallback(preset, args.fallback)(args.preset, k_guess=K_GUESS)
    from oracle import oracle as O
    from paper_2403_18901_gb300.workloads import CODES
    cores = O.default_threads()
    dem = O.OracleDEM(CODES[CODE_KEY], P_PHYS, ROUNDS)
    nwin = dem.n_windows(params["W"], params["F"])
    n = 2 * cores
    for w in range(args.warmup):
        det, obs = dem.sample(args.seed, 10_000_000 + w * n, n)
        dem.run_shots(params, det, obs, threads=cores)
    times = []
    for s in range(args.steps):
        det, obs = dem.sample(args.seed, s * n, n)
        t0 = time.perf_counter()
        dem.run_shots(params, det, obs, threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * nwin * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "windows/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded DEM sampling)",
        "config": {"workload": workload_name(args.preset, args.fallback), "shots_per_step": n,
                   "windows_per_shot": nwin, "parallelism": f"{cores} host threads"},
        "cpu_baseline": {"value": value, "unit": "windows/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {n} shots"},
        "e2e": {"value": value, "unit": "windows/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def batched_uneven(args, torch, qdec, CODES, preset):
    """[[90,8,10]], [[108,8,10]] and [[144,12,12]] (p = 0.003, d rounds) with
    W = 2 + (shot mod 3): one decoder per (code, W) holding a third of the
    code's shots, all advanced together by qd_batch_step (one decode and one
    commit launch per window step), shapes from qd_batch_autotune, the whole
    window loop replayed as one CUDA graph.  Compared with the same decoders
    run one after another (qd_decode_all each)."""
    p = 0.003
    codes = [("90", 10), ("108", 10), ("144", 12)]
    per = args.batch_shots // 3
    mem = []
    for ci, (key, R) in enumerate(codes):
        dem = qdec.Dem(CODES[key], p, R)
        for W in (2, 3, 4):
            params = preset(args.preset, k_guess=K_GUESS, p=p, W=W)
            dec = qdec.Decoder(dem, params, max_shots=per)
            det, obs = dem.sample(args.seed + 7 * ci, W * per, per)  # disjoint shot ranges per (code, W)
            mem.append(dict(key=key, R=R, W=W, dem=dem, dec=dec, det=det, obs=obs))
    n = [per] * len(mem)
    b = qdec.Batch([m["dec"] for m in mem])
    # autotune the interior step on a slice of the shots; use that shape everywhere it fits
    tune_n = [min(per, 1024)] * len(mem)
    default = b.info(1)
    tune_ms = b.autotune(1, [m["det"] for m in mem], tune_n, reps=1)
    shape = b.info(1)
    for j in range(b.n_steps):
        try:
            b.set_shape(j, shape["warps"], shape["ctas_per_sm"])
        except qdec.QdError:
            pass
    det = [m["det"].clone() for m in mem]
    pred = [torch.zeros(per, dtype=torch.int32, device="cuda") for _ in mem]
    resid = [torch.zeros(per, dtype=torch.int32, device="cuda") for _ in mem]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for j in range(b.n_steps):
            b.step(j, det, n, pred, resid, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for j in range(b.n_steps):
            b.step(j, det, n, pred, resid, stream=s)

    def reset():
        for i, m in enumerate(mem):
            det[i].copy_(m["det"])
            pred[i].zero_()
            resid[i].zero_()

    reset()
    g.replay()  # warm-up
    torch.cuda.synchronize()
    reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1000.0
    windows = sum(per * m["dec"].n_windows for m in mem)
    out_members = []
    for i, m in enumerate(mem):
        pr = pred[i].cpu().numpy().view(np.uint32)
        rs = resid[i].cpu().numpy().view(np.uint32)
        ob = m["obs"].cpu().numpy().view(np.uint32)
        f = int(((rs & 1) | (pr != ob)).astype(bool).sum())
        lo, hi = wilson(f, per)
        out_members.append({"code": CODES[m["key"]]["name"], "rounds": m["R"], "W": m["W"], "shots": per,
                            "windows": per * m["dec"].n_windows, "failures": f,
                            "p_L": per_round(f / per, m["R"]),
                            "wilson95": [per_round(lo, m["R"]), per_round(hi, m["R"])]})
    # the same decoders one after another
    wk = [m["det"].clone() for m in mem]
    pr2 = torch.zeros(per, dtype=torch.int32, device="cuda")
    fl2 = torch.zeros(per, dtype=torch.int32, device="cuda")
    nf2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    for i, m in enumerate(mem):  # warm-up
        m["dec"].decode_all(wk[i], m["obs"], per, pr2, fl2, nf2)
    for i, m in enumerate(mem):
        wk[i].copy_(m["det"])
    torch.cuda.synchronize()
    e0.record()
    for i, m in enumerate(mem):
        m["dec"].decode_all(wk[i], m["obs"], per, pr2, fl2, nf2)
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1000.0
    return {"workload": "[[90,8,10]] x10 rounds, [[108,8,10]] x10, [[144,12,12]] x12; p=0.003; "
                        "W = 2 + (shot mod 3); GDG 2^4 paths",
            "shots_per_code": 3 * per, "members": len(mem), "window_steps": b.n_steps,
            "launches_per_pass": 3 * b.n_steps,
            "value": windows / t_batch, "unit": "windows/s", "seconds": t_batch,
            "sequential_value": windows / t_seq, "sequential_seconds": t_seq,
            "autotune": {"step": 1, "default": default, "chosen": shape, "ms": tune_ms,
                         "shots_per_member": tune_n[0]},
            "cuda_graph": "one graph of all window steps", "per_member": out_members}


def paper_tree(args, torch, qdec, CODES, preset, latency_fn):
    """The paper's own decoder (Sec. IV-C, Fig. 2): alpha = 1.0, 8 pre-BP
    iterations, 6 iterations per step, main branch D_max 25, 2^4 tree, side
    branches at D_split = 4..10 -- on the headline workload."""
    params = preset("paper", k_guess=K_GUESS, p=P_PHYS)
    dem = qdec.Dem(CODES[CODE_KEY], P_PHYS, ROUNDS)
    n = args.paper_shots
    dec = qdec.Decoder(dem, params, max_shots=n)
    det, obs = dem.sample(args.seed + 1, 0, n)
    work = torch.empty_like(det)
    pred = torch.empty(n, dtype=torch.int32, device="cuda")
    fail = torch.empty(n, dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # warm-up
        work.copy_(det)
        dec.decode_all(work, obs, n, pred, fail, nf)
    work.copy_(det)
    nf.zero_()
    dec.reset_counters()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    dec.decode_all(work, obs, n, pred, fail, nf)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0
    c = dec.counters()
    f = int(nf.item())
    resid_only = int((fail == 1).sum().item())  # Eq. (11) failed, Eq. (12) held
    lo, hi = wilson(f, n)
    pi = np.zeros(2, np.int32)
    qdec._check(qdec.lib().qd_decoder_path_info(dec.h, qdec._ptr(pi)))
    ldec = qdec.Decoder(dem, params, max_shots=1)
    lat = latency_fn(ldec, det[:max(1, args.latency_shots)].clone())
    # the appendix's snapshot variant: paths restart their messages where they split
    rdec = qdec.Decoder(dem, dict(params, reinit_on_split=1), max_shots=n)
    work.copy_(det)
    nf.zero_()
    e0.record()
    rdec.decode_all(work, obs, n, pred, fail, nf)
    e1.record()
    torch.cuda.synchronize()
    tr_ = e0.elapsed_time(e1) / 1000.0
    fr = int(nf.item())
    rlo, rhi = wilson(fr, n)
    reinit = {"value": n * rdec.n_windows / tr_, "unit": "windows/s",
              "ler_per_round": {"failures": fr, "shots": n, "p_L": per_round(fr / n),
                                "wilson95": [per_round(rlo), per_round(rhi)]}}
    return {"preset": "paper (alpha 1.0, n_pre 8, 6 iterations/step, Fig. 2 tree)", "paths": int(pi[0]),
            "reinit_on_split": reinit,
            "shots": n, "value": n * dec.n_windows / t, "unit": "windows/s", "seconds": t,
            "gdg_windows_frac": float(c[3]) / (n * dec.n_windows),
            "latency_ms": lat,
            "failures_eq11_only": resid_only,
            "ler_per_round": {"failures": f, "shots": n, "p_L": per_round(f / n),
                              "wilson95": [per_round(lo), per_round(hi)]}}


def ler_sweep(args, torch, qdec, CODES, preset):
    """[[144,12,12]], 12 rounds, (3,1) windows, k = 4, configured preset: LER per
    round at p = 0.001 .. 0.004 (seeds 144_00{1..4}), shots decoded in batches
    with the whole pass on the GPU; windows/s of each point."""
    from paper_2403_18901_gb300.workloads import SWEEP_144
    out = []
    B = min(args.shots, args.sweep_shots)
    for w in SWEEP_144:
        p = w["p"]
        dem = qdec.Dem(CODES[CODE_KEY], p, ROUNDS)
        dec = qdec.Decoder(dem, preset("configured", k_guess=K_GUESS, p=p), max_shots=B)
        pred = torch.empty(B, dtype=torch.int32, device="cuda")
        fail = torch.empty(B, dtype=torch.int32, device="cuda")
        nf = torch.zeros(1, dtype=torch.int64, device="cuda")
        n_done, t, resid_only = 0, 0.0, 0
        while n_done < args.sweep_shots:
            n = min(B, args.sweep_shots - n_done)
            det, obs = dem.sample(w["seed"], n_done, n)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dec.decode_all(det, obs, n, pred, fail, nf)
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1000.0
            resid_only += int((fail[:n] == 1).sum().item())  # Eq. (11) failed, Eq. (12) held
            n_done += n
        f = int(nf.item())
        lo, hi = wilson(f, n_done)
        out.append({"p": p, "shots": n_done, "failures": f, "p_L": per_round(f / n_done),
                    "failures_eq11_only": resid_only,
                    "wilson95": [per_round(lo), per_round(hi)], "windows_per_s": n_done * dec.n_windows / t,
                    "low_error_mode": p <= 0.002})
    return out


def code_capacity(args, torch, qdec, CODES):
    """Appendix workloads on [[288,12,18]]: BSC(p_d) decoded with H_X, and
    [H_X | I] with syndrome noise p_s (the appendix's decoder: alpha 0.625,
    low-error mode, D_max 40, depth-5 tree, side branches to D_split 20)."""
    from paper_2403_18901_gb300.workloads import CAPACITY
    out = []
    n = args.capacity_shots
    for pd, ps in [(0.04, 0.0), (0.04, 1e-3)]:
        dem = qdec.Dem(CODES["288"], 0, 0, capacity=(pd, ps))
        dec = qdec.Decoder(dem, dict(CAPACITY), max_shots=n)
        det, obs = dem.sample(args.seed + 288, 0, n)
        work = torch.empty_like(det)
        pred = torch.empty(n, dtype=torch.int32, device="cuda")
        fail = torch.empty(n, dtype=torch.int32, device="cuda")
        nf = torch.zeros(1, dtype=torch.int64, device="cuda")
        work.copy_(det)
        dec.decode_all(work, obs, n, pred, fail, nf)  # warm-up
        work.copy_(det)
        nf.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dec.decode_all(work, obs, n, pred, fail, nf)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        f = int(nf.item())
        lo, hi = wilson(f, n)
        r = {"code": "[[288,12,18]]", "p_data": pd, "p_synd": ps, "shots": n, "shots_per_s": n / t,
             "failures": f, "p_fail": f / n, "wilson95": [lo, hi]}
        if ps > 0:
            r["lower_bound_terms_864_2592"] = 864 * ps * ps + 2592 * pd * ps * ps
        out.append(r)
    return out


def ranker_288(args, torch, qdec, CODES, preset, latency_fn):
    """[[288,12,18]], 18 rounds, (3,1) windows, p = 0.002 (low-error mode),
    k = 4, D_max 40 on the main path and 20 steps after the last guess
    (Sec. IV-C for N = 288): a decimation ranker trained on the decoder's own
    interior-window records against Alg. 1's argmin, on the same fresh shots."""
    from paper_2403_18901_gb300 import ranker as rk
    p, R = 0.002, 18
    params = preset("configured", k_guess=K_GUESS, p=p, d_max_main=40, d_max_other=K_GUESS + 20)
    dem = qdec.Dem(CODES["288"], p, R)
    n = args.r288_shots
    B = min(n, args.shots)
    dec = qdec.Decoder(dem, params, max_shots=max(B, args.ranker_shots))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rparams, rinfo = rk.train(dec, 1, steps=max(args.ranker_steps, 1), shots_per_round=args.ranker_shots, rounds=4,
                              cap=1 << 24, batch=65536, lr=1e-2, seed=2_403_189_02)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    rhost = rparams.cpu().numpy()
    out = {"workload": "[[288,12,18]] BB memory, 18 rounds, (3,1) windows, p=0.002, GDG 2^4 paths, low-error mode, "
                       "D_max 40 / 24",
           "shots": n, "windows_per_shot": dec.n_windows,
           "train": dict(rinfo, steps=max(args.ranker_steps, 1), window=1, rounds=4,
                         shots_per_round=args.ranker_shots, seconds=train_s)}
    ldec = qdec.Decoder(dem, params, max_shots=1)
    lsrc, _ = dem.sample(args.seed + 2880, 0, max(1, args.r288_latency_shots))
    for name, rp in (("plain", None), ("ranker", rhost)):
        dec.set_ranker(rp)
        t, f, f11, gdg = decode_pass(torch, dec, dem, args.seed + 288, n, B)
        ldec.set_ranker(rp)
        out[name] = {"windows_per_s": n * dec.n_windows / t, "seconds": t, "gdg_windows_frac": gdg / (n * dec.n_windows),
                     "ler_per_round": ler_entry(f, n, R), "failures_eq11_only": f11,
                     "latency_ms": latency_fn(ldec, lsrc)}
    dec.set_ranker(None)
    return out


def readings(args, torch, qdec, CODES, preset, latency_fn=None):
    """The configured preset (alpha = 0.625, 100 initial BP iterations, steps
    of 10) on the headline workload under single changes: the second reading
    of "100 initial BP iterations" (no pre-BP and no shortening; GDG's first
    step runs 100 iterations on the whole window), alpha = 1.0 (the paper's)
    with the preset otherwise unchanged, and the two readings of the H_1
    merge of Sec. III; the paper preset with and without the H_1 merges;
    message reuse between windows (Sec. VI) with both presets, with
    per-window latency against reuse off; each output rule for windows in
    which no decision path converges (path 0's estimate; fewest unsatisfied
    checks; committed checks first), which Alg. 2 leaves open.  Every entry
    takes the run's rule (--fallback) unless it names its own."""
    dem = qdec.Dem(CODES[CODE_KEY], P_PHYS, ROUNDS)
    out = {}
    for name, pname, over, n in (
            ("initial_bp_as_first_step", "configured", dict(n_pre=0, shorten=0, iters_first=100), args.reading_shots),
            ("alpha_1.0", "configured", dict(alpha=1.0), args.shots),
            ("h1_merge_equal_restrictions", "configured", dict(merge_h1=1), args.shots),
            ("h1_merge_identity", "configured", dict(merge_h1=2), args.shots),
            ("paper_preset", "paper", {}, args.shots),
            ("paper_h1_merge_equal_restrictions", "paper", dict(merge_h1=1), args.shots),
            ("paper_h1_merge_identity", "paper", dict(merge_h1=2), args.shots),
            ("message_reuse", "configured", dict(reuse_msgs=1), args.shots),
            ("paper_message_reuse", "paper", dict(reuse_msgs=1), args.shots),
            ("fallback_path0", "configured", dict(fallback=0), args.shots),
            ("fallback_fewest_unsatisfied", "configured", dict(fallback=1), args.shots),
            ("fallback_committed_first", "configured", dict(fallback=2), args.shots),
            ("paper_fallback_path0", "paper", dict(fallback=0), args.shots),
            ("paper_fallback_committed_first", "paper", dict(fallback=2), args.shots)):
        params = preset(pname, k_guess=K_GUESS, p=P_PHYS, **over)
        B = min(n, args.shots)
        dec = qdec.Decoder(dem, params, max_shots=B)
        t, f, f11, gdg = decode_pass(torch, dec, dem, args.seed + 5, n, B)
        out[name] = {"preset": pname, "change": over, "shots": n, "windows_per_s": n * dec.n_windows / t,
                     "gdg_windows_frac": gdg / (n * dec.n_windows), "ler_per_round": ler_entry(f, n),
                     "failures_eq11_only": f11}
        if over.get("reuse_msgs") and latency_fn is not None:
            # per-window latency with and without reuse, on the same shots
            src, _ = dem.sample(args.seed + 5, 0, max(1, args.latency_shots // 4))
            ld = qdec.Decoder(dem, params, max_shots=1)
            out[name]["latency_ms"] = latency_fn(ld, src)
            ld0 = qdec.Decoder(dem, dict(params, reuse_msgs=0), max_shots=1)
            out[name]["latency_ms_without_reuse"] = latency_fn(ld0, src)
    return out


def window_shapes(args, torch, qdec, CODES, preset):
    """The other window shapes of Sec. IV-C with the paper's decoder: (5,2)
    windows for [[144,12,12]] (12 rounds, p = 0.003, the Fig. 2 tree) and (4,1)
    windows for [[288,12,18]] (18 rounds, p = 0.002, its own tree: D_max 40,
    depth-5 tree, side branches to D_split 20, 16 pre-BP iterations)."""
    out = []
    n = args.shape_shots
    for key, R, p, params in (
            ("144", 12, 0.003, preset("paper", 4, p=0.003, W=5, F=2)),
            ("288", 18, 0.002, preset("paper", 5, p=0.002, d_max_main=40, d_max_other=25, side_max=20, n_pre=16,
                                      W=4, F=1))):
        dem = qdec.Dem(CODES[key], p, R)
        B = min(n, args.shots)
        dec = qdec.Decoder(dem, params, max_shots=B)
        t, f, f11, gdg = decode_pass(torch, dec, dem, args.seed + 17, n, B)
        out.append({"code": CODES[key]["name"], "rounds": R, "p": p, "W": params["W"], "F": params["F"],
                    "shots": n, "windows_per_shot": dec.n_windows, "windows_per_s": n * dec.n_windows / t,
                    "gdg_windows_frac": gdg / (n * dec.n_windows), "ler_per_round": ler_entry(f, n, R),
                    "failures_eq11_only": f11})
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2403_18901_gb300 import build as qbuild
    from paper_2403_18901_gb300 import qdec, replicas
    from paper_2403_18901_gb300.workloads import CODES, preset
    preset = with_fallback(preset, args.fallback)

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    qbuild.build()
    qdec.lib()
    params = preset(args.preset, k_guess=K_GUESS)
    dem = qdec.Dem(CODES[CODE_KEY], P_PHYS, ROUNDS)
    B = args.shots
    dec = qdec.Decoder(dem, params, max_shots=B)
    nwin = dec.n_windows
    dw = dem.det_words
    n_batches = args.warmup + args.steps
    # inputs resident in HBM before timing: one fresh batch per step
    pristine = []
    for b in range(n_batches):
        d, o = dem.sample(args.seed, replicas.shot_offset(rank, n_batches, B, b), B)
        pristine.append((d, o))
    work = torch.empty((B, dw), dtype=torch.int32, device="cuda")
    pred = torch.empty(B, dtype=torch.int32, device="cuda")
    fail = torch.empty(B, dtype=torch.int32, device="cuda")
    nfail = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2
    stream = torch.cuda.current_stream()

    def step(b):
        work.copy_(pristine[b][0])
        dec.decode_all(work, pristine[b][1], B, pred, fail, nfail)

    def timed(local_idx):
        """Warm-up + exactly K timed steps; returns (seconds, failures, clocks)."""
        for b in range(args.warmup):
            step(b)
        torch.cuda.synchronize()
        dec.reset_counters()
        nfail.zero_()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_idx) as clk:
            for s_ in range(args.steps):
                flush.fill_(s_)  # L2 flushed between timed steps (outside the events)
                ev[s_][0].record(stream)
                step(args.warmup + s_)
                ev[s_][1].record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, "cuda")
        return t, int(nfail.item()), clk.summary()

    t_wall0 = time.perf_counter()
    tot_s, failures, clocks = timed(local)
    t_wall = time.perf_counter() - t_wall0
    counters = dec.counters()
    windows = B * nwin * args.steps * world
    value = windows / tot_s

    # ---- decode-kernel time alone (CUDA events on the launching stream) ----
    kern_ms = []
    corr = torch.empty((B, dec.corr_words), dtype=torch.int32, device="cuda")
    resid = torch.zeros(B, dtype=torch.int32, device="cuda")
    b = args.warmup
    work.copy_(pristine[b][0])
    pred.zero_()
    dec.reset_counters()
    for k in range(nwin):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dec.decode_window(k, work, B, corr)
        e1.record(stream)
        dec.commit(k, corr, B, work, pred, resid)
        kern_ms.append((e0, e1))
    torch.cuda.synchronize()
    kern_ms = [a.elapsed_time(b) for a, b in kern_ms]
    kc = dec.counters_ex()
    edge_iters = int(kc[0] + kc[1])  # every decision path counted from the root (Alg. 2)
    edge_exec = int(kc[0] + kc[5])   # what the GPU ran (shared path prefixes once)
    kern_s = sum(kern_ms) / 1000.0
    peaks, peak_kind = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12  # T op/s, one FP32 op per lane per clock
    achieved = OPS_PER_EDGE_ITER * edge_iters / kern_s / 1e12
    smem_peak = n_sm * 128 * sm_mhz * 1e6 / 1e9  # GB/s, 32 banks x 4 B per clock per SM
    smem_achieved = BYTES_PER_EDGE_ITER * edge_iters / kern_s / 1e9

    # ---- learned weighted min-sum: train on the GPU, then time the same shots ----
    learned = None
    if args.train_steps > 0:
        from paper_2403_18901_gb300 import learn
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        logs = []
        wts = learn.train(dem, dec, alpha=params["alpha"], T=25, ckpt=5, batch=args.train_batch,
                          steps=args.train_steps, lr=1e-3, seed=2_403_189_01, log=logs.append)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        for k, w in wts.items():
            dec.set_weights(k, w)
        tot_l, fail_l, clocks_l = timed(local)
        cl = dec.counters()
        for k in wts:
            dec.set_weights(k, None)
        n_types = len({id(w) for w in wts.values()})
        learned = {"train": {"steps_per_window_type": args.train_steps, "batch": args.train_batch,
                             "window_types": n_types,
                             "samples": args.train_steps * args.train_batch * n_types,
                             "seconds": train_s, "T": 25, "checkpoint_every": 5, "adam_lr": 1e-3,
                             "loss_log": logs},
                   "value": windows / tot_l, "ms_per_step": 1000 * tot_l / args.steps,
                   "edge_iterations_per_window": float(cl[0] + cl[1]) / (B * nwin * args.steps),
                   "gdg_windows_frac": float(cl[3]) / (B * nwin * args.steps),
                   "clocks": clocks_l}
    # ---- learned decimation ranker: train on the decoder's own records ----
    ranked = None
    if args.ranker_steps > 0:
        from paper_2403_18901_gb300 import ranker as rk
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rdec = qdec.Decoder(dem, params, max_shots=max(B, args.ranker_shots))
        rparams, rinfo = rk.train(rdec, 1, steps=args.ranker_steps, shots_per_round=args.ranker_shots, rounds=4,
                                  cap=1 << 24, batch=65536, lr=1e-2, seed=2_403_189_01)
        torch.cuda.synchronize()
        rtrain_s = time.perf_counter() - t0
        del rdec
        rhost = rparams.cpu().numpy()
        dec.set_ranker(rhost)
        tot_r, fail_r, clocks_r = timed(local)
        cr = dec.counters()
        rlaunch = dec.launch_info(1)
        dec.set_ranker(None)
        ranked = {"train": dict(rinfo, steps=args.ranker_steps, window=1, rounds=4,
                                shots_per_round=args.ranker_shots, batch=65536, adam_lr=1e-2,
                                seconds=rtrain_s),
                  "value": windows / tot_r, "ms_per_step": 1000 * tot_r / args.steps, "clocks": clocks_r,
                  "edge_iterations_per_window": float(cr[0] + cr[1]) / (B * nwin * args.steps),
                  "gdg_windows_frac": float(cr[3]) / (B * nwin * args.steps),
                  "launch": rlaunch, "failures": fail_r}
    batched = None
    if args.batch_shots > 0 and rank == 0:
        batched = batched_uneven(args, torch, qdec, CODES, preset)
    failures = int(replicas.sum_over_ranks(failures, "cuda"))

    line = None
    if rank == 0:
        # ---- end to end: host buffers through qd_decode_shots_host ----
        hd = pristine[args.warmup][0].cpu().numpy().view(np.uint32).copy()
        ho = pristine[args.warmup][1].cpu().numpy().view(np.uint32).copy()
        hd_t = torch.from_numpy(hd.view(np.int32)).pin_memory()
        ho_t = torch.from_numpy(ho.view(np.int32)).pin_memory()
        hd_p = hd_t.numpy().view(np.uint32)
        ho_p = ho_t.numpy().view(np.uint32)
        dec.decode_host(hd_p, ho_p)
        e2e_times = []
        for _ in range(max(1, min(3, args.steps))):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dec.decode_host(hd_p, ho_p)
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = statistics.median(e2e_times)
        h2d = hd_p.nbytes + ho_p.nbytes
        d2h = 4 * B + 4 * B + 8

        # ---- latency mode: one shot per window step, CUDA-graph replay ----
        L = max(1, args.latency_shots)
        ldec = qdec.Decoder(dem, params, max_shots=1)
        lsrc = pristine[args.warmup][0][:L].clone()

        def latency(ld, src=None):
            src = lsrc if src is None else src
            nwin = ld.n_windows
            ldet = torch.empty((1, ld.dem.det_words), dtype=torch.int32, device="cuda")
            lcorr = torch.empty((1, ld.corr_words), dtype=torch.int32, device="cuda")
            lpred = torch.zeros(1, dtype=torch.int32, device="cuda")
            lres = torch.zeros(1, dtype=torch.int32, device="cuda")
            gs = torch.cuda.Stream()
            graphs = []
            with torch.cuda.stream(gs):
                for k in range(nwin):  # warm the launch path before capture
                    ld.decode_window(k, ldet, 1, lcorr)
                    ld.commit(k, lcorr, 1, ldet, lpred, lres)
            torch.cuda.synchronize()
            for k in range(nwin):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=gs):
                    ld.decode_window(k, ldet, 1, lcorr)
                    ld.commit(k, lcorr, 1, ldet, lpred, lres)
                graphs.append(g)
            lat = []
            for sidx in range(src.shape[0]):
                ldet.copy_(src[sidx:sidx + 1])
                for k in range(nwin):
                    a = torch.cuda.Event(enable_timing=True)
                    b2 = torch.cuda.Event(enable_timing=True)
                    a.record()
                    graphs[k].replay()
                    b2.record()
                    lat.append((a, b2))
            torch.cuda.synchronize()
            lat_ms = sorted(a.elapsed_time(b2) for a, b2 in lat)
            return {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))],
                    "max": lat_ms[-1], "windows": len(lat_ms)}

        lat_plain = latency(ldec)
        n_shots_total = B * args.steps * world
        if learned is not None:
            for k, w in wts.items():
                ldec.set_weights(k, w)
            learned["latency_ms"] = latency(ldec)
            for k in wts:
                ldec.set_weights(k, None)
            fl_tot = fail_l if world == 1 else None
            lo, hi = wilson(failures, n_shots_total)
            llo, lhi = wilson(fail_l, B * args.steps)
            learned["ler_per_round"] = {
                "plain": {"failures": failures, "shots": n_shots_total,
                          "p_L": per_round(failures / n_shots_total),
                          "wilson95": [per_round(lo), per_round(hi)]},
                "learned": {"failures": fail_l, "shots": B * args.steps,
                            "p_L": per_round(fail_l / (B * args.steps)),
                            "wilson95": [per_round(llo), per_round(lhi)]}}
            del fl_tot

        if ranked is not None:
            ldec.set_ranker(rhost)
            ranked["latency_ms"] = latency(ldec)
            ldec.set_ranker(None)
            lo, hi = wilson(failures, n_shots_total)
            rlo, rhi = wilson(ranked["failures"], B * args.steps)
            ranked["ler_per_round"] = {
                "plain": {"failures": failures, "shots": n_shots_total,
                          "p_L": per_round(failures / n_shots_total),
                          "wilson95": [per_round(lo), per_round(hi)]},
                "ranker": {"failures": ranked["failures"], "shots": B * args.steps,
                           "p_L": per_round(ranked["failures"] / (B * args.steps)),
                           "wilson95": [per_round(rlo), per_round(rhi)]}}

        capacity = code_capacity(args, torch, qdec, CODES) if args.capacity_shots > 0 else None
        sweep = ler_sweep(args, torch, qdec, CODES, preset) if args.sweep_shots > 0 else None
        paper = None
        if args.paper_shots > 0:
            paper = paper_tree(args, torch, qdec, CODES, preset, latency)
        r288 = ranker_288(args, torch, qdec, CODES, preset, latency) if args.r288_shots > 0 else None
        rdg = readings(args, torch, qdec, CODES, preset, latency) if args.reading_shots > 0 else None
        shapes = window_shapes(args, torch, qdec, CODES, preset) if args.shape_shots > 0 else None

        # the metric's own numbers first: plain vs learned GDG on the headline
        # workload (windows/s, per-window latency, LER per round), and the
        # [[288,12,18]] ranker workload
        def hl(v, lat, ler):
            return {"windows_per_s": v, "latency_ms": {k: lat[k] for k in ("p50", "p99", "max", "windows")},
                    "ler_per_round": ler}
        headline = {"workload": workload_name(args.preset, args.fallback),
                    "plain": hl(value, lat_plain, ler_entry(failures, n_shots_total))}
        if learned is not None:
            headline["learned_weights"] = hl(learned["value"], learned["latency_ms"],
                                             learned["ler_per_round"]["learned"])
        if ranked is not None:
            headline["learned_ranker"] = hl(ranked["value"], ranked["latency_ms"], ranked["ler_per_round"]["ranker"])
        if r288 is not None:
            headline["bb288_p002"] = {k: hl(r288[k]["windows_per_s"], r288[k]["latency_ms"], r288[k]["ler_per_round"])
                                      for k in ("plain", "ranker")}

        cpu_rate, cores, cpu_shots, cpu_s = cpu_oracle_rate(params, args.cpu_seconds, args.seed)
        line = {
            "headline": headline,
            "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (DEM shots sampled on the GPU, seeded Philox)",
            "config": {"workload": workload_name(args.preset, args.fallback), "shots_per_step": B * world,
                       "windows_per_shot": nwin, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write)",
                       "cuda_graph": "latency mode replays one captured graph per window"},
            "shots_per_s": B * args.steps * world / tot_s,
            "logical_failures": failures, "shots_decoded": B * args.steps * world,
            "latency_ms": dict(lat_plain,
                               mode="1 shot per window step (decode + commit, one CUDA graph); path mode: "
                                    "one 512-thread CTA per decision path, the shot's "
                                    f"{ldec.launch_info(0)['path_ctas_per_shot']} CTAs in clusters of "
                                    f"{ldec.launch_info(0)['path_cluster']} that split the pre-BP"),
            "paper_context": {"worst_case_ms_per_window": 3.0,
                              "hardware": "Intel i9-13900K, multi-threaded"},
            "e2e": {"value": B * nwin / e2e_s, "unit": "windows/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (2 * nwin + 1),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Top/s",
                         "frac": achieved / alu_peak,
                         "traffic": TRAFFIC_PER_LAUNCH.get((args.preset, B, args.fallback)),
                         "kernel": "decode_shot_kernel",
                         "work": f"{OPS_PER_EDGE_ITER} ops x {edge_iters} edge-iterations in "
                                 f"{nwin} launches",
                         "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz "
                                       f"({peak_kind} sm_max_mhz)",
                         "smem": {"achieved": smem_achieved, "peak": smem_peak, "unit": "GB/s",
                                  "frac": smem_achieved / smem_peak,
                                  "basis": f"{BYTES_PER_EDGE_ITER} B per counted edge-iteration (two FP32 messages "
                                           f"read and written) against {n_sm} SMs x 128 B/clk x {sm_mhz:.0f} MHz "
                                           f"({peak_kind} sm_max_mhz); the kernel keeps compressed check state "
                                           f"and moves fewer bytes than this count"},
                         "edge_iterations_executed": edge_exec,
                         "ncu_pipes": PIPES_PER_LAUNCH.get((args.preset, args.fallback))},
            "launch": dec.launch_info(1),
            "edge_iterations_per_window": edge_iters / (B * nwin),
            "gdg_windows_frac": float(kc[3]) / (B * nwin),
            "clocks": clocks,
            "cpu_baseline": {"value": cpu_rate, "unit": "windows/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{cpu_shots} shots ({cpu_shots * nwin} windows) in "
                                       f"{cpu_s:.1f} s"},
            "wall_s_timed": t_wall,
            "learned": learned,
            "ranker": ranked,
            "batched_uneven": batched,
            "paper_tree": paper,
            "code_capacity": capacity,
            "ler_sweep_144": sweep,
            "ranker_288": r288,
            "readings": rdg,
            "window_shapes": shapes,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
