"""Learned decimation ranker: a 2-layer MLP (8 -> 64 -> 1) that replaces the
argmin of Alg. 1 (SELECT-VN) inside GDG; aggressive decimation (Alg. 3), the
guess rule of Alg. 2 and f = [L_g <= 0] stay.

Training data are the decoder's own candidate records: window-local samples
(qd_window_sample) decoded with the candidate dump on (qd_decoder_set_dump),
labelled 1 when the candidate's column is in the sampled fault set and Alg. 1
would give it the value 1.  Training
runs the library's forward / backward kernel (qd_ranker_eval) with the
decoder's parameter rounding in the forward pass, and Adam (qd_adam_step).
Inference (qd_decoder_set_ranker) scores the candidates with BF16 tensor-core
MMAs inside the decode kernel.

Every numerical step runs in libqdec; torch provides device memory and
streams.
"""
import torch

from . import qdec
from .learn import adam_step

N_PARAMS = 641
REC_BYTES = 48


def fields(recs):
    """Views of a [n, 48] uint8 record tensor: x [n, 8], shot, wcol, depth, flags."""
    f = recs.view(torch.float32)
    i = recs.view(torch.int32)
    h = recs.view(torch.int16)
    return f[:, :8], i[:, 8], i[:, 9], h[:, 20], i[:, 11]


def labels_of(recs, fault):
    """1 where the record's window column is in its shot's sampled fault set."""
    _, shot, wcol, _, _ = fields(recs)
    word = fault[shot.long(), (wcol >> 5).long()]
    return ((word >> (wcol & 31)) & 1).to(torch.uint8)


def train_labels(recs, in_fault):
    """The training target: the candidate is a sampled fault AND Alg. 1's
    value for it is 1 ([L <= 0]), i.e. decimating it now is a right guess of
    a flipped bit -- the event the argmin of Alg. 1 bets on."""
    _, _, _, _, flags = fields(recs)
    return in_fault & (flags & 1).to(torch.uint8)


def collect(dec, k, seed, offset, n, cap):
    """Decode n window-local samples of window k with the dump on; returns
    (records [m, 48] uint8, labels [m] uint8, m_total) where m_total counts
    records beyond the capacity too."""
    dw, cw = dec.dem.det_words, dec.corr_words
    det = torch.zeros((n, dw), dtype=torch.int32, device="cuda")
    fault = torch.zeros((n, cw), dtype=torch.int32, device="cuda")
    dec.window_sample(k, seed, offset, n, det, fault)
    recs = torch.zeros((cap, REC_BYTES), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    corr = torch.zeros((n, cw), dtype=torch.int32, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    dec.set_dump(recs, cnt)
    try:
        dec.decode_window(k, det, n, corr, status, None)
    finally:
        dec.set_dump(None, None)
    total = int(cnt.item())
    recs = recs[:min(total, cap)]
    return recs, labels_of(recs, fault), total


def evaluate(params, recs, labels=None, quantize=True, pos_weight=1.0):
    """Scores (and per-record losses when labels are given)."""
    n = recs.shape[0]
    score = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.empty(n, dtype=torch.float32, device="cuda") if labels is not None else None
    qdec._check(qdec.lib().qd_ranker_eval(qdec._ptr(params), qdec._ptr(recs), qdec._ptr(labels), n,
                                          int(quantize), float(pos_weight), 0.0, None, qdec._ptr(loss),
                                          qdec._ptr(score), qdec._stream(None)))
    return score, loss


def grad(params, recs, labels, quantize=True, pos_weight=1.0, scale=1.0, out=None):
    """Accumulates scale * d(sum of losses)/d params into out; returns (out, losses)."""
    n = recs.shape[0]
    if out is None:
        out = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(n, dtype=torch.float32, device="cuda")
    qdec._check(qdec.lib().qd_ranker_eval(qdec._ptr(params), qdec._ptr(recs), qdec._ptr(labels), n,
                                          int(quantize), float(pos_weight), float(scale), qdec._ptr(out),
                                          qdec._ptr(loss), None, qdec._stream(None)))
    return out, loss


def init_params(seed=0):
    """Starts at (almost) the rule it replaces: hidden unit 0 = relu(-L/4), so
    the score ranks the most negative history sum first, plus small random
    units."""
    g = torch.Generator().manual_seed(seed)
    p = torch.zeros(N_PARAMS)
    p[:512] = 0.25 * torch.randn(512, generator=g)
    p[512:576] = 0.1 * torch.randn(64, generator=g)
    p[576:640] = 0.05 * torch.randn(64, generator=g)
    p[0:8] = 0.0
    p[0] = -1.0
    p[512] = 0.0
    p[576] = 1.0
    p[640] = -4.0
    return p.cuda()


def decision_accuracy(score, recs, labels):
    """Per selection step (shot, depth): the fraction of steps whose chosen
    candidate gets the right value f = [L <= 0] against the sampled faults,
    for the ranker's argmax (ties to the lowest column) and for the candidate
    the decoder selected when the records were made.  Returns (ranker, recorded, steps)."""
    _, shot, wcol, depth, flags = fields(recs)
    key = shot.long() * 1024 + depth.long()
    uk, grp = torch.unique(key, return_inverse=True)
    ng = uk.shape[0]
    best = torch.full((ng,), -float("inf"), device=score.device).scatter_reduce(0, grp, score, "amax")
    at_best = score == best[grp]
    big = torch.iinfo(torch.int32).max
    wmin = torch.full((ng,), big, dtype=torch.int32, device=score.device).scatter_reduce(
        0, grp, torch.where(at_best, wcol, torch.full_like(wcol, big)), "amin")
    pick = at_best & (wcol == wmin[grp])
    right = ((flags & 1).to(torch.uint8) == labels)
    acc_r = float(right[pick].float().sum()) / ng
    sel = (flags & 2) != 0
    acc_a = float(right[sel].float().sum()) / max(int(sel.sum()), 1)
    return acc_r, acc_a, ng


def train(dec, k, steps=300, shots_per_round=2048, rounds=4, cap=1 << 22, batch=65536, lr=1e-2,
          pos_weight=None, seed=2_403_189_01, log=None):
    """Collects `rounds` x `shots_per_round` window-local samples of window k,
    then runs `steps` Adam steps on minibatches of their candidate records.
    Returns (params [641] CUDA float32, info)."""
    rs, ls = [], []
    for r in range(rounds):
        rec, lab, _ = collect(dec, k, seed, r * shots_per_round, shots_per_round, cap)
        rs.append(rec)
        ls.append(lab)
    recs = torch.cat(rs)
    labels = train_labels(recs, torch.cat(ls))
    n = recs.shape[0]
    pos = float(labels.float().sum())
    if pos_weight is None:
        pos_weight = max(1.0, (n - pos) / max(pos, 1.0))
    p = init_params(seed & 0xFFFF)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.Generator(device="cuda").manual_seed(seed & 0xFFFF)
    for step in range(1, steps + 1):
        idx = torch.randint(0, n, (min(batch, n),), device="cuda", generator=g)
        b = recs[idx].contiguous()
        gr, loss = grad(p, b, labels[idx].contiguous(), True, pos_weight, 1.0 / b.shape[0])
        adam_step(p, gr, m, v, lr, step)
        if log and (step % 50 == 0 or step == 1):
            log(f"ranker step {step}: loss {float(loss.mean()):.4f}")
    return p, dict(records=n, positives=int(pos), pos_weight=pos_weight)
