"""GPU tests of the learned weighted min-sum (training kernels).

The adjoint kernel (qd_wms_grad) is compared with the oracle's FP64
reverse-mode gradient and with FP64 central finite differences of the oracle
loss on 64 random (iteration, edge) weights at generic points (relative
error <= 1e-3).  Training through the autograd wrapper lowers the held-out
loss and raises the fraction of windows whose T-iteration decision already
satisfies the syndrome -- what the trained weights gain over plain alpha.
"""
import numpy as np
import pytest

from conftest import oracle_dem
from oracle import wms_ref
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


def _window_samples(o, k, n, seed):
    """Window syndromes s = H_win e with every window column firing with its
    prior (numpy RNG, test side)."""
    win = o.window(3, 1, k)
    rng = np.random.default_rng(seed)
    p = o.col_p[win["gcols"]]
    out = np.zeros((n, win["n_rows"]), np.uint8)
    for s in range(n):
        fired = np.nonzero(rng.random(win["n_cols"]) < p)[0]
        for c in fired:
            out[s, win["col_rows"][win["col_ptr"][c]:win["col_ptr"][c + 1]]] ^= 1
    return win, out


def _pack(bits):
    n, r = bits.shape
    rw = (r + 31) // 32
    words = np.zeros((n, rw), np.uint32)
    for j in range(r):
        words[:, j >> 5] |= bits[:, j].astype(np.uint32) << np.uint32(j & 31)
    return torch.from_numpy(words.view(np.int32)).cuda()


def _setup(T=25, ckpt=5):
    from paper_2403_18901_gb300.learn import Wms
    d = qdec.Dem(CODES["72"], 0.003, 6)
    dec = qdec.Decoder(d, preset("configured", k_guess=3), max_shots=16)
    return d, dec, Wms(dec, 1, T, ckpt)


def test_adjoint_matches_oracle_and_finite_differences():
    o = oracle_dem("72", 0.003, 6)
    _, _, wms = _setup(T=25, ckpt=5)
    win, bits = _window_samples(o, 1, 4, seed=7)
    g = wms_ref.Graph(win["n_rows"], win["col_ptr"], win["col_rows"], win["llr"])
    rng = np.random.default_rng(1)
    w = rng.uniform(0.55, 0.75, size=(25, g.ne)).astype(np.float32)
    wt = torch.from_numpy(w).cuda()
    synd = _pack(bits)
    loss = wms.loss(wt, synd).cpu().numpy()
    for s in range(bits.shape[0]):
        gg, lg = wms.grad(wt, synd[s:s + 1].contiguous())
        gg = gg.cpu().numpy().astype(np.float64)
        L, gref = wms_ref.loss_and_grad(g, w.astype(np.float64), bits[s])
        assert abs(loss[s] - L) <= 1e-4 * abs(L) + 1e-7
        assert abs(float(lg[0]) - L) <= 1e-4 * abs(L) + 1e-7
        scale = np.abs(gref).max()
        assert np.abs(gg - gref).max() <= 1e-3 * scale
        # FP64 finite differences of the oracle loss on 64 random weights
        idx = [(t, e) for t in range(25) for e in range(g.ne) if abs(gref[t, e]) > 1e-3 * scale]
        pick = rng.choice(len(idx), min(64, len(idx)) if s == 0 else 8, replace=False)
        h = 1e-6
        for q in pick:
            t, e = idx[q]
            wp = w.astype(np.float64).copy()
            wm = wp.copy()
            wp[t, e] += h
            wm[t, e] -= h
            fd = (wms_ref.forward(g, wp, bits[s]) - wms_ref.forward(g, wm, bits[s])) / (2 * h)
            assert abs(gg[t, e] - fd) <= 1e-3 * abs(fd) + 1e-6 * scale, (t, e, gg[t, e], fd)


def test_checkpoint_spacing_does_not_change_gradient():
    from paper_2403_18901_gb300.learn import Wms
    d, dec, _ = _setup()
    a = Wms(dec, 1, 25, 5)
    b = Wms(dec, 1, 25, 1)
    c = Wms(dec, 1, 25, 25)
    synd = a.sample(3, 0, 64)
    w = torch.full((25, a.n_edges), 0.7, device="cuda") + 0.01 * torch.rand((25, a.n_edges), device="cuda")
    ga, _ = a.grad(w, synd)
    gb, _ = b.grad(w, synd)
    gc, _ = c.grad(w, synd)
    torch.cuda.synchronize()
    # sums over samples use atomics, so compare to rounding
    assert torch.allclose(ga, gb, rtol=1e-5, atol=1e-7) and torch.allclose(ga, gc, rtol=1e-5, atol=1e-7)


def test_autograd_function_uses_the_adjoint():
    from paper_2403_18901_gb300.learn import WeightedMinSumLoss
    d, dec, wms = _setup()
    synd = wms.sample(9, 0, 32)
    w = torch.full((25, wms.n_edges), 0.625, device="cuda", requires_grad=True)
    L = WeightedMinSumLoss.apply(w, synd, wms)
    L.backward()
    ref, losses = wms.grad(w.detach(), synd, scale=1.0 / 32)
    torch.cuda.synchronize()
    assert abs(float(L.detach()) - float(losses.mean())) < 1e-6
    assert torch.allclose(w.grad, ref, rtol=1e-5, atol=1e-8)


def _converged_fraction(wms, o, w, synd_bits):
    win = o.window(3, 1, wms.k)
    synd = _pack(synd_bits)
    _, post = wms.loss(w, synd, want_post=True)
    e = (post.cpu().numpy() <= 0).astype(np.uint8)
    ok = 0
    for s in range(e.shape[0]):
        acc = np.zeros(win["n_rows"], np.uint8)
        for c in np.nonzero(e[s])[0]:
            acc[win["col_rows"][win["col_ptr"][c]:win["col_ptr"][c + 1]]] ^= 1
        ok += int((acc == synd_bits[s]).all())
    return ok / e.shape[0]


def test_training_lowers_loss_and_helps_convergence():
    from paper_2403_18901_gb300.learn import WeightedMinSumLoss, Wms, adam_step
    o = oracle_dem("72", 0.003, 6)
    d = qdec.Dem(CODES["72"], 0.003, 6)
    dec = qdec.Decoder(d, preset("configured", k_guess=3), max_shots=16)
    wms = Wms(dec, 1, 25, 5)
    w = torch.full((25, wms.n_edges), 0.625, device="cuda", requires_grad=True)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    _, held = _window_samples(o, 1, 400, seed=99)
    held_t = _pack(held)
    base_loss = float(wms.loss(w.detach(), held_t).mean())
    base_conv = _converged_fraction(wms, o, w.detach(), held)
    for step in range(1, 61):
        synd = wms.sample(11, step * 1024, 1024)
        w.grad = None
        L = WeightedMinSumLoss.apply(w, synd, wms)
        L.backward()
        with torch.no_grad():
            adam_step(w.data, w.grad, m, v, 1e-2, step)
    new_loss = float(wms.loss(w.detach(), held_t).mean())
    new_conv = _converged_fraction(wms, o, w.detach(), held)
    assert new_loss < base_loss
    assert new_conv > base_conv, (base_conv, new_conv)
