"""Learned weighted min-sum: per-edge, per-iteration weights in place of the
normalisation alpha of Eq. (1), trained on window samples with the library's
hand-written adjoint (qd_wms_grad) behind a torch.autograd.Function, and
Adam (qd_adam_step).  The trained weights plug into the GDG decoder with
qd_decoder_set_weights; plain GDG stays available by passing no weights.

Every numerical step runs in libqdec; torch provides device memory, streams
and the autograd plumbing.
"""
import ctypes as C

import numpy as np
import torch

from . import qdec


class Wms:
    """Training context of one window (qd_wms_*)."""

    def __init__(self, dec, k, T=25, ckpt=5):
        h = C.c_void_p()
        qdec._check(qdec.lib().qd_wms_create(dec.h, k, T, ckpt, C.byref(h)))
        self.h, self.dec, self.k = h, dec, k
        info = np.zeros(6, np.int32)
        qdec._check(qdec.lib().qd_wms_info(self.h, qdec._ptr(info)))
        self.n_rows, self.n_cols, self.n_edges, self.T, self.ckpt, self.rw = (int(x) for x in info)

    def __del__(self):
        if getattr(self, "h", None) and qdec._lib is not None:
            qdec._lib.qd_wms_destroy(self.h)
            self.h = None

    def sample(self, seed, offset, n):
        synd = torch.empty((n, self.rw), dtype=torch.int32, device="cuda")
        qdec._check(qdec.lib().qd_wms_sample(self.h, seed, offset, n, qdec._ptr(synd), qdec._stream(None)))
        return synd

    def loss(self, w, synd, want_post=False):
        n = synd.shape[0]
        loss = torch.empty(n, dtype=torch.float32, device="cuda")
        post = torch.empty((n, self.n_cols), dtype=torch.float32, device="cuda") if want_post else None
        qdec._check(qdec.lib().qd_wms_loss(self.h, qdec._ptr(w), qdec._ptr(synd), n, qdec._ptr(loss),
                                           qdec._ptr(post), qdec._stream(None)))
        return (loss, post) if want_post else loss

    def grad(self, w, synd, scale=1.0, out=None):
        """Accumulates scale * dL/dw (summed over samples) into out; returns (out, loss)."""
        n = synd.shape[0]
        if out is None:
            out = torch.zeros_like(w)
        loss = torch.empty(n, dtype=torch.float32, device="cuda")
        qdec._check(qdec.lib().qd_wms_grad(self.h, qdec._ptr(w), qdec._ptr(synd), n, float(scale),
                                           qdec._ptr(out), qdec._ptr(loss), qdec._stream(None)))
        return out, loss


class WeightedMinSumLoss(torch.autograd.Function):
    """Mean soft-syndrome BCE of T unrolled weighted min-sum iterations.
    Forward: qd_wms_loss; backward: the adjoint kernel qd_wms_grad (which
    recomputes the unrolled iterations from message checkpoints)."""

    @staticmethod
    def forward(ctx, w, synd, wms):
        loss = wms.loss(w.detach().contiguous(), synd)
        ctx.save_for_backward(w, synd)
        ctx.wms = wms
        return loss.mean()

    @staticmethod
    def backward(ctx, gout):
        w, synd = ctx.saved_tensors
        n = synd.shape[0]
        g = torch.zeros_like(w)
        ctx.wms.grad(w.detach().contiguous(), synd, scale=float(gout) / n, out=g)
        return g, None, None


def adam_step(w, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    qdec._check(qdec.lib().qd_adam_step(qdec._ptr(w), qdec._ptr(g), qdec._ptr(m), qdec._ptr(v), w.numel(),
                                        lr, b1, b2, eps, step, qdec._stream(None)))


def window_types(dem, dec):
    """Groups of windows whose matrices and priors are identical (so one weight
    set serves them all), from the DEM columns relative to each window's
    first block."""
    cols = dem.columns()
    sig = {}
    for k in range(dec.n_windows):
        wi = dec.window_info(k)
        r0 = wi["r0"] * dem.w
        key = [wi["n_rows"], wi["n_commit"]]
        for c in wi["gcols"]:
            d = cols["col_dets"][cols["col_ptr"][c]:cols["col_ptr"][c + 1]]
            key.append((tuple(int(x) - r0 for x in d if x - r0 < wi["n_rows"]), float(cols["llr"][c])))
        sig.setdefault(tuple(key), []).append(k)
    return list(sig.values())


def train(dem, dec, alpha, T=25, ckpt=5, batch=4096, steps=245, lr=1e-3, seed=2_403_189_01, log=None):
    """Train one weight set per window type; returns {window k: weights [T][edges]}
    (the tensors of windows of one type are shared)."""
    out = {}
    for group in window_types(dem, dec):
        k0 = group[0]
        wms = Wms(dec, k0, T, ckpt)
        w = torch.full((T, wms.n_edges), float(alpha), dtype=torch.float32, device="cuda",
                       requires_grad=True)
        m = torch.zeros_like(w)
        v = torch.zeros_like(w)
        for step in range(1, steps + 1):
            synd = wms.sample(seed, (k0 * steps + step) * batch, batch)
            w.grad = None
            loss = WeightedMinSumLoss.apply(w, synd, wms)
            loss.backward()
            with torch.no_grad():
                adam_step(w.data, w.grad, m, v, lr, step)
            if log is not None and (step == 1 or step % 50 == 0 or step == steps):
                log(f"window type {group}: step {step} loss {float(loss.detach()):.5f}")
        wf = w.detach()
        for k in group:
            out[k] = wf
    return out
