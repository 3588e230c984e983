"""CPU ORACLE (test infrastructure only): learned weighted min-sum and its
gradient, in FP64 with numpy.

The model has no counterpart in the paper: Eq. (1) with the normalisation
alpha replaced by a weight w[t, e] per edge and iteration, unrolled for T
flooding iterations on a window's full parity-check matrix from
mu_{i->j} = Lambda_i (Sec. II-A), VN->CN messages clipped to [-clip, clip]
(Sec. IV), loss = soft-syndrome binary cross entropy at t = T:
P(check j odd) = (1 - prod_{i in N(j)} (1 - 2 sigma(-Lambda_i^(T)))) / 2,
averaged over the checks.

The gradient is reverse-mode differentiation of exactly these steps, written
out by hand: an edge's CN->VN message is w * |v2c| of the smallest OTHER
input of its check (found by brute force over the other inputs), so its
gradient flows to that input with d|x|/dx = sign(x); sign() has derivative
0; a clipped message passes no gradient.
"""
import numpy as np


class Graph:
    def __init__(self, n_rows, col_ptr, col_rows, llr):
        self.nr = int(n_rows)
        self.col_ptr = np.asarray(col_ptr, np.int64)
        self.col_rows = np.asarray(col_rows, np.int64)
        self.nc = len(self.col_ptr) - 1
        self.ne = int(self.col_ptr[-1])
        self.llr = np.asarray(llr, np.float64)
        self.edge_col = np.repeat(np.arange(self.nc), np.diff(self.col_ptr))
        deg = np.bincount(self.col_rows, minlength=self.nr)
        self.dmax = int(deg.max())
        # rows as padded edge lists [nr, dmax]; -1 = padding
        self.pad = -np.ones((self.nr, self.dmax), np.int64)
        fill = np.zeros(self.nr, np.int64)
        for e in range(self.ne):
            r = self.col_rows[e]
            self.pad[r, fill[r]] = e
            fill[r] += 1
        self.valid = self.pad >= 0
        # for each slot k of a row: the smallest input among the OTHER slots
        # is found by masking slot k out
        self.eye = np.eye(self.dmax, dtype=bool)


def _check_update(g, v2c, s, w_t):
    """Weighted Eq. (1): c2v, the source edge of each message's magnitude,
    and the message's sign (+-1)."""
    e = np.where(g.valid, g.pad, 0)
    a = np.where(g.valid, np.abs(v2c[e]), np.inf)            # [nr, dmax]
    neg = np.where(g.valid, v2c[e] < 0, False).astype(np.int64)
    tot = neg.sum(1) & 1                                     # [nr]
    # brute force: for slot k, min over slots != k
    a_rep = np.where(g.eye[None, :, :], np.inf, a[:, None, :])  # [nr, k, other]
    kk = np.argmin(a_rep, axis=2)                            # [nr, dmax]
    m = np.take_along_axis(a, kk, axis=1)
    src = np.take_along_axis(e, kk, axis=1)
    sgn = (tot[:, None] ^ neg ^ s[:, None].astype(np.int64)) & 1
    unit = np.where(sgn == 1, -1.0, 1.0)
    c2v = np.zeros(g.ne)
    src_e = np.zeros(g.ne, np.int64)
    unit_e = np.zeros(g.ne)
    m_e = np.zeros(g.ne)
    ev = g.pad[g.valid]
    c2v[ev] = (unit * w_t[e] * m)[g.valid]
    src_e[ev] = src[g.valid]
    unit_e[ev] = unit[g.valid]
    m_e[ev] = m[g.valid]
    return c2v, src_e, unit_e, m_e


def _var_update(g, c2v, clip):
    post = g.llr.copy()
    np.add.at(post, g.edge_col, c2v)
    raw = post[g.edge_col] - c2v
    v2c = np.clip(raw, -clip, clip)
    inside = (raw > -clip) & (raw < clip)
    return post, v2c, inside


def _loss_and_dpost(g, post, s):
    th = np.tanh(post / 2.0)
    e = np.where(g.valid, g.pad, 0)
    tv = np.where(g.valid, th[g.edge_col[e]], 1.0)          # [nr, dmax]
    prod = tv.prod(1)
    eps = 1e-7
    P = 0.5 * (1.0 - prod)
    clamped = (P < eps) | (P > 1 - eps)
    P = np.clip(P, eps, 1 - eps)
    s = s.astype(bool)
    loss = np.where(s, -np.log(P), -np.log(1 - P)).sum() / g.nr
    dP = np.where(clamped, 0.0, np.where(s, -1.0 / P, 1.0 / (1 - P))) / g.nr
    dprod = -0.5 * dP                                        # [nr]
    excl = np.where(g.eye[None, :, :], 1.0, tv[:, None, :]).prod(2)  # [nr, dmax]
    contrib = dprod[:, None] * excl * 0.5 * (1 - tv ** 2)
    dpost = np.zeros(g.nc)
    np.add.at(dpost, g.edge_col[g.pad[g.valid]], contrib[g.valid])
    return loss, dpost


def forward(g, w, s, clip=50.0):
    """Loss of one sample (s: 0/1 per row); w: [T, ne]."""
    s = np.asarray(s, np.int64)
    v2c = g.llr[g.edge_col].copy()
    post = g.llr.copy()
    for t in range(w.shape[0]):
        c2v, _, _, _ = _check_update(g, v2c, s, w[t])
        post, v2c, _ = _var_update(g, c2v, clip)
    return _loss_and_dpost(g, post, s)[0]


def loss_and_grad(g, w, s, clip=50.0):
    """Loss of one sample and dLoss/dw [T, ne] (reverse mode, FP64)."""
    s = np.asarray(s, np.int64)
    T = w.shape[0]
    v2c = g.llr[g.edge_col].copy()
    tape = []
    for t in range(T):
        c2v, src, unit, m = _check_update(g, v2c, s, w[t])
        post, v2c_new, inside = _var_update(g, c2v, clip)
        tape.append((v2c, src, unit, m, inside))
        v2c = v2c_new
    loss, dpost = _loss_and_dpost(g, post, s)
    gw = np.zeros((T, g.ne))
    g_v2c = np.zeros(g.ne)  # v2c^(T) does not enter the loss
    for t in range(T - 1, -1, -1):
        v_in, src, unit, m, inside = tape[t]
        gp = dpost.copy() if t == T - 1 else np.zeros(g.nc)
        passed = np.where(inside, g_v2c, 0.0)
        np.add.at(gp, g.edge_col, passed)
        g_c2v = gp[g.edge_col] - passed
        gw[t] = g_c2v * unit * m
        gm = g_c2v * unit * w[t]
        g_new = np.zeros(g.ne)
        np.add.at(g_new, src, gm * np.where(v_in[src] < 0, -1.0, 1.0))
        g_v2c = g_new
    return loss, gw


def posteriors(g, w, s, clip=50.0):
    """Lambda^(T) of the weighted model (for cross-checks)."""
    s = np.asarray(s, np.int64)
    v2c = g.llr[g.edge_col].copy()
    post = g.llr.copy()
    for t in range(w.shape[0]):
        c2v, _, _, _ = _check_update(g, v2c, s, w[t])
        post, v2c, _ = _var_update(g, c2v, clip)
    return post
