"""ctypes wrapper around the CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this module.  The product package never does.
"""
import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_lib = None


class QdoCode(C.Structure):
    _fields_ = [("l", C.c_int), ("m", C.c_int), ("ax", C.c_int * 3), ("ay", C.c_int * 3),
                ("bx", C.c_int * 3), ("by", C.c_int * 3)]


def ranker_score(params, x):
    """Oracle ranker scores of feature rows x [n, 8] (FP32)."""
    p = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 8)
    out = np.zeros(x.shape[0], np.float32)
    lib().qdo_ranker_score(_ptr(p), _ptr(x), x.shape[0], _ptr(out))
    return out


# one ranker candidate record (qdo_rank_rec)
RANK_REC = np.dtype([("x", "<f4", (8,)), ("shot", "<i4"), ("wcol", "<i4"), ("depth", "<i2"),
                     ("path", "<i2"), ("flags", "<i4")])


class QdoParams(C.Structure):
    _fields_ = [("W", C.c_int), ("F", C.c_int), ("alpha", C.c_float), ("n_pre", C.c_int),
                ("iters_per_step", C.c_int), ("d_max_main", C.c_int), ("d_max_other", C.c_int),
                ("k_guess", C.c_int), ("low_error_mode", C.c_int), ("peel_at_init", C.c_int),
                ("shorten", C.c_int), ("clip", C.c_float), ("pa_main", C.c_float),
                ("pa_other", C.c_float), ("pb_main", C.c_float), ("pb_other", C.c_float),
                ("pb_d1", C.c_float), ("pc", C.c_float), ("pd", C.c_float),
                ("pc_max_depth", C.c_int), ("n_unsat_min", C.c_int), ("side_max", C.c_int),
                ("reinit_on_split", C.c_int), ("iters_first", C.c_int), ("merge_h1", C.c_int),
                ("reuse_msgs", C.c_int),
                ("fallback", C.c_int),
                ("wts", C.POINTER(C.c_void_p)), ("wT", C.c_int), ("ranker", C.c_void_p),
                ("dump", C.c_void_p), ("dump_n", C.c_void_p), ("dump_cap", C.c_int)]


class QdoBranch(C.Structure):
    _fields_ = [("status", C.c_int), ("depth", C.c_int), ("iters", C.c_int), ("pm", C.c_double)]


class QdoStep(C.Structure):
    _fields_ = [("g", C.c_int), ("value", C.c_int), ("n_agg", C.c_int), ("n_peel", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.qdo_ranker_score.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.qdo_n_paths.argtypes = [C.c_void_p]
        L.qdo_path_dmax_all.argtypes = [C.c_void_p]
        L.qdo_dem_build.restype = C.c_void_p
        L.qdo_dem_code_capacity.restype = C.c_void_p
        L.qdo_dem_code_capacity.argtypes = [P(QdoCode), C.c_double, C.c_double]
        L.qdo_logical_x.argtypes = [P(QdoCode), C.c_void_p, C.c_int]
        L.qdo_dem_build.argtypes = [P(QdoCode), C.c_double, C.c_int]
        L.qdo_dem_free.argtypes = [C.c_void_p]
        L.qdo_dem_info.argtypes = [C.c_void_p, C.c_void_p]
        L.qdo_dem_columns.argtypes = [C.c_void_p] + [C.c_void_p] * 5
        L.qdo_n_fault_locations.argtypes = [C.c_void_p]
        L.qdo_fault_effect.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.c_void_p, C.c_void_p]
        L.qdo_circuit_ops.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
        L.qdo_logical_matrix.argtypes = [C.c_void_p, C.c_void_p]
        L.qdo_noiseless_detectors.argtypes = [C.c_void_p, C.c_void_p]
        L.qdo_n_windows.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.qdo_window_info.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.qdo_window_graph.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 4
        L.qdo_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.qdo_sample.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p,
                                 C.c_void_p]
        L.qdo_code_matrices.argtypes = [P(QdoCode), C.c_void_p, C.c_void_p]
        L.qdo_gf2_rank.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.qdo_logical_z.argtypes = [P(QdoCode), C.c_void_p, C.c_int]
        L.qdo_bp_run.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_float, C.c_float, C.c_int, C.c_int,
                                 C.c_void_p, C.c_void_p]
        L.qdo_decode_window.argtypes = [C.c_void_p, P(QdoParams), C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
        L.qdo_gdg_graph.argtypes = [P(QdoParams), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.qdo_run_shots.argtypes = [C.c_void_p, P(QdoParams), C.c_void_p, C.c_void_p,
                                    C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.qdo_decode_window_ex.argtypes = [C.c_void_p, P(QdoParams), C.c_int] + [C.c_void_p] * 5
        L.qdo_decode_window_paths.argtypes = [C.c_void_p, P(QdoParams), C.c_int] + [C.c_void_p] * 4
        L.qdo_window_build.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 6
        declare_select(L)
        _lib = L
    return _lib


def declare_select(L):
    """Argument types of the SELECT-VN / AGG-DEC test-access calls of an
    oracle library handle (also used on rebuilt copies of the oracle)."""
    L.qdo_agg_dec.argtypes = [C.POINTER(QdoParams), C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.qdo_select_vn.argtypes = [C.POINTER(QdoParams), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                C.c_void_p, C.c_void_p]
    return L


def agg_dec(params, h, D, main_branch, n_unsat, lib_=None):
    """Alg. 3 on one VN's four-iteration history h (oldest first): 1, 0 or -1."""
    q = make_params(params)
    hv = np.ascontiguousarray(h, np.float32)
    assert hv.size == 4
    return (lib_ or lib()).qdo_agg_dec(C.byref(q), _ptr(hv), int(D), int(main_branch), int(n_unsat))


def select_vn(params, H, hist, status, synd, D, main_branch, lib_=None):
    """One SELECT-VN call (Alg. 1, with Alg. 3 outside the low-error mode) on
    the dense matrix H [nr][nc] with history hist [4][nc] (oldest first; the
    newest row is the current posterior), status [nc] (-1 active) and current
    syndrome synd [nr].  Returns (g, f, n_agg, status after, synd after)."""
    H = np.asarray(H, np.uint8)
    nr, nc = H.shape
    cols = [np.nonzero(H[:, i])[0] for i in range(nc)]
    ptr = np.cumsum([0] + [len(c) for c in cols]).astype(np.int32)
    rows = (np.concatenate(cols) if nc else np.zeros(0)).astype(np.int32)
    hv = np.ascontiguousarray(hist, np.float32).reshape(4, nc)
    st = np.ascontiguousarray(status, np.int8).copy()
    sp = np.ascontiguousarray(synd, np.uint8).copy()
    f = C.c_int(-7)
    nagg = C.c_int(-7)
    q = make_params(params)
    g = (lib_ or lib()).qdo_select_vn(C.byref(q), nr, nc, _ptr(ptr), _ptr(rows), _ptr(hv), _ptr(st),
                                      _ptr(sp), int(D), int(main_branch), C.byref(f), C.byref(nagg))
    return g, f.value, nagg.value, st, sp


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_code(code):
    """code: dict(l, m, A=[(ax, ay)]*3, B=[(bx, by)]*3)."""
    c = QdoCode()
    c.l, c.m = code["l"], code["m"]
    for k in range(3):
        c.ax[k], c.ay[k] = code["A"][k]
        c.bx[k], c.by[k] = code["B"][k]
    return c


def make_params(p, weights=None, ranker=None):
    """weights: None or {window index: float32 array [T][n_edges of the window]};
    ranker: None or 641 float32 parameters of the decimation ranker."""
    assert p.get("side_max", 0) == 0 or p["side_max"] >= p["k_guess"], "side_max must be 0 or >= k_guess"
    q = QdoParams()
    for name, _ in QdoParams._fields_:
        if name in ("wts", "wT", "ranker", "dump", "dump_n", "dump_cap"):
            continue
        setattr(q, name, p.get(name, 0) if name == "fallback" else p[name])
    q.ranker = None
    if ranker is not None:
        r = np.ascontiguousarray(ranker, np.float32)
        assert r.size == 641
        q.ranker = r.ctypes.data
        q._keep_r = r
    q.wT = 0
    q.wts = None
    if weights:
        T = {w.shape[0] for w in weights.values()}
        assert len(T) == 1
        n = max(weights) + 1
        arr = (C.c_void_p * n)()
        keep = []
        for k in range(n):
            if k in weights:
                a = np.ascontiguousarray(weights[k], np.float32)
                keep.append(a)
                arr[k] = a.ctypes.data
        q.wts = C.cast(arr, C.POINTER(C.c_void_p))
        q.wT = T.pop()
        q._keep = (arr, keep)
    return q


def code_matrices(code):
    c = make_code(code)
    w = code["l"] * code["m"]
    HX = np.zeros((w, 2 * w), np.uint8)
    HZ = np.zeros((w, 2 * w), np.uint8)
    lib().qdo_code_matrices(C.byref(c), _ptr(HX), _ptr(HZ))
    return HX, HZ


def gf2_rank(M):
    M = np.ascontiguousarray(M, dtype=np.uint8)
    return lib().qdo_gf2_rank(_ptr(M), M.shape[0], M.shape[1])


def logical_z(code):
    c = make_code(code)
    w = code["l"] * code["m"]
    LZ = np.zeros((64, 2 * w), np.uint8)
    K = lib().qdo_logical_z(C.byref(c), _ptr(LZ), 64)
    return LZ[:K].copy()


def logical_x(code):
    """Logical operators flipped by errors decoded with H_X (kernel of H_Z
    modulo the row span of H_X)."""
    c = make_code(code)
    w = code["l"] * code["m"]
    LX = np.zeros((64, 2 * w), np.uint8)
    K = lib().qdo_logical_x(C.byref(c), _ptr(LX), 64)
    return LX[:K].copy()


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().qdo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def bp_run(n_rows, col_ptr, col_rows, llr, synd, alpha=1.0, clip=50.0, max_iter=100,
           early_stop=True):
    col_ptr = np.ascontiguousarray(col_ptr, np.int32)
    col_rows = np.ascontiguousarray(col_rows, np.int32)
    llr = np.ascontiguousarray(llr, np.float32)
    synd = np.ascontiguousarray(synd, np.uint8)
    n = len(col_ptr) - 1
    e = np.zeros(n, np.uint8)
    post = np.zeros(n, np.float32)
    it = lib().qdo_bp_run(n_rows, n, _ptr(col_ptr), _ptr(col_rows), _ptr(llr), _ptr(synd),
                          alpha, clip, max_iter, int(early_stop), _ptr(e), _ptr(post))
    return it, e, post


def gdg_graph(params, n_rows, col_ptr, col_rows, llr, synd):
    col_ptr = np.ascontiguousarray(col_ptr, np.int32)
    col_rows = np.ascontiguousarray(col_rows, np.int32)
    llr = np.ascontiguousarray(llr, np.float32)
    synd = np.ascontiguousarray(synd, np.uint8)
    n = len(col_ptr) - 1
    e = np.zeros(n, np.uint8)
    P = make_params(params)
    nb = lib().qdo_n_paths(C.byref(P))
    br = (QdoBranch * nb)()
    best = lib().qdo_gdg_graph(C.byref(P), n_rows, n, _ptr(col_ptr), _ptr(col_rows), _ptr(llr),
                               _ptr(synd), _ptr(e), br)
    return best, e, [(b.status, b.depth, b.iters, b.pm) for b in br]


class OracleDEM:
    """Detector error model built by the oracle (direct per-fault simulation)."""

    def __init__(self, code, p, rounds, capacity=None):
        """Circuit-level DEM of the Z-basis memory (rounds noisy rounds), or,
        with capacity=(p_data, p_synd), the code-capacity model of the
        appendices decoded with H_X ([H_X | I] when p_synd > 0)."""
        self.code = code
        self.p = p
        self.rounds = rounds
        self._c = make_code(code)
        if capacity is None:
            self.h = lib().qdo_dem_build(C.byref(self._c), p, rounds)
        else:
            self.h = lib().qdo_dem_code_capacity(C.byref(self._c), float(capacity[0]), float(capacity[1]))
        info = np.zeros(6, np.int32)
        lib().qdo_dem_info(self.h, _ptr(info))
        self.n_det, self.n_cols, self.K, self.n_blocks, self.w, nnz = (int(x) for x in info)
        self.col_ptr = np.zeros(self.n_cols + 1, np.int32)
        self.col_dets = np.zeros(max(nnz, 1), np.int32)
        self.col_obs = np.zeros(self.n_cols, np.uint32)
        self.col_p = np.zeros(self.n_cols, np.float64)
        self.col_llr = np.zeros(self.n_cols, np.float32)
        lib().qdo_dem_columns(self.h, _ptr(self.col_ptr), _ptr(self.col_dets), _ptr(self.col_obs),
                              _ptr(self.col_p), _ptr(self.col_llr))
        self.det_words = (self.n_det + 31) // 32

    def __del__(self):
        if getattr(self, "h", None):
            lib().qdo_dem_free(self.h)
            self.h = None

    def column(self, c):
        return tuple(self.col_dets[self.col_ptr[c]:self.col_ptr[c + 1]].tolist()), int(self.col_obs[c])

    def n_fault_locations(self):
        return lib().qdo_n_fault_locations(self.h)

    def fault_effect(self, loc, pattern):
        dets = np.zeros(self.n_det, np.int32)
        obs = np.zeros(1, np.uint32)
        info = np.zeros(4, np.int32)
        nd = lib().qdo_fault_effect(self.h, loc, pattern, _ptr(dets), self.n_det, _ptr(obs),
                                    _ptr(info))
        return tuple(dets[:nd].tolist()), int(obs[0]), info.tolist()

    def circuit_ops(self):
        n = lib().qdo_circuit_ops(self.h, None, 0)
        out = np.zeros((n, 4), np.int32)
        lib().qdo_circuit_ops(self.h, _ptr(out), n)
        return out

    def logical_matrix(self):
        LZ = np.zeros((self.K, 2 * self.w), np.uint8)
        lib().qdo_logical_matrix(self.h, _ptr(LZ))
        return LZ

    def noiseless_detectors(self):
        out = np.zeros(self.n_det, np.uint8)
        lib().qdo_noiseless_detectors(self.h, _ptr(out))
        return out

    # ---- windows ----
    def n_windows(self, W, F):
        return lib().qdo_n_windows(self.h, W, F)

    def window(self, W, F, k, merge=0):
        """Window k as GDG decodes it (merge: the H_1 merge of Sec. III, 0 none)."""
        info = np.zeros(7, np.int32)
        lib().qdo_window_build(self.h, W, F, k, merge, _ptr(info), None, None, None, None, None)
        r0, nb, nr, nc, ne, ncom, last = (int(x) for x in info)
        gcols = np.zeros(nc, np.int32)
        cp = np.zeros(nc + 1, np.int32)
        cr = np.zeros(max(ne, 1), np.int32)
        com = np.zeros(nc, np.uint8)
        llr = np.zeros(nc, np.float32)
        lib().qdo_window_build(self.h, W, F, k, merge, _ptr(info), _ptr(gcols), _ptr(cp), _ptr(cr), _ptr(com),
                               _ptr(llr))
        return dict(r0=r0, n_blocks=nb, n_rows=nr, n_cols=nc, n_edges=ne, n_commit=ncom,
                    last=bool(last), gcols=gcols, col_ptr=cp, col_rows=cr[:ne], commit=com, llr=llr)

    # ---- sampling ----
    def sample(self, seed, shot_offset, n_shots):
        det = np.zeros((n_shots, self.det_words), np.uint32)
        obs = np.zeros(n_shots, np.uint32)
        lib().qdo_sample(self.h, seed, shot_offset, n_shots, _ptr(det), _ptr(obs))
        return det, obs

    # ---- decoding ----
    def decode_window(self, params, k, synd, trace=False, weights=None, ranker=None, dump=None):
        """dump: None or a RANK_REC array that receives path 0's candidate
        records (the returned info carries 'n_dump', the number produced)."""
        W, F = params["W"], params["F"]
        win = self.window(W, F, k, params.get("merge_h1", 0))
        synd = np.ascontiguousarray(synd, np.uint8)
        corr = np.zeros(win["n_cols"], np.uint8)
        info = np.zeros(4, np.int32)
        P = make_params(params, weights, ranker)
        dn = np.zeros(1, np.int32)
        if dump is not None:
            assert dump.dtype == RANK_REC and dump.flags.c_contiguous
            P.dump = dump.ctypes.data
            P.dump_n = dn.ctypes.data
            P.dump_cap = dump.shape[0]
        nb = lib().qdo_n_paths(C.byref(P))
        dmx = lib().qdo_path_dmax_all(C.byref(P))
        if trace:
            sc = np.zeros(win["n_cols"], np.int32)
            br = (QdoBranch * nb)()
            steps = (QdoStep * (nb * dmx))()
            fst = np.zeros(nb * win["n_cols"], np.int8)
            lib().qdo_decode_window(self.h, C.byref(P), k, _ptr(synd), _ptr(corr), _ptr(info),
                                    _ptr(sc), br, steps, _ptr(fst))
            ns = int(info[2])
            tr = dict(short_cols=sc[:ns].copy(),
                      branches=[(b.status, b.depth, b.iters, b.pm) for b in br],
                      steps=[[(s.g, s.value, s.n_agg, s.n_peel) for s in steps[i * dmx:(i + 1) * dmx]]
                             for i in range(nb)],
                      final_status=fst[:nb * ns].reshape(nb, ns).copy())
        else:
            lib().qdo_decode_window(self.h, C.byref(P), k, _ptr(synd), _ptr(corr), _ptr(info),
                                    None, None, None, None)
            tr = None
        return corr, dict(n_dump=int(dn[0]), prebp_converged=bool(info[0]), winner=int(info[1]),
                          n_short=int(info[2]), prebp_iters=int(info[3])), tr

    def decode_window_reuse(self, params, k, synd, init=None):
        """One window with message reuse: returns (corrections, info dict, kept
        values [n_cols]); init [n_cols] or None (NaN entries: the prior)."""
        win = self.window(params["W"], params["F"], k, params.get("merge_h1", 0))
        synd = np.ascontiguousarray(synd, np.uint8)
        corr = np.zeros(win["n_cols"], np.uint8)
        info = np.zeros(4, np.int32)
        keep = np.zeros(win["n_cols"], np.float32)
        ini = None if init is None else np.ascontiguousarray(init, np.float32)
        P = make_params(params)
        lib().qdo_decode_window_ex(self.h, C.byref(P), k, _ptr(synd), _ptr(corr), _ptr(info), _ptr(ini), _ptr(keep))
        return corr, dict(prebp_converged=bool(info[0]), winner=int(info[1]), n_short=int(info[2]),
                          prebp_iters=int(info[3])), keep

    def decode_window_paths(self, params, k, synd):
        """One window, with every decision path's final estimate: returns
        (corrections [n_cols], info dict, estimates [n_paths][n_cols]; zeros
        when the pre-BP converged)."""
        win = self.window(params["W"], params["F"], k, params.get("merge_h1", 0))
        synd = np.ascontiguousarray(synd, np.uint8)
        corr = np.zeros(win["n_cols"], np.uint8)
        info = np.zeros(4, np.int32)
        P = make_params(params)
        est = np.zeros((lib().qdo_n_paths(C.byref(P)), win["n_cols"]), np.uint8)
        lib().qdo_decode_window_paths(self.h, C.byref(P), k, _ptr(synd), _ptr(corr), _ptr(info), _ptr(est))
        return corr, dict(prebp_converged=bool(info[0]), winner=int(info[1]), n_short=int(info[2]),
                          prebp_iters=int(info[3])), est

    def run_shots(self, params, det, obs, threads=1, want_corr=False, weights=None, ranker=None):
        """Sliding-window decode of every shot.  Returns (fail, obs_pred, corr_words)."""
        det = np.ascontiguousarray(det, np.uint32)
        obs = np.ascontiguousarray(obs, np.uint32)
        n = det.shape[0]
        fail = np.zeros(n, np.uint8)
        pred = np.zeros(n, np.uint32)
        nwin = self.n_windows(params["W"], params["F"])
        maxc = max(self.window(params["W"], params["F"], k, params.get("merge_h1", 0))["n_cols"] for k in range(nwin))
        cw = (maxc + 31) // 32
        corr = np.zeros((n, nwin, cw), np.uint32) if want_corr else None
        P = make_params(params, weights, ranker)

        def work(a, b):
            lib().qdo_run_shots(self.h, C.byref(P), _ptr(det[a:b]), _ptr(obs[a:b]), b - a,
                                _ptr(fail[a:b]), _ptr(pred[a:b]),
                                _ptr(corr[a:b]) if want_corr else None, cw)

        threads = max(1, min(threads, n))
        if threads == 1:
            work(0, n)
        else:
            bounds = np.linspace(0, n, threads + 1).astype(int)
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda ab: work(*ab), zip(bounds[:-1], bounds[1:])))
        return fail, pred, corr


def default_threads():
    return max(1, len(os.sched_getaffinity(0)))
