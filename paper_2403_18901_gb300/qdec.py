"""Python binding of libqdec (argument marshalling only).

Every step of the decoder runs in the CUDA library; this module converts
torch tensors to raw pointers, numpy arrays to host pointers and C status
codes to exceptions.  There is no fallback: if libqdec.so is missing or a
call fails, it raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqdec.so")

QD_OK, QD_EINVAL, QD_ENOMEM, QD_ECUDA, QD_ETIMEOUT, QD_EUNSUPPORTED = range(6)
_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}


class QdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqdec {_NAMES.get(code, code)}: {msg}")
        self.code = code


class BBCode(C.Structure):
    _fields_ = [("l", C.c_int), ("m", C.c_int), ("a_x", C.c_int * 3), ("a_y", C.c_int * 3),
                ("b_x", C.c_int * 3), ("b_y", C.c_int * 3)]


class Noise(C.Structure):
    _fields_ = [("p", C.c_double), ("rounds", C.c_int)]


class GdgParams(C.Structure):
    _fields_ = [("W", C.c_int), ("F", C.c_int), ("alpha", C.c_float), ("n_pre", C.c_int),
                ("iters_per_step", C.c_int), ("d_max_main", C.c_int), ("d_max_other", C.c_int),
                ("k_guess", C.c_int), ("low_error_mode", C.c_int), ("peel_at_init", C.c_int),
                ("shorten", C.c_int), ("clip", C.c_float), ("pa_main", C.c_float),
                ("pa_other", C.c_float), ("pb_main", C.c_float), ("pb_other", C.c_float),
                ("pb_d1", C.c_float), ("pc", C.c_float), ("pd", C.c_float),
                ("pc_max_depth", C.c_int), ("n_unsat_min", C.c_int), ("side_max", C.c_int),
                ("reinit_on_split", C.c_int), ("iters_first", C.c_int), ("merge_h1", C.c_int),
                ("reuse_msgs", C.c_int), ("fallback", C.c_int)]


class DemInfo(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("n_det", "n_cols", "n_obs", "n_blocks", "w", "det_words",
                                       "n_edges")]


class WindowInfo(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("r0", "n_blocks", "n_rows", "n_cols", "n_edges", "n_commit",
                                       "is_last", "n_short")]


# symbol -> (restype, argtypes)
_VP, _I, _I64, _U64, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_size_t
_SIGS = {
    "qd_last_error_message": (C.c_char_p, []),
    "qd_build_dem": (_I, [C.POINTER(BBCode), C.POINTER(Noise), C.POINTER(_VP)]),
    "qd_build_dem_code_capacity": (_I, [C.POINTER(BBCode), C.c_double, C.c_double, C.POINTER(_VP)]),
    "qd_dem_info": (_I, [_VP, C.POINTER(DemInfo)]),
    "qd_dem_columns": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "qd_dem_window": (_I, [_VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, _VP, _VP]),
    "qd_path_plan": (_I, [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP]),
    "qd_dem_destroy": (_I, [_VP]),
    "qd_sample_shots": (_I, [_VP, _U64, _U64, _I64, _VP, _VP, _VP]),
    "qd_decoder_create": (_I, [_VP, C.POINTER(GdgParams), _I64, C.POINTER(_VP)]),
    "qd_decoder_destroy": (_I, [_VP]),
    "qd_decoder_n_windows": (_I, [_VP, C.POINTER(_I)]),
    "qd_decoder_corr_words": (_I, [_VP, C.POINTER(_I)]),
    "qd_decoder_path_info": (_I, [_VP, _VP]),
    "qd_window_info": (_I, [_VP, _I, C.POINTER(WindowInfo), _VP]),
    "qd_decoder_trace_bytes": (_I, [_VP, C.POINTER(_SZ)]),
    "qd_decode_windows": (_I, [_VP, _I, _VP, _I64, _VP, _VP, _VP, _VP]),
    "qd_commit_and_slide": (_I, [_VP, _I, _VP, _I64, _VP, _VP, _VP, _VP]),
    "qd_evaluate": (_I, [_VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "qd_decode_all": (_I, [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP]),
    "qd_decode_shots_host": (_I, [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP]),
    "qd_decode_commit_static": (_I, [_VP, _I, _VP, _I64, _VP, _VP, _VP]),
    "qd_decoder_set_launch": (_I, [_VP, _I]),
    "qd_decoder_launch_info": (_I, [_VP, _I, _VP]),
    "qd_decoder_set_weights": (_I, [_VP, _I, _VP, _I]),
    "qd_decoder_set_ranker": (_I, [_VP, _VP]),
    "qd_decoder_set_dump": (_I, [_VP, _VP, _VP, _I]),
    "qd_batch_create": (_I, [_VP, _I, C.POINTER(_VP)]),
    "qd_batch_destroy": (_I, [_VP]),
    "qd_batch_n_steps": (_I, [_VP, C.POINTER(_I)]),
    "qd_batch_step": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "qd_batch_set_shape": (_I, [_VP, _I, _I, _I]),
    "qd_batch_info": (_I, [_VP, _I, _VP]),
    "qd_batch_autotune": (_I, [_VP, _I, _VP, _VP, _I, _VP, _VP]),
    "qd_window_sample": (_I, [_VP, _I, _U64, _U64, _I64, _VP, _VP, _VP]),
    "qd_ranker_eval": (_I, [_VP, _VP, _VP, _I64, _I, C.c_float, C.c_float, _VP, _VP, _VP, _VP]),
    "qd_wms_create": (_I, [_VP, _I, _I, _I, C.POINTER(_VP)]),
    "qd_wms_destroy": (_I, [_VP]),
    "qd_wms_info": (_I, [_VP, _VP]),
    "qd_wms_sample": (_I, [_VP, _U64, _U64, _I64, _VP, _VP]),
    "qd_wms_loss": (_I, [_VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "qd_wms_grad": (_I, [_VP, _VP, _VP, _I64, C.c_float, _VP, _VP, _VP]),
    "qd_adam_step": (_I, [_VP, _VP, _VP, _VP, _I64, C.c_float, C.c_float, C.c_float, C.c_float, _I,
                          _VP]),
    "qd_decoder_counters": (_I, [_VP, _VP]),
    "qd_decoder_counters_ex": (_I, [_VP, _VP, C.c_int]),
    "qd_decoder_set_fork": (_I, [_VP, C.c_int]),
    "qd_decoder_reset_counters": (_I, [_VP, _VP]),
}

_lib = None


def lib():
    """Load libqdec.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libqdec.so not built ({LIB_PATH}); run paper_2403_18901_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != QD_OK:
        raise QdError(code, lib().qd_last_error_message().decode(errors="replace"))


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or numpy array; None passes through."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data_as(C.c_void_p)
    assert x.is_contiguous()
    return C.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_code(code):
    c = BBCode()
    c.l, c.m = code["l"], code["m"]
    for k in range(3):
        c.a_x[k], c.a_y[k] = code["A"][k]
        c.b_x[k], c.b_y[k] = code["B"][k]
    return c


def make_params(p):
    q = GdgParams()
    for name, _ in GdgParams._fields_:
        setattr(q, name, p.get(name, 0) if name in ("side_max", "reinit_on_split", "fallback") else p[name])
    return q


def path_plan(params, wave):
    """Shot mode's decision-path plan (host only): dict of nb, dmx, n_nodes
    (-1: no plan) and, with a plan, order [nb], chain [nb][dmx], fnode [nb],
    fdep [nb]."""
    info = np.zeros(3, np.int32)
    p = make_params(params)
    _check(lib().qd_path_plan(C.byref(p), int(wave), _ptr(info), None, None, None, None))
    nb, dmx, nn = (int(x) for x in info)
    out = dict(nb=nb, dmx=dmx, n_nodes=nn)
    if nn >= 0:
        order = np.zeros(nb, np.int16)
        chain = np.zeros(nb * dmx, np.int16)
        fnode = np.zeros(nb, np.int16)
        fdep = np.zeros(nb, np.int16)
        _check(lib().qd_path_plan(C.byref(p), int(wave), _ptr(info), _ptr(order), _ptr(chain), _ptr(fnode),
                                  _ptr(fdep)))
        out.update(order=order, chain=chain.reshape(nb, dmx), fnode=fnode, fdep=fdep)
    return out


class Dem:
    """Detector error model of the Z-basis memory experiment (qd_build_dem),
    or with capacity=(p_data, p_synd) the code-capacity model of the
    appendices (qd_build_dem_code_capacity; p and rounds are then ignored)."""

    def __init__(self, code, p, rounds, capacity=None):
        self.code, self.p, self.rounds = code, p, rounds
        h = C.c_void_p()
        if capacity is None:
            _check(lib().qd_build_dem(C.byref(make_code(code)), C.byref(Noise(p, rounds)), C.byref(h)))
        else:
            _check(lib().qd_build_dem_code_capacity(C.byref(make_code(code)), float(capacity[0]),
                                                    float(capacity[1]), C.byref(h)))
        self.h = h
        inf = DemInfo()
        _check(lib().qd_dem_info(self.h, C.byref(inf)))
        self.info = inf
        self.n_det, self.n_cols, self.K = inf.n_det, inf.n_cols, inf.n_obs
        self.w, self.det_words, self.n_blocks = inf.w, inf.det_words, inf.n_blocks

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qd_dem_destroy(self.h)
            self.h = None

    def columns(self):
        cp = np.zeros(self.n_cols + 1, np.int32)
        cd = np.zeros(max(self.info.n_edges, 1), np.int32)
        ob = np.zeros(self.n_cols, np.uint32)
        pr = np.zeros(self.n_cols, np.float64)
        ll = np.zeros(self.n_cols, np.float32)
        _check(lib().qd_dem_columns(self.h, _ptr(cp), _ptr(cd), _ptr(ob), _ptr(pr), _ptr(ll)))
        return dict(col_ptr=cp, col_dets=cd[:self.info.n_edges], obs=ob, prob=pr, llr=ll)

    def window(self, W, F, k, merge_h1=0):
        """Window k as the decoder builds it (host only): dict of r0, n_blocks,
        n_rows, n_cols, n_edges, n_commit, last, gcols, col_ptr, col_rows, llr."""
        info = np.zeros(7, np.int32)
        _check(lib().qd_dem_window(self.h, W, F, k, merge_h1, _ptr(info), None, None, None, None))
        r0, nb, nr, nc, ne, ncom, last = (int(x) for x in info)
        g = np.zeros(nc, np.int32)
        cp = np.zeros(nc + 1, np.int32)
        cr = np.zeros(max(ne, 1), np.int32)
        ll = np.zeros(nc, np.float32)
        _check(lib().qd_dem_window(self.h, W, F, k, merge_h1, _ptr(info), _ptr(g), _ptr(cp), _ptr(cr), _ptr(ll)))
        return dict(r0=r0, n_blocks=nb, n_rows=nr, n_cols=nc, n_edges=ne, n_commit=ncom, last=bool(last),
                    gcols=g, col_ptr=cp, col_rows=cr[:ne], llr=ll)

    def sample(self, seed, shot_offset, n_shots, det=None, obs=None, stream=None):
        import torch
        if det is None:
            det = torch.empty((n_shots, self.det_words), dtype=torch.int32, device="cuda")
        if obs is None:
            obs = torch.empty((n_shots,), dtype=torch.int32, device="cuda")
        _check(lib().qd_sample_shots(self.h, seed, shot_offset, n_shots, _ptr(det), _ptr(obs),
                                     _stream(stream)))
        return det, obs


class Decoder:
    """Sliding-window GDG decoder on the GPU (qd_decoder_create)."""

    def __init__(self, dem, params, max_shots):
        self.dem, self.params, self.max_shots = dem, dict(params), max_shots
        h = C.c_void_p()
        _check(lib().qd_decoder_create(dem.h, C.byref(make_params(params)), max_shots, C.byref(h)))
        self.h = h
        n = C.c_int()
        _check(lib().qd_decoder_n_windows(self.h, C.byref(n)))
        self.n_windows = n.value
        _check(lib().qd_decoder_corr_words(self.h, C.byref(n)))
        self.corr_words = n.value
        b = C.c_size_t()
        _check(lib().qd_decoder_trace_bytes(self.h, C.byref(b)))
        self.trace_bytes = b.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qd_decoder_destroy(self.h)
            self.h = None

    def window_info(self, k):
        wi = WindowInfo()
        _check(lib().qd_window_info(self.h, k, C.byref(wi), None))
        g = np.zeros(wi.n_cols, np.int32)
        _check(lib().qd_window_info(self.h, k, C.byref(wi), _ptr(g)))
        return dict(r0=wi.r0, n_blocks=wi.n_blocks, n_rows=wi.n_rows, n_cols=wi.n_cols,
                    n_edges=wi.n_edges, n_commit=wi.n_commit, last=bool(wi.is_last),
                    n_short=wi.n_short, gcols=g)

    def decode_window(self, k, det, n_shots, corr, status=None, trace=None, stream=None):
        _check(lib().qd_decode_windows(self.h, k, _ptr(det), n_shots, _ptr(corr), _ptr(status),
                                       _ptr(trace), _stream(stream)))

    def commit(self, k, corr, n_shots, det, obs_pred, resid, stream=None):
        _check(lib().qd_commit_and_slide(self.h, k, _ptr(corr), n_shots, _ptr(det), _ptr(obs_pred),
                                         _ptr(resid), _stream(stream)))

    def decode_commit_static(self, k, det, n_shots, obs_pred, resid, stream=None):
        """Decode + commit window k using the library's fixed scratch array
        (no device allocation; see qd_decode_commit_static)."""
        _check(lib().qd_decode_commit_static(self.h, k, _ptr(det), n_shots, _ptr(obs_pred),
                                             _ptr(resid), _stream(stream)))

    def decode_all(self, det, obs, n_shots, obs_pred, fail, n_fail=None, stream=None):
        _check(lib().qd_decode_all(self.h, _ptr(det), _ptr(obs), n_shots, _ptr(obs_pred),
                                   _ptr(fail), _ptr(n_fail), _stream(stream)))

    def decode_host(self, det, obs, stream=None):
        """Host numpy buffers in and out (qd_decode_shots_host)."""
        det = np.ascontiguousarray(det, np.uint32)
        obs = np.ascontiguousarray(obs, np.uint32)
        n = det.shape[0]
        pred = np.zeros(n, np.uint32)
        fail = np.zeros(n, np.uint32)
        nf = np.zeros(1, np.int64)
        _check(lib().qd_decode_shots_host(self.h, _ptr(det), _ptr(obs), n, _ptr(pred), _ptr(fail),
                                          _ptr(nf), _stream(stream)))
        return pred, fail, int(nf[0])

    def set_weights(self, k, w):
        """w: CUDA float32 tensor [T][n_edges of window k] (kept referenced), or None."""
        if w is None:
            _check(lib().qd_decoder_set_weights(self.h, k, None, 0))
            self._w = getattr(self, "_w", {})
            self._w.pop(k, None)
            return
        assert w.is_cuda and w.dtype.is_floating_point and w.dim() == 2
        self._w = getattr(self, "_w", {})
        self._w[k] = w
        _check(lib().qd_decoder_set_weights(self.h, k, _ptr(w), w.shape[0]))

    def set_ranker(self, params):
        """params: 641 float32 values W1[64][8], b1[64], W2[64], b2 (host
        array, copied), or None for the argmin of Alg. 1."""
        if params is None:
            _check(lib().qd_decoder_set_ranker(self.h, None))
            return
        r = np.ascontiguousarray(params, np.float32).reshape(-1)
        assert r.size == 641
        _check(lib().qd_decoder_set_ranker(self.h, _ptr(r)))

    def set_dump(self, records, count):
        """records: CUDA uint8 tensor [capacity, 48] (qd_rank_rec_t rows),
        count: CUDA int32 tensor [1] (caller zeroes it); None turns the dump off."""
        if records is None:
            _check(lib().qd_decoder_set_dump(self.h, None, None, 0))
            self._dump = None
            return
        assert records.is_cuda and records.dim() == 2 and records.shape[1] == 48
        self._dump = (records, count)
        _check(lib().qd_decoder_set_dump(self.h, _ptr(records), _ptr(count), records.shape[0]))

    def window_sample(self, k, seed, offset, n, det, fault=None, stream=None):
        """Window-local samples of window k into det [n][det_words] (and the
        fired window columns into fault [n][corr_words])."""
        _check(lib().qd_window_sample(self.h, k, seed, offset, n, _ptr(det), _ptr(fault) if fault is not None
                                      else None, _stream(stream)))

    def launch_info(self, k=0):
        out = np.zeros(8, np.int32)
        _check(lib().qd_decoder_launch_info(self.h, k, _ptr(out)))
        return dict(shot_smem=int(out[0]), shot_threads=int(out[1]), shot_ctas_per_sm=int(out[2]),
                    path_smem=int(out[3]), path_threads=int(out[4]), sms=int(out[5]),
                    path_cluster=int(out[6]), path_ctas_per_shot=int(out[7]))

    def set_launch(self, mode):
        """0 automatic, 1 shot mode (throughput), 2 path mode (latency), 3 shot
        mode with the path states in global memory."""
        _check(lib().qd_decoder_set_launch(self.h, int(mode)))

    def counters(self):
        """[pre-BP edge-iterations, GDG edge-iterations, pre-BP converged
        windows, GDG windows, bulk staging waits that ran out]"""
        out = np.zeros(5, np.int64)
        _check(lib().qd_decoder_counters(self.h, _ptr(out)))
        return out

    def counters_ex(self, n=8):
        """counters() then [5] the GDG edge-iterations actually executed (shared
        path prefixes computed once), [6..7] reserved."""
        out = np.zeros(n, np.int64)
        _check(lib().qd_decoder_counters_ex(self.h, _ptr(out), int(n)))
        return out

    def set_fork(self, mode):
        """Shot mode's path scheduling: 0 every path from the root, in a fixed
        order; 1 paths resume from snapshots of shared prefixes; 2 (default)
        also preemption at step boundaries, longest remaining work first."""
        _check(lib().qd_decoder_set_fork(self.h, int(mode)))

    def reset_counters(self, stream=None):
        _check(lib().qd_decoder_reset_counters(self.h, _stream(stream)))

    # ---- trace decoding (layout of the per-shot trace buffer) ----
    def parse_trace(self, buf):
        """buf: numpy uint8 [trace_bytes] of one shot."""
        pi = np.zeros(2, np.int32)
        _check(lib().qd_decoder_path_info(self.h, _ptr(pi)))
        nb, dmx = int(pi[0]), int(pi[1])
        ns_max = self._ns_max()
        head = np.frombuffer(buf[:16].tobytes(), np.int32)
        br_dt = np.dtype([("status", "<i4"), ("depth", "<i4"), ("iters", "<i4"), ("pad", "<i4"),
                          ("pm", "<f8")])
        st_dt = np.dtype([("g", "<i2"), ("value", "i1"), ("pad", "i1"), ("n_agg", "<i2"),
                          ("n_peel", "<i2")])
        o = 16
        br = np.frombuffer(buf[o:o + 24 * nb].tobytes(), br_dt)
        o += 24 * nb
        st = np.frombuffer(buf[o:o + 8 * nb * dmx].tobytes(), st_dt).reshape(nb, dmx)
        o += 8 * nb * dmx
        fs = np.frombuffer(buf[o:o + nb * ns_max].tobytes(), np.int8).reshape(nb, ns_max)
        o = (o + nb * ns_max + 1) & ~1
        sel = np.frombuffer(buf[o:o + 2 * ns_max].tobytes(), np.uint16)
        return dict(head=head, branches=br, steps=st, final_status=fs, short_cols=sel)

    def _ns_max(self):
        return max(self.window_info(k)["n_short"] for k in range(self.n_windows))


class Batch:
    """Several decoders advanced one window step at a time, each step one
    decode launch and one commit launch over all members (qd_batch_*)."""

    def __init__(self, decoders):
        arr = (C.c_void_p * len(decoders))(*[d.h for d in decoders])
        h = C.c_void_p()
        _check(lib().qd_batch_create(arr, len(decoders), C.byref(h)))
        self.h, self.members = h, list(decoders)
        n = C.c_int()
        _check(lib().qd_batch_n_steps(self.h, C.byref(n)))
        self.n_steps = n.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qd_batch_destroy(self.h)
            self.h = None

    @staticmethod
    def _ptrs(ts):
        return (C.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])

    def _args(self, det, n, pred=None, resid=None):
        self._keep = (self._ptrs(det), (C.c_int64 * len(n))(*n),
                      self._ptrs(pred) if pred is not None else None,
                      self._ptrs(resid) if resid is not None else None)
        return self._keep

    def step(self, j, det, n, pred, resid, stream=None):
        """det, pred, resid: per-member CUDA tensors; n: per-member shot counts."""
        a = self._args(det, n, pred, resid)
        _check(lib().qd_batch_step(self.h, j, a[0], a[1], a[2], a[3], _stream(stream)))

    def set_shape(self, j, warps, ctas_per_sm=2):
        _check(lib().qd_batch_set_shape(self.h, j, int(warps), int(ctas_per_sm)))

    def info(self, j):
        out = np.zeros(4, np.int32)
        _check(lib().qd_batch_info(self.h, j, _ptr(out)))
        return dict(warps=int(out[0]), smem=int(out[1]), ctas_per_sm=int(out[2]), members=int(out[3]))

    def autotune(self, j, det, n, reps=3, stream=None):
        a = self._args(det, n)
        ms = C.c_float()
        _check(lib().qd_batch_autotune(self.h, j, a[0], a[1], int(reps), _stream(stream), C.byref(ms)))
        return ms.value
