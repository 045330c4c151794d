"""Thin ctypes binding of include/seg.h (argument marshalling only).

Every step of the path runs in the CUDA kernels of ``libseg.so``; this module
only converts torch tensors to device pointers, calls the C entry points of the
same names and turns negative return codes into :class:`SegError`.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the library
is missing the import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libseg.so")

SEG_OK = 0
SEG_EINVAL = -1
SEG_ENOMEM = -2
SEG_ENOTCONVERGED = -3
SEG_ECUDA = -4
SEG_ETIMEOUT = -5
SEG_ECAPACITY = -6
SEG_MINCUT_STATIC_MAX_PIXELS = 131072


class SegError(RuntimeError):
    def __init__(self, code: int, where: str):
        detail = ""
        if code == SEG_ECUDA and "lib" in globals():
            detail = ": " + lib.seg_last_cuda_error().decode(errors="replace")
        super().__init__(f"{where}: {strerror(code)} ({code}){detail}")
        self.code = code


class seg_params(C.Structure):
    _fields_ = [
        ("levels", C.c_int32), ("c_min", C.c_int32), ("c_max", C.c_int32), ("d_min", C.c_int32),
        ("d_max", C.c_int32), ("n_orient", C.c_int32), ("gabor_lambda", C.c_float),
        ("gabor_sigma", C.c_float), ("gabor_radius", C.c_int32), ("norm_tile", C.c_int32),
        ("norm_flat", C.c_float), ("w", C.c_float * 4), ("cs_opponent_sum", C.c_int32),
        ("border_px", C.c_int32), ("sigma1", C.c_double), ("sigma2", C.c_double),
        ("f_sigma", C.c_float), ("f_radius", C.c_int32), ("eps", C.c_float),
        ("lambda_u", C.c_double), ("lambda_p", C.c_double), ("lambda_s", C.c_double),
        ("sigma_I", C.c_double), ("cap_scale", C.c_double), ("neighbourhood", C.c_int32),
        ("max_cycles", C.c_int32), ("global_relabel_every", C.c_int32), ("local_iters", C.c_int32),
        ("use_graph", C.c_int32), ("gmm_components", C.c_int32), ("em_iters", C.c_int32),
        ("warm_start", C.c_int32), ("barrier_timeout_us", C.c_int32), ("kmeans_iters", C.c_int32),
        ("gmm_update", C.c_int32), ("relabel_frontier", C.c_int32), ("cut_tile", C.c_int32),
    ]


class seg_frame_io(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("sal", C.c_void_p), ("prior", C.c_void_p), ("mask", C.c_void_p),
                ("cut", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i32, P = C.c_void_p, C.c_int, C.POINTER
    sig = {
        "seg_default_params": ([P(seg_params)], i32),
        "seg_create": ([vp, i32, i32, P(seg_params), P(vp)], i32),
        "seg_create_batch": ([vp, i32, i32, i32, P(seg_params), P(vp)], i32),
        "seg_reset_stream": ([vp, i32], i32),
        "seg_set_stream_active": ([vp, i32, i32], i32),
        "seg_workspace_bytes": ([i32, i32, i32, P(seg_params), P(C.c_size_t)], i32),
        "seg_destroy": ([vp], i32),
        "seg_reset": ([vp], i32),
        "seg_set_barrier_timeout": ([vp, i32], i32),
        "seg_push_frame": ([vp, vp, vp, vp, vp, vp], i32),
        "seg_push_frame_host": ([vp, vp, vp, vp, vp, vp], i32),
        "seg_sync": ([vp, P(C.c_int)], i32),
        "seg_last_cuda_error": ([], C.c_char_p),
        "seg_group_create": ([vp, P(vp), i32, P(vp)], i32),
        "seg_group_push": ([vp, P(seg_frame_io)], i32),
        "seg_group_sync": ([vp, P(C.c_int), P(C.c_int)], i32),
        "seg_group_destroy": ([vp], i32),
        "seg_get_state": ([vp, vp, P(C.c_size_t)], i32),
        "seg_set_state": ([vp, vp, C.c_size_t], i32),
        "seg_strerror": ([i32], C.c_char_p),
        "seg_saliency": ([vp, vp, vp], i32),
        "seg_prior": ([vp, vp, vp, C.c_double, vp], i32),
        "seg_terms": ([vp, vp, vp, vp, vp, vp], i32),
        "seg_mincut": ([vp, vp, vp, vp, vp, vp], i32),
        "seg_mincut_grid": ([vp, i32, i32, i32, vp, vp, vp, vp, vp, i32, P(C.c_int)], i32),
        "seg_mincut_grid_static": ([vp, i32, i32, i32, vp, vp, vp, vp, vp, i32, P(C.c_int)], i32),
        "seg_debug_copy": ([vp, i32, i32, vp, C.c_size_t], i32),
        "seg_level_dim": ([i32, i32], i32),
        "seg_profile_enable": ([vp, i32], i32),
        "seg_profile_read": ([vp, P(C.c_double), P(C.c_int), P(C.c_longlong), vp, i32], i32),
        "seg_profile_read_ex": ([vp, P(C.c_double), P(C.c_int), P(C.c_longlong), vp, vp, i32], i32),
        "seg_pipeline_enable": ([vp, i32], i32),
        "seg_saliency_grid": ([vp, i32, i32, P(seg_params), vp, vp], i32),
        "seg_push_frame_ev": ([vp, vp, vp, vp, vp, vp, vp], i32),
        "seg_push_frame_host_async": ([vp, vp, vp, vp], i32),
        "seg_diff_workspace_bytes": ([i32, i32, i32, P(seg_params), P(C.c_size_t)], i32),
        "seg_diff_create": ([vp, i32, i32, i32, P(seg_params), P(vp)], i32),
        "seg_diff_destroy": ([vp], i32),
        "seg_diff_forward": ([vp, vp, vp, vp, i32, vp, vp], i32),
        "seg_diff_backward": ([vp, vp, vp, vp, vp, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def strerror(code: int) -> str:
    return lib.seg_strerror(code).decode()


def _check(code: int, where: str) -> int:
    if code != SEG_OK:
        raise SegError(code, where)
    return code


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype, shape, name):
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def _host(t, dtype, numel, name):
    """Pointer to a host buffer, after checking that it holds exactly what the
    library copies through it (the C side trusts the size it derives from H, W, B)."""
    if t is None:
        return None
    if t.device.type != "cpu":
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype or t.numel() != numel:
        raise ValueError(f"{name}: expected {dtype} with {numel} elements, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def default_params(**over) -> seg_params:
    p = seg_params()
    _check(lib.seg_default_params(C.byref(p)), "seg_default_params")
    for k, v in over.items():
        if k == "w":
            p.w = (C.c_float * 4)(*v)
        else:
            setattr(p, k, v)
    return p


def params_from(cfg: dict, **over) -> seg_params:
    """seg_params from a plain dict of field values (unknown keys are an error)."""
    d = dict(cfg)
    d.update(over)
    return default_params(**d)


def workspace_bytes(B: int, H: int, W: int, params: seg_params) -> int:
    n = C.c_size_t(0)
    _check(lib.seg_workspace_bytes(B, H, W, C.byref(params), C.byref(n)), "seg_workspace_bytes")
    return n.value


def level_dim(n: int, level: int) -> int:
    return lib.seg_level_dim(n, level)


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Segmenter:
    """One video stream: owns a seg_ctx (workspace + temporal state) on a CUDA stream."""

    def __init__(self, H: int, W: int, params: seg_params | None = None, stream=None, device=None,
                 batch: int = 1, pipeline: bool = False):
        self.H, self.W, self.B = H, W, batch
        self.device = torch.device(device) if device is not None else torch.device("cuda",
                                                                                   torch.cuda.current_device())
        self.params = params if params is not None else default_params()
        with torch.cuda.device(self.device):
            # a stream of its own (not the legacy default stream) lets the library replay
            # one captured CUDA graph per frame; it is a blocking stream, so work queued on
            # the default stream before a call is ordered before it
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            h = C.c_void_p()
            _check(lib.seg_create_batch(_stream_handle(self.stream), batch, H, W, C.byref(self.params),
                                        C.byref(h)), "seg_create_batch")
        self.handle = h
        self.nk = self.params.neighbourhood // 2
        # pipelined frames: frame t's saliency overlaps frame t-1's prior, terms and cut.
        # push_frame then does not order the caller's stream after the outputs: call
        # outputs_ready() (or sync()) before using them.
        self.pipeline = bool(pipeline)
        if self.pipeline:
            _check(lib.seg_pipeline_enable(h, 1), "seg_pipeline_enable")

    # The context runs on its own stream; every call orders it after the caller's
    # current stream (inputs ready) and the caller's stream after it (outputs ready),
    # so tensors can be used on the current stream as usual.
    def _begin(self):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
        return cur

    def _end(self, cur):
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def close(self):
        if getattr(self, "handle", None):
            lib.seg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- buffers
    def _shape(self, *tail):
        return (self.H, self.W) + tail if self.B == 1 else (self.B, self.H, self.W) + tail

    def empty_outputs(self):
        d = self.device
        return (torch.empty(self._shape(), dtype=torch.float32, device=d),
                torch.empty(self._shape(), dtype=torch.float32, device=d),
                torch.empty(self._shape(), dtype=torch.uint8, device=d),
                torch.empty(self.B, dtype=torch.int64, device=d))

    # --- whole method
    def push_frame(self, rgb, saliency=None, prior=None, mask=None, cut=None):
        """One frame of every stream (rgb (H,W,3), or (B,H,W,3) for a batch)."""
        if mask is None:
            saliency, prior, mask, cut = self.empty_outputs()
        args = (_dev(rgb, torch.uint8, self._shape(3), "rgb"),
                _dev(saliency, torch.float32, self._shape(), "saliency") if saliency is not None else None,
                _dev(prior, torch.float32, self._shape(), "prior") if prior is not None else None,
                _dev(mask, torch.uint8, self._shape(), "mask"),
                _dev(cut, torch.int64, (self.B,), "cut") if cut is not None else None)
        if self.pipeline:
            cur = torch.cuda.current_stream(self.device)
            ready = torch.cuda.Event()
            ready.record(cur)  # the frame's data is ready on the caller's stream
            if cur != self.stream:
                self.stream.wait_stream(cur)  # outputs: earlier readers on the caller's stream come first
            _check(lib.seg_push_frame_ev(self.handle, *args, C.c_void_p(ready.cuda_event)), "seg_push_frame_ev")
            for t in (rgb, saliency, prior, mask, cut):
                if t is not None:
                    t.record_stream(self.stream)
            self._ready_events = getattr(self, "_ready_events", [])[-7:] + [ready]  # keep alive until used
            return saliency, prior, mask, cut
        cur = self._begin()
        _check(lib.seg_push_frame(self.handle, *args), "seg_push_frame")
        self._end(cur)
        return saliency, prior, mask, cut

    def push_frame_host_async(self, rgb_host, mask_host, cut_host=None):
        """Pipelined host-buffer frame: no host wait; results complete after sync().
        The host buffers must stay untouched until then."""
        n = self.B * self.H * self.W
        args = (_host(rgb_host, torch.uint8, 3 * n, "rgb_host"), _host(mask_host, torch.uint8, n, "mask_host"),
                _host(cut_host, torch.int64, self.B, "cut_host"))
        _check(lib.seg_push_frame_host_async(self.handle, *args), "seg_push_frame_host_async")

    def outputs_ready(self, stream=None):
        """Orders `stream` (default: the current stream) after every frame pushed so far."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        if s != self.stream:
            s.wait_stream(self.stream)

    def push_frame_host(self, rgb_host, mask_host, cut_host=None, saliency_host=None, prior_host=None):
        n = self.B * self.H * self.W
        args = (_host(rgb_host, torch.uint8, 3 * n, "rgb_host"),
                _host(saliency_host, torch.float32, n, "saliency_host"),
                _host(prior_host, torch.float32, n, "prior_host"),
                _host(mask_host, torch.uint8, n, "mask_host"), _host(cut_host, torch.int64, self.B, "cut_host"))
        return _check(lib.seg_push_frame_host(self.handle, *args), "seg_push_frame_host")

    def sync(self, check=True):
        cyc = C.c_int(0)
        code = lib.seg_sync(self.handle, C.byref(cyc))
        if check:
            _check(code, "seg_sync")
        return code, cyc.value

    def reset(self, stream_index=None):
        cur = self._begin()
        if stream_index is None:
            _check(lib.seg_reset(self.handle), "seg_reset")
        else:
            _check(lib.seg_reset_stream(self.handle, int(stream_index)), "seg_reset_stream")
        self._end(cur)

    def set_barrier_timeout(self, us: int):
        """Time limit of the min cut's grid-barrier waits (seg_set_barrier_timeout); waits for
        the context's stream and re-captures its graphs on the next frame."""
        _check(lib.seg_set_barrier_timeout(self.handle, int(us)), "seg_set_barrier_timeout")
        self.params.barrier_timeout_us = int(us)

    def set_stream_active(self, b: int, on: bool):
        """Slot b of a batch holds a stream (True) or is empty (False: its frame is skipped)."""
        cur = self._begin()
        _check(lib.seg_set_stream_active(self.handle, int(b), int(bool(on))), "seg_set_stream_active")
        self._end(cur)

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib.seg_get_state(self.handle, None, C.byref(n)), "seg_get_state")
        buf = C.create_string_buffer(n.value)
        _check(lib.seg_get_state(self.handle, buf, C.byref(n)), "seg_get_state")
        return buf.raw

    def set_state(self, state: bytes):
        _check(lib.seg_set_state(self.handle, C.c_char_p(state), len(state)), "seg_set_state")

    def profile_enable(self, on=True):
        _check(lib.seg_profile_enable(self.handle, int(on)), "seg_profile_enable")

    def profile_read(self, max_frames=4096):
        ms = (C.c_double * 4)()
        n = C.c_int(0)
        cyc = C.c_longlong(0)
        fr = (C.c_float * max_frames)()
        st = (C.c_int * (7 * max_frames))()
        _check(lib.seg_profile_read_ex(self.handle, ms, C.byref(n), C.byref(cyc), fr, st, max_frames),
               "seg_profile_read_ex")
        k = min(n.value, max_frames)
        return {"stage_ms": list(ms), "frames": n.value, "cycles": cyc.value, "frame_ms": list(fr[:k]),
                "mincut_stats": [tuple(st[7 * i:7 * i + 7]) for i in range(k)]}

    # --- stage entry points
    def saliency(self, rgb, out=None):
        out = out if out is not None else torch.empty(self._shape(), dtype=torch.float32, device=self.device)
        cur = self._begin()
        _check(lib.seg_saliency(self.handle, _dev(rgb, torch.uint8, self._shape(3), "rgb"),
                                _dev(out, torch.float32, self._shape(), "saliency")), "seg_saliency")
        self._end(cur)
        return out

    def prior(self, saliency, prev_mask, w_f, out=None):
        out = out if out is not None else torch.empty(self.H, self.W, dtype=torch.float32, device=self.device)
        pm = _dev(prev_mask, torch.uint8, (self.H, self.W), "prev_mask") if prev_mask is not None else None
        cur = self._begin()
        _check(lib.seg_prior(self.handle, _dev(saliency, torch.float32, (self.H, self.W), "saliency"), pm,
                             float(w_f), _dev(out, torch.float32, (self.H, self.W), "prior")), "seg_prior")
        self._end(cur)
        return out

    def terms(self, rgb, prior):
        H, W, d = self.H, self.W, self.device
        cs = torch.empty(H, W, dtype=torch.int32, device=d)
        ct = torch.empty(H, W, dtype=torch.int32, device=d)
        nc = torch.empty(self.nk, H, W, dtype=torch.int32, device=d)
        cur = self._begin()
        _check(lib.seg_terms(self.handle, _dev(rgb, torch.uint8, (H, W, 3), "rgb"),
                             _dev(prior, torch.float32, (H, W), "prior"), _ptr(cs), _ptr(ct), _ptr(nc)),
               "seg_terms")
        self._end(cur)
        return cs, ct, nc

    def mincut(self, cs, ct, ncap, mask=None, cut=None):
        H, W, d = self.H, self.W, self.device
        mask = mask if mask is not None else torch.empty(H, W, dtype=torch.uint8, device=d)
        cut = cut if cut is not None else torch.empty(1, dtype=torch.int64, device=d)
        cur = self._begin()
        _check(lib.seg_mincut(self.handle, _dev(cs, torch.int32, (H, W), "cs"), _dev(ct, torch.int32, (H, W), "ct"),
                              _dev(ncap, torch.int32, (self.nk, H, W), "ncap"), _ptr(mask), _ptr(cut)),
               "seg_mincut")
        self._end(cur)
        return mask, cut

    def debug_copy(self, which: int, index: int, shape):
        out = torch.empty(*shape, dtype=torch.float32)
        _check(lib.seg_debug_copy(self.handle, which, index, _ptr(out), out.numel()), "seg_debug_copy")
        return out


def saliency_grid(rgb, params: seg_params | None = None, stream=None, out=None):
    """Saliency map of one (H, W, 3) uint8 CUDA frame without a context (own workspace)."""
    H, W = int(rgb.shape[0]), int(rgb.shape[1])
    p = params if params is not None else default_params()
    if out is None:
        out = torch.empty(H, W, dtype=torch.float32, device=rgb.device)
    st = stream if stream is not None else torch.cuda.current_stream(rgb.device)
    _check(lib.seg_saliency_grid(C.c_void_p(st.cuda_stream), H, W, C.byref(p), _dev(rgb, torch.uint8, (H, W, 3), "rgb"),
                                 _dev(out, torch.float32, (H, W), "out")), "seg_saliency_grid")
    return out


def mincut_grid(cs, ct, ncap, max_cycles: int = 0, stream=None):
    """Standalone exact min cut of an H x W grid.  Returns (mask, cut, status, cycles)."""
    H, W = cs.shape
    nk = ncap.shape[0]
    mask = torch.empty(H, W, dtype=torch.uint8, device=cs.device)
    cut = torch.empty(1, dtype=torch.int64, device=cs.device)
    cyc = C.c_int(0)
    code = lib.seg_mincut_grid(_stream_handle(stream), H, W, 2 * nk, _dev(cs, torch.int32, (H, W), "cs"),
                               _dev(ct, torch.int32, (H, W), "ct"), _dev(ncap, torch.int32, (nk, H, W), "ncap"),
                               _ptr(mask), _ptr(cut), int(max_cycles), C.byref(cyc))
    if code not in (SEG_OK, SEG_ENOTCONVERGED, SEG_ETIMEOUT, SEG_ECAPACITY):
        raise SegError(code, "seg_mincut_grid")
    return mask, cut, code, cyc.value


def mincut_grid_static(cs, ct, ncap, max_cycles: int = 0, stream=None, mask=None, cut=None):
    """seg_mincut_grid_static: the standalone min cut with the library's fixed
    device scratch instead of an allocation (H*W <= SEG_MINCUT_STATIC_MAX_PIXELS).
    Pass preallocated ``mask``/``cut`` tensors to keep the call allocation-free.
    Returns (mask, cut, status, cycles)."""
    H, W = cs.shape
    nk = ncap.shape[0]
    mask = mask if mask is not None else torch.empty(H, W, dtype=torch.uint8, device=cs.device)
    cut = cut if cut is not None else torch.empty(1, dtype=torch.int64, device=cs.device)
    cyc = C.c_int(0)
    code = lib.seg_mincut_grid_static(_stream_handle(stream), H, W, 2 * nk, _dev(cs, torch.int32, (H, W), "cs"),
                                      _dev(ct, torch.int32, (H, W), "ct"),
                                      _dev(ncap, torch.int32, (nk, H, W), "ncap"),
                                      _dev(mask, torch.uint8, (H, W), "mask"), _dev(cut, torch.int64, (1,), "cut"),
                                      int(max_cycles), C.byref(cyc))
    if code not in (SEG_OK, SEG_ENOTCONVERGED, SEG_ETIMEOUT, SEG_ECAPACITY):
        raise SegError(code, "seg_mincut_grid_static")
    return mask, cut, code, cyc.value


# ---------------------------------------------------------------- backward form
def diff_workspace_bytes(B: int, H: int, W: int, params: seg_params) -> int:
    n = C.c_size_t(0)
    _check(lib.seg_diff_workspace_bytes(B, H, W, C.byref(params), C.byref(n)), "seg_diff_workspace_bytes")
    return n.value


def theta_from(params: seg_params, device=None) -> torch.Tensor:
    """theta = (w_I, w_RG, w_BY, w_O, Q = sigma1^2, R = sigma2^2) of a params struct, float64 on the device."""
    v = [float(params.w[k]) for k in range(4)] + [params.sigma1 ** 2, params.sigma2 ** 2]
    return torch.tensor(v, dtype=torch.float64, device=device if device is not None else "cuda")


class DiffContext:
    """Backward-form context (seg_diff) for batches of B float frames of H x W:
    saliency and Kalman-updated prior of clip times t0..t0+B-1, and their reverse
    pass with respect to the frames and theta."""

    def __init__(self, B: int, H: int, W: int, params: seg_params | None = None, device=None):
        self.B, self.H, self.W = B, H, W
        self.device = torch.device(device) if device is not None else torch.device("cuda",
                                                                                   torch.cuda.current_device())
        self.params = params if params is not None else default_params()
        self.generation = 0  # counts forwards: the context holds the checkpoints of the last one
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(self.device)
            h = C.c_void_p()
            _check(lib.seg_diff_create(_stream_handle(self.stream), B, H, W, C.byref(self.params), C.byref(h)),
                   "seg_diff_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib.seg_diff_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _begin(self):
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        return cur

    def _end(self, cur):
        cur.wait_stream(self.stream)

    def _args(self, rgb, theta, fmap):
        B, H, W = self.B, self.H, self.W
        r = _dev(rgb, torch.float32, (B, H, W, 3), "rgb")
        th = _dev(theta, torch.float64, (6,), "theta")
        f = _dev(fmap, torch.float32, (B, H, W), "fmap") if fmap is not None else None
        return r, th, f

    def forward(self, rgb, theta, fmap=None, t0: int = 0, saliency=None, prior=None):
        B, H, W = self.B, self.H, self.W
        r, th, f = self._args(rgb, theta, fmap)
        if saliency is None:
            saliency = torch.empty(B, H, W, dtype=torch.float32, device=self.device)
        if prior is None:
            prior = torch.empty(B, H, W, dtype=torch.float32, device=self.device)
        cur = self._begin()
        _check(lib.seg_diff_forward(self.handle, r, f, th, int(t0), _dev(saliency, torch.float32, (B, H, W), "sal"),
                                    _dev(prior, torch.float32, (B, H, W), "prior")), "seg_diff_forward")
        self._end(cur)
        for t in (rgb, theta, fmap, saliency, prior):
            if t is not None:
                t.record_stream(self.stream)
        self.generation += 1
        return saliency, prior

    def backward(self, rgb, theta, g_prior, g_sal=None, fmap=None, g_rgb=None, g_theta=None):
        """Reverse pass of the last forward (same rgb, theta, fmap)."""
        B, H, W = self.B, self.H, self.W
        r, th, f = self._args(rgb, theta, fmap)
        gp = _dev(g_prior, torch.float32, (B, H, W), "g_prior")
        gs = _dev(g_sal, torch.float32, (B, H, W), "g_sal") if g_sal is not None else None
        if g_rgb is None:
            g_rgb = torch.empty(B, H, W, 3, dtype=torch.float32, device=self.device)
        if g_theta is None:
            g_theta = torch.empty(6, dtype=torch.float64, device=self.device)
        cur = self._begin()
        _check(lib.seg_diff_backward(self.handle, r, f, th, gp, gs, _dev(g_rgb, torch.float32, (B, H, W, 3), "g_rgb"),
                                     _dev(g_theta, torch.float64, (6,), "g_theta")), "seg_diff_backward")
        self._end(cur)
        for t in (rgb, theta, fmap, g_prior, g_sal, g_rgb, g_theta):
            if t is not None:
                t.record_stream(self.stream)
        return g_rgb, g_theta


class SaliencyFn(torch.autograd.Function):
    """(saliency, prior) = f(rgb, theta) as a torch.autograd.Function over a DiffContext.

    rgb: (B, H, W, 3) float32 frames at clip times t0..t0+B-1; theta: (6,) float64
    (w_I, w_RG, w_BY, w_O, Q, R); fmap: (B, H, W) float32 smoothed previous masks or
    None (a constant).  If the context ran another forward before this backward,
    the backward first recomputes this forward's checkpoints."""

    @staticmethod
    def forward(ctx, rgb, theta, fmap, t0, dctx):
        rgb, theta = rgb.contiguous(), theta.contiguous()
        fmap = fmap.contiguous() if fmap is not None else None
        sal, prior = dctx.forward(rgb, theta, fmap, t0)
        ctx.dctx, ctx.generation, ctx.t0, ctx.has_fmap = dctx, dctx.generation, t0, fmap is not None
        ctx.save_for_backward(rgb, theta, fmap if fmap is not None else rgb.new_empty(0))
        return sal, prior

    @staticmethod
    def backward(ctx, g_sal, g_prior):
        rgb, theta, fmap = ctx.saved_tensors
        fmap = fmap if ctx.has_fmap else None
        d = ctx.dctx
        if d.generation != ctx.generation:
            d.forward(rgb, theta, fmap, ctx.t0)
            ctx.generation = d.generation
        if g_prior is None:
            g_prior = torch.zeros(d.B, d.H, d.W, dtype=torch.float32, device=d.device)
        g_rgb, g_theta = d.backward(rgb, theta, g_prior.contiguous(),
                                    g_sal.contiguous() if g_sal is not None else None, fmap)
        return (g_rgb if ctx.needs_input_grad[0] else None, g_theta if ctx.needs_input_grad[1] else None,
                None, None, None)


_diff_cache: dict = {}


def saliency_prior(rgb, theta, fmap=None, t0: int = 0, params: seg_params | None = None):
    """Differentiable saliency and prior of a clip batch (see SaliencyFn).  Contexts
    are cached per (B, H, W, device, params)."""
    B, H, W = int(rgb.shape[0]), int(rgb.shape[1]), int(rgb.shape[2])
    p = params if params is not None else default_params()
    key = (B, H, W, str(rgb.device), bytes(p))
    d = _diff_cache.get(key)
    if d is None:
        d = _diff_cache[key] = DiffContext(B, H, W, p, device=rgb.device)
    return SaliencyFn.apply(rgb, theta, fmap, t0, d)


class Group:
    """seg_group: member Segmenters (batch contexts of different resolutions, say)
    advanced by one CUDA graph launch per frame step on the group's own stream.
    Results equal each member's push_frame; members keep their state and their
    per-stream calls (reset, set_stream_active, sync) between steps stay ordered."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (C.c_void_p * len(self.members))(*[m.handle for m in self.members])
        h = C.c_void_p()
        _check(lib.seg_group_create(C.c_void_p(self.stream.cuda_stream), arr, len(self.members), C.byref(h)),
               "seg_group_create")
        self.handle = h

    def push(self, frames, outs=None):
        """frames[i]: member i's frame tensor(s), shaped as its push_frame takes them;
        outs[i]: its (saliency, prior, mask, cut) buffers (allocated when None).
        Returns the outs."""
        if len(frames) != len(self.members):
            raise ValueError(f"{len(frames)} frames for {len(self.members)} members")
        outs = list(outs) if outs is not None else [m.empty_outputs() for m in self.members]
        io = (seg_frame_io * len(self.members))()
        for i, (m, f, o) in enumerate(zip(self.members, frames, outs)):
            sal, pr, mask, cut = o
            io[i].rgb = _dev(f, torch.uint8, m._shape(3), "rgb")
            io[i].sal = _dev(sal, torch.float32, m._shape(), "saliency") if sal is not None else None
            io[i].prior = _dev(pr, torch.float32, m._shape(), "prior") if pr is not None else None
            io[i].mask = _dev(mask, torch.uint8, m._shape(), "mask")
            io[i].cut = _dev(cut, torch.int64, (m.B,), "cut") if cut is not None else None
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            self.stream.wait_stream(cur)  # the frames are ready on the caller's stream
        _check(lib.seg_group_push(self.handle, io), "seg_group_push")
        if cur != self.stream:
            cur.wait_stream(self.stream)
        return outs

    def sync(self):
        """[(status, cycles)] of every member."""
        n = len(self.members)
        codes, cyc = (C.c_int * n)(), (C.c_int * n)()
        code = lib.seg_group_sync(self.handle, codes, cyc)
        if code == SEG_ECUDA or code == SEG_EINVAL:
            raise SegError(code, "seg_group_sync")
        return [(codes[i], cyc[i]) for i in range(n)]

    def close(self):
        if getattr(self, "handle", None):
            lib.seg_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
