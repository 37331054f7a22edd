"""ctypes binding of libstereovae.so (include/stereovae.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA
kernels.  torch tensors provide device memory and streams.  If the library is
missing the binding raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_void_p
from dataclasses import dataclass

import numpy as np

from . import synth

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstereovae.so")

SV_OK, SV_ERR_INVALID_ARG, SV_ERR_CUDA, SV_ERR_OOM, SV_ERR_UNSUPPORTED, SV_ERR_TIMEOUT, SV_ERR_STATE = range(7)
SV_FP32, SV_BF16, SV_FP64_CHECK, SV_FP8 = 0, 1, 2, 3
SV_NET_TABLE1 = 1
PRECISIONS = {"fp32": SV_FP32, "bf16": SV_BF16, "fp64": SV_FP64_CHECK, "fp8": SV_FP8}


class SvConfig(ctypes.Structure):
    _fields_ = [("window", c_int), ("enc_ch", c_int * 3), ("latent_ch", c_int), ("dec_ch", c_int * 3),
                ("precision", c_int), ("flags", c_int)]


class SvPair(ctypes.Structure):
    _fields_ = [("left", c_void_p), ("right", c_void_p), ("width", c_int), ("height", c_int), ("pitch", c_int),
                ("max_disp", c_int)]


class SvCoarseOpts(ctypes.Structure):
    _fields_ = [("cost", c_int), ("census_window", c_int), ("aggregation", c_int), ("P1", c_float), ("P2", c_float),
                ("npaths", c_int), ("dt_sigma_s", c_float), ("dt_sigma_r", c_float), ("dt_iters", c_int),
                ("post", c_int)]


SV_COST_ZNCC, SV_COST_CENSUS = 0, 1
SV_AGG_NONE, SV_AGG_SGM, SV_AGG_DT = 0, 1, 2
SV_POST_SMP, SV_POST_MEDIAN = 1, 2


def coarse_opts(cost="zncc", aggregation="none", census_window=5, P1=0.1, P2=0.5, npaths=4, dt_sigma_s=8.0,
                dt_sigma_r=20.0, dt_iters=2, smp=False, median=False) -> SvCoarseOpts:
    """sv_coarse_opts from names: cost "zncc" | "census", aggregation "none" | "sgm" | "dt"."""
    o = SvCoarseOpts()
    o.cost = {"zncc": SV_COST_ZNCC, "census": SV_COST_CENSUS}[cost]
    o.census_window = census_window
    o.aggregation = {"none": SV_AGG_NONE, "sgm": SV_AGG_SGM, "dt": SV_AGG_DT}[aggregation]
    o.P1, o.P2, o.npaths = P1, P2, npaths
    o.dt_sigma_s, o.dt_sigma_r, o.dt_iters = dt_sigma_s, dt_sigma_r, dt_iters
    o.post = (SV_POST_SMP if smp else 0) | (SV_POST_MEDIAN if median else 0)
    return o


class SvProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", c_double)]


class SvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None

API = {
    "sv_status_string": ([c_int], c_char_p),
    "sv_last_error": ([c_void_p], c_char_p),
    "sv_param_count": ([POINTER(SvConfig)], c_size_t),
    "sv_create": ([POINTER(SvConfig), c_int, POINTER(c_void_p)], c_int),
    "sv_destroy": ([c_void_p], c_int),
    "sv_set_weights": ([c_void_p, c_void_p, c_size_t], c_int),
    "sv_get_weights": ([c_void_p, c_void_p, c_size_t], c_int),
    "sv_coarse_match": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                         c_void_p], c_int),
    "sv_coarse_match_sgm": ([c_void_p, POINTER(SvPair), c_int, c_float, c_float, c_int, POINTER(c_void_p),
                             POINTER(c_void_p), c_void_p], c_int),
    "sv_coarse_match_ex": ([c_void_p, POINTER(SvPair), c_int, POINTER(SvCoarseOpts), POINTER(c_void_p),
                            POINTER(c_void_p), c_void_p], c_int),
    "sv_postprocess": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), c_int, POINTER(c_void_p), c_void_p],
                       c_int),
    "sv_pipeline_ex": ([c_void_p, POINTER(SvPair), c_int, POINTER(SvCoarseOpts), POINTER(c_void_p), c_void_p], c_int),
    "sv_refine": ([c_void_p, POINTER(SvPair), POINTER(c_void_p), c_int, POINTER(c_void_p), c_void_p], c_int),
    "sv_pipeline": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), c_void_p], c_int),
    "sv_refine_train": ([c_void_p, POINTER(SvPair), POINTER(c_void_p), POINTER(c_void_p), c_int, POINTER(c_void_p),
                         POINTER(c_void_p), POINTER(c_void_p), c_void_p], c_int),
    "sv_refine_backward": ([c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p), c_void_p,
                            POINTER(c_void_p), c_void_p], c_int),
    "sv_loss": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                 POINTER(c_void_p), c_double, c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                 c_void_p], c_int),
    "sv_adam_step": ([c_void_p, c_void_p, c_int, c_double, c_double, c_double, c_double, c_void_p], c_int),
    "sv_loss_paper": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                       POINTER(c_void_p), POINTER(c_void_p), c_void_p, POINTER(c_void_p), POINTER(c_void_p),
                       POINTER(c_void_p), c_void_p], c_int),
    "sv_pipeline_host": ([c_void_p, POINTER(SvPair), c_int, POINTER(c_void_p), c_void_p], c_int),
    "sv_profile_enable": ([c_void_p, c_int], c_int),
    "sv_profile_read": ([c_void_p, POINTER(SvProfileEntry), c_int, POINTER(c_int), c_int], c_int),
    "sv_launch_count": ([c_void_p], ctypes.c_longlong),
    "sv_synchronize": ([c_void_p, c_void_p], c_int),
    "sv_set_option": ([c_void_p, c_char_p, ctypes.c_longlong], c_int),
    "sv_debug_activation": ([c_void_p, c_int, c_int, c_void_p, c_size_t], c_int),
    "sv_coarse_match_static": ([POINTER(SvPair), c_int, c_int, POINTER(c_void_p), POINTER(c_void_p),
                                POINTER(c_void_p), c_void_p], c_int),
    "sv_autotune": ([c_void_p, POINTER(SvPair), c_int, c_char_p, c_void_p], c_int),
    "sv_tuning": ([c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_double)], c_int),
}


def lib():
    """Load libstereovae.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2305_11566_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in API.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    try:
        return lib().sv_status_string(s).decode()
    except Exception:  # pragma: no cover
        return str(s)


def make_config(shape, window: int, precision: str | int = "fp32") -> SvConfig:
    """sv_config for a NetShape, or for the paper's Table I network when shape is "table1"."""
    c = SvConfig()
    c.window = window
    t1 = isinstance(shape, str) and shape == "table1"
    if not t1:
        c.enc_ch[:] = list(shape.enc)
        c.latent_ch = shape.latent
        c.dec_ch[:] = list(shape.dec)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.flags = SV_NET_TABLE1 if t1 else 0
    return c


def param_count(shape: synth.NetShape, window: int = 9) -> int:
    c = make_config(shape, window)
    return int(lib().sv_param_count(ctypes.byref(c)))


def _ptrs(items):
    arr = (c_void_p * max(1, len(items)))()
    for i, t in enumerate(items):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


@dataclass
class DevicePair:
    """A stereo pair resident on the GPU: pitched uint8 images [H, pitch]."""
    left: "object"
    right: "object"
    width: int
    height: int
    max_disp: int

    def __setattr__(self, name, value):
        object.__setattr__(self, name, value)
        object.__setattr__(self, "_fields", None)  # the marshalled fields follow any change

    @property
    def pitch(self) -> int:
        return int(self.left.stride(0))

    def fields(self) -> tuple:
        """(left, right, width, height, pitch, max_disp) as the C struct holds them (cached)."""
        f = self._fields
        if f is None:
            f = (self.left.data_ptr(), self.right.data_ptr(), self.width, self.height, self.pitch, self.max_disp)
            object.__setattr__(self, "_fields", f)
        return f

    def sv(self) -> SvPair:
        return SvPair(*self.fields())

    @property
    def coarse_hw(self):
        return self.height // 4, self.width // 4


def to_device(pair: synth.Pair, max_disp: int, device="cuda") -> DevicePair:
    import torch
    L = torch.from_numpy(synth.pitched(pair.left)).to(device)
    R = torch.from_numpy(synth.pitched(pair.right)).to(device)
    return DevicePair(L, R, pair.width, pair.height, max_disp)


# numpy view of an sv_pair array: one array build instead of one ctypes struct per pair
_SV_PAIR_DTYPE = np.dtype({"names": ["left", "right", "width", "height", "pitch", "max_disp"],
                           "formats": ["<u8", "<u8", "<i4", "<i4", "<i4", "<i4"],
                           "offsets": [SvPair.left.offset, SvPair.right.offset, SvPair.width.offset,
                                       SvPair.height.offset, SvPair.pitch.offset, SvPair.max_disp.offset],
                           "itemsize": ctypes.sizeof(SvPair)})


def _pairs_array(pairs):
    a = np.array([p.fields() for p in pairs] if len(pairs) else [(0, 0, 0, 0, 0, 0)], dtype=_SV_PAIR_DTYPE)
    return (SvPair * len(a)).from_buffer(a)


class Context:
    """One sv_ctx: configuration, weights and workspaces on one GPU.  shape: a NetShape, or
    "table1" for the paper's Table I network (FP32)."""

    def __init__(self, shape, window: int, precision: str = "fp32", device: int = 0):
        self.shape = shape
        self.latent = 1 if isinstance(shape, str) else shape.latent
        self.window = window
        self.precision = precision
        self.device = device
        cfg = make_config(shape, window, precision)
        h = c_void_p()
        s = lib().sv_create(ctypes.byref(cfg), device, ctypes.byref(h))
        if s != SV_OK:
            raise SvError(s, "sv_create failed")
        self._h = h
        self.n_params = int(lib().sv_param_count(ctypes.byref(cfg)))

    def close(self):
        if getattr(self, "_h", None):
            lib().sv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int):
        if s != SV_OK:
            raise SvError(s, lib().sv_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def set_weights(self, params):
        import torch
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, dtype=np.float32)
            self._check(lib().sv_set_weights(self._h, params.ctypes.data_as(c_void_p), params.size))
        else:
            t = params.detach().to(torch.float32).contiguous()
            self._check(lib().sv_set_weights(self._h, c_void_p(t.data_ptr()), t.numel()))

    def get_weights(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(lib().sv_get_weights(self._h, out.ctypes.data_as(c_void_p), out.size))
        return out

    # ---------------------------------------------------------------- inference
    def coarse_match(self, pairs, scores: bool = False, stream=None, out=None):
        import torch
        dev = pairs[0].left.device if pairs else "cuda"
        disp = out if out is not None else [torch.empty(p.coarse_hw, dtype=torch.int16, device=dev) for p in pairs]
        best = [torch.empty(p.coarse_hw, dtype=torch.float32, device=dev) for p in pairs] if scores else None
        second = [torch.empty(p.coarse_hw, dtype=torch.float32, device=dev) for p in pairs] if scores else None
        self._check(lib().sv_coarse_match(self._h, _pairs_array(pairs), len(pairs), _ptrs(disp),
                                          _ptrs(best) if scores else None, _ptrs(second) if scores else None,
                                          _stream(stream)))
        return (disp, best, second) if scores else disp

    def coarse_match_sgm(self, pairs, P1: float, P2: float, npaths: int = 4, costs: bool = False, stream=None):
        """sv_coarse_match_sgm: int16 coarse maps (and the aggregated FP32 cost volumes
        [h, w, D] when `costs`)."""
        import torch
        dev = pairs[0].left.device if pairs else "cuda"
        disp = [torch.empty(p.coarse_hw, dtype=torch.int16, device=dev) for p in pairs]
        vols = [torch.empty((*p.coarse_hw, p.max_disp), dtype=torch.float32, device=dev) for p in pairs] if costs else None
        self._check(lib().sv_coarse_match_sgm(self._h, _pairs_array(pairs), len(pairs), float(P1), float(P2), int(npaths),
                                              _ptrs(disp), _ptrs(vols) if costs else None, _stream(stream)))
        return (disp, vols) if costs else disp

    def coarse_match_ex(self, pairs, opts: SvCoarseOpts, costs: bool = False, stream=None):
        """sv_coarse_match_ex: int16 coarse maps (and the aggregated FP32 volumes [h, w, D]
        when `costs`)."""
        import torch
        dev = pairs[0].left.device if pairs else "cuda"
        disp = [torch.empty(p.coarse_hw, dtype=torch.int16, device=dev) for p in pairs]
        vols = [torch.empty((*p.coarse_hw, p.max_disp), dtype=torch.float32, device=dev) for p in pairs] if costs else None
        self._check(lib().sv_coarse_match_ex(self._h, _pairs_array(pairs), len(pairs), ctypes.byref(opts), _ptrs(disp),
                                             _ptrs(vols) if costs else None, _stream(stream)))
        return (disp, vols) if costs else disp

    def postprocess(self, pairs, maps, smp: bool = True, median: bool = True, stream=None):
        """sv_postprocess: occlusion check and / or median filter of given int16 coarse maps."""
        import torch
        outs = [torch.empty_like(m) for m in maps]
        post = (SV_POST_SMP if smp else 0) | (SV_POST_MEDIAN if median else 0)
        self._check(lib().sv_postprocess(self._h, _pairs_array(pairs), len(pairs), _ptrs(maps), post, _ptrs(outs),
                                         _stream(stream)))
        return outs

    def pipeline_ex(self, pairs, opts: SvCoarseOpts, stream=None, out=None):
        import torch
        outs = out if out is not None else [
            torch.empty((p.height, p.width), dtype=torch.float32, device=p.left.device) for p in pairs]
        self._check(lib().sv_pipeline_ex(self._h, _pairs_array(pairs), len(pairs), ctypes.byref(opts), _ptrs(outs),
                                         _stream(stream)))
        return outs

    def refine(self, pairs, coarse, stream=None, out=None):
        import torch
        outs = out if out is not None else [
            torch.empty((p.height, p.width), dtype=torch.float32, device=p.left.device) for p in pairs]
        self._check(lib().sv_refine(self._h, _pairs_array(pairs), _ptrs(coarse), len(pairs), _ptrs(outs),
                                    _stream(stream)))
        return outs

    def pipeline(self, pairs, stream=None, out=None):
        import torch
        outs = out if out is not None else [
            torch.empty((p.height, p.width), dtype=torch.float32, device=p.left.device) for p in pairs]
        self._check(lib().sv_pipeline(self._h, _pairs_array(pairs), len(pairs), _ptrs(outs), _stream(stream)))
        return outs

    def pipeline_host(self, lefts, rights, widths, heights, pitches, Ds, outs, stream=None):
        """sv_pipeline_host: host images (numpy / pinned torch tensors) in, host results out."""
        arr = (SvPair * max(1, len(lefts)))()
        for i in range(len(lefts)):
            arr[i] = SvPair(_host_ptr(lefts[i]), _host_ptr(rights[i]), widths[i], heights[i], pitches[i], Ds[i])
        optr = (c_void_p * max(1, len(outs)))(*[_host_ptr(o) for o in outs])
        self._check(lib().sv_pipeline_host(self._h, arr, len(lefts), optr, _stream(stream)))
        return outs

    # ---------------------------------------------------------------- profiling
    def profile(self, enable: bool):
        self._check(lib().sv_profile_enable(self._h, int(enable)))

    def profile_read(self, reset: bool = True) -> dict:
        buf = (SvProfileEntry * 64)()
        n = c_int()
        self._check(lib().sv_profile_read(self._h, buf, 64, ctypes.byref(n), int(reset)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, 64))}

    def synchronize(self, stream=None):
        self._check(lib().sv_synchronize(self._h, _stream(stream)))

    def set_option(self, key: str, value: int):
        self._check(lib().sv_set_option(self._h, key.encode(), int(value)))

    def debug_activation(self, which: int, pair: int, shape) -> np.ndarray:
        """Activation of the last tensor-core refinement as float32 [H, W, C]: BF16 values, or
        on an FP8 context the E4M3 codes of e1 .. d1 (which 0 .. 4) decoded."""
        import torch
        n = int(np.prod(shape))
        if self.precision == "fp8" and 0 <= which <= 4:
            buf = torch.empty(n, dtype=torch.uint8)
            self._check(lib().sv_debug_activation(self._h, which, pair, c_void_p(buf.data_ptr()), n))
            return buf.view(torch.float8_e4m3fn).float().numpy().reshape(shape)
        buf = torch.empty(n, dtype=torch.bfloat16)
        self._check(lib().sv_debug_activation(self._h, which, pair, c_void_p(buf.data_ptr()), n * 2))
        return buf.float().numpy().reshape(shape)

    def autotune(self, pairs, cache_path=None, stream=None):
        """Tune the tensor-core layers on this batch (SV_BF16 contexts); returns the choice."""
        p = None if cache_path is None else str(cache_path).encode()
        self._check(lib().sv_autotune(self._h, _pairs_array(pairs), len(pairs), p, _stream(stream)))
        return self.tuning()

    def tuning(self):
        rows = (c_int * 6)()
        nt = (c_int * 6)()
        ctas = (c_int * 6)()
        us = (c_double * 6)()
        self._check(lib().sv_tuning(self._h, rows, nt, ctas, us))
        return {"rows": list(rows), "nt": list(nt), "ctas": list(ctas), "us": list(us)}

    def launch_count(self) -> int:
        return int(lib().sv_launch_count(self._h))

    # ---------------------------------------------------------------- training
    def refine_train(self, pairs, coarse, eps, stream=None):
        import torch
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        dev = pairs[0].left.device
        Y = [torch.empty((p.height, p.width), dtype=dt, device=dev) for p in pairs]
        mu, lv = [], []
        for p in pairs:
            H3, W3 = latent_hw(p.height, p.width)
            mu.append(torch.empty((H3, W3, self.latent), dtype=dt, device=dev))
            lv.append(torch.empty((H3, W3, self.latent), dtype=dt, device=dev))
        self._check(lib().sv_refine_train(self._h, _pairs_array(pairs), _ptrs(coarse), _ptrs(eps), len(pairs),
                                          _ptrs(Y), _ptrs(mu), _ptrs(lv), _stream(stream)))
        return Y, mu, lv

    def refine_backward(self, grad_Y, grad_mu, grad_lv, want_coarse: bool, coarse_like, stream=None):
        import torch
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        dev = grad_Y[0].device
        gparams = torch.empty(self.n_params, dtype=dt, device=dev)
        gc = [torch.empty_like(c, dtype=dt) for c in coarse_like] if want_coarse else None
        self._check(lib().sv_refine_backward(self._h, _ptrs(grad_Y), _ptrs(grad_mu), _ptrs(grad_lv),
                                             c_void_p(gparams.data_ptr()), _ptrs(gc) if want_coarse else None,
                                             _stream(stream)))
        return gparams, gc

    def loss(self, pairs, Y, gt, mu, lv, kl_weight=1e-3, want_grads=True, stream=None):
        import torch
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        dev = Y[0].device
        out = torch.empty(3, dtype=dt, device=dev)
        gY = [torch.empty_like(t) for t in Y] if want_grads else None
        gmu = [torch.empty_like(t) for t in mu] if want_grads else None
        glv = [torch.empty_like(t) for t in lv] if want_grads else None
        self._check(lib().sv_loss(self._h, _pairs_array(pairs), len(pairs), _ptrs(Y), _ptrs(gt), _ptrs(mu), _ptrs(lv),
                                  float(kl_weight), c_void_p(out.data_ptr()),
                                  _ptrs(gY) if want_grads else None, _ptrs(gmu) if want_grads else None,
                                  _ptrs(glv) if want_grads else None, _stream(stream)))
        return out, gY, gmu, glv

    def loss_paper(self, pairs, Y, gt, noc, mu, sigma, want_grads=True, stream=None):
        """sv_loss_paper (Eq. 9-11 of the Table I network): (float64 [total, Loss_1, Loss_2],
        grad_Y, grad_mu, grad_sigma)."""
        import torch
        dev = Y[0].device
        out = torch.empty(3, dtype=torch.float64, device=dev)
        gY = [torch.empty_like(t) for t in Y] if want_grads else None
        gmu = [torch.empty_like(t) for t in mu] if want_grads else None
        gsg = [torch.empty_like(t) for t in sigma] if want_grads else None
        self._check(lib().sv_loss_paper(self._h, _pairs_array(pairs), len(pairs), _ptrs(Y), _ptrs(gt), _ptrs(noc),
                                        _ptrs(mu), _ptrs(sigma), c_void_p(out.data_ptr()),
                                        _ptrs(gY) if want_grads else None, _ptrs(gmu) if want_grads else None,
                                        _ptrs(gsg) if want_grads else None, _stream(stream)))
        return out, gY, gmu, gsg

    def adam_step(self, grad, step: int, lr=5e-4, beta1=0.99, beta2=0.999, eps=1e-8, stream=None):
        self._check(lib().sv_adam_step(self._h, c_void_p(grad.data_ptr()), int(step), lr, beta1, beta2, eps,
                                       _stream(stream)))


def _host_ptr(a):
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def latent_hw(H: int, W: int):
    for _ in range(3):
        H, W = (H + 1) // 2, (W + 1) // 2
    return H, W
