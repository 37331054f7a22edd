"""FP64 CPU oracle of the StereoVAE hot path (arXiv 2305.11566).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

This module is argument marshalling around ``sv_oracle.c`` (plain C, FP64,
direct loops; see the header of that file for the passage each function
follows).  It shares no code with the CUDA library.

Parity status per function (what pins each one, in tests/test_oracle_*.py):
  downsample4      brute force on tiny images, exact integers
  zncc_volume      brute-force numpy restatement of Eq. 1-3 on tiny pairs; rho in
                   [-1, 1]; gain/offset invariance; rho(I, I) = 1; shift recovery
  zncc_wta         exact integer argmax agrees with FP64 argmax where it is
                   unambiguous; exact recovery of a constant integer shift
  upsample4        affine ramps reproduced exactly; torch interpolate at W = 4w
  conv2d           torch.nn.functional.conv2d in FP64 (library routine),
                   nearest-x2 via torch interpolate
  refine_forward   composed of the pinned pieces; layer-by-layer against torch FP64
  refine_backward  central finite differences in FP64 and torch FP64 autograd
  sgm_path / sgm   brute-force minimum over every disparity sequence of a path (tiny D, w);
                   P1 = P2 = 0 reduces to the cost itself; constant-shift invariance;
                   direction symmetry under flips / transposes; 0 <= C_r - C <= P2
  sgm_wta          ties to the lowest d; equals the plain argmin of C when P1 = P2 = 0
  smp              hand-made collisions; injective rows unchanged; no two valid pixels share a
                   target afterwards
  census_volume    hand-made 3 x 3 codes; invariance under increasing intensity maps; zero
                   cost of an image against itself and of a constant shift at its disparity;
                   the mirror identity (both images flipped, roles swapped)
  e4m3             torch's float8_e4m3fn conversion (round to nearest even) over the whole
                   finite range, saturation above 448
  refine_forward_q with its roundings off: refine_forward (the folded decoder interior and
                   the unfolded border recompute together equal the plain nearest-x2 conv);
                   activations on the E4M3 grid (d2, d3 on the BF16 grid); the BF16 form's bar
                   against refine_forward
  qconv_layer      the layer refine_forward_q applies: chaining it layer by layer gives that
                   forward's activations exactly; stride-2 and pointwise layers whose weights
                   are E4M3 values times 2^-8 (each channel reaching 448 x 2^-8, so its scale
                   is 2^-8 and every code exact) equal torch's FP64 conv2d
  t1_layer         torch.nn.functional conv2d / conv_transpose2d / leaky_relu in FP64
  t1_inputs        torch avg_pool2d and interpolate (bilinear, half-pixel centres) where the
                   sizes are exact multiples
  t1_forward       the same network composed from torch FP64 library routines (torch.cat,
                   conv2d, conv_transpose2d, leaky_relu), with and without eps
  t1_loss          closed forms of the weighted L1 term; torch.distributions.kl_divergence
                   of Normal(mu - 1, exp(sigma - 1)) from Normal(0, 1)
  dt_aggregate     uniform guide: scipy.signal.lfilter (first-order recursive filter) along
                   each axis; constant slices unchanged; a hard edge (sigma_r -> 0) separates
                   the two sides exactly; linearity in the cost; bounds min C <= out <= max C
  median3          scipy.ndimage.median_filter (3 x 3, nearest) as an independent routine
  end-to-end disparity error vs synthetic ground truth: parity unpinned
  (random weights; the paper's trained weights and KITTI are absent).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_size_t, c_uint8, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sv_oracle.c into liboracle.so with gcc (-O2, OpenMP, IEEE math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = c_void_p
        L.orc_downsample4.argtypes = [P, c_int, c_int, c_int, P]
        L.orc_zncc_at.argtypes = [P, P, c_int, c_int, c_int, c_int, c_int, c_int]
        L.orc_zncc_at.restype = c_double
        L.orc_zncc_volume.argtypes = [P, P, c_int, c_int, c_int, c_int, P]
        L.orc_zncc_wta.argtypes = [P, P, c_int, c_int, c_int, c_int, P, P, P]
        L.orc_upsample4.argtypes = [P, c_int, c_int, c_int, c_int, P]
        L.orc_sgm_path.argtypes = [P, c_int, c_int, c_int, c_double, c_double, c_int, P]
        L.orc_sgm.argtypes = [P, c_int, c_int, c_int, c_double, c_double, c_int, P]
        L.orc_sgm_wta.argtypes = [P, c_int, c_int, c_int, P]
        L.orc_smp.argtypes = [P, c_int, c_int, c_int, P]
        L.orc_median3.argtypes = [P, c_int, c_int, P]
        L.orc_census_volume.argtypes = [P, P, c_int, c_int, c_int, c_int, P]
        L.orc_e4m3.argtypes = [c_double]
        L.orc_e4m3.restype = c_double
        L.orc_refine_forward_q.argtypes = [P, P, P, c_int, c_int, c_int, P, c_int, c_int, c_int, P, c_int, P]
        L.orc_qconv_layer.argtypes = [P, c_int, c_int, c_int, P, P, c_int, c_int, c_int, c_int, c_int, c_int, c_int, P]
        L.orc_t1_param_offset.argtypes = [c_int, c_int]
        L.orc_t1_param_offset.restype = c_size_t
        L.orc_t1_param_count.restype = c_size_t
        L.orc_t1_layer.argtypes = [P, c_int, c_int, c_int, P, P, c_int, c_int, c_int, c_int, c_int, c_int, P]
        L.orc_t1_inputs.argtypes = [P, c_int, c_int, c_int, P, c_int, c_int, P, P]
        L.orc_t1_forward.argtypes = [P, P, c_int, c_int, c_int, P, c_int, c_int, P, P, P, P, c_int, P]
        L.orc_t1_loss.argtypes = [P, P, P, c_size_t, P, P, c_size_t, P]
        L.orc_t1_loss.restype = c_double
        L.orc_dt_aggregate.argtypes = [P, c_int, c_int, c_int, P, c_double, c_double, c_int, P]
        L.orc_upsample4_backward.argtypes = [P, c_int, c_int, c_int, c_int, P]
        L.orc_conv2d.argtypes = [P, c_int, c_int, c_int, P, P, c_int, c_int, c_int, c_int, c_int, c_int, c_int,
                                 c_int, P]
        L.orc_conv2d_backward.argtypes = [P, c_int, c_int, c_int, P, c_int, c_int, c_int, c_int, c_int, c_int,
                                          c_int, P, P, P, P]
        L.orc_param_offset.argtypes = [P, c_int, c_int]
        L.orc_param_offset.restype = c_size_t
        L.orc_refine_forward.argtypes = [P, P, P, c_int, c_int, c_int, P, c_int, c_int, P, P, P, P, P]
        L.orc_refine_activation.argtypes = [P, P, P, c_int, c_int, c_int, P, c_int, c_int, P, c_int, P]
        L.orc_refine_loss.argtypes = [P, P, P, c_int, c_int, c_int, P, c_int, c_int, P, P, c_double, c_double,
                                      c_double]
        L.orc_refine_loss.restype = c_double
        L.orc_refine_backward.argtypes = [P, P, P, c_int, c_int, c_int, P, c_int, c_int, P, P, c_double,
                                          c_double, c_double, P, P]
        L.orc_refine_backward.restype = c_double
        L.orc_adam.argtypes = [P, P, P, P, c_size_t, c_int, c_double, c_double, c_double, c_double]
        L.orc_num_threads.restype = c_int
        L.orc_set_threads.argtypes = [c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(c_void_p)


def _opt(a):
    return None if a is None else _p(a)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(n)


# ---------------------------------------------------------------- coarse stage
def downsample4(img: np.ndarray) -> np.ndarray:
    """4x4 box sums (int32 [H//4, W//4]) of a uint8 [H, W] image."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    S = np.zeros((H // 4, W // 4), dtype=np.int32)
    lib().orc_downsample4(_p(img), W, H, W, _p(S))
    return S


def zncc_at(SL, SR, k, x, y, d) -> float:
    SL = np.ascontiguousarray(SL, dtype=np.int32)
    SR = np.ascontiguousarray(SR, dtype=np.int32)
    h, w = SL.shape
    return lib().orc_zncc_at(_p(SL), _p(SR), w, h, k, x, y, d)


def zncc_volume(SL, SR, k: int, D: int) -> np.ndarray:
    """rho [h, w, D] by Eq. 1-3 in FP64; NaN where x - d < 0."""
    SL = np.ascontiguousarray(SL, dtype=np.int32)
    SR = np.ascontiguousarray(SR, dtype=np.int32)
    h, w = SL.shape
    rho = np.zeros((h, w, D))
    lib().orc_zncc_volume(_p(SL), _p(SR), w, h, k, D, _p(rho))
    return rho


def zncc_wta(SL, SR, k: int, D: int):
    """(disp int32 [h, w], best rho, second-best rho) by Eq. 6, exact integer decisions."""
    SL = np.ascontiguousarray(SL, dtype=np.int32)
    SR = np.ascontiguousarray(SR, dtype=np.int32)
    h, w = SL.shape
    disp = np.zeros((h, w), dtype=np.int32)
    best = np.zeros((h, w))
    second = np.zeros((h, w))
    lib().orc_zncc_wta(_p(SL), _p(SR), w, h, k, D, _p(disp), _p(best), _p(second))
    return disp, best, second


def coarse_match(left: np.ndarray, right: np.ndarray, k: int, D: int):
    """Downsample both images and run ZNCC + WTA: (disp, best, second)."""
    return zncc_wta(downsample4(left), downsample4(right), k, D)


# ---------------------------------------------------------------- semi-global matching
def sgm_cost(rho: np.ndarray) -> np.ndarray:
    """Cost volume of Eq. 1, C = 1 - rho, with the largest cost (2) where x - d < 0."""
    return np.where(np.isnan(rho), 2.0, 1.0 - rho)


def sgm_path(C: np.ndarray, P1: float, P2: float, direction: int) -> np.ndarray:
    """C_r of Eq. 4 along one direction (0: left to right, 1: right to left, 2: top to
    bottom, 3: bottom to top), FP64 [h, w, D]."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    h, w, D = C.shape
    out = np.zeros_like(C)
    lib().orc_sgm_path(_p(C), w, h, D, float(P1), float(P2), int(direction), _p(out))
    return out


def sgm(C: np.ndarray, P1: float, P2: float, npaths: int = 4) -> np.ndarray:
    """C_SGM of Eq. 5: the sum of sgm_path over the first `npaths` directions."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    h, w, D = C.shape
    out = np.zeros_like(C)
    lib().orc_sgm(_p(C), w, h, D, float(P1), float(P2), int(npaths), _p(out))
    return out


def sgm_wta(Csgm: np.ndarray) -> np.ndarray:
    """Eq. 6 on an aggregated volume: argmin over d, lowest d on ties (int32 [h, w])."""
    Csgm = np.ascontiguousarray(Csgm, dtype=np.float64)
    h, w, D = Csgm.shape
    disp = np.zeros((h, w), dtype=np.int32)
    lib().orc_sgm_wta(_p(Csgm), w, h, D, _p(disp))
    return disp


def smp(disp: np.ndarray, D: int) -> np.ndarray:
    """Single-matching-phase check (Eq. 7 read as uniqueness of the target column): invalid
    pixels take the nearest valid disparity of their row (int32 [h, w])."""
    d = np.ascontiguousarray(disp, dtype=np.int32)
    h, w = d.shape
    out = np.zeros_like(d)
    lib().orc_smp(_p(d), w, h, int(D), _p(out))
    return out


def median3(disp: np.ndarray) -> np.ndarray:
    """3 x 3 median filter with edge clamping (int32 [h, w])."""
    d = np.ascontiguousarray(disp, dtype=np.int32)
    h, w = d.shape
    out = np.zeros_like(d)
    lib().orc_median3(_p(d), w, h, _p(out))
    return out


# ---------------------------------------------------------------- census cost, DT aggregation
def census_volume(SL, SR, kc: int, D: int) -> np.ndarray:
    """Census cost [h, w, D] (FP64, integer valued) of the quarter-size box sums: Hamming
    distance of the kc x kc census codes of (x, y) and (x - d, y); kc^2 - 1 where x - d < 0."""
    SL = np.ascontiguousarray(SL, dtype=np.int32)
    SR = np.ascontiguousarray(SR, dtype=np.int32)
    h, w = SL.shape
    out = np.zeros((h, w, D), dtype=np.float64)
    lib().orc_census_volume(_p(SL), _p(SR), w, h, int(kc), int(D), _p(out))
    return out


def dt_aggregate(C: np.ndarray, guide: np.ndarray, sigma_s: float, sigma_r: float, iters: int) -> np.ndarray:
    """Domain-transform aggregation of a cost volume [h, w, D] guided by the left box sums
    [h, w] (intensity = sum / 16): recursive edge-aware filter along rows then columns,
    both ways, `iters` times."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    g = np.ascontiguousarray(guide, dtype=np.int32)
    h, w, D = C.shape
    out = np.zeros_like(C)
    lib().orc_dt_aggregate(_p(C), w, h, D, _p(g), float(sigma_s), float(sigma_r), int(iters), _p(out))
    return out


def coarse_cost(left, right, cost: str, k: int, D: int, census_window: int = 5):
    """The cost volume of the chosen matcher on the quarter-size pair: "zncc" (1 - rho of
    Eq. 1, 2 where x - d < 0) or "census"."""
    SL, SR = downsample4(left), downsample4(right)
    if cost == "zncc":
        return sgm_cost(zncc_volume(SL, SR, k, D))
    return census_volume(SL, SR, census_window, D)


# ---------------------------------------------------------------- the paper's Table I network
T1_LAYERS = ["FE_1", "FE_2", "EN_1", "EN_1_R", "EN_2", "EN_2_R", "heads", "D_1", "D_1_R", "D_2", "D_2_R", "D", "Y"]
T1_ACTS = ["FE_1", "FE_2", "EN_1", "EN_1_R", "EN_2", "EN_2_R", "heads", "D_1", "D_1_R", "D_2", "D_2_R", "D", "X_0",
           "X_1"]


def t1_levels(H: int, W: int):
    """(H, W), half, quarter and eighth resolution sizes (ceil at every halving)."""
    out = [(H, W)]
    for _ in range(3):
        H, W = (H + 1) // 2, (W + 1) // 2
        out.append((H, W))
    return out


def t1_param_count() -> int:
    return int(lib().orc_t1_param_count())


def t1_param_slices():
    """{layer name: (W slice, b slice)} into the flat Table I parameter vector."""
    out = {}
    for i, n in enumerate(T1_LAYERS):
        a = lib().orc_t1_param_offset(i, 0)
        b = lib().orc_t1_param_offset(i, 1)
        c = lib().orc_t1_param_offset(i + 1, 0)
        out[n] = (slice(a, b), slice(b, c))
    return out


def t1_layer(x: np.ndarray, wt: np.ndarray, b: np.ndarray, mode: int, out_hw, act: bool) -> np.ndarray:
    """One Table I layer: mode 0 conv s1, 1 conv s2, 2 deconv s2 (cropped to out_hw); x
    [Hi, Wi, Ci], wt [Co, k, k, Ci] float32, b [Co]; leaky ReLU 0.1 when act."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    Hi, Wi, Ci = x.shape
    Co, k = wt.shape[0], wt.shape[1]
    Ho, Wo = out_hw
    out = np.zeros((Ho, Wo, Co), dtype=np.float64)
    lib().orc_t1_layer(_p(x), Hi, Wi, Ci, _p(wt), _p(b), Co, k, int(mode), Ho, Wo, int(act), _p(out))
    return out


def t1_inputs(left: np.ndarray, coarse: np.ndarray):
    """(X_0, X_1) at half resolution from the left image and the coarse map (coarse pixels)."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    H, W = left.shape
    c = np.ascontiguousarray(coarse, dtype=np.float64)
    h, w = c.shape
    Hh, Wh = (H + 1) // 2, (W + 1) // 2
    X0 = np.zeros((Hh, Wh), dtype=np.float64)
    X1 = np.zeros((Hh, Wh), dtype=np.float64)
    lib().orc_t1_inputs(_p(left), W, H, W, _p(c), w, h, _p(X0), _p(X1))
    return X0, X1


def t1_forward(params: np.ndarray, left: np.ndarray, coarse: np.ndarray, eps=None, act: str | None = None):
    """Forward pass of the Table I network: {"Y": [H, W] normalised disparity (256 Y in pixels),
    "mu", "sigma": [H8, W8]} and, with `act`, that activation."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    H, W = left.shape
    c = np.ascontiguousarray(coarse, dtype=np.float64)
    h, w = c.shape
    (_, _), (H2, W2), (H4, W4), (H8, W8) = t1_levels(H, W)
    Y = np.zeros((H, W), dtype=np.float64)
    mu = np.zeros((H8, W8), dtype=np.float64)
    sg = np.zeros((H8, W8), dtype=np.float64)
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64).reshape(H8, W8)
    which, buf = -1, None
    if act is not None:
        which = T1_ACTS.index(act)
        lv = {"FE_1": (H2, W2, 32), "FE_2": (H2, W2, 32), "EN_1": (H4, W4, 16), "EN_1_R": (H4, W4, 8),
              "EN_2": (H8, W8, 32), "EN_2_R": (H8, W8, 16), "heads": (H8, W8, 2), "D_1": (H8, W8, 32),
              "D_1_R": (H8, W8, 16), "D_2": (H4, W4, 16), "D_2_R": (H4, W4, 8), "D": (H2, W2, 16),
              "X_0": (H2, W2, 1), "X_1": (H2, W2, 1)}[act]
        buf = np.zeros(lv, dtype=np.float64)
    lib().orc_t1_forward(_p(params), _p(left), W, H, W, _p(c), w, h, _opt(e), _p(Y), _p(mu), _p(sg), which,
                         _opt(buf))
    out = {"Y": Y, "mu": mu, "sigma": sg}
    if act is not None:
        out[act] = buf
    return out


def t1_loss(Y, gt, noc, mu, sigma):
    """Loss of Eq. 9-11 for the Table I network: (total, Loss_1, Loss_2)."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    gt = np.ascontiguousarray(gt, dtype=np.float32)
    noc = np.ascontiguousarray(noc, dtype=np.uint8)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    parts = np.zeros(2, dtype=np.float64)
    tot = lib().orc_t1_loss(_p(Y), _p(gt), _p(noc), Y.size, _p(mu), _p(sigma), mu.size, _p(parts))
    return float(tot), float(parts[0]), float(parts[1])


def upsample4(disp: np.ndarray, W: int, H: int) -> np.ndarray:
    d = np.ascontiguousarray(disp, dtype=np.float64)
    h, w = d.shape
    U = np.zeros((H, W))
    lib().orc_upsample4(_p(d), w, h, W, H, _p(U))
    return U


def upsample4_backward(gU: np.ndarray, w: int, h: int) -> np.ndarray:
    gU = np.ascontiguousarray(gU, dtype=np.float64)
    H, W = gU.shape
    g = np.zeros((h, w))
    lib().orc_upsample4_backward(_p(gU), w, h, W, H, _p(g))
    return g


# ---------------------------------------------------------------- convolution
def conv2d(x: np.ndarray, wt: np.ndarray, b, stride: int, pad: int, relu: bool = False,
           up2: bool = False, out_hw=None) -> np.ndarray:
    """x: [Hi, Wi, Ci] float64; wt: [Co, k, k, Ci] float32; b: [Co] float32 or None."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float32)
    Hi, Wi, Ci = x.shape
    Co, ks = wt.shape[0], wt.shape[1]
    if up2:
        Ho, Wo = out_hw
    else:
        Ho = (Hi + 2 * pad - ks) // stride + 1
        Wo = (Wi + 2 * pad - ks) // stride + 1
    out = np.zeros((Ho, Wo, Co))
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float32)
    lib().orc_conv2d(_p(x), Hi, Wi, Ci, _p(wt), _opt(bb), Co, ks, stride, pad, int(up2), Ho, Wo, int(relu), _p(out))
    return out


def conv2d_backward(x, wt, stride, pad, gout, up2=False):
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float32)
    gout = np.ascontiguousarray(gout, dtype=np.float64)
    Hi, Wi, Ci = x.shape
    Co, ks = wt.shape[0], wt.shape[1]
    Ho, Wo = gout.shape[:2]
    gin = np.zeros_like(x)
    gw = np.zeros(wt.shape)
    gb = np.zeros(Co)
    lib().orc_conv2d_backward(_p(x), Hi, Wi, Ci, _p(wt), Co, ks, stride, pad, int(up2), Ho, Wo, _p(gout), _p(gin),
                              _p(gw), _p(gb))
    return gin, gw, gb


# ---------------------------------------------------------------- the net
def widths7(shape) -> np.ndarray:
    return np.array([*shape.enc, shape.latent, *shape.dec], dtype=np.int32)


def level_sizes(H: int, W: int):
    H1, W1 = (H + 1) // 2, (W + 1) // 2
    H2, W2 = (H1 + 1) // 2, (W1 + 1) // 2
    H3, W3 = (H2 + 1) // 2, (W2 + 1) // 2
    return (H, W), (H1, W1), (H2, W2), (H3, W3)


def param_slices(shape):
    """{layer: (w_offset, w_shape, b_offset, cout)} of the flat parameter vector."""
    w7 = widths7(shape)
    out = {}
    for i, (name, co, ci, k) in enumerate(shape.layers()):
        ow = lib().orc_param_offset(_p(w7), i, 0)
        ob = lib().orc_param_offset(_p(w7), i, 1)
        out[name] = (ow, (co, k, k, ci), ob, co)
    return out


def refine_forward(shape, params: np.ndarray, left: np.ndarray, coarse: np.ndarray, eps=None):
    """Returns dict with Y, U (float64 [H, W]) and mu, logvar ([H3, W3, lat])."""
    w7 = widths7(shape)
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    H, W = left.shape
    h, w = coarse.shape
    _, _, _, (H3, W3) = level_sizes(H, W)
    Y = np.zeros((H, W))
    U = np.zeros((H, W))
    mu = np.zeros((H3, W3, shape.latent))
    lv = np.zeros((H3, W3, shape.latent))
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float32)
    lib().orc_refine_forward(_p(w7), _p(params), _p(left), W, H, W, _p(coarse), w, h, _opt(e), _p(Y), _p(U), _p(mu),
                             _p(lv))
    return {"Y": Y, "U": U, "mu": mu, "logvar": lv}


ACTIVATIONS = ["U", "e1", "e2", "e3", "mu", "logvar", "z", "d1", "d2", "d3", "Y"]


def e4m3(x: float) -> float:
    """E4M3 (FP8) rounding of the quantised form: nearest, ties to even, saturating at 448."""
    return float(lib().orc_e4m3(float(x)))


def refine_forward_q(shape, params: np.ndarray, left: np.ndarray, coarse: np.ndarray, quant: bool = True,
                     act: str | None = None):
    """The FP8 form's refinement (inference): {"Y": [H, W]} and, with `act`, that activation
    ("e1" .. "d3") as the layer passes it on.  quant=False skips every rounding."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    H, W = left.shape
    c = np.ascontiguousarray(coarse, dtype=np.float64)
    h, w = c.shape
    w7 = widths7(shape)
    Y = np.zeros((H, W), dtype=np.float64)
    names = ["e1", "e2", "e3", "z", "d1", "d2", "d3"]
    which, buf = -1, None
    if act is not None:
        which = names.index(act)
        L0, L1, L2, L3 = level_sizes(H, W)
        c1, c2, c3 = shape.enc
        d1, d2, d3 = shape.dec
        shp = {"e1": (*L1, c1), "e2": (*L2, c2), "e3": (*L3, c3), "z": (*L3, shape.latent), "d1": (*L2, d1),
               "d2": (*L1, d2), "d3": (*L0, d3)}[act]
        buf = np.zeros(shp, dtype=np.float64)
    lib().orc_refine_forward_q(_p(w7), _p(params), _p(left), W, H, W, _p(c), w, h, int(quant), _p(Y), which, _opt(buf))
    out = {"Y": Y}
    if act is not None:
        out[act] = buf
    return out


def qconv_layer(x: np.ndarray, wt: np.ndarray, b: np.ndarray, mode: int, out_hw, relu: bool = True,
                out_round: str = "e4m3", quant_weights: bool = True) -> np.ndarray:
    """One FP8-form layer from the given input values x [Hi, Wi, Ci]: wt [Co, k, k, Ci] FP32
    weights (k = 3, or 1 for mode 1), mode 0 stride-2 3 x 3, 1 pointwise, 2 nearest x2 + crop +
    3 x 3; weights quantised per output channel (quant_weights, the form's quantised layers)
    or used as they are (its last decoder layer); out_round "none", "e4m3" or "bf16".
    Returns [Ho, Wo, Co]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    Hi, Wi, Ci = x.shape
    Co = wt.shape[0]
    Ho, Wo = out_hw
    out = np.zeros((Ho, Wo, Co), dtype=np.float64)
    r = {"none": 0, "e4m3": 1, "bf16": 2}[out_round]
    lib().orc_qconv_layer(_p(x), Hi, Wi, Ci, _p(wt), _p(b), Co, mode, Ho, Wo, int(relu), int(quant_weights), r,
                          _p(out))
    return out


def refine_activation(shape, params, left, coarse, which: str, eps=None) -> np.ndarray:
    w7 = widths7(shape)
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    H, W = left.shape
    h, w = coarse.shape
    L0, L1, L2, L3 = level_sizes(H, W)
    c1, c2, c3 = shape.enc
    d1, d2, d3 = shape.dec
    dims = {"U": (*L0, 1), "e1": (*L1, c1), "e2": (*L2, c2), "e3": (*L3, c3), "mu": (*L3, shape.latent),
            "logvar": (*L3, shape.latent), "z": (*L3, shape.latent), "d1": (*L2, d1), "d2": (*L1, d2),
            "d3": (*L0, d3), "Y": (*L0, 1)}[which]
    out = np.zeros(dims)
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float32)
    lib().orc_refine_activation(_p(w7), _p(params), _p(left), W, H, W, _p(coarse), w, h, _opt(e),
                                ACTIVATIONS.index(which), _p(out))
    return out


def refine_loss(shape, params, left, coarse, eps, gt, n_pix, n_lat, kl_w=1e-3) -> float:
    w7 = widths7(shape)
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    gt = np.ascontiguousarray(gt, dtype=np.float32)
    H, W = left.shape
    h, w = coarse.shape
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float32)
    return lib().orc_refine_loss(_p(w7), _p(params), _p(left), W, H, W, _p(coarse), w, h, _opt(e), _p(gt),
                                 float(n_pix), float(n_lat), float(kl_w))


def refine_backward(shape, params, left, coarse, eps, gt, n_pix, n_lat, kl_w=1e-3, want_coarse=False):
    """(loss, grad params float64 flat, grad coarse [h, w] or None)."""
    w7 = widths7(shape)
    params = np.ascontiguousarray(params, dtype=np.float32)
    left = np.ascontiguousarray(left, dtype=np.uint8)
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    gt = np.ascontiguousarray(gt, dtype=np.float32)
    H, W = left.shape
    h, w = coarse.shape
    g = np.zeros(params.size)
    gc = np.zeros((h, w)) if want_coarse else None
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float32)
    L = lib().orc_refine_backward(_p(w7), _p(params), _p(left), W, H, W, _p(coarse), w, h, _opt(e), _p(gt),
                                  float(n_pix), float(n_lat), float(kl_w), _p(g), _opt(gc))
    return L, g, gc


def adam(p, m, v, g, t, lr=5e-4, b1=0.99, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    for a in (p, m, v, g):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().orc_adam(_p(p), _p(m), _p(v), _p(g), p.size, int(t), lr, b1, b2, eps)


def pipeline(shape, params, left, right, k, D):
    """Coarse match + refinement of one pair (inference): returns (Y, disp, best, second)."""
    disp, best, second = coarse_match(left, right, k, D)
    out = refine_forward(shape, params, left, disp.astype(np.float64))
    return out["Y"], disp, best, second
