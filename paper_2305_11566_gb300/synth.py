"""Seeded synthetic stereo pairs, ground truth, weights and noise.

This module generates inputs only; it holds none of the method's arithmetic
(no ZNCC, no winner-take-all, no upsampling, no convolution).  Both the CUDA
path and the CPU oracle receive exactly the arrays produced here.

KITTI 2015 (the paper's dataset, Sec. IV-A) is not available, so these pairs
stand in for it: grayscale uint8, about 1242x375, disparity up to ~190 px.

Recipe (one pair):
  * left: 4-octave value noise (lattice cells 32, 16, 8, 4 px; amplitudes 1,
    1/2, 1/4, 1/8; uniform lattice values; smoothstep-bilinear interpolation),
    min-max scaled to 0..255 and rounded to uint8;
  * ground-truth disparity on the left grid: 4 random planes
    d = c + a (x - sx) + b (y - sy), region = Voronoi cell of 4 random seed
    points, clamped to [0, d_max];
  * right: forward splat of left pixel (x, y) to column round(x - d) with a
    z-buffer (larger disparity wins); unfilled right pixels take fresh value
    noise; N(0, 2^2) noise added; clamped and rounded to uint8;
  * occlusion mask: left pixels that lose the z-test or land outside.

All random numbers come from a counter-based splitmix64 stream, so results are
identical on every platform and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based splitmix64 stream: value i = mix64(key + (i + 1) * golden)."""

    def __init__(self, seed: int, tag: int = 0):
        with np.errstate(over="ignore"):
            k = _mix64(np.array([(seed * 1000003 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
        self.key = k[0]
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + idx * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller on pairs of uniforms."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
        t = 2.0 * math.pi * u2
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(t)
        out[1::2] = r * np.sin(t)
        return out[:n]


def value_noise(W: int, H: int, st: Stream) -> np.ndarray:
    """4-octave value noise in [0, 1] (before scaling), float64 [H, W]."""
    acc = np.zeros((H, W))
    ys = np.arange(H, dtype=np.float64)
    xs = np.arange(W, dtype=np.float64)
    for cell, amp in ((32, 1.0), (16, 0.5), (8, 0.25), (4, 0.125)):
        gh = H // cell + 2
        gw = W // cell + 2
        lat = st.uniform(gh * gw).reshape(gh, gw)
        fy = ys / cell
        fx = xs / cell
        iy = np.floor(fy).astype(np.int64)
        ix = np.floor(fx).astype(np.int64)
        ty = fy - iy
        tx = fx - ix
        sy = ty * ty * (3.0 - 2.0 * ty)
        sx = tx * tx * (3.0 - 2.0 * tx)
        v00 = lat[iy][:, ix]
        v01 = lat[iy][:, ix + 1]
        v10 = lat[iy + 1][:, ix]
        v11 = lat[iy + 1][:, ix + 1]
        top = v00 + (v01 - v00) * sx[None, :]
        bot = v10 + (v11 - v10) * sx[None, :]
        acc += amp * (top + (bot - top) * sy[:, None])
    return acc


def _to_u8(a: np.ndarray) -> np.ndarray:
    lo, hi = a.min(), a.max()
    s = (a - lo) / (hi - lo if hi > lo else 1.0) * 255.0
    return np.clip(np.rint(s), 0, 255).astype(np.uint8)


@dataclass
class Pair:
    left: np.ndarray       # uint8 [H, W]
    right: np.ndarray      # uint8 [H, W]
    gt: np.ndarray         # float32 [H, W] disparity on the left grid, px
    occ: np.ndarray        # bool [H, W] left pixels occluded in the right view
    seed: int

    @property
    def width(self) -> int:
        return self.left.shape[1]

    @property
    def height(self) -> int:
        return self.left.shape[0]


def make_pair(W: int, H: int, d_max: float, seed: int) -> Pair:
    st = Stream(seed, 1)
    left_f = value_noise(W, H, st)
    left = _to_u8(left_f)
    # piecewise-planar ground truth: Voronoi cells of 4 seeds, one plane each
    px = st.uniform(4) * W
    py = st.uniform(4) * H
    c0 = (0.1 + 0.8 * st.uniform(4)) * d_max
    ga = (st.uniform(4) - 0.5) * 0.6 * d_max / W
    gb = (st.uniform(4) - 0.5) * 0.6 * d_max / H
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    dist = (xx[None] - px[:, None, None]) ** 2 + (yy[None] - py[:, None, None]) ** 2
    cell = np.argmin(dist, axis=0)
    gt = c0[cell] + ga[cell] * (xx - px[cell]) + gb[cell] * (yy - py[cell])
    gt = np.clip(gt, 0.0, d_max)
    # forward splat with z-buffer: larger disparity wins (write in ascending d)
    xr = np.rint(xx - gt).astype(np.int64)
    inside = xr >= 0
    order = np.argsort(gt, axis=None, kind="stable")
    fy = yy.ravel()[order].astype(np.int64)
    fx = xx.ravel()[order].astype(np.int64)
    fxr = xr.ravel()[order]
    keep = inside.ravel()[order]
    fy, fx, fxr = fy[keep], fx[keep], fxr[keep]
    owner = np.full((H, W), -1, dtype=np.int64)
    owner[fy, fxr] = fy * W + fx            # later (larger d) writes win
    right_f = np.zeros((H, W))
    filled = owner >= 0
    lf_flat = left.astype(np.float64).ravel()
    right_f[filled] = lf_flat[owner[filled]]
    fresh = _to_u8(value_noise(W, H, st)).astype(np.float64)
    right_f[~filled] = fresh[~filled]
    right_f += 2.0 * st.normal(H * W).reshape(H, W)
    right = np.clip(np.rint(right_f), 0, 255).astype(np.uint8)
    visible = np.zeros(H * W, dtype=bool)
    visible[owner[filled]] = True
    occ = ~visible.reshape(H, W)
    return Pair(left=left, right=right, gt=gt.astype(np.float32), occ=occ, seed=seed)


# ---------------------------------------------------------------- networks
@dataclass(frozen=True)
class NetShape:
    """Channel widths of the refinement net (encoder, latent, decoder)."""
    enc: tuple = (16, 32, 64)
    latent: int = 64
    dec: tuple = (64, 32, 16)

    def layers(self):
        """(name, cout, cin, k) in the canonical weight order."""
        c1, c2, c3 = self.enc
        d1, d2, d3 = self.dec
        return [
            ("enc1", c1, 2, 3), ("enc2", c2, c1, 3), ("enc3", c3, c2, 3),
            ("mu", self.latent, c3, 1), ("logvar", self.latent, c3, 1),
            ("dec1", d1, self.latent, 3), ("dec2", d2, d1, 3), ("dec3", d3, d2, 3),
            ("final", 1, d3, 3),
        ]

    def n_params(self) -> int:
        return sum(co * k * k * ci + co for _, co, ci, k in self.layers())


NET_SMALL = NetShape((16, 32, 64), 64, (64, 32, 16))
NET_WIDE = NetShape((32, 64, 128), 128, (128, 64, 32))


def he_normal_weights(shape: NetShape, seed: int = 7) -> np.ndarray:
    """Flat float32 parameters: per layer W[cout][kh][kw][cin] then b[cout].

    W ~ N(0, 2 / (cin * kh * kw)) (He-normal), b = 0."""
    st = Stream(seed, 2)
    parts = []
    for _, co, ci, k in shape.layers():
        n = co * k * k * ci
        std = math.sqrt(2.0 / (ci * k * k))
        parts.append((st.normal(n) * std).astype(np.float32))
        parts.append(np.zeros(co, dtype=np.float32))
    return np.concatenate(parts)


# The paper's Table I network (Sec. III-B1): (name, cout, cin, k) in the flat parameter order.
TABLE1_LAYERS = [
    ("FE_1", 32, 1, 5), ("FE_2", 32, 1, 5), ("EN_1", 16, 64, 5), ("EN_1_R", 8, 16, 5), ("EN_2", 32, 24, 5),
    ("EN_2_R", 16, 32, 5), ("heads", 2, 48, 1), ("D_1", 32, 1, 1), ("D_1_R", 16, 80, 5), ("D_2", 16, 96, 5),
    ("D_2_R", 8, 40, 5), ("D", 16, 48, 5), ("Y", 1, 81, 5),
]


def table1_weights(seed: int = 7) -> np.ndarray:
    """Flat float32 parameters of the Table I network: per layer W[cout][k][k][cin] then
    b[cout], W ~ N(0, 2 / (cin k k)) (He-normal), b = 0."""
    st = Stream(seed, 5)
    parts = []
    for _, co, ci, k in TABLE1_LAYERS:
        parts.append((st.normal(co * k * k * ci) * math.sqrt(2.0 / (ci * k * k))).astype(np.float32))
        parts.append(np.zeros(co, dtype=np.float32))
    return np.concatenate(parts)


def reparam_noise(n: int, seed: int) -> np.ndarray:
    """epsilon ~ N(0, 1) for the reparameterisation (float32)."""
    return Stream(seed, 3).normal(n).astype(np.float32)


def pitched(img: np.ndarray, align: int = 16) -> np.ndarray:
    """Copy an [H, W] uint8 image into an [H, pitch] buffer, pitch % align == 0."""
    H, W = img.shape
    pitch = (W + align - 1) // align * align
    out = np.zeros((H, pitch), dtype=np.uint8)
    out[:, :W] = img
    return out


# ------------------------------------------------------------- workloads
def workload_small(seed: int = 1000) -> Pair:
    """One 256x128 pair, disparity 0-60 px (coarse 64x32, D=16, 7x7 window)."""
    return make_pair(256, 128, 60.0, seed)


def workload_kitti(seed: int = 1000) -> Pair:
    """One 1242x375 pair, disparity 0-190 px (coarse 310x93, D=48, 9x9 window)."""
    return make_pair(1242, 375, 190.0, seed)


def batch_uneven(n: int = 64, seed: int = 2000):
    """Pairs of widths drawn uniformly from {320, 640, 960, 1242}, height
    round(0.302 W), disparity range D = ceil(W / 26) coarse px
    (ground truth up to 4 (D - 1) full-res px)."""
    st = Stream(seed, 4)
    widths = np.array([320, 640, 960, 1242])[(st.uniform(n) * 4).astype(np.int64)]
    out = []
    for i, W in enumerate(widths):
        W = int(W)
        H = int(round(0.302 * W))
        D = -(-W // 26)
        out.append((make_pair(W, H, 4.0 * (D - 1), seed + 1 + i), D))
    return out
