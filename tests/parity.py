"""Shared parity rules of the end-to-end GPU tests.

A refined disparity depends on the coarse WTA map through the network's receptive
field.  Where the oracle's best and second-best ZNCC scores are closer than the FP32
rounding of the GPU's scores, the two sides may pick different (equally correct)
disparities (Eq. 6 on a near tie), and every refined pixel that sees such a coarse
pixel may differ by up to a few pixels.  The end-to-end comparisons therefore:

  1. require every WTA difference to sit on a near tie of the oracle (margin <= 1e-4),
  2. mask the receptive field of each difference (a square of `radius` coarse pixels,
     i.e. 4 * radius full-resolution pixels, around it),
  3. require the kept part to cover more than 90 % of the image, and
  4. apply the form's bar to every kept pixel.

Nothing is conditional: a pair with a WTA difference is still compared everywhere
else, and a pair without one is compared everywhere.
"""
import numpy as np

WTA_MARGIN = 1e-4
RF_RADIUS = 16  # coarse pixels; the refined output sees about 9 coarse pixels each way


def wta_differences(d_gpu, d_oracle, best_o, second_o):
    """Coarse pixels where the two WTA maps differ; asserts each is a near tie."""
    diff = np.asarray(d_gpu) != np.asarray(d_oracle)
    clear = (best_o - second_o) > WTA_MARGIN
    bad = diff & clear
    assert not bad.any(), f"{int(bad.sum())} WTA differences where the oracle's margin exceeds {WTA_MARGIN}"
    return diff


def keep_mask(diff, H, W, radius=RF_RADIUS):
    """Full-resolution pixels outside the receptive field of every coarse difference."""
    near = np.zeros_like(diff)
    for y, x in zip(*np.nonzero(diff)):
        near[max(0, y - radius):y + radius + 1, max(0, x - radius):x + radius + 1] = True
    keep = ~np.repeat(np.repeat(near, 4, 0), 4, 1)
    keep = np.pad(keep, ((0, H - keep.shape[0]), (0, W - keep.shape[1])), mode="edge")
    assert keep.mean() > 0.9, f"only {keep.mean():.3f} of the pixels are outside the WTA differences' reach"
    return keep


def compare_refined(Y_gpu, Y_oracle, keep, max_px, mean_px=None, gt=None, epe_px=None, label=""):
    """The form's bar on the kept pixels: max |dY|, optionally mean |dY| and the EPE change
    against the ground truth."""
    Yg = np.asarray(Y_gpu, dtype=np.float64)
    err = np.abs(Yg - Y_oracle)[keep]
    assert err.max() <= max_px, f"{label}: max |dY| = {err.max():.3g} (bar {max_px})"
    if mean_px is not None:
        assert err.mean() <= mean_px, f"{label}: mean |dY| = {err.mean():.3g} (bar {mean_px})"
    if gt is not None and epe_px is not None:
        epe_g = np.abs(Yg - gt)[keep].mean()
        epe_o = np.abs(Y_oracle - gt)[keep].mean()
        assert abs(epe_g - epe_o) <= epe_px, f"{label}: EPE {epe_g:.4f} vs oracle {epe_o:.4f}"
    return float(err.max())
