"""Pins of the oracle's semi-global matching (Sec. III-A, Eq. 4-6) and post-processing
(Eq. 7 and the text after it), on the CPU.

Each check is independent of the oracle's own recursion: an exhaustive minimum over
every disparity sequence of a path, closed forms of special penalties, invariances of
Eq. 4 and the symmetry of its directions; hand-made collisions and the uniqueness
property for the occlusion check; a library median filter."""
import itertools

import numpy as np
import pytest

import oracle


def brute_force_path(c_line: np.ndarray, P1: float, P2: float) -> np.ndarray:
    """Unnormalised path cost L(s, d): the minimum over every disparity sequence
    d_0 .. d_s = d of sum_j c(j, d_j) plus the penalties of its steps (0 for no change,
    P1 for a change of one, P2 for more), by enumeration."""
    n, D = c_line.shape
    L = np.full((n, D), np.inf)
    for s in range(n):
        for seq in itertools.product(range(D), repeat=s + 1):
            cost = sum(c_line[j, seq[j]] for j in range(s + 1))
            for j in range(1, s + 1):
                step = abs(seq[j] - seq[j - 1])
                cost += 0.0 if step == 0 else P1 if step == 1 else P2
            L[s, seq[-1]] = min(L[s, seq[-1]], cost)
    return L


@pytest.mark.parametrize("direction", [0, 1, 2, 3])
def test_sgm_path_is_the_minimum_over_disparity_sequences(direction):
    # Eq. 4 subtracts the previous pixel's minimum at every step, so C_r(s, d) equals the
    # unnormalised minimum path cost L(s, d) minus min_k L(s - 1, k).
    rng = np.random.default_rng(11 + direction)
    h, w, D = 3, 5, 3
    C = rng.random((h, w, D)) * 2.0
    P1, P2 = 0.3, 0.8
    Cr = oracle.sgm_path(C, P1, P2, direction)
    lines = range(h) if direction < 2 else range(w)
    for line in lines:
        if direction == 0:
            c_line, got = C[line], Cr[line]
        elif direction == 1:
            c_line, got = C[line, ::-1], Cr[line, ::-1]
        elif direction == 2:
            c_line, got = C[:, line], Cr[:, line]
        else:
            c_line, got = C[::-1, line], Cr[::-1, line]
        L = brute_force_path(c_line, P1, P2)
        want = L.copy()
        want[1:] -= L[:-1].min(axis=1, keepdims=True)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_sgm_without_penalties_is_the_cost_times_paths():
    rng = np.random.default_rng(3)
    C = rng.random((6, 9, 5)) * 2.0
    for npaths in (1, 2, 4):
        np.testing.assert_allclose(oracle.sgm(C, 0.0, 0.0, npaths), npaths * C, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(oracle.sgm_wta(oracle.sgm(C, 0.0, 0.0)), C.argmin(axis=2))


def test_sgm_shifts_with_a_constant_cost():
    rng = np.random.default_rng(4)
    C = rng.random((5, 7, 6))
    a = oracle.sgm(C, 0.2, 0.7)
    b = oracle.sgm(C + 0.375, 0.2, 0.7)
    np.testing.assert_allclose(b - a, 4 * 0.375, rtol=0, atol=1e-12)


def test_sgm_directions_are_flips_and_transposes_of_each_other():
    rng = np.random.default_rng(5)
    C = rng.random((6, 8, 5)) * 2.0
    P1, P2 = 0.15, 0.6
    # right-to-left on C = left-to-right on the mirrored volume, mirrored back
    np.testing.assert_allclose(oracle.sgm_path(C, P1, P2, 1),
                               oracle.sgm_path(C[:, ::-1], P1, P2, 0)[:, ::-1], atol=1e-12)
    # top-to-bottom on C = left-to-right on the transposed volume
    Ct = np.ascontiguousarray(C.transpose(1, 0, 2))
    np.testing.assert_allclose(oracle.sgm_path(C, P1, P2, 2),
                               oracle.sgm_path(Ct, P1, P2, 0).transpose(1, 0, 2), atol=1e-12)
    np.testing.assert_allclose(oracle.sgm_path(C, P1, P2, 3),
                               oracle.sgm_path(C[::-1], P1, P2, 2)[::-1], atol=1e-12)


def test_sgm_step_bounds():
    # the bracket of Eq. 4 minus the previous minimum lies in [0, P2]
    rng = np.random.default_rng(6)
    C = rng.random((7, 9, 8)) * 2.0
    P1, P2 = 0.25, 0.9
    for d in range(4):
        diff = oracle.sgm_path(C, P1, P2, d) - C
        assert diff.min() >= -1e-12 and diff.max() <= P2 + 1e-12


def test_sgm_wta_ties_and_smoothing():
    # ties go to the lowest disparity
    C = np.ones((2, 3, 4))
    np.testing.assert_array_equal(oracle.sgm_wta(C), np.zeros((2, 3), dtype=np.int32))
    # a field with its minimum at d = 2 everywhere but one pixel that prefers d = 4 by a
    # small margin: large penalties pull that pixel back, no penalties leave it
    h, w, D = 5, 7, 6
    C = np.full((h, w, D), 1.0)
    C[:, :, 2] = 0.2
    C[2, 3, 2] = 0.35
    C[2, 3, 4] = 0.3
    assert oracle.sgm_wta(oracle.sgm(C, 0.0, 0.0))[2, 3] == 4
    smooth = oracle.sgm_wta(oracle.sgm(C, 0.2, 0.5))
    np.testing.assert_array_equal(smooth, np.full((h, w), 2, dtype=np.int32))


def test_sgm_cost_of_the_zncc_volume():
    # Eq. 1: cost 1 - rho; invalid candidates (x - d < 0) take the largest cost
    rho = np.array([[[1.0, np.nan], [-0.5, 0.25]]])
    np.testing.assert_array_equal(oracle.sgm_cost(rho), [[[0.0, 2.0], [1.5, 0.75]]])


# ------------------------------------------------------------------ post-processing (Eq. 7)
def test_smp_resolves_a_shared_target_column():
    # targets x - d = 0, 1, 2, 2, 2, 3: pixels 3 and 4 match column 2 like pixel 2, which
    # keeps it (leftmost).  Pixel 3 takes its nearest valid neighbour's disparity (pixel 2,
    # left, distance 1); pixel 4 has no valid pixel at distance 1 on the left (pixel 3) but
    # pixel 5 on the right (d = 2)
    row = np.array([[0, 0, 0, 1, 2, 2]], dtype=np.int32)
    np.testing.assert_array_equal(oracle.smp(row, D=8), [[0, 0, 0, 0, 2, 2]])
    # a collision farther apart than the disparity range is no collision
    far = np.array([[0, 0, 0, 3]], dtype=np.int32)  # pixel 3 matches column 0 like pixel 0
    np.testing.assert_array_equal(oracle.smp(far, D=3), far)
    np.testing.assert_array_equal(oracle.smp(far, D=4), [[0, 0, 0, 0]])


def test_smp_leaves_injective_rows_and_leaves_no_collision():
    # a constant disparity maps every pixel to its own column: nothing changes
    const = np.full((3, 12), 4, dtype=np.int32)
    np.testing.assert_array_equal(oracle.smp(const, D=8), const)
    # random maps: after the check, the pixels that were valid keep their value, and no two
    # of them within D share a target
    rng = np.random.default_rng(21)
    D = 6
    disp = rng.integers(0, D, size=(4, 30)).astype(np.int32)
    for x in range(30):
        disp[:, x] = np.minimum(disp[:, x], x)  # a candidate needs x - d >= 0
    out = oracle.smp(disp, D)
    for y in range(4):
        valid = [all(x - disp[y, x] != x - k - disp[y, x - k] for k in range(1, min(D, x + 1))) for x in range(30)]
        for x in range(30):
            if valid[x]:
                assert out[y, x] == disp[y, x]
        tv = [x - disp[y, x] for x in range(30) if valid[x]]
        xs = [x for x in range(30) if valid[x]]
        for i in range(len(xs)):
            for j in range(i + 1, len(xs)):
                if xs[j] - xs[i] < D:
                    assert tv[i] != tv[j]


def test_median3_matches_the_library_filter():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(22)
    d = rng.integers(0, 40, size=(9, 13)).astype(np.int32)
    np.testing.assert_array_equal(oracle.median3(d), ndi.median_filter(d, size=3, mode="nearest"))
    spike = np.full((5, 5), 7, dtype=np.int32)
    spike[2, 2] = 30
    np.testing.assert_array_equal(oracle.median3(spike), np.full((5, 5), 7, dtype=np.int32))


def test_sgm_degenerate_shapes():
    rng = np.random.default_rng(23)
    # one disparity: no neighbour terms and the previous minimum is the previous cost, so
    # every path returns the cost itself
    C = rng.random((4, 6, 1)) * 2.0
    for d in range(4):
        np.testing.assert_allclose(oracle.sgm_path(C, 0.3, 0.9, d), C, atol=1e-12)
    np.testing.assert_array_equal(oracle.sgm_wta(oracle.sgm(C, 0.3, 0.9)), np.zeros((4, 6), dtype=np.int32))
    # one column / one row: the paths across it have a single pixel and keep the cost
    col = rng.random((5, 1, 4)) * 2.0
    np.testing.assert_allclose(oracle.sgm_path(col, 0.3, 0.9, 0), col, atol=1e-12)
    np.testing.assert_allclose(oracle.sgm_path(col, 0.3, 0.9, 1), col, atol=1e-12)
    row = rng.random((1, 5, 4)) * 2.0
    np.testing.assert_allclose(oracle.sgm_path(row, 0.3, 0.9, 2), row, atol=1e-12)
    np.testing.assert_allclose(oracle.sgm_path(row, 0.3, 0.9, 3), row, atol=1e-12)
