"""Pins of the oracle's segmentation (Sec. IV-C: SNIC superpixels in YCbCr, compactness m = 5,
8-connected segments): the sequential SNIC the paper uses, the data-parallel clustering the GPU
computes, and its connectivity step. Expected values are closed forms or worked by hand below; none
comes from the code under test."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

EIGHT = np.ones((3, 3), bool)


def _frame(Y, U=None, V=None, dtype=np.uint8):
    Y = np.atleast_2d(np.asarray(Y, dtype))
    U = np.zeros_like(Y) if U is None else np.atleast_2d(np.asarray(U, dtype))
    V = np.zeros_like(Y) if V is None else np.atleast_2d(np.asarray(V, dtype))
    return synth.View(Y, U, V)


def _grid(W, H, S):
    gw = -(-W // S)
    ys, xs = np.mgrid[0:H, 0:W]
    return (ys // S) * gw + xs // S


def _components_per_label(lab):
    return {int(k): ndimage.label(lab == k, EIGHT)[1] for k in np.unique(lab)}


def boundary_recall(seg, gt, tol=2):
    def edges(l):
        b = np.zeros(l.shape, bool)
        h, v = l[:, :-1] != l[:, 1:], l[:-1] != l[1:]
        b[:, :-1] |= h
        b[:, 1:] |= h
        b[:-1] |= v
        b[1:] |= v
        return b
    g = edges(gt)
    s = ndimage.binary_dilation(edges(seg), np.ones((2 * tol + 1,) * 2, bool))
    return (g & s).sum() / max(1, g.sum())


def undersegmentation_error(seg, gt):
    tot = 0
    for s in np.unique(seg):
        m = seg == s
        _, cnt = np.unique(gt[m], return_counts=True)
        tot += np.minimum(cnt, m.sum() - cnt).sum()
    return tot / seg.size


# ------------------------------------------------------------------ clustering (GPU's reformulation)

def _nearest_seed_labels(W, H, S):
    """Closed form of one pass on a one-colour image: D is m^2 (dx^2 + dy^2), separable, so the label
    is (nearest seed row) * gw + (nearest seed column), the smaller index on ties."""
    def axis(n):
        cells = -(-n // S)
        seeds = np.array([i * S + (min(S, n - i * S) - 1) // 2 for i in range(cells)])
        d = np.abs(np.arange(n)[:, None] - seeds[None, :])
        return np.argmin(d, axis=1)  # first minimum = smaller index on ties
    gw = -(-W // S)
    return axis(H)[:, None] * gw + axis(W)[None, :]


@pytest.mark.parametrize("W,H,S", [(48, 32, 8), (50, 37, 7), (61, 29, 6), (33, 21, 4), (9, 5, 1), (17, 3, 5)])
def test_one_pass_on_a_uniform_image_takes_the_nearest_seed(W, H, S):
    f = _frame(np.full((H, W), 77), np.full((H, W), 3), np.full((H, W), 200))
    lab = oracle.superpixels(f, 1, 8, S, 5, 1, connect=False)
    assert np.array_equal(lab, _nearest_seed_labels(W, H, S))
    assert oracle.grid_segments(W, H, S) == _grid(W, H, S).max() + 1


@pytest.mark.parametrize("W,H,S", [(48, 32, 8), (49, 35, 7), (60, 30, 6), (36, 20, 4), (9, 5, 1)])
@pytest.mark.parametrize("iterations", [1, 5])
def test_uniform_image_gives_the_grid_cells(W, H, S, iterations):
    """Closed form when S divides W and H: every pixel is nearest to its own cell's seed (for even S the
    pixels half-way between two seeds tie and go to the smaller label, their own cell), the cell means
    are the cell centres, and the grid is a fixed point of the passes."""
    f = _frame(np.full((H, W), 77), np.full((H, W), 3), np.full((H, W), 200))
    for connect in (False, True):
        lab = oracle.superpixels(f, 1, 8, S, 5, iterations, connect=connect)
        assert np.array_equal(lab, _grid(W, H, S))


def _strip(values, channel=0, bd=8):
    vals = np.asarray(values)
    planes = [np.zeros((1, len(vals)), np.uint16 if bd > 8 else np.uint8) for _ in range(3)]
    planes[channel][0] = vals
    return synth.View(*planes)


@pytest.mark.parametrize("channel", [0, 1, 2])
def test_colour_against_space_weights_worked_example(channel):
    """1x8 strip, S = 4: seeds at x = 1 (colour 0) and x = 5 (colour 100); pixel 2 has colour 60.
    In 1/16 units, D_k = S^2 (16*60 - C_k)^2 + m^2 (16*2 - X_k)^2:
      D_0 = 16 * 960^2 + m^2 * 16^2 = 14745600 + 256 m^2
      D_1 = 16 * 640^2 + m^2 * 48^2 = 6553600 + 2304 m^2
    so pixel 2 joins cluster 0 exactly when m^2 > 4000, i.e. m >= 64. Every channel counts alike."""
    vals = [0, 0, 60, 60, 100, 100, 100, 100]
    lab63 = oracle.superpixels(_strip(vals, channel), 1, 8, 4, 63, 1, connect=False)
    lab64 = oracle.superpixels(_strip(vals, channel), 1, 8, 4, 64, 1, connect=False)
    assert lab63.ravel().tolist() == [0, 0, 1, 1, 1, 1, 1, 1]
    assert lab64.ravel().tolist() == [0, 0, 0, 1, 1, 1, 1, 1]


def test_bit_depth_scales_the_spatial_weight():
    """At 10 bits colours are 4x larger; the spatial term is multiplied by 4^2, so the decision of the
    8-bit worked example is unchanged (threshold still m >= 64)."""
    vals = [0, 0, 240, 240, 400, 400, 400, 400]
    assert oracle.superpixels(_strip(vals, 0, 10), 2, 10, 4, 63, 1, False).ravel().tolist() == [0, 0, 1, 1, 1, 1, 1, 1]
    assert oracle.superpixels(_strip(vals, 0, 10), 2, 10, 4, 64, 1, False).ravel().tolist() == [0, 0, 0, 1, 1, 1, 1, 1]


def test_columns_behave_like_rows():
    """The worked example transposed into an 8x1 column gives the transposed labels (y is handled like x)."""
    vals = np.array([0, 0, 60, 60, 100, 100, 100, 100], np.uint8).reshape(8, 1)
    f = synth.View(vals, np.zeros_like(vals), np.zeros_like(vals))
    assert oracle.superpixels(f, 1, 8, 4, 63, 1, False).ravel().tolist() == [0, 0, 1, 1, 1, 1, 1, 1]
    assert oracle.superpixels(f, 1, 8, 4, 64, 1, False).ravel().tolist() == [0, 0, 0, 1, 1, 1, 1, 1]


def test_mean_update_rounds_half_up_worked_example():
    """1x6 strip, S = 3, m = 0 (colour only), colours [1, 0, 1, 10, 19, 29]; seeds x = 1 (0), x = 4 (19).
    Pass 1: pixels 0..2 -> cluster 0, pixel 3: |10-0| = 10 > |10-19| = 9 -> cluster 1, 4, 5 -> cluster 1.
    Update: cluster 0 sum 2 over 3 -> 16 * 2/3 = 10.67 -> 11 (floor would give 10);
            cluster 1 sum 58 over 3 -> 16 * 58/3 = 309.33 -> 309.
    Pass 2, pixel 3 (160): |160 - 11| = 149 = |160 - 309| -> tie -> the smaller label 0."""
    f = _strip([1, 0, 1, 10, 19, 29])
    assert oracle.superpixels(f, 1, 8, 3, 0, 1, False).ravel().tolist() == [0, 0, 0, 1, 1, 1]
    assert oracle.superpixels(f, 1, 8, 3, 0, 2, False).ravel().tolist() == [0, 0, 0, 0, 1, 1]


def test_cluster_without_pixels_keeps_its_mean_worked_example():
    """1x9 strip, S = 3, m = 0, colours [50, 50, 60, 70, 50, 50, 200, 200, 200]. Seeds 0 and 1 both
    have colour 50, so in pass 1 every pixel that sees both ties and takes cluster 0: cluster 1 is
    empty and keeps its seed colour 50 (800). Cluster 0 (pixels 0..5) moves to 55 (880). Pass 2: the
    pixels of colour 50 are at 0 from cluster 1 and at 80 from cluster 0."""
    f = _strip([50, 50, 60, 70, 50, 50, 200, 200, 200])
    assert oracle.superpixels(f, 1, 8, 3, 0, 1, False).ravel().tolist() == [0, 0, 0, 0, 0, 0, 2, 2, 2]
    assert oracle.superpixels(f, 1, 8, 3, 0, 2, False).ravel().tolist() == [1, 1, 0, 0, 1, 1, 2, 2, 2]


def test_candidates_are_the_three_by_three_neighbouring_cells():
    """12x9 image, S = 3: a 4x3 grid, label = 4 j + i. All pixels 0 except pixel (0,0) = 90, the seed
    of cell (1,1) (label 5, pixel (4,4)) = 100, and the seed of cell (2,2) (label 10, pixel (7,7)) = 90.
    With m = 0 pixel (0,0) sees cells (0..1, 0..1) only and takes label 5, not the exact match 10."""
    Y = np.zeros((9, 12), np.uint8)
    Y[0, 0] = 90
    Y[4, 4] = 100
    Y[7, 7] = 90
    lab = oracle.superpixels(_frame(Y), 1, 8, 3, 0, 1, False)
    assert lab[0, 0] == 5
    assert lab[4, 4] == 5 and lab[7, 7] == 10


# ------------------------------------------------------------------------------ connectivity step

def test_connectivity_main_tie_and_smallest_name_worked_example():
    """Uniform colour, so every colour distance is 0 and ties go to the smallest group name.
    Label 2 has two components of 8 pixels: the ring (named 8) is earlier and stays; the block in
    rows 5-6 (named 35) touches groups 0 and 39 and joins 0. The centre pixel of label 3 (named 16)
    touches only the ring and joins it."""
    lab = np.array([[0, 0, 0, 0, 0, 1, 1],
                    [0, 2, 2, 2, 0, 1, 1],
                    [0, 2, 3, 2, 0, 1, 1],
                    [0, 2, 2, 2, 0, 1, 1],
                    [0, 0, 0, 0, 0, 1, 1],
                    [2, 2, 2, 2, 3, 3, 1],
                    [2, 2, 2, 2, 3, 3, 1]], np.int32)
    want = np.array([[0, 0, 0, 0, 0, 1, 1],
                     [0, 2, 2, 2, 0, 1, 1],
                     [0, 2, 2, 2, 0, 1, 1],
                     [0, 2, 2, 2, 0, 1, 1],
                     [0, 0, 0, 0, 0, 1, 1],
                     [0, 0, 0, 0, 3, 3, 1],
                     [0, 0, 0, 0, 3, 3, 1]], np.int32)
    got = oracle.connectivity(lab, 4, _frame(np.full(lab.shape, 9)), 1)
    assert np.array_equal(got, want)


def test_connectivity_nested_orphans_merge_in_one_round():
    """Label 2's ring (named 6) is smaller than its 9-pixel block; the ring touches groups 0, 3 and
    the centre (12) and picks 0; the centre touches only the ring and picks it; both links merge in
    the same round, so the centre ends in label 0 too."""
    lab = np.array([[0, 0, 0, 1, 1],
                    [0, 2, 2, 2, 1],
                    [0, 2, 3, 2, 1],
                    [0, 2, 2, 2, 1],
                    [0, 0, 1, 1, 1],
                    [2, 2, 2, 3, 3],
                    [2, 2, 2, 3, 3],
                    [2, 2, 2, 3, 3]], np.int32)
    want = lab.copy()
    want[1:4, 1:4] = 0
    got = oracle.connectivity(lab, 4, _frame(np.zeros(lab.shape)), 1)
    assert np.array_equal(got, want)


def test_connectivity_picks_the_nearest_mean_colour_worked_example():
    """The orphan {(1,1), (2,1)} of label 2 (colour 45) touches group 0 (colour 10) and group 3
    (label 1, colour 50): |720 - 160| = 560 > |720 - 800| = 80 in 1/16 units, so it joins label 1
    although group 3 has the larger name."""
    lab = np.array([[0, 0, 0, 1, 1, 1],
                    [0, 2, 2, 1, 1, 1],
                    [0, 0, 0, 1, 1, 1],
                    [2, 2, 2, 2, 2, 2]], np.int32)
    Y = np.where(lab == 0, 10, np.where(lab == 1, 50, 100))
    Y[1, 1] = Y[1, 2] = 45
    got = oracle.connectivity(lab, 3, _frame(Y), 1)
    want = lab.copy()
    want[1, 1] = want[1, 2] = 1
    assert np.array_equal(got, want)


def test_connectivity_mutual_picks_merge_then_use_the_merged_mean():
    """Strip [0 0 | A | B | 3 3 | 1 1 | 2 2] with colours [0, 0, 40, 62, 100, 100, ...]. A (label 1)
    and B (label 2) are orphans. A: |40 - 0| = 40 vs |40 - 62| = 22 -> B; B: 22 vs |62 - 100| = 38 -> A.
    Round 1 merges them into an unanchored group of mean 51 (816); round 2: |816 - 0| = 816 >
    |816 - 1600| = 784, so both join label 3 (A alone would have joined label 0)."""
    lab = np.array([[0, 0, 1, 2, 3, 3, 1, 1, 2, 2]], np.int32)
    Y = np.array([[0, 0, 40, 62, 100, 100, 7, 7, 250, 250]])
    got = oracle.connectivity(lab, 4, _frame(Y), 1)
    assert got.ravel().tolist() == [0, 0, 3, 3, 3, 3, 1, 1, 2, 2]


@pytest.mark.parametrize("seed", [0, 1])
def test_connectivity_invariants_on_noisy_clusterings(seed):
    """On a noisy mosaic the raw clustering is fragmented; afterwards every label is one 8-connected
    set, and every pixel of a label's largest raw component (scipy's 8-connected labelling) keeps it."""
    f = synth.mosaic(96, 64, 10, noise_sigma=12, seed=seed)
    raw = oracle.superpixels(f, 1, 8, 6, 5, 3, connect=False)
    K = oracle.grid_segments(96, 64, 6)
    assert max(_components_per_label(raw).values()) > 1
    out = oracle.connectivity(raw, K, f, 1)
    assert all(n == 1 for n in _components_per_label(out).values())
    assert np.array_equal(out, oracle.superpixels(f, 1, 8, 6, 5, 3, connect=True))
    for k in np.unique(raw):
        cc, n = ndimage.label(raw == k, EIGHT)
        sizes = np.bincount(cc.ravel())[1:]
        largest = np.flatnonzero(sizes == sizes.max())
        # the earliest in raster order among equally large components
        first = min(largest, key=lambda i: np.flatnonzero((cc == i + 1).ravel())[0])
        assert np.all(out[cc == first + 1] == k)


# ------------------------------------------------------------------------------------------ SNIC

def test_snic_worked_example_running_mean_and_push_order():
    """1x6 strip, S = 3, m = 0, colours [0, 0, 9, 11, 20, 20]; seeds x = 1 (0) and x = 4 (20).
    Pops: seed 0 (pushes x0 at 0, x2 at 9*81 = 729), seed 1 (pushes x3 at 9*81 = 729, x5 at 0), x0, x5,
    then x2 (729, pushed before x3's 729): the mean of cluster 0 becomes 3, x3 is pushed again at
    9*64 = 576 and joins cluster 0, although its colour is nearer to seed 1's."""
    assert oracle.snic(_strip([0, 0, 9, 11, 20, 20]), 1, 8, 3, 0).ravel().tolist() == [0, 0, 0, 0, 1, 1]


def test_snic_worked_example_equal_distances_leave_in_push_order():
    """1x6 strip, S = 3, m = 0, colours [40, 50, 60, 70, 88, 88]; seeds x = 1 (50), x = 4 (88).
    Seed 0 pushes x0 then x2, both at 9*10^2 = 900; seed 1 pushes x3 at 9*18^2 = 2916 and x5 at 0.
    x0 leaves first (pushed first): mean 45; then x2: mean 50, and x2 pushes x3 at 9*20^2 = 3600.
    x3 then goes to cluster 1 (2916). Had x2 left before x0, the mean would have been 55 and x3's
    push 9*15^2 = 2025, taking it into cluster 0."""
    assert oracle.snic(_strip([40, 50, 60, 70, 88, 88]), 1, 8, 3, 0).ravel().tolist() == [0, 0, 0, 1, 1, 1]


def test_snic_worked_example_grows_through_diagonal_neighbours():
    """6x3 image, S = 3, m = 0, colour 100 except the diagonal chain (1,1), (2,0), (3,1) of colour 0;
    seeds (1,1) (cluster 0, colour 0) and (4,1) (cluster 1, colour 100). Cluster 0 reaches (2,0) and
    then (3,1) diagonally at distance 0; cluster 1 takes every pixel of colour 100 at distance 0. With
    4-neighbours only, cluster 0 could not leave its seed."""
    Y = np.full((3, 6), 100)
    for x, y in ((1, 1), (2, 0), (3, 1)):
        Y[y, x] = 0
    want = np.ones((3, 6), np.int32)
    for x, y in ((1, 1), (2, 0), (3, 1)):
        want[y, x] = 0
    assert np.array_equal(oracle.snic(_frame(Y), 1, 8, 3, 0), want)


@pytest.mark.parametrize("W,H,S,m", [(64, 48, 8, 5), (57, 31, 6, 0), (40, 40, 5, 40)])
def test_snic_invariants(W, H, S, m):
    """Every pixel is labelled with a grid label, every label is one 8-connected set grown from its
    seed, and each seed pixel carries its own label (seeds leave the queue first)."""
    f = synth.mosaic(W, H, 7, noise_sigma=10, seed=W)
    lab = oracle.snic(f, 1, 8, S, m)
    K = oracle.grid_segments(W, H, S)
    assert lab.min() >= 0 and lab.max() < K
    assert all(n == 1 for n in _components_per_label(lab).values())
    gw, gh = -(-W // S), -(-H // S)
    for j in range(gh):
        for i in range(gw):
            w, h = min(S, W - i * S), min(S, H - j * S)
            assert lab[j * S + (h - 1) // 2, i * S + (w - 1) // 2] == j * gw + i


# --------------------------------------------------------------- quality against the paper's SNIC

@pytest.mark.parametrize("noise", [0, 8, 16])
def test_reformulation_segments_as_well_as_snic(noise):
    """Ground truth: the mosaic's regions. The data-parallel clustering with its connectivity step
    keeps segments inside regions as well as SNIC does (undersegmentation error within 0.005) and
    finds the region boundaries as well (boundary recall within 0.01)."""
    f = synth.mosaic(240, 160, 24, noise_sigma=noise, seed=noise + 5)
    ours = oracle.superpixels(f, 1, 8, 8, 5, 10)
    ref = oracle.snic(f, 1, 8, 8, 5)
    ue_o, ue_r = undersegmentation_error(ours, f.plane_id), undersegmentation_error(ref, f.plane_id)
    br_o, br_r = boundary_recall(ours, f.plane_id), boundary_recall(ref, f.plane_id)
    assert ue_o <= ue_r + 0.005, (ue_o, ue_r)
    assert br_o >= br_r - 0.01, (br_o, br_r)
    assert all(n == 1 for n in _components_per_label(ours).values())
