"""Pins of the oracle's descriptor step (Sec. III.A, Fig. 1(b-d); Sec. VI.A)
against hand-derived values, closed forms, the mirror symmetry and a library
correlation."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_impulse_golden(orc):
    g = json.load(open(os.path.join(GOLD, "impulse_descriptor.json")))
    img = np.zeros((g["h"], g["w"]), np.uint8)
    x0, y0, val = g["impulse"]
    img[y0, x0] = val
    du, dv = orc.sobel(img)
    exp_du = np.zeros_like(du)
    exp_dv = np.zeros_like(dv)
    for x, y, s in g["du_nonzero"]:
        exp_du[y, x] = s
    for x, y, s in g["dv_nonzero"]:
        exp_dv[y, x] = s
    np.testing.assert_array_equal(du, exp_du)
    np.testing.assert_array_equal(dv, exp_dv)
    desc = orc.descriptors(img)
    for key, bytes_ in g["descriptors"].items():
        x, y = map(int, key.split(","))
        np.testing.assert_array_equal(desc[y, x], np.array(bytes_, np.uint8))


def test_constant_image_is_flat(orc):
    img = np.full((17, 23), 77, np.uint8)
    desc = orc.descriptors(img)
    assert (desc == 128).all()


def test_vertical_step_edge_and_saturation(orc):
    # step of height s at column u0: du = 4s at u0-1 and u0 (interior rows), 0 elsewhere
    h, w, u0 = 9, 12, 6
    for s, q in [(100, 228), (255, 255), (30, 158)]:
        img = np.zeros((h, w), np.uint8)
        img[:, u0:] = s
        du, dv = orc.sobel(img)
        exp = np.zeros((h, w), np.int32)
        exp[1:h - 1, u0 - 1] = 4 * s
        exp[1:h - 1, u0] = 4 * s
        np.testing.assert_array_equal(du, exp)
        assert (dv == 0).all()
        desc = orc.descriptors(img)
        # byte 2 samples du at (-1, 0), byte 3 at (+1, 0)
        assert desc[4, u0, 2] == q and desc[4, u0, 3] == 128
        assert desc[4, u0 - 2, 3] == q
        # falling edge saturates at 1 (not 0): q(-s) = 256 - q(s)
        desc_m = orc.descriptors(255 - img)
        assert desc_m[4, u0, 2] == 256 - q


def test_frame_and_outside_read_128(orc):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (10, 14), dtype=np.uint8)
    du, dv = orc.sobel(img)
    assert (du[0] == 0).all() and (du[-1] == 0).all() and (du[:, 0] == 0).all() and (du[:, -1] == 0).all()
    desc = orc.descriptors(img)
    # pixel (0,0): every sample with a negative offset is outside -> 128
    assert desc[0, 0, 0] == 128 and desc[0, 0, 8] == 128


def _mirror_perm():
    du = [(-2, -2), (2, -2), (-1, 0), (1, 0), (-2, 2), (2, 2), (0, -1), (0, 1)]
    dv = [(0, -2), (0, 2), (-2, 0), (2, 0), (-1, -1), (1, -1), (-1, 1), (1, 1)]
    perm = [du.index((-x, y)) for x, y in du] + [8 + dv.index((-x, y)) for x, y in dv]
    return perm


def test_mirror_invariant(orc):
    """desc(mirror I)(W-1-u, v) is desc(I)(u, v) with the sample offsets
    mirrored (x -> -x) and the du bytes complemented (256 - q)."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, (31, 45), dtype=np.uint8)
    d = orc.descriptors(img).astype(np.int32)
    dm = orc.descriptors(img[:, ::-1].copy()).astype(np.int32)
    perm = _mirror_perm()
    expect = d[:, ::-1][:, :, perm]
    expect[:, :, :8] = 256 - expect[:, :, :8]
    np.testing.assert_array_equal(dm, expect)


def test_transpose_swaps_gradients(orc):
    """Transposing the image swaps du and dv exactly (the stencils are
    transposes of each other)."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (19, 27), dtype=np.uint8)
    du, dv = orc.sobel(img)
    duT, dvT = orc.sobel(img.T.copy())
    np.testing.assert_array_equal(duT, dv.T)
    np.testing.assert_array_equal(dvT, du.T)


def test_interior_gradients_match_a_library_correlation(orc):
    """Inside the one-pixel frame, du and dv are the correlations of the image
    with the 3x3 Sobel kernels (a library routine): a wrong weight, sign or a
    transposed kernel fails here."""
    ndimage = pytest.importorskip("scipy.ndimage")
    K = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.int64)
    rng = np.random.default_rng(8)
    for h, w in ((37, 53), (5, 5), (64, 200)):
        img = rng.integers(0, 256, (h, w)).astype(np.uint8)
        du, dv = orc.sobel(img)
        inner = (slice(1, -1), slice(1, -1))
        np.testing.assert_array_equal(du[inner], ndimage.correlate(img.astype(np.int64), K)[inner])
        np.testing.assert_array_equal(dv[inner], ndimage.correlate(img.astype(np.int64), K.T)[inner])
