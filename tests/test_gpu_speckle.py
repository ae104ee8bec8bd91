"""Parity of the GPU small-segment (speckle) removal with the oracle, bit for
bit: piecewise maps with holes over several tiles and a ragged tail, the
LR-checked maps of the path at the paper's workload sizes, segments that
wind across many tile borders, and the degenerate maps (one pixel, one row,
one column, nothing valid, one segment covering everything)."""
import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _check(d, thr, min_size, in_place=False):
    B = _B()
    t = dev(d)
    if in_place:
        out, st = B.elas_speckle(t, thr, min_size, out=t, with_status=True)
    else:
        out, st = B.elas_speckle(t, thr, min_size, with_status=True)
    exp = oracle.speckle(d, thr, min_size)
    np.testing.assert_array_equal(host(out), exp)
    assert int(host(st)[0]) == 0
    return exp


def _piecewise(w, h, seed, hole=0.15):
    rng = np.random.default_rng(seed)
    base = np.add.outer(np.arange(h) // 7, np.arange(w) // 11) * 3
    d = (base + rng.integers(-2, 3, base.shape)).astype(np.int16)
    d[rng.random(d.shape) < hole] = -1
    return d


@pytest.mark.parametrize("size", [(37, 29), (203, 117), (640, 480), (1242, 375)])
@pytest.mark.parametrize("thr,min_size", [(0, 3), (1, 20), (2, 200)])
def test_piecewise_maps(size, thr, min_size):
    w, h = size
    exp = _check(_piecewise(w, h, w + thr), thr, min_size)
    assert (exp >= 0).any()


def test_in_place():
    _check(_piecewise(203, 117, 5), 1, 30, in_place=True)


@pytest.mark.parametrize("name,wl,cfg", [("vga_640", synth.VGA_640, 2), ("kitti_1242", synth.KITTI_1242, 0)])
def test_lr_checked_maps_of_the_path(name, wl, cfg):
    """ELAS's defaults (threshold 1, 200 pixels) on the path's LR-checked maps."""
    B = _B()
    L, R, _ = synth.workload_pair(wl, 0, cfg)
    h, w = L.shape
    pl = B.Pipeline(w, h, wl.params)
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    pl.run(dev(L), dev(R), dL)
    pl.close()
    d = host(dL)
    exp = _check(d, 1, 200)
    assert (exp != d).any() and (exp >= 0).sum() > 0.3 * d.size


def test_winding_segments_cross_many_tiles():
    """A one-pixel-wide serpentine of equal values (one segment thousands of
    pixels long through every tile), a comb whose teeth meet only at the
    bottom, and a staircase that drifts by one per pixel."""
    w, h = 300, 130
    d = np.full((h, w), -1, np.int16)
    for y in range(0, h, 2):
        d[y, :] = 9
        d[y + 1 if y + 1 < h else y, (w - 1) if (y // 2) % 2 == 0 else 0] = 9
    _check(d, 0, 5000)
    _check(d, 0, 100)
    comb = np.full((h, w), -1, np.int16)
    comb[:, ::3] = 4
    comb[h - 1, :] = 4
    _check(comb, 0, 200)
    comb[h - 1, 150] = -1   # cut the spine: two halves
    _check(comb, 0, 5000)
    stair = np.tile((np.arange(w) % 200).astype(np.int16), (h, 1))
    _check(stair, 1, 1000)
    _check(stair, 0, 200)


@pytest.mark.parametrize("size", [(1, 1), (1, 57), (61, 1), (33, 17)])
def test_degenerate_maps(size):
    w, h = size
    _check(np.full((h, w), -1, np.int16), 1, 2)
    _check(np.full((h, w), 5, np.int16), 1, w * h)
    _check(np.full((h, w), 5, np.int16), 1, w * h + 1)
    rng = np.random.default_rng(w * h)
    _check(rng.integers(-1, 6, (h, w)).astype(np.int16), 1, 3)


def test_one_segment_covering_a_large_map():
    d = np.full((1080, 1920), 40, np.int16)
    _check(d, 0, 200)
    d[::97, :] = -1   # horizontal cuts every 97 rows: 12 bands
    exp = _check(d, 0, 96 * 1920)
    assert (exp == 40).sum() == 11 * 96 * 1920
