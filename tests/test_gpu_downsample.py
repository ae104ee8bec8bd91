"""Parity of support down-sampling (Sec. VII: 1/8, 1/14, 1/32 of the
extracted support points) with the oracle through the C-ABI: the candidate
grid, the list and its count, the grid vectors, and the whole one-pair path,
on the default lattice and on the every-pixel lattice the paper's variant
extracts from (batches and the server: test_gpu_variants_batched.py)."""

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, grid_as_i32, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _support_case(wl, cfg, prm):
    B = _B()
    L, R, _ = synth.workload_pair(wl, 0, cfg)
    h, w = L.shape
    dL, dR = oracle.descriptors(L), oracle.descriptors(R)
    exp = oracle.support_points(dL, dR, prm)
    lst = oracle.support_list(exp, prm)
    r = B.elas_support_points(dev(dL), dev(dR), prm)
    np.testing.assert_array_equal(host(r["d_can"]), exp)
    n = int(host(r["count"])[0])
    assert n == len(lst)
    np.testing.assert_array_equal(host(r["list"])[:n], lst)
    np.testing.assert_array_equal(host(r["grid_L"]), grid_as_i32(oracle.grid_vectors(lst, w, h, prm)))
    np.testing.assert_array_equal(host(r["grid_R"]), grid_as_i32(oracle.grid_vectors(lst, w, h, prm, right=True)))
    return n


@pytest.mark.parametrize("k", [2, 8, 14, 32])
@pytest.mark.parametrize("name,wl,cfg", [("small_320", synth.SMALL_320, 1), ("vga_640", synth.VGA_640, 2)])
def test_downsampled_support(name, wl, cfg, k):
    n = _support_case(wl, cfg, dict(wl.params, support_downsample=k))
    assert n >= 1


def test_every_pixel_lattice_downsampled():
    """Candidates at every pixel (the paper's variant extracts support
    everywhere), then 1/14 of the filtered points; the row-organised
    matcher runs (one lattice row per pixel row)."""
    wl = synth.scaled_workload(180, 320, 48)
    n = _support_case(wl, 2, dict(wl.params, candidate_stepsize=1, support_downsample=14))
    assert n > 50


@pytest.mark.parametrize("k", [8, 14])
def test_pipeline_downsampled(k):
    B = _B()
    for wl, cfg in ((synth.SMALL_320, 1), (synth.scaled_workload(203, 117, 48), 7)):
        prm = dict(wl.params, support_downsample=k)
        L, R, _ = synth.workload_pair(wl, 0, cfg)
        ref = oracle.pipeline(L, R, prm, postprocess_on=False)
        h, w = L.shape
        pl = B.Pipeline(w, h, prm)
        dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
        dR = torch.empty_like(dL)
        for _ in range(2):
            pl.run(dev(L), dev(R), dL, dR)
            np.testing.assert_array_equal(host(dL), ref["lrL"])
            np.testing.assert_array_equal(host(dR), ref["lrR"])
        assert pl.stats()["n_support"] == len(ref["list"])
        pl.close()
