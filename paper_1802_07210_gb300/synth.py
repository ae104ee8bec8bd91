"""Seeded synthetic stereo pairs shaped like the paper's workloads.

The paper evaluates on KITTI (1242x375) and New Tsukuba (640x480), Sec. VII.
Neither dataset is available, so every input here is generated: a
piecewise-planar disparity field (Voronoi cells, one slanted plane per cell,
integer-rounded), band-limited texture (uniform noise, 3x3 box blur), the right
image obtained by forward-warping the left one by the disparity field (larger
disparity wins; disoccluded pixels get fresh texture) and additive Gaussian
noise clipped to uint8.

This module holds no step of the stereo method itself: it only makes inputs,
and both the CUDA path and the oracle consume them.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class SceneSpec:
    w: int
    h: int
    n_planes: int
    d_lo: float
    d_hi: float
    noise_sigma: float = 2.0
    ground_max: float = 0.0     # >0: ground plane rising 0 -> ground_max top to bottom
    slope: float = 0.12         # max |dd/du|, |dd/dv| of a plane


@dataclass
class Workload:
    name: str
    spec: SceneSpec
    disp_max: int
    postprocess: bool = False
    params: dict = field(default_factory=dict)


def _box3(a: np.ndarray) -> np.ndarray:
    p = np.pad(a.astype(np.int32), 1, mode="edge")
    s = sum(p[dy:dy + a.shape[0], dx:dx + a.shape[1]] for dy in range(3) for dx in range(3))
    return (s + 4) // 9


def _texture(rng, h, w):
    return _box3(rng.integers(0, 256, size=(h, w), dtype=np.int32)).astype(np.float64)


def disparity_field(spec: SceneSpec, rng) -> np.ndarray:
    """Integer disparity per left-image pixel (int32)."""
    h, w, k = spec.h, spec.w, spec.n_planes
    sx = rng.uniform(0, w, size=k)
    sy = rng.uniform(0, h, size=k)
    dc = rng.uniform(spec.d_lo, spec.d_hi, size=k)
    a = rng.uniform(-spec.slope, spec.slope, size=k)
    b = rng.uniform(-spec.slope, spec.slope, size=k)
    uu = np.arange(w, dtype=np.float64)[None, :]
    out = np.empty((h, w), np.int32)
    chunk = max(1, (1 << 22) // max(1, w * k))
    for v0 in range(0, h, chunk):
        vv = np.arange(v0, min(h, v0 + chunk), dtype=np.float64)[:, None]
        d2 = (uu[..., None] - sx) ** 2 + (vv[..., None] - sy) ** 2  # (rows, w, k)
        lab = np.argmin(d2, axis=-1)
        d = dc[lab] + a[lab] * (uu - sx[lab]) + b[lab] * (vv - sy[lab])
        if spec.ground_max > 0:
            g = spec.ground_max * vv / max(1, h - 1)
            d = np.maximum(d, np.broadcast_to(g, d.shape))
        out[v0:v0 + len(vv)] = np.rint(np.clip(d, spec.d_lo, spec.d_hi)).astype(np.int32)
    return out


def make_pair(spec: SceneSpec, seed: int):
    """Returns (left uint8 [h][w], right uint8 [h][w], gt int32 [h][w])."""
    rng = np.random.default_rng(seed)
    h, w = spec.h, spec.w
    D = disparity_field(spec, rng)
    L = _texture(rng, h, w)
    fill = _texture(rng, h, w)
    # forward warp R(u - D, v) = L(u, v); larger disparity (closer) wins, then larger u
    vv, uu = np.mgrid[0:h, 0:w]
    x = uu - D
    ok = x >= 0
    key = (vv * w + x)[ok]
    dd = D[ok]
    src = (vv * w + uu)[ok]
    order = np.lexsort((src, dd, key))
    ks = key[order]
    last = np.ones(len(ks), bool)
    last[:-1] = ks[:-1] != ks[1:]
    R = fill.reshape(-1).copy()
    R[ks[last]] = L.reshape(-1)[src[order][last]]
    R = R.reshape(h, w)
    nl = rng.normal(0.0, spec.noise_sigma, size=(h, w))
    nr = rng.normal(0.0, spec.noise_sigma, size=(h, w))
    Li = np.clip(np.rint(L + nl), 0, 255).astype(np.uint8)
    Ri = np.clip(np.rint(R + nr), 0, 255).astype(np.uint8)
    return Li, Ri, D


def fronto_parallel_pair(w: int, h: int, shift: int, seed: int, noise_sigma: float = 0.0):
    """Textured pair with one constant integer disparity `shift`:
    R(u - shift, v) = L(u, v) exactly where u - shift >= 0 (noise-free unless
    noise_sigma > 0)."""
    rng = np.random.default_rng(seed)
    T = _texture(rng, h, w + shift)
    Lw = T[:, 0:w]                      # left(u)  = T(u)
    Rw = T[:, shift:shift + w]          # right(x) = T(x + shift) -> right(u - shift) = left(u)
    if noise_sigma > 0:
        Lw = Lw + rng.normal(0, noise_sigma, Lw.shape)
        Rw = Rw + rng.normal(0, noise_sigma, Rw.shape)
    return (np.clip(np.rint(Lw), 0, 255).astype(np.uint8),
            np.clip(np.rint(Rw), 0, 255).astype(np.uint8))


# The workloads (sizes, disparity ranges, plane counts, noise) of the paper's
# datasets and the serving mix.  ELAS parameters are the "robotics" set.
ROBOTICS = dict(support_threshold=0.85, support_texture=10, candidate_stepsize=5,
                incon_window_size=5, incon_threshold=5, incon_min_support=5,
                redun_max_dist=5, grid_size=20, beta=0.02, gamma=3.0, sigma=1.0,
                sradius=2, match_texture=1, lr_threshold=2)

SMALL_320 = Workload("320x240_D64", SceneSpec(320, 240, 6, 2, 60, 2.0, slope=0.10), 63,
                     postprocess=False, params=dict(ROBOTICS, disp_min=0, disp_max=63,
                                                    ipol_gap_width=0, filter_adaptive_mean=0))
VGA_640 = Workload("640x480_D256", SceneSpec(640, 480, 20, 0, 250, 2.0, slope=0.15), 255,
                   postprocess=True, params=dict(ROBOTICS, disp_min=0, disp_max=255,
                                                 ipol_gap_width=3, filter_adaptive_mean=1))
KITTI_1242 = Workload("1242x375_D256", SceneSpec(1242, 375, 40, 0, 250, 3.0, ground_max=120,
                                                  slope=0.15), 255,
                      postprocess=False, params=dict(ROBOTICS, disp_min=0, disp_max=255,
                                                     ipol_gap_width=0, filter_adaptive_mean=0))

MIXED_SIZES = [(320, 240), (640, 480), (1242, 375), (1280, 720), (1920, 1080)]
MIXED_D = [64, 128, 256]


def scaled_workload(w: int, h: int, D: int) -> Workload:
    """Generator scaled to an arbitrary size and disparity count D."""
    n = int(np.clip(round(20 * w * h / 307200), 6, 60))
    spec = SceneSpec(w, h, n, 0, 0.98 * (D - 1), 2.0, slope=0.12)
    return Workload(f"{w}x{h}_D{D}", spec, D - 1,
                    params=dict(ROBOTICS, disp_min=0, disp_max=D - 1,
                                ipol_gap_width=0, filter_adaptive_mean=0))


def mixed_batch(n: int, seed: int):
    """(workload, pair seed) list for the mixed-size batch."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w, h = MIXED_SIZES[rng.integers(len(MIXED_SIZES))]
        D = MIXED_D[rng.integers(len(MIXED_D))]
        out.append((scaled_workload(w, h, D), seed * 1000 + i))
    return out


def workload_pair(wl: Workload, index: int, cfg_id: int = 0):
    """Pair `index` of a workload, seeded as 1000*cfg_id + index."""
    return make_pair(wl.spec, 1000 * cfg_id + index)
