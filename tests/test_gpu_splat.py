"""GPU parity of the tile-based splat rasteriser (Sec. 3.5, Eqs. 7-9) against the oracle on the same seeded Gaussians.

The projection, the reach test and the depth order are float decisions both sides take alike, so the only
differences are float accumulation, exp rounding and the GPU's stop once a pixel's transmittance is below 1e-4
(which changes its colour by less than 1e-4 times the largest colour, 1 here): colour and transmittance within 2e-4
absolute. Whole images on small cameras (ragged 16 x 16 tiles), sampled pixels at the 640 x 480 camera with a
million Gaussians, and the degenerate cases."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_21459_b300 import build
    build.build()


def mrh():
    import paper_2511_21459_b300 as m
    return m


def small_camera(wl, w, h):
    s = w / wl.width
    return dataclasses.replace(wl, width=w, height=h, fx=wl.fx * s, fy=wl.fy * s, cx=(w - 1) / 2, cy=(h - 1) / 2)


def to_dev(g):
    return {k: torch.from_numpy(v).cuda() for k, v in g.items()}


def render_gpu(gd, K, T, trans=None):
    rgb, tr, pairs = mrh().splat_render(gd["means"], gd["covs"], gd["opacity"], gd["colors"], K, T, trans=trans)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), (tr.cpu().numpy() if tr is not None else None), pairs


@pytest.mark.parametrize("size,n,frame", [((150, 110), 20000, 20), ((160, 120), 60000, 75), ((97, 61), 5000, 140)])
def test_whole_images_match_the_oracle(size, n, frame):
    wl = small_camera(synth.rgbd(), *size)
    g = synth.gaussians(synth.rgbd(), n)
    T = wl.pose(frame)
    rgb_o, tr_o, drawn = oracle.splat_render(g["means"], g["covs"], g["opacity"], g["colors"], oracle.pinhole_from(wl), T)
    rgb_g, tr_g, pairs = render_gpu(to_dev(g), mrh().pinhole_from(wl), T)
    assert drawn > n // 10 and pairs > 0
    assert np.abs(rgb_g - rgb_o).max() <= TOL
    assert np.abs(tr_g - tr_o).max() <= TOL
    assert (tr_o < 0.99).mean() > 0.3  # most pixels receive some Gaussian


def test_needles_and_discs_match_the_oracle():
    """Thin, tilted Gaussians (standard deviations 100:1:1 and 1:1:0.01): elongated image ellipses, whose boxes hold
    many tiles the ellipse misses; the culled tiles must be ones no pixel of which the ellipse reaches."""
    rng = np.random.default_rng(21)
    wl = small_camera(synth.rgbd(), 160, 120)
    n = 3000
    T = wl.pose(30)
    pc = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-0.9, 0.9, n), rng.uniform(1.0, 4.0, n)], 1)
    means = pc @ T[:3, :3].T + T[:3, 3]
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y), 2 * (x * y + w * z),
                  1 - 2 * (x * x + z * z), 2 * (y * z - w * x), 2 * (x * z - w * y), 2 * (y * z + w * x),
                  1 - 2 * (x * x + y * y)], 1).reshape(n, 3, 3)
    sd = np.where(rng.uniform(size=(n, 1)) < 0.5, [0.08, 0.0008, 0.0008], [0.03, 0.03, 0.0003])
    S = np.einsum("nij,nj,nkj->nik", R, sd * sd, R)
    g = {"means": means.astype(np.float32),
         "covs": np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1).astype(np.float32),
         "opacity": rng.uniform(0.3, 0.95, n).astype(np.float32), "colors": rng.uniform(0, 1, (n, 3)).astype(np.float32)}
    rgb_o, tr_o, drawn = oracle.splat_render(g["means"], g["covs"], g["opacity"], g["colors"], oracle.pinhole_from(wl), T)
    rgb_g, tr_g, pairs = render_gpu(to_dev(g), mrh().pinhole_from(wl), T)
    assert drawn > n // 2 and pairs > 0
    assert np.abs(rgb_g - rgb_o).max() <= TOL
    assert np.abs(tr_g - tr_o).max() <= TOL


def test_full_size_camera_at_sampled_pixels():
    wl = synth.rgbd()
    g = synth.gaussians(wl, 1_000_000)
    gd = to_dev(g)
    rng = np.random.default_rng(11)
    for frame in (10, 130):
        T = wl.pose(frame)
        rgb_g, tr_g, pairs = render_gpu(gd, mrh().pinhole_from(wl), T)
        assert pairs > 1_000_000
        uv = np.stack([rng.integers(0, wl.width, 300), rng.integers(0, wl.height, 300)], 1)
        uv = np.concatenate([uv, [[0, 0], [wl.width - 1, wl.height - 1], [wl.width - 1, 0], [0, wl.height - 1]]])
        rgb_o, tr_o = oracle.splat_pixels(g["means"], g["covs"], g["opacity"], g["colors"], oracle.pinhole_from(wl), T,
                                          uv)
        assert np.abs(rgb_g[uv[:, 1], uv[:, 0]] - rgb_o).max() <= TOL
        assert np.abs(tr_g[uv[:, 1], uv[:, 0]] - tr_o).max() <= TOL


def test_degenerate_inputs():
    m = mrh()
    wl = small_camera(synth.rgbd(), 48, 40)
    K = m.pinhole_from(wl)
    Ko = oracle.pinhole_from(wl)
    T = np.eye(4)
    z3 = lambda *s: torch.zeros(s, dtype=torch.float32, device="cuda")  # noqa: E731
    # no Gaussians: nothing drawn, full transmittance
    rgb, tr, pairs = m.splat_render(z3(0, 3), z3(0, 6), z3(0), z3(0, 3), K, T)
    assert pairs == 0 and torch.all(rgb == 0) and torch.all(tr == 1)
    # behind the camera, beyond max depth, a zero covariance, a NaN mean: none drawn
    means = np.array([[0, 0, -1.0], [0, 0, wl.max_depth * 2], [0, 0, 2.0], [np.nan, 0, 2.0]], np.float32)
    covs = np.tile(np.array([1e-3, 0, 0, 1e-3, 0, 1e-3], np.float32), (4, 1))
    covs[2] = 0
    g = {"means": means, "covs": covs, "opacity": np.full(4, 0.5, np.float32), "colors": np.ones((4, 3), np.float32)}
    rgb, tr, pairs = render_gpu(to_dev(g), K, T)
    assert pairs == 0 and np.all(rgb == 0) and np.all(tr == 1)
    # one Gaussian covering every tile, a tie in depth (index order decides), an opaque front
    means = np.array([[0, 0, 1.0], [0.05, 0, 1.5], [0.05, 0, 1.5], [-0.1, 0.02, 0.8]], np.float32)
    covs = np.array([[0.5, 0.1, 0, 0.4, 0, 0.2], [1e-3, 0, 0, 1e-3, 0, 1e-3], [2e-3, 0, 0, 1e-3, 0, 1e-3],
                     [4e-4, 1e-4, 0, 3e-4, 0, 1e-4]], np.float32)
    g = {"means": means, "covs": covs, "opacity": np.array([0.3, 0.6, 0.9, 1.0], np.float32),
         "colors": np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float32)}
    rgb_g, tr_g, pairs = render_gpu(to_dev(g), K, T)
    rgb_o, tr_o, _ = oracle.splat_render(g["means"], g["covs"], g["opacity"], g["colors"], Ko, T)
    assert pairs >= 6
    assert np.abs(rgb_g - rgb_o).max() <= TOL and np.abs(tr_g - tr_o).max() <= TOL
    assert tr_o.min() < 0.1  # near the opaque Gaussian's centre
    # transmittance output is optional
    rgb2, tr2, _ = render_gpu(to_dev(g), K, T, trans=False)
    assert tr2 is None and np.array_equal(rgb2, rgb_g)


def test_invalid_arguments_are_rejected():
    m = mrh()
    wl = small_camera(synth.rgbd(), 32, 32)
    g = to_dev(synth.gaussians(synth.rgbd(), 100))
    for field, value in (("min_depth", 0.0), ("width", 0), ("fx", -1.0), ("max_depth", 0.01)):
        K = m.pinhole_from(wl)
        setattr(K, field, value)
        with pytest.raises(m.MrhError):
            m.splat_render(g["means"], g["covs"], g["opacity"], g["colors"], K, np.eye(4))
    with pytest.raises(ValueError):
        m.splat_render(g["means"], g["covs"][:, :3].contiguous(), g["opacity"], g["colors"], m.pinhole_from(wl),
                       np.eye(4))
