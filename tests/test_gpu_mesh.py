"""GPU parity of the multi-resolution Marching Cubes extraction (Sec. 3.4) against the oracle.

Both sides compute every vertex with the same float operations, so the triangle sets are compared exactly after a
canonical order (each triangle rotated to start at its smallest vertex, keeping its winding; triangles sorted).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_21459_b300 import build
    build.build()


def mrh():
    import paper_2511_21459_b300 as m
    return m


def canonical(tris):
    """Triangles (n, 9) rotated to start at their lexicographically smallest vertex (winding kept), sorted."""
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 3, 3)
    best = np.zeros(len(t), np.int64)
    for k in (1, 2):
        a, b = t[:, k], t[np.arange(len(t)), best]
        less = (a[:, 0] < b[:, 0]) | ((a[:, 0] == b[:, 0]) & ((a[:, 1] < b[:, 1]) |
                                                           ((a[:, 1] == b[:, 1]) & (a[:, 2] < b[:, 2]))))
        best = np.where(less, k, best)
    idx = (best[:, None] + np.arange(3)[None, :]) % 3
    flat = t[np.arange(len(t))[:, None], idx].reshape(len(t), 9)
    return flat[np.lexsort(flat.T[::-1])]


def same_mesh(g, o):
    a, b = canonical(g), canonical(o)
    assert a.shape == b.shape, (a.shape, b.shape)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def run_camera(wl, frames, **kw):
    m = mrh()
    g = m.Map(m.params_from(wl, **kw))
    o = oracle.OracleMap(oracle.params_from(wl, "f32s", **kw))
    K_g, K_o = m.pinhole_from(wl), oracle.pinhole_from(wl)
    for depth, rgb, T in frames:
        g.integrate_depth(K_g, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        o.integrate_depth(K_o, T, depth, rgb)
    return g, o


def test_tiny_frame_mesh_matches_oracle():
    wl = synth.tiny()
    g, o = run_camera(wl, [synth.render_depth(wl, 0)])
    tg = g.extract_mesh().cpu().numpy()
    assert len(tg) > 10000
    same_mesh(tg, o.extract_mesh())


def test_relevelled_views_mesh_matches_oracle():
    """Ten noisy views from one pose: blocks merge to level 1 next to level-0 blocks, so the seams between levels are
    meshed on both sides."""
    wl = synth.tiny()
    g, o = run_camera(wl, [synth.render_depth(wl, 0, seed=s) for s in range(10)])
    assert (o.block_stats()["levels"] == 1).sum() > 100
    same_mesh(g.extract_mesh().cpu().numpy(), o.extract_mesh())


def test_fp16_storage_mesh_matches_oracle():
    wl = synth.tiny()
    wl.fp16 = True
    g, o = run_camera(wl, [synth.render_depth(wl, 0, seed=s) for s in range(6)])
    same_mesh(g.extract_mesh().cpu().numpy(), o.extract_mesh())


def test_rgbd_sequence_prefix_mesh_matches_oracle():
    """Full-size frames of the RGB-D sequence, every 10th pose, with thresholds that make blocks of all three
    levels: the mesh of the whole map."""
    wl = synth.rgbd()
    scene = wl.scene()
    frames = [synth.render_depth(wl, k, scene=scene) for k in range(0, 60, 10)]
    wl.var_threshold = (1e-4, 4e-4)
    g, o = run_camera(wl, frames)
    lv = o.block_stats()["levels"]
    assert (lv == 1).sum() > 0 and (lv == 2).sum() > 0
    tg = g.extract_mesh().cpu().numpy()
    assert len(tg) > 200000
    same_mesh(tg, o.extract_mesh())


def test_lidar_map_mesh_matches_oracle():
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 64, 512
    wl.min_obs = 2
    m = mrh()
    g = m.Map(m.params_from(wl))
    o = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    scene = wl.scene()
    for f in range(3):
        xyz, T = synth.render_lidar(wl, f, scene=scene)
        g.integrate_points(T, torch.from_numpy(xyz).cuda())
        o.integrate_points(T, xyz)
    same_mesh(g.extract_mesh().cpu().numpy(), o.extract_mesh())


def test_capacity_error_reports_the_count_and_empty_map_has_no_triangles():
    m = mrh()
    wl = synth.tiny()
    g, _ = run_camera(wl, [synth.render_depth(wl, 0)])
    n = len(g.extract_mesh())
    with pytest.raises(m.MrhError) as e:
        g.extract_mesh(capacity=n - 1)
    assert e.value.code == 7
    e2 = m.Map(m.params_from(wl))
    assert len(e2.extract_mesh()) == 0


def test_vertex_collapse_matches_oracle():
    """The GPU collapse of the GPU soup equals the oracle's collapse of the oracle soup: the same vertices in the same
    (cell) order, and the same faces once each is rotated to its smallest index and the list sorted (the soups'
    triangle orders differ)."""
    wl = synth.tiny()
    g, o = run_camera(wl, [synth.render_depth(wl, 0, seed=s) for s in range(10)])
    delta = 0.01 / 8
    vg, fg = g.weld_mesh(g.extract_mesh(), delta)
    vo, fo = oracle.weld_mesh(o.extract_mesh(), delta)
    vg, fg = vg.cpu().numpy(), fg.cpu().numpy()
    assert len(vo) > 5000 and len(fo) > 10000
    assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32))

    def canon(f):
        r = np.argmin(f, axis=1)
        f = f[np.arange(len(f))[:, None], (r[:, None] + np.arange(3)[None, :]) % 3]
        return f[np.lexsort(f.T[::-1])]
    assert np.array_equal(canon(fg), canon(fo))
    # fewer vertices than the soup has corners, and triangles dropped only where they collapsed
    assert len(vg) < 3 * len(fg)
