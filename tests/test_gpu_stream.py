"""GPU parity of capacity-driven streaming (Sec. 3.3): after every frame the resident blocks (keys, levels, payload)
and the per-frame eviction and restore counts equal the oracle's. Pools are sized so that the peak resident count
fits while the fraction is crossed: camera frames go to the opposite side of the orbit and back (blocks leave and
return), LiDAR scans advance along the street (blocks beyond the radius leave, some come back)."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare_extracts

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


KEYS = ("valid_rays", "touched", "new_blocks", "merged", "split", "evicted", "restored")


def test_camera_streaming_matches_oracle():
    wl = synth.rgbd()
    wl.max_blocks = (14000, 2000, 4000)
    sc = wl.scene()
    g = mrh().Map(mrh().params_from(wl))
    o = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    g.set_streaming(0.85, 0.0, 40000)
    o.set_streaming(0.85, 0.0, wl.max_blocks)
    Kg, Ko = mrh().pinhole_from(wl), oracle.pinhole_from(wl)
    ev = rs = 0
    for k in (0, 2, 4, 150, 152, 2, 4):
        d, c, T = synth.render_depth(wl, k, scene=sc)
        g.integrate_depth(Kg, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        so = o.integrate_depth(Ko, T, d, c)
        sg = g.stats()
        assert sg["status_code"] == 0, sg
        for key in KEYS:
            assert sg[key] == so[key], (k, key, sg[key], so[key])
        assert sg["archived"] == o.archived()
        ev += so["evicted"]
        rs += so["restored"]
        compare_extracts(g.extract(), o.extract(), wl.truncation, wl.var_threshold[0], check_color=True)
    assert ev > 10000 and rs > 5000


def test_lidar_streaming_matches_oracle():
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    wl.max_blocks = (40000, 3000, 3000)
    sc = wl.scene()
    g = mrh().Map(mrh().params_from(wl))
    o = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    g.set_streaming(0.5, 25.0, 60000)
    o.set_streaming(0.5, 25.0, wl.max_blocks)
    ev = rs = 0
    for f in range(0, 24, 3):
        xyz, T = synth.render_lidar(wl, f, scene=sc)
        g.integrate_points(T, torch.from_numpy(xyz).cuda())
        so = o.integrate_points(T, xyz)
        sg = g.stats()
        assert sg["status_code"] == 0, sg
        for key in KEYS:
            assert sg[key] == so[key], (f, key, sg[key], so[key])
        ev += so["evicted"]
        rs += so["restored"]
    compare_extracts(g.extract(), o.extract(), wl.truncation, wl.var_threshold[0], check_color=False)
    assert ev > 10000 and rs > 5000


def test_streaming_arguments_and_exclusions():
    m = mrh()
    wl = synth.tiny()
    g = m.Map(m.params_from(wl))
    for bad in ((1.5, 0.0, 100), (-0.1, 0.0, 100), (0.5, -1.0, 100), (0.5, 0.0, 0)):
        with pytest.raises(m.MrhError):
            g.set_streaming(*bad)
    g.set_streaming(0.8, 0.0, 1000)
    with pytest.raises(m.MrhError):
        g.set_feature_capture(100)
    with pytest.raises(m.MrhError):
        m.Batch([g], [m.pinhole_from(wl)])
