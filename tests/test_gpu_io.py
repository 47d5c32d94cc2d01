"""GPU map save / load (the persistence half of streaming, Sec. 3.3): a loaded map holds exactly the saved blocks
(keys, levels, payload bit for bit), raycasts the same depth, and keeps fusing like the map it was saved from; a
streaming map's file holds its resident and archived blocks, which together equal the oracle's map that never
streamed. FP32 storage with colour (RGB-D) and FP16 storage (LiDAR) both round-trip."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare_extracts, to_numpy

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


def same_blocks(a, b):
    a, b = to_numpy(a), to_numpy(b)
    assert set(a) == set(b)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_rgbd_round_trip_and_continued_fusion(tmp_path):
    m = mrh()
    wl = synth.rgbd()
    sc = wl.scene()
    K = m.pinhole_from(wl)
    g = m.Map(m.params_from(wl))
    frames = [synth.render_depth(wl, k, scene=sc) for k in (0, 3, 6, 9, 12)]
    for d, c, T in frames[:3]:
        g.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
    path = str(tmp_path / "rgbd.mrhmap")
    g.save(path)
    h = m.Map.load(path)
    assert bytes(h.params) == bytes(g.params)
    assert h.count() == g.count()
    same_blocks(h.extract(), g.extract())
    T = frames[2][2]
    for x, y in zip(g.raycast(K, T, normals=True, rgb=True), h.raycast(K, T, normals=True, rgb=True)):
        assert torch.equal(x, y)
    for d, c, T in frames[3:]:
        for mp in (g, h):
            mp.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        sg, sh = g.stats(), h.stats()
        for key in ("touched", "new_blocks", "merged", "split", "live_blocks"):
            assert sg[key] == sh[key], key
    same_blocks(h.extract(), g.extract())


def test_lidar_fp16_round_trip(tmp_path):
    m = mrh()
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    sc = wl.scene()
    g = m.Map(m.params_from(wl, storage=m.MRH_STORAGE_FP16))
    for f in (0, 2, 4):
        xyz, T = synth.render_lidar(wl, f, scene=sc)
        g.integrate_points(T, torch.from_numpy(xyz).cuda())
    path = str(tmp_path / "lidar.mrhmap")
    g.save(path)
    h = m.Map.load(path)
    same_blocks(h.extract(), g.extract())


def test_streaming_map_file_equals_the_map_that_never_streamed(tmp_path):
    m = mrh()
    wl = synth.rgbd()
    wl.max_blocks = (14000, 2000, 4000)
    sc = wl.scene()
    g = m.Map(m.params_from(wl))
    g.set_streaming(0.85, 0.0, 40000)
    ctl = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    Kg, Ko = m.pinhole_from(wl), oracle.pinhole_from(wl)
    for k in (0, 2, 4, 150, 152):
        d, c, T = synth.render_depth(wl, k, scene=sc)
        g.integrate_depth(Kg, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        ctl.integrate_depth(Ko, T, d, c)
    st = g.stats()
    assert st["status_code"] == 0 and st["archived"] > 5000
    path = str(tmp_path / "stream.mrhmap")
    g.save(path)
    # the saved capacities cannot hold the union: load it into a map with larger pools
    raw = bytearray(open(path, "rb").read())
    p = m.Params.from_buffer_copy(raw[16:16 + len(bytes(g.params))])
    p.max_blocks[0], p.max_blocks[1], p.max_blocks[2] = 400000, 100000, 100000
    raw[16:16 + len(bytes(p))] = bytes(p)
    big = str(tmp_path / "stream_big.mrhmap")
    open(big, "wb").write(bytes(raw))
    with pytest.raises(m.MrhError):
        m.Map.load(path)
    h = m.Map.load(big)
    assert h.count()[0] == g.count()[0] + st["archived"]
    compare_extracts(h.extract(), ctl.extract(), wl.truncation, wl.var_threshold[0], check_color=True)


def test_malformed_files_are_rejected(tmp_path):
    m = mrh()
    wl = synth.tiny()
    g = m.Map(m.params_from(wl))
    path = str(tmp_path / "empty.mrhmap")
    g.save(path)
    h = m.Map.load(path)
    assert h.count()[0] == 0
    raw = open(path, "rb").read()
    for bad in (raw[:-1], raw[:8], b"XXXXXXXX" + raw[8:], raw[:8] + b"\x02" + raw[9:]):
        p = str(tmp_path / "bad.mrhmap")
        open(p, "wb").write(bad)
        with pytest.raises(m.MrhError):
            m.Map.load(p)
