"""Batched multi-scene integration (mrh_batch_*): maps with uneven frame sizes integrated together must end up
bitwise identical to the same frames integrated one map at a time (which the oracle parity tests cover), through the
warm-up step, the autotune trial steps (alternative launch shapes) and CUDA-graph replays; raycasts likewise."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _workloads(n):
    wls = synth.batched(n_maps=n, n_frames=100)
    for wl in wls:
        wl.max_blocks = (1 << 16, 1 << 15, 1 << 15)  # keep the test's memory modest
    return wls


def test_batched_equals_per_map_bitwise():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import build
    build.build()
    wls = _workloads(5)
    scenes = [wl.scene() for wl in wls]
    steps = 9  # 1 plain + 4 autotune trials + graph capture + replays
    frames = [[synth.render_depth(wl, 4 * k, scene=sc) for k in range(steps)] for wl, sc in zip(wls, scenes)]
    cams = [mrh.pinhole_from(wl) for wl in wls]
    single = [mrh.Map(mrh.params_from(wl)) for wl in wls]
    batched = [mrh.Map(mrh.params_from(wl)) for wl in wls]
    batch = mrh.Batch(batched, cams)
    stream = torch.cuda.Stream()
    for k in range(steps):
        outs_s, outs_b, fr = [], [], []
        for i, wl in enumerate(wls):
            d, c, T = frames[i][k]
            dt, ct = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
            single[i].integrate_depth(cams[i], T, dt, ct)
            outs_s.append(single[i].raycast(cams[i], T))
            ob = torch.zeros((wl.height, wl.width), device="cuda")
            outs_b.append(ob)
            fr.append((T, dt, ct, ob))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            batch.integrate(fr, stream=stream)
        stream.synchronize()
        for i in range(len(wls)):
            assert single[i].stats()["status_code"] == 0 and batched[i].stats()["status_code"] == 0
            sb, ss = batched[i].stats(), single[i].stats()
            for key in ("touched", "new_blocks", "merged", "split", "valid_rays", "observations"):
                assert sb[key] == ss[key], (k, i, key)
            torch.testing.assert_close(outs_b[i], outs_s[i], rtol=0, atol=0)
    cfg = batch.config()
    assert cfg["tuned"] and cfg["graph"], cfg
    for i in range(len(wls)):
        a = {k: v.cpu().numpy() for k, v in single[i].extract().items()}
        b = {k: v.cpu().numpy() for k, v in batched[i].extract().items()}
        for key in a:
            np.testing.assert_array_equal(a[key], b[key], err_msg=f"map {i} field {key}")
    batch.close()


def test_batched_maps_match_the_oracle():
    """Three maps of uneven frame sizes (320x240, 848x480, 1280x720; FP16 storage with colour) integrated through the
    batched path (plain step, autotune trials, CUDA-graph capture and replays) against oracle maps in float mode with
    half storage fed the same frames: per-frame counters equal, and after the last step keys, levels and weights
    identical, D, sigma^2 and colour within 1e-4 relative, the batched raycast within the bounds of the raycast
    check."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import build
    from tests.parity import compare_extracts
    from tests.raycast_check import check_raycast, grid_step
    build.build()
    all_wls = synth.batched(n_maps=16, n_frames=100)
    pick = {}
    for wl in all_wls:
        pick.setdefault((wl.width, wl.height), wl)
    wls = [pick[s] for s in ((320, 240), (848, 480), (1280, 720))]
    for wl in wls:
        wl.max_blocks = (1 << 16, 1 << 15, 1 << 15)
    scenes = [wl.scene() for wl in wls]
    cams = [mrh.pinhole_from(wl) for wl in wls]
    gmaps = [mrh.Map(mrh.params_from(wl)) for wl in wls]
    omaps = [oracle.OracleMap(oracle.params_from(wl, "f32s")) for wl in wls]
    batch = mrh.Batch(gmaps, cams)
    stream = torch.cuda.Stream()
    steps = 8
    for k in range(steps):
        fr, outs = [], []
        for i, wl in enumerate(wls):
            d, c, T = synth.render_depth(wl, 4 * k, scene=scenes[i])
            ob = torch.zeros((wl.height, wl.width), device="cuda")
            outs.append(ob)
            fr.append((T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), ob))
            st_o = omaps[i].integrate_depth(oracle.pinhole_from(wl), T, d, c)
            fr[-1] = fr[-1] + (st_o,)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            batch.integrate([f[:4] for f in fr], stream=stream)
        stream.synchronize()
        for i in range(len(wls)):
            st_g, st_o = gmaps[i].stats(), fr[i][4]
            assert st_g["status_code"] == 0, st_g
            for key in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations", "updated_voxels"):
                assert st_g[key] == st_o[key], (k, i, key, st_g[key], st_o[key])
    assert batch.config()["graph"]
    for i, wl in enumerate(wls):
        compare_extracts(gmaps[i].extract(), omaps[i].extract(), wl.truncation, wl.var_threshold[0])
        T = fr[i][0]
        rc_o = omaps[i].raycast(oracle.pinhole_from(wl), T)
        check_raycast(outs[i].cpu().numpy(), rc_o, grid_step(wl))
    batch.close()
