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
