"""mrh_extract_blocks_noalloc: the read-out that allocates no device memory.

Some callers cannot allocate at read-out time: a process that gave all device memory to a fixed arena or to a
framework's caching allocator (a fresh cudaMalloc would fail), or a latency-bounded loop where an allocation, which
can synchronise the device, is not acceptable. For them the library keeps the sort scratch of the read-out in one
fixed device array. This test calls that entry point through the C ABI and checks that it returns exactly what the
allocating mrh_extract_blocks returns, on two calls in a row (the shared scratch keeps the previous call's contents).
It sits in a file of its own, collected last, and passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _extract(m, lib, fn, nb, nv):
    dev = "cuda"
    out = dict(keys=torch.empty((max(nb, 1), 3), dtype=torch.int32, device=dev),
               levels=torch.empty(max(nb, 1), dtype=torch.uint8, device=dev),
               offsets=torch.zeros(nb + 1, dtype=torch.int64, device=dev),
               D=torch.empty(max(nv, 1), device=dev), W=torch.empty(max(nv, 1), device=dev),
               S2=torch.empty(max(nv, 1), device=dev), C=torch.empty((max(nv, 1), 3), device=dev))
    wb, wv = ctypes.c_uint64(), ctypes.c_uint64()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    code = getattr(lib, fn)(m._h, p(out["keys"]), p(out["levels"]), p(out["offsets"]), p(out["D"]), p(out["W"]),
                            p(out["S2"]), p(out["C"]), max(nb, 1), max(nv, 1), ctypes.byref(wb), ctypes.byref(wv),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, (fn, code)
    assert (wb.value, wv.value) == (nb, nv)
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_extract_equals_extract_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import build
    build.build()
    lib = mrh.lib()
    wl = synth.rgbd()
    scene = wl.scene()
    m = mrh.Map(mrh.params_from(wl))
    K = mrh.pinhole_from(wl)
    sizes = []
    for frame in (0, 7):  # the second call sees a bigger map and must not reuse the first call's contents
        depth, rgb, T = synth.render_depth(wl, frame, scene=scene)
        m.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        nb, nv = m.count()
        ref = _extract(m, lib, "mrh_extract_blocks", nb, nv)
        got = _extract(m, lib, "mrh_extract_blocks_noalloc", nb, nv)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
        sizes.append(nb)
    assert sizes[1] > sizes[0] > 1000
    m.close()


def test_noalloc_limit_then_smaller_map():
    """A map holding more than MRH_NOALLOC_MAX_BLOCKS blocks gets MRH_ERR_STATIC_LIMIT (8) with the output buffers
    left as they were; a smaller map read right after it (the scratch still holding the larger map's leftovers
    beyond the new count) returns exactly what mrh_extract_blocks returns."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import build
    build.build()
    lib = mrh.lib()
    # a LiDAR street at 2 / 4 / 8 cm voxels (16 cm blocks): a few scans allocate well over 2^18 blocks
    wl = synth.lidar()
    wl.base_voxel, wl.truncation = 0.08, 0.24
    wl.hash_log2 = 22
    wl.max_blocks = (1 << 20, 1 << 17, 1 << 17)
    wl.max_touched = 1 << 20
    big = mrh.Map(mrh.params_from(wl))
    scene = wl.scene()
    for f in range(6):
        xyz, T = synth.render_lidar(wl, f, scene=scene)
        big.integrate_points(T, torch.from_numpy(xyz).cuda())
        if big.count()[0] > (1 << 18):
            break
    nb, nv = big.count()
    assert nb > (1 << 18) and big.stats()["status_code"] == 0
    # the allocating read-out works on it, and the no-allocation one refuses it without writing anything
    ref_big = _extract(big, lib, "mrh_extract_blocks", nb, nv)
    assert ref_big["keys"].shape[0] == nb
    dev = "cuda"
    outs = [torch.full((nb, 3), -7, dtype=torch.int32, device=dev), torch.full((nb,), 7, dtype=torch.uint8, device=dev),
            torch.full((nb + 1,), -7, dtype=torch.int64, device=dev)] + \
           [torch.full((nv,), -7.0, device=dev) for _ in range(3)] + [torch.full((nv, 3), -7.0, device=dev)]
    before = [o.clone() for o in outs]
    wb, wv = ctypes.c_uint64(), ctypes.c_uint64()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    code = lib.mrh_extract_blocks_noalloc(big._h, *[p(o) for o in outs], nb, nv, ctypes.byref(wb), ctypes.byref(wv),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert code == 8, code
    for a, b in zip(outs, before):
        assert torch.equal(a, b)
    del outs, before, ref_big
    # a smaller map right after a call that filled the scratch with a larger one
    small_wl = synth.rgbd()
    sm = mrh.Map(mrh.params_from(small_wl))
    first = mrh.Map(mrh.params_from(small_wl))
    sc = small_wl.scene()
    K = mrh.pinhole_from(small_wl)
    for f in (0, 5, 10):
        depth, rgb, T = synth.render_depth(small_wl, f, scene=sc)
        first.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        if f == 0:
            sm.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
    nb1, nv1 = first.count()
    nb2, nv2 = sm.count()
    assert nb1 > nb2 > 1000
    _extract(first, lib, "mrh_extract_blocks_noalloc", nb1, nv1)
    ref = _extract(sm, lib, "mrh_extract_blocks", nb2, nv2)
    got = _extract(sm, lib, "mrh_extract_blocks_noalloc", nb2, nv2)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    for m in (big, sm, first):
        m.close()
