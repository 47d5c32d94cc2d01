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
