"""GPU parity of the contrast quadtree (Sec. 3.5, Eq. 10, Algorithm 1) against the oracle: the same leaves (sets of
(x, y, w, h)), exactly, since both take every split decision from the same exact integer sums."""
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


def leaves_gpu(img, thr, min_size=1):
    out = mrh().quadtree(torch.from_numpy(np.ascontiguousarray(img)).cuda(), thr, min_size).cpu().numpy()
    return out[np.lexsort(out.T[::-1])]


def leaves_oracle(img, thr, min_size=1):
    out = oracle.quadtree(img, thr, min_size)
    return out[np.lexsort(out.T[::-1])]


@pytest.mark.parametrize("frame", [0, 57, 211])
def test_rgbd_frames_match_oracle(frame):
    wl = synth.rgbd()
    _, rgb, _ = synth.render_depth(wl, frame)
    g, o = leaves_gpu(rgb, 0.1), leaves_oracle(rgb, 0.1)
    assert len(o) > 10000
    np.testing.assert_array_equal(g, o)


@pytest.mark.parametrize("w,h,thr,min_size", [(13, 7, -1.0, 1), (1, 1, 0.0, 1), (64, 48, 1e9, 1), (97, 61, 500.0, 1),
                                              (128, 96, 50.0, 3), (1280, 720, 20.0, 1)])
def test_random_images_match_oracle(w, h, thr, min_size):
    rng = np.random.default_rng(w * 1000 + h)
    # blocky noise: constant 8 x 8 tiles with some noisy ones, so that the tree has both deep and shallow leaves
    base = rng.integers(0, 256, ((h + 7) // 8, (w + 7) // 8, 3), dtype=np.uint8).repeat(8, 0).repeat(8, 1)[:h, :w]
    noisy = rng.random((h, w)) < 0.02
    img = base.copy()
    img[noisy] = rng.integers(0, 256, (noisy.sum(), 3), dtype=np.uint8)
    np.testing.assert_array_equal(leaves_gpu(img, thr, min_size), leaves_oracle(img, thr, min_size))


def test_leaves_tile_a_full_hd_frame():
    wl = synth.rgbd()
    _, rgb, _ = synth.render_depth(wl, 3)
    big = np.ascontiguousarray(np.repeat(np.repeat(rgb, 2, 0), 2, 1)[:720, :1280])
    lv = leaves_gpu(big, 0.1)
    cover = np.zeros(big.shape[:2], np.int32)
    for x, y, w, h in lv:
        cover[y:y + h, x:x + w] += 1
    assert np.all(cover == 1)
