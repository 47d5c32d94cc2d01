"""GPU tests of the learned level predictor (an addition to the paper's method) through the C ABI.

- Inference kernel: logits bit-exact with the float oracle (same sums in the same order, BF16 products exact).
- Training kernels: the loss and gradient against the float64 oracle (oracle/mlp.py, itself pinned to central
  differences); the first Adam step against its closed form; the BF16 copy equals the rounded master weights.
- In the map: with a predictor set, new blocks start at the predicted level; keys, levels, weights and the per-frame
  counters are bit-exact with the oracle map running the same predictor, fields within the parity tolerance, and the
  captured features are bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp
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


def _init(seed, noise=0.05):
    from paper_2511_21459_b300 import predictor
    w = predictor.init_weights(seed)
    return (w + noise * np.random.default_rng(seed + 100).standard_normal(w.size)).astype(np.float32)


# ---------------------------------------------------------------------------------------------- network kernels

def test_predict_bit_exact_with_oracle():
    net = mrh().Mlp(_init(1))
    _, wbf = net.weights()
    x = (np.random.default_rng(2).standard_normal((1000, 16)) * 1.5).astype(np.float32)  # 1000: ragged last CTA
    got = net.predict(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.mlp_forward(wbf, x)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_bf16_copy_is_rounded_master():
    w = _init(3)
    net = mrh().Mlp(w)
    master, wbf = net.weights()
    np.testing.assert_array_equal(master, w)
    np.testing.assert_array_equal(wbf, mlp.bf16_bits(w.astype(np.float64)))


@pytest.mark.parametrize("n", [1, 31, 777, 4096, 100_000])
def test_loss_and_gradient_match_float64_oracle(n):
    """The tensor-core gradient against float64. Forward products are exact BF16 products summed in FP32; in the
    backward products the FP32 gradient factor is split into a BF16 part and a BF16 remainder (16 of its 24 mantissa
    bits, relative error below 2^-16 = 1.5e-5 per term); the sums and the atomic accumulation add errors of order
    1e-6; a rare flip of one BF16 activation rounding moves one sample's share by about 2^-8. Tolerance: 1e-4 of the
    largest gradient entry. 100 000 samples make every CTA loop over several tiles."""
    net = mrh().Mlp(_init(4))
    _, wbf = net.weights()
    rng = np.random.default_rng(5 + n)
    x = (rng.standard_normal((n, 16)) * 1.5).astype(np.float32)
    y = rng.integers(0, 3, n).astype(np.int32)
    loss, grad = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    L_ref, g_ref = mlp.loss_and_grad(mlp.from_bf16_bits(wbf), mlp.bf16_round(x), y, act_round=True)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_labels_outside_range_contribute_nothing():
    """A label outside [0, 3) adds no loss and no gradient; the mean still divides by the batch size."""
    net = mrh().Mlp(_init(6))
    _, wbf = net.weights()
    rng = np.random.default_rng(7)
    x = rng.standard_normal((300, 16)).astype(np.float32)
    y = rng.integers(0, 3, 300).astype(np.int32)
    y[::3] = 3
    y[1::7] = -1
    ok = (y >= 0) & (y < 3)
    loss, grad = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    L_ref, g_ref = mlp.loss_and_grad(mlp.from_bf16_bits(wbf), mlp.bf16_round(x[ok]), y[ok], act_round=True)
    frac = ok.sum() / len(y)
    assert abs(float(loss.item()) - frac * L_ref) <= 1e-5
    assert np.max(np.abs(grad.cpu().numpy() - frac * g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_first_adam_step_closed_form():
    w = _init(8)
    net = mrh().Mlp(w)
    _, wbf = net.weights()
    rng = np.random.default_rng(9)
    x = rng.standard_normal((512, 16)).astype(np.float32)
    y = rng.integers(0, 3, 512).astype(np.int32)
    lr = 1e-3
    loss = torch.zeros(1, device="cuda")
    net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), lr, loss)
    master, wbf1 = net.weights()
    L_ref, g = mlp.loss_and_grad(mlp.from_bf16_bits(wbf), mlp.bf16_round(x), y, act_round=True)
    assert abs(float(loss.item()) - L_ref) <= 1e-5 * max(1.0, L_ref)
    step = master.astype(np.float64) - w
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    expect = -lr * g / (np.abs(g) + 1e-8)
    assert np.all(np.abs(step[big] - expect[big]) <= 1e-3 * lr + 2.0 ** -23 * np.abs(w[big]))
    assert np.all(np.abs(step) <= lr * (1 + 1e-5) + 2.0 ** -23 * np.abs(w))
    np.testing.assert_array_equal(wbf1, mlp.bf16_bits(master.astype(np.float64)))


def test_training_learns_a_teacher():
    """Labels from a fixed random teacher network of the same shape: GPU training reaches low error."""
    from paper_2511_21459_b300 import predictor
    rng = np.random.default_rng(10)
    teacher = mlp.bf16_bits(mlp.init_params(11, scale=1.0))
    x = rng.uniform(-1, 1, (20000, 16)).astype(np.float32)
    y = np.argmax(oracle.mlp_forward(teacher, x), axis=1).astype(np.int32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net, hist = predictor.train(xt, yt, epochs=40, batch=1024, lr=3e-3, seed=0)
    assert hist[-1] < 0.5 * hist[0]
    err = float((predictor.predicted_levels(net, xt) != yt).float().mean().item())
    assert err < 0.1, err


# ---------------------------------------------------------------------------------------------- in the map

def _run_both(wl, frames, w_bf16, capture=True, **kw):
    m = mrh()
    gmap = m.Map(m.params_from(wl, **kw))
    omap = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    if w_bf16 is not None:
        gmap.set_predictor(w_bf16)
        omap.set_predictor(w_bf16)
    if capture:
        gmap.set_feature_capture(1 << 20)
        omap.set_capture(True)
    K_g, K_o = m.pinhole_from(wl), oracle.pinhole_from(wl)
    for f, (depth, rgb, T) in enumerate(frames):
        gmap.integrate_depth(K_g, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        st_o = omap.integrate_depth(K_o, T, depth, rgb)
        st_g = gmap.stats()
        assert st_g["status_code"] == 0, st_g
        for k in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations"):
            assert st_g[k] == st_o[k], (f, k, st_g[k], st_o[k])
    compare_extracts(gmap.extract(), omap.extract(), wl.truncation, wl.var_threshold[0], check_color=wl.has_color)
    return gmap, omap


def _compare_features(gmap, omap):
    keys, feats, seen = gmap.features()
    keys, feats = keys.cpu().numpy(), feats.cpu().numpy()
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    ok, of = omap.features()
    assert seen == len(keys) == len(ok)
    np.testing.assert_array_equal(keys[order], ok)
    np.testing.assert_array_equal(feats[order].view(np.uint32), of.view(np.uint32))
    return len(keys)


def _spread_weights(seed):
    """Random weights whose argmax spreads over the three levels on real features."""
    w = mlp.init_params(seed, scale=1.0)
    w[-3:] = [0.0, 0.3, 0.6]
    return mlp.bf16_bits(w)


def test_learned_allocation_parity_tiny():
    wl = synth.tiny()
    frames = [synth.render_depth(wl, f) for f in range(5)]
    gmap, omap = _run_both(wl, frames, _spread_weights(12))
    n = _compare_features(gmap, omap)
    assert n > 100
    levels = omap.extract()["levels"]
    assert len(np.unique(levels)) == 2  # both levels occur


def test_learned_allocation_parity_rgbd_full_frames():
    wl = synth.rgbd()
    frames = [synth.render_depth(wl, f) for f in range(3)]
    gmap, omap = _run_both(wl, frames, _spread_weights(13))
    _compare_features(gmap, omap)
    counts = np.bincount(omap.extract()["levels"], minlength=3)
    assert np.all(counts > 0), counts


def test_learned_allocation_parity_fp16_storage():
    wl = synth.rgbd(fp16=True)
    frames = [synth.render_depth(wl, f) for f in range(2)]
    m = mrh()
    gmap = m.Map(m.params_from(wl))
    omap = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    w = _spread_weights(14)
    gmap.set_predictor(w)
    omap.set_predictor(w)
    K_g, K_o = m.pinhole_from(wl), oracle.pinhole_from(wl)
    for depth, rgb, T in frames:
        gmap.integrate_depth(K_g, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        omap.integrate_depth(K_o, T, depth, rgb)
    compare_extracts(gmap.extract(), omap.extract(), wl.truncation, wl.var_threshold[0], check_color=wl.has_color)


def test_feature_capture_plain_rule_parity():
    """Capture without a predictor (the training-data path): the plain rule's map and the recorded features."""
    wl = synth.rgbd()
    frames = [synth.render_depth(wl, f) for f in range(2)]
    gmap, omap = _run_both(wl, frames, None)
    assert _compare_features(gmap, omap) > 1000
    assert np.all(omap.extract()["levels"] == 0)


def _run_both_lidar(wl, n_scans, w_bf16, capture=True):
    m = mrh()
    gmap = m.Map(m.params_from(wl))
    omap = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    if w_bf16 is not None:
        gmap.set_predictor(w_bf16)
        omap.set_predictor(w_bf16)
    if capture:
        gmap.set_feature_capture(1 << 21)
        omap.set_capture(True)
    sc = wl.scene()
    for f in range(n_scans):
        xyz, T = synth.render_lidar(wl, f, scene=sc)
        gmap.integrate_points(T, torch.from_numpy(xyz).cuda())
        st_o = omap.integrate_points(T, xyz)
        st_g = gmap.stats()
        assert st_g["status_code"] == 0, st_g
        for k in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations", "updated_voxels"):
            assert st_g[k] == st_o[k], (f, k, st_g[k], st_o[k])
    compare_extracts(gmap.extract(), omap.extract(), wl.truncation, wl.var_threshold[0], check_color=False)
    return gmap, omap


def test_learned_allocation_parity_lidar_small_scans():
    """LiDAR scans with a predictor: the end-point moments, the features, the levels of the new blocks and the whole
    map against the oracle (four 32 x 256 scans, FP16 storage, merges at two observations)."""
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    wl.min_obs = 2
    gmap, omap = _run_both_lidar(wl, 4, _spread_weights(12))
    assert _compare_features(gmap, omap) > 10000
    counts = np.bincount(omap.extract()["levels"], minlength=3)
    assert np.all(counts > 0), counts


def test_learned_allocation_parity_lidar_full_scans():
    """Two full 128 x 2048 scans of the benchmark's LiDAR configuration with a predictor."""
    wl = synth.lidar()
    gmap, omap = _run_both_lidar(wl, 2, _spread_weights(12))
    assert _compare_features(gmap, omap) > 50000


def test_feature_capture_plain_rule_parity_lidar():
    """LiDAR capture without a predictor (the training-data path): the plain rule's map and the recorded
    features."""
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 64, 512
    gmap, omap = _run_both_lidar(wl, 3, None)
    assert _compare_features(gmap, omap) > 10000


def test_capture_capacity_and_reset():
    wl = synth.tiny()
    m = mrh()
    gmap = m.Map(m.params_from(wl))
    gmap.set_feature_capture(10)
    depth, rgb, T = synth.render_depth(wl, 0)
    gmap.integrate_depth(m.pinhole_from(wl), T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
    keys, feats, seen = gmap.features(reset=True)
    assert keys.shape == (10, 3) and feats.shape == (10, 16) and seen > 10
    keys, feats, seen = gmap.features()
    assert keys.shape[0] == 0 and seen == 0
    gmap.set_feature_capture(0)
    with pytest.raises(m.MrhError):
        gmap.features()


def test_predictor_argument_errors():
    wl = synth.tiny()
    m = mrh()
    gmap = m.Map(m.params_from(wl))
    with pytest.raises(m.MrhError):
        gmap.set_predictor(np.zeros(100, np.uint16))
    bad = np.zeros(m.MLP_PARAMS, np.uint16)
    bad[7] = 0x7F80  # +inf
    with pytest.raises(m.MrhError):
        gmap.set_predictor(bad)
    gmap.set_predictor(np.zeros(m.MLP_PARAMS, np.uint16))
    gmap.set_predictor(None)
    with pytest.raises(m.MrhError):
        m.Mlp(np.full(m.MLP_PARAMS, np.nan, np.float32))


# ---------------------------------------------------------------------------------------------- what it gains

def test_trained_predictor_gain():
    """Train on the plain rule's final levels of one seeded RGB-D scene, run a different scene with and without the
    predictor: blocks predicted coarse are never fused at the fine level, so the fine-level block updates and the
    fused voxel observations drop, while the map stays within 1 mm of the plain rule's Chamfer error (Sec. 4.1.2) and
    the predictor's misclassification against the plain rule's own final levels stays low."""
    import dataclasses
    from paper_2511_21459_b300 import metrics, predictor
    m_ = mrh()
    n_frames = 100

    def frames(wl):
        sc = wl.scene()
        return [synth.render_depth(wl, k, scene=sc) for k in range(n_frames)]

    def run(wl, frs, w=None, capture=False):
        gmap = m_.Map(m_.params_from(wl))
        if w is not None:
            gmap.set_predictor(w)
        if capture:
            gmap.set_feature_capture(1 << 20)
        K = m_.pinhole_from(wl)
        obs, fine = 0, 0
        for d, c, T in frs:
            gmap.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
            st = gmap.stats()
            assert st["status_code"] == 0
            obs += st["observations"]
            fine += st["touched_level"][0]
        return gmap, obs, fine

    def labelled(gmap):
        keys, feats, _ = gmap.features()
        ex = gmap.extract()
        y = predictor.level_labels(keys.cpu().numpy(), ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy())
        ok = y >= 0
        return feats[torch.from_numpy(ok).cuda()].contiguous(), torch.from_numpy(y[ok]).cuda()

    train_wl = synth.rgbd(seed=11)
    x, y = labelled(run(train_wl, frames(train_wl), capture=True)[0])
    net, hist = predictor.train(x, y, epochs=20, batch=4096, lr=2e-3, seed=0)
    assert hist[-1] < hist[0]
    _, w = net.weights()

    wl = synth.rgbd(seed=1)
    frs = frames(wl)
    plain, obs_p, fine_p = run(wl, frs, capture=True)
    xe, ye = labelled(plain)
    misclass = float((predictor.predicted_levels(net, xe) != ye).float().mean().item())
    learned, obs_l, fine_l = run(wl, frs, w=w)
    assert misclass < 0.2, misclass
    assert fine_l < fine_p and obs_l < obs_p, (fine_l, fine_p, obs_l, obs_p)

    K = m_.pinhole_from(wl)
    clean = dataclasses.replace(wl, noise_coef=0.0, dropout=0.0)
    sc = wl.scene()

    def cloud(gmap, k):
        T = wl.pose(k)
        return metrics.backproject(gmap.raycast(K, T).cpu().numpy(), wl.fx, wl.fy, wl.cx, wl.cy, T, stride=4)

    views = range(0, n_frames, 20)
    gt = []
    for k in views:
        d, _, _ = synth.render_depth(clean, k, scene=sc)
        gt.append(metrics.backproject(np.where((d >= wl.min_depth) & (d <= wl.max_depth), d, 0.0), wl.fx, wl.fy,
                                      wl.cx, wl.cy, wl.pose(k), stride=4))
    gt = np.concatenate(gt)
    ch_p = metrics.chamfer(np.concatenate([cloud(plain, k) for k in views]), gt)["chamfer"]
    ch_l = metrics.chamfer(np.concatenate([cloud(learned, k) for k in views]), gt)["chamfer"]
    assert ch_l - ch_p <= 1e-3, (ch_l, ch_p)
