"""Pins for the learned level predictor's oracles (an addition to the paper's method, which allocates every new block
at the finest level, Sec. 3.2.1).

Two oracles are pinned here:
  - oracle/level_predictor.cpp (float, decides levels bit for bit): its exp / erf / GELU against the math library within
    their published error bounds, its BF16 rounding against torch's bfloat16 conversion, its forward pass against an
    independent float64 evaluation and against hand-built networks with closed-form outputs, and its features against
    closed forms on constant and linear range images;
  - oracle/mlp.py (float64 training): its gradient against central differences, its loss and Adam step against closed
    forms.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp


# ---------------------------------------------------------------------------------------------- scalar functions

def test_exp_within_taylor_bound():
    """Cody-Waite reduction leaves |r| <= ln2 / 2; the degree-6 Taylor remainder is below r^7 / 7! * e^r < 1.7e-7
    relative, plus a few float roundings."""
    xs = np.concatenate([np.linspace(-87.0, 87.0, 20001), np.linspace(-1.0, 1.0, 2001)])
    worst = max(abs(oracle.exp_cw(float(x)) / math.exp(float(np.float32(x))) - 1.0) for x in xs)
    assert worst < 1.7e-7 + 6 * 2.0 ** -24
    assert oracle.exp_cw(0.0) == 1.0
    assert oracle.exp_cw(-100.0) == 0.0


def test_erf_within_abramowitz_stegun_bound():
    """A&S 7.1.26: |error| <= 1.5e-7; float evaluation adds a few ulps of 1."""
    xs = np.linspace(-6.0, 6.0, 24001)
    worst = max(abs(oracle.erf_as(float(x)) - math.erf(float(np.float32(x)))) for x in xs)
    assert worst < 1.5e-7 + 8 * 2.0 ** -24
    assert oracle.erf_as(0.0) == 0.0
    assert oracle.erf_as(-1.25) == -oracle.erf_as(1.25)  # odd


def test_gelu_close_to_exact():
    for x in np.linspace(-8.0, 8.0, 3201):
        xf = float(np.float32(x))
        exact = 0.5 * xf * (1.0 + math.erf(xf / math.sqrt(2.0)))
        assert abs(oracle.gelu(xf) - exact) <= abs(xf) * 1.6e-7 + 4e-7 * max(1.0, abs(xf))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 4000),
                        np.float32([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, -0.0, 3.0e38])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(float(v)) for v in x], np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    np.testing.assert_array_equal(mlp.bf16_round(x).astype(np.float32).view(np.uint32), ref.view(np.uint32))


# ---------------------------------------------------------------------------------------------- network

def _random_bf16_weights(seed, scale=1.0):
    return mlp.bf16_bits(mlp.init_params(seed, scale) + 0.05 * np.random.default_rng(seed + 1).standard_normal(
        mlp.N_PARAMS))


def test_forward_matches_float64_network():
    """The float forward pass (sums in index order, BF16 activations) against the float64 network with the same BF16
    weights and activation rounding. A float/double difference can flip one activation's BF16 rounding (one BF16 ulp,
    2^-8 relative), so most logits agree to float precision and all within the effect of a few such flips."""
    w = _random_bf16_weights(3)
    rng = np.random.default_rng(4)
    x = mlp.bf16_round(rng.standard_normal((512, 16)) * 2.0)
    got = oracle.mlp_forward(w, x.astype(np.float32)).astype(np.float64)
    ref = mlp.forward(mlp.from_bf16_bits(w), x, act_round=True)["z"]
    err = np.abs(got - ref)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.mean(err <= 2e-5 * scale) > 0.97
    assert np.all(err <= 0.05 * scale)


def test_forward_closed_forms():
    """Hand-built networks: biases only gives logits = b3; one path x0 -> h1_0 -> h2_0 -> logits gives
    logits_c = c h2_0 + b3_c with h1_0 = BF16(GELU(x0)), h2_0 = BF16(GELU(h1_0))."""
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["b3"] = np.array([0.5, -1.25, 2.0])
    w = mlp.bf16_bits(mlp.pack(p))
    x = np.random.default_rng(5).standard_normal((4, 16)).astype(np.float32)
    np.testing.assert_array_equal(oracle.mlp_forward(w, x), np.tile(np.float32([0.5, -1.25, 2.0]), (4, 1)))
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, :] = [0.0, 1.0, 2.0]
    w = mlp.bf16_bits(mlp.pack(p))
    for x0 in (-2.0, -0.5, 0.25, 1.0, 3.0):
        x = np.zeros((1, 16), np.float32)
        x[0, 0] = x0
        g = lambda t: 0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0)))  # noqa: E731
        h1 = float(mlp.bf16_round(np.array([g(x0)]))[0])
        h2 = float(mlp.bf16_round(np.array([g(h1)]))[0])
        expect = np.array([0.5, h2 - 1.25, 2.0 * h2 + 2.0])
        np.testing.assert_allclose(oracle.mlp_forward(w, x)[0], expect, rtol=0, atol=2.0 * 2.0 ** -8 * max(1, abs(h2)))


# ---------------------------------------------------------------------------------------------- features

def _cam(width=64, height=48):
    K = oracle.Pinhole()
    K.fx = K.fy = 50.0
    K.cx, K.cy = 31.5, 23.5
    K.width, K.height = width, height
    K.min_depth, K.max_depth = 0.1, 10.0
    return K


E, TAU = 0.08, 0.12


def _centre(key):
    return (np.asarray(key, np.float64) + 0.5) * E


def _bf(x):
    return float(mlp.bf16_round(np.array([x]))[0])


def _soft(x):
    return x / (1.0 + abs(x))


def _near(a, b, rel=2.0 ** -7):
    """Equal up to the BF16 rounding of a float-evaluated value (one BF16 ulp)."""
    return abs(a - b) <= rel * max(abs(b), 1e-30) + 1e-30


def test_features_constant_range_image():
    K = _cam()
    rho0 = 2.0
    rho = np.full((K.height, K.width), rho0, np.float32)
    key = (1, -1, 25)
    f = oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, key)
    c = _centre(key)
    r = float(np.linalg.norm(c))
    u, v = K.fx * c[0] / c[2] + K.cx, K.fy * c[1] / c[2] + K.cy
    expect = [r, _soft((rho0 - r) / TAU), 0.0, 0.0, 1.0, E / r, 0.0, 0.0, 0.0, 2 * abs(u / K.width - 0.5),
              2 * abs(v / K.height - 0.5), c[2] / r, 1.0 / r, 0.0, TAU / E, 1.0]
    for i, (a, b) in enumerate(zip(f, expect)):
        assert _near(float(a), _bf(b)), (i, a, b)


def test_features_linear_ramp():
    """rho = a + b u: the u-slope feature is b fx / r, the v-slope 0, the curvature 0, the spread over the 5 x 5 grid
    (offsets -2s..2s) b s sqrt 2 and the range b 4 s."""
    K = _cam(200, 150)
    K.cx, K.cy = 99.5, 74.5
    a, b = 1.5, 0.0078125  # dyadic: every sample and difference is exact in float
    u = np.arange(K.width, dtype=np.float64)
    rho = np.tile((a + b * u).astype(np.float32), (K.height, 1))
    key = (0, 0, 12)  # centre (0.04, 0.04, 1.0): projects to (101.5, 76.5), rounded to (102, 77)
    f = oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, key)
    c = _centre(key)
    r = float(np.linalg.norm(c))
    s = max(1, min(16, int(np.floor(0.5 * K.fx * 0.5 * E / c[2]))))
    assert s == 1
    u0 = 102
    mean = a + b * u0
    assert _near(float(f[1]), _bf(_soft((mean - r) / TAU)))
    # var = E[x^2] - mean^2 cancels in float
    assert _near(float(f[2]), _bf(_soft(b * s * math.sqrt(2.0) / TAU)), rel=2e-2)
    assert _near(float(f[3]), _bf(_soft(4 * b * s / E)))
    assert _near(float(f[6]), _bf(_soft(b * K.fx / r)))
    assert float(f[7]) == 0.0 and float(f[8]) == 0.0


def test_features_missing_samples_and_visibility():
    K = _cam()
    rho = np.full((K.height, K.width), 2.0, np.float32)
    rho[:, ::2] = -1.0  # every even column invalid
    key = (0, 0, 25)  # centre projects to pixel (32.3, 24.3) -> (32, 24); spacing s = 1
    f = oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, key)
    # columns 30..34: 31 and 33 present -> 2 of 5 per row
    assert float(f[4]) == _bf(10.0 / 25.0)
    assert float(f[6]) == 0.0  # neighbours 31, 33 present, equal
    assert float(f[8]) == 0.0  # no three consecutive samples present
    assert oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, (0, 0, -5)) is None  # behind
    assert oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, (40, 0, 5)) is None  # outside the image


def test_level_is_first_argmax_clamped():
    K = _cam()
    rho = np.full((K.height, K.width), 2.0, np.float32)
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    for b3, lvl3, lvl2 in (([1.0, 0.0, 0.0], 0, 0), ([0.0, 1.0, 1.0], 1, 1), ([0.0, 0.5, 1.0], 2, 1)):
        p["b3"] = np.array(b3)
        w = mlp.bf16_bits(mlp.pack(p))
        _, l3 = oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, (0, 0, 25), w, 3)
        _, l2 = oracle.block_features(K, np.eye(3), np.zeros(3), rho, E, TAU, (0, 0, 25), w, 2)
        assert (l3, l2) == (lvl3, lvl2)


# ---------------------------------------------------------------------------------------------- training oracle

def test_gradient_matches_central_differences():
    theta = mlp.init_params(0) + 0.01 * np.random.default_rng(1).standard_normal(mlp.N_PARAMS)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((9, 16))
    y = rng.integers(0, 3, 9)
    _, g = mlp.loss_and_grad(theta, x, y)
    h = 1e-5
    # every bias and output weight, and a sample of the rest
    idx = np.concatenate([np.arange(1024, 1088), np.arange(5120, 5443), rng.choice(5120, 200, replace=False)])
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, x, y) - mlp.loss(theta - e, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-8 + 1e-6 * abs(g[i]), i


def test_loss_and_gradient_of_zero_network():
    """All weights zero: logits 0, loss ln 3, d loss / d b3 = mean(1/3 - onehot), every other gradient 0."""
    theta = np.zeros(mlp.N_PARAMS)
    x = np.random.default_rng(3).standard_normal((6, 16))
    y = np.array([0, 1, 2, 2, 2, 1])
    L, g = mlp.loss_and_grad(theta, x, y)
    assert abs(L - math.log(3.0)) < 1e-15
    gb3 = g[-3:]
    np.testing.assert_allclose(gb3, [1 / 3 - 1 / 6, 1 / 3 - 2 / 6, 1 / 3 - 3 / 6], atol=1e-15)
    # W3 gradient: h2 = GELU(GELU(0)) = 0 for zero weights -> zero
    assert np.all(g[:-3] == 0.0)


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected first step is -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m1, m2 = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 1e-3)
    np.testing.assert_allclose(th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 0.001 * g * g)


# ---------------------------------------------------------------------------------------------- in the map

def _const_level_weights(level):
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["b3"] = np.eye(3)[level] * 4.0
    return mlp.bf16_bits(mlp.pack(p))


@pytest.mark.parametrize("level", [0, 1])
def test_predicted_level_in_oracle_map(level):
    """A network that always answers `level`: every new block that projects into the image starts at that level
    (blocks that do not project keep the finest level); the key set is the plain rule's."""
    wl = synth.tiny(noise=False)
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    plain = oracle.OracleMap(oracle.params_from(wl, "f32s", var_threshold=(-1.0, -1.0), split_hysteresis=0.0))
    plain.integrate_depth(K, T, depth, rgb)
    learned = oracle.OracleMap(oracle.params_from(wl, "f32s", var_threshold=(-1.0, -1.0), split_hysteresis=0.0))
    learned.set_predictor(_const_level_weights(level))
    learned.set_capture(True)
    st = learned.integrate_depth(K, T, depth, rgb)
    a, b = plain.extract(), learned.extract()
    np.testing.assert_array_equal(a["keys"], b["keys"])
    keys, feats = learned.features()
    assert len(keys) > 0.9 * st["new_blocks"] and feats.shape == (len(keys), 16)
    captured = {tuple(k) for k in keys}
    lv = {tuple(k): int(l) for k, l in zip(b["keys"], b["levels"])}
    assert all(lv[k] == level for k in captured)
    assert all(lv[k] == 0 for k in lv if k not in captured)
    # the captured features are the oracle's own features of each block
    rho = np.where((depth >= wl.min_depth) & (depth <= wl.max_depth), depth * np.sqrt(
        ((np.arange(wl.width, dtype=np.float32) - np.float32(wl.cx)) / np.float32(wl.fx))[None, :] ** 2 +
        ((np.arange(wl.height, dtype=np.float32) - np.float32(wl.cy)) / np.float32(wl.fy))[:, None] ** 2 + 1),
        -1).astype(np.float32)
    E_f = np.float32(np.float32(wl.base_voxel) / np.float32(2 ** (wl.n_levels - 1))) * np.float32(8)
    Rf, tf = T[:3, :3].astype(np.float32), T[:3, 3].astype(np.float32)
    for i in range(0, len(keys), max(1, len(keys) // 20)):
        f = oracle.block_features(K, Rf, tf, rho, float(E_f), float(np.float32(wl.truncation)), keys[i])
        np.testing.assert_array_equal(f, feats[i])


# ---------------------------------------------------------------------------------------------- LiDAR features

EL, TAUL = 0.5, 0.75  # LiDAR block edge and truncation (dyadic: block centres are exact in float and double)


def _grid_moments(qs):
    """The 10 end-point moments of integer positions qs (n, 3) in a block."""
    q = np.asarray(qs, np.uint64)
    x, y, z = q[:, 0], q[:, 1], q[:, 2]
    return np.array([len(q), x.sum(), y.sum(), z.sum(), (x * x).sum(), (y * y).sum(), (z * z).sum(), (x * y).sum(),
                     (x * z).sum(), (y * z).sum()], np.uint64)


def _pose_at(o):
    T = np.eye(4)
    T[:3, 3] = o
    return T


def _grid_var(step, m):
    """Population variance of the m equally spaced values 0, step, ..., (m - 1) step: step^2 (m^2 - 1) / 12."""
    return step * step * (m * m - 1) / 12.0


def test_lidar_features_horizontal_plane_seen_from_above():
    """End points on an 8 x 8 grid of a horizontal plane, the sensor straight above the block centre: the spread along
    the view (f2) and the vertical spread (f6) are zero, the lateral spread (f3, f11) is that of the grid in x and y,
    and the centroid offsets follow from the grid's mean."""
    key = (2, 3, -1)
    c = (np.asarray(key, np.float64) + 0.5) * EL
    h = 7.0
    T = _pose_at(c + [0.0, 0.0, h])
    step, m, qz = 128, 8, 300
    qs = [(step * i, step * j, qz) for i in range(m) for j in range(m)]
    f = oracle.lidar_block_features(_grid_moments(qs), T, EL, TAUL, key)
    off_xy = (step * (m - 1) / 2 + 0.5) / 1024 - 0.5
    off_z = (qz + 0.5) / 1024 - 0.5
    lat = math.sqrt(2 * _grid_var(step, m)) / 1024
    expect = [h, _soft(-off_z * EL / TAUL), 0.0, lat, _soft(64 / 16), EL / h, 0.0, math.sqrt(2) * abs(off_xy), 1.0,
              1.0, -1.0, lat, 1.0 / h, 1.0, TAUL / EL, 1.0]
    for i, (a, b) in enumerate(zip(f, expect)):
        assert _near(float(a), _bf(b)), (i, a, b)


def test_lidar_features_vertical_plane_seen_edge_on():
    """End points on a grid of the plane y = const, viewed along +x (inside the plane): the spread along the view is
    the grid's spread in x, the lateral spread its spread in z (a swapped axis or a transposed covariance fails)."""
    key = (-4, 0, 1)
    c = (np.asarray(key, np.float64) + 0.5) * EL
    h = 12.0
    T = _pose_at(c - [h, 0.0, 0.0])
    qs = [(64 * i, 700, 32 * j) for i in range(16) for j in range(4)]
    f = oracle.lidar_block_features(_grid_moments(qs), T, EL, TAUL, key)
    sx, sz = math.sqrt(_grid_var(64, 16)) / 1024, math.sqrt(_grid_var(32, 4)) / 1024
    off = np.array([(64 * 7.5 + 0.5) / 1024 - 0.5, 700.5 / 1024 - 0.5, (32 * 1.5 + 0.5) / 1024 - 0.5])
    assert _near(float(f[0]), _bf(h))
    assert _near(float(f[1]), _bf(_soft(off[0] * EL / TAUL)))
    assert _near(float(f[2]), _bf(_soft(sx * EL / TAUL)))
    assert _near(float(f[3]), _bf(sz))
    assert _near(float(f[6]), _bf(sz))
    assert _near(float(f[7]), _bf(math.hypot(off[1], off[2])))
    assert _near(float(f[11]), _bf(math.hypot(sx, sz)))
    assert float(f[9]) == 0.0 and float(f[10]) == 0.0


def test_lidar_features_block_without_end_points():
    """A block crossed only by free space: every end-point statistic is zero, the geometry features remain."""
    key = (10, -2, 0)
    c = (np.asarray(key, np.float64) + 0.5) * EL
    o = np.array([1.0, 2.0, 3.0])
    T = _pose_at(o)
    f = oracle.lidar_block_features(np.zeros(10, np.uint64), T, EL, TAUL, key)
    r = float(np.linalg.norm(c - o))
    uz = (c[2] - o[2]) / r
    assert all(float(f[i]) == 0.0 for i in (1, 2, 3, 4, 6, 7, 8, 11))
    for i, b in ((0, r), (5, EL / r), (9, abs(uz)), (10, uz), (12, 1.0 / r), (13, 1.0), (14, TAUL / EL), (15, 1.0)):
        assert _near(float(f[i]), _bf(b)), (i, f[i], b)


def test_lidar_features_against_numpy_covariance():
    """Random end points in random blocks seen from random sensor positions: the oracle's moment formulas (float)
    against numpy's float64 mean and covariance of the quantised points, projected on the view direction by a matrix
    product."""
    rng = np.random.default_rng(5)
    for trial in range(50):
        key = tuple(int(k) for k in rng.integers(-50, 50, 3))
        n = int(rng.integers(1, 400))
        spread = rng.uniform(0.02, 1.0, 3)
        q = np.clip(np.floor((0.5 + (rng.random((n, 3)) - 0.5) * spread) * 1024), 0, 1023).astype(np.int64)
        o = rng.uniform(-30, 30, 3)
        T = _pose_at(o)
        f = oracle.lidar_block_features(_grid_moments(q), T, EL, TAUL, key)
        c = (np.asarray(key, np.float64) + 0.5) * EL - o
        r = np.linalg.norm(c)
        u = c / r
        pos = (q + 0.5) / 1024 - 0.5
        mean = pos.mean(0)
        C = np.cov(pos.T, bias=True) if n > 1 else np.zeros((3, 3))
        along = mean @ u
        thick = math.sqrt(max(u @ C @ u, 0.0))
        lat = math.sqrt(max(np.trace(C) - u @ C @ u, 0.0))
        expect = {0: r, 1: _soft(along * EL / TAUL), 2: _soft(thick * EL / TAUL), 3: lat, 4: _soft(n / 16),
                  5: EL / r, 6: math.sqrt(max(C[2, 2], 0.0)), 7: np.linalg.norm(mean - along * u), 10: u[2],
                  11: math.sqrt(max(np.trace(C), 0.0)), 12: 1.0 / r}
        for i, b in expect.items():
            # spreads are float differences of large moments (E[q^2] - E[q]^2): allow 1e-6 block units absolute
            ok = _near(float(f[i]), _bf(b)) or abs(float(f[i]) - b) <= abs(b) * 2.0 ** -7 + 1e-6
            assert ok, (trial, i, f[i], b)


def _lidar_small():
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    return wl


def _end_point_moments(T, xyz, E_f, wl):
    """Moments of every end point's block, from the raw points: p = R x + t evaluated left to right in float64 as
    the map does, fixed point floor(p 65536 / E), block key floor(fixed / 65536), q = (fixed - key 65536) // 64."""
    x = xyz.astype(np.float64)
    n2 = (x * x).sum(1)
    ok = np.isfinite(n2) & (n2 >= np.float64(np.float32(wl.r_min)) ** 2) & (n2 <= np.float64(np.float32(wl.r_max)) ** 2)
    x = x[ok]
    p = np.stack([((T[a, 0] * x[:, 0] + T[a, 1] * x[:, 1]) + T[a, 2] * x[:, 2]) + T[a, 3] for a in range(3)], 1)
    fixed = np.floor(p * (65536.0 / float(E_f))).astype(np.int64)
    keys = fixed // 65536
    q = (fixed - keys * 65536) // 64
    out = {}
    for k in np.unique(keys, axis=0):
        sel = np.all(keys == k, axis=1)
        out[tuple(int(v) for v in k)] = _grid_moments(q[sel])
    return out


@pytest.mark.parametrize("level", [0, 2])
def test_predicted_level_in_oracle_map_lidar(level):
    """LiDAR scans: a network that always answers `level` puts every block new to the scan at that level (blocks of
    earlier scans keep theirs); the key set is the plain rule's; each captured record equals the features of the
    block's end-point moments computed from the raw points."""
    wl = _lidar_small()
    sc = wl.scene()
    scans = [synth.render_lidar(wl, k, scene=sc) for k in range(2)]
    prm = dict(var_threshold=(-1.0, -1.0), split_hysteresis=0.0)
    plain = oracle.OracleMap(oracle.params_from(wl, "f32s", **prm))
    learned = oracle.OracleMap(oracle.params_from(wl, "f32s", **prm))
    learned.set_predictor(_const_level_weights(level))
    E_f = float(np.float32(np.float32(wl.base_voxel) / np.float32(2 ** (wl.n_levels - 1))) * np.float32(8))
    total = 0
    for xyz, T in scans:
        learned.set_capture(True)  # records of this scan only
        plain.integrate_points(T, xyz)
        st = learned.integrate_points(T, xyz)
        keys, feats = learned.features()
        assert len(keys) == st["new_blocks"] > 0
        total += len(keys)
    a, b = plain.extract(), learned.extract()
    np.testing.assert_array_equal(a["keys"], b["keys"])
    assert np.all(b["levels"] == level)
    assert total == len(b["keys"])  # every block was new to some scan
    mom = _end_point_moments(scans[-1][1], scans[-1][0], E_f, wl)
    seen = 0
    for k, f in zip(keys, feats):
        m = mom.get(tuple(int(v) for v in k), np.zeros(10, np.uint64))
        g = oracle.lidar_block_features(m, scans[-1][1], E_f, float(np.float32(wl.truncation)), k)
        np.testing.assert_array_equal(g, f)
        seen += int(m[0] > 0)
    assert seen > 0.1 * len(keys)  # most new blocks hold only the truncation band in front of or behind a surface
