"""Pins of the splat oracle (Sec. 3.5, Eqs. 7-9) against closed forms, a finite-difference Jacobian, rigid-motion
invariance and hand-computed blends. No GPU."""
import math

import numpy as np
import pytest

import oracle


def f32(x):
    return float(np.float32(x))


def cam(width=64, height=48, f=(80.0, 90.0), c=(32.0, 24.0), near=0.1, far=20.0):
    return oracle.Pinhole(f[0], f[1], c[0], c[1], width, height, near, far)


def rot(axis, angle):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def cov6(S):
    return np.array([S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]], np.float32)


def random_spd(rng, scale):
    A = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(A)
    return Q @ np.diag((scale * rng.uniform(0.3, 1.5, 3)) ** 2) @ Q.T


def test_projection_on_the_optical_axis_is_the_closed_form():
    K = cam()
    for sx, sy, sz, z in ((0.05, 0.05, 0.05, 2.0), (0.02, 0.07, 0.3, 3.5)):
        p = oracle.splat_project([0, 0, z], cov6(np.diag([sx * sx, sy * sy, sz * sz])), K, np.eye(4))
        np.testing.assert_allclose(p["mu"], [K.cx, K.cy], rtol=0, atol=1e-5)
        np.testing.assert_allclose(p["cov"], [(K.fx * sx / z) ** 2, 0.0, (K.fy * sy / z) ** 2], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(p["conic"], [(z / (K.fx * sx)) ** 2, 0.0, (z / (K.fy * sy)) ** 2], rtol=1e-5,
                                   atol=1e-7)
        assert p["z"] == np.float32(z)


def test_projection_off_axis_matches_a_finite_difference_jacobian():
    rng = np.random.default_rng(3)
    K = cam()
    for _ in range(20):
        R = rot(rng.normal(size=3), rng.uniform(-1, 1))
        t = rng.normal(size=3)
        T = pose(R, t)
        pc = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(1.5, 5)])
        mu = R @ pc + t
        S = random_spd(rng, 0.05)

        def pi(m):
            c = R.T @ (m - t)
            return np.array([K.fx * c[0] / c[2] + K.cx, K.fy * c[1] / c[2] + K.cy])

        h = 1e-6
        J = np.stack([(pi(mu + h * e) - pi(mu - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        Si = J @ S @ J.T
        p = oracle.splat_project(mu.astype(np.float32), cov6(S), K, T)
        np.testing.assert_allclose(p["mu"], pi(mu), rtol=0, atol=2e-3)
        np.testing.assert_allclose(p["cov"], [Si[0, 0], Si[0, 1], Si[1, 1]], rtol=2e-3, atol=1e-3 * Si[0, 0])
        np.testing.assert_allclose(p["z"], pc[2], rtol=1e-5)
        inv = np.linalg.inv(Si)
        np.testing.assert_allclose(p["conic"], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=5e-3,
                                   atol=1e-3 * abs(inv[0, 0]))


def test_culling_by_depth_and_definiteness():
    K = cam(near=0.5, far=4.0)
    S = cov6(np.eye(3) * 1e-3)
    assert oracle.splat_project([0, 0, 0.4], S, K, np.eye(4)) is None
    assert oracle.splat_project([0, 0, 4.1], S, K, np.eye(4)) is None
    assert oracle.splat_project([0, 0, -2.0], S, K, np.eye(4)) is None
    assert oracle.splat_project([0, 0, 2.0], np.zeros(6, np.float32), K, np.eye(4)) is None
    assert oracle.splat_project([0, 0, 2.0], S, K, np.eye(4)) is not None
    rgb, tr, drawn = oracle.splat_render([[0, 0, 0.4], [0, 0, 2.0]], [S, S], [0.5, 0.5], [[1, 1, 1], [1, 1, 1]], K,
                                         np.eye(4))
    assert drawn == 1


def test_one_gaussian_blends_alpha_times_the_gaussian():
    K = cam(width=40, height=30, f=(60.0, 60.0), c=(20.0, 15.0))
    z, s, a = 2.0, 0.06, f32(0.7)
    C = np.array([0.2, 0.5, 0.9], np.float32).astype(np.float64)
    rgb, tr, drawn = oracle.splat_render([[0, 0, z]], [cov6(np.eye(3) * s * s)], [a], [C], K, np.eye(4))
    assert drawn == 1
    np.testing.assert_allclose(rgb[15, 20], a * C, rtol=1e-12)
    assert tr[15, 20] == pytest.approx(1 - a, rel=1e-12)
    sig = K.fx * s / z  # 1.8 px
    v, u = np.mgrid[0:30, 0:40]
    q = ((u - 20.0) ** 2 + (v - 15.0) ** 2) / sig ** 2
    inside = q <= 9.0 * (1 - 1e-5)
    outside = q >= 9.0 * (1 + 1e-5)
    w = a * np.exp(-0.5 * q)
    np.testing.assert_allclose(rgb[inside], w[inside][:, None] * C, rtol=2e-5)
    np.testing.assert_allclose(tr[inside], 1 - w[inside], rtol=2e-5)
    assert np.all(rgb[outside] == 0) and np.all(tr[outside] == 1)
    assert inside.sum() > 80


def test_one_tilted_gaussian_follows_its_image_covariance():
    """On the optical axis Sigma_I is diag(f/z) Sigma_W[:2, :2] diag(f/z) exactly, off-diagonal terms included."""
    K = cam(width=40, height=30, f=(60.0, 70.0), c=(20.0, 15.0))
    z, a = 2.0, f32(0.8)
    S = np.array([[0.004, 0.0025, 0.001], [0.0025, 0.003, 0.0], [0.001, 0.0, 0.002]])
    S32 = cov6(S)
    Sf = np.array([[S32[0], S32[1]], [S32[1], S32[3]]], np.float64)
    D = np.diag([K.fx / z, K.fy / z])
    Si = D @ Sf @ D
    rgb, tr, _ = oracle.splat_render([[0, 0, z]], [S32], [a], [[1, 1, 1]], K, np.eye(4))
    v, u = np.mgrid[0:30, 0:40]
    d = np.stack([u - 20.0, v - 15.0], -1)
    q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(Si), d)
    box = (np.abs(d[..., 0]) <= 3 * np.sqrt(Si[0, 0]) * (1 - 1e-5)) & (np.abs(d[..., 1]) <= 3 * np.sqrt(Si[1, 1]) * (1 - 1e-5))
    inside = (q <= 9.0 * (1 - 1e-4)) & box
    outside = q >= 9.0 * (1 + 1e-4)
    np.testing.assert_allclose(tr[inside], 1 - a * np.exp(-0.5 * q[inside]), rtol=1e-5)
    assert np.all(tr[outside] == 1)
    assert inside.sum() > 50 and outside.sum() > 50


def test_two_gaussians_blend_front_to_back_whatever_their_index():
    K = cam(width=20, height=20, f=(50.0, 50.0), c=(10.0, 10.0))
    S = cov6(np.eye(3) * 0.05 ** 2)
    near = ([0, 0, 1.0], 0.6, [1.0, 0.0, 0.0])
    far = ([0, 0, 2.0], 0.8, [0.0, 0.0, 1.0])
    outs = []
    for first, second in ((near, far), (far, near)):
        rgb, tr, _ = oracle.splat_render([first[0], second[0]], [S, S], [first[1], second[1]], [first[2], second[2]],
                                         K, np.eye(4))
        outs.append((rgb, tr))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    rgb, tr = outs[0]
    # at the centre both Gaussians evaluate to 1
    a1, a2 = f32(0.6), f32(0.8)
    np.testing.assert_allclose(rgb[10, 10], [a1, 0.0, a2 * (1 - a1)], rtol=1e-12)
    assert tr[10, 10] == pytest.approx((1 - a1) * (1 - a2), rel=1e-12)
    # one pixel off: G = exp(-q/2) with the footprint of each depth
    g1 = math.exp(-0.5 * (1.0 / (50 * 0.05 / 1.0) ** 2))
    g2 = math.exp(-0.5 * (1.0 / (50 * 0.05 / 2.0) ** 2))
    np.testing.assert_allclose(rgb[10, 11], [a1 * g1, 0.0, a2 * g2 * (1 - a1 * g1)], rtol=2e-6)


def test_equal_depths_blend_in_index_order_and_an_opaque_front_hides_the_rest():
    K = cam(width=20, height=20, f=(50.0, 50.0), c=(10.0, 10.0))
    S = cov6(np.eye(3) * 0.05 ** 2)
    rgb, tr, _ = oracle.splat_render([[0, 0, 1.0], [0, 0, 1.0]], [S, S], [0.5, 0.5], [[1, 0, 0], [0, 1, 0]], K,
                                     np.eye(4))
    np.testing.assert_allclose(rgb[10, 10], [0.5, 0.25, 0.0], rtol=1e-12)
    rgb, tr, _ = oracle.splat_render([[0, 0, 2.0], [0, 0, 1.0]], [S, S], [0.9, 1.0], [[1, 0, 0], [0, 1, 0]], K,
                                     np.eye(4))
    np.testing.assert_array_equal(rgb[10, 10], [0.0, 1.0, 0.0])
    assert tr[10, 10] == 0.0


def test_moving_camera_and_gaussians_together_changes_nothing():
    rng = np.random.default_rng(5)
    K = cam(width=48, height=36, f=(60.0, 60.0), c=(24.0, 18.0))
    n = 60
    pc = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n), rng.uniform(1.5, 3.0, n)], 1)
    covs = [random_spd(rng, 0.05) for _ in range(n)]
    op = rng.uniform(0.2, 0.9, n).astype(np.float32)
    col = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    ref_rgb, ref_tr, _ = oracle.splat_render(pc, np.stack([cov6(S) for S in covs]), op, col, K, np.eye(4))
    assert ref_tr.min() < 0.5
    for k in range(3):
        R = rot(rng.normal(size=3), rng.uniform(-2, 2))
        t = rng.normal(size=3) * 2
        mu = pc @ R.T + t
        rgb, tr, _ = oracle.splat_render(mu, np.stack([cov6(R @ S @ R.T) for S in covs]), op, col, K, pose(R, t))
        # float projection: footprints move by rounding only; pixels near a support edge may flip, so compare robustly
        bad = np.abs(rgb - ref_rgb).max(axis=2) > 1e-3
        assert bad.mean() < 0.01
        assert np.median(np.abs(tr - ref_tr)) < 1e-5
