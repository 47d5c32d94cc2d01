"""Pins for multi-resolution Marching Cubes (Sec. 3.4, Figs. 5 and 6).

The case table is built by the oracle from its definition (loops of face segments, inside corners of a face kept
apart). It is pinned by brute-force properties of every case: triangles only on edges whose ends change sign and every
such edge used; single-corner cases cut that corner off facing away from it; planar cases give two triangles. The cell
layout and corner rule are pinned by fields with known surfaces: a sphere's exact distance on one level gives a closed,
consistently oriented mesh (every edge in two triangles, once in each direction; Euler characteristic 2) whose
vertices lie within the linear-interpolation error of the sphere; a linear field gives vertices on its plane at every
level and triangles facing along its gradient. The blending across resolution boundaries is a reading (the paper gives
only the idea); its vertices are held to a bound.
"""
import numpy as np
import pytest

import oracle
import synth

E = 0.08


def _map(precision="f32s"):
    return oracle.OracleMap(oracle.params_from(synth.rgbd(), precision))


def _centres(key, level):
    n = 8 >> level
    v = 0.01 * (1 << level)
    i = np.arange(n ** 3)
    loc = np.stack([i % n, (i // n) % n, i // (n * n)], axis=1) + 0.5
    return np.asarray(key, np.float64) * E + loc * v


def _fill(m, keys, level_of, field):
    for k in keys:
        lv = level_of(k)
        X = _centres(k, lv)
        m.set_block(k, lv, field(X), np.ones(len(X)))


def _box(lo, hi):
    return [(x, y, z) for x in range(lo[0], hi[0]) for y in range(lo[1], hi[1]) for z in range(lo[2], hi[2])]


# ---------------------------------------------------------------------------------------------- the case table

def test_table_uses_exactly_the_sign_changing_edges():
    nt, tri, ec = oracle.mc_table()
    for cs in range(256):
        inside = [(cs >> c) & 1 for c in range(8)]
        crossing = {e for e in range(12) if inside[ec[e, 0]] != inside[ec[e, 1]]}
        used = set(tri[cs, :nt[cs]].ravel().tolist())
        assert used == crossing, cs
    assert nt[0] == 0 and nt[255] == 0 and nt.max() <= 5


def _corner(c):
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], np.float64)


def _mid(ec, e):
    return 0.5 * (_corner(ec[e, 0]) + _corner(ec[e, 1]))


def test_single_corner_cases_cut_the_corner_off_facing_outside():
    nt, tri, ec = oracle.mc_table()
    for c in range(8):
        for cs, sign in ((1 << c, 1.0), (255 ^ (1 << c), -1.0)):
            assert nt[cs] == 1
            a, b, d = (_mid(ec, e) for e in tri[cs, 0])
            normal = np.cross(b - a, d - a)
            away = (a + b + d) / 3 - _corner(c)   # from the lone corner towards the triangle
            # one inside corner: the normal points away from it; one outside corner: towards it
            assert sign * np.dot(normal, away) > 0, cs


def test_planar_cases_give_two_triangles_facing_the_outside():
    nt, tri, ec = oracle.mc_table()
    for a in range(3):
        low = sum(1 << c for c in range(8) if not (c >> a) & 1)   # the low half along axis a is inside
        for cs, out in ((low, 1.0), (255 ^ low, -1.0)):
            assert nt[cs] == 2
            for t in tri[cs, :2]:
                p, q, r = (_mid(ec, e) for e in t)
                nrm = np.cross(q - p, r - p)
                assert out * nrm[a] > 0 and abs(nrm[(a + 1) % 3]) < 1e-12 and abs(nrm[(a + 2) % 3]) < 1e-12


# ---------------------------------------------------------------------------------------------- fields

def _edges(tris):
    """Weld bit-identical positions; return vertex count, directed edges, undirected edge count."""
    flat = tris.reshape(-1, 3)
    uniq, inv = np.unique(flat.view(np.dtype((np.void, 12))), return_inverse=True)
    ids = inv.reshape(-1, 3)
    ids = ids[(ids[:, 0] != ids[:, 1]) & (ids[:, 1] != ids[:, 2]) & (ids[:, 0] != ids[:, 2])]
    directed = np.concatenate([ids[:, [0, 1]], ids[:, [1, 2]], ids[:, [2, 0]]])
    return len(uniq), ids, directed


@pytest.mark.parametrize("level", [0, 1, 2])
def test_sphere_on_one_level_is_closed_oriented_and_accurate(level):
    c = np.array([0.013, -0.007, 1.004])
    r = 0.19
    m = _map()
    _fill(m, _box((-4, -4, 9), (4, 4, 17)), lambda k: level, lambda X: np.linalg.norm(X - c, axis=1) - r)
    tris = m.extract_mesh()
    assert len(tris) > 100
    nv, ids, directed = _edges(tris)
    # every directed edge once, and its reverse once: closed and consistently oriented
    d = {tuple(e) for e in directed.tolist()}
    assert len(d) == len(directed)
    assert all((b, a) in d for a, b in d)
    n_edges = len(directed) // 2
    assert nv - n_edges + len(ids) == 2
    # vertices on the sphere up to linear interpolation of |x - c| along an edge of length h: h^2 / (8 r)
    h = 0.01 * (1 << level)
    dist = np.abs(np.linalg.norm(tris.reshape(-1, 3).astype(np.float64) - c, axis=1) - r)
    assert dist.max() <= h * h / (8 * r) + 2e-6
    # outward, and enclosing the sphere's volume (divergence theorem over the oriented triangles) less what the flat
    # triangles cut off: their vertices are inside by at most h^2 / (8 r) and their edges (at most sqrt 2 h) sag by at
    # most 2 h^2 / (8 r), so at most 3 h^2 / (4 r^2) of the volume
    p0, p1, p2 = (tris[:, i].astype(np.float64) - c for i in range(3))
    vol = np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6 / (4 / 3 * np.pi * r ** 3)
    assert 1 - 3 * h * h / (4 * r * r) - 0.002 < vol < 1.002


N_HAT = np.array([0.25, -0.15, -1.0]) / np.linalg.norm([0.25, -0.15, -1.0])
P0 = np.array([0.02, -0.01, 1.0])


@pytest.mark.parametrize("precision,tol", [("f64", 1e-7), ("f32s", 3e-6)])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_linear_field_vertices_lie_on_the_plane(precision, tol, level):
    m = _map(precision)
    _fill(m, _box((-2, -2, 10), (2, 2, 15)), lambda k: level, lambda X: (X - P0) @ N_HAT)
    tris = m.extract_mesh().astype(np.float64)
    assert len(tris) > 50
    assert np.abs((tris.reshape(-1, 3) - P0) @ N_HAT).max() <= tol
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    big = np.linalg.norm(nrm, axis=1) > 1e-12
    assert np.all(nrm[big] @ N_HAT > 0)


def test_mixed_levels_stay_near_the_plane_and_fill_the_seams():
    """Blocks alternate between levels 0 and 1 along x. The cells of each block reach the first voxel centre of the
    next block, so the meshes of the two levels meet; a corner read across the boundary takes the coarse voxel that
    contains a fine centre (or the reverse), which is off by at most half a coarse voxel along the gradient."""
    m = _map()
    keys = _box((-2, -2, 10), (2, 2, 15))
    _fill(m, keys, lambda k: k[0] & 1, lambda X: (X - P0) @ N_HAT)
    tris = m.extract_mesh().astype(np.float64)
    dev = np.abs((tris.reshape(-1, 3) - P0) @ N_HAT)
    assert dev.max() <= 0.5 * 0.02
    # across the seams the cells of the two levels tile space: seen along z (the plane is a graph over x, y) every
    # interior point is covered by exactly one triangle, up to the slivers that the blend leaves along the seams
    cover = _coverage(tris[:, :, :2], np.arange(-0.11, 0.11, 0.0017), np.arange(-0.11, 0.11, 0.0017))
    assert np.mean(cover == 1) > 0.995 and np.mean(cover == 0) < 0.003 and cover.max() <= 2


def _coverage(tri2, xs, ys):
    """Number of triangles (projected to 2D) containing each point of the grid xs x ys."""
    X, Y = np.meshgrid(xs, ys)
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    cnt = np.zeros(len(P), np.int32)
    for t in tri2:
        lo, hi = t.min(axis=0), t.max(axis=0)
        sel = np.nonzero(np.all((P >= lo) & (P <= hi), axis=1))[0]
        if len(sel) == 0:
            continue
        a, b, c = t
        q = P[sel]
        d1 = (b[0] - a[0]) * (q[:, 1] - a[1]) - (b[1] - a[1]) * (q[:, 0] - a[0])
        d2 = (c[0] - b[0]) * (q[:, 1] - b[1]) - (c[1] - b[1]) * (q[:, 0] - b[0])
        d3 = (a[0] - c[0]) * (q[:, 1] - c[1]) - (a[1] - c[1]) * (q[:, 0] - c[0])
        inside = ((d1 >= 0) & (d2 >= 0) & (d3 >= 0)) | ((d1 <= 0) & (d2 <= 0) & (d3 <= 0))
        cnt[sel[inside]] += 1
    return cnt


def test_fused_frame_mesh_follows_the_scene():
    """A fused noise-free frame: vertices on the sphere and on the back wall lie within the projective bound of Eq. 2
    (the voxel reads the range of its nearest pixel, whose ray is up to 0.71 / f rad off the voxel's own: a surface at
    incidence theta moves by at most rho tan(theta) 0.71 / f) plus half a millimetre."""
    wl = synth.tiny(noise=False)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    depth, rgb, T = synth.render_depth(wl, 0)
    m.integrate_depth(oracle.pinhole_from(wl), T, depth, rgb)
    V = m.extract_mesh().reshape(-1, 3).astype(np.float64)
    assert len(V) > 30000
    rho = np.linalg.norm(V, axis=1)
    ray = V / rho[:, None]
    c = np.array([0.0, 0.0, 1.5])
    n_s = (V - c) / np.linalg.norm(V - c, axis=1)[:, None]
    d_s = np.abs(np.linalg.norm(V - c, axis=1) - 0.5)
    cos_s = np.abs(np.sum(ray * n_s, axis=1))
    on_s = (d_s < 0.03) & (cos_s > 0.3)
    bound_s = rho * np.sqrt(1 - cos_s ** 2) / cos_s * 0.71 / wl.fx + 5e-4
    assert on_s.sum() > 20000
    assert np.all(d_s[on_s] <= bound_s[on_s])
    cos_b = np.abs(ray[:, 2])
    on_b = (np.abs(V[:, 2] - 3.0) < 0.03) & (np.abs(V[:, 0]) < 1.4) & (np.abs(V[:, 1]) < 1.4) & ~(d_s < 0.05)
    bound_b = rho * np.sqrt(1 - cos_b ** 2) / cos_b * 0.71 / wl.fx + 5e-4
    assert on_b.sum() > 100000
    assert np.all(np.abs(V[on_b, 2] - 3.0) <= bound_b[on_b])


# ---------------------------------------------------------------------------------------------- vertex collapse

def _sphere_soup(level=0):
    c = np.array([0.013, -0.007, 1.004])
    m = _map()
    _fill(m, _box((-4, -4, 9), (4, 4, 17)), lambda k: level, lambda X: np.linalg.norm(X - c, axis=1) - 0.19)
    return m.extract_mesh()


def test_collapse_at_a_tiny_spacing_only_joins_equal_vertices():
    soup = _sphere_soup()
    verts, faces = oracle.weld_mesh(soup, 1e-7)
    flat = soup.reshape(-1, 3)
    assert len(verts) == len(np.unique(flat, axis=0))
    assert len(faces) == len(soup)
    # the welded closed surface: V - E + F = 2, every edge in exactly two faces
    e = np.sort(np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]]), axis=1)
    ue, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(cnt == 2)
    assert len(verts) - len(ue) + len(faces) == 2
    # faces point at the soup's own vertices, in the same winding
    np.testing.assert_array_equal(verts[faces], soup)


@pytest.mark.parametrize("delta", [0.00125, 0.005])
def test_collapse_keeps_members_inside_their_cluster_cell(delta):
    soup = _sphere_soup()
    verts, faces = oracle.weld_mesh(soup, delta)
    flat = soup.reshape(-1, 3)
    # every representative is one of the soup's vertices
    soup_set = {tuple(v) for v in flat.tolist()}
    assert all(tuple(v) in soup_set for v in verts.tolist())
    # each face vertex moved by less than a cluster cell's diagonal, and the faces kept are the non-degenerate ones
    kept = (np.abs(np.diff(np.sort(faces, axis=1), axis=1)) > 0).all(axis=1)
    assert kept.all() and len(faces) <= len(soup)
    # coarser grids merge more
    v2, f2 = oracle.weld_mesh(soup, 2 * delta)
    assert len(v2) < len(verts) and len(f2) <= len(faces)
    # representatives are the smallest member of their cell
    cells = np.floor(flat * np.float32(1.0 / delta)).astype(np.int64)
    order = np.lexsort((flat[:, 2], flat[:, 1], flat[:, 0]))
    first = {}
    for i in order:
        first.setdefault(tuple(cells[i]), tuple(flat[i]))
    assert len(first) == len(verts)
    assert sorted(first.values()) == sorted(tuple(v) for v in verts.tolist())
