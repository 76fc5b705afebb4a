"""Pins for the oracle's z-buffer rasteriser (CPU only): hand-computed coverage, the
top-left rule on shared edges, depth interpolation, the (depth, index) tie-break,
order independence and flat headlight shading."""
import numpy as np

import sem_inputs as si


def _ortho_cam(W, H):
    # looking down -z from z=10 at the origin, up +y, half-height H/2: one world unit per pixel
    return si.camera(True, (W / 2, H / 2, 10.0), (W / 2, H / 2, 0.0), (0, 1, 0), W, H,
                     half_h=H / 2, znear=1.0, zfar=19.0)


def _tri(*pts):
    return np.array(pts, dtype=float).reshape(1, 3, 3)


def test_single_triangle_coverage(orc):
    W = H = 8
    cam = _ortho_cam(W, H)
    # world (x, y) maps to screen (x, H - y): triangle (1,7),(6,7),(1,2) in world
    # -> screen (1,1),(6,1),(1,6): pixel centres with px+py+1 <= 7 and px,py >= 1 (the
    # diagonal edge passes through centres exactly and is a right edge: excluded)
    t = _tri((1, 7, 0), (6, 7, 0), (1, 2, 0))
    rgba, depth, win = orc.render(t, [1], [[1, 1, 1]], cam)
    cov = win >= 0
    exp = np.zeros((H, W), bool)
    for py in range(H):
        for px in range(W):
            cx, cy = px + 0.5, py + 0.5
            inside = cx > 1 and cy > 1 and cx + cy < 7
            on_top = cy == 1 and 1 < cx < 6
            on_left = cx == 1 and 1 < cy < 6
            exp[py, px] = inside or on_top or on_left
    np.testing.assert_array_equal(cov, exp)


def test_shared_edges_covered_exactly_once(orc):
    # a square with corners on pixel centres and a fan of 4 triangles around its centre: every
    # covered pixel is claimed by exactly one triangle (edges pass through centres)
    # (power-of-two view size keeps every projected coordinate exact)
    W = H = 16
    cam = _ortho_cam(W, H)
    c = (7.5, 7.5, 0)
    corners = [(1.5, 1.5, 0), (13.5, 1.5, 0), (13.5, 13.5, 0), (1.5, 13.5, 0)]
    tris = np.array([[corners[i], corners[(i + 1) % 4], c] for i in range(4)], float)
    counts = np.zeros((H, W), int)
    for i in range(4):
        _, _, win = orc.render(tris[i:i + 1], [1], [[1, 1, 1]], cam)
        counts += win >= 0
    assert counts.max() == 1
    # the union is the square, screen x in [1.5, 13.5), screen y = H - y in [2.5, 14.5),
    # with its left and top edges (through pixel centres) included
    exp = np.zeros((H, W), bool)
    for py in range(H):
        for px in range(W):
            cx, cy = px + 0.5, py + 0.5
            exp[py, px] = 1.5 <= cx < 13.5 and 2.5 <= cy < 14.5
    np.testing.assert_array_equal(counts == 1, exp)


def test_depth_plane_and_tie_break(orc):
    W = H = 16
    cam = _ortho_cam(W, H)
    # a tilted plane z = 0.1 x: z_view = 10 - 0.1 x, depth = (z_view - 1)/18
    t = _tri((0, 0, 0), (16, 0, 1.6), (0, 16, 0))
    _, depth, win = orc.render(t, [1], [[1, 1, 1]], cam)
    py, px = np.nonzero(win >= 0)
    cx = px + 0.5
    np.testing.assert_allclose(depth[py, px], (10 - 0.1 * cx - 1) / 18, atol=1e-14)
    # two coincident triangles: the lower index wins everywhere
    two = np.concatenate([_tri((0, 0, 1), (16, 0, 1), (0, 16, 1))] * 2)
    _, _, win2 = orc.render(two, [2], [[1, 1, 1]], cam)
    assert set(np.unique(win2)) <= {-1, 0}


def test_perspective_depth(orc):
    W, H = 20, 10
    cam = si.camera(False, (0, 0, 5.0), (0, 0, 0), (0, 1, 0), W, H, fovy_deg=60.0, znear=1.0, zfar=9.0)
    t = _tri((-50, -50, 2), (50, -50, 2), (0, 50, 2))  # plane at z_view = 3
    _, depth, win = orc.render(t, [1], [[1, 1, 1]], cam)
    assert (win >= 0).all()
    np.testing.assert_allclose(depth, 9 / 8 * (1 - 1 / 3), atol=1e-14)


def test_order_independence_and_shading(orc):
    rng = np.random.default_rng(0)
    W, H = 32, 24
    cam = si.camera(False, (3, 2, 9.0), (0, 0, 0), (0, 1, 0), W, H, fovy_deg=50.0, znear=1.0, zfar=20.0)
    tris = rng.uniform(-3, 3, size=(60, 3, 3))
    seg = [20, 25, 15]
    rgb = [[0.9, 0.3, 0.2], [0.2, 0.6, 0.9], [1.0, 1.0, 1.0]]
    img, dep, win = orc.render(tris, seg, rgb, cam)
    perm = rng.permutation(60)
    # permuting changes indices and segments; compare per-pixel winning geometry instead
    segid = np.repeat(np.arange(3), seg)
    img2, dep2, win2 = orc.render(tris[perm], [60], [[1, 1, 1]], cam)
    cov = win >= 0
    np.testing.assert_array_equal(cov, win2 >= 0)
    np.testing.assert_array_equal(dep[cov], dep2[cov])
    # with distinct depths the winner is the same triangle after permutation
    np.testing.assert_array_equal(perm[win2[cov]], win[cov])
    # shading: headlight factor 0.15 + 0.85 |n.l| applied to the segment colour
    f = np.array(cam["center"]) - np.array(cam["eye"])
    f /= np.linalg.norm(f)
    for py, px in zip(*np.nonzero(cov)):
        t = tris[win[py, px]]
        n = np.cross(t[1] - t[0], t[2] - t[0])
        s = 0.15 + 0.85 * abs(n @ f) / np.linalg.norm(n)
        exp = np.floor(np.clip(np.array(rgb[segid[win[py, px]]]) * s, 0, 1) * 255 + 0.5)
        np.testing.assert_array_equal(img[py, px, :3], exp)
        assert img[py, px, 3] == 255
    assert (img[~cov] == 0).all() and (dep[~cov] == 1.0).all()


def test_near_plane_drop(orc):
    W = H = 8
    cam = _ortho_cam(W, H)
    t = _tri((0, 0, 9.5), (8, 0, 0), (0, 8, 0))  # first vertex at z_view = 0.5 < znear
    _, _, win = orc.render(t, [1], [[1, 1, 1]], cam)
    assert (win < 0).all()
