"""Pins for the oracle's marching-cubes table and extraction (CPU only).

Brute force over all 256 cases of one cell, closed-form sphere area/volume with O(h^2)
convergence, watertightness with consistent orientation, and exact vertex placement.
"""
import math

import numpy as np
import pytest

import sem_inputs as si

EDGES = [(lo, hi) for lo in range(8) for hi in range(lo + 1, 8) if (lo ^ hi) in (1, 2, 4)]


def _pos(v):
    return np.array([v & 1, (v >> 1) & 1, (v >> 2) & 1], float)


def _trilinear_grad(vals, p):
    g = np.zeros(3)
    for v in range(8):
        c = _pos(v)
        w = [p[d] if c[d] else 1 - p[d] for d in range(3)]
        for d in range(3):
            dw = list(w)
            dw[d] = 1.0 if c[d] else -1.0
            g[d] += vals[v] * dw[0] * dw[1] * dw[2]
    return g


def test_edge_numbering():
    assert EDGES == [(0, 1), (0, 2), (0, 4), (1, 3), (1, 5), (2, 3), (2, 6), (3, 7), (4, 5), (4, 6),
                     (5, 7), (6, 7)]


def test_table_brute_force(orc):
    n, t = orc.mc_table()
    assert n[0] == 0 and n[255] == 0
    for v in range(8):
        assert n[1 << v] == 1 and n[255 ^ (1 << v)] == 1
    for cs in range(256):
        cut = {e for e, (lo, hi) in enumerate(EDGES) if ((cs >> lo) & 1) != ((cs >> hi) & 1)}
        used = set()
        # every triangle edge between two loop vertices: count directed boundary edges
        directed = {}
        for q in range(n[cs]):
            tri = list(t[cs, q])
            assert all(e in cut for e in tri)
            used.update(tri)
            for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
                directed[(a, b)] = directed.get((a, b), 0) + 1
        assert used == cut, cs
        assert (t[cs, n[cs]:] == -1).all()
        # interior fan edges appear once in each direction; boundary (loop) edges once:
        # the boundary of the fan is a union of closed loops through the cut edges, each
        # cut edge having one outgoing and one incoming boundary edge
        boundary = [(a, b) for (a, b), c in directed.items() if (b, a) not in directed]
        outdeg = {}
        indeg = {}
        for a, b in boundary:
            outdeg[a] = outdeg.get(a, 0) + 1
            indeg[b] = indeg.get(b, 0) + 1
        assert set(outdeg) == cut and set(indeg) == cut
        assert all(v == 1 for v in outdeg.values()) and all(v == 1 for v in indeg.values())
        # orientation: with corner values +-1, every triangle normal has a positive
        # component along the trilinear interpolant's gradient at the triangle centroid
        vals = [1.0 if (cs >> v) & 1 else -1.0 for v in range(8)]
        for q in range(n[cs]):
            P = [(_pos(EDGES[e][0]) + _pos(EDGES[e][1])) / 2 for e in t[cs, q]]
            nn = np.cross(P[1] - P[0], P[2] - P[0])
            assert nn @ _trilinear_grad(vals, sum(P) / 3) > 0, (cs, q)


def test_single_cell_every_case(orc):
    # one element of order N=1 is one cell; corner values +-1 put vertices at midpoints,
    # random values put them at the linear-interpolation points
    rng = np.random.default_rng(5)
    m = si.uniform_box((1, 1, 1), (0, 0, 0), (2, 3, 5), 1)
    xyz = m.xyz().numpy()
    n, t = orc.mc_table()
    for cs in range(256):
        mag = rng.uniform(0.1, 1.0, 8)
        f = np.array([[mag[v] if (cs >> v) & 1 else -mag[v] for v in range(8)]])
        r = orc.isosurface(1, xyz, f, 0.0)
        assert r["cases"][0, 0] == cs
        assert r["ntri"] == n[cs]
        for q in range(n[cs]):
            for s in range(3):
                lo, hi = EDGES[t[cs, q, s]]
                tt = -f[0, lo] / (f[0, hi] - f[0, lo])
                pa, pb = xyz[:, 0, lo], xyz[:, 0, hi]
                np.testing.assert_allclose(r["tris"][q, s], pa + tt * (pb - pa), rtol=1e-15, atol=1e-15)


def test_isovalue_tie_counts_as_inside(orc):
    m = si.uniform_box((1, 1, 1), (0, 0, 0), (1, 1, 1), 1)
    f = np.array([[0.5, -1, -1, -1, -1, -1, -1, -1]])
    assert orc.isosurface(1, m.xyz().numpy(), f, 0.5)["cases"][0, 0] == 1
    assert orc.isosurface(1, m.xyz().numpy(), f, np.nextafter(0.5, 1))["cases"][0, 0] == 0


def _weld(tris):
    pts = tris.reshape(-1, 3)
    _, inv = np.unique(pts, axis=0, return_inverse=True)
    return inv.reshape(-1, 3)


@pytest.mark.parametrize("nel,N", [(2, 2), (3, 4), (4, 7)])
def test_sphere_watertight_and_oriented(orc, nel, N):
    m = si.uniform_box((nel,) * 3, (0,) * 3, (1,) * 3, N)
    f = si.sphere_field(m, (0.47, 0.52, 0.5), 0.31).numpy()
    r = orc.isosurface(N, m.xyz().numpy(), f, 0.0)
    idx = _weld(r["tris"])
    # drop zero-area triangles (two vertices welded) before the manifold check
    keep = (idx[:, 0] != idx[:, 1]) & (idx[:, 1] != idx[:, 2]) & (idx[:, 0] != idx[:, 2])
    idx = idx[keep]
    directed = {}
    for a, b, c in idx:
        for e in ((a, b), (b, c), (c, a)):
            directed[e] = directed.get(e, 0) + 1
    assert all(v == 1 for v in directed.values())
    assert all((b, a) in directed for (a, b) in directed)
    area, vol = orc.surface_measures(r["tris"])
    assert vol > 0


def test_sphere_area_volume_converge(orc):
    r0 = 0.3
    for N in (2, 4, 7):
        ea, ev = [], []
        for nel in (2, 4, 8):
            m = si.uniform_box((nel,) * 3, (0,) * 3, (1,) * 3, N)
            f = si.sphere_field(m, (0.5, 0.5, 0.5), r0).numpy()
            r = orc.isosurface(N, m.xyz().numpy(), f, 0.0)
            A, V = orc.surface_measures(r["tris"])
            ea.append(abs(A / (4 * math.pi * r0 * r0) - 1))
            ev.append(abs(V / (4 / 3 * math.pi * r0 ** 3) - 1))
        for err in (ea, ev):
            rates = [math.log2(err[i] / err[i + 1]) for i in range(2)]
            assert all(1.6 < q < 2.6 for q in rates), (N, err, rates)


def test_element_order_and_tri_elem(orc):
    w = si.tgv_box(nel=3, N=4, noise=1e-3)
    xyz = w.mesh.xyz().numpy()
    Q = orc.qcriterion(4, xyz, w.fields.numpy())
    iso = 0.1 * Q.max()
    r = orc.isosurface(4, xyz, Q, iso)
    assert r["ntri"] == r["elem_ntri"].sum()
    assert (np.diff(r["tri_elem"]) >= 0).all()
    np.testing.assert_array_equal(np.bincount(r["tri_elem"], minlength=w.E), r["elem_ntri"])
    # an element's triangles equal those of the element extracted alone
    e = int(r["tri_elem"][len(r["tri_elem"]) // 2])
    one = orc.isosurface(4, xyz[:, e:e + 1], Q[e:e + 1], iso)
    np.testing.assert_array_equal(one["tris"], r["tris"][r["tri_elem"] == e])
