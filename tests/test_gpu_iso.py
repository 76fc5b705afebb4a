"""GPU parity of sem_isosurface against the oracle (through the C ABI).

Isolated-stage comparisons: both sides get the same FP32 field, so cell cases, per-element
triangle counts, triangle counts and triangle-to-element maps are bit-exact, and vertex
positions agree within 1e-5 relative to the domain size.
"""
import math

import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import dev32, host64

pytestmark = pytest.mark.gpu


def _run_gpu(S, sess, mesh_xyz, N, f32, iso, cap=None, cases=True):
    m = sess.mesh(N, mesh_xyz)
    E = f32.shape[0]
    cs = torch.zeros(E * N ** 3, dtype=torch.uint8, device="cuda") if cases else None
    n = S.sem_isosurface(sess.ctx, m, f32, iso, None, None, cs, cap=0) if cap is None else cap
    tris = torch.full((max(n, 1) * 9,), -7.0, device="cuda")
    te = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    n2 = S.sem_isosurface(sess.ctx, m, f32, iso, tris, te, cs)
    torch.cuda.synchronize()
    return m, n2, host64(tris)[:n2 * 9].reshape(-1, 3, 3), te.cpu().numpy()[:n2], \
        (cs.cpu().numpy().reshape(E, -1) if cases else None)


def _compare(orc, N, xyz, f64, iso32, got, L):
    m, n, tris, te, cases = got
    ref = orc.isosurface(N, xyz, f64, float(iso32))
    np.testing.assert_array_equal(cases, ref["cases"])
    assert n == ref["ntri"]
    np.testing.assert_array_equal(te, ref["tri_elem"])
    if n:
        # NaN vertices (edges touching a NaN node) must match as NaN
        nan = np.isnan(ref["tris"])
        np.testing.assert_array_equal(np.isnan(tris), nan)
        assert np.abs(tris[~nan] - ref["tris"][~nan]).max() <= 1e-5 * L
    return ref


def test_all_256_cases_single_cells(gpu, sess, orc):
    # 256 elements of order 1 in a row, element c holding case c with random magnitudes
    mesh = si.uniform_box((256, 1, 1), (0, 0, 0), (256.0, 1.3, 0.7), 1)
    rng = np.random.default_rng(3)
    f = np.zeros((256, 8))
    for c in range(256):
        mag = rng.uniform(0.1, 1.0, 8)
        f[c] = [mag[v] if (c >> v) & 1 else -mag[v] for v in range(8)]
    f32 = dev32(f)
    xyz = mesh.xyz().numpy()
    got = _run_gpu(gpu, sess, xyz, 1, f32, 0.0)
    ref = _compare(orc, 1, xyz, host64(f32), np.float32(0.0), got, 256.0)
    np.testing.assert_array_equal(got[4][:, 0], np.arange(256))
    assert ref["ntri"] == orc.mc_table()[0].sum()


def test_taylor_green_q_isosurface(gpu, sess, orc):
    """8^3 elements, N=7: the oracle's Q of the FP32 velocity, rounded to FP32, is given to
    both sides; iso = 0.1 max Q."""
    w = si.tgv_box()
    xyz = w.mesh.xyz().numpy()
    vel32 = w.fields.float().double().numpy()
    Q = orc.qcriterion(7, xyz, vel32)
    q32 = dev32(Q)
    iso = np.float32(0.1 * Q.max())
    got = _run_gpu(gpu, sess, xyz, 7, q32, float(iso))
    ref = _compare(orc, 7, xyz, host64(q32), iso, got, 2 * math.pi)
    assert ref["ntri"] > 10000


@pytest.mark.parametrize("N,nel", [(2, (3, 4, 2)), (3, (5, 2, 3)), (5, (3, 3, 3)), (7, (5, 3, 3)), (9, (2, 3, 2)),
                                   (10, (2, 2, 2)), (12, (2, 1, 2)), (15, (2, 2, 1))])
def test_sphere_orders(gpu, sess, orc, N, nel):
    mesh = si.stretched_box(nel, N, seed=N)
    xyz = mesh.xyz().numpy()
    c = [(mesh.xf[0] + mesh.xf[-1]) / 2, (mesh.yf[0] + mesh.yf[-1]) / 2, (mesh.zf[0] + mesh.zf[-1]) / 2]
    r = 0.35 * min(mesh.xf[-1] - mesh.xf[0], mesh.yf[-1] - mesh.yf[0], mesh.zf[-1] - mesh.zf[0])
    f32 = dev32(si.sphere_field(mesh, c, r).numpy())
    got = _run_gpu(gpu, sess, xyz, N, f32, 0.0)
    ref = _compare(orc, N, xyz, host64(f32), np.float32(0.0), got, 10.0)
    # FP64 reductions on the GPU agree with the oracle's on the oracle's triangles
    tris = dev32(got[2].reshape(-1))
    A, V = gpu.sem_surface_measures(sess.ctx, tris, got[1])
    Ao, Vo = orc.surface_measures(ref["tris"])
    assert abs(A - Ao) < 1e-5 * Ao and abs(V - Vo) < 1e-5 * abs(Vo)
    assert V > 0


def test_capacity_error_writes_nothing(gpu, sess, orc):
    mesh = si.uniform_box((3, 3, 3), (0, 0, 0), (1, 1, 1), 4)
    f32 = dev32(si.sphere_field(mesh, (0.5, 0.5, 0.5), 0.3).numpy())
    m = sess.mesh(4, mesh.xyz().numpy())
    n = gpu.sem_isosurface(sess.ctx, m, f32, 0.0, None, cap=0)
    assert n > 0
    tris = torch.full(((n - 1) * 9,), 3.25, device="cuda")
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_isosurface(sess.ctx, m, f32, 0.0, tris)
    assert ex.value.status == gpu.SEM_ERR_CAPACITY and ex.value.required == n
    gpu.sem_synchronize(sess.ctx)
    assert (tris == 3.25).all()


def test_nan_counts_below_and_flat_elements(gpu, sess, orc):
    mesh = si.uniform_box((4, 1, 1), (0, 0, 0), (4, 1, 1), 3)
    f = si.random_nodal(mesh, 1, seed=9)[0].numpy()
    f[1] = 5.0          # all inside
    f[2] = -5.0         # all outside
    f[3, ::7] = np.nan  # NaN nodes count as below
    xyz = mesh.xyz().numpy()
    f32 = dev32(f)
    got = _run_gpu(gpu, sess, xyz, 3, f32, 0.0)
    _compare(orc, 3, xyz, host64(f32), np.float32(0.0), got, 4.0)
    assert (got[4][1] == 255).all() and (got[4][2] == 0).all()


def test_multi_isovalues_match_oracle_and_single_calls(gpu, sess, orc):
    """Three isovalues in one call: each segment equals the oracle's extraction (cases,
    counts, element map, positions) and the single-isovalue call."""
    w = si.tgv_box(nel=5, N=7)
    xyz = w.mesh.xyz().numpy()
    m = sess.mesh(7, xyz)
    u, v, ww = (dev32(w.fields[c].numpy()) for c in range(3))
    Q = torch.empty_like(u)
    gpu.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    qmax = gpu.sem_field_max(sess.ctx, Q)
    isos = [float(np.float32(f * qmax)) for f in (0.05, 0.1, 0.2, -0.05)]
    E, N3 = w.E, 343
    counts = gpu.sem_isosurface_multi(sess.ctx, m, Q, isos, None)
    tris = torch.empty(sum(counts) * 9, device="cuda")
    te = torch.empty(sum(counts), dtype=torch.int32, device="cuda")
    cs = torch.zeros(len(isos) * E * N3, dtype=torch.uint8, device="cuda")
    assert gpu.sem_isosurface_multi(sess.ctx, m, Q, isos, tris, te, cs) == counts
    torch.cuda.synchronize()
    q64 = host64(Q)
    t_h, e_h, c_h = host64(tris).reshape(-1, 3, 3), te.cpu().numpy(), cs.cpu().numpy().reshape(len(isos), E, N3)
    off = 0
    for q, iso in enumerate(isos):
        ref = orc.isosurface(7, xyz, q64, iso)
        n = counts[q]
        assert n == ref["ntri"]
        np.testing.assert_array_equal(c_h[q], ref["cases"])
        np.testing.assert_array_equal(e_h[off:off + n], ref["tri_elem"])
        assert np.abs(t_h[off:off + n] - ref["tris"]).max() <= 1e-5 * 2 * math.pi
        one = torch.empty(n * 9, device="cuda")
        assert gpu.sem_isosurface(sess.ctx, m, Q, iso, one) == n
        assert torch.equal(one, tris[off * 9:(off + n) * 9])
        off += n
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_isosurface_multi(sess.ctx, m, Q, isos, tris[:9 * (sum(counts) - 1)])
    assert ex.value.status == gpu.SEM_ERR_CAPACITY and ex.value.required == sum(counts)


def test_channel_full_size_sampled(gpu, sess, orc):
    """32^3 elements, N = 7, the benchmark's three isovalues; GPU Q on the full mesh, the
    oracle extracts 256 sampled elements from the same FP32 Q."""
    w = si.channel(device="cuda")
    xyz_d = w.mesh.xyz("cuda")
    m = sess.mesh(7, xyz_d.cpu().numpy())
    u, v, ww = (w.fields[c].float().contiguous() for c in range(3))
    Q = torch.empty_like(u)
    gpu.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    qmax = gpu.sem_field_max(sess.ctx, Q)
    assert qmax == float(Q.max())
    rng = np.random.default_rng(5)
    E = w.E
    cs = torch.zeros(E * 343, dtype=torch.uint8, device="cuda")
    for frac in w.iso_fracs:
        iso = float(np.float32(frac * qmax))
        n = gpu.sem_isosurface(sess.ctx, m, Q, iso, None, cap=0)
        tris = torch.empty(n * 9, device="cuda")
        te = torch.empty(n, dtype=torch.int32, device="cuda")
        assert gpu.sem_isosurface(sess.ctx, m, Q, iso, tris, te, cs) == n
        te_h = te.cpu().numpy()
        counts = np.bincount(te_h, minlength=E)
        starts = np.concatenate([[0], np.cumsum(counts)])
        act = np.nonzero(counts)[0]
        sample = np.sort(np.concatenate([rng.choice(E, 128, replace=False), rng.choice(act, 128, replace=False)]))
        sample = np.unique(sample)
        sidx = torch.as_tensor(sample, device="cuda")
        xs = xyz_d[:, sidx].cpu().numpy()
        qs = Q.view(E, 512)[sidx].double().cpu().numpy()
        ref = orc.isosurface(7, xs, qs, iso)
        np.testing.assert_array_equal(cs.view(E, 343)[sidx].cpu().numpy(), ref["cases"])
        np.testing.assert_array_equal(counts[sample], ref["elem_ntri"])
        tri_h = tris.view(-1, 3, 3)
        got = np.concatenate([tri_h[starts[e]:starts[e + 1]].double().cpu().numpy() for e in sample])
        assert np.abs(got - ref["tris"]).max() <= 1e-5 * 2 * math.pi


@pytest.mark.parametrize("shape", [(64, 32, 32), (65537, 1, 1)])
def test_scan_at_the_one_launch_limit(gpu, sess, orc, shape):
    """2 isovalues x 65536 elements = 131072 counts (exactly 32 tiles of 4096 of the look-back
    scan) and x 65537 = 131074 counts (33 tiles, the last holding 2 counts); counts and the
    triangles' elements against the oracle.  Per-node random values, so nearly every element
    holds triangles."""
    mesh = si.uniform_box(shape, (0, 0, 0), (1, 1, 1), 1)
    xyz = mesh.xyz().numpy()
    f32 = dev32(si.random_nodal(mesh, 1, seed=shape[0])[0].numpy())  # (E, 8)
    m = sess.mesh(1, xyz)
    isos = [0.0, 0.5]
    counts = gpu.sem_isosurface_multi(sess.ctx, m, f32, isos, None)
    tris = torch.empty(sum(counts) * 9, device="cuda")
    te = torch.empty(sum(counts), dtype=torch.int32, device="cuda")
    assert gpu.sem_isosurface_multi(sess.ctx, m, f32, isos, tris, te) == counts
    torch.cuda.synchronize()
    f64 = host64(f32)
    off = 0
    e_h = te.cpu().numpy()
    for q, iso in enumerate(isos):
        ref = orc.isosurface(1, xyz, f64, float(np.float32(iso)), want_tris=False)
        assert counts[q] == ref["ntri"]
        np.testing.assert_array_equal(e_h[off:off + counts[q]], np.repeat(np.arange(mesh.E), ref["elem_ntri"]))
        off += counts[q]


def test_emit_autotuner_choice_does_not_change_the_triangles(gpu, sess):
    """The first emitting call of an (order, elements, isovalues) picks the units per work
    atomic; the triangles are bit-identical to the untuned launch's."""
    S = gpu
    w = si.tgv_box(nel=6)
    m = sess.mesh(7, w.mesh.xyz().numpy())
    u, v, ww = (dev32(w.fields[c].numpy()) for c in range(3))
    Q = torch.empty_like(u)
    S.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    qmax = S.sem_field_max(sess.ctx, Q)
    isos = [float(np.float32(f * qmax)) for f in (0.05, 0.1, 0.2, 0.3)]
    S.sem_autotune_set(sess.ctx, True)
    counts = S.sem_isosurface_multi(sess.ctx, m, Q, isos, None)
    tuned = torch.empty(sum(counts) * 9, device="cuda")
    S.sem_isosurface_multi(sess.ctx, m, Q, isos, tuned)
    mine = [c for c in S.sem_autotune_emit_choices(sess.ctx) if c[:3] == (7, w.E, 4)]
    assert len(mine) == 1 and mine[0][3] in (1, 2, 4, 8) and mine[0][4] > 0
    again = torch.empty_like(tuned)
    S.sem_isosurface_multi(sess.ctx, m, Q, isos, again)
    assert len([c for c in S.sem_autotune_emit_choices(sess.ctx) if c[:3] == (7, w.E, 4)]) == 1
    S.sem_autotune_set(sess.ctx, False)
    assert S.sem_autotune_emit_choices(sess.ctx) == []
    plain = torch.empty_like(tuned)
    S.sem_isosurface_multi(sess.ctx, m, Q, isos, plain)
    S.sem_autotune_set(sess.ctx, True)
    torch.cuda.synchronize()
    assert torch.equal(tuned.view(torch.int32), plain.view(torch.int32))
    assert torch.equal(again.view(torch.int32), plain.view(torch.int32))


def test_many_elements_multi_isovalue_uses_the_multi_block_scan(gpu, sess, orc):
    """64^3 elements of order 1 x 2 isovalues = 524288 counts: 128 tiles of the look-back scan
    (the single-block scan takes at most 8192), so tiles fold up to four 32-tile windows of
    their predecessors; counts and offsets against the oracle."""
    mesh = si.uniform_box((64, 64, 64), (0, 0, 0), (1, 1, 1), 1)
    xyz = mesh.xyz().numpy()
    f32 = dev32(si.sphere_field(mesh, (0.5, 0.5, 0.5), 0.3).numpy())
    m = sess.mesh(1, xyz)
    isos = [0.0, 0.02]
    counts = gpu.sem_isosurface_multi(sess.ctx, m, f32, isos, None)
    tris = torch.empty(sum(counts) * 9, device="cuda")
    te = torch.empty(sum(counts), dtype=torch.int32, device="cuda")
    assert gpu.sem_isosurface_multi(sess.ctx, m, f32, isos, tris, te) == counts
    torch.cuda.synchronize()
    f64 = host64(f32)
    off = 0
    e_h = te.cpu().numpy()
    for q, iso in enumerate(isos):
        ref = orc.isosurface(1, xyz, f64, float(np.float32(iso)))
        assert counts[q] == ref["ntri"]
        np.testing.assert_array_equal(e_h[off:off + counts[q]], ref["tri_elem"])
        off += counts[q]
