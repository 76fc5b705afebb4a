"""Host-synchronisation-free frames (sem_isosurface_multi_async + sem_render_async) and their
capture in one CUDA graph per time step, against the synchronous path; batches of partitions
with uneven element counts and mixed orders in one graph."""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import host64

pytestmark = pytest.mark.gpu


class Frame:
    """Device buffers of one partition's frame: Q, triangles of all isovalues, image."""

    def __init__(self, S, ctx, w, isos, cap, mesh=None):
        self.S, self.ctx, self.w = S, ctx, w
        self.mesh = mesh if mesh is not None else S.sem_load_mesh(ctx, w.mesh.N, w.mesh.xyz().numpy())
        self.vel = [w.fields[c].float().cuda().contiguous() for c in range(3)]
        self.Q = torch.empty_like(self.vel[0])
        self.isos = isos
        self.cap = cap
        self.tris = torch.full((cap * 9,), -1.0, device="cuda")
        self.counts = torch.zeros(len(isos) + 1, dtype=torch.int64, device="cuda")
        W, H = w.camera["W"], w.camera["H"]
        self.rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
        self.depth = torch.zeros(H * W, device="cuda")

    def run(self):
        S = self.S
        S.sem_qcriterion(self.ctx, self.mesh, *self.vel, self.Q)
        S.sem_isosurface_multi_async(self.ctx, self.mesh, self.Q, self.isos, self.tris, self.counts, cap=self.cap)
        S.sem_render_async(self.ctx, self.tris, self.cap, self.counts, len(self.isos), None, self.w.camera,
                           self.w.camera["W"], self.w.camera["H"], self.rgba, self.depth)


def _sync_reference(S, ctx, mesh, vel, isos, cam):
    Q = torch.empty_like(vel[0])
    S.sem_qcriterion(ctx, mesh, *vel, Q)
    counts = S.sem_isosurface_multi(ctx, mesh, Q, isos, None)
    tris = torch.empty(max(1, sum(counts)) * 9, device="cuda")
    S.sem_isosurface_multi(ctx, mesh, Q, isos, tris)
    W, H = cam["W"], cam["H"]
    rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
    depth = torch.zeros(H * W, device="cuda")
    S.sem_render(ctx, tris, sum(counts), counts, None, cam, W, H, rgba, depth)
    torch.cuda.synchronize()
    return counts, tris[:sum(counts) * 9].clone(), rgba.clone(), depth.clone()


def test_async_frame_equals_sync(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=6)
    isos = [0.05, 0.2, 0.4]
    fr = Frame(S, sess.ctx, w, isos, cap=400000)
    fr.run()
    S.sem_synchronize(sess.ctx)
    counts, tris, rgba, depth = _sync_reference(S, sess.ctx, fr.mesh, fr.vel, isos, w.camera)
    starts = fr.counts.cpu().numpy()
    assert list(np.diff(starts)) == counts and starts[0] == 0
    assert torch.equal(fr.tris[:sum(counts) * 9], tris)
    assert torch.equal(fr.rgba, rgba) and torch.equal(fr.depth, depth)
    S.sem_mesh_free(fr.mesh)


def test_graph_replay_on_new_snapshots(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=6)
    isos = [0.05, 0.2, 0.4]
    fr = Frame(S, sess.ctx, w, isos, cap=400000)
    fr.run()  # sizes the library's scratch before capture
    S.sem_synchronize(sess.ctx)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        fr.run()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    for snap in (1, 2):
        ws = si.tgv_box(nel=6, snapshot=snap, phase=0.3 * snap)
        for c in range(3):
            fr.vel[c].copy_(ws.fields[c].float())
        g.replay()
        torch.cuda.synchronize()
        S.sem_synchronize(sess.ctx)
        g_rgba, g_depth = fr.rgba.clone(), fr.depth.clone()
        counts, tris, rgba, depth = _sync_reference(S, sess.ctx, fr.mesh, fr.vel, isos, w.camera)
        assert list(np.diff(fr.counts.cpu().numpy())) == counts
        assert torch.equal(fr.tris[:sum(counts) * 9], tris)
        fr.run()  # the same frame, eager
        torch.cuda.synchronize()
        assert torch.equal(g_rgba, rgba) and torch.equal(g_depth, depth), snap
        assert torch.equal(fr.rgba, rgba) and torch.equal(fr.depth, depth), snap
    S.sem_mesh_free(fr.mesh)


def test_async_render_ignores_triangles_past_the_device_count(gpu, sess):
    """The device count, not ntri_max, bounds the rasterised triangles: a buffer whose tail
    holds valid triangles past the count renders like the synchronous call on the prefix
    (the raster grid is sized by ntri_max, so most of its blocks have nothing to do)."""
    S = gpu
    w = si.tgv_box(nel=6)
    fr = Frame(S, sess.ctx, w, [0.05, 0.2], cap=200000)
    fr.run()
    S.sem_synchronize(sess.ctx)
    n = int(fr.counts[-1])
    keep = n // 5
    cam, W, H = w.camera, w.camera["W"], w.camera["H"]
    for k in (0, 1, keep, n):
        cnt = torch.tensor([0, min(k, int(fr.counts[1])), k], dtype=torch.int64, device="cuda")
        rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
        depth = torch.zeros(H * W, device="cuda")
        S.sem_render_async(sess.ctx, fr.tris, n, cnt, 2, None, cam, W, H, rgba, depth)
        segs = [int(cnt[1]), k - int(cnt[1])]
        r2 = torch.zeros_like(rgba)
        d2 = torch.zeros_like(depth)
        torch.cuda.synchronize()
        S.sem_render(sess.ctx, fr.tris[:max(k, 1) * 9].clone(), k, segs, None, cam, W, H, r2, d2)
        torch.cuda.synchronize()
        assert torch.equal(rgba, r2) and torch.equal(depth, d2), k
        if k == 0:
            assert (rgba == 0).all() and (depth == 1.0).all()
    S.sem_mesh_free(fr.mesh)


def test_async_overflow_is_flagged_and_writes_nothing(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=4)
    fr = Frame(S, sess.ctx, w, [0.1], cap=50)
    S.sem_qcriterion(sess.ctx, fr.mesh, *fr.vel, fr.Q)
    S.sem_isosurface_multi_async(sess.ctx, fr.mesh, fr.Q, [0.1], fr.tris, fr.counts, cap=50)
    with pytest.raises(S.SemError) as ex:
        S.sem_synchronize(sess.ctx)
    assert ex.value.status == S.SEM_ERR_CAPACITY
    assert fr.counts[-1].item() > 50
    assert (fr.tris == -1.0).all()
    S.sem_synchronize(sess.ctx)  # the flag was cleared
    S.sem_mesh_free(fr.mesh)


def test_batched_partitions_mixed_orders_one_graph(gpu, sess, orc):
    """Partitions of uneven element counts and orders N in {5, 7, 9}, two fields (Q and the
    x-velocity) x 4 isovalues each, all captured in one CUDA graph per time step; checked
    against the oracle's isosurfaces (cases are bit-exact, so triangle counts match)."""
    S = gpu
    rng = np.random.default_rng(si.seed_for(4))
    parts = []
    for p in range(5):
        N = int(rng.choice([5, 7, 9]))
        nel = (int(rng.integers(2, 5)), int(rng.integers(2, 5)), int(rng.integers(1, 4)))
        lo = np.array([p * 1.3, 0.0, 0.0])
        mesh = si.uniform_box(nel, lo, lo + np.array([1.2, 1.5, 1.1]), N)
        vel = si.taylor_green(mesh, 1e-3, si.seed_for(4, p), phase=0.2 * p)
        cam = si.box_camera_persp(lo, lo + np.array([1.2, 1.5, 1.1]), 96, 64)
        parts.append((mesh, vel, cam))
    frames = []
    for mesh, vel, cam in parts:
        w = si.Workload("part", 4, mesh, [], cam, vel)
        f = Frame(S, sess.ctx, w, [-0.2, -0.05, 0.05, 0.2], cap=200000)
        f.ufield = f.vel[0]
        f.tris2 = torch.zeros(200000 * 9, device="cuda")
        f.counts2 = torch.zeros(5, dtype=torch.int64, device="cuda")
        frames.append(f)

    def step():
        for f in frames:
            f.run()
            S.sem_isosurface_multi_async(sess.ctx, f.mesh, f.ufield, [-0.5, 0.0, 0.25, 0.5], f.tris2, f.counts2)

    step()
    S.sem_synchronize(sess.ctx)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        step()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    for f in frames:
        f.Q.zero_()
    g.replay()
    torch.cuda.synchronize()
    S.sem_synchronize(sess.ctx)
    for f, (mesh, vel, cam) in zip(frames, parts):
        xyz = mesh.xyz().numpy()
        for field, isos, counts in ((host64(f.Q), f.isos, f.counts), (host64(f.ufield), [-0.5, 0.0, 0.25, 0.5],
                                                                      f.counts2)):
            c = counts.cpu().numpy()
            for q, iso in enumerate(isos):
                ref = orc.isosurface(mesh.N, xyz, field, float(np.float32(iso)), want_tris=False)
                assert c[q + 1] - c[q] == ref["ntri"], (mesh.N, q)
        S.sem_mesh_free(f.mesh)


def test_qcriterion_batch_equals_per_partition_calls(gpu, sess):
    """12 partitions of uneven element counts (including counts that leave partial 4-element
    groups) and mixed orders in one batch call: Q bit-identical to one call per partition,
    also when the batch call is captured in a CUDA graph."""
    S = gpu
    rng = np.random.default_rng(si.seed_for(4, 77))
    parts = []
    for p in range(12):
        N = int(rng.choice([5, 7, 9]))
        nel = (int(rng.integers(1, 6)), int(rng.integers(1, 6)), int(rng.integers(1, 5)))
        lo = np.array([p * 1.1, 0.3, 0.0])
        mesh = si.uniform_box(nel, lo, lo + np.array([1.0, 1.3, 0.9]), N)
        vel = si.taylor_green(mesh, 1e-3, si.seed_for(4, 100 + p), phase=0.1 * p)
        m = sess.mesh(N, mesh.xyz().numpy())
        f = [vel[c].float().cuda().contiguous() for c in range(3)]
        parts.append((m, f))
    metas = [m for m, _ in parts]
    us, vs, ws = ([f[c] for _, f in parts] for c in range(3))
    ref = []
    for m, f in parts:
        q = torch.empty_like(f[0])
        S.sem_qcriterion(sess.ctx, m, *f, q)
        ref.append(q)
    got = [torch.full_like(f[0], float("nan")) for _, f in parts]
    S.sem_qcriterion_batch(sess.ctx, metas, us, vs, ws, got)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    # captured
    got2 = [torch.full_like(f[0], float("nan")) for _, f in parts]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        S.sem_qcriterion_batch(sess.ctx, metas, us, vs, ws, got2)
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    S.sem_synchronize(sess.ctx)
    for a, b in zip(got2, ref):
        assert torch.equal(a, b)


def _two_field_case(nel=5):
    """The Rayleigh-Benard-like field on a small box: velocity (Q) and temperature."""
    import math
    mesh = si.BoxMesh(7, np.linspace(0, 2 * math.pi, nel + 1), np.linspace(0, 2 * math.pi, nel + 1),
                      np.linspace(0, 1.0, nel + 1))
    f = si.rayleigh_benard(mesh, 64, si.seed_for(3, 5))
    cam = si.box_camera_persp((0.0, 0.0, 0.0), (2 * math.pi, 2 * math.pi, 1.0), 320, 180,
                              direction=(1.0, -1.2, 0.8), up=(0.0, 0.0, 1.0))
    return mesh, f, cam


def test_append_second_field_in_one_graph(gpu, sess):
    """Q isosurfaces then the temperature's appended behind them on the device (counts_dev[0] of
    the second call is the first call's total), drawn by one sem_render_async as consecutive
    segments, captured in one graph: triangles, segment starts and frame equal the
    host-synchronised calls written back to back."""
    S = gpu
    mesh, f, cam = _two_field_case()
    m = sess.mesh(7, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    T = f[3].float().cuda().contiguous()
    Q = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Q)
    qmax = S.sem_field_max(sess.ctx, Q)
    qisos = [float(np.float32(0.1 * qmax)), float(np.float32(0.3 * qmax))]
    tisos = [0.5]
    cq = S.sem_isosurface_multi(sess.ctx, m, Q, qisos, None)
    ct = S.sem_isosurface_multi(sess.ctx, m, T, tisos, None)
    nq, nt = sum(cq), sum(ct)
    assert nq > 0 and nt > 0
    ref = torch.empty((nq + nt) * 9, device="cuda")
    S.sem_isosurface_multi(sess.ctx, m, Q, qisos, ref[:nq * 9])
    S.sem_isosurface_multi(sess.ctx, m, T, tisos, ref[nq * 9:])
    W, H = cam["W"], cam["H"]
    cols = [[0.9, 0.3, 0.2], [0.7, 0.2, 0.1], [0.2, 0.5, 0.9]]
    r_rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
    r_depth = torch.zeros(H * W, device="cuda")
    S.sem_render(sess.ctx, ref, nq + nt, cq + ct, cols, cam, W, H, r_rgba, r_depth)
    cap = nq + nt + 100
    tris = torch.full((cap * 9,), -1.0, device="cuda")
    cnt = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    rgba = torch.zeros_like(r_rgba)
    depth = torch.zeros_like(r_depth)

    def step():
        S.sem_isosurface_multi_async(sess.ctx, m, Q, qisos, tris, cnt[:3], cap=cap)
        S.sem_isosurface_multi_append_async(sess.ctx, m, T, tisos, tris, cnt[2:], cap=cap)
        S.sem_render_async(sess.ctx, tris, cap, cnt, 3, cols, cam, W, H, rgba, depth)

    step()
    S.sem_synchronize(sess.ctx)
    assert cnt.cpu().tolist() == [0, cq[0], nq, nq + nt]
    assert torch.equal(tris[:(nq + nt) * 9], ref)
    assert (tris[(nq + nt) * 9:] == -1.0).all()
    assert torch.equal(rgba, r_rgba) and torch.equal(depth, r_depth)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        step()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    tris.fill_(-1.0)
    rgba.zero_()
    cnt.fill_(-7)
    g.replay()
    S.sem_synchronize(sess.ctx)
    assert cnt.cpu().tolist() == [0, cq[0], nq, nq + nt]
    assert torch.equal(tris[:(nq + nt) * 9], ref)
    assert torch.equal(rgba, r_rgba) and torch.equal(depth, r_depth)


def test_append_overflow_is_flagged_and_writes_nothing(gpu, sess):
    """An append whose start plus its own total exceeds the buffer writes no triangle and raises
    the capacity flag; the segment ends still report the required size."""
    S = gpu
    mesh, f, _ = _two_field_case(nel=3)
    m = sess.mesh(7, mesh.xyz().numpy())
    T = f[3].float().cuda().contiguous()
    nt = S.sem_isosurface_multi(sess.ctx, m, T, [0.5], None)[0]
    assert nt > 10
    cap = nt + 5
    tris = torch.full((cap * 9,), -1.0, device="cuda")
    cnt = torch.tensor([10, -1], dtype=torch.int64, device="cuda")  # 10 + nt > cap
    S.sem_isosurface_multi_append_async(sess.ctx, m, T, [0.5], tris, cnt, cap=cap)
    with pytest.raises(S.SemError) as ex:
        S.sem_synchronize(sess.ctx)
    assert ex.value.status == S.SEM_ERR_CAPACITY
    assert cnt.cpu().tolist() == [10, 10 + nt]
    assert (tris == -1.0).all()
    cnt = torch.tensor([5, -1], dtype=torch.int64, device="cuda")  # fits exactly
    S.sem_isosurface_multi_append_async(sess.ctx, m, T, [0.5], tris, cnt, cap=cap)
    S.sem_synchronize(sess.ctx)
    ref = torch.empty(nt * 9, device="cuda")
    S.sem_isosurface_multi(sess.ctx, m, T, [0.5], ref)
    assert torch.equal(tris[5 * 9:], ref) and (tris[:5 * 9] == -1.0).all()


@pytest.mark.parametrize("N,nel,isos", [(7, (6, 6, 6), [0.05, 0.2, 0.4]), (7, (7, 5, 3), [0.1]),
                                        (7, (1, 1, 1), [0.1, 0.3]), (5, (4, 3, 3), [0.1, 0.2])])
def test_fused_q_isosurface_equals_separate_calls(gpu, sess, N, nel, isos):
    """sem_qcriterion_isosurface_async (for N = 7 the counting pass runs inside the Q kernel)
    against sem_qcriterion + sem_isosurface_multi_async on the same velocity: Q, segment starts
    and triangles bit for bit, eager and replayed from a CUDA graph; element counts that leave a
    partial 4-element group, a single element, and an order that runs the passes unfused."""
    S = gpu
    import math
    mesh = si.uniform_box(nel, (0.0,) * 3, (2 * math.pi,) * 3, N)
    m = sess.mesh(N, mesh.xyz().numpy())
    f = si.taylor_green(mesh, 1e-3, si.seed_for(1, 9))
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    Q0 = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Q0)
    counts = S.sem_isosurface_multi(sess.ctx, m, Q0, isos, None)
    cap = sum(counts) + 64
    ref_t = torch.full((cap * 9,), -1.0, device="cuda")
    ref_c = torch.zeros(len(isos) + 1, dtype=torch.int64, device="cuda")
    S.sem_isosurface_multi_async(sess.ctx, m, Q0, isos, ref_t, ref_c, cap=cap)
    Q = torch.full_like(vel[0], float("nan"))
    tris = torch.full((cap * 9,), -1.0, device="cuda")
    cnt = torch.full((len(isos) + 1,), -5, dtype=torch.int64, device="cuda")

    def fused():
        S.sem_qcriterion_isosurface_async(sess.ctx, m, *vel, Q, isos, tris, cnt, cap=cap)

    fused()
    S.sem_synchronize(sess.ctx)
    assert torch.equal(Q, Q0)
    assert torch.equal(cnt, ref_c) and int(cnt[-1]) == sum(counts)
    assert torch.equal(tris, ref_t)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        fused()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    Q.fill_(float("nan"))
    tris.fill_(-1.0)
    cnt.fill_(-5)
    g.replay()
    S.sem_synchronize(sess.ctx)
    assert torch.equal(Q, Q0) and torch.equal(cnt, ref_c) and torch.equal(tris, ref_t)


def test_fused_q_isosurface_overflow_is_flagged(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=4)
    m = sess.mesh(7, w.mesh.xyz().numpy())
    vel = [w.fields[c].float().cuda().contiguous() for c in range(3)]
    Q = torch.empty_like(vel[0])
    tris = torch.full((50 * 9,), -1.0, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    S.sem_qcriterion_isosurface_async(sess.ctx, m, *vel, Q, [0.1], tris, cnt, cap=50)
    with pytest.raises(S.SemError) as ex:
        S.sem_synchronize(sess.ctx)
    assert ex.value.status == S.SEM_ERR_CAPACITY
    assert int(cnt[-1]) > 50 and (tris == -1.0).all()


def test_batching_partitions_against_the_oracle_sampled(gpu, sess, orc):
    """The batching workload's partitions at full size (16 partitions of U{4096..40960} elements,
    orders 5, 7 and 9), snapshot 1: Q of all partitions in one batched call, then the Q and u
    isosurfaces at the workload's four isovalues.  On 48 seeded sampled elements per partition,
    Q within its per-node bound and every cell's case equal the oracle's (from the GPU's FP32 Q
    for the isosurface), and the elements' triangle counts equal the oracle's."""
    import math
    from _helpers import box_factors, grad_bounds, q_bound
    S = gpu
    parts = si.batching_partitions()
    for p in parts:
        p["xyz"] = p["mesh"].xyz_range(0, p["E"])
        p["m"] = sess.mesh(p["N"], p["xyz"])
        p["vel"] = si.taylor_green_snapshots(p["mesh"], p["E"], [2 * math.pi / 64], 1e-3, si.seed_for(4, 17))[0]
        p["Q"] = torch.empty(p["E"] * (p["N"] + 1) ** 3, device="cuda")
    S.sem_qcriterion_batch(sess.ctx, [p["m"] for p in parts], [p["vel"][0].reshape(-1) for p in parts],
                           [p["vel"][1].reshape(-1) for p in parts], [p["vel"][2].reshape(-1) for p in parts],
                           [p["Q"] for p in parts])
    qmax = max(S.sem_field_max(sess.ctx, p["Q"]) for p in parts)
    umax = max(S.sem_field_max(sess.ctx, p["vel"][0].reshape(-1)) for p in parts)
    fr = (0.05, 0.1, 0.2, 0.4)
    isos = [[float(np.float32(f * qmax)) for f in fr], [float(np.float32(f * umax)) for f in fr]]
    rng = np.random.default_rng(si.seed_for(4, 3))
    for p in parts:
        N, E = p["N"], p["E"]
        NP3, N3 = (N + 1) ** 3, N ** 3
        sample = np.sort(rng.choice(E, 48, replace=False))
        st = torch.as_tensor(sample, device="cuda")
        vel = p["vel"][:, st].double().cpu().numpy()
        xs = p["xyz"][:, sample]
        J = orc.gradient(N, xs, vel)
        ref = orc.q_from_gradient(J)
        Qs = p["Q"].view(E, NP3)[st].double().cpu().numpy()
        dJ = np.stack([grad_bounds(orc.dmat(N), vel[c], box_factors(xs), N + 1, J[c]) for c in range(3)])
        assert (np.abs(Qs - ref) <= q_bound(J, dJ)).all(), (N, E)
        for f, fld in enumerate((p["Q"], p["vel"][0].reshape(-1))):
            cs = torch.empty(4 * E * N3, dtype=torch.uint8, device="cuda")
            counts = S.sem_isosurface_multi(sess.ctx, p["m"], fld, isos[f], None, cases=cs)
            tris = torch.empty(max(1, sum(counts)) * 9, device="cuda")
            te = torch.empty(max(1, sum(counts)), dtype=torch.int32, device="cuda")
            S.sem_isosurface_multi(sess.ctx, p["m"], fld, isos[f], tris, tri_elem=te)
            starts = np.concatenate([[0], np.cumsum(counts)])
            tev = te.cpu().numpy()
            fs = fld.view(E, NP3)[st].double().cpu().numpy()
            for q in range(4):
                r = orc.isosurface(N, xs, fs, isos[f][q], want_tris=False)
                got = cs.view(4, E, N3)[q][st].cpu().numpy()
                np.testing.assert_array_equal(got, r["cases"])
                per_elem = np.bincount(tev[starts[q]:starts[q + 1]], minlength=E)[sample]
                np.testing.assert_array_equal(per_elem, r["elem_ntri"])
