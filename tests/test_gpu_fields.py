"""sem_qcriterion_isosurface_fields_async: Q with its isosurfaces and further fields' isosurfaces
in one call, the further fields' passes on the context's auxiliary stream.

The call must equal the call sequence it stands for -- sem_qcriterion_isosurface_async then one
sem_isosurface_multi_append_async per field -- bit for bit (Q, triangles, triangle elements,
segment starts): on its first call (the emit autotuner still timing, so one stream), on later
eager calls and with tuning off (forked), and replayed from a CUDA graph (forked under capture).
Results must be complete in the caller's stream order when the call returns: a kernel queued on
the caller's stream right after the call sees every segment.
"""
import math

import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu


def _case(N, nel):
    mesh = si.BoxMesh(N, np.linspace(0, 2 * math.pi, nel + 1), np.linspace(0, 2 * math.pi, nel + 1),
                      np.linspace(0, 1.0, nel + 1))
    f = si.rayleigh_benard(mesh, 64, si.seed_for(3, 6))
    return mesh, f


def _reference(S, ctx, m, vel, T, qisos, fields, fisos, E):
    """The separate calls, host-synchronised: Q, triangles, triangle elements, segment starts."""
    Q = torch.empty_like(vel[0])
    S.sem_qcriterion(ctx, m, *vel, Q)
    counts = [S.sem_isosurface_multi(ctx, m, Q, qisos, None)]
    counts += [S.sem_isosurface_multi(ctx, m, f, iv, None) for f, iv in zip(fields, fisos)]
    total = sum(sum(c) for c in counts)
    tris = torch.empty(max(total, 1) * 9, device="cuda")
    te = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    at = 0
    for f, iv, c in zip([Q] + list(fields), [qisos] + list(fisos), counts):
        n = sum(c)
        S.sem_isosurface_multi(ctx, m, f, iv, tris[at * 9:(at + n) * 9], tri_elem=te[at:at + n])
        at += n
    starts = [0]
    for c in counts:
        for x in c:
            starts.append(starts[-1] + x)
    torch.cuda.synchronize()
    return Q, tris[:total * 9].clone(), te[:total].clone(), starts, total


@pytest.mark.parametrize("N,nel", [(7, 5), (7, 3), (5, 4)])
def test_fields_call_equals_the_call_sequence(gpu, sess, N, nel):
    S = gpu
    mesh, f = _case(N, nel)
    m = sess.mesh(N, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    T = f[3].float().cuda().contiguous()
    U = vel[0].clone()  # a second further field: the first velocity component at two levels
    Qr = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Qr)
    qmax = S.sem_field_max(sess.ctx, Qr)
    qisos = [float(np.float32(0.1 * qmax)), float(np.float32(0.3 * qmax))]
    fields, fisos = [T, U], [[0.5], [0.0, 0.05]]
    Q0, ref_t, ref_e, starts, total = _reference(S, sess.ctx, m, vel, T, qisos, fields, fisos, mesh.E)
    assert total > 0 and all(b > a for a, b in zip(starts[2:], starts[3:])), starts
    cap = total + 77
    Q = torch.empty_like(vel[0])
    tris = torch.empty(cap * 9, device="cuda")
    te = torch.empty(cap, dtype=torch.int32, device="cuda")
    cnt = torch.empty(len(starts), dtype=torch.int64, device="cuda")

    def call():
        S.sem_qcriterion_isosurface_fields_async(sess.ctx, m, *vel, Q, qisos, fields, fisos, tris, cnt,
                                                 tri_elem=te, cap=cap)

    def check(label):
        # queued on the caller's stream right behind the call: must see the joined results
        snap = (Q.clone(), tris[:total * 9].clone(), te[:total].clone(), cnt.clone())
        S.sem_synchronize(sess.ctx)
        assert torch.equal(snap[0], Q0), label
        assert snap[3].cpu().tolist() == starts, (label, snap[3].cpu().tolist(), starts)
        assert torch.equal(snap[1], ref_t), label
        assert torch.equal(snap[2], ref_e), label
        assert (tris[total * 9:] == -2.0).all(), label  # nothing past the total

    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    for label in ("first call (tuning)", "second call (forked)"):
        Q.fill_(float("nan"))
        tris.fill_(-2.0)
        te.fill_(-1)
        cnt.fill_(-9)
        call()
        check(label)
    # the call's kernels (one stream while tracing): on N = 7 box meshes Q's triangles are
    # counted by the Q kernel, the further fields' by the counting pass
    S.sem_trace_enable(sess.ctx, True)
    S.sem_trace_collect(sess.ctx)
    call()
    S.sem_synchronize(sess.ctx)
    names = S.sem_trace_collect(sess.ctx)
    S.sem_trace_enable(sess.ctx, False)
    if N == 7:
        assert names["k_sem_q8_count"][1] == 1 and names["k_iso_count_p"][1] == 2, names
    else:
        assert "k_sem_q8_count" not in names and names["k_iso_count_p"][1] == 3, names
    assert names["k_iso_emit_m"][1] == 3, names
    check("traced")
    S.sem_autotune_set(sess.ctx, False)
    try:
        Q.fill_(float("nan"))
        tris.fill_(-2.0)
        te.fill_(-1)
        cnt.fill_(-9)
        call()
        check("tuning off")
    finally:
        S.sem_autotune_set(sess.ctx, True)
    call()  # sizes scratch and settles the tuner outside the capture
    S.sem_synchronize(sess.ctx)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        call()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    for rep in range(2):
        Q.fill_(float("nan"))
        tris.fill_(-2.0)
        te.fill_(-1)
        cnt.fill_(-9)
        g.replay()
        check(f"graph replay {rep}")


def test_no_further_fields_equals_the_fused_call(gpu, sess):
    S = gpu
    mesh, f = _case(7, 4)
    m = sess.mesh(7, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    Q0 = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Q0)
    isos = [float(np.float32(0.2 * S.sem_field_max(sess.ctx, Q0)))]
    n = sum(S.sem_isosurface_multi(sess.ctx, m, Q0, isos, None))
    out = []
    for fields_call in (False, True):
        Q = torch.empty_like(vel[0])
        tris = torch.full(((n + 5) * 9,), -1.0, device="cuda")
        cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
        if fields_call:
            S.sem_qcriterion_isosurface_fields_async(sess.ctx, m, *vel, Q, isos, [], [], tris, cnt)
        else:
            S.sem_qcriterion_isosurface_async(sess.ctx, m, *vel, Q, isos, tris, cnt)
        S.sem_synchronize(sess.ctx)
        out.append((Q, tris, cnt))
    assert all(torch.equal(a, b) for a, b in zip(*out))
    assert out[1][2].cpu().tolist() == [0, n]


def test_overflowing_field_writes_nothing_of_it_or_later(gpu, sess):
    """cap covers Q's and the first field's triangles but not the second's: those two segments
    are written, the second field's and the third's are not, the capacity flag is raised and
    the segment starts still report the sizes needed."""
    S = gpu
    mesh, f = _case(7, 4)
    m = sess.mesh(7, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    T = f[3].float().cuda().contiguous()
    U = vel[0].clone()
    Qr = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Qr)
    qisos = [float(np.float32(0.1 * S.sem_field_max(sess.ctx, Qr)))]
    fields, fisos = [T, U, T], [[0.5], [0.0], [0.45]]
    _, ref_t, _, starts, total = _reference(S, sess.ctx, m, vel, T, qisos, fields, fisos, mesh.E)
    cap = starts[2] + (starts[3] - starts[2]) // 2  # inside the second field's segment
    tris = torch.full((cap * 9,), -3.0, device="cuda")
    cnt = torch.empty(len(starts), dtype=torch.int64, device="cuda")
    Q = torch.empty_like(vel[0])
    for rep in range(2):  # the tuning call, then the forked one
        tris.fill_(-3.0)
        S.sem_qcriterion_isosurface_fields_async(sess.ctx, m, *vel, Q, qisos, fields, fisos, tris, cnt, cap=cap)
        with pytest.raises(S.SemError) as ex:
            S.sem_synchronize(sess.ctx)
        assert ex.value.status == S.SEM_ERR_CAPACITY
        assert cnt.cpu().tolist() == starts
        assert torch.equal(tris[:starts[2] * 9], ref_t[:starts[2] * 9])
        assert (tris[starts[2] * 9:] == -3.0).all()


def test_fields_call_argument_errors(gpu, sess):
    S = gpu
    mesh, f = _case(7, 2)
    m = sess.mesh(7, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    T = f[3].float().cuda().contiguous()
    Q = torch.empty_like(vel[0])
    tris = torch.empty(900, device="cuda")
    cnt = torch.zeros(12, dtype=torch.int64, device="cuda")
    bad = [
        dict(fields=[T] * (S.SEM_MAX_FIELDS + 1), fisos=[[0.5]] * (S.SEM_MAX_FIELDS + 1)),
        dict(fields=[T], fisos=[[]]),
        dict(fields=[T], fisos=[[float("nan")]]),
        dict(fields=[Q], fisos=[[0.5]]),
        dict(fields=[T], fisos=[[0.5] * (S.SEM_MAX_ISO + 1)]),
    ]
    for kw in bad:
        with pytest.raises(S.SemError) as ex:
            S.sem_qcriterion_isosurface_fields_async(sess.ctx, m, *vel, Q, [0.1], kw["fields"], kw["fisos"], tris, cnt)
        assert ex.value.status == S.SEM_ERR_ARG, kw


@pytest.mark.parametrize("N,nel", [(7, 5), (5, 4)])
def test_frame_call_equals_fields_call_and_render(gpu, sess, N, nel):
    """sem_frame_async against sem_qcriterion_isosurface_fields_async + sem_render_async: frame
    (RGBA and depth), triangles and segment starts bit for bit -- on its first call (the render's
    launch widths still to be chosen: the two calls as such), later calls (each stream draws its
    own segments, one resolve), traced (one stream), with tuning off, and replayed from a graph."""
    S = gpu
    mesh, f = _case(N, nel)
    m = sess.mesh(N, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    T = f[3].float().cuda().contiguous()
    U = vel[0].clone()
    Qr = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Qr)
    qisos = [float(np.float32(0.1 * S.sem_field_max(sess.ctx, Qr)))]
    fields, fisos = [T, U], [[0.5], [0.0, 0.05]]
    nseg = 1 + 1 + 2
    cols = [[0.9, 0.3, 0.2], [0.2, 0.5, 0.9], [0.3, 0.8, 0.3], [0.8, 0.8, 0.2]]
    cam = si.box_camera_persp((0.0, 0.0, 0.0), (2 * math.pi, 2 * math.pi, 1.0), 320, 180,
                              direction=(1.0, -1.2, 0.8), up=(0.0, 0.0, 1.0))
    W, H = cam["W"], cam["H"]
    total = sum(sum(S.sem_isosurface_multi(sess.ctx, m, x, iv, None)) for x, iv in ((Qr, qisos), (T, [0.5]),
                                                                                (U, [0.0, 0.05])))
    cap = total + 64
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    S.sem_autotune_set(sess.ctx, False)  # the reference at the default launch widths
    Q = torch.empty_like(vel[0])
    rt = torch.full((cap * 9,), -2.0, device="cuda")
    rc = torch.empty(nseg + 1, dtype=torch.int64, device="cuda")
    r_rgba = torch.empty(H * W * 4, dtype=torch.uint8, device="cuda")
    r_depth = torch.empty(H * W, device="cuda")
    S.sem_qcriterion_isosurface_fields_async(sess.ctx, m, *vel, Q, qisos, fields, fisos, rt, rc, cap=cap)
    S.sem_render_async(sess.ctx, rt, cap, rc, nseg, cols, cam, W, H, r_rgba, r_depth)
    S.sem_synchronize(sess.ctx)
    assert int(rc[-1]) == total and (r_rgba.view(H, W, 4)[..., 3] == 255).float().mean() > 0.05
    S.sem_autotune_set(sess.ctx, True)
    tris = torch.empty_like(rt)
    cnt = torch.empty_like(rc)
    rgba = torch.empty_like(r_rgba)
    depth = torch.empty_like(r_depth)

    def call():
        S.sem_frame_async(sess.ctx, m, *vel, Q, qisos, fields, fisos, tris, cnt, cols, cam, W, H, rgba, depth,
                          cap=cap)

    def check(label):
        snap = (rgba.clone(), depth.clone(), tris.clone(), cnt.clone())
        S.sem_synchronize(sess.ctx)
        assert torch.equal(snap[3], rc), label
        assert torch.equal(snap[2], rt), label
        assert torch.equal(snap[0], r_rgba), label
        assert torch.equal(snap[1], r_depth), label

    def reset():
        tris.fill_(-2.0)
        cnt.fill_(-9)
        rgba.fill_(7)
        depth.fill_(-1.0)

    for label in ("first call (tuning)", "second call (in parts)"):
        reset()
        call()
        check(label)
    S.sem_trace_enable(sess.ctx, True)
    S.sem_trace_collect(sess.ctx)
    reset()
    call()
    S.sem_synchronize(sess.ctx)
    names = S.sem_trace_collect(sess.ctx)
    S.sem_trace_enable(sess.ctx, False)
    # Q's part from the buffer's start as one tile per block, the T and U parts as ranges
    assert names["k_raster_small"][1] == 1 and names["k_raster_range"][1] == 2, names
    assert names["k_resolve"][1] == 1, names
    check("traced")
    S.sem_autotune_set(sess.ctx, False)
    try:
        reset()
        call()
        check("tuning off")
    finally:
        S.sem_autotune_set(sess.ctx, True)
    call()  # settles the tuners outside the capture
    S.sem_synchronize(sess.ctx)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        call()
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    for rep in range(2):
        reset()
        g.replay()
        check(f"graph replay {rep}")


def test_frame_call_without_further_fields(gpu, sess):
    """No further fields: the fused call and one render, as such (k_raster_small, no parts)."""
    S = gpu
    mesh, f = _case(7, 4)
    m = sess.mesh(7, mesh.xyz().numpy())
    vel = [f[c].float().cuda().contiguous() for c in range(3)]
    Q0 = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Q0)
    isos = [float(np.float32(x * S.sem_field_max(sess.ctx, Q0))) for x in (0.1, 0.3)]
    n = sum(S.sem_isosurface_multi(sess.ctx, m, Q0, isos, None))
    cam = si.box_camera_persp((0.0, 0.0, 0.0), (2 * math.pi, 2 * math.pi, 1.0), 200, 120,
                              direction=(1.0, -1.2, 0.8), up=(0.0, 0.0, 1.0))
    W, H = cam["W"], cam["H"]
    out = []
    for frame_call in (False, True):
        Q = torch.empty_like(vel[0])
        tris = torch.full(((n + 5) * 9,), -1.0, device="cuda")
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
        depth = torch.zeros(H * W, device="cuda")
        S.sem_trace_enable(sess.ctx, True)
        S.sem_trace_collect(sess.ctx)
        if frame_call:
            S.sem_frame_async(sess.ctx, m, *vel, Q, isos, [], [], tris, cnt, None, cam, W, H, rgba, depth)
        else:
            S.sem_qcriterion_isosurface_async(sess.ctx, m, *vel, Q, isos, tris, cnt)
            S.sem_render_async(sess.ctx, tris, n + 5, cnt, 2, None, cam, W, H, rgba, depth)
        S.sem_synchronize(sess.ctx)
        names = S.sem_trace_collect(sess.ctx)
        S.sem_trace_enable(sess.ctx, False)
        assert "k_raster_range" not in names and names["k_raster_small"][1] == 1, names
        out.append((Q, tris, cnt, rgba, depth))
    assert all(torch.equal(a, b) for a, b in zip(*out))
    assert (out[1][3].view(H, W, 4)[..., 3] == 255).any()
