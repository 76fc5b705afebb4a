"""Kernel trace (sem_trace_*): per-kernel launch counts and device times of one frame, and
no records for launches made while the stream is captured into a CUDA graph."""
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu


def test_trace_counts_the_frame_kernels(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=4)
    m = sess.mesh(w.mesh.N, w.mesh.xyz().numpy())
    vel = [w.fields[c].float().cuda().contiguous() for c in range(3)]
    Q = torch.empty_like(vel[0])
    S.sem_trace_enable(sess.ctx, True)
    for _ in range(3):
        S.sem_qcriterion(sess.ctx, m, *vel, Q)
    counts = S.sem_isosurface_multi(sess.ctx, m, Q, [0.1, 0.3], None)
    tr = S.sem_trace_collect(sess.ctx)
    qk = "k_sem_q8"  # the Q kernel of order 7
    assert tr[qk][1] == 3 and tr[qk][0] > 0.0
    assert tr["k_iso_count_p"][1] == 1  # the persistent counting pass (N <= 9)
    assert list(tr)[0] == qk  # first-launch order
    assert sum(counts) > 0
    assert S.sem_trace_collect(sess.ctx) == {}  # collecting cleared the record
    # captured launches are not traced (events cannot be recorded into a capture this way)
    g = torch.cuda.CUDAGraph()
    S.sem_qcriterion(sess.ctx, m, *vel, Q)
    S.sem_trace_collect(sess.ctx)
    with torch.cuda.graph(g):
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
        S.sem_qcriterion(sess.ctx, m, *vel, Q)
    S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    assert S.sem_trace_collect(sess.ctx) == {}
    S.sem_trace_enable(sess.ctx, False)
    S.sem_qcriterion(sess.ctx, m, *vel, Q)
    assert S.sem_trace_collect(sess.ctx) == {}


def test_memory_in_use_and_high_water_mark(gpu):
    S = gpu
    s = S.Session(0)
    try:
        base, peak0 = S.sem_memory(s.ctx)
        assert base > 0 and peak0 >= base
        w = si.tgv_box(nel=4)
        m = S.sem_load_mesh(s.ctx, w.mesh.N, w.mesh.xyz().numpy())
        with_mesh, _ = S.sem_memory(s.ctx)
        assert with_mesh == base + 3 * 16 * w.E  # three float4 per element
        ae = S.sem_ae_create(s.ctx, 128)
        with_ae, peak1 = S.sem_memory(s.ctx)
        assert with_ae > with_mesh + 26 * 2 ** 20 and peak1 >= with_ae
        S.sem_ae_destroy(ae)
        S.sem_mesh_free(m)
        after, peak2 = S.sem_memory(s.ctx)
        assert after == base and peak2 == peak1
    finally:
        s.close()
