"""Failure detection without a device fault: the Q kernels' bounded waits on their input
copies.  sem_debug_set_wait_limit(ctx, 0) makes every consumer wait give up at once, so the
timeout path runs deterministically: the kernel records SEM_ERR_TIMEOUT on the context's device
flag, drains its copies still in flight (with the default limit) and returns.  The test checks
that sem_synchronize reports the timeout and clears the flag, and that the next normal call on
the same context is correct against the oracle."""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import box_factors, dev32, grad_bounds, host64, q_bound

pytestmark = pytest.mark.gpu


def _q_parity(S, ctx, orc, m, xyz, uvw32, N):
    Q = torch.full_like(uvw32[0], float("nan"))
    S.sem_qcriterion(ctx, m, *uvw32, Q)
    S.sem_synchronize(ctx)
    uvw = np.stack([host64(c) for c in uvw32])
    J = orc.gradient(N, xyz, uvw)
    ref = orc.q_from_gradient(J)
    D, g = orc.dmat(N), box_factors(xyz)
    dJ = np.stack([grad_bounds(D, uvw[c], g, N + 1, J[c]) for c in range(3)])
    err = np.abs(host64(Q) - ref)
    assert (err <= q_bound(J, dJ)).all()


# N = 7: k_sem_q8 (4-element stages); N = 5: k_sem_qd<6> (7-element stages; the last,
# partial group is loaded without a copy); both fill their stages with bulk copies
@pytest.mark.parametrize("N,nel", [(7, (5, 4, 3)), (5, (5, 4, 3))])
def test_bounded_wait_runs_out_and_context_recovers(gpu, sess, orc, N, nel):
    S = gpu
    mesh = si.stretched_box(nel, N, seed=N)
    xyz = mesh.xyz().numpy()
    m = sess.mesh(N, xyz)
    uvw32 = [dev32(c) for c in si.random_nodal(mesh, 3, seed=10 + N).numpy()]
    Q = torch.zeros_like(uvw32[0])
    S.sem_debug_set_wait_limit(sess.ctx, 0)
    try:
        S.sem_qcriterion(sess.ctx, m, *uvw32, Q)
        with pytest.raises(S.SemError) as ex:
            S.sem_synchronize(sess.ctx)
        assert ex.value.status == S.SEM_ERR_TIMEOUT
        assert "wait ran out" in str(ex.value)
        S.sem_synchronize(sess.ctx)  # reported once: the flag was cleared
    finally:
        S.sem_debug_set_wait_limit(sess.ctx, -1)
    _q_parity(S, sess.ctx, orc, m, xyz, uvw32, N)


def test_timeout_inside_a_graph_is_reported_after_replay(gpu, sess, orc):
    """The limit is read when the launch is recorded: a graph captured with the limit at 0
    raises the flag on every replay, while direct calls with the default limit stay correct."""
    S = gpu
    mesh = si.stretched_box((4, 3, 2), 7, seed=3)
    xyz = mesh.xyz().numpy()
    m = sess.mesh(7, xyz)
    uvw32 = [dev32(c) for c in si.random_nodal(mesh, 3, seed=3).numpy()]
    Q = torch.zeros_like(uvw32[0])
    S.sem_qcriterion(sess.ctx, m, *uvw32, Q)
    S.sem_synchronize(sess.ctx)
    S.sem_debug_set_wait_limit(sess.ctx, 0)
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
            S.sem_qcriterion(sess.ctx, m, *uvw32, Q)
        S.sem_set_stream(sess.ctx, torch.cuda.current_stream())
    finally:
        S.sem_debug_set_wait_limit(sess.ctx, -1)
    for _ in range(2):
        g.replay()
        with pytest.raises(S.SemError) as ex:
            S.sem_synchronize(sess.ctx)
        assert ex.value.status == S.SEM_ERR_TIMEOUT
    _q_parity(S, sess.ctx, orc, m, xyz, uvw32, 7)
