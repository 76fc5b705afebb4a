"""GPU parity of sem_derivatives / sem_qcriterion against the FP64 oracle (through the C ABI).

Tolerances: per-node FP32 error bounds derived from the arithmetic (tests/_helpers.py), and for
the derivatives also the field-level bar max |du - du_64| <= 1e-5 max |du_64|.
Sizes: small cases spanning several blocks with ragged tails, every supported order, and
the 32^3-element channel workload at full size in the launch configuration bench.py times,
checked on sampled elements.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import box_factors, dev32, grad_bounds, host64, q_bound

pytestmark = pytest.mark.gpu
DERIV_BAR = 1e-5


def _grad_check(S, sess, orc, mesh, u64, seed_note=""):
    N, NP = mesh.N, mesh.NP
    xyz = mesh.xyz().numpy()
    m = sess.mesh(N, xyz)
    u32 = dev32(u64)
    out = [torch.empty_like(u32) for _ in range(3)]
    S.sem_derivatives(sess.ctx, m, u32, *out)
    torch.cuda.synchronize()
    got = np.stack([host64(o) for o in out])
    u = host64(u32)
    ref = orc.gradient(N, xyz, u)[0]
    bound = grad_bounds(orc.dmat(N), u, box_factors(xyz), NP, ref)
    err = np.abs(got - ref)
    assert (err <= bound).all(), (seed_note, N, float((err / bound).max()))
    # the field-level bar for FP32 derivatives: max |du - du_64| <= 1e-5 max |du_64|
    assert err.max() <= DERIV_BAR * np.abs(ref).max(), (seed_note, N, err.max() / np.abs(ref).max())
    return got, ref


@pytest.mark.parametrize("N,nel", [(7, (3, 5, 3)), (7, (1, 1, 1)), (7, (2, 1, 3)), (1, (2, 3, 4)), (2, (3, 3, 3)),
                                   (3, (4, 2, 3)), (4, (2, 2, 3)), (5, (4, 4, 3)), (6, (3, 1, 2)), (8, (2, 2, 2)),
                                   (9, (2, 3, 3)), (10, (1, 2, 3)), (11, (1, 1, 3)), (13, (1, 1, 2)), (15, (1, 2, 2))])
def test_derivatives_random_field(gpu, sess, orc, N, nel):
    mesh = si.stretched_box(nel, N, seed=N)
    u = si.random_nodal(mesh, 1, seed=100 + N)[0].numpy()
    _grad_check(gpu, sess, orc, mesh, u, "random")


@pytest.mark.parametrize("N", [3, 7])
def test_derivatives_polynomial(gpu, sess, orc, N):
    mesh = si.stretched_box((3, 2, 2), N, seed=3)
    X, Y, Z = mesh.xyz().numpy()
    u = X ** 3 * Y - 2.0 * Y ** 2 * Z + Z ** 3 + X * Y * Z
    got, _ = _grad_check(gpu, sess, orc, mesh, u, "poly")
    exact = np.stack([3 * X ** 2 * Y + Y * Z, X ** 3 - 4 * Y * Z + X * Z, -2 * Y ** 2 + 3 * Z ** 2 + X * Y])
    assert np.abs(got - exact).max() < 1e-4 * np.abs(exact).max()


def _q_check(S, sess, orc, xyz, uvw64, N, sample=None):
    m = sess.mesh(N, xyz)
    u, v, w = (dev32(c) for c in uvw64)
    Q = torch.empty_like(u)
    S.sem_qcriterion(sess.ctx, m, u, v, w, Q)
    S.sem_synchronize(sess.ctx)
    got = host64(Q)
    uvw = np.stack([host64(c) for c in (u, v, w)])
    if sample is not None:
        xyz, uvw, got = xyz[:, sample], uvw[:, sample], got[sample]
    J = orc.gradient(N, xyz, uvw)            # (3 comps, 3 dirs, E, NP3) = J[i][j]
    ref = orc.q_from_gradient(J)
    D = orc.dmat(N)
    g = box_factors(xyz)
    dJ = np.stack([grad_bounds(D, uvw[c], g, N + 1, J[c]) for c in range(3)])
    bound = q_bound(J, dJ)
    err = np.abs(got - ref)
    assert (err <= bound).all(), float((err / bound).max())
    return got, ref


def test_qcriterion_taylor_green_box(gpu, sess, orc):
    """8^3 elements, N = 7, Taylor-Green + seeded 1e-3 noise (the small workload)."""
    w = si.tgv_box()
    got, ref = _q_check(gpu, sess, orc, w.mesh.xyz().numpy(), w.fields.numpy(), 7)
    assert abs(got.max() - ref.max()) < 1e-5 * ref.max()


def test_qcriterion_noise_free_analytic(gpu, sess, orc):
    w = si.tgv_box(noise=0.0)
    xyz = w.mesh.xyz().numpy()
    got, _ = _q_check(gpu, sess, orc, xyz, w.fields.numpy(), 7)
    X, Y, Z = xyz
    Qa = -(1 + np.cos(2 * Z)) * (np.cos(2 * X) + np.cos(2 * Y)) / 4
    assert np.abs(got - Qa).max() < 2e-5


@pytest.mark.parametrize("E", [1, 2, 3, 4, 5, 7, 9, 33])
def test_qcriterion_ragged_counts(gpu, sess, orc, E):
    # element counts around the 4-element groups the N=7 kernel stages per copy
    mesh = si.stretched_box((E, 1, 1), 7, seed=E)
    uvw = si.random_nodal(mesh, 3, seed=E).numpy()
    _q_check(gpu, sess, orc, mesh.xyz().numpy(), uvw, 7)


@pytest.mark.parametrize("N", [2, 4, 5, 9])
def test_qcriterion_orders(gpu, sess, orc, N):
    mesh = si.stretched_box((3, 2, 5), N, seed=N)
    uvw = si.random_nodal(mesh, 3, seed=7 * N).numpy()
    _q_check(gpu, sess, orc, mesh.xyz().numpy(), uvw, N)


def test_qcriterion_channel_full_size_sampled(gpu, sess, orc):
    """32^3 elements (16.8M nodes), N = 7: the benchmark's workload and launch; the oracle
    checks 384 seeded sampled elements."""
    w = si.channel(device="cuda")
    xyz = w.mesh.xyz("cuda").cpu().numpy()
    uvw = w.fields.cpu().numpy()
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(w.E, 384, replace=False))
    sample[-1] = w.E - 1
    _q_check(gpu, sess, orc, xyz, uvw, 7, sample=sample)


def test_empty_mesh_is_noop(gpu, sess):
    m = sess.mesh(7, np.zeros((3, 0, 512)))
    assert gpu.sem_mesh_info(m) == (7, 0)
    t = torch.zeros(4, device="cuda")
    gpu.sem_qcriterion(sess.ctx, m, t, t.clone(), t.clone(), torch.zeros(4, device="cuda"))


def test_argument_errors(gpu, sess):
    mesh = si.uniform_box((2, 1, 1), (0, 0, 0), (1, 1, 1), 7)
    m = sess.mesh(7, mesh.xyz().numpy())
    u = torch.zeros(2 * 512 + 4, device="cuda")
    Q = torch.zeros_like(u)
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_qcriterion(sess.ctx, m, u[1:], u, u, Q)  # 4-byte offset: misaligned
    assert ex.value.status == gpu.SEM_ERR_ARG
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_qcriterion(sess.ctx, m, u, u, u, u)
    assert ex.value.status == gpu.SEM_ERR_ARG
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_qcriterion(sess.ctx, m, u, u, u, Q, 17)
    assert ex.value.status == gpu.SEM_ERR_ARG
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_load_mesh(sess.ctx, 16, np.zeros((3, 1, 17 ** 3)))
    assert ex.value.status == gpu.SEM_ERR_ARG
    # a non-box element makes the mesh general (isoparametric path); an inverted one is refused
    xyz = mesh.xyz().numpy().copy()
    xyz[0, 0, 100] += 0.01
    gpu.sem_mesh_free(gpu.sem_load_mesh(sess.ctx, 7, xyz))
    xyz[0] = -xyz[0]  # mirrored: every Jacobian determinant of the general mesh is negative
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_load_mesh(sess.ctx, 7, xyz)
    assert ex.value.status == gpu.SEM_ERR_ARG
    gpu.sem_synchronize(sess.ctx)
