"""General (curved) meshes through the C ABI against the FP64 oracle: derivatives and Q by the
isoparametric chain rule, the isosurface with vertices between the nodes' own coordinates.

Mesh: the element-corner grid with its interior corners moved at random, each element the
trilinear map of its corners (conforming, non-affine).  Bound per node for the derivatives:
the reference derivative along direction d is an FP32 sum of NP products with FP32 D, error
<= (NP + 1) u A_d with A_d = sum_m |D||u| along d; the inverse Jacobian G = d r / d x is
rounded to FP32 (u |G|), and the three-term sum d u / d x_j = sum_d (d u / d r_d) G_dj adds
3 u sum_d |d u / d r_d| |G_dj|; together (NP + 5) u sum_d |G_dj| A_d to first order, u = 2^-24
(the test takes NP + 6 for the second-order terms).  Q's bound follows from the derivatives'
(q_bound).
"""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import EPS32, dev32, host64, q_bound, ref_abs_contractions

pytestmark = pytest.mark.gpu


def _inverse_jacobian(D, xyz, NP):
    """(E, NP^3, 3, 3) G[d][j] = d r_d / d x_j from the node coordinates (FP64)."""
    E = xyz.shape[1]
    X = xyz.reshape(3, E, NP, NP, NP)  # [c][e][k][j][i]
    J = np.stack([np.stack([np.einsum("im,ekjm->ekji", D, X[c]), np.einsum("jm,ekmi->ekji", D, X[c]),
                            np.einsum("km,emji->ekji", D, X[c])], axis=-1) for c in range(3)], axis=-2)
    return np.linalg.inv(J.reshape(E, NP ** 3, 3, 3))  # J[c][d] -> G[d][c]


def _deriv_bounds(D, u, G, NP, ref):
    """(3, E, NP^3) bound on |du/dx_j (GPU) - du/dx_j (oracle)| for one field u (E, NP^3)."""
    A = ref_abs_contractions(D, u, NP)
    out = []
    for j in range(3):
        b = sum(np.abs(G[..., d, j]) * A[d] for d in range(3))
        out.append((NP + 6) * EPS32 * b + 1e-12 * np.abs(ref).max())
    return np.stack(out)


def _velocity(xyz):
    X, Y, Z = xyz
    return np.stack([np.sin(2 * X) * np.cos(Y) + 0.3 * Z * Z, -np.cos(2 * X) * np.sin(Y) + X * Z,
                     0.5 * np.sin(X + Y) * np.cos(3 * Z)])


@pytest.mark.parametrize("N,n", [(3, (3, 2, 2)), (7, (3, 3, 2)), (10, (2, 2, 1))])
def test_curved_derivatives_and_q(gpu, sess, orc, N, n):
    S = gpu
    xyz = si.perturbed_box(n, (0, 0, 0), (1.5, 1.2, 1.0), N, amp=0.2, seed=N)
    NP = N + 1
    m = sess.mesh(N, xyz)
    uvw32 = [dev32(c) for c in _velocity(xyz)]
    uvw = np.stack([host64(c) for c in uvw32])
    J = orc.gradient(N, xyz, uvw)
    D = orc.dmat(N)
    G = _inverse_jacobian(D, xyz, NP)
    dJ = np.stack([_deriv_bounds(D, uvw[c], G, NP, J[c]) for c in range(3)])
    # derivatives of each component
    for c in range(3):
        d = [torch.full_like(uvw32[0], float("nan")) for _ in range(3)]
        S.sem_derivatives(sess.ctx, m, uvw32[c], *d)
        S.sem_synchronize(sess.ctx)
        got = np.stack([host64(x) for x in d])
        assert np.isfinite(got).all()
        err = np.abs(got - J[c])
        assert (err <= dJ[c]).all(), (c, float((err / dJ[c]).max()))
        # the field-level bar for FP32 derivatives: max |du - du_64| <= 1e-5 max |du_64|
        assert err.max() <= 1e-5 * np.abs(J[c]).max(), (c, err.max() / np.abs(J[c]).max())
    # Q
    Q = torch.full_like(uvw32[0], float("nan"))
    S.sem_qcriterion(sess.ctx, m, *uvw32, Q)
    S.sem_synchronize(sess.ctx)
    ref = orc.q_from_gradient(J)
    err = np.abs(host64(Q) - ref)
    bound = q_bound(J, dJ)
    assert (err <= bound).all(), float((err / bound).max())


def test_curved_exact_quadratic_gradient(gpu, sess, orc):
    """A field of total degree 2 in x is degree <= 2 per reference direction on trilinear
    elements, so the chain rule is exact: the GPU result is the analytic gradient to FP32."""
    S = gpu
    N = 4
    xyz = si.perturbed_box((2, 2, 2), (0, 0, 0), (1, 1, 1), N, amp=0.25, seed=3)
    X, Y, Z = xyz
    f = 1.0 + 2 * X - Y + 0.5 * Z + X * Y - 0.3 * Z * Z + 0.7 * X * Z
    exact = np.stack([2 + Y + 0.7 * Z, -1 + X, 0.5 - 0.6 * Z + 0.7 * X])
    m = sess.mesh(N, xyz)
    f32 = dev32(f)
    d = [torch.empty_like(f32) for _ in range(3)]
    S.sem_derivatives(sess.ctx, m, f32, *d)
    S.sem_synchronize(sess.ctx)
    got = np.stack([host64(x) for x in d])
    NP = N + 1
    G = _inverse_jacobian(orc.dmat(N), xyz, NP)
    bound = _deriv_bounds(orc.dmat(N), host64(f32), G, NP, exact)
    # plus the FP32 rounding of f itself, carried through the exact (linear) chain rule
    bound += 4 * EPS32 * np.abs(host64(f32)).max() * np.abs(G).sum(axis=2).transpose(2, 0, 1) * \
        np.abs(orc.dmat(N)).sum(axis=1).max()
    assert (np.abs(got - exact) <= bound).all()


def test_curved_isosurface(gpu, sess, orc):
    """Sphere field on a curved mesh: cases, counts and element of every triangle exact, vertices
    (between the nodes' own coordinates) within 1e-5 of the domain size."""
    S = gpu
    N = 5
    xyz = si.perturbed_box((4, 3, 3), (0, 0, 0), (1.2, 1.0, 1.0), N, amp=0.2, seed=11)
    X, Y, Z = xyz
    f = (X - 0.6) ** 2 + (Y - 0.5) ** 2 + (Z - 0.45) ** 2 - 0.3 ** 2
    m = sess.mesh(N, xyz)
    f32 = dev32(f)
    iso = 0.0
    cases = torch.empty(f.shape[0] * N ** 3, dtype=torch.uint8, device="cuda")
    n = S.sem_isosurface(sess.ctx, m, f32, iso, None, cases=cases)
    tris = torch.empty(max(n, 1) * 9, device="cuda")
    te = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    S.sem_isosurface(sess.ctx, m, f32, iso, tris, tri_elem=te)
    torch.cuda.synchronize()
    ref = orc.isosurface(N, xyz, host64(f32), iso)
    np.testing.assert_array_equal(cases.view(-1, N ** 3).cpu().numpy(), ref["cases"])
    assert n == ref["ntri"] and n > 100
    np.testing.assert_array_equal(te[:n].cpu().numpy(), ref["tri_elem"])
    got = tris[:n * 9].view(n, 3, 3).double().cpu().numpy()
    assert np.abs(got - ref["tris"]).max() <= 1e-5 * 1.2


def test_curved_mesh_limits(gpu, sess):
    """What a general mesh does not take: tensor-core precisions, the batched Q, the
    allocation-free isosurface (SEM_ERR_UNSUPPORTED)."""
    S = gpu
    xyz = si.perturbed_box((2, 2, 2), (0, 0, 0), (1, 1, 1), 7, amp=0.1, seed=2)  # the centre corner moves
    m = sess.mesh(7, xyz)
    u = torch.zeros(8 * 512, device="cuda")
    Q = torch.zeros_like(u)
    with pytest.raises(S.SemError) as ex:
        S.sem_qcriterion(sess.ctx, m, u, u.clone(), u.clone(), Q, S.SEM_BF16)
    assert ex.value.status == S.SEM_ERR_UNSUPPORTED
    with pytest.raises(S.SemError) as ex:
        S.sem_qcriterion_batch(sess.ctx, [m], [u], [u.clone()], [u.clone()], [Q])
    assert ex.value.status == S.SEM_ERR_UNSUPPORTED
    tris = torch.zeros(9 * 64, device="cuda")
    with pytest.raises(S.SemError) as ex:
        S.sem_isosurface_noalloc(sess.ctx, m, u, 0.0, tris, cap=64)
    assert ex.value.status == S.SEM_ERR_UNSUPPORTED
    S.sem_qcriterion(sess.ctx, m, u, u.clone(), u.clone(), Q)  # FP32 works
    S.sem_synchronize(sess.ctx)
    assert (Q == 0).all()
