"""Tensor-core precision variants of sem_qcriterion (s- and t-contractions on tcgen05 in BF16,
FP16, split BF16 hi+lo or TF32; r in FP32) against the FP64 oracle.

Bound per node: the FP32 bound of the plain path plus the rounding of the element data and of
D to the operand type on the s/t contractions (unit roundoff 2^-9 BF16, 2^-11 FP16 and TF32,
2^-17 for the hi+lo pair); FP16 subnormals round with absolute error 2^-25 (TF32 keeps the
FP32 exponent range).  The measured maximum
errors are printed (pytest -s) per precision.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import box_factors, dev32, grad_bounds_prec, host64, q_bound

pytestmark = pytest.mark.gpu

EPS = {"BF16": 2.0 ** -9, "FP16": 2.0 ** -11, "BF16X2": 4.0 * 2.0 ** -17, "TF32": 2.0 ** -11}
# FP16 subnormals (|x| < 2^-14, e.g. the velocity near a no-slip wall) round with absolute error
ABS = {"BF16": 0.0, "FP16": 2.0 ** -25, "BF16X2": 0.0, "TF32": 0.0}


def _prec(S, name):
    return {"BF16": S.SEM_BF16, "FP16": S.SEM_FP16, "BF16X2": S.SEM_BF16X2, "TF32": S.SEM_TF32}[name]


def _check(S, sess, orc, xyz, uvw64, name, sample=None):
    m = sess.mesh(7, xyz)
    u, v, w = (dev32(c) for c in uvw64)
    Q = torch.full_like(u, float("nan"))
    S.sem_qcriterion(sess.ctx, m, u, v, w, Q, _prec(S, name))
    S.sem_synchronize(sess.ctx)
    got = host64(Q)
    uvw = np.stack([host64(c) for c in (u, v, w)])
    if sample is not None:
        xyz, uvw, got = xyz[:, sample], uvw[:, sample], got[sample]
    J = orc.gradient(7, xyz, uvw)
    ref = orc.q_from_gradient(J)
    D, g = orc.dmat(7), box_factors(xyz)
    dJ = np.stack([grad_bounds_prec(D, uvw[c], g, 8, J[c], EPS[name], ABS[name]) for c in range(3)])
    bound = q_bound(J, dJ)
    err = np.abs(got - ref)
    assert np.isfinite(got).all()
    assert (err <= bound).all(), (name, float((err / bound).max()))
    rel = err.max() / np.abs(ref).max()
    print(f"\n{name}: max |Q - Q_fp64| / max |Q_fp64| = {rel:.3e}, worst err/bound = {(err / bound).max():.3f}")
    return rel


@pytest.mark.parametrize("name", ["BF16", "FP16", "BF16X2", "TF32"])
def test_tc_taylor_green_box(gpu, sess, orc, name):
    w = si.tgv_box()
    _check(gpu, sess, orc, w.mesh.xyz().numpy(), w.fields.numpy(), name)


@pytest.mark.parametrize("name", ["BF16", "BF16X2", "TF32"])
@pytest.mark.parametrize("E", [1, 3, 4, 5, 9, 37])
def test_tc_ragged_counts(gpu, sess, orc, name, E):
    mesh = si.stretched_box((E, 1, 1), 7, seed=E)
    uvw = si.random_nodal(mesh, 3, seed=E + 50).numpy()
    _check(gpu, sess, orc, mesh.xyz().numpy(), uvw, name)


@pytest.mark.parametrize("name", ["BF16", "FP16", "BF16X2", "TF32"])
def test_tc_channel_full_size_sampled(gpu, sess, orc, name):
    w = si.channel(device="cuda")
    xyz = w.mesh.xyz("cuda").cpu().numpy()
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(w.E, 256, replace=False))
    _check(gpu, sess, orc, xyz, w.fields.cpu().numpy(), name, sample=sample)


def test_tc_split_is_more_accurate_than_single(gpu, sess, orc):
    w = si.tgv_box()
    xyz, f = w.mesh.xyz().numpy(), w.fields.numpy()
    single = _check(gpu, sess, orc, xyz, f, "BF16")
    split = _check(gpu, sess, orc, xyz, f, "BF16X2")
    assert split < single / 20


def test_tc_tf32_between_bf16_and_split(gpu, sess, orc):
    """TF32 operands (11 significant bits) against BF16 (8) and the hi+lo pair (16)."""
    w = si.tgv_box()
    xyz, f = w.mesh.xyz().numpy(), w.fields.numpy()
    single = _check(gpu, sess, orc, xyz, f, "BF16")
    tf32 = _check(gpu, sess, orc, xyz, f, "TF32")
    split = _check(gpu, sess, orc, xyz, f, "BF16X2")
    assert split < tf32 < single / 4


@pytest.mark.parametrize("prec", ["SEM_BF16", "SEM_TF32"])
def test_tc_rejects_other_orders(gpu, sess, prec):
    mesh = si.uniform_box((2, 2, 2), (0, 0, 0), (1, 1, 1), 5)
    m = sess.mesh(5, mesh.xyz().numpy())
    t = torch.zeros(8 * 216, device="cuda")
    with pytest.raises(gpu.SemError) as ex:
        gpu.sem_qcriterion(sess.ctx, m, t, t.clone(), t.clone(), torch.zeros_like(t), getattr(gpu, prec))
    assert ex.value.status == gpu.SEM_ERR_UNSUPPORTED
