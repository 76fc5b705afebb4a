"""End-to-end parity on the 8^3-element, N = 7 Taylor-Green workload: GPU (Q -> isosurface ->
frame) against the oracle (Q -> isosurface -> frame) from the same FP32 velocity.

Nodes whose Q lies within the FP32 error bound of the isovalue can legitimately classify
differently; cells touching such a node are masked (and counted), all other cell cases must
be identical.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import box_factors, dev32, grad_bounds, host64, q_bound

pytestmark = pytest.mark.gpu


def test_tgv_end_to_end(gpu, sess, orc):
    w = si.tgv_box()
    xyz = w.mesh.xyz().numpy()
    m = sess.mesh(7, xyz)
    u, v, ww = (dev32(w.fields[c].numpy()) for c in range(3))
    vel = np.stack([host64(t) for t in (u, v, ww)])
    # oracle chain
    J = orc.gradient(7, xyz, vel)
    Qo = orc.q_from_gradient(J)
    iso = np.float32(0.1 * Qo.max())
    ro = orc.isosurface(7, xyz, Qo, float(iso))
    img_o, dep_o, _ = orc.render(ro["tris"], [ro["ntri"]], [[0.9, 0.35, 0.25]], w.camera)
    # GPU chain
    Q = torch.empty_like(u)
    gpu.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    cs = torch.zeros(w.E * 343, dtype=torch.uint8, device="cuda")
    n = gpu.sem_isosurface(sess.ctx, m, Q, float(iso), None, None, cs, cap=0)
    tris = torch.empty(n * 9, device="cuda")
    gpu.sem_isosurface(sess.ctx, m, Q, float(iso), tris, None, cs)
    W, H = w.camera["W"], w.camera["H"]
    rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
    depth = torch.zeros(H * W, device="cuda")
    gpu.sem_render(sess.ctx, tris, n, [n], [[0.9, 0.35, 0.25]], w.camera, W, H, rgba, depth)
    torch.cuda.synchronize()
    # mask cells with a corner inside the Q error band around iso
    D = orc.dmat(7)
    g = box_factors(xyz)
    dJ = np.stack([grad_bounds(D, vel[c], g, 8, J[c]) for c in range(3)])
    band = np.abs(Qo - iso) <= q_bound(J, dJ) + abs(float(iso)) * 2.0 ** -23
    bnd = band.reshape(-1, 8, 8, 8)
    near = np.zeros((w.E, 7, 7, 7), bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                near |= bnd[:, dk:dk + 7, dj:dj + 7, di:di + 7]
    near = near.reshape(w.E, -1)
    got = cs.cpu().numpy().reshape(w.E, -1)
    assert (got[~near] == ro["cases"][~near]).all()
    assert near.mean() < 0.01
    assert abs(n - ro["ntri"]) <= 5 * near.sum()
    img = rgba.cpu().numpy().reshape(H, W, 4)
    close = (np.abs(img.astype(int) - img_o.astype(int)) <= 1).all(axis=2).mean()
    assert close >= 0.999, close
