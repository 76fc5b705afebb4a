"""The precision workload at full size: 64^3 = 262144 elements of order 7 (134M nodes), a
Rayleigh-Benard-like field (convection rolls + 64 seeded modes, amplitude 0.1) with velocity
and temperature (2.15 GB of FP32), Q at every arithmetic of sem_qcriterion against the FP64
oracle on sampled elements (per-node bounds from the arithmetic, errors printed per result: FP32, BF16,
FP16, split BF16, TF32),
the temperature isosurface T = 0.5 next to the Q isosurface (cases bit-exact on sampled
elements) and one 3840x2160 frame holding both fields' surfaces, compared pixel by pixel with
the oracle's raster of the same triangles."""
import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import box_factors, compare_images, grad_bounds, grad_bounds_prec, host64, q_bound

pytestmark = pytest.mark.gpu

EPS = {"BF16": 2.0 ** -9, "FP16": 2.0 ** -11, "BF16X2": 4.0 * 2.0 ** -17, "TF32": 2.0 ** -11}
ABS = {"BF16": 0.0, "FP16": 2.0 ** -25, "BF16X2": 0.0, "TF32": 0.0}


@pytest.fixture(scope="module")
def rb(gpu):
    w = si.rb_box(device="cuda")
    f32 = w.fields.float()
    w.fields = None
    w.extra["xyz"] = w.mesh.xyz("cuda").cpu().numpy()  # (3, E, 512) float64, 3.2 GB on the host
    torch.cuda.empty_cache()
    return w, f32


def test_q_every_precision_full_size_sampled(gpu, sess, orc, rb):
    S = gpu
    w, f = rb
    xyz = w.extra["xyz"]
    m = sess.mesh(7, xyz)
    rng = np.random.default_rng(si.seed_for(3, 7))
    sample = np.sort(rng.choice(w.E, 128, replace=False))
    sample[-1] = w.E - 1
    uvw = np.stack([f[c][torch.as_tensor(sample, device="cuda")].double().cpu().numpy() for c in range(3)])
    xs = xyz[:, sample]
    J = orc.gradient(7, xs, uvw)
    ref = orc.q_from_gradient(J)
    D, g = orc.dmat(7), box_factors(xs)
    Q = torch.empty_like(f[0])
    report = {}
    for name in ("FP32", "BF16", "FP16", "BF16X2", "TF32"):
        Q.fill_(float("nan"))
        S.sem_qcriterion(sess.ctx, m, f[0], f[1], f[2], Q, getattr(S, "SEM_" + name))
        S.sem_synchronize(sess.ctx)
        got = Q[torch.as_tensor(sample, device="cuda")].double().cpu().numpy()
        if name == "FP32":
            dJ = np.stack([grad_bounds(D, uvw[c], g, 8, J[c]) for c in range(3)])
        else:
            dJ = np.stack([grad_bounds_prec(D, uvw[c], g, 8, J[c], EPS[name], ABS[name]) for c in range(3)])
        bound = q_bound(J, dJ)
        err = np.abs(got - ref)
        assert np.isfinite(got).all(), name
        assert (err <= bound).all(), (name, float((err / bound).max()))
        report[name] = err.max() / np.abs(ref).max()
    # the derivative itself (plain path): max |du - du_64| / max |du_64|
    du = [torch.empty_like(f[0]) for _ in range(3)]
    S.sem_derivatives(sess.ctx, m, f[0], *du)
    torch.cuda.synchronize()
    dgot = np.stack([d[torch.as_tensor(sample, device="cuda")].double().cpu().numpy() for d in du])
    derr = np.abs(dgot - J[0])
    assert (derr <= grad_bounds(D, uvw[0], g, 8, J[0])).all()  # per-node FP32 bound
    drel = derr.max() / np.abs(J[0]).max()
    assert drel <= 1e-5, drel  # the field-level bar for FP32 derivatives
    print("\n64^3 precision workload, sampled elements:", f"du/dx_j FP32 {drel:.3e};",
          "; ".join(f"Q {k} {v:.3e}" for k, v in report.items()), "(max error / max |Q_fp64|)")
    assert report["FP32"] < report["BF16X2"] < report["TF32"] < report["BF16"] and report["FP16"] < report["BF16"]


def test_temperature_and_q_isosurfaces_and_one_frame(gpu, sess, orc, rb):
    S = gpu
    w, f = rb
    xyz = w.extra["xyz"]
    m = sess.mesh(7, xyz)
    Q = torch.empty_like(f[0])
    S.sem_qcriterion(sess.ctx, m, f[0], f[1], f[2], Q)
    q_iso = float(np.float32(0.1 * S.sem_field_max(sess.ctx, Q)))
    t_iso = float(np.float32(w.extra["t_iso"]))
    rng = np.random.default_rng(si.seed_for(3, 8))
    sample = np.sort(rng.choice(w.E, 96, replace=False))
    si_ = torch.as_tensor(sample, device="cuda")
    counts, cases = [], []
    for field, iso in ((Q, q_iso), (f[3], t_iso)):
        cs = torch.empty(w.E * 343, dtype=torch.uint8, device="cuda")
        n = S.sem_isosurface(sess.ctx, m, field, iso, None, cases=cs)
        counts.append(n)
        cases.append(cs.view(w.E, 343)[si_].cpu().numpy())
        ref = orc.isosurface(7, xyz[:, sample], field[si_].double().cpu().numpy(), iso, want_tris=False)
        np.testing.assert_array_equal(cases[-1].reshape(-1), ref["cases"].reshape(-1))
    nq, nt = counts
    assert nq > 0 and nt > 0
    # the fused form (counting inside the Q kernel) at full size: the same Q and count
    Qf = torch.empty_like(Q)
    cf = torch.zeros(2, dtype=torch.int64, device="cuda")
    S.sem_qcriterion_isosurface_async(sess.ctx, m, f[0], f[1], f[2], Qf, [q_iso], None, cf)
    S.sem_synchronize(sess.ctx)
    assert torch.equal(Qf, Q) and cf.cpu().tolist() == [0, nq]
    del Qf
    tris = torch.empty((nq + nt) * 9, device="cuda")
    S.sem_isosurface(sess.ctx, m, Q, q_iso, tris[:nq * 9])
    S.sem_isosurface(sess.ctx, m, f[3], t_iso, tris[nq * 9:])
    Wd, Hd = w.camera["W"], w.camera["H"]
    rgba = torch.empty(Hd * Wd * 4, dtype=torch.uint8, device="cuda")
    depth = torch.empty(Hd * Wd, device="cuda")
    colours = np.array([[0.9, 0.3, 0.2], [0.2, 0.5, 0.9]], np.float32)
    S.sem_render(sess.ctx, tris, nq + nt, [nq, nt], colours, w.camera, Wd, Hd, rgba, depth)
    torch.cuda.synchronize()
    img = rgba.view(Hd, Wd, 4).int().cpu().numpy()
    covered = img[..., 3] == 255
    assert covered.mean() > 0.05
    # both fields' surfaces are visible: red-dominant (Q) and blue-dominant (T) pixels
    red = covered & (img[..., 0] > img[..., 2])
    blue = covered & (img[..., 2] > img[..., 0])
    assert red.sum() > 1000 and blue.sum() > 1000
    used, peak = S.sem_memory(sess.ctx)
    # the whole 3840x2160 frame against the oracle's raster of the same FP32 triangles
    ref_img, ref_dep, _ = orc.render(host64(tris).reshape(-1, 3, 3), [nq, nt], colours.astype(np.float64),
                                     w.camera)
    frac, dfrac = compare_images(img.astype(np.uint8), depth.view(Hd, Wd).cpu().numpy(), ref_img, ref_dep)
    print(f"\n64^3: {nq} Q triangles, {nt} T triangles, {covered.mean():.3f} of 3840x2160 covered, "
          f"{frac * 100:.3f}% of pixels within 1/255 of the oracle, {dfrac * 100:.3f}% of compared depths "
          f"within 1e-5; "
          f"library memory {used / 2**20:.1f} MiB (peak {peak / 2**20:.1f} MiB)")
