"""What the learned compression gains over the method without it, and what its error does to
the Q-isosurface frame.

The autoencoder is trained on the GPU by the library's own BF16 kernels on 200 snapshots of
the Taylor-Green field (32^3 elements, N = 7, phase 2 pi s / 250, 1e-3 noise) and evaluated on
held-out snapshots s = 200, 225, 249.  The baseline at the same payload (48 BF16 values per
element) keeps, per component, the 16 Legendre modes with the most energy on the training data
(oracle/ae.py).  The decoded field then goes through the plain path (Q, isosurface, frame)
and is compared with the input field (the plain path) and with the noise-free field.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import sem_inputs as si
from oracle import ae as ora

pytestmark = pytest.mark.gpu

STEPS, BATCH, LR0 = 20000, 8192, 1e-3
HELD_OUT = tuple(range(200, 250))  # every held-out snapshot


@pytest.fixture(scope="module")
def trained(gpu):
    S = gpu
    sess = S.Session(0)
    train = torch.empty(si.AE_SNAPSHOTS_TRAIN * 32768, 1536, device="cuda")
    for s in range(si.AE_SNAPSHOTS_TRAIN):
        train[s * 32768:(s + 1) * 32768] = si.ae_samples(si.ae_snapshot(s, nel=32, device="cuda"))
    ae = S.sem_ae_create(sess.ctx, BATCH)
    S.sem_ae_set_params(sess.ctx, ae, si.ae_init_params())
    S.sem_ae_fit_normalization(sess.ctx, ae, train[:4 * 32768])
    g = torch.Generator(device="cuda")
    g.manual_seed(si.seed_for(5, 1000))
    loss = torch.zeros(1, device="cuda")
    for it in range(STEPS):
        idx = torch.randint(0, train.shape[0], (BATCH,), generator=g, device="cuda")
        lr = LR0 * 0.5 * (1.0 + math.cos(math.pi * it / STEPS)) + 1e-5
        S.sem_ae_train_step(sess.ctx, ae, train, idx, lr=lr, loss_dev=loss)
    S.sem_synchronize(sess.ctx)
    final = loss.item() / (BATCH * 1536)
    # the baseline's modes, chosen on a sample of the training data
    rng = np.random.default_rng(si.seed_for(5, 1001))
    xi = oracle.gll(7)[0]
    sample = train[torch.as_tensor(rng.choice(train.shape[0], 4096, replace=False), device="cuda")]
    sample = sample.cpu().double().numpy()
    modes = [ora.choose_modes(ora.modal_coefficients(sample[:, c * 512:(c + 1) * 512], xi), 16) for c in range(3)]
    del train, sample
    torch.cuda.empty_cache()
    yield S, sess, ae, modes, final
    S.sem_ae_destroy(ae)
    sess.close()


def _roundtrip(S, sess, ae, f):
    E = f.shape[1]
    lat = torch.empty(E * 48, dtype=torch.bfloat16, device="cuda")
    S.sem_ae_encode(sess.ctx, ae, f[0].contiguous(), f[1].contiguous(), f[2].contiguous(), lat)
    out = [torch.empty(E, 512, device="cuda") for _ in range(3)]
    S.sem_ae_decode(sess.ctx, ae, lat, E, *out)
    torch.cuda.synchronize()
    return torch.stack(out)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_autoencoder_beats_legendre_truncation_at_equal_payload(trained):
    S, sess, ae, modes, final = trained
    xi = oracle.gll(7)[0]
    report = []
    for s in HELD_OUT:
        f = si.ae_snapshot(s, nel=32, device="cuda")
        fc = si.ae_snapshot(s, nel=32, noise=0.0, device="cuda")
        rec = _roundtrip(S, sess, ae, f)
        sel = np.random.default_rng(s).choice(f.shape[1], 256, replace=False)
        fin = f[:, sel].cpu().double().numpy()
        fcl = fc[:, sel].cpu().double().numpy()
        r_ae = rec[:, sel].cpu().double().numpy()
        r_leg = np.stack([ora.truncate(fin[c], xi, modes[c], coef_round=ora.round_bf16) for c in range(3)])
        e_ae, e_leg = _rel(r_ae, fin), _rel(r_leg, fin)
        c_ae, c_leg = _rel(r_ae, fcl), _rel(r_leg, fcl)
        report.append((s, e_ae, e_leg, c_ae, c_leg))
        # vs the transmitted (noisy) field and vs the noise-free field.  Against the input, both
        # errors sit on the same floor: the i.i.d. 1e-3 noise (relative ~3e-3 of the field) that no
        # 48-value code of a 1536-value element can carry, so the margin there is small; against
        # the noise-free field -- what the in situ frame is meant to show -- the code must be
        # better on every snapshot by 10 % and on average by 15 % (below).  The per-snapshot
        # ratio moves by about 0.02 from one training run to the next: the GEMM autotuner's
        # K-split choice, which depends on timings, changes the summation order of the weight
        # gradients and so the trained weights.
        assert e_ae < e_leg, (s, e_ae, e_leg)
        assert c_ae <= 0.90 * c_leg, (s, c_ae, c_leg)
    print(f"\nfinal training loss {final:.3e}")
    for s, e_ae, e_leg, c_ae, c_leg in report:
        if s in (200, 225, 249):
            print(f"held-out s={s}: rel. L2 error vs input  AE {e_ae:.3e}  Legendre-16/BF16 {e_leg:.3e}; "
                  f"vs noise-free  AE {c_ae:.3e}  Legendre-16/BF16 {c_leg:.3e}")
    r = np.array([x[1:] for x in report])
    assert np.mean(r[:, 2] / r[:, 3]) <= 0.85, np.mean(r[:, 2] / r[:, 3])
    print(f"all {len(report)} held-out snapshots: AE / Legendre error ratio vs input {np.min(r[:, 0] / r[:, 1]):.3f}.."
          f"{np.max(r[:, 0] / r[:, 1]):.3f}, vs noise-free {np.min(r[:, 2] / r[:, 3]):.3f}..{np.max(r[:, 2] / r[:, 3]):.3f} "
          f"(mean {np.mean(r[:, 2] / r[:, 3]):.3f})")


def test_decoded_field_through_q_isosurface_and_frame(trained):
    """Q relative L2 error, isosurface Hausdorff distance and pixel error of the decoded
    field, against the plain path (the input field) and the noise-free field."""
    S, sess, ae, modes, final = trained
    s = 225
    f = si.ae_snapshot(s, nel=32, device="cuda")
    fc = si.ae_snapshot(s, nel=32, noise=0.0, device="cuda")
    dec = _roundtrip(S, sess, ae, f)
    mesh = si.uniform_box((32,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, 7)
    m = sess.mesh(7, mesh.xyz().numpy())
    Q = {}
    for name, fld in (("plain", f), ("decoded", dec), ("clean", fc)):
        q = torch.empty_like(fld[0])
        S.sem_qcriterion(sess.ctx, m, fld[0].contiguous(), fld[1].contiguous(), fld[2].contiguous(), q)
        Q[name] = q
    torch.cuda.synchronize()
    qn = {k: v.double().cpu().numpy() for k, v in Q.items()}
    e_dec_plain = _rel(qn["decoded"], qn["plain"])
    e_dec_clean = _rel(qn["decoded"], qn["clean"])
    e_plain_clean = _rel(qn["plain"], qn["clean"])
    # the decoded field is closer to the noise-free field than the input is (noise does not
    # survive the 48-value latent), and derivatives amplify noise
    assert e_dec_clean < e_plain_clean, (e_dec_clean, e_plain_clean)
    iso = float(np.float32(0.1 * S.sem_field_max(sess.ctx, Q["clean"])))
    cam = si.box_camera_persp((0.0,) * 3, (2 * math.pi,) * 3, 1920, 1080)
    # frames of the whole domain; vertices of the 8^3-element corner block for the distances
    ex = torch.arange(32, device="cuda")
    blk = (ex[None, None, :8] + 32 * (ex[None, :8, None] + 32 * ex[:8, None, None])).reshape(-1)
    sub = si.uniform_box((8,) * 3, (0.0,) * 3, (2 * math.pi / 4,) * 3, 7)
    msub = sess.mesh(7, sub.xyz().numpy())
    verts, imgs = {}, {}
    for name, q in Q.items():
        n = S.sem_isosurface(sess.ctx, m, q, iso, None)
        tris = torch.empty(max(n, 1) * 9, device="cuda")
        S.sem_isosurface(sess.ctx, m, q, iso, tris)
        rgba = torch.empty(1080 * 1920 * 4, dtype=torch.uint8, device="cuda")
        S.sem_render(sess.ctx, tris, n, [n], None, cam, 1920, 1080, rgba, None)
        qs = q[blk].contiguous()
        ns = S.sem_isosurface(sess.ctx, msub, qs, iso, None)
        ts = torch.empty(max(ns, 1) * 9, device="cuda")
        S.sem_isosurface(sess.ctx, msub, qs, iso, ts)
        torch.cuda.synchronize()
        verts[name] = np.unique(ts[:ns * 9].view(-1, 3).double().cpu().numpy(), axis=0)
        imgs[name] = rgba.view(1080, 1920, 4).int().cpu().numpy()
    h_dec_clean = ora.hausdorff_kd(verts["decoded"], verts["clean"])
    h_plain_clean = ora.hausdorff_kd(verts["plain"], verts["clean"])
    h_dec_plain = ora.hausdorff_kd(verts["decoded"], verts["plain"])
    cell = 2 * math.pi / 32 / 7  # mean sub-hex size
    assert h_dec_clean < h_plain_clean
    px = lambda a, b: float((np.abs(a - b).max(axis=2) > 1).mean())  # noqa: E731
    p_dec_plain, p_dec_clean, p_plain_clean = px(imgs["decoded"], imgs["plain"]), px(imgs["decoded"], imgs["clean"]), \
        px(imgs["plain"], imgs["clean"])
    assert p_dec_clean < p_plain_clean
    print(f"\nQ rel. L2: decoded vs plain {e_dec_plain:.3e}, decoded vs noise-free {e_dec_clean:.3e}, "
          f"plain vs noise-free {e_plain_clean:.3e}")
    print(f"isosurface Hausdorff (sub-hex size {cell:.3e}): decoded-plain {h_dec_plain:.3e}, "
          f"decoded-noise-free {h_dec_clean:.3e}, plain-noise-free {h_plain_clean:.3e}")
    print(f"pixels differing by more than 1/255: decoded-plain {p_dec_plain:.4f}, decoded-noise-free "
          f"{p_dec_clean:.4f}, plain-noise-free {p_plain_clean:.4f}")
