"""GPU parity of the learned per-element compression (sem_ae_*, sem_gemm_bf16) against the FP64
oracle (oracle/ae.py).

Tolerances (from the arithmetic):
* GEMM: BF16 x BF16 products are exact in FP32; the FP32 accumulation of K terms errs by at
  most K 2^-24 sum_k |a_k b_k| (bound used with a factor 2 margin).
* Forward / gradients: the GPU stores every activation and back-propagated gradient in BF16
  (unit roundoff u = 2^-8) and computes gelu, gelu' in FP32.  Along the longest path a gradient
  entry passes through at most 8 BF16 roundings, so its relative error is at most ~8u = 3%
  when they align; the tests bound the relative L2 error of each gradient tensor by 5% and the
  loss by 1% (the loss is a mean over 1536 B squared residuals, each perturbed by a few u).
* AdamW: FP32 update of the same gradients; a few ulps of each weight.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si
from oracle import ae as ora

pytestmark = pytest.mark.gpu


def _bf(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (384, 192, 320), (256, 256, 576), (128, 128, 1536)])
def test_gemm_bf16_matches_fp64_product(gpu, sess, M, N, K):
    S = gpu
    rng = np.random.default_rng(M + N + K)
    A = _bf(rng.normal(size=(M, K))).cuda()
    B = _bf(rng.normal(size=(N, K))).cuda()
    Cd = torch.full((M, N), float("nan"), device="cuda")
    S.sem_gemm_bf16(sess.ctx, A, B, Cd)
    torch.cuda.synchronize()
    a = A.float().cpu().double().numpy()
    b = B.float().cpu().double().numpy()
    ref = a @ b.T
    bound = 2.0 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(Cd.cpu().double().numpy() - ref)
    assert np.isfinite(Cd.cpu().numpy()).all()
    assert (err <= bound).all(), float((err / bound).max())


def test_gemm_autotuner_choices_and_determinism(gpu, sess):
    """The first product of a shape tunes (tile width, stages, K split); later products reuse the
    choice bit for bit; with tuning off the default configuration agrees within the FP32 bound."""
    S = gpu
    rng = np.random.default_rng(5)
    M, N, K = 512, 1536, 8192  # a weight-gradient shape: few tiles, long K -> split candidates
    A = _bf(rng.normal(size=(M, K))).cuda()
    B = _bf(rng.normal(size=(N, K))).cuda()
    C1, C2, C3 = (torch.empty(M, N, device="cuda") for _ in range(3))
    S.sem_autotune_set(sess.ctx, True)
    S.sem_gemm_bf16(sess.ctx, A, B, C1)
    S.sem_gemm_bf16(sess.ctx, A, B, C2)
    torch.cuda.synchronize()
    ch = [c for c in S.sem_autotune_choices(sess.ctx) if c[:3] == (M, N, K)]
    assert len(ch) == 1
    _, _, _, mode, bn, stages, split, persistent, ms = ch[0]
    assert bn in (64, 128, 256) and stages in (3, 4) and split in (1, 2, 4, 8, 16, 32) and ms > 0
    assert persistent in (0, 1) and (not persistent or (split == 1 and bn <= 128))
    assert torch.equal(C1, C2)
    S.sem_autotune_set(sess.ctx, False)
    S.sem_gemm_bf16(sess.ctx, A, B, C3)
    torch.cuda.synchronize()
    S.sem_autotune_set(sess.ctx, True)
    a, b = A.float().cpu().double().numpy(), B.float().cpu().double().numpy()
    bound = 2.0 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T)
    ref = a @ b.T
    for Cx in (C1, C3):
        assert (np.abs(Cx.cpu().double().numpy() - ref) <= bound).all()
    print(f"\n{M}x{N}x{K}: BN {bn}, {stages} stages, K split {split}, persistent {persistent}, {ms * 1e3:.1f} us")


def test_gemm_rejects_untileable_shapes(gpu, sess):
    S = gpu
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(64, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(100, 64, device="cuda")
    with pytest.raises(S.SemError) as ex:
        S.sem_gemm_bf16(sess.ctx, A, B, C)
    assert ex.value.status == S.SEM_ERR_ARG


def _data(nel=4, snaps=(0, 1)):
    fields = [si.ae_snapshot(s, nel=nel, device="cuda") for s in snaps]
    return torch.cat([si.ae_samples(f) for f in fields])


def _oracle_inputs(samples, idx, mean, std, params):
    x = samples[idx].cpu().double().numpy()
    xn = np.empty_like(x)
    for c in range(3):
        xn[:, c * 512:(c + 1) * 512] = (np.float32(x[:, c * 512:(c + 1) * 512]) - np.float32(mean[c])) * np.float32(
            1.0 / np.float32(std[c]))
    xn = ora.round_bf16(xn.astype(np.float32).astype(np.float64))
    p64 = {}
    for k, v in params.items():
        p64[k] = ora.round_bf16(v.astype(np.float64)) if k.startswith("W") else v.astype(np.float64)
    return xn, p64


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_loss_and_gradients_match_oracle_backprop(gpu, sess):
    S = gpu
    samples = _data(nel=6)  # 432 samples
    params = si.ae_init_params()
    ae = S.sem_ae_create(sess.ctx, 256)
    try:
        S.sem_ae_set_params(sess.ctx, ae, params)
        S.sem_ae_fit_normalization(sess.ctx, ae, samples)
        mean, std = S.sem_ae_get_normalization(sess.ctx, ae)
        # normalisation: per-component means, one common scale
        x = samples.double().cpu().numpy().reshape(-1, 3, 512)
        assert np.allclose(mean, x.mean(axis=(0, 2)), rtol=1e-5, atol=1e-7)
        assert np.allclose(std, np.sqrt(x.var(axis=(0, 2)).mean()), rtol=1e-5)
        rng = np.random.default_rng(7)
        idx_h = rng.choice(samples.shape[0], 200, replace=False)  # a partial batch (200 of 256 rows)
        idx = torch.as_tensor(idx_h, dtype=torch.int64, device="cuda")
        loss, g = S.sem_ae_loss_grad(sess.ctx, ae, samples, idx)
        xn, p64 = _oracle_inputs(samples, idx_h, mean, std, params)
        l_ref, cache = ora.forward(p64, xn, latent_round=ora.round_bf16)
        g_ref = ora.backward(p64, cache)
        assert abs(loss - l_ref) <= 1e-2 * l_ref, (loss, l_ref)
        # The bar for the gradients.  The oracle runs the same network in FP64 with the same
        # BF16 weights and BF16 latent; the GPU also rounds every activation and back-propagated
        # tensor to BF16 (unit roundoff u = 2^-8).  A gradient entry depends on at most 8 such
        # rounded tensors (X, H1/A1, the latent, H3/A3, dY, dH3, dZ, dH1), so its relative error
        # is below 8u = 3.1 % if every rounding pushed the same way, and near sqrt(8/3) u = 0.6 %
        # for uncorrelated roundings; the FP32 accumulation (K <= 1536 terms, 2^-24 each) and
        # the GELU' evaluation add well under 0.1 %.  Relative L2 error < 5 % (the aligned case with
        # margin) and cosine > 0.998 (an error of that size at right angles to the gradient).
        for k in g_ref:
            r = _rel(g[k].astype(np.float64), g_ref[k])
            cos = float(np.dot(g[k].ravel(), g_ref[k].ravel()) /
                        (np.linalg.norm(g[k]) * np.linalg.norm(g_ref[k]) + 1e-300))
            assert r < 5e-2 and cos > 0.998, (k, r, cos)
        # a second call after a full batch must not see the full batch's rows
        full = torch.as_tensor(rng.choice(samples.shape[0], 256, replace=False), dtype=torch.int64, device="cuda")
        S.sem_ae_loss_grad(sess.ctx, ae, samples, full, want_grad=False)
        loss2, g2 = S.sem_ae_loss_grad(sess.ctx, ae, samples, idx)
        assert abs(loss2 - loss) <= 1e-6 * loss  # the loss is summed with float atomics; gradients are not
        for k in g:
            assert np.array_equal(g2[k], g[k]), k
    finally:
        S.sem_ae_destroy(ae)


def test_adamw_step_matches_oracle_update(gpu, sess):
    S = gpu
    samples = _data(snaps=(3, 4))  # 128 samples
    params = si.ae_init_params(seed=11)
    ae = S.sem_ae_create(sess.ctx, 128)
    try:
        S.sem_ae_set_params(sess.ctx, ae, params)
        S.sem_ae_fit_normalization(sess.ctx, ae, samples)
        idx = torch.arange(0, 128, dtype=torch.int64, device="cuda")
        _, g = S.sem_ae_loss_grad(sess.ctx, ae, samples, idx)
        hp = dict(lr=3e-3, beta1=0.9, beta2=0.99, eps=1e-8, weight_decay=0.01)
        S.sem_ae_train_step(sess.ctx, ae, samples, idx, **hp)
        got = S.sem_ae_get_params(sess.ctx, ae)
        m, v, step = S.sem_ae_get_state(sess.ctx, ae)
        assert step == 1
        p64 = {k: v_.astype(np.float64) for k, v_ in params.items()}
        g64 = {k: v_.astype(np.float64) for k, v_ in g.items()}
        z = {k: np.zeros_like(v_) for k, v_ in p64.items()}
        ref, M, V = ora.adamw_step(p64, g64, z, z, 1, hp["lr"], hp["beta1"], hp["beta2"], hp["eps"], hp["weight_decay"])
        for k in ref:
            # FP32 update: a few ulps of the weight, plus the normalised step's own rounding
            # (1 - beta and the bias corrections in FP32 move m/sqrt(v) by ~1e-6 relative)
            tol = 4 * 2.0 ** -24 * np.abs(ref[k]) + 1e-5 * hp["lr"] + 1e-12
            assert (np.abs(got[k] - ref[k]) <= tol).all(), k
        mm = S.ae_unflatten(m)
        for k in M:
            assert np.allclose(mm[k], M[k], rtol=1e-6, atol=1e-30), k
    finally:
        S.sem_ae_destroy(ae)


def test_padded_latent_weights_stay_zero_and_training_lowers_the_loss(gpu, sess):
    S = gpu
    samples = _data(nel=6, snaps=(0, 5, 10, 15))
    ae = S.sem_ae_create(sess.ctx, 512)
    try:
        S.sem_ae_set_params(sess.ctx, ae, si.ae_init_params())
        S.sem_ae_fit_normalization(sess.ctx, ae, samples)
        g = torch.Generator(device="cuda")
        g.manual_seed(si.seed_for(5, 999))
        evalidx = torch.arange(0, 512, dtype=torch.int64, device="cuda")
        l0, _ = S.sem_ae_loss_grad(sess.ctx, ae, samples, evalidx, want_grad=False)
        for _ in range(300):
            idx = torch.randint(0, samples.shape[0], (512,), generator=g, device="cuda")
            S.sem_ae_train_step(sess.ctx, ae, samples, idx, lr=1e-3, weight_decay=0.0)
        l1, _ = S.sem_ae_loss_grad(sess.ctx, ae, samples, evalidx, want_grad=False)
        assert l1 < 0.2 * l0, (l0, l1)
        S.sem_synchronize(sess.ctx)
    finally:
        S.sem_ae_destroy(ae)


def test_encode_decode_match_oracle(gpu, sess):
    S = gpu
    samples = _data(snaps=(2,))
    params = si.ae_init_params(seed=5)
    E = samples.shape[0]  # 64 elements: one partial chunk of 128
    f = si.ae_snapshot(2, nel=4, device="cuda")
    ae = S.sem_ae_create(sess.ctx, 128)
    try:
        S.sem_ae_set_params(sess.ctx, ae, params)
        S.sem_ae_fit_normalization(sess.ctx, ae, samples)
        mean, std = S.sem_ae_get_normalization(sess.ctx, ae)
        lat = torch.empty(E * 48, dtype=torch.bfloat16, device="cuda")
        S.sem_ae_encode(sess.ctx, ae, f[0].contiguous(), f[1].contiguous(), f[2].contiguous(), lat)
        out = [torch.full((E, 512), float("nan"), device="cuda") for _ in range(3)]
        S.sem_ae_decode(sess.ctx, ae, lat, E, *out)
        torch.cuda.synchronize()
        xn, p64 = _oracle_inputs(samples, np.arange(E), mean, std, params)
        z_ref = ora.encode(p64, xn)
        z = lat.float().cpu().double().numpy().reshape(E, 48)
        assert _rel(z, z_ref) < 2e-2
        y_ref = ora.decode(p64, ora.round_bf16(z))
        y = np.concatenate([((o.cpu().double().numpy() - mean[c]) / std[c]) for c, o in enumerate(out)], axis=1)
        assert np.isfinite(y).all()
        assert _rel(y, y_ref) < 2e-2
    finally:
        S.sem_ae_destroy(ae)


def test_sample_index_out_of_range_is_flagged(gpu, sess):
    S = gpu
    samples = _data(snaps=(1,))  # 64 samples
    ae = S.sem_ae_create(sess.ctx, 128)
    try:
        S.sem_ae_set_params(sess.ctx, ae, si.ae_init_params())
        S.sem_ae_fit_normalization(sess.ctx, ae, samples)
        idx = torch.tensor([0, 1, 64, -1], dtype=torch.int64, device="cuda")
        S.sem_ae_loss_grad(sess.ctx, ae, samples, idx, want_grad=False)
        with pytest.raises(S.SemError) as ex:
            S.sem_synchronize(sess.ctx)
        assert ex.value.status == S.SEM_ERR_ARG
        S.sem_synchronize(sess.ctx)  # cleared
    finally:
        S.sem_ae_destroy(ae)


def test_checkpoint_resume_continues_identically(gpu, sess):
    S = gpu
    samples = _data(snaps=(4,))
    a = S.sem_ae_create(sess.ctx, 128)
    b = S.sem_ae_create(sess.ctx, 128)
    try:
        S.sem_ae_set_params(sess.ctx, a, si.ae_init_params(seed=2))
        S.sem_ae_fit_normalization(sess.ctx, a, samples)
        idx = torch.arange(0, 64, dtype=torch.int64, device="cuda")
        for _ in range(3):
            S.sem_ae_train_step(sess.ctx, a, samples, idx, lr=1e-3)
        # checkpoint a -> b
        S.sem_ae_set_params(sess.ctx, b, S.sem_ae_get_params(sess.ctx, a))
        m, v, step = S.sem_ae_get_state(sess.ctx, a)
        S.sem_ae_set_state(sess.ctx, b, m, v, step)
        mu, sd = S.sem_ae_get_normalization(sess.ctx, a)
        S.sem_ae_set_normalization(sess.ctx, b, mu, sd)
        for x in (a, b):
            S.sem_ae_train_step(sess.ctx, x, samples, idx, lr=1e-3)
        pa, pb = S.sem_ae_get_params(sess.ctx, a), S.sem_ae_get_params(sess.ctx, b)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), k
    finally:
        S.sem_ae_destroy(a)
        S.sem_ae_destroy(b)
