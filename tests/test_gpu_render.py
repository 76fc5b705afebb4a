"""GPU parity of sem_render against the oracle's rasteriser (through the C ABI).

Same FP32 triangles on both sides.  Bar: every channel within 1/255 on at least 99.9% of
pixels; depth within 1e-5 on at least 99.9% (and within 1e-3 on all) of the pixels both sides
cover with colours within 1/255; exact coverage on cases whose projected coordinates are exact
in FP32.
"""
import math

import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import compare_images as _compare_images, dev32, host64

pytestmark = pytest.mark.gpu


def _render(S, sess, tris32, seg, rgb, cam):
    W, H = cam["W"], cam["H"]
    rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
    depth = torch.zeros(H * W, device="cuda")
    n = tris32.numel() // 9
    S.sem_render(sess.ctx, tris32 if n else None, n, seg, rgb, cam, W, H, rgba, depth)
    torch.cuda.synchronize()
    return rgba.cpu().numpy().reshape(H, W, 4), depth.cpu().numpy().reshape(H, W)


def test_random_triangles_perspective(gpu, sess, orc):
    rng = np.random.default_rng(1)
    cam = si.camera(False, (3, 2, 9.0), (0, 0, 0), (0, 1, 0), 320, 200, fovy_deg=50.0, znear=1.0, zfar=20.0)
    c = rng.uniform(-3, 3, size=(3000, 1, 3))
    tris = c + rng.normal(0, 0.3, size=(3000, 3, 3))
    t32 = dev32(tris.reshape(-1))
    seg, rgb = [1000, 1500, 500], [[0.9, 0.3, 0.2], [0.2, 0.6, 0.9], [0.95, 0.95, 0.95]]
    img, dep = _render(gpu, sess, t32, seg, rgb, cam)
    ref_img, ref_dep, _ = orc.render(host64(t32).reshape(-1, 3, 3), seg, rgb, cam)
    _compare_images(img, dep, ref_img, ref_dep)


def test_random_triangles_ortho_large_and_clipped(gpu, sess, orc):
    rng = np.random.default_rng(2)
    cam = si.camera(True, (0, 0, 10.0), (0, 0, 0), (0, 1, 0), 257, 131, half_h=4.0, znear=2.0, zfar=18.0)
    tris = rng.uniform(-9, 9, size=(400, 3, 3))  # large, partly off-screen, some crossing the clip range
    t32 = dev32(tris.reshape(-1))
    img, dep = _render(gpu, sess, t32, [400], None, cam)
    pal = [[0.90, 0.35, 0.25]]
    ref_img, ref_dep, _ = orc.render(host64(t32).reshape(-1, 3, 3), [400], pal, cam)
    _compare_images(img, dep, ref_img, ref_dep)


def test_every_box_size_class(gpu, sess, orc):
    """Triangles whose boxes (clamped to the image) hold <= 32 pixel centres (the warps' balanced
    lists) and more (the large-triangle pass: a warp per triangle, its lanes stepping 32
    candidates at a time), from 33 up to well over 4096 centres, overlapping at random depths,
    one pixel per world unit."""
    rng = np.random.default_rng(6)
    W, H = 160, 128
    cam = si.camera(True, (W / 2, H / 2, 10.0), (W / 2, H / 2, 0), (0, 1, 0), W, H, half_h=H / 2, znear=1.0,
                    zfar=19.0)
    tris, classes = [], []
    for size, count in ((4.0, 600), (12.0, 200), (40.0, 60), (90.0, 24)):
        for _ in range(count):
            c = rng.uniform((0, 0), (W, H))
            ang = rng.uniform(0, 2 * np.pi) + np.array([0.0, 2.1, 4.2]) + rng.uniform(-0.4, 0.4, 3)
            r = size * rng.uniform(0.5, 1.0, 3)
            z = rng.uniform(-3, 3, 3)
            v = np.stack([c[0] + r * np.cos(ang), c[1] + r * np.sin(ang), z], axis=1)
            tris.append(v)
            # pixel centres of the box clamped to the image (the y flip does not change counts)
            x0, x1 = max(0, np.ceil(v[:, 0].min() - 0.5)), min(W - 1, np.floor(v[:, 0].max() - 0.5))
            y0, y1 = max(0, np.ceil(v[:, 1].min() - 0.5)), min(H - 1, np.floor(v[:, 1].max() - 0.5))
            classes.append(max(0, x1 - x0 + 1) * max(0, y1 - y0 + 1))
    classes = np.array(classes)
    assert (classes <= 32).sum() > 100 and ((classes > 32) & (classes <= 4096)).sum() > 100
    assert (classes > 4096).sum() >= 10
    t32 = dev32(np.array(tris).reshape(-1))
    n = len(tris)
    seg, rgb = [n // 2, n - n // 2], [[0.9, 0.3, 0.2], [0.2, 0.6, 0.9]]
    img, dep = _render(gpu, sess, t32, seg, rgb, cam)
    ref_img, ref_dep, _ = orc.render(host64(t32).reshape(-1, 3, 3), seg, rgb, cam)
    _compare_images(img, dep, ref_img, ref_dep)
    assert (img[..., 3] > 0).mean() > 0.5


def test_exact_fan_coverage(gpu, sess, orc):
    # pixel-centre-aligned square split into 4 triangles: every covered pixel exactly once
    W = H = 16
    cam = si.camera(True, (8, 8, 10.0), (8, 8, 0), (0, 1, 0), W, H, half_h=8.0, znear=1.0, zfar=19.0)
    corners = [(1.5, 1.5, 0), (13.5, 1.5, 0), (13.5, 13.5, 0), (1.5, 13.5, 0)]
    c = (7.5, 7.5, 0)
    tris = np.array([[corners[i], corners[(i + 1) % 4], c] for i in range(4)], float)
    cnt = np.zeros((H, W), int)
    for i in range(4):
        img, _ = _render(gpu, sess, dev32(tris[i].reshape(-1)), [1], [[1, 1, 1]], cam)
        _, _, win = orc.render(tris[i:i + 1], [1], [[1, 1, 1]], cam)
        np.testing.assert_array_equal(img[..., 3] > 0, win >= 0)
        cnt += img[..., 3] > 0
    assert cnt.max() == 1
    assert cnt.sum() == 12 * 12


def test_tie_break_lower_index_and_determinism(gpu, sess, orc):
    cam = si.camera(True, (0, 0, 10.0), (0, 0, 0), (0, 1, 0), 64, 64, half_h=2.0, znear=1.0, zfar=19.0)
    t = np.array([[(-1.5, -1.5, 0.5), (1.7, -1.1, 0.5), (0.2, 1.8, 0.5)]])
    tris = np.concatenate([t, t])
    img, _ = _render(gpu, sess, dev32(tris.reshape(-1)), [1, 1], [[1, 0, 0], [0, 1, 0]], cam)
    cov = img[..., 3] > 0
    assert cov.any() and (img[cov][:, 1] == 0).all()  # the first triangle (red) wins every tie
    rng = np.random.default_rng(4)
    many = dev32(rng.uniform(-2, 2, size=(5000 * 9,)))
    a = _render(gpu, sess, many, [5000], None, cam)
    b = _render(gpu, sess, many, [5000], None, cam)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_empty_scene(gpu, sess):
    cam = si.camera(True, (0, 0, 10.0), (0, 0, 0), (0, 1, 0), 40, 30, half_h=2.0, znear=1.0, zfar=19.0)
    img, dep = _render(gpu, sess, torch.zeros(0, device="cuda"), [0], None, cam)
    assert (img == 0).all() and (dep == 1.0).all()


def test_taylor_green_frame(gpu, sess, orc):
    """The 8^3, N=7 workload's Q-isosurface (GPU triangles) rendered 256x256 by both sides."""
    w = si.tgv_box()
    xyz = w.mesh.xyz().numpy()
    m = sess.mesh(7, xyz)
    u, v, ww = (dev32(w.fields[c].numpy()) for c in range(3))
    Q = torch.empty_like(u)
    gpu.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    iso = float(np.float32(0.1 * gpu.sem_field_max(sess.ctx, Q)))
    n = gpu.sem_isosurface(sess.ctx, m, Q, iso, None, cap=0)
    tris = torch.empty(n * 9, device="cuda")
    gpu.sem_isosurface(sess.ctx, m, Q, iso, tris)
    img, dep = _render(gpu, sess, tris, [n], None, w.camera)
    ref_img, ref_dep, _ = orc.render(host64(tris).reshape(-1, 3, 3), [n], [[0.90, 0.35, 0.25]], w.camera)
    _compare_images(img, dep, ref_img, ref_dep)
    assert (img[..., 3] > 0).mean() > 0.2


def test_bad_camera_and_segments(gpu, sess):
    cam = si.camera(True, (0, 0, 10.0), (0, 0, 0), (0, 0, 1), 8, 8, half_h=2.0, znear=1.0, zfar=19.0)
    rgba = torch.zeros(8 * 8 * 4, dtype=torch.uint8, device="cuda")
    t = torch.zeros(9, device="cuda")
    with pytest.raises(gpu.SemError):  # up parallel to the view direction
        gpu.sem_render(sess.ctx, t, 1, [1], None, cam, 8, 8, rgba)
    cam["up"] = [0, 1, 0]
    with pytest.raises(gpu.SemError):  # segments do not sum to ntri
        gpu.sem_render(sess.ctx, t, 1, [2], None, cam, 8, 8, rgba)


def test_channel_benchmark_frame_full_size(gpu, sess, orc):
    """The benchmark's secondary frame at full size: the 32^3-element channel's three
    Q-isosurfaces (about 5.1M GPU triangles, mean area ~1.3 px) rendered 1920x1080 by both
    sides from the same FP32 triangles, in the launch configuration bench.py times."""
    w = si.channel(device="cuda")
    m = sess.mesh(7, w.mesh.xyz("cuda").cpu().numpy())
    vel = [w.fields[c].float().contiguous() for c in range(3)]
    w.fields = None
    Q = torch.empty_like(vel[0])
    gpu.sem_qcriterion(sess.ctx, m, *vel, Q)
    qmax = gpu.sem_field_max(sess.ctx, Q)
    isos = [float(np.float32(f * qmax)) for f in w.iso_fracs]
    counts = gpu.sem_isosurface_multi(sess.ctx, m, Q, isos, None)
    n = sum(counts)
    assert n > 4_000_000
    tris = torch.empty(n * 9, device="cuda")
    gpu.sem_isosurface_multi(sess.ctx, m, Q, isos, tris)
    img, dep = _render(gpu, sess, tris, counts, None, w.camera)
    pal = [[0.90, 0.35, 0.25], [0.25, 0.60, 0.90], [0.35, 0.85, 0.40]]
    ref_img, ref_dep, _ = orc.render(host64(tris).reshape(-1, 3, 3), counts, pal, w.camera)
    frac, dfrac = _compare_images(img, dep, ref_img, ref_dep)
    assert (img[..., 3] > 0).mean() > 0.2
    print(f"\nchannel 32^3 frame: {n} triangles, {frac * 100:.3f}% of pixels within 1/255, "
          f"{dfrac * 100:.3f}% of compared depths within 1e-5")


@pytest.mark.parametrize("nseg,seed", [(3, 1), (40, 2), (64, 3)])
def test_render_segments_mask_draws_only_the_chosen_segments(gpu, sess, nseg, seed):
    """sem_render_segments_async with a segment mask equals sem_render of the same buffer in which
    the triangles of the segments not drawn are made degenerate (zero area: dropped) at the same
    indices, bit for bit in colour and depth; one colour for all segments, up to 64 segments with
    uneven boundaries."""
    S = gpu
    w = si.tgv_box(nel=6)
    m = sess.mesh(7, w.mesh.xyz().numpy())
    vel = [w.fields[c].float().cuda().contiguous() for c in range(3)]
    Q = torch.empty_like(vel[0])
    S.sem_qcriterion(sess.ctx, m, *vel, Q)
    qmax = S.sem_field_max(sess.ctx, Q)
    isos = [float(np.float32(f * qmax)) for f in (0.05, 0.1, 0.2)]
    counts = S.sem_isosurface_multi(sess.ctx, m, Q, isos, None)
    n = sum(counts)
    tris = torch.empty(n * 9, device="cuda")
    S.sem_isosurface_multi(sess.ctx, m, Q, isos, tris)
    rng = np.random.default_rng(seed)
    if nseg == 3:
        starts = np.concatenate([[0], np.cumsum(counts)])
        mask = 0b101
    else:
        starts = np.concatenate([[0], np.sort(rng.choice(np.arange(1, n), nseg - 1, replace=False)), [n]])
        mask = int(rng.integers(1, 1 << 62)) | (1 << (nseg - 1))
    sd = torch.as_tensor(starts.astype(np.int64), device="cuda")
    cam, W, H = w.camera, w.camera["W"], w.camera["H"]
    rgba = torch.zeros(H * W * 4, dtype=torch.uint8, device="cuda")
    depth = torch.zeros(H * W, device="cuda")
    S.sem_render_segments_async(sess.ctx, tris, n, sd, nseg, [[0.8, 0.4, 0.2]] * nseg, mask, cam, W, H, rgba, depth)
    ref_t = tris.clone().view(-1, 9)
    for sgm in range(nseg):
        if not (mask >> sgm) & 1:
            ref_t[starts[sgm]:starts[sgm + 1]] = 0.0
    r_rgba = torch.zeros_like(rgba)
    r_depth = torch.zeros_like(depth)
    S.sem_render(sess.ctx, ref_t.view(-1), n, [n], [[0.8, 0.4, 0.2]], cam, W, H, r_rgba, r_depth)
    S.sem_synchronize(sess.ctx)
    assert torch.equal(rgba, r_rgba) and torch.equal(depth, r_depth)
    assert (rgba.view(-1, 4)[:, 3] > 0).any()
