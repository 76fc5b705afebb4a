"""sem_isosurface_noalloc, the allocation-free isosurface entry point, against sem_isosurface.

Some callers may not allocate device memory while they run (an in situ hook inside a solver
step whose GPU memory the solver has already committed); for them the library keeps the
isosurface scratch in a fixed device array.  This file runs last (its name sorts last) so a
failure here stops a `-x` run only after every other test has run.  It also passes alone in a
fresh process: sem_create looks the array's address up and loads the entry point's kernels.
The cases span both scan forms whose state the fixed scratch holds: one block (up to 8192
elements) and the single-pass look-back scan over tiles of 4096 beyond, up to the limit;
results are checked against the regular entry point and against the oracle.
"""
import math

import numpy as np
import pytest
import torch

import sem_inputs as si
from _helpers import host64

pytestmark = pytest.mark.gpu


def _both(S, ctx, m, f, iso, E, N):
    """Run the regular and the allocation-free entry point on the same input."""
    out = []
    for fn in (S.sem_isosurface, S.sem_isosurface_noalloc):
        cases = torch.zeros(E * N ** 3, dtype=torch.uint8, device="cuda")
        n = fn(ctx, m, f, iso, None)
        tris = torch.full((max(n, 1) * 9,), -3.0, device="cuda")
        te = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        assert fn(ctx, m, f, iso, tris, te, cases) == n
        torch.cuda.synchronize()
        out.append((n, tris[:n * 9].cpu(), te[:n].cpu(), cases.cpu()))
    return out


def test_noalloc_matches_regular_entry_point_twice(gpu, sess):
    S = gpu
    w = si.tgv_box(nel=6, N=7)
    m = sess.mesh(7, w.mesh.xyz().numpy())
    u, v, ww = (w.fields[c].float().cuda().contiguous() for c in range(3))
    Q = torch.empty_like(u)
    S.sem_qcriterion(sess.ctx, m, u, v, ww, Q)
    qmax = S.sem_field_max(sess.ctx, Q)
    # two calls in a row with different isovalues: the second must not see the first's scratch
    for frac in (0.1, 0.3):
        iso = float(np.float32(frac * qmax))
        (n0, t0, e0, c0), (n1, t1, e1, c1) = _both(S, sess.ctx, m, Q, iso, w.E, 7)
        assert n0 == n1 and n0 > 0
        assert torch.equal(c0, c1)
        assert torch.equal(e0, e1)
        assert (t0.double() - t1.double()).abs().max().item() <= 1e-5 * 2 * math.pi


def test_noalloc_rejects_meshes_beyond_its_limit(gpu, sess):
    S = gpu
    E = S.SEM_NOALLOC_MAX_ELEMENTS + 1
    mesh = si.uniform_box((E, 1, 1), (0, 0, 0), (float(E), 1, 1), 1)
    m = sess.mesh(1, mesh.xyz().numpy())
    f = torch.zeros(E * 8, device="cuda")
    with pytest.raises(S.SemError) as ex:
        S.sem_isosurface_noalloc(sess.ctx, m, f, 0.5, None)
    assert ex.value.status == S.SEM_ERR_ARG
    assert str(S.SEM_NOALLOC_MAX_ELEMENTS) in str(ex.value)


@pytest.mark.parametrize("N,nel", [(2, 47), (1, 58)])
def test_noalloc_large_meshes_against_oracle(gpu, sess, orc, N, nel):
    """103823 elements of order 2 (26 tiles of the look-back scan) and 195112 elements of
    order 1 (48 tiles, their status words in the fixed array), a sphere |x - c|^2 = r^2 at two
    radii in a row: every cell's case and every element's triangle count equal the oracle's from
    the same FP32 field, and the triangles equal sem_isosurface's."""
    S = gpu
    mesh = si.uniform_box((nel,) * 3, (0.0,) * 3, (1.0,) * 3, N)
    xyz = mesh.xyz().numpy()
    m = sess.mesh(N, xyz)
    E = mesh.E
    assert E > (131072 if N == 1 else 8192)
    for r in (0.31, 0.42):
        f = si.sphere_field(mesh, (0.47, 0.52, 0.5), r)
        f32 = f.float().cuda().contiguous()
        (n0, t0, e0, c0), (n1, t1, e1, c1) = _both(S, sess.ctx, m, f32, 0.0, E, N)
        assert n0 == n1 and n0 > 1000
        assert torch.equal(c0, c1) and torch.equal(e0, e1)
        assert (t0.double() - t1.double()).abs().max().item() <= 1e-5
        ref = orc.isosurface(N, xyz, host64(f32).reshape(E, -1), 0.0, want_tris=False)
        np.testing.assert_array_equal(c1.numpy().reshape(E, -1), ref["cases"])
        np.testing.assert_array_equal(np.bincount(e1.numpy(), minlength=E), ref["elem_ntri"])
        assert n1 == ref["ntri"]
