"""The arithmetic identities the rasteriser's kernels rely on, checked exhaustively or on large
samples on the CPU (no GPU): each replaces a costlier exact computation, so each must hold for
every input the kernel can see.

* Coverage on float bits: for a float e that is neither -0 nor NaN, "e > 0, or e == 0 on a
  top-left edge" equals int_bits(e) + tl > 0.
* Box row of candidate k: (k * ceil(1024 / nx)) >> 10 == k // nx for 0 <= k < 32, nx <= 32, with
  the multiplier from an approximate quotient int(q - 2^-8) + 1; and floor((k + .5) RN(1/nx))
  in FP32 == k // nx for k, nx <= 1024.
* Stepping: lane l starting at candidate l and advancing 32 candidates as q rows and r columns
  visits every candidate of an nx x ny box once.
* Candidate owner: with the warp's lists placed back to back, the owner of candidate idx has
  rank (list starts before the round) + popc(starts in the round at or below idx) - 1 among the
  lanes that have candidates.
"""
import numpy as np

import sem_inputs as si


def _bits(x):
    return np.asarray(x, np.float32).view(np.int32).astype(np.int64)


def test_top_left_coverage_on_float_bits():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(200000).astype(np.float32),
                           (rng.standard_normal(20000) * 1e-38).astype(np.float32),  # subnormals
                           np.array([0.0, 1e-45, -1e-45, 3.4e38, -3.4e38, np.inf, -np.inf], np.float32),
                           (rng.integers(-8, 9, 4000) * np.float32(0.25)).astype(np.float32)])
    for tl in (0, 1):
        ref = (vals > 0) | ((vals == 0) & bool(tl))
        np.testing.assert_array_equal((_bits(vals) + tl) > 0, ref)


def test_exact_zero_of_a_sum_is_plus_zero():
    """x + 0 turns -0 into +0; a round-to-nearest sum of exactly cancelling terms is +0, so a
    plane value a + b kx + c ky with a != -0 and kx, ky >= 0 is never -0."""
    z = np.float32(-0.0) + np.float32(0.0)
    assert not np.signbit(z)
    rng = np.random.default_rng(1)
    for _ in range(20000):
        a = np.float32(rng.integers(-8, 9) * 0.25) + np.float32(0.0)
        b, c = (np.float32(rng.integers(-8, 9) * 0.25) for _ in range(2))
        kx, ky = np.float32(rng.integers(0, 4)), np.float32(rng.integers(0, 4))
        e = c * ky + (b * kx + a)  # exact for these dyadic values, so equal to the FMA chain
        if e == 0:
            assert not np.signbit(e)


def test_box_row_multiply_shift():
    for nx in range(1, 33):
        q = np.float32(1024) / np.float32(nx)
        for ulps in range(-4, 5):  # the approximate quotient's error, with margin
            qq = q
            for _ in range(abs(ulps)):
                qq = np.nextafter(qq, np.float32(np.inf if ulps > 0 else -np.inf), dtype=np.float32)
            assert int(np.float32(qq - np.float32(1 / 256))) + 1 == -(-1024 // nx)
        mul = -(-1024 // nx)
        for k in range(32):
            assert (k * mul) >> 10 == k // nx


def test_box_row_float_reciprocal():
    k = np.arange(1024, dtype=np.int64)
    for nx in range(1, 1025):
        rnx = np.float32(1.0) / np.float32(nx)
        ky = ((k.astype(np.float32) + np.float32(0.5)) * rnx).astype(np.float32).astype(np.int64)
        np.testing.assert_array_equal(ky, k // nx)


def test_stepping_visits_every_candidate_once():
    for step in (32, 256):
        for nx in list(range(1, 70)) + [255, 256, 257, 1000]:
            for ny in (1, 2, 5, 33):
                seen = []
                for lane in range(step):
                    dq, dr = step // nx, step - (step // nx) * nx
                    ky, kx = lane // nx, lane - (lane // nx) * nx
                    while ky < ny:
                        seen.append(ky * nx + kx)
                        kx += dr
                        ky += dq
                        if kx >= nx:
                            kx -= nx
                            ky += 1
                assert sorted(seen) == list(range(nx * ny)), (step, nx, ny)


def test_candidate_owner_from_list_starts():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        npx = np.where(rng.random(32) < 0.3, 0, rng.integers(1, 33, 32))
        incl = np.cumsum(npx)
        excl = incl - npx
        total = int(incl[-1])
        owners = [L for L in range(32) if npx[L] > 0]
        before = 0
        for r in range(0, total, 32):
            starts = 0
            for L in owners:
                if 0 <= excl[L] - r < 32:
                    starts |= 1 << int(excl[L] - r)
            for lane in range(32):
                idx = r + lane
                rank = before + bin(starts & ((2 << lane) - 1) & 0xFFFFFFFF).count("1") - 1
                assert 0 <= rank < len(owners)
                if idx < total:
                    L = owners[rank]
                    assert excl[L] <= idx < incl[L]
            before += bin(starts).count("1")


def test_perturbed_box_is_conforming_and_curved():
    N, NP = 4, 5
    xyz = si.perturbed_box((3, 2, 2), (0, 0, 0), (1.5, 1, 1), N, amp=0.2, seed=1)
    X = xyz.reshape(3, 2, 2, 3, NP, NP, NP)  # [c][ez][ey][ex][k][j][i]
    # neighbours share their faces exactly
    assert np.abs(X[:, :, :, :-1, :, :, -1] - X[:, :, :, 1:, :, :, 0]).max() == 0
    assert np.abs(X[:, :, :-1, :, :, -1, :] - X[:, :, 1:, :, :, 0, :]).max() == 0
    assert np.abs(X[:, :-1, :, :, -1, :, :] - X[:, 1:, :, :, 0, :, :]).max() == 0
    # and the elements around the moved interior corners are not boxes
    box = si.uniform_box((3, 2, 2), (0, 0, 0), (1.5, 1, 1), N).xyz().numpy()
    assert np.abs(xyz - box).max() > 1e-3
