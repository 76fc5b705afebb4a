"""Shared test helpers: FP32 error bounds for the derivative / Q kernels and comparisons.

The bounds follow from the arithmetic: an FP32 dot product of n terms (fused multiply-adds)
has error at most about n * 2^-24 * sum |D_im u_m|; rounding D to FP32 adds 2^-24 * sum |D_im
u_m|; scaling by the FP32 factor 2/h adds 2 * 2^-24 |result|.  A safety factor of 2 covers
the remaining second-order terms.  The FP64 oracle's own error is added as a floor of
1e-12 times the node's largest gradient entry (its general chain rule carries D's row-sum
rounding, ~1e-14, times coordinate/size ratios).  Q = -1/2 sum J_ij J_ji then inherits
|dQ| <= sum_ij (|J_ij| + dJ_ij) dJ_ji + 16 * 2^-24 sum |J_ij J_ji| (each of the six product
terms carries at most 5 roundings from its coefficient -g_i g_j/2 and products, and the
accumulation of six terms at most 6 more).
"""
import numpy as np
import torch

EPS32 = 2.0 ** -24


def dev32(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda().contiguous()


def host64(t):
    return t.detach().cpu().double().numpy()


def ref_abs_contractions(D, u, NP):
    """sum_m M[i][m] (|u_m| + |u_0| + |u_N|) along r, s, t for u (E, NP^3) -> three (E, NP^3)
    arrays, with M[i][m] = max(|D[i][m]|, |D[i][N-m]|) and u_0, u_N the ends of the line through
    the node.  D is centro-antisymmetric (GLL nodes are symmetric), so a kernel may contract with
    the even/odd parts u_m +- u_{N-m} and the coefficients (D[i][m] +- D[i][N-m])/2; their
    rounding error is bounded by the same sums with |(x+y)/2| + |(x-y)/2| = max(|x|, |y|) in
    place of |D[i][m]|.  M >= |D|, so the bound also covers the plain contraction.  The kernels
    subtract the line's first value (or, in the even/odd form, the first even part u_0 + u_N)
    from the line before the products (D's rows sum to zero, so the result is unchanged in exact
    arithmetic); that subtraction rounds each operand with an error of at most
    eps (|u_m| + |u_0| + |u_N|), hence the ends' term."""
    A = np.maximum(np.abs(D), np.abs(D[:, ::-1]))
    rs = A.sum(axis=1)
    U = np.abs(u).reshape(-1, NP, NP, NP)  # [e][k][j][i]
    ends_r = U[:, :, :, :1] + U[:, :, :, -1:]
    ends_s = U[:, :, :1, :] + U[:, :, -1:, :]
    ends_t = U[:, :1, :, :] + U[:, -1:, :, :]
    br = np.einsum("im,ekjm->ekji", A, U) + rs[None, None, None, :] * ends_r
    bs = np.einsum("jm,ekmi->ekji", A, U) + rs[None, None, :, None] * ends_s
    bt = np.einsum("km,emji->ekji", A, U) + rs[None, :, None, None] * ends_t
    return [b.reshape(u.shape) for b in (br, bs, bt)]


def grad_bounds(D, u, g, NP, ref):
    """Per-node bounds on |grad_gpu - grad_oracle| for one FP32 field u (E, NP^3); g (E, 3) the
    factors 2/h; ref (3, E, NP^3) the oracle gradient."""
    bs = ref_abs_contractions(D, u, NP)
    floor = 1e-12 * np.abs(ref).max(axis=0)
    return np.stack([2.0 * ((NP + 1) * np.abs(g[:, a:a + 1]) * bs[a] + 2.0 * np.abs(ref[a])) * EPS32 + floor
                     for a in range(3)])


def grad_bounds_prec(D, u, g, NP, ref, eps_st, abs_st=0.0):
    """As grad_bounds, with the s- and t-contractions done in a 16-bit type: rounding the
    element data and D to it (unit roundoff eps_st each) adds 2 eps_st sum |D||u - c| per node,
    where c is the value the kernel subtracts from the node's column (i fixed) before rounding,
    the column's first value u[0][0][i] (the contraction operators' rows sum to zero, so the
    shift leaves the result unchanged); |u - c| <= |u| + |c|.  Values below the type's normal
    range round with an absolute error abs_st instead (FP16: 2^-25), adding abs_st sum |D|."""
    bs = ref_abs_contractions(D, u, NP)
    A = np.maximum(np.abs(D), np.abs(D[:, ::-1]))
    U = np.abs(u).reshape(-1, NP, NP, NP)
    col = np.broadcast_to(U[:, :1, :1, :], U.shape)  # |c| of each node's column
    cs = [None, (np.einsum("jm->j", A)[None, None, :, None] * col).reshape(u.shape),
          (np.einsum("km->k", A)[None, :, None, None] * col).reshape(u.shape)]
    dsum = np.abs(D).sum(axis=1).max()
    floor = 1e-12 * np.abs(ref).max(axis=0)
    out = []
    for a in range(3):
        e_in = 0.0 if a == 0 else 2.0 * eps_st
        a_in = 0.0 if a == 0 else 2.0 * abs_st * dsum
        data = bs[a] if a == 0 else bs[a] + cs[a]
        out.append(((2.0 * (NP + 1) * EPS32) * bs[a] + 2.0 * e_in * data + a_in) * np.abs(g[:, a:a + 1])
                   + 4.0 * EPS32 * np.abs(ref[a]) + floor)
    return np.stack(out)


def q_bound(J, dJ):
    """J, dJ: (3, 3, ...) gradient and its per-entry bound -> per-node bound on Q."""
    b = np.zeros(J.shape[2:])
    s = np.zeros(J.shape[2:])
    for i in range(3):
        for j in range(3):
            b += (np.abs(J[i, j]) + dJ[i, j]) * dJ[j, i]
            s += np.abs(J[i, j] * J[j, i])
    return b + 16.0 * EPS32 * s + 1e-30


def box_factors(xyz):
    """2/h per element and axis from node coordinates (3, E, NP^3)."""
    NP = round(xyz.shape[2] ** (1 / 3))
    x0 = xyz[:, :, 0]
    x1 = np.stack([xyz[0, :, NP - 1], xyz[1, :, NP * (NP - 1)], xyz[2, :, NP * NP * (NP - 1)]])
    return (2.0 / (x1 - x0)).T


def compare_images(img, dep, ref_img, ref_dep, min_frac=0.999):
    """GPU frame against the oracle's from the same FP32 triangles.  Colour: every channel
    within 1/255 on >= 99.9% of pixels; the pixels beyond are those whose centre lies within
    FP32 rounding of a triangle edge, where the two sides can pick different winners (often on
    different surfaces, at any depth).  Depth, where both sides cover the pixel with colours
    within 1/255 (the same winner, or an adjacent one of the same surface): within 1e-5 on
    >= 99.9% of those pixels (the rest are sliver triangles, whose FP32 depth plane has steep
    gradients) and within 1e-3 on all of them.  Returns (fraction of pixels within 1/255,
    fraction of the depth-compared pixels within 1e-5)."""
    close = (np.abs(img.astype(int) - ref_img.astype(int)) <= 1).all(axis=2)
    frac = close.mean()
    assert frac >= min_frac, frac
    both = (img[..., 3] > 0) & (ref_img[..., 3] > 0) & close
    dfrac = 1.0
    if both.any():
        dz = np.abs(dep[both] - ref_dep[both])
        dfrac = (dz <= 1e-5).mean()
        assert dfrac >= min_frac, dfrac
        assert dz.max() <= 1e-3, dz.max()
    return frac, dfrac
