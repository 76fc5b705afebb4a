"""FP64 CPU oracle of the learned per-element compression (an MLP autoencoder) and of the
baseline it is judged against.

TEST INFRASTRUCTURE ONLY: the test-suite and bench.py's CPU-baseline leg are the only
callers; the CUDA library never imports this module and shares no code with it.

The paper moves NekRS fields off the simulation nodes for in-transit analysis (Sec. 4.2,
ADIOS2/SST) and names the transfer volume as the cost.  The learned part compresses each
spectral element's velocity before transfer: per element the 3 x (N+1)^3 = 1536 nodal values
(N = 7), z-scored per component with training statistics, go through

    encoder:  H1 = X W1^T + b1,  A1 = gelu(H1),  Z = A1 W2^T + b2          (1536 -> 512 -> 48)
    decoder:  H3 = Z W3^T + b3,  A3 = gelu(H3),  Y = A3 W4^T + b4          (48 -> 512 -> 1536)

with gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 (exact, no tanh approximation), no
activation on the latent Z or the output Y, loss = mean over all entries of (Y - X)^2, and
AdamW (Loshchilov & Hutter 2019: Adam moments with bias correction, weight decay decoupled
from the gradient).  The latent is what would be transferred.  Every function below is plain
numpy in float64 and follows those definitions term by term; the pins are in
tests/test_oracle_ae.py (central finite differences for the backward pass, closed forms for
gelu and the first AdamW step, exactness of the Legendre transform on polynomials, brute
force for the Hausdorff distance).

Baseline ("the method without it"): per element and component, the Legendre modal expansion
of the nodal values on the GLL grid (the interpolating tensor-product polynomial), truncated
to 16 modes per component: 48 values per element, the same payload as the 48-value latent.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)

LAYERS = (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4"))


def _erf(x: np.ndarray) -> np.ndarray:
    from scipy.special import erf
    return erf(x)


def gelu(x: np.ndarray) -> np.ndarray:
    """x Phi(x) with the standard normal CDF Phi(x) = (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + _erf(x / SQRT2))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d/dx x Phi(x) = Phi(x) + x phi(x), phi the standard normal density."""
    return 0.5 * (1.0 + _erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def forward(params: dict, X: np.ndarray, latent_round=None):
    """Loss and the intermediate values the backward pass needs.  X: (n, d_in) normalised
    input (also the target).  latent_round, if given, maps Z to the value the decoder sees
    (e.g. rounding to BF16); the gradient passes through it unchanged (straight-through)."""
    X = np.asarray(X, dtype=np.float64)
    H1 = X @ params["W1"].T + params["b1"]
    A1 = gelu(H1)
    Z = A1 @ params["W2"].T + params["b2"]
    Zq = latent_round(Z) if latent_round is not None else Z
    H3 = Zq @ params["W3"].T + params["b3"]
    A3 = gelu(H3)
    Y = A3 @ params["W4"].T + params["b4"]
    R = Y - X
    loss = float(np.mean(R * R))
    cache = dict(X=X, H1=H1, A1=A1, Z=Z, Zq=Zq, H3=H3, A3=A3, Y=Y, R=R)
    return loss, cache


def backward(params: dict, cache: dict) -> dict:
    """Gradients of the loss with respect to every weight and bias (chain rule, layer by
    layer from the output)."""
    X, R = cache["X"], cache["R"]
    n_out = R.size
    dY = 2.0 * R / n_out
    g = {}
    g["W4"] = dY.T @ cache["A3"]
    g["b4"] = dY.sum(axis=0)
    dA3 = dY @ params["W4"]
    dH3 = dA3 * gelu_grad(cache["H3"])
    g["W3"] = dH3.T @ cache["Zq"]
    g["b3"] = dH3.sum(axis=0)
    dZ = dH3 @ params["W3"]
    g["W2"] = dZ.T @ cache["A1"]
    g["b2"] = dZ.sum(axis=0)
    dA1 = dZ @ params["W2"]
    dH1 = dA1 * gelu_grad(cache["H1"])
    g["W1"] = dH1.T @ X
    g["b1"] = dH1.sum(axis=0)
    return g


def encode(params: dict, X: np.ndarray) -> np.ndarray:
    return gelu(np.asarray(X, np.float64) @ params["W1"].T + params["b1"]) @ params["W2"].T + params["b2"]


def decode(params: dict, Z: np.ndarray) -> np.ndarray:
    return gelu(np.asarray(Z, np.float64) @ params["W3"].T + params["b3"]) @ params["W4"].T + params["b4"]


def adamw_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr: float, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8, weight_decay: float = 0.0):
    """One AdamW step (t counts from 1).  Returns new (params, m, v)."""
    P, M, V = {}, {}, {}
    for k, p in params.items():
        gk = grads[k]
        M[k] = beta1 * m[k] + (1.0 - beta1) * gk
        V[k] = beta2 * v[k] + (1.0 - beta2) * gk * gk
        mhat = M[k] / (1.0 - beta1 ** t)
        vhat = V[k] / (1.0 - beta2 ** t)
        P[k] = p - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * p)
    return P, M, V


# ----------------------------------------------------------------------------- baseline

def legendre_vandermonde(xi: np.ndarray) -> np.ndarray:
    """V[n][p] = L_p(xi_n), the Legendre polynomials normalised to unit L2 norm on [-1, 1]
    (L_p = sqrt((2p + 1)/2) P_p), by the three-term recurrence."""
    xi = np.asarray(xi, dtype=np.float64)
    n = xi.size
    P = np.zeros((n, n))
    P[:, 0] = 1.0
    if n > 1:
        P[:, 1] = xi
    for p in range(2, n):
        P[:, p] = ((2 * p - 1) * xi * P[:, p - 1] - (p - 1) * P[:, p - 2]) / p
    return P * np.sqrt((2.0 * np.arange(n) + 1.0) / 2.0)


def modal_coefficients(u: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """u: (..., NP^3) nodal values (node i + NP j + NP^2 k) -> modal coefficients
    c (..., NP^3) (mode p + NP q + NP^2 r) of the interpolating tensor-product polynomial,
    u = sum_pqr c_pqr L_p(xi) L_q(eta) L_r(zeta) at every node."""
    NP = xi.size
    Vinv = np.linalg.inv(legendre_vandermonde(xi))
    U = np.asarray(u, np.float64).reshape(u.shape[:-1] + (NP, NP, NP))  # [.., k, j, i]
    C = np.einsum("pi,qj,rk,...kji->...rqp", Vinv, Vinv, Vinv, U)
    return C.reshape(u.shape)


def modal_to_nodal(c: np.ndarray, xi: np.ndarray) -> np.ndarray:
    NP = xi.size
    V = legendre_vandermonde(xi)
    C = np.asarray(c, np.float64).reshape(c.shape[:-1] + (NP, NP, NP))  # [.., r, q, p]
    U = np.einsum("ip,jq,kr,...rqp->...kji", V, V, V, C)
    return U.reshape(c.shape)


def choose_modes(coeffs: np.ndarray, keep: int) -> np.ndarray:
    """The `keep` mode indices with the largest mean squared coefficient over the samples
    (coeffs: (n, NP^3)), ascending: the best fixed truncation for that data."""
    energy = np.mean(np.asarray(coeffs, np.float64) ** 2, axis=0)
    order = np.argsort(-energy, kind="stable")[:keep]
    return np.sort(order)


def truncate(u: np.ndarray, xi: np.ndarray, modes: np.ndarray, coef_round=None) -> np.ndarray:
    """Nodal values of the expansion of u kept to `modes`; coef_round (optional) maps the kept
    coefficients to the values transmitted (e.g. BF16)."""
    c = modal_coefficients(u, xi)
    kept = np.zeros_like(c)
    ck = c[..., modes]
    kept[..., modes] = coef_round(ck) if coef_round is not None else ck
    return modal_to_nodal(kept, xi)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest BF16 (8 significant bits, ties to even) in one
    step: x = m 2^e with 1/2 <= |m| < 1, m rounded to a multiple of 2^-8 (np.rint: half to
    even).  Normal range only (|x| >= 2^-126), which covers the values used here."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


# ----------------------------------------------------------------------------- surfaces

def hausdorff(P: np.ndarray, Q: np.ndarray, chunk: int = 2048) -> float:
    """Symmetric Hausdorff distance between point sets P (n, 3) and Q (m, 3), by brute force:
    max(max_p min_q |p - q|, max_q min_p |p - q|)."""
    P = np.asarray(P, np.float64)
    Q = np.asarray(Q, np.float64)
    if P.size == 0 or Q.size == 0:
        return 0.0 if P.size == Q.size else math.inf

    def directed(A, B):
        worst = 0.0
        for a0 in range(0, len(A), chunk):
            a = A[a0:a0 + chunk]
            best = np.full(len(a), np.inf)
            for b0 in range(0, len(B), chunk):
                b = B[b0:b0 + chunk]
                d2 = ((a[:, None, :] - b[None, :, :]) ** 2).sum(axis=2)
                best = np.minimum(best, d2.min(axis=1))
            worst = max(worst, float(best.max()))
        return math.sqrt(worst)

    return max(directed(P, Q), directed(Q, P))


def hausdorff_kd(P: np.ndarray, Q: np.ndarray) -> float:
    """hausdorff() for large point sets: the nearest-neighbour distances come from a k-d tree
    (scipy.spatial.cKDTree) instead of all pairs; same definition, pinned against the brute
    force in the tests."""
    from scipy.spatial import cKDTree
    P = np.asarray(P, np.float64)
    Q = np.asarray(Q, np.float64)
    if P.size == 0 or Q.size == 0:
        return 0.0 if P.size == Q.size else math.inf
    d_pq = cKDTree(Q).query(P)[0].max()
    d_qp = cKDTree(P).query(Q)[0].max()
    return float(max(d_pq, d_qp))
