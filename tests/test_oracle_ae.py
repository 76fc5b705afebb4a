"""Pins of the FP64 autoencoder oracle (oracle/ae.py) against what mathematics fixes:
central finite differences for every gradient, closed forms of gelu and of the first AdamW
steps, exactness of the Legendre modal transform on polynomials, brute force Hausdorff."""
import math

import numpy as np
import pytest

import oracle
from oracle import ae


def _tiny(seed=0, dims=(12, 7, 3, 7, 12), n=5):
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(4):
        p[f"W{l + 1}"] = rng.normal(0, 0.6, size=(dims[l + 1], dims[l]))
        p[f"b{l + 1}"] = rng.normal(0, 0.2, size=dims[l + 1])
    X = rng.normal(0, 1, size=(n, dims[0]))
    return p, X


def test_gradients_match_central_differences():
    """Every parameter entry of a small network: rel. error of the analytic gradient against
    the 5-point central difference (8 (L(+h) - L(-h)) - (L(+2h) - L(-2h))) / 12h, whose
    truncation error is O(h^4), below 1e-6 (h = 1e-4 relative; entries above 1e-7 of the
    tensor's largest)."""
    p, X = _tiny()
    _, cache = ae.forward(p, X)
    g = ae.backward(p, cache)

    def loss_at(k, idx, val):
        q = {kk: vv.copy() for kk, vv in p.items()}
        q[k][idx] = val
        return ae.forward(q, X)[0]

    worst = 0.0
    for k, v in p.items():
        scale = np.abs(g[k]).max()
        for idx in np.ndindex(v.shape):
            h = 1e-4 * max(1.0, abs(v[idx]))
            x0 = v[idx]
            fd = (8.0 * (loss_at(k, idx, x0 + h) - loss_at(k, idx, x0 - h))
                  - (loss_at(k, idx, x0 + 2 * h) - loss_at(k, idx, x0 - 2 * h))) / (12.0 * h)
            if abs(g[k][idx]) > 1e-7 * scale:
                worst = max(worst, abs(fd - g[k][idx]) / abs(g[k][idx]))
    assert worst < 1e-6, worst


def test_straight_through_latent_rounding_gradient():
    """With a latent rounding the decoder sees the rounded Z and the encoder gradient is
    that of the identity through it: equal to the unrounded gradient at a Z already on the
    grid."""
    p, X = _tiny(1)
    _, c0 = ae.forward(p, X)
    grid = lambda z: np.round(z * 8.0) / 8.0  # noqa: E731
    p2 = {k: v.copy() for k, v in p.items()}
    p2["b2"] = p["b2"] + (grid(c0["Z"]) - c0["Z"])[0]  # shift one sample's Z onto the grid
    _, c1 = ae.forward(p2, X[:1], latent_round=grid)
    _, c2 = ae.forward(p2, X[:1])
    assert np.allclose(c1["Zq"], c2["Z"], atol=1e-12)
    g1, g2 = ae.backward(p2, c1), ae.backward(p2, c2)
    for k in g1:
        assert np.allclose(g1[k], g2[k], rtol=1e-10, atol=1e-14)


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 241)
    # Phi(x) + Phi(-x) = 1  =>  gelu(x) - gelu(-x) = x exactly
    assert np.abs(ae.gelu(x) - ae.gelu(-x) - x).max() < 1e-14
    assert ae.gelu(np.array([0.0]))[0] == 0.0
    assert abs(ae.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16
    # Phi(1) = 0.841344746068543 (tables of the normal distribution)
    assert abs(ae.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-14
    assert abs(ae.gelu(np.array([12.0]))[0] - 12.0) < 1e-15
    h = 1e-6
    fd = (ae.gelu(x + h) - ae.gelu(x - h)) / (2 * h)
    assert np.abs(fd - ae.gelu_grad(x)).max() < 1e-8


def test_loss_of_zero_network_and_identity_gradient_sign():
    p, X = _tiny(2)
    z = {k: np.zeros_like(v) for k, v in p.items()}
    loss, cache = ae.forward(z, X)
    assert abs(loss - np.mean(X * X)) < 1e-15
    g = ae.backward(z, cache)
    # with every weight zero only the output bias moves the loss: d/db4 = -2 mean_rows(X) / d
    assert np.allclose(g["b4"], -2.0 * X.sum(axis=0) / X.size)
    for k in ("W1", "W2", "W3", "W4", "b1", "b2", "b3"):
        assert np.abs(g[k]).max() == 0.0


def test_adamw_first_steps_closed_form():
    theta = {"a": np.array([1.0, -2.0, 0.5])}
    g1 = {"a": np.array([0.3, -0.1, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 0.1
    P, M, V = ae.adamw_step(theta, g1, m, v, 1, lr, b1, b2, eps, wd)
    # step 1: mhat = g, vhat = g^2  ->  theta - lr (g / (|g| + eps) + wd theta)
    exp1 = theta["a"] - lr * (g1["a"] / (np.abs(g1["a"]) + eps) + wd * theta["a"])
    assert np.allclose(P["a"], exp1, rtol=0, atol=1e-15)
    # step 2 with g2: m = 0.9*0.1 g1 + 0.1 g2, v = 0.999*0.001 g1^2 + 0.001 g2^2
    g2 = {"a": np.array([0.1, 0.2, -0.4])}
    P2, M2, V2 = ae.adamw_step(P, g2, M, V, 2, lr, b1, b2, eps, wd)
    m2 = 0.9 * 0.1 * g1["a"] + 0.1 * g2["a"]
    v2 = 0.999 * 0.001 * g1["a"] ** 2 + 0.001 * g2["a"] ** 2
    exp2 = P["a"] - lr * ((m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + eps) + wd * P["a"])
    assert np.allclose(M2["a"], m2) and np.allclose(V2["a"], v2)
    assert np.allclose(P2["a"], exp2, rtol=0, atol=1e-14)


def _xi(N=7):
    return oracle.gll(N)[0]


def test_legendre_transform_is_exact_on_polynomials():
    """The modal transform interpolates: a tensor polynomial of degree <= N per direction is
    reproduced exactly at the nodes, and each single Legendre product has one coefficient."""
    xi = _xi()
    NP = xi.size
    X = xi[None, None, :] + 0 * xi[:, None, None]
    Y = xi[None, :, None] + 0 * xi[:, None, None]
    Z = xi[:, None, None] + 0 * xi[None, :, None]
    u = (X ** 3 * Y - 2 * Y ** 2 * Z ** 5 + X ** 7 * Z ** 7 + 0.25).reshape(1, -1)
    c = ae.modal_coefficients(u, xi)
    assert np.abs(ae.modal_to_nodal(c, xi) - u).max() < 1e-12
    V = ae.legendre_vandermonde(xi)
    for (p, q, r) in [(0, 0, 0), (3, 1, 2), (7, 7, 7), (2, 0, 5)]:
        f = (V[:, p][None, None, :] * V[:, q][None, :, None] * V[:, r][:, None, None]).reshape(1, -1)
        cf = ae.modal_coefficients(f, xi)[0]
        e = p + NP * q + NP * NP * r
        assert abs(cf[e] - 1.0) < 1e-11
        cf[e] = 0.0
        assert np.abs(cf).max() < 1e-11
    # L_p normalisation: integral of L_p^2 over [-1, 1] = 1 (GLL quadrature exact to degree 2N-1)
    w = oracle.gll(7)[1]
    for pdeg in range(4):
        assert abs(np.sum(w * V[:, pdeg] ** 2) - 1.0) < 1e-13


def test_truncation_keeps_the_kept_modes():
    xi = _xi()
    rng = np.random.default_rng(3)
    c = np.zeros((4, 512))
    modes = np.array([0, 1, 8, 64, 9, 72, 65, 2, 16, 128, 3, 24, 192, 10, 17, 80])
    c[:, modes] = rng.normal(size=(4, modes.size))
    u = ae.modal_to_nodal(c, xi)
    assert np.abs(ae.truncate(u, xi, np.sort(modes)) - u).max() < 1e-12
    # dropping every mode leaves zero; keeping all is the identity
    noise = rng.normal(size=(2, 512))
    assert np.abs(ae.truncate(noise, xi, np.arange(512)) - noise).max() < 1e-11
    assert np.abs(ae.truncate(noise, xi, np.array([], dtype=int))).max() == 0.0
    # the data-chosen modes are those with the most energy
    assert list(ae.choose_modes(c, 16)) == sorted(modes.tolist())


def test_round_bf16():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 1e-3, 65504.0])
    r = ae.round_bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # exactly halfway between 1 and 1 + 2^-7: ties to even
    assert r[2] == 1.0 + 2 ** -7  # 3/4 of the way to 1 + 2^-7 -> rounds up
    for x, y in zip(vals, r):
        m, e = math.frexp(y)
        assert m * 256 == int(m * 256)  # 8 significant bits
        assert abs(x - y) <= abs(x) * 2 ** -8 * (1 + 1e-15)  # unit roundoff of 8 significant bits


def test_hausdorff_brute_force():
    P = np.array([[0.0, 0.0, 0.0]])
    Q = np.array([[1.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    assert ae.hausdorff(P, Q) == 2.0
    assert ae.hausdorff(Q, P) == 2.0
    rng = np.random.default_rng(4)
    A = rng.normal(size=(300, 3))
    assert ae.hausdorff(A, A) == 0.0
    t = np.array([0.3, -0.4, 0.0])
    assert ae.hausdorff(A, A + t) <= 0.5 + 1e-12  # every point's translate is 0.5 away
    assert abs(ae.hausdorff(A[:1], A[:1] + t) - 0.5) < 1e-15
    # against a direct double loop on a small case
    B = rng.normal(size=(40, 3))
    d = np.sqrt(((A[:50, None] - B[None]) ** 2).sum(-1))
    ref = max(d.min(axis=1).max(), d.min(axis=0).max())
    assert abs(ae.hausdorff(A[:50], B, chunk=7) - ref) < 1e-12


def test_hausdorff_kd_equals_brute_force():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(700, 3))
    B = rng.normal(size=(500, 3)) * 1.3 + 0.2
    assert abs(ae.hausdorff_kd(A, B) - ae.hausdorff(A, B)) < 1e-12
    assert ae.hausdorff_kd(A, A) == 0.0


def test_encode_decode_equal_the_forward_pass():
    """encode() and decode() restate the forward pass for the latent and the reconstruction;
    they must give forward()'s Z and Y exactly (forward() is the path the finite-difference
    test pins), on a network whose layers are all of different widths so a transposed or
    swapped weight cannot broadcast."""
    rng = np.random.default_rng(11)
    dims = (9, 6, 4, 5, 9)
    p = {}
    for l in range(4):
        p[f"W{l + 1}"] = rng.normal(0, 0.7, size=(dims[l + 1], dims[l]))
        p[f"b{l + 1}"] = rng.normal(0, 0.3, size=dims[l + 1])
    X = rng.normal(0, 1, size=(7, dims[0]))
    _, cache = ae.forward(p, X)
    np.testing.assert_array_equal(ae.encode(p, X), cache["Z"])
    np.testing.assert_array_equal(ae.decode(p, cache["Z"]), cache["Y"])
    # with a rounded latent, decode of the rounded Z is the decoder forward() ran
    rnd = ae.round_bf16
    _, cq = ae.forward(p, X, latent_round=rnd)
    np.testing.assert_array_equal(ae.decode(p, rnd(ae.encode(p, X))), cq["Y"])


def test_encode_decode_scalar_network_closed_form():
    """A 1-1-1-1-1 network evaluated by hand with the tabulated Phi(1) = 0.8413447460685429
    (Abramowitz & Stegun 26.2): x = 1, H1 = 2x - 1 = 1, A1 = Phi(1), Z = 3 Phi(1) + 0.5;
    the decoder's b3 is chosen so that H3 = Z - (Z* - 1) = 1 at the tabulated Z*, then
    Y = -2 Phi(1) + 0.25.  A dropped bias, a GELU on the latent or on the output, or a wrong
    sign changes the values."""
    phi1 = 0.8413447460685429
    z_star = 3.0 * phi1 + 0.5
    p = {"W1": np.array([[2.0]]), "b1": np.array([-1.0]), "W2": np.array([[3.0]]), "b2": np.array([0.5]),
         "W3": np.array([[1.0]]), "b3": np.array([1.0 - z_star]), "W4": np.array([[-2.0]]), "b4": np.array([0.25])}
    z = ae.encode(p, np.array([[1.0]]))
    assert abs(z[0, 0] - z_star) < 1e-15
    y = ae.decode(p, z)
    assert abs(y[0, 0] - (-2.0 * phi1 + 0.25)) < 1e-14
