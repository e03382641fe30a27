"""Learned PM force correction, FP64 reference (test infrastructure only).

The paper names a learned, space- and time-dependent optimisation of the PM
gravity solver as ongoing work built on pmwd (Statement of Need) without
describing it, so the network here is a design choice [reading]: a per-cell
multilayer perceptron on the coarse CIC density mesh that predicts a force
correction on the same mesh, added to the PM force meshes before the CIC
read.

  features   asinh(rho(c + o) - 1) for the 27 offsets o in {-1, 0, 1}^3
             (periodic; rho = alpha sum W, so rho - 1 is the density
             contrast), then the scale factor a, then 4 zeros (32 inputs);
             offsets in lexicographic order (ox slowest, oz fastest)
  network    h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3,
             32 -> 128 -> 128 -> 3
  output     dF_j(c) = s_out y_j(c), s_out = 3/2 Om h (h = cell size)
  loss       force matching: L = mean_i |read(dF)(x_i) - T_i|^2 over
             particles, T_i = F_fine(x_i) - F_coarse(x_i)

Precision points mirrored from the BF16 tensor-core kernels: features,
weights and the hidden activations h1, h2 are rounded to bfloat16 (round to
nearest even) before each product; products accumulate in FP64 here.  In the
backward pass the activation cotangents and the per-cell output cotangent
are rounded to bfloat16 before the weight-gradient products.

Parity status: the arithmetic (forward, loss gradient, the correction's
VJPs, the corrected adjoint) is pinned by central finite differences of the
unrounded FP64 maps, and the bf16 rounding by its ties-to-even definition
(tests/test_oracle_learned.py).  Parity unpinned: the architecture above
(features, sizes, output scale), a design choice the paper does not fix.
"""

import itertools

import numpy as np

from . import pm

N_IN, N_HID, N_OUT = 32, 128, 3
OFFSETS = np.array(list(itertools.product((-1, 0, 1), repeat=3)))


def bf16(x):
    """Round float values to bfloat16 (round to nearest, ties to even),
    returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def param_shapes():
    return [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
            ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(theta):
    out, k = {}, 0
    for name, shape in param_shapes():
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + size], dtype=np.float64).reshape(shape)
        k += size
    return out


def features(rho, a):
    """(n^3, 32) features of the painted mesh rho (rho = alpha sum W)."""
    n = rho.shape[0]
    f = np.zeros((n ** 3, N_IN))
    d = np.arcsinh(rho - 1.0)
    for q, (ox, oy, oz) in enumerate(OFFSETS):
        f[:, q] = np.roll(d, shift=(-ox, -oy, -oz), axis=(0, 1, 2)).ravel()
    f[:, 27] = a
    return f


def forward(x, theta, rounding=True):
    """Per-cell outputs y (cells, 3) and the intermediates."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    p = unflatten(theta)
    x = r(x)
    z1 = x @ r(p["W1"]) + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(p["W2"]) + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ r(p["W3"]) + p["b3"]
    return y, (x, h1, h2)


def correction_mesh(s, a, theta, setup, rounding=True):
    """dF on the coarse mesh, (n^3, 3), for particles at displacement s."""
    rho = setup.alpha * pm.cic_paint(pm.positions(s, setup), setup.n_m, setup.cell, order=setup.order)
    y, _ = forward(features(rho, a), theta, rounding)
    return output_scale(setup) * y


def output_scale(setup):
    return 1.5 * setup.cosmo.omega_m * setup.cell


def predict(s, a, theta, setup, rounding=True):
    """Per-particle correction read from the dF mesh, (N, 3)."""
    dfm = correction_mesh(s, a, theta, setup, rounding)
    x = pm.positions(s, setup)
    n = setup.n_m
    return np.stack([pm.cic_read(x, dfm[:, j].reshape(n, n, n), setup.cell, setup.order) for j in range(3)], axis=1)


def loss(s, target, a, theta, setup, rounding=True):
    d = predict(s, a, theta, setup, rounding) - target
    return float(np.mean(np.sum(d * d, axis=1)))


def loss_and_grad(s, target, a, theta, setup, rounding=True):
    """Force-matching loss and its gradient with respect to theta (flat),
    with the kernels' bfloat16 rounding points when ``rounding``."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    p = unflatten(theta)
    n = setup.n_m
    xpos = pm.positions(s, setup)
    rho = setup.alpha * pm.cic_paint(xpos, n, setup.cell, order=setup.order)
    feat = features(rho, a)
    y, (x, h1, h2) = forward(feat, theta, rounding)
    so = output_scale(setup)
    pred = np.stack([pm.cic_read(xpos, (so * y[:, j]).reshape(n, n, n), setup.cell, setup.order) for j in range(3)], axis=1)
    d = pred - target
    npart = len(s)
    L = float(np.sum(d * d) / npart)
    # adjoint of the read: paint the residual cotangent 2 d / N
    gy = np.stack([pm.cic_paint(xpos, n, setup.cell, 2.0 * d[:, j] / npart, setup.order).ravel() for j in range(3)], axis=1)
    gy = r(so * gy)
    g = {}
    g["W3"] = h2.T @ gy
    g["b3"] = gy.sum(0)
    g2 = (gy @ r(p["W3"]).T) * (h2 > 0)
    g["b2"] = g2.sum(0)
    g2 = r(g2)
    g["W2"] = h1.T @ g2
    g1 = (g2 @ r(p["W2"]).T) * (h1 > 0)
    g["b1"] = g1.sum(0)
    g1 = r(g1)
    g["W1"] = x.T @ g1
    flat = np.concatenate([g[name].ravel() for name, _ in param_shapes()])
    return L, flat


def init_params(seed):
    """He-normal weights, zero biases, zero last layer (the untrained
    network leaves the PM force unchanged)."""
    rng = np.random.default_rng(seed)
    theta = []
    for name, shape in param_shapes():
        if name == "W3" or name.startswith("b"):
            theta.append(np.zeros(shape))
        else:
            theta.append(rng.standard_normal(shape) * np.sqrt(2.0 / shape[0]))
    return np.concatenate([t.ravel() for t in theta])


# ------------------------------------------- through the trajectory -------
#
# Training the correction on the trajectory (rather than on forces) needs
# its vector-Jacobian products inside the reverse-time adjoint.  With
# dF(c) = s_out y(x(c)), x(c)_q = asinh(rho(c + o_q) - 1), rho = alpha sum W
# and the corrected particle force F_i = sum_c W(x_i - c) dF(c), the
# cotangent v of F gives
#   u(c)        = sum_i W(x_i - c) v_i                     (paint of v)
#   g_s (read)  = sum_c dW(x_i - c)/dx_i (v_i . dF(c))
#   g_y(c)      = s_out u(c);  g_x = MLP backward of g_y;  g_theta likewise
#   g_rho(c')   = sum_q g_x(c' - o_q, q) / sqrt(1 + (rho(c') - 1)^2)
#   g_s (paint) = alpha sum_c dW(x_i - c)/dx_i g_rho(c)
# The bf16 rounding points are those of loss_and_grad (activation and output
# cotangents rounded before the products), with the feature cotangent g_x
# taken from the rounded g1 and W1.


def _mlp_backward(x, h1, h2, gy, theta, r):
    """MLP backward from the output cotangent gy (cells, 3): returns the
    feature cotangent (cells, 32) and the flat parameter gradient."""
    p = unflatten(theta)
    g = {}
    gy = r(gy)
    g["W3"] = h2.T @ gy
    g["b3"] = gy.sum(0)
    g2 = (gy @ r(p["W3"]).T) * (h2 > 0)
    g["b2"] = g2.sum(0)
    g2 = r(g2)
    g["W2"] = h1.T @ g2
    g1 = (g2 @ r(p["W2"]).T) * (h1 > 0)
    g["b1"] = g1.sum(0)
    g1 = r(g1)
    g["W1"] = x.T @ g1
    gx = g1 @ r(p["W1"]).T
    return gx, np.concatenate([g[name].ravel() for name, _ in param_shapes()])


def correction_vjp(s, v, a, theta, setup, rounding=True):
    """(g_s, g_theta): cotangents of the particles' displacements and of the
    network parameters for the cotangent v (N, 3) of predict(s, a, ...)."""
    r = bf16 if rounding else (lambda t: np.asarray(t, dtype=np.float64))
    n, h, order = setup.n_m, setup.cell, setup.order
    xpos = pm.positions(s, setup)
    rho = setup.alpha * pm.cic_paint(xpos, n, h, order=order)
    y, (x, h1, h2) = forward(features(rho, a), theta, rounding)
    so = output_scale(setup)
    dfm = [(so * y[:, j]).reshape(n, n, n) for j in range(3)]
    g_read = np.zeros((len(s), 3))
    for j in range(3):
        g_read += pm.cic_read_grad(xpos, dfm[j], h, order) * v[:, j:j + 1]
    u = np.stack([pm.cic_paint(xpos, n, h, v[:, j], order).ravel() for j in range(3)], axis=1)
    gx, g_theta = _mlp_backward(x, h1, h2, so * u, theta, r)
    g_d = np.zeros((n, n, n))
    for q, (ox, oy, oz) in enumerate(OFFSETS):
        # x(c)_q reads d(c + o_q): its cotangent lands on cell c + o_q
        g_d += np.roll(gx[:, q].reshape(n, n, n), shift=(ox, oy, oz), axis=(0, 1, 2))
    g_rho = g_d / np.sqrt(1.0 + (rho - 1.0) ** 2)
    g_paint = setup.alpha * pm.cic_read_grad(xpos, g_rho, h, order)
    return g_read + g_paint, g_theta


def integrate_corrected(s, p, theta, setup, rounding=True):
    """Forward KDK with the force PM + correction, the correction at each
    evaluation's scale factor (step boundaries a_n)."""
    c = pm.coefficients(setup)
    a = c["a"]
    s, p = s.copy(), p.copy()
    f = pm.force(s, setup) + predict(s, a[0], theta, setup, rounding)
    for n in range(setup.n_steps):
        p = p + c["K_a"][n] * f
        s = s + c["Dr"][n] * p
        f = pm.force(s, setup) + predict(s, a[n + 1], theta, setup, rounding)
        p = p + c["K_b"][n] * f
    return s, p, f


def adjoint_corrected(s, p, f, lam, mu, theta, setup, rounding=True):
    """Discrete adjoint of integrate_corrected, backward in time along the
    reconstructed trajectory: returns the initial (s, p), the cotangents of
    the initial s and p, and the gradient with respect to the network
    parameters (Om is held fixed here)."""
    c = pm.coefficients(setup)
    a = c["a"]
    g_theta = np.zeros(n_params())
    s, p, lam, mu = s.copy(), p.copy(), lam.copy(), mu.copy()

    def vjp(y, v, ak, coef):
        gs_nn, gt = correction_vjp(y, v, ak, theta, setup, rounding)
        return coef * (pm.force_vjp(y, v, setup) + gs_nn), coef * gt

    for n in reversed(range(setup.n_steps)):
        gl, gt = vjp(s, mu, a[n + 1], c["K_b"][n])
        lam, g_theta = lam + gl, g_theta + gt
        p_half = p - c["K_b"][n] * f
        mu = mu + c["Dr"][n] * lam
        s = s - c["Dr"][n] * p_half
        f = pm.force(s, setup) + predict(s, a[n], theta, setup, rounding)
        gl, gt = vjp(s, mu, a[n], c["K_a"][n])
        lam, g_theta = lam + gl, g_theta + gt
        p = p_half - c["K_a"][n] * f
    return s, p, lam, mu, g_theta
