"""Pins of the optimiser references (oracle/optim.py): closed forms
of the SE(3) exponential and of Adam's first step."""

import numpy as np

from oracle import optim as op


def test_exp_of_translation_and_rotation():
    E = op.se3_exp([0.1, -0.2, 0.3, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(E, np.hstack([np.eye(3), [[0.1], [-0.2], [0.3]]]), atol=1e-15)
    th = 0.3
    E = op.se3_exp([0.0, 0.0, 0.0, 0.0, 0.0, th])
    c, s = np.cos(th), np.sin(th)
    np.testing.assert_allclose(E[:, :3], [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)
    np.testing.assert_allclose(E[:, 3], 0.0, atol=1e-15)


def test_exp_inverse_and_screw_translation():
    """Exp(xi) Exp(-xi) = I; a screw about z moves a point on the axis by
    rho_z only."""
    xi = np.array([0.05, -0.02, 0.07, 0.1, -0.3, 0.2])
    A, B = op.se3_exp(xi), op.se3_exp(-xi)
    np.testing.assert_allclose(A[:, :3] @ B[:, :3], np.eye(3), atol=1e-14)
    np.testing.assert_allclose(A[:, :3] @ B[:, 3] + A[:, 3], 0.0, atol=1e-14)
    E = op.se3_exp([0.0, 0.0, 0.4, 0.0, 0.0, 1.1])
    np.testing.assert_allclose(E[:, 3], [0.0, 0.0, 0.4], atol=1e-15)


def test_adam_first_step_is_sign_step():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is
    lr * g / (|g| + eps) = lr * sign(g) up to eps."""
    P = np.hstack([np.eye(3), [[1.0], [2.0], [3.0]]])
    g = np.array([0.3, -2.0, 1e-3, -0.5, 0.25, 4.0])
    lr = np.array([2e-3] * 3 + [4e-4] * 3)
    Pn, m, v, t = op.adam_pose_step(P, g, np.zeros(6), np.zeros(6), 0.0, lr, eps=0.0)
    assert t == 1.0
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)   # 1 - 0.999 rounds
    E = op.se3_exp(-lr * np.sign(g))
    np.testing.assert_allclose(Pn[:, :3], E[:, :3], atol=1e-15)
    np.testing.assert_allclose(Pn[:, 3], E[:, 3] + P[:, 3], atol=1e-15)


def test_attr_adam_first_step_and_chain_rule():
    """First step: theta moves by lr * sign(g) (eps = 0) with g the chain-rule
    gradient; a zero gradient leaves theta unchanged; the activated outputs
    are sigmoid / exp of the new theta."""
    rng = np.random.default_rng(0)
    n = 7
    theta = np.stack([rng.random(n), rng.random(n), rng.random(n),
                      rng.normal(0, 1, n), np.log(0.01 + rng.random(n))])
    dc = rng.normal(0, 1, (n, 3))
    do = rng.normal(0, 1, n)
    dr = rng.normal(0, 1, n)
    dr[2] = 0.0
    lr = [0.0025] * 3 + [0.05, 0.005]
    th, m, v, t, col, op_, rad = op.attr_adam_step(theta, np.zeros((5, n)), np.zeros((5, n)),
                                                   0.0, dc, do, dr, lr, eps=1e-300)
    o = 1 / (1 + np.exp(-theta[3]))
    g = np.stack([dc[:, 0], dc[:, 1], dc[:, 2], do * o * (1 - o), dr * np.exp(theta[4])])
    np.testing.assert_allclose(th, theta - np.array(lr)[:, None] * np.sign(g), rtol=0,
                               atol=1e-15)
    assert th[4, 2] == theta[4, 2]     # zero gradient: 0 / (0 + eps)
    np.testing.assert_allclose(op_, 1 / (1 + np.exp(-th[3])), rtol=1e-15)
    np.testing.assert_allclose(rad, np.exp(th[4]), rtol=1e-15)
    np.testing.assert_array_equal(col, th[:3].T)


def test_shape_gradient_matches_finite_differences():
    """shape_grads is the gradient of L(theta_s) = <a, exp(log s)> + <b, q>
    in theta_s (central differences of that L, whose gradient with respect
    to the activated values is (a, b))."""
    rng = np.random.default_rng(3)
    n = 5
    th = np.concatenate([np.log(rng.uniform(0.01, 0.1, (3, n))), rng.normal(size=(4, n))])
    a, b = rng.normal(size=(n, 3)), rng.normal(size=(n, 4))
    L = lambda t: (a * np.exp(t[:3]).T).sum() + (b * t[3:].T).sum()
    g = op.shape_grads(th, a, b)
    for i in range(7):
        for j in range(n):
            e = np.zeros_like(th)
            e[i, j] = 1e-6
            fd = (L(th + e) - L(th - e)) / 2e-6
            assert abs(fd - g[i, j]) <= 1e-8 * (1 + abs(fd))


def test_shape_adam_first_step_is_sign_step():
    """At t = 1 every parameter moves by its rate against the sign of its
    gradient (log scales by lr_scale, quaternion components by lr_rot); the
    outputs are exp of the log scales and the quaternion as stored."""
    rng = np.random.default_rng(4)
    n = 6
    th = np.concatenate([np.log(rng.uniform(0.01, 0.1, (3, n))), rng.normal(size=(4, n))])
    ds, dq = rng.normal(size=(n, 3)), rng.normal(size=(n, 4))
    out, m, v, t, s, q = op.shape_adam_step(th, np.zeros((7, n)), np.zeros((7, n)), 0.0, ds, dq,
                                            5e-3, 1e-3, eps=0.0)
    assert t == 1.0
    step = np.concatenate([np.full((3, n), 5e-3), np.full((4, n), 1e-3)])
    g = np.concatenate([ds.T, dq.T])          # signs of dL/dlog s = dL/ds s (s > 0)
    np.testing.assert_allclose(out, th - step * np.sign(g), rtol=0, atol=1e-15)
    np.testing.assert_allclose(s, np.exp(out[:3]).T, rtol=1e-15)
    np.testing.assert_array_equal(q, out[3:].T)
