"""Plain float64 NumPy reference of the tracking optimiser step (test
infrastructure; see the package docstring for who may import it).

Adam on the camera-pose twist (Sec. 3.3 optimises the pose of the latest
frame; the supplementary gives the Adam learning rates lr_rot, lr_trans),
with the pose retracted by right-multiplication with the SE(3) exponential:

    t += 1,  m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
    s = lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
    P <- P Exp(-s),  xi = (rho, phi).

The exponential is evaluated here as the matrix exponential of the 4 x 4
twist matrix [[phi]x, rho; 0, 0] (SciPy's expm), independently of the
closed form the kernel uses.
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import expm


def se3_exp(xi) -> np.ndarray:
    """(3, 4) [R | t] = Exp of the twist xi = (rho, phi)."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    A = np.zeros((4, 4))
    A[:3, :3] = [[0.0, -phi[2], phi[1]], [phi[2], 0.0, -phi[0]], [-phi[1], phi[0], 0.0]]
    A[:3, 3] = rho
    return expm(A)[:3, :]


def adam_pose_step(pose, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One step; returns (new pose (3, 4), m, v, t)."""
    g = np.asarray(grad, np.float64)
    t = t + 1.0
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    s = np.asarray(lr, np.float64) * (m / (1 - beta1 ** t)) / (np.sqrt(v / (1 - beta2 ** t)) + eps)
    E = se3_exp(-s)
    P = np.asarray(pose, np.float64).reshape(3, 4)
    R = P[:, :3] @ E[:, :3]
    tr = P[:, :3] @ E[:, 3] + P[:, 3]
    return np.hstack([R, tr[:, None]]), m, v, t


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def attr_adam_step(theta, m, v, t, d_colour, d_opacity, d_radius, lr, beta1=0.9, beta2=0.999,
                   eps=1e-8):
    """One Adam step of the mapping optimiser on theta (5, n) =
    (c0, c1, c2, logit o, log r): the gradients with respect to the activated
    values (d_colour (n, 3), d_opacity (n,), d_radius (n,)) are taken to theta
    by the chain rule at the current theta,
        m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
        theta -= lr m / (1 - b1^t) / (sqrt(v) / sqrt(1 - b2^t) + eps).
    Returns (theta, m, v, t, colour (n, 3), opacity (n,), radius (n,))."""
    theta = np.asarray(theta, np.float64)
    o = sigmoid(theta[3])
    r = np.exp(theta[4])
    g = np.stack([d_colour[:, 0], d_colour[:, 1], d_colour[:, 2],
                  np.asarray(d_opacity, np.float64) * o * (1 - o),
                  np.asarray(d_radius, np.float64) * r]).astype(np.float64)
    t = t + 1.0
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    lr = np.asarray(lr, np.float64)[:, None]
    theta = theta - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v) / np.sqrt(1 - beta2 ** t) + eps)
    return theta, m, v, t, theta[:3].T.copy(), sigmoid(theta[3]), np.exp(theta[4])


def shape_grads(theta_s, d_scale, d_rot):
    """Gradient with respect to theta_s (7, n) = (log s0, log s1, log s2,
    q0, q1, q2, q3) of the ellipsoid shape from the gradients with respect
    to the activated scale s = exp(log s) (n, 3) and the stored quaternion
    (n, 4): the chain rule dL/dlog s = dL/ds s, the quaternion as stored."""
    theta_s = np.asarray(theta_s, np.float64)
    s = np.exp(theta_s[:3])
    return np.concatenate([np.asarray(d_scale, np.float64).T * s,
                           np.asarray(d_rot, np.float64).T]).astype(np.float64)


def shape_adam_step(theta_s, m, v, t, d_scale, d_rot, lr_scale, lr_rot, beta1=0.9,
                    beta2=0.999, eps=1e-8):
    """One Adam step of the ellipsoid shape (the anisotropic variant of the
    attribute ablation, Sec. 4) in the parametrisation of shape_grads, with
    one rate for the three log scales and one for the four quaternion
    components (the 3D Gaussian splatting convention; the quaternion is
    normalised where it is used, not here).  Returns (theta_s, m, v, t,
    scale (n, 3), rot (n, 4))."""
    g = shape_grads(theta_s, d_scale, d_rot)
    t = t + 1.0
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    lr = np.array([lr_scale] * 3 + [lr_rot] * 4, np.float64)[:, None]
    theta_s = np.asarray(theta_s, np.float64) - lr * (m / (1 - beta1 ** t)) / (
        np.sqrt(v) / np.sqrt(1 - beta2 ** t) + eps)
    return theta_s, m, v, t, np.exp(theta_s[:3]).T.copy(), theta_s[3:].T.copy()
