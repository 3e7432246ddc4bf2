"""Camera tracking driver (Sec. 3.3): optimise the pose of the latest frame
against fixed Gaussians by minimising Eq. 1,

    alpha * W |V - V'|_1 + beta * W |D - D'|_1,

with W masking pixels without depth or not covered by the render (here:
silhouette > 0.99).  The render and its pose gradient run in the vtsplat
kernels; the loss gradient and the Adam step on the pose twist are a handful
of torch element-wise ops on the device (no host synchronisation).

The L1 norms are averaged over the pixels (a reading: the paper writes
||.||_1 without a normaliser).  Pose updates are right-multiplicative,
P <- P Exp(-step), matching the twist gradient of vt_render_backward.
"""

from __future__ import annotations

import numpy as np
import torch

from . import api


def _skew(w):
    z = torch.zeros((), dtype=w.dtype, device=w.device)
    return torch.stack([torch.stack([z, -w[2], w[1]]), torch.stack([w[2], z, -w[0]]),
                        torch.stack([-w[1], w[0], z])])


def se3_exp(xi: torch.Tensor):
    """Exp of a twist (rho, phi) -> (R (3,3), t (3,)), float64 on the device."""
    rho, phi = xi[:3], xi[3:]
    th2 = (phi * phi).sum()
    th = torch.sqrt(th2 + 1e-300)
    K = _skew(phi)
    K2 = K @ K
    small = th2 < 1e-16
    a = torch.where(small, 1.0 - th2 / 6.0, torch.sin(th) / th)
    b = torch.where(small, 0.5 - th2 / 24.0, (1.0 - torch.cos(th)) / (th2 + 1e-300))
    c = torch.where(small, 1.0 / 6.0 - th2 / 120.0, (th - torch.sin(th)) / (th2 * th + 1e-300))
    eye = torch.eye(3, dtype=xi.dtype, device=xi.device)
    R = eye + a * K + b * K2
    J = eye + b * K + c * K2
    return R, J @ rho


class PoseTracker:
    """Adam on the pose twist (learning rates per rotation / translation,
    supplementary: lr_rot, lr_trans)."""

    def __init__(self, renderer: api.Renderer, sections, K, W: int, H: int, pose0,
                 lr_rot: float = 4e-4, lr_trans: float = 2e-3, alpha: float = 0.5,
                 beta: float = 0.025, device="cuda"):
        self.R = renderer
        self.sections = sections
        self.K, self.W, self.H = tuple(K), int(W), int(H)
        self.pose = api.pose12(pose0, device)
        self.alpha, self.beta = float(alpha), float(beta)
        self.lr = torch.tensor([lr_trans] * 3 + [lr_rot] * 3, dtype=torch.float64, device=device)
        self.m = torch.zeros(6, dtype=torch.float64, device=device)
        self.v = torch.zeros(6, dtype=torch.float64, device=device)
        self.t = torch.zeros((), dtype=torch.float64, device=device)
        self.d_twist = torch.zeros(6, dtype=torch.float64, device=device)
        self.d_mat = torch.zeros(12, dtype=torch.float64, device=device)
        self.rgb = torch.empty(3, H, W, device=device)
        self.depth = torch.empty(H, W, device=device)
        self.sil = torch.empty(H, W, device=device)
        self.loss = torch.zeros((), device=device)
        self.obs_rgb = torch.zeros(3, H, W, device=device)
        self.obs_depth = torch.zeros(H, W, device=device)
        self.graph = None

    def set_target(self, rgb: torch.Tensor, depth: torch.Tensor):
        """Copy the observed frame into the tracker's fixed buffers."""
        self.obs_rgb.copy_(rgb, non_blocking=True)
        self.obs_depth.copy_(depth, non_blocking=True)

    def reset_optimiser(self):
        self.m.zero_()
        self.v.zero_()
        self.t.zero_()

    def step(self):
        """One tracking iteration: render, Eq. 1 loss and its image gradient,
        pose backward, Adam step and retraction.  All on the device."""
        self.R.render(self.sections, self.pose, self.K, self.W, self.H, self.rgb, self.depth,
                      self.sil)
        P = float(self.W * self.H)
        mask = ((self.obs_depth > 0) & (self.sil > 0.99)).float()
        dr = self.rgb - self.obs_rgb
        dd = self.depth - self.obs_depth
        self.loss = (self.alpha * (dr.abs() * mask).sum() / (3 * P) +
                     self.beta * (dd.abs() * mask).sum() / P)
        g_rgb = (torch.sign(dr) * mask * (self.alpha / (3 * P))).contiguous()
        g_d = (torch.sign(dd) * mask * (self.beta / P)).contiguous()
        self.d_twist.zero_()
        self.R.backward(g_rgb, g_d, None, pose_grad=True, d_twist=self.d_twist, d_mat=self.d_mat)
        g = self.d_twist
        b1, b2, eps = 0.9, 0.999, 1e-15
        self.t += 1
        self.m.mul_(b1).add_((1 - b1) * g)
        self.v.mul_(b2).add_((1 - b2) * g * g)
        mh = self.m / (1 - b1 ** self.t)
        vh = self.v / (1 - b2 ** self.t)
        step = self.lr * mh / (torch.sqrt(vh) + eps)
        Rd, td = se3_exp(-step)
        Rm = self.pose[:9].reshape(3, 3)
        tm = self.pose[9:]
        new = torch.cat([(Rm @ Rd).reshape(-1), Rm @ td + tm])
        self.pose.copy_(new)
        return self.loss

    def capture(self, warmup: int = 3):
        """Record one step() in a CUDA graph (the renderer's workspace must be
        reserved first: a captured render allocates nothing).  Afterwards
        replay() runs the step with one launch; the pose, optimiser state and
        observation buffers are updated in place."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.loss


def pose_error(P, Q):
    """(translation error m, rotation error deg) between two (3,4) poses."""
    P = api.matrix_of(P) if not isinstance(P, np.ndarray) or P.shape == (12,) else P
    Q = api.matrix_of(Q) if not isinstance(Q, np.ndarray) or Q.shape == (12,) else Q
    dt = float(np.linalg.norm(P[:, 3] - Q[:, 3]))
    dR = P[:, :3].T @ Q[:, :3]
    ang = float(np.degrees(np.arccos(np.clip((np.trace(dR) - 1) / 2, -1, 1))))
    return dt, ang
