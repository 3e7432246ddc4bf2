"""Scene mapping driver (Sec. 3.4): learn the colour, opacity and radius of
the Gaussians of the current section by rendering it from the views of the
section and minimising the L1 terms of Eq. 2,

    rho |V - V'|_1 + sigma U |D - D'|_1        (rho = 0.8, sigma = 1.0),

with U masking pixels without valid depth.  The SSIM term of Eq. 2 is not
part of this driver.  The render and its attribute gradient run in the vtsplat
kernels, the loss and its image gradient in one kernel (vt_masked_l1); the
Adam step (learning rates of the supplementary: colour 0.0025, radius 0.005,
opacity 0.05) is a torch fused optimiser on the device.

The learning rates apply, as in the 3D Gaussian splatting family the paper
builds on, to logit(opacity) and log(radius) (a reading: the paper gives the
rates, not the parametrisation); the kernels take and return the activated
values, and this driver applies the chain rule.  Attributes may be stored in
FP16 (all arithmetic stays FP32): the optimiser keeps FP32 master copies and
writes the storage after each step.
"""

from __future__ import annotations

import numpy as np
import torch

from . import api


class SectionMapper:
    def __init__(self, renderer: api.Renderer, section: api.Section, frames_rgb: torch.Tensor,
                 lr_colour: float = 0.0025, lr_opacity: float = 0.05, lr_radius: float = 0.005,
                 rho: float = 0.8, sigma: float = 1.0):
        self.R = renderer
        self.sec = section
        self.rgb_obs = frames_rgb                      # (V, 3, H, W) float32, device
        self.depth_obs = section.depth                 # (V, H, W)
        self.V, self.H, self.W = section.depth.shape
        self.rho, self.sigma = float(rho), float(sigma)
        dev = section.colour.device
        o = section.opacity.detach().float().clamp(1e-4, 1 - 1e-4)
        self.master = [section.colour.detach().float().clone(), torch.log(o / (1 - o)),
                       torch.log(section.radius.detach().float())]
        for m in self.master:
            m.grad = torch.zeros_like(m)
        self.d_o = torch.zeros_like(self.master[1])
        self.d_r = torch.zeros_like(self.master[2])
        self.opt = torch.optim.Adam(
            [{"params": [self.master[0]], "lr": lr_colour},
             {"params": [self.master[1]], "lr": lr_opacity},
             {"params": [self.master[2]], "lr": lr_radius}], fused=True)
        self.rgb = torch.empty(3, self.H, self.W, device=dev)
        self.depth = torch.empty(self.H, self.W, device=dev)
        self.sil = torch.empty(self.H, self.W, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.g_rgb = torch.zeros(3, self.H, self.W, device=dev)
        self.g_depth = torch.zeros(self.H, self.W, device=dev)

    def step(self, view: int):
        """One mapping iteration rendering from section view ``view``."""
        pose = self.sec.poses[view]
        K = self.sec.K
        self.R.render([self.sec], pose, K, self.W, self.H, self.rgb, self.depth, self.sil)
        self.R.masked_l1(self.rgb, self.depth, None, self.rgb_obs[view], self.depth_obs[view],
                         self.rho, self.sigma, d_rgb=self.g_rgb, d_depth=self.g_depth,
                         loss=self.loss)
        self.master[0].grad.zero_()
        self.d_o.zero_()
        self.d_r.zero_()
        self.R.backward(self.g_rgb, self.g_depth, None,
                        attr_grads=[(self.master[0].grad, self.d_o, self.d_r)])
        with torch.no_grad():
            o = torch.sigmoid(self.master[1])
            r = torch.exp(self.master[2])
            torch.mul(self.d_o, o * (1 - o), out=self.master[1].grad)   # d/dlogit
            torch.mul(self.d_r, r, out=self.master[2].grad)             # d/dlog r
        self.opt.step()
        with torch.no_grad():
            self.sec.colour.copy_(self.master[0])
            self.sec.opacity.copy_(torch.sigmoid(self.master[1]))
            self.sec.radius.copy_(torch.exp(self.master[2]))
        return self.loss


def random_views(n_views: int, iters: int, seed: int = 0):
    """Views to map from, drawn uniformly (Sec. 3.4: a random view of the section)."""
    return np.random.default_rng(seed).integers(0, n_views, iters).tolist()
