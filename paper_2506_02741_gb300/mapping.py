"""Scene mapping loop (Sec. 3.4): learn the colour, opacity and radius of
the Gaussians of the current section by rendering it from the views of the
section and minimising the L1 terms of Eq. 2,

    rho |V - V'|_1 + sigma U |D - D'|_1        (rho = 0.8, sigma = 1.0),

with U masking pixels without valid depth, plus tau L_S (tau = 0.2, Sec. 4;
ssim=False leaves it out).  Every step of an iteration runs in the vtsplat
kernels: render, the masked L1 loss and its image gradient (vt_masked_l1),
the SSIM term accumulated into the same gradient (vt_ssim), the attribute
backward and one fused Adam step (vt_attr_adam; learning rates of the
supplementary: colour 0.0025, radius 0.005, opacity 0.05).  Ellipsoid
sections (the anisotropic variant of the attribute ablation) also learn
their scales and rotations (vt_shape_adam; rates 0.005 for the log scales
and 0.001 for the quaternion, the 3D Gaussian splatting defaults).

The learning rates apply, as in the 3D Gaussian splatting family the paper
builds on, to logit(opacity) and log(radius) (a reading: the paper gives the
rates, not the parametrisation); the kernels take and return the activated
values, and the optimiser applies the chain rule.  Attributes may be stored in
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
                 rho: float = 0.8, sigma: float = 1.0, tau: float = 0.2, ssim: bool = True,
                 lr_scale: float = 0.005, lr_rot: float = 0.001):
        self.R = renderer
        self.sec = section
        self.rgb_obs = frames_rgb                      # (V, 3, H, W) float32, device
        self.depth_obs = section.depth                 # (V, H, W)
        self.V, self.H, self.W = section.depth.shape
        self.rho, self.sigma, self.tau = float(rho), float(sigma), float(tau)
        self.use_ssim = bool(ssim)
        self.lr = [lr_colour] * 3 + [lr_opacity, lr_radius]
        dev = section.colour.device
        n = section.n
        # (c, logit o, log r) and zero moments, formed by the library
        self.theta, self.m, self.v, self.step_state = api.adam_init(section, renderer=renderer)
        self.d_colour = torch.zeros(n, 3, device=dev)
        self.d_opacity = torch.zeros(n, device=dev)
        self.d_radius = torch.zeros(n, device=dev)
        self.rgb = torch.empty(3, self.H, self.W, device=dev)
        self.depth = torch.empty(self.H, self.W, device=dev)
        self.sil = torch.empty(self.H, self.W, device=dev)
        self.losses = torch.zeros(2, dtype=torch.float64, device=dev)   # L1 terms, SSIM term
        self.loss = self.losses[:1]
        self.g_rgb = torch.zeros(3, self.H, self.W, device=dev)
        self.g_depth = torch.zeros(self.H, self.W, device=dev)
        self.shape = None
        if section.ellipsoids:
            self.lr_shape = (float(lr_scale), float(lr_rot))
            self.shape, self.shape_m, self.shape_v, self.shape_step = api.adam_init(
                section, shape=True, renderer=renderer)
            self.d_scale = torch.zeros(n, 3, device=dev)
            self.d_rot = torch.zeros(n, 4, device=dev)

    def step(self, view: int):
        """One mapping iteration rendering from section view ``view``.  Returns
        the device tensor (L1 terms, SSIM term) of the iteration (the SSIM
        entry stays 0 without the SSIM term); the Eq. 2 loss is their sum,
        left to the caller so that the iteration launches no reduction of
        its own."""
        self.R.render([self.sec], self.sec.poses[view], self.sec.K, self.W, self.H, self.rgb,
                      self.depth, self.sil)
        self.R.masked_l1(self.rgb, self.depth, None, self.rgb_obs[view], self.depth_obs[view],
                         self.rho, self.sigma, d_rgb=self.g_rgb, d_depth=self.g_depth,
                         loss=self.losses[0:1])
        if self.use_ssim:
            self.R.ssim(self.rgb, self.rgb_obs[view], self.tau, d_rgb=self.g_rgb,
                        loss=self.losses[1:2])
        # the gradients were zeroed by the previous Adam step (and at construction)
        if self.shape is None:
            grads = (self.d_colour, self.d_opacity, self.d_radius)
        else:
            grads = (self.d_colour, self.d_opacity, None, self.d_scale, self.d_rot)
        self.R.backward(self.g_rgb, self.g_depth, None, attr_grads=[grads])
        api.attr_adam(self.sec, self.theta, self.m, self.v, self.step_state, self.d_colour,
                      self.d_opacity, self.d_radius, self.lr, renderer=self.R)
        if self.shape is not None:
            api.shape_adam(self.sec, self.shape, self.shape_m, self.shape_v, self.shape_step,
                           self.d_scale, self.d_rot, *self.lr_shape, renderer=self.R)
        return self.losses


def random_views(n_views: int, iters: int, seed: int = 0):
    """Views to map from, drawn uniformly (Sec. 3.4: a random view of the section)."""
    return np.random.default_rng(seed).integers(0, n_views, iters).tolist()
