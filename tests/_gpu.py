"""Test-only bridge: the same seeded inputs for the oracle and the CUDA path.

Attributes are first rounded to the storage precision (float32 or float16)
so that both sides read identical values.
"""

from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2506_02741_gb300 import api


def quantise(sec: "oracle.Section", prec: str = "f32") -> "oracle.Section":
    dt = np.float16 if prec == "f16" else np.float32
    q = lambda a: np.asarray(a, dt).astype(np.float64)
    return oracle.Section(sec.W, sec.H, sec.K, sec.poses, sec.depth, sec.src, q(sec.colour),
                          q(sec.opacity), q(sec.radius))


def to_device(sec: "oracle.Section", prec: str = "f32", device="cuda") -> api.Section:
    dt = torch.float16 if prec == "f16" else torch.float32
    t = lambda a, d=dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=d)
    return api.Section(api.pose12(sec.poses, device).reshape(-1, 12).contiguous(),
                       t(sec.depth, torch.float32).contiguous(), tuple(sec.K),
                       torch.from_numpy(sec.src.astype(np.uint32).view(np.int32).copy()).to(device),
                       t(sec.colour.reshape(-1, 3)).contiguous(), t(sec.opacity).contiguous(),
                       t(sec.radius).contiguous())


def clean_mask(ref: dict, tau_incl=1e-5, tau_T=2e-4, tau_clamp=None) -> np.ndarray:
    """Pixels whose every inclusion / termination decision is farther than the
    given relative margins from its threshold: there FP32 and FP64 must take
    the same decisions.  The FP32 kernels compute q to ~6e-7 and ahat to
    ~3e-6 relative (exp of an argument up to 4.5), and the transmittance to
    ~1e-4 after many steps near the 0.99 clamp, hence the default margins."""
    m = (ref["margin"] > tau_incl) & (ref["margin_T"] > tau_T)
    if tau_clamp is not None:
        m &= ref["margin_clamp"] > tau_clamp
    return m


def assert_forward_close(out, ref, mask, tol=1e-5, depth_scale=4.0):
    rgb, depth, sil = (x.detach().cpu().numpy().astype(np.float64) for x in out)
    err = {}
    for name, g, r, s in (("rgb", rgb, ref["rgb"], 1.0), ("depth", depth, ref["depth"], depth_scale),
                          ("sil", sil, ref["sil"], 1.0)):
        m = np.broadcast_to(mask, g.shape)
        bound = tol * np.maximum(np.abs(r), s)
        bad = (np.abs(g - r) > bound) & m
        err[name] = float(np.max(np.abs(g - r)[m])) if m.any() else 0.0
        assert not bad.any(), (name, int(bad.sum()), float(np.max((np.abs(g - r) / bound)[m])))
    return err


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Bound on the rounding noise of a pose-gradient component summed per pixel
# in FP32 and across pixels in FP64, in units of the oracle's noise scale
# sqrt(sum_p n_p m_p^2): per pixel, each of the n_p terms and each running
# sum rounds with relative error <= 2^-24 (a few roundings per term), and the
# pixels' errors are independent, so the total stays within a few units of
# 2^-24 x the scale; 8 leaves room for the tail.
POSE_NOISE = 8.0 * 2.0 ** -24


def assert_grad_close(g, ref, tol=1e-4, name="", abs_ref=None, noise=None):
    """Per-tensor relative L2 <= tol, and per element
    |g - ref| <= tol * max(|ref|, 1e-3 max|ref|) + tol * sum|terms|
                 + POSE_NOISE * noise.

    The second term applies the same relative tolerance to the componentwise
    magnitude of each pixel's term (the oracle reports, per element, the sum
    over pixels of the absolute values of the products the derivative formula
    adds): terms cancel within a pixel's formula and across pixels, and each
    FP32 product carries the error of the transmittance product in front of
    it, about sum_i (alpha_i / (1 - alpha_i)) x 1e-7 (~1e-5 to 1e-4 after 50
    Gaussians of alpha ~0.9)."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert rel_l2(g, ref) <= tol, (name, rel_l2(g, ref))
    floor = 1e-3 * np.max(np.abs(ref)) if ref.size else 0.0
    bound = tol * np.maximum(np.abs(ref), floor)
    if abs_ref is not None:
        bound = bound + tol * np.asarray(abs_ref, np.float64).ravel()
    if noise is not None:
        bound = bound + POSE_NOISE * np.asarray(noise, np.float64).ravel()
    bad = np.abs(g - ref) > bound
    assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(g - ref) / bound)))
