"""Test-only bridge: the same seeded inputs for the oracle and the CUDA path.

Attributes are first rounded to the storage precision (float32 or float16)
so that both sides read identical values.
"""

from __future__ import annotations

import os

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


# Relative margins within which a decision of the definition may go either
# way between the FP32 kernels and the FP64 oracle: the kernels compute q to
# ~6e-7 and ahat to ~3e-6 relative (exp of an argument up to 4.5), and the
# transmittance to ~1e-4 after many steps near the 0.99 clamp.
TAU_INCL = 1e-5
TAU_T = 2e-4

# Per-case decision statistics of the parity tests (printed with -s).
STATS = []


def _case() -> str:
    return os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]


def _report(kind, name, ratio, strict=None, rel=None):
    """Prints the achieved error of one compared tensor as a fraction of its
    bound (ratio <= 1 passes); strict: the same against the plain per-element
    bound tol * max(|ref|, floor) without the magnitude and noise terms."""
    rec = dict(case=_case(), tensor=name, ratio=round(float(ratio), 4))
    if strict is not None:
        rec["strict_ratio"] = round(float(strict), 4)
    if rel is not None:
        rec["rel_l2"] = float(f"{rel:.3g}")
    print(kind, rec)


def gpu_lists(R, W, H, box=None, id_map=None):
    """The GPU's decisions: per-pixel lists of added Gaussians (ids (h, w,
    cap) int64 and counts (h, w)) of the last render of renderer R for the
    rectangle box = (x0, y0, w, h) (default: the whole W x H image).  Every
    pixel's list must be complete (no pixel added more than the context
    keeps).  id_map translates the GPU's ids (positions in the concatenation
    of the render's sections) to the oracle's."""
    x0, y0, w, h = box or (0, 0, W, H)
    ids, _T, counts, kept = R.pixel_lists(x0, y0, w, h)
    assert counts.max(initial=0) <= kept, ("a pixel list overflowed", int(counts.max()), kept)
    if id_map is not None:
        ids = id_map(ids)
        assert np.all(ids[np.arange(ids.shape[2])[None, None, :] < counts[:, :, None]] >= 0), \
            "a Gaussian the GPU added is missing from the oracle's input"
    return ids, counts


def subset_map(keep_masks):
    """id_map for an oracle input made of the Gaussians keep_masks[s] of each
    section s of the GPU render, in their order (-1 for a Gaussian left
    out)."""
    bases = np.cumsum([0] + [len(k) for k in keep_masks[:-1]])
    kept = np.concatenate([np.flatnonzero(k) + b for k, b in zip(keep_masks, bases)])
    kept = kept.astype(np.int64)

    def f(ids):
        if kept.size == 0:
            return np.full_like(ids, -1)
        pos = np.minimum(np.searchsorted(kept, np.maximum(ids, 0)), kept.size - 1)
        return np.where((ids >= 0) & (kept[pos] == ids), pos, -1)
    return f


def check_decisions(ref, name=""):
    """Every pixel's GPU list is one of the definition's up to decisions
    within the margins render_lists was given (status 0); records and
    returns the count of pixels with a decision taken otherwise than in
    FP64."""
    st = ref["status"]
    bad = np.argwhere(st != 0)
    assert bad.size == 0, (name, int((st != 0).sum()), [tuple(b) for b in bad[:5]],
                           [int(st[tuple(b)]) for b in bad[:5]])
    rec = dict(case=name, pixels=int(st.size), flip_pixels=int((ref["flips"] > 0).sum()),
               flips=int(ref["flips"].sum()),
               max_flip_margin=float(ref["flip_margin"].max(initial=0.0)))
    STATS.append(rec)
    print("PARITY_DECISIONS", rec)
    return rec


def assert_forward_close(out, ref, mask=None, tol=1e-5, depth_scale=4.0):
    """|gpu - ref| <= tol max(|ref|, s) at every pixel (of mask, if given),
    s = 1 for colour and silhouette, depth_scale for depth."""
    rgb, depth, sil = (x.detach().cpu().numpy().astype(np.float64) for x in out)
    if mask is None:
        mask = np.ones(depth.shape, bool)
    err = {}
    for name, g, r, s in (("rgb", rgb, ref["rgb"], 1.0), ("depth", depth, ref["depth"], depth_scale),
                          ("sil", sil, ref["sil"], 1.0)):
        m = np.broadcast_to(mask, g.shape)
        bound = tol * np.maximum(np.abs(r), s)
        bad = (np.abs(g - r) > bound) & m
        err[name] = float(np.max(np.abs(g - r)[m])) if m.any() else 0.0
        ratio = float(np.max((np.abs(g - r) / bound)[m])) if m.any() else 0.0
        _report("PARITY_ERROR", name, ratio)
        assert not bad.any(), (name, int(bad.sum()), ratio)
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
    floor = 1e-3 * np.max(np.abs(ref)) if ref.size else 0.0
    bound = tol * np.maximum(np.abs(ref), floor)
    diff = np.abs(g - ref)
    strict = float(np.max(diff / np.maximum(bound, 1e-300))) if ref.size else 0.0
    assert rel_l2(g, ref) <= tol, (name, rel_l2(g, ref))
    if abs_ref is not None:
        bound = bound + tol * np.asarray(abs_ref, np.float64).ravel()
    if noise is not None:
        bound = bound + POSE_NOISE * np.asarray(noise, np.float64).ravel()
    bad = diff > bound
    ratio = float(np.max(diff / np.maximum(bound, 1e-300))) if ref.size else 0.0
    _report("PARITY_ERROR", name, ratio, strict, rel_l2(g, ref))
    assert not bad.any(), (name, int(bad.sum()), ratio)


def decisions(dsecs, pose12, K, W, H, out=None, box=None, id_map=None, cap=None):
    """The GPU's decisions of a render of dsecs taken on a fresh context that
    keeps per-pixel lists (capacity cap, default the library's); with out
    (the images of another render of the same inputs) the images must be
    bit-identical: the decisions do not depend on whether lists are kept."""
    R = api.Renderer()
    if cap:
        R.set_list_capacity(cap)
    o = R.render(dsecs, pose12, K, W, H, checked=True)
    torch.cuda.synchronize()
    if out is not None:
        for a, b in zip(o, out):
            assert torch.equal(a, b)
    return gpu_lists(R, W, H, box, id_map)
