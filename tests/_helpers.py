"""Test-only helpers: small hand-built sections and pose perturbations.

Nothing here computes the splatting method; it assembles inputs.
"""

from __future__ import annotations

import math

import numpy as np

from paper_2506_02741_gb300 import synthetic as syn


def hand_section(views, W, H, K, colour=None, opacity=None, radius=None):
    """Build an oracle.Section from explicit views.

    views: list of (pose (3,4), {(u, v): depth}) -- every listed pixel is a
    valid depth pixel, every other pixel invalid (depth 0).  colour/opacity/
    radius default to grey, 0.9 and D/fx (the initial values)."""
    import oracle
    V = len(views)
    depth = np.zeros((V, H, W), np.float32)
    poses = np.zeros((V, 3, 4))
    for k, (pose, pix) in enumerate(views):
        poses[k] = pose
        for (u, v), d in pix.items():
            depth[k, v, u] = d
    src = np.flatnonzero(depth.reshape(-1) > 0).astype(np.uint32)
    n = src.size
    D = depth.reshape(-1)[src].astype(np.float64)
    fx = float(np.float32(K[0]))
    col = np.full((n, 3), 0.5) if colour is None else np.asarray(colour, np.float64).reshape(n, 3)
    op = np.full(n, 0.9) if opacity is None else np.asarray(opacity, np.float64).reshape(n)
    rad = D / fx if radius is None else np.asarray(radius, np.float64).reshape(n)
    return oracle.Section(W, H, tuple(float(np.float32(k)) for k in K), poses, depth, src,
                          col, op, rad)


def tiny_section(randomise=True, seed=5):
    """The 64x48 single-view workload as an oracle.Section plus its target pose.
    With ``randomise`` the attributes are replaced by seeded random values so
    that every gradient path is exercised."""
    import oracle
    room, fr, target = syn.tiny_workload()
    K = syn.TINY
    sec = oracle.section_init(fr.depth, fr.rgb, K.astuple(), np.stack(fr.poses))
    if randomise:
        col, op, rs = syn.random_attributes(sec.n, seed, opacity_range=(0.3, 0.95))
        sec.colour = col
        sec.opacity = op
        sec.radius = sec.radius * rs
    return sec, target, K


def multiview_section(K, n_views=2, key_every=5, randomise=True, seed=7):
    import oracle
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(n_views * key_every + 3)
    keys = [path[i * key_every] for i in range(n_views)]
    fr = syn.render_frames(room, K, keys)
    sec = oracle.section_init(fr.depth, fr.rgb, K.astuple(), np.stack(keys))
    if randomise:
        col, op, rs = syn.random_attributes(sec.n, seed, opacity_range=(0.2, 0.97))
        sec.colour = col
        sec.opacity = op
        sec.radius = sec.radius * rs
    target = path[(n_views - 1) * key_every + 2]
    return sec, target


def right_perturb(pose, k, h):
    """P * Exp(h e_k) for twist component k (0-2 translation, 3-5 rotation)."""
    P = np.asarray(pose, np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    if k < 3:
        e = np.zeros(3)
        e[k] = h
        return np.hstack([R, (t + R @ e)[:, None]])
    w = np.zeros(3)
    w[k - 3] = h
    return np.hstack([R @ syn.rotvec_to_matrix(w), t[:, None]])


def entry_perturb(pose, k, h):
    """Add h to entry k of (R row-major, t)."""
    P = np.asarray(pose, np.float64).reshape(3, 4).copy()
    if k < 9:
        P[k // 3, k % 3] += h
    else:
        P[k - 9, 3] += h
    return P


def random_rigid(rng):
    R = syn.rotvec_to_matrix(rng.normal(0, 0.7, 3))
    t = rng.normal(0, 3.0, 3)
    return np.hstack([R, t[:, None]])


def l_of(out, g_rgb, g_depth, g_sil):
    return float(np.sum(out["rgb"] * g_rgb) + np.sum(out["depth"] * g_depth) +
                 np.sum(out["sil"] * g_sil))


def l_diff(a, b, g_rgb, g_depth, g_sil):
    """<g, a - b>: the difference of two linear losses, formed pixel-wise so
    that untouched pixels cancel exactly."""
    return float(np.sum((a["rgb"] - b["rgb"]) * g_rgb) + np.sum((a["depth"] - b["depth"]) * g_depth)
                 + np.sum((a["sil"] - b["sil"]) * g_sil))


def deg(x):
    return math.degrees(x)
