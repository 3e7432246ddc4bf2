"""Pins of the source-view pose gradients (head-frame bundle adjustment,
Sec. 3.4): central differences of the oracle's render when one view's pose
moves all the Gaussians tied to that view."""

import copy

import numpy as np

import oracle
from paper_2506_02741_gb300 import synthetic as syn
from tests import _helpers as h


def _stable(base, others):
    m = np.ones(base["n_added"].shape, bool)
    for o in others:
        m &= np.all(o["lists"] == base["lists"], axis=-1) & (o["n_added"] == base["n_added"])
    return m


def _with_view_pose(sec, k, P):
    s = copy.copy(sec)
    s.poses = sec.poses.copy()
    s.poses[k] = P
    return s


def test_view_pose_gradient_finite_differences():
    K = syn.scaled_intrinsics(48, 36)
    sec, target = h.multiview_section(K, n_views=3, seed=9)
    args = (K.astuple(), K.W, K.H)
    cap = 192
    base = oracle.render(sec, target, *args, list_cap=cap)
    assert base["n_added"].max() < cap
    hstep = 1e-6
    renders = {}
    for kind, fn, nk in (("twist", h.right_perturb, 6), ("mat", h.entry_perturb, 12)):
        for v in range(3):
            for k in range(nk):
                for s in (+1, -1):
                    renders[(kind, v, k, s)] = oracle.render(
                        _with_view_pose(sec, v, fn(sec.poses[v], k, s * hstep)), target, *args,
                        list_cap=cap)
    stable = _stable(base, renders.values()) & (base["margin"] > 1e-6) & (base["margin_T"] > 1e-6)
    assert stable.mean() > 0.8
    rng = np.random.default_rng(31)
    gR = rng.normal(0, 1, (3, K.H, K.W)) * stable
    gD = rng.normal(0, 1, (K.H, K.W)) * stable
    gS = rng.normal(0, 1, (K.H, K.W)) * stable
    g = oracle.backward(sec, target, *args, g_rgb=gR, g_depth=gD, g_sil=gS)
    tw, mat = oracle.view_pose_grads(sec, target, g["x"][0])
    for kind, an, nk in (("twist", tw, 6), ("mat", mat, 12)):
        fd = np.array([[h.l_diff(renders[(kind, v, k, 1)], renders[(kind, v, k, -1)], gR, gD, gS) /
                        (2 * hstep) for k in range(nk)] for v in range(3)])
        scale = np.max(np.abs(an))
        assert scale > 1.0
        np.testing.assert_allclose(an, fd, rtol=2e-6, atol=2e-6 * scale, err_msg=kind)


def test_rigid_motion_of_everything_has_no_view_gradient_sum():
    """Moving the target camera and every source view by the same rigid
    motion leaves the render unchanged, so for the world-frame translation
    the source-view gradients cancel the target's: sum_k dL/dt_k + dL/dt = 0
    (a one-section render)."""
    K = syn.scaled_intrinsics(48, 36)
    sec, target = h.multiview_section(K, n_views=3, seed=10)
    rng = np.random.default_rng(32)
    gR = rng.normal(0, 1, (3, K.H, K.W))
    g = oracle.backward(sec, target, K.astuple(), K.W, K.H, g_rgb=gR)
    tw, mat = oracle.view_pose_grads(sec, target, g["x"][0])
    tot = mat[:, 9:].sum(0) + g["mat"][9:]
    assert np.abs(tot).max() <= 1e-9 * np.abs(g["mat"][9:]).max()


def test_depth_gradient_finite_differences():
    """Moving single Gaussians along their rays (their depth-map values)
    changes the loss as dL/dD predicts."""
    K = syn.scaled_intrinsics(48, 36)
    sec, target = h.multiview_section(K, n_views=2, seed=12)
    args = (K.astuple(), K.W, K.H)
    cap = 192
    base = oracle.render(sec, target, *args, list_cap=cap)
    rng = np.random.default_rng(33)
    gR = rng.normal(0, 1, (3, K.H, K.W))
    gD = rng.normal(0, 1, (K.H, K.W))
    g = oracle.backward(sec, target, *args, g_rgb=gR, g_depth=gD)
    dd = oracle.depth_grads(sec, target, g["x"][0])
    order = np.argsort(-np.abs(dd))
    checked = 0
    for i in order[:40]:
        src = int(sec.src[i])
        D = sec.depth.reshape(-1)[src]
        renders = []
        for s in (+1, -1):
            t = copy.copy(sec)
            t.depth = sec.depth.copy()
            t.depth.reshape(-1)[src] = np.float32(D * (1 + s * 2e-6))
            renders.append((oracle.render(t, target, *args, list_cap=cap),
                            float(t.depth.reshape(-1)[src])))
        (rp, dp), (rm, dm) = renders
        if not _stable(base, [rp, rm]).all():
            continue                     # a decision moved: the loss is not smooth here
        fd = h.l_diff(rp, rm, gR, gD, np.zeros_like(gD)) / (dp - dm)
        np.testing.assert_allclose(dd[i], fd, rtol=2e-3, atol=1e-6 * np.abs(dd).max())
        checked += 1
        if checked == 8:
            break
    assert checked >= 5
