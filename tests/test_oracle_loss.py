"""Pins of the oracle's visibility check (Sec. 3.3) and masked L1 loss
(Eq. 1, Eq. 2): closed forms of simple geometry, invariants and finite
differences."""

import numpy as np
import pytest

import oracle
from paper_2506_02741_gb300 import synthetic as syn

W, H = 40, 30
K = (30.0, 36.0, (W - 1) / 2, (H - 1) / 2)   # fx != fy on purpose


def _pose(t=(0.0, 0.0, 0.0), R=None):
    P = np.zeros((3, 4))
    P[:, :3] = np.eye(3) if R is None else R
    P[:, 3] = t
    return P


def _plane(z, w=W, h=H):
    return np.full((h, w), z, np.float32)


def test_self_visibility_interior():
    """A frame checked against itself: every interior valid pixel projects
    (to rounding) onto itself, so it is visible; invalid pixels never are."""
    K64 = syn.TINY
    fr = syn.render_frames(syn.make_room(syn.SCENE_SEED), K64, [syn.identity_pose()])
    d = fr.depth[0].copy()
    d[5, 7] = 0.0
    d[9, 11] = np.nan
    d[20, 30] = -1.0
    vis = oracle.visibility(d, K64.astuple(), syn.identity_pose(), [(d, K64.astuple(), syn.identity_pose())])
    assert not vis[5, 7] and not vis[9, 11] and not vis[20, 30]
    inner = np.zeros_like(vis)
    inner[1:-1, 1:-1] = True
    bad = np.zeros_like(vis)
    for (j, i) in ((5, 7), (9, 11), (20, 30)):   # neighbourhoods of the invalid pixels
        bad[j - 1:j + 2, i - 1:i + 2] = True
    assert vis[inner & ~bad].all()


@pytest.mark.parametrize("scale, expect", [(1.0, True), (1.009, True), (1.011, False)])
def test_plane_seen_from_behind(scale, expect):
    """Fronto-parallel plane at 2 m; the view sits 0.5 m behind with the same
    orientation, so every point lies at 2.5 m in the view and projects to
    cx + 0.8 (u - cx), inside the image.  The view's depth map holds
    2.5 * scale: visible iff |2.5 - 2.5 s| <= 0.01 * 2.5 s."""
    d = _plane(2.0)
    vd = _plane(np.float32(2.5 * scale))
    vis = oracle.visibility(d, K, _pose(), [(vd, K, _pose((0.0, 0.0, -0.5)))])
    assert vis.all() == expect and vis.any() == expect


def test_behind_the_view_is_invisible():
    """The same view turned around (180 degrees about y) sees nothing."""
    R = np.diag([-1.0, 1.0, -1.0])
    vis = oracle.visibility(_plane(2.0), K, _pose(), [(_plane(2.5), K, _pose((0.0, 0.0, -0.5), R))])
    assert not vis.any()


@pytest.mark.parametrize("axis", [0, 1])
def test_half_pixel_shift_interpolates(axis):
    """The view moved by 0.5 * 2 / f m along x (axis 0) or y (axis 1) at the
    plane's depth 2 m: every point lands half a pixel before its own column
    (row), between two view pixels with weights 1/2.  Alternate view columns
    (rows) hold 2 and 2 (1 + b): the interpolated depth is 2 (1 + b/2),
    visible iff b/2 <= 0.01 (1 + b/2).  Column (row) 0 lands at -0.5, outside."""
    d = _plane(2.0)
    t = [0.0, 0.0, 0.0]
    t[axis] = 0.5 * 2.0 / K[axis]
    for b, expect in ((0.015, True), (0.025, False)):
        vd = _plane(2.0)
        if axis == 0:
            vd[:, 1::2] = np.float32(2.0 * (1 + b))
        else:
            vd[1::2, :] = np.float32(2.0 * (1 + b))
        vis = oracle.visibility(d, K, _pose(), [(vd, K, _pose(tuple(t)))])
        first = vis[:, 0] if axis == 0 else vis[0, :]
        rest = vis[:, 1:] if axis == 0 else vis[1:, :]
        assert not first.any()
        assert (rest == expect).all()


def _room_case():
    K64 = syn.TINY
    path = syn.trajectory(30)
    fr = syn.render_frames(syn.make_room(syn.SCENE_SEED), K64, [path[i] for i in (0, 10, 20, 29)])
    cur = fr.depth[3]
    views = [(fr.depth[k], K64.astuple(), path[i]) for k, i in enumerate((0, 10, 20))]
    return K64, cur, path[29], views


def test_rigid_motion_invariance_and_self_check():
    """Moving every camera by the same rigid motion G leaves the mask
    unchanged (depth maps live in camera frames), which fails for a
    transposed rotation anywhere in the transform chain; a frame checked
    against itself under a rotated pose sees its interior."""
    K64, cur, P, views = _room_case()
    vis = oracle.visibility(cur, K64.astuple(), P, views)
    assert 0.05 < vis.mean() < 0.999
    G = syn.compose(syn.perturb_pose(syn.identity_pose(), np.random.default_rng(5), 0.7, 40.0),
                    syn.identity_pose())
    moved = [(d, k, syn.compose(G, p)) for d, k, p in views]
    vis2 = oracle.visibility(cur, K64.astuple(), syn.compose(G, P), moved)
    assert (vis == vis2).all()
    own = oracle.visibility(cur, K64.astuple(), syn.compose(G, P),
                            [(cur, K64.astuple(), syn.compose(G, P))])
    assert own[1:-1, 1:-1].all()


def _occluded(cols):
    vd = _plane(2.5)
    vd[:, cols] = 1.0
    return vd


def test_occluder_and_union():
    """View 0.5 m behind: the point of column u projects to
    x = cx + 0.8 (u - cx).  An occluder (depth 1 m) over view columns
    [0, 20) hides the points whose interpolation stencil [floor x, floor x + 1]
    lies in it and leaves those whose stencil lies outside; a second view
    occluded over [20, 40) complements it, and the union sees every point
    whose stencil is clear in one of the two."""
    d = _plane(2.0)
    Pv = _pose((0.0, 0.0, -0.5))
    x = K[2] + 0.8 * (np.arange(W) - K[2])
    x0 = np.floor(x).astype(int)
    x1 = np.minimum(x0 + 1, W - 1)
    a = oracle.visibility(d, K, _pose(), [(_occluded(slice(0, 20)), K, Pv)])
    b = oracle.visibility(d, K, _pose(), [(_occluded(slice(20, 40)), K, Pv)])
    ab = oracle.visibility(d, K, _pose(), [(_occluded(slice(0, 20)), K, Pv),
                                          (_occluded(slice(20, 40)), K, Pv)])
    left, right = x1 < 20, x0 >= 20
    assert not a[:, left].any() and a[:, right].all()
    assert b[:, left].all() and not b[:, right].any()
    assert (ab == (a | b)).all()
    assert ab[:, left | right].all()


def _images(seed, h=6, w=7):
    rng = np.random.default_rng(seed)
    rgb = rng.random((3, h, w)).astype(np.float32)
    obs = rng.random((3, h, w)).astype(np.float32)
    depth = (1 + rng.random((h, w))).astype(np.float32)
    od = (1 + rng.random((h, w))).astype(np.float32)
    sil = rng.random((h, w)).astype(np.float32)
    return rgb, depth, sil, obs, od


def test_l1_constant_images():
    """Constant residuals: L = w_rgb |0.5 - 0.2| + w_depth |2 - 2.1| (FP32
    inputs), gradients -w_rgb/(3P) and -w_depth/P everywhere."""
    h, w = 5, 9
    P = h * w
    rgb = np.full((3, h, w), 0.5, np.float32)
    obs = np.full((3, h, w), 0.2, np.float32)
    dep = np.full((h, w), 2.0, np.float32)
    od = np.full((h, w), 2.1, np.float32)
    sil = np.ones((h, w), np.float32)
    L, gr, gd = oracle.masked_l1(rgb, dep, sil, obs, od, 0.5, 0.025, 0.99, True)
    e_c = 0.5 - float(np.float32(0.2))
    e_d = float(np.float32(2.1)) - 2.0
    assert L == pytest.approx(0.5 * e_c + 0.025 * e_d, rel=1e-14)
    assert np.all(gr == 0.5 / (3 * P)) and np.all(gd == -0.025 / P)


def test_l1_masks():
    """Invalid observed depth (0, NaN, negative) drops a pixel from both terms
    under Eq. 1 (rgb_needs_depth) and from the depth term only under Eq. 2;
    the coverage test is strict (silhouette == threshold is uncovered); the
    visibility mask drops pixels from both terms."""
    rgb, dep, sil, obs, od = _images(1)
    P = dep.size
    od[0, 0], od[1, 2], od[3, 4] = 0.0, np.nan, -1.0
    sil[:] = 1.0
    sil[2, 2] = np.float32(0.99)
    vis = np.ones(dep.shape, bool)
    vis[4, 5] = False
    er = np.abs(rgb.astype(np.float64) - obs)
    ed = np.abs(dep.astype(np.float64) - od)
    valid = np.isfinite(od) & (od > 0)
    for needs, smin, vmask in ((True, 0.99, vis), (False, -1.0, None)):
        L, gr, gd = oracle.masked_l1(rgb, dep, sil, obs, od, 0.8, 1.0, smin, needs, vmask)
        cov = sil > np.float32(smin) if smin >= 0 else np.ones(dep.shape, bool)
        vv = vmask if vmask is not None else np.ones(dep.shape, bool)
        m_d = valid & cov & vv
        m_c = cov & vv & (valid if needs else True)
        want = 0.8 / (3 * P) * er[:, m_c].sum() + 1.0 / P * ed[m_d].sum()
        assert L == pytest.approx(want, rel=1e-13)
        assert np.all(gr[:, ~m_c] == 0) and np.all(gd[~m_d] == 0)
        assert np.all(np.abs(gr[:, m_c]) == 0.8 / (3 * P))
    assert not (sil[2, 2] > np.float32(0.99))


def test_l1_gradient_is_finite_difference():
    """Away from zero residuals the loss is linear in each input, so central
    differences reproduce the gradient to rounding."""
    rgb, dep, sil, obs, od = _images(2)
    sil[:] = 1.0
    L0, gr, gd = oracle.masked_l1(rgb, dep, sil, obs, od, 0.5, 0.025, 0.99, True)
    h = 1e-3
    rng = np.random.default_rng(3)
    for _ in range(8):
        c, j, i = rng.integers(3), rng.integers(dep.shape[0]), rng.integers(dep.shape[1])
        if abs(float(rgb[c, j, i]) - float(obs[c, j, i])) < 2 * h:
            continue
        rp, rm = rgb.copy(), rgb.copy()
        rp[c, j, i] += np.float32(h)
        rm[c, j, i] -= np.float32(h)
        fd = (oracle.masked_l1(rp, dep, sil, obs, od, 0.5, 0.025, 0.99, True)[0] -
              oracle.masked_l1(rm, dep, sil, obs, od, 0.5, 0.025, 0.99, True)[0]) / \
            (float(rp[c, j, i]) - float(rm[c, j, i]))
        assert fd == pytest.approx(gr[c, j, i], rel=1e-6)
    dp, dm = dep.copy(), dep.copy()
    dp[1, 1] += np.float32(h)
    dm[1, 1] -= np.float32(h)
    fd = (oracle.masked_l1(rgb, dp, sil, obs, od, 0.5, 0.025, 0.99, True)[0] -
          oracle.masked_l1(rgb, dm, sil, obs, od, 0.5, 0.025, 0.99, True)[0]) / \
        (float(dp[1, 1]) - float(dm[1, 1]))
    assert fd == pytest.approx(gd[1, 1], rel=1e-6)


def test_l1_zero_residual_has_zero_gradient():
    rgb, dep, sil, obs, od = _images(4)
    L, gr, gd = oracle.masked_l1(rgb, dep, sil, rgb.copy(), dep.copy(), 0.5, 0.025)
    assert L == 0.0 and not gr.any() and not gd.any()
