"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test would catch a plausible slip in the oracle: a wrong footprint scale
or pixel convention (closed forms), a wrong compositing order or weight
(two-Gaussian and termination cases), a binning bug (brute vs binned), a
wrong transform (rigid-motion and source-pose invariance, back-projection
onto the generator's planes) and every gradient (central differences).
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2506_02741_gb300 import synthetic as syn
from tests import _helpers as h

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
IDENT = syn.identity_pose()


def test_single_gaussian_closed_form():
    """Sec. 3.2 + supplementary r = D/f: seen from its own camera a Gaussian
    has sigma = 1 px, so alpha = 0.9 exp(-d^2/2) inside the 3-pixel disc."""
    W, H, f = 16, 12, 20.0
    K = (f, f, 7.5, 5.5)
    u0, v0, D = 8, 6, 2.0
    col = np.array([[0.2, 0.5, 0.9]])
    sec = h.hand_section([(IDENT, {(u0, v0): D})], W, H, K, colour=col)
    out = oracle.render(sec, IDENT, K, W, H, binned=False)
    seen = set()
    for c in GOLD["single_gaussian"]["cases"]:
        du, dv = c["offset"]
        a = c["alpha"]
        u, v = u0 + du, v0 + dv
        seen.add((u, v))
        np.testing.assert_allclose(out["rgb"][:, v, u], col[0] * a, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out["sil"][v, u], a, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out["depth"][v, u], D * a, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out["T_final"][v, u], 1 - a, rtol=1e-12)
        assert out["n_added"][v, u] == (1 if a > 0 else 0)
    # nothing outside the 3-pixel disc
    vv, uu = np.mgrid[0:H, 0:W]
    outside = (uu - u0) ** 2 + (vv - v0) ** 2 > 9
    assert np.all(out["sil"][outside] == 0.0)
    assert np.all(out["rgb"][:, outside] == 0.0)


def test_two_gaussians_front_back_and_ties():
    """Front-to-back compositing: C = c1 a1 + c2 a2 (1 - a1); swapping the
    depths swaps the roles; equal depth keys are ordered by id (view order)."""
    W, H, f = 16, 12, 20.0
    K = (f, f, 7.5, 5.5)
    c1, c2 = np.array([1.0, 0.0, 0.25]), np.array([0.0, 1.0, 0.5])
    o1, o2 = 0.6, 0.7

    def run(d1, d2):
        sec = h.hand_section([(IDENT, {(8, 6): d1}), (IDENT, {(8, 6): d2})], W, H, K,
                             colour=np.stack([c1, c2]), opacity=[o1, o2])
        return oracle.render(sec, IDENT, K, W, H, binned=False)

    a = run(1.5, 2.5)
    np.testing.assert_allclose(a["rgb"][:, 6, 8], c1 * o1 + c2 * o2 * (1 - o1), rtol=1e-12)
    np.testing.assert_allclose(a["depth"][6, 8], 1.5 * o1 + 2.5 * o2 * (1 - o1), rtol=1e-12)
    e = math.exp(-0.5)
    np.testing.assert_allclose(a["rgb"][:, 6, 9],
                               c1 * o1 * e + c2 * o2 * e * (1 - o1 * e), rtol=1e-12)
    b = run(2.5, 1.5)
    np.testing.assert_allclose(b["rgb"][:, 6, 8], c2 * o2 + c1 * o1 * (1 - o2), rtol=1e-12)
    t = run(2.0, 2.0)
    np.testing.assert_allclose(t["rgb"][:, 6, 8], c1 * o1 + c2 * o2 * (1 - o1), rtol=1e-12)
    assert np.all(t["n_added"][6, 8] == 2)


def test_termination_exact():
    """T after i Gaussians of alpha 0.5 is 2^-i exactly: the 13th (1.22e-4)
    is added, the 14th (6.1e-5 < 1e-4) stops the walk."""
    g = GOLD["termination"]
    W, H, f = 16, 12, 20.0
    K = (f, f, 7.5, 5.5)
    n = g["n"]
    rng = np.random.default_rng(11)
    depths = 1.0 + 0.1 * rng.permutation(n)
    cols = rng.uniform(0, 1, (n, 3))
    sec = h.hand_section([(IDENT, {(8, 6): float(d)}) for d in depths], W, H, K, colour=cols,
                         opacity=np.full(n, g["opacity"]))
    out = oracle.render(sec, IDENT, K, W, H, binned=False, list_cap=32)
    assert out["n_added"][6, 8] == g["n_added"]
    assert out["sil"][6, 8] == pytest.approx(g["silhouette"], abs=1e-15)
    assert out["T_final"][6, 8] == g["T_final"]
    order = np.argsort(np.float32(depths), kind="stable")[: g["n_added"]]
    np.testing.assert_array_equal(out["lists"][6, 8, : g["n_added"]], order)
    expect = sum(2.0 ** -(i + 1) * cols[j] for i, j in enumerate(order))
    np.testing.assert_allclose(out["rgb"][:, 6, 8], expect, rtol=1e-14)


def test_layout_param_count():
    """Sec. 3.2 / Gaussian-type ablation: 5 learnable values per view-tied
    Gaussian versus 14, a saving of 9/14 = 64.3%."""
    g = GOLD["layout"]
    sec, _, _ = h.tiny_section(randomise=False)
    per = sec.colour.shape[1] + 1 + 1
    assert per == g["params_view_tied"]
    assert round(100 * (1 - per / g["params_3dgs"]), 1) == g["saving_percent"]


@pytest.mark.parametrize("case", ["tiny", "qqvga2"])
def test_brute_equals_binned(case):
    if case == "tiny":
        sec, target, K = h.tiny_section()
    else:
        K = syn.scaled_intrinsics(160, 120)
        sec, target = h.multiview_section(K, n_views=2)
    a = oracle.render(sec, target, K.astuple(), K.W, K.H, binned=False, list_cap=48)
    b = oracle.render(sec, target, K.astuple(), K.W, K.H, binned=True, list_cap=48)
    for k in ("rgb", "depth", "sil", "T_final", "n_added", "lists", "margin", "margin_T"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["n_added"].max() > 5


def test_silhouette_plus_transmittance_is_one():
    sec, target, K = h.tiny_section()
    out = oracle.render(sec, target, K.astuple(), K.W, K.H)
    assert np.max(np.abs(out["sil"] + out["T_final"] - 1.0)) < 1e-12
    assert np.all(out["T_final"] >= 1e-4 * (1 - 1e-12))


def test_rigid_world_motion_invariance():
    K = syn.scaled_intrinsics(96, 72)
    sec, target = h.multiview_section(K, n_views=2)
    G = h.random_rigid(np.random.default_rng(3))
    moved = oracle.Section(sec.W, sec.H, sec.K, np.stack([syn.compose(G, p) for p in sec.poses]),
                           sec.depth, sec.src, sec.colour, sec.opacity, sec.radius)
    a = oracle.render(sec, target, K.astuple(), K.W, K.H)
    b = oracle.render(moved, syn.compose(G, target), K.astuple(), K.W, K.H)
    for k in ("rgb", "depth", "sil", "T_final"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-9, err_msg=k)


def test_own_view_independent_of_pose():
    """A view rendered from its own pose sees x = back-projected X_c whatever
    that pose is.  The poses are axis-permutation rotations about the origin,
    for which every step is exact in floating point: a fronto-parallel wall
    seen from its own view puts neighbours at exactly q = 9 and gives all its
    Gaussians one depth key, so any rounding would flip decisions."""
    room, fr, _ = syn.tiny_workload()
    K = syn.TINY
    outs = []
    cyc = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    for R, t in ((np.eye(3), [0.0, 0.0, 0.0]), (cyc, [0.0, 0.0, 0.0]), (cyc.T, [0.0, 0.0, 0.0])):
        P = np.hstack([R, np.array(t)[:, None]])
        sec = oracle.section_init(fr.depth, fr.rgb, K.astuple(), P[None])
        outs.append(oracle.render(sec, P, K.astuple(), K.W, K.H))
    for o in outs[1:]:
        for k in ("rgb", "depth", "sil", "n_added"):
            np.testing.assert_array_equal(outs[0][k], o[k], err_msg=k)


def test_section_split_and_order():
    """Ids are (section, view, pixel): splitting a section keeps them; with no
    equal depth keys across sections the section order does not matter."""
    K = syn.scaled_intrinsics(96, 72)
    sec, target = h.multiview_section(K, n_views=2)
    plane = sec.W * sec.H
    view = sec.src // plane
    parts = []
    for k in range(2):
        m = view == k
        parts.append(oracle.Section(sec.W, sec.H, sec.K, sec.poses[k:k + 1], sec.depth[k:k + 1],
                                    (sec.src[m] - k * plane).astype(np.uint32), sec.colour[m],
                                    sec.opacity[m], sec.radius[m]))
    whole = oracle.render(sec, target, K.astuple(), K.W, K.H)
    split = oracle.render(parts, target, K.astuple(), K.W, K.H)
    for k in ("rgb", "depth", "sil", "n_added"):
        np.testing.assert_array_equal(whole[k], split[k], err_msg=k)
    # Swapping the sections changes the ids, hence the order of Gaussians
    # with equal depth keys across the two sections; every other pixel must
    # be bit-identical.
    za, _ = oracle.zkeys(parts[0], target, K.astuple(), K.W, K.H)
    zb, _ = oracle.zkeys(parts[1], target, K.astuple(), K.W, K.H)
    tied = np.concatenate([np.flatnonzero(np.isin(za, zb)),
                           parts[0].n + np.flatnonzero(np.isin(zb, za))])
    cap = 256
    whole = oracle.render(parts, target, K.astuple(), K.W, K.H, list_cap=cap)
    swapped = oracle.render(parts[::-1], target, K.astuple(), K.W, K.H, list_cap=cap)
    back = swapped["lists"].copy()        # ids of [B, A] -> ids of [A, B]
    nb = parts[1].n
    m = back >= 0
    back[m] = np.where(back[m] < nb, back[m] + parts[0].n, back[m] - nb)
    clean = ~(np.isin(whole["lists"], tied).any(-1) | np.isin(back, tied).any(-1))
    assert whole["n_added"].max() < cap and clean.mean() > 0.7
    np.testing.assert_array_equal(whole["lists"][clean], back[clean])
    for k in ("rgb", "depth", "sil"):
        np.testing.assert_array_equal(whole[k][..., clean], swapped[k][..., clean], err_msg=k)


def test_backprojection_lies_on_generator_planes():
    """Back-projected centres of back-wall pixels satisfy the generator's
    plane equation (independent ray-casting geometry)."""
    room = syn.make_room()
    K = syn.TINY
    P = syn.trajectory(8)[7]
    depth, _ = syn.raycast(room, K, P)
    cen, pix = oracle.backproject(depth, K.astuple(), P)
    assert cen.shape[0] == K.W * K.H
    n, hh = room.plane_n[2], room.plane_h[2]          # back wall z = 3.6
    resid = cen @ n - hh
    # float32 depth rounding bounds the residual by ~|X| * 2^-24 per step
    on = np.abs(resid) < 1e-3
    assert np.sum(np.abs(resid[on]) < 3.6 * 2e-7 * 4) > 0.99 * on.sum() > 1000
    # round trip: projecting back with the same camera recovers the pixel
    Xc = (cen - P[:, 3]) @ P[:, :3]
    u = K.fx * Xc[:, 0] / Xc[:, 2] + K.cx
    v = K.fy * Xc[:, 1] / Xc[:, 2] + K.cy
    np.testing.assert_allclose(u, pix % K.W, atol=1e-9)
    np.testing.assert_allclose(v, pix // K.W, atol=1e-9)
    np.testing.assert_allclose(Xc[:, 2], depth.reshape(-1)[pix], rtol=1e-12)


def test_section_init_values():
    room, fr, _ = syn.tiny_workload()
    K = syn.TINY
    d = fr.depth.copy()
    d[0, 3, 4] = 0.0
    d[0, 10, 11] = np.nan
    d[0, 20, 21] = -1.0
    sec = oracle.section_init(d, fr.rgb, K.astuple(), np.stack(fr.poses))
    assert sec.n == K.W * K.H - 3
    assert np.all(np.diff(sec.src.astype(np.int64)) > 0)
    D = d.reshape(-1)[sec.src]
    np.testing.assert_allclose(sec.radius, D.astype(np.float64) / np.float32(K.fx), rtol=1e-15)
    assert np.all(sec.opacity == 0.9)
    np.testing.assert_array_equal(sec.colour[:, 1], fr.rgb[0, 1].reshape(-1)[sec.src])


# ---------------------------------------------------------------------------
# gradients by central differences on the FP64 oracle


def _stable_mask(base, others):
    """Pixels whose added lists are identical in every perturbed render."""
    m = np.ones(base["n_added"].shape, bool)
    for o in others:
        m &= np.all(o["lists"] == base["lists"], axis=-1) & (o["n_added"] == base["n_added"])
    return m


def _upstream(shape, seed):
    H, W = shape
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1, (3, H, W)), rng.normal(0, 1, (H, W)), rng.normal(0, 1, (H, W))


def test_pose_gradient_finite_differences():
    sec, target, K = h.tiny_section()
    args = (K.astuple(), K.W, K.H)
    cap = 64
    base = oracle.render(sec, target, *args, list_cap=cap)
    assert base["n_added"].max() < cap
    hstep = 1e-6
    renders = {}
    for kind, fn, nk in (("twist", h.right_perturb, 6), ("mat", h.entry_perturb, 12)):
        for k in range(nk):
            for s in (+1, -1):
                renders[(kind, k, s)] = oracle.render(sec, fn(target, k, s * hstep), *args,
                                                      list_cap=cap)
    stable = _stable_mask(base, renders.values()) & (base["margin"] > 1e-6) & \
        (base["margin_T"] > 1e-6)
    assert stable.mean() > 0.95
    gR, gD, gS = _upstream((K.H, K.W), 21)
    gR, gD, gS = gR * stable, gD * stable, gS * stable
    g = oracle.backward(sec, target, *args, g_rgb=gR, g_depth=gD, g_sil=gS)
    for kind, nk in (("twist", 6), ("mat", 12)):
        fd = np.array([h.l_diff(renders[(kind, k, 1)], renders[(kind, k, -1)], gR, gD, gS) /
                       (2 * hstep) for k in range(nk)])
        an = g[kind]
        scale = np.max(np.abs(an))
        assert scale > 1.0
        np.testing.assert_allclose(an, fd, rtol=2e-6, atol=2e-6 * scale, err_msg=kind)


def test_pose_noise_scale():
    """The pose noise scale sqrt(sum_p n_p m_p^2) bounds each component from
    above by Cauchy-Schwarz (|g_i| <= sum_p m_p <= sqrt(P) x scale), is zero
    without upstream gradients and scales linearly with them."""
    sec, target, K = h.tiny_section()
    args = (K.astuple(), K.W, K.H)
    gR, gD, gS = _upstream((K.H, K.W), 23)
    g = oracle.backward(sec, target, *args, g_rgb=gR, g_depth=gD, g_sil=gS)
    P = K.W * K.H
    for kind in ("twist", "mat"):
        nz = g[kind + "_noise"]
        assert np.all(nz > 0)
        assert np.all(np.abs(g[kind]) <= np.sqrt(P) * nz * (1 + 1e-12))
    g2 = oracle.backward(sec, target, *args, g_rgb=2 * gR, g_depth=2 * gD, g_sil=2 * gS)
    np.testing.assert_allclose(g2["twist_noise"], 2 * g["twist_noise"], rtol=1e-12)
    z = oracle.backward(sec, target, *args, g_rgb=0 * gR)
    assert np.all(z["twist_noise"] == 0) and np.all(z["mat_noise"] == 0)


def test_attribute_gradient_finite_differences():
    sec, target, K = h.tiny_section()
    args = (K.astuple(), K.W, K.H)
    cap = 64
    base = oracle.render(sec, target, *args, list_cap=cap)
    gR, gD, gS = _upstream((K.H, K.W), 22)
    keep = (base["margin"] > 1e-6) & (base["margin_T"] > 1e-6) & (base["margin_clamp"] > 1e-6)
    gR, gD, gS = gR * keep, gD * keep, gS * keep
    g = oracle.backward(sec, target, *args, g_rgb=gR, g_depth=gD, g_sil=gS)
    rng = np.random.default_rng(4)
    touched = np.flatnonzero(np.abs(g["opacity"][0]) > 1e-3)
    picks = rng.choice(touched, 25, replace=False)
    checked = 0
    for i in picks:
        for attr, key, comp, step in (("opacity", "opacity", None, 1e-7),
                                      ("radius", "radius", None, 1e-6 * sec.radius[i]),
                                      ("colour", "colour", 1, 1e-6)):
            outs = []
            for s in (+1, -1):
                arr = getattr(sec, attr).copy()
                if comp is None:
                    arr[i] += s * step
                else:
                    arr[i, comp] += s * step
                mod = oracle.Section(sec.W, sec.H, sec.K, sec.poses, sec.depth, sec.src,
                                     arr if attr == "colour" else sec.colour,
                                     arr if attr == "opacity" else sec.opacity,
                                     arr if attr == "radius" else sec.radius)
                outs.append(oracle.render(mod, target, *args, list_cap=cap))
            if not np.all(_stable_mask(base, outs) | ~keep):
                continue
            fd = h.l_diff(outs[0], outs[1], gR, gD, gS) / (2 * step)
            an = g[key][0][i] if comp is None else g[key][0][i, comp]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, abs(an))), (attr, i)
            checked += 1
    assert checked >= 60


def test_pose_gradient_vanishes_at_optimum_of_l2():
    """For L = 1/2 |render(P) - render(P0)|^2 the gradient at P0 is zero; a
    small motion away from P0 gives a positive derivative along that motion
    (moving back lowers L)."""
    sec, target, K = h.tiny_section()
    args = (K.astuple(), K.W, K.H)
    ref = oracle.render(sec, target, *args)
    for eps, k in ((0.0, 3), (2e-4, 3), (2e-4, 4), (1e-4, 0), (1e-4, 2)):
        P = h.right_perturb(target, k, eps)
        out = oracle.render(sec, P, *args)
        g = oracle.backward(sec, P, *args, g_rgb=out["rgb"] - ref["rgb"],
                            g_depth=out["depth"] - ref["depth"], g_sil=out["sil"] - ref["sil"])
        if eps == 0.0:
            assert np.all(g["twist"] == 0.0) and np.all(g["mat"] == 0.0)
        else:
            assert g["twist"][k] > 0.0


def test_zkey_is_fp32_camera_depth():
    """The FP32 depth key agrees with the FP64 camera depth of the
    back-projected centre to a few FP32 ulps (a wrong transform entry would
    be far off), and culls centres in front of z_near = 0.1."""
    K = syn.scaled_intrinsics(96, 72)
    sec, target = h.multiview_section(K, n_views=3)
    z, ok = oracle.zkeys(sec, target, K.astuple(), K.W, K.H)
    plane = sec.W * sec.H
    zs = []
    for k in range(3):
        cen, pix = oracle.backproject(sec.depth[k], sec.K, sec.poses[k])
        R, t = target[:, :3], target[:, 3]
        zs.append(((cen - t) @ R)[:, 2])
    z64 = np.concatenate(zs)
    assert ok.all() and z64.shape == z.shape
    np.testing.assert_allclose(z, z64, rtol=8 * 2.0 ** -24)
    # push the target camera forward until part of the scene is behind z_near
    P = target.copy()
    P[:, 3] += 2.5 * P[:, 2]
    z2, ok2 = oracle.zkeys(sec, P, K.astuple(), K.W, K.H)
    assert 0 < ok2.sum() < ok2.size
    assert np.all(z2[ok2] >= np.float32(0.1)) and np.all(z2[~ok2] < np.float32(0.1))


def test_gradient_term_magnitudes_bound_the_gradients():
    """abs_* (sum over pixels of |term|) bounds |gradient| element-wise and
    equals it when every term has one sign (all upstream gradients >= 0 and
    a colour gradient is w * gC)."""
    sec, target, K = h.tiny_section()
    args = (K.astuple(), K.W, K.H)
    rng = np.random.default_rng(2)
    g = oracle.backward(sec, target, *args, g_rgb=rng.normal(0, 1, (3, K.H, K.W)),
                        g_depth=rng.normal(0, 1, (K.H, K.W)), g_sil=rng.normal(0, 1, (K.H, K.W)))
    for k in ("colour", "opacity", "radius"):
        assert np.all(g["abs_" + k][0] >= np.abs(g[k][0]) * (1 - 1e-12))
    g = oracle.backward(sec, target, *args, g_rgb=np.abs(rng.normal(0, 1, (3, K.H, K.W))))
    np.testing.assert_allclose(g["abs_colour"][0], g["colour"][0], rtol=1e-12)
