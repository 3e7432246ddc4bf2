"""Pins of the anisotropic (EWA) oracle (oracle/aniso.py) against facts that
do not come from its own formulas: the projected covariance of sampled 3D
points, the isotropic oracle on the optical axis, the symmetries of the
ellipsoid parametrisation, and finite differences of its forward."""

import numpy as np
import pytest

import oracle
from oracle import aniso
from paper_2506_02741_gb300 import synthetic as syn

from . import _helpers as h

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def _small_case(seed=3, crop=(40, 30)):
    """The 64x48 single-view section with random ellipsoids, rendered into a
    40x30 crop of the target view (same focal lengths, shifted principal
    point)."""
    sec, target, K = h.tiny_section(seed=seed)
    scale, quat = syn.random_ellipsoids(sec.radius, seed)
    W, H = crop
    Kc = (K.fx, K.fy, K.cx - (K.W - W) / 2, K.cy - (K.H - H) / 2)
    return sec, scale, quat, target, Kc, W, H


def test_projected_covariance_matches_sampled_points():
    """Sigma_2D - eps I is the covariance of the projections of points drawn
    from the ellipsoid (small ellipsoids: the linearisation error is of
    order (s/z)^2), with the ellipsoid built from scipy's rotation of the
    quaternion and the points moved to the target camera through world
    coordinates."""
    sec, target, K = h.tiny_section()
    n = sec.n
    rng = np.random.default_rng(11)
    idx = rng.choice(n, 6, replace=False)
    scale = np.zeros((n, 3)) + 1e-3
    scale[idx] = np.array([[4e-3, 1e-3, 2e-3], [1e-3, 5e-3, 1e-3], [3e-3, 3e-3, 1e-3],
                           [6e-3, 2e-3, 4e-3], [1e-3, 1e-3, 6e-3], [2e-3, 5e-3, 3e-3]])
    quat = rng.normal(size=(n, 4))
    Kt = K.astuple()
    geo = aniso._geometry(sec, scale, quat, target, Kt, K.W, K.H, aniso.EPS_LOWPASS)
    P = np.asarray(target, np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    plane = sec.W * sec.H
    N = 400_000
    for i in idx:
        src = int(sec.src[i])
        k, pix = divmod(src, plane)
        v, u = divmod(pix, sec.W)
        D = float(sec.depth.reshape(-1)[src])
        Xc = np.array([D * (u - np.float32(K.cx)) / np.float32(K.fx),
                       D * (v - np.float32(K.cy)) / np.float32(K.fy), D])
        Rq = Rotation.from_quat(np.roll(quat[i], -1)).as_matrix()   # scipy: (x, y, z, w)
        pts = Xc + (rng.normal(size=(N, 3)) * scale[i]) @ Rq.T       # view-k camera frame
        Rk, tk = sec.poses[k][:, :3], sec.poses[k][:, 3]
        world = pts @ Rk.T + tk
        cam = (world - t) @ R                                          # R^T (X - t)
        uv = np.stack([np.float32(K.fx) * cam[:, 0] / cam[:, 2] + np.float32(K.cx),
                       np.float32(K.fy) * cam[:, 1] / cam[:, 2] + np.float32(K.cy)], 1)
        cov = np.cov(uv.T)
        want = geo["S2"][i] - aniso.EPS_LOWPASS * np.eye(2)
        scl = np.sqrt(np.outer(np.diag(want), np.diag(want)))
        assert np.all(np.abs(cov - want) <= 1.5e-2 * scl), (i, cov, want)
        mean = uv.mean(0)
        sd = np.sqrt(np.diag(want) / N)
        assert np.all(np.abs(mean - [geo["uc"][i], geo["vc"][i]]) <= 6 * sd + 1e-9)


def _on_axis_section(depths, radii, fx=30.0, fy=24.0, W=33, H=25):
    """One Gaussian per view at the principal pixel (cx, cy) = (16, 12); the
    views look along the target's axis from behind it, so every centre lies
    on the target's optical axis."""
    rng = np.random.default_rng(2)
    Rt = syn.rotvec_to_matrix(np.array([0.1, -0.2, 0.05]))
    t0 = np.array([0.3, -0.1, 0.2])
    target = np.hstack([Rt, t0[:, None]])
    V = len(depths)
    cx, cy = 16.0, 12.0
    poses = []
    depth = np.zeros((V, H, W), np.float32)
    for j, (D, back) in enumerate(zip(depths, rng.uniform(0.0, 0.5, V))):
        poses.append(np.hstack([Rt, (t0 - Rt @ np.array([0.0, 0.0, back]))[:, None]]))
        depth[j, int(cy), int(cx)] = np.float32(D + back)
    src = np.array([j * W * H + int(cy) * W + int(cx) for j in range(V)], np.uint32)
    col, op, _ = syn.random_attributes(V, 4, opacity_range=(0.3, 0.9))
    K = (fx, fy, cx, cy)
    sec = oracle.Section(W, H, K, np.stack(poses), depth, src, col, op, np.asarray(radii, float))
    return sec, target, K, W, H


def test_on_axis_spheres_match_isotropic_render():
    """An ellipsoid with three equal scales r centred on the target's optical
    axis projects to the isotropic footprint (J J^T = diag(fx^2, fy^2) / z^2
    there), so without the low-pass the two oracles render the same image
    whatever the quaternion."""
    sec, target, K, W, H = _on_axis_section([1.0, 1.4, 2.2, 3.1], [0.03, 0.05, 0.04, 0.09])
    iso = oracle.render([sec], target, K, W, H)
    quat = np.random.default_rng(5).normal(size=(sec.n, 4))
    scale = np.repeat(sec.radius[:, None], 3, 1)
    an = aniso.render(sec, scale, quat, target, K, W, H, eps=0.0)
    for key in ("rgb", "depth", "sil", "T_final"):
        np.testing.assert_allclose(an[key], iso[key], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(an["n_added"], iso["n_added"])
    assert iso["n_added"].max() >= 3      # the spheres overlap and composite


def test_ellipsoid_parametrisation_symmetries():
    """The render depends on the ellipsoid only: any quaternion for a sphere;
    q, -q and 2.5 q alike; scales permuted together with the matching
    quarter turn of the axes (scipy composes the rotations)."""
    sec, scale, quat, target, K, W, H = _small_case()
    base = aniso.render(sec, scale, quat, target, K, W, H)
    for q2 in (-quat, 2.5 * quat):
        o = aniso.render(sec, scale, q2, target, K, W, H)
        np.testing.assert_allclose(o["rgb"], base["rgb"], rtol=0, atol=1e-11)
    # quarter turn about the local z axis swaps the first two scales
    rq = Rotation.from_quat(np.roll(quat, -1, axis=1)) * Rotation.from_euler("z", 90, degrees=True)
    q_turn = np.roll(rq.as_quat(), 1, axis=1)
    s_turn = scale[:, [1, 0, 2]]
    o = aniso.render(sec, s_turn, q_turn, target, K, W, H)
    np.testing.assert_allclose(o["rgb"], base["rgb"], rtol=0, atol=1e-10)
    # spheres: the quaternion does not matter
    sph = np.repeat(scale[:, :1], 3, 1)
    a = aniso.render(sec, sph, quat, target, K, W, H)
    b = aniso.render(sec, sph, np.random.default_rng(1).normal(size=quat.shape), target, K, W, H)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-11)


def _loss(sec, scale, quat, pose, K, W, H, gR, gD, gS):
    o = aniso.render(sec, scale, quat, pose, K, W, H)
    L = (gR * o["rgb"]).sum() + (gD * o["depth"]).sum() + (gS * o["sil"]).sum()
    return L, o["n_added"]


def test_gradients_match_finite_differences():
    """Analytic gradients of <g, render> against central differences of the
    oracle's forward for colour, opacity, scale, quaternion and the target
    pose twist (right perturbation); a difference whose perturbed renders
    add a different number of Gaussians somewhere (a decision flipped) is
    skipped."""
    sec, scale, quat, target, K, W, H = _small_case(crop=(24, 18))
    rng = np.random.default_rng(8)
    gR = rng.normal(size=(3, H, W))
    gD = rng.normal(size=(H, W)) * 0.1
    gS = rng.normal(size=(H, W)) * 0.2
    g = aniso.backward(sec, scale, quat, target, K, W, H, gR, gD, gS)
    L0, n0 = _loss(sec, scale, quat, target, K, W, H, gR, gD, gS)
    # Gaussians that matter: largest scale gradients
    live = np.argsort(-np.abs(g["scale"]).sum(1))[:6]
    checked = 0

    def fd(make, hstep):
        nonlocal checked
        a = _loss(*make(+hstep), gR, gD, gS)
        b = _loss(*make(-hstep), gR, gD, gS)
        if not (np.array_equal(a[1], n0) and np.array_equal(b[1], n0)):
            return None
        checked += 1
        return (a[0] - b[0]) / (2 * hstep)

    for i in live:
        for j in range(3):
            def mk(e, i=i, j=j):
                s = scale.copy()
                s[i, j] += e
                return sec, s, quat, target, K, W, H
            d = fd(mk, 1e-7 * scale[i, j])
            if d is not None:
                assert abs(d - g["scale"][i, j]) <= 1e-5 * g["abs_scale"][i, j] + 1e-6 * abs(d), (i, j, d, g["scale"][i, j])
        for j in range(4):
            def mk(e, i=i, j=j):
                q = quat.copy()
                q[i, j] += e
                return sec, scale, q, target, K, W, H
            d = fd(mk, 1e-7)
            if d is not None:
                assert abs(d - g["quat"][i, j]) <= 1e-5 * g["abs_quat"][i, j] + 1e-6 * abs(d), (i, j, d, g["quat"][i, j])

        def mko(e, i=i):
            s2 = _with(sec, opacity=sec.opacity.copy())
            s2.opacity[i] += e
            return s2, scale, quat, target, K, W, H
        d = fd(mko, 1e-7)
        if d is not None:
            assert abs(d - g["opacity"][i]) <= 1e-5 * g["abs_opacity"][i] + 1e-6 * abs(d)
        for j in range(3):
            def mkc(e, i=i, j=j):
                s2 = _with(sec, colour=sec.colour.copy())
                s2.colour[i, j] += e
                return s2, scale, quat, target, K, W, H
            d = fd(mkc, 1e-3)
            if d is not None:
                assert abs(d - g["colour"][i, j]) <= 1e-8 * (1 + abs(d))
    for k in range(6):
        d = fd(lambda e, k=k: (sec, scale, quat, h.right_perturb(target, k, e), K, W, H), 1e-7)
        if d is not None:
            assert abs(d - g["twist"][k]) <= 1e-5 * g["abs_twist"][k] + 1e-6 * abs(d), (k, d, g["twist"][k])
    assert checked >= 40


def _with(sec, **kw):
    import dataclasses
    return dataclasses.replace(sec, **kw)


def test_magnitudes_bound_the_gradients():
    sec, scale, quat, target, K, W, H = _small_case()
    rng = np.random.default_rng(4)
    g = aniso.backward(sec, scale, quat, target, K, W, H, rng.normal(size=(3, H, W)),
                       rng.normal(size=(H, W)), None)
    for k in ("colour", "opacity", "scale", "quat", "x", "twist", "mat"):
        assert np.all(np.abs(g[k]) <= g["abs_" + k] * (1 + 1e-9) + 1e-300), k
    assert np.abs(g["scale"]).max() > 0 and np.abs(g["quat"]).max() > 0


def test_invalid_shapes_are_not_rendered():
    """Gaussians with a non-positive or non-finite scale or a zero
    quaternion are left out: the render equals that of the section without
    them (their opacity set below the 1/255 skip)."""
    sec, scale, quat, target, K, W, H = _small_case()
    rng = np.random.default_rng(9)
    bad = rng.choice(sec.n, 40, replace=False)
    s2, q2 = scale.copy(), quat.copy()
    s2[bad[:10], 0] = 0.0
    s2[bad[10:20], 1] = -1e-3
    s2[bad[20:30], 2] = np.nan
    q2[bad[30:]] = 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        got = aniso.render(sec, s2, q2, target, K, W, H)
    op = sec.opacity.copy()
    op[bad] = 0.0
    import dataclasses
    ref = aniso.render(dataclasses.replace(sec, opacity=op), scale, quat, target, K, W, H)
    np.testing.assert_array_equal(got["rgb"], ref["rgb"])
    np.testing.assert_array_equal(got["n_added"], ref["n_added"])
