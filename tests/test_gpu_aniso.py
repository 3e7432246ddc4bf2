"""Parity of the ellipsoid (anisotropic, EWA footprint) path through the C ABI
with the FP64 oracle of oracle/aniso.py.

Forward: FP32 within 2e-5 relative (floor 1 for colour / silhouette, 4 m
for depth) at every pixel, against the oracle composited along the GPU's own
per-pixel lists, which must be the definition's up to decisions within 1e-4
(relative) of their inclusion thresholds or 2e-4 of the termination
threshold.  The conic is formed in FP32 from J, M, R(q) and s (about
ten rounded products and sums per entry before the 2 x 2 inverse), so q
carries a few 1e-7 relative error where the sphere form has one or two
roundings; alpha = o exp(-q/2) turns a relative error d of q into q d / 2
<= 4.5 d of alpha, and the composite adds the transmittance's rounding:
twice the sphere bound covers it.  Gradients within 1e-4 relative per tensor
(L2) and per element, plus 1e-4 of each element's componentwise magnitude.
"""

import numpy as np
import pytest
import torch

from oracle import aniso
from paper_2506_02741_gb300 import _lib as L
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G
from tests import _helpers as h

pytestmark = pytest.mark.gpu

FWD_TOL = 2e-5
TAU_INCL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _q32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _case(name):
    if name == "tiny":
        sec, target, K = h.tiny_section()
        Kt, W, H, seed = K.astuple(), K.W, K.H, 21
    elif name == "qqvga_2views":
        K = syn.scaled_intrinsics(160, 120)
        sec, target = h.multiview_section(K, n_views=2)
        Kt, W, H, seed = K.astuple(), K.W, K.H, 22
    else:   # ragged image, three views
        K = syn.scaled_intrinsics(200, 130)
        sec, target = h.multiview_section(K, n_views=3, seed=9)
        Kt, W, H, seed = K.astuple(), 203, 131, 23
    sec = G.quantise(sec)
    scale, quat = syn.random_ellipsoids(sec.radius, seed)
    return sec, _q32(scale), _q32(quat), target, Kt, W, H


def _device(sec, scale, quat):
    return G.to_device(sec).with_ellipsoids(torch.from_numpy(scale), torch.from_numpy(quat))


CASES = ["tiny", "qqvga_2views", "ragged_3views"]


def _lists_ref(R, sec, scale, quat, target, K, W, H, name, keep=False):
    """The oracle composited along the last render's per-pixel lists, after
    checking them against the definition."""
    ids, cnt = G.gpu_lists(R, W, H)
    ref = aniso.render_lists(sec, scale, quat, target, K, W, H, ids, cnt, tau_incl=TAU_INCL,
                             keep=keep)
    G.check_decisions(ref, name)
    return ref


@pytest.mark.parametrize("case", CASES)
def test_ellipsoid_forward_parity(dev, case):
    sec, scale, quat, target, K, W, H = _case(case)
    R = api.Renderer()
    out = R.render([_device(sec, scale, quat)], api.pose12(target, dev), K, W, H, checked=True)
    torch.cuda.synchronize()
    ref = _lists_ref(R, sec, scale, quat, target, K, W, H, "ellipsoids_" + case)
    assert ref["n_added"].mean() > 5
    G.assert_forward_close(out, ref, tol=FWD_TOL)


@pytest.mark.parametrize("case", CASES)
def test_ellipsoid_gradients(dev, case):
    """Colour, opacity, scale, quaternion and target-pose gradients against
    the oracle's chain rule along the GPU's own per-pixel lists."""
    sec, scale, quat, target, K, W, H = _case(case)
    R = api.Renderer()
    dsec = _device(sec, scale, quat)
    R.render([dsec], api.pose12(target, dev), K, W, H, checked=True)
    ref = _lists_ref(R, sec, scale, quat, target, K, W, H, "ellipsoid_grads_" + case, keep=True)
    rng = np.random.default_rng(31)
    gR = rng.normal(0, 1, (3, H, W)).astype(np.float32)
    gD = rng.normal(0, 1, (H, W)).astype(np.float32)
    gS = rng.normal(0, 1, (H, W)).astype(np.float32)
    want = aniso.backward(sec, scale, quat, target, K, W, H, gR, gD, gS, fwd=ref)
    n = sec.n
    z = lambda *s: torch.zeros(*s, device=dev)
    grads = [(z(n, 3), z(n), None, z(n, 3), z(n, 4))]
    t = lambda a: torch.from_numpy(a).to(dev)
    dtw, dmat = R.backward(t(gR), t(gD), t(gS), attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    got = dict(colour=grads[0][0], opacity=grads[0][1], scale=grads[0][3], quat=grads[0][4])
    for k, v in got.items():
        G.assert_grad_close(v.cpu().numpy(), want[k], name=k, abs_ref=want["abs_" + k])
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", abs_ref=want["abs_twist"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", abs_ref=want["abs_mat"])
    assert np.abs(want["scale"]).max() > 0 and np.abs(want["twist"]).max() > 0


def test_ellipsoid_replay_matches_lists(dev):
    """Without per-pixel lists (memory budget) the tile replay gives the same
    forward and the same gradients up to the order of float atomics."""
    sec, scale, quat, target, K, W, H = _case("qqvga_2views")
    dsec = _device(sec, scale, quat)
    res = []
    for budget in (None, 1):
        R = api.Renderer()
        if budget is not None:
            R.set_budget(budget)
        out = R.render([dsec], api.pose12(target, dev), K, W, H, checked=True)
        assert R.used_lists == (budget is None)
        rng = np.random.default_rng(3)
        gR = torch.from_numpy(rng.normal(0, 1, (3, H, W)).astype(np.float32)).to(dev)
        gD = torch.from_numpy(rng.normal(0, 1, (H, W)).astype(np.float32)).to(dev)
        n = sec.n
        gr = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), None,
               torch.zeros(n, 3, device=dev), torch.zeros(n, 4, device=dev))]
        tw, mat = R.backward(gR, gD, None, attr_grads=gr, pose_grad=True)
        torch.cuda.synchronize()
        res.append((out, gr[0], tw, mat))
    (o1, g1, tw1, m1), (o2, g2, tw2, m2) = res
    for a, b in zip(o1, o2):
        assert torch.equal(a, b)
    for a, b in zip(g1, g2):
        if a is None:
            continue
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))
    torch.testing.assert_close(tw1, tw2, rtol=1e-4, atol=1e-5 * float(tw2.abs().max()))


def test_ellipsoid_argument_errors(dev):
    sec, scale, quat, target, K, W, H = _case("tiny")
    ell = _device(sec, scale, quat)
    sph = G.to_device(sec)
    R = api.Renderer()
    with pytest.raises(L.VTError):
        R.render([ell, sph], api.pose12(target, dev), K, W, H)
    R.render([ell], api.pose12(target, dev), K, W, H)
    g = torch.zeros(W * H * 3, device=dev).reshape(3, H, W)
    vt = torch.zeros(1, 6, dtype=torch.float64, device=dev)
    with pytest.raises(L.VTError):
        R.backward(g, None, None, view_grads=[(vt, None)])
    with pytest.raises(ValueError):
        api.Section(ell.poses, ell.depth, ell.K, ell.src, ell.colour, ell.opacity, ell.radius,
                    scale=ell.scale).validate()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_shape_adam_matches_reference(dev, prec):
    """Three Adam steps on the ellipsoid shape against the float64 reference
    (FP32 arithmetic: 1e-5 relative on the parameters); storage written in
    the section's precision; gradients zeroed; its own step counter."""
    from oracle import optim as op
    rng = np.random.default_rng(6)
    n = 777
    dt = torch.float16 if prec == "f16" else torch.float32
    sc = rng.uniform(0.002, 0.02, (n, 3)).astype(np.float32)
    qt = rng.normal(size=(n, 4)).astype(np.float32)
    ones = torch.ones(n, device=dev, dtype=dt)
    sec = api.Section(poses=torch.zeros(1, 12, dtype=torch.float64, device=dev),
                      depth=torch.ones(1, 1, n, device=dev), K=(1.0, 1.0, 0.0, 0.0),
                      src=torch.arange(n, dtype=torch.int32, device=dev),
                      colour=torch.zeros(n, 3, device=dev, dtype=dt), opacity=ones * 0.5,
                      radius=ones * 0.01, scale=torch.from_numpy(sc).to(dev, dt),
                      rot=torch.from_numpy(qt).to(dev, dt))
    th = np.ascontiguousarray(np.concatenate([np.log(sc).T, qt.T]), np.float32)
    th_d = torch.from_numpy(th).to(dev)
    m_d, v_d = torch.zeros(7, n, device=dev), torch.zeros(7, n, device=dev)
    st = torch.zeros(3, dtype=torch.float64, device=dev)
    th64, m, v, t = th.astype(np.float64), np.zeros((7, n)), np.zeros((7, n)), 0.0
    for _ in range(3):
        ds = rng.normal(0, 1e-2, (n, 3)).astype(np.float32)
        dq = rng.normal(0, 1e-3, (n, 4)).astype(np.float32)
        gds, gdq = torch.from_numpy(ds).to(dev), torch.from_numpy(dq).to(dev)
        api.shape_adam(sec, th_d, m_d, v_d, st, gds, gdq, 0.005, 0.001)
        th64, m, v, t, s_ref, q_ref = op.shape_adam_step(th64, m, v, t, ds, dq, 0.005, 0.001)
        torch.cuda.synchronize()
        assert not gds.any() and not gdq.any()
        np.testing.assert_allclose(th_d.cpu().numpy(), th64, rtol=1e-5, atol=1e-6)
        # m sums terms of both signs: its FP32 rounding is relative to the terms
        np.testing.assert_allclose(m_d.cpu().numpy(), m, rtol=1e-4, atol=1e-6 * np.abs(m).max())
        tol = 1e-3 if prec == "f16" else 1e-5
        np.testing.assert_allclose(sec.scale.float().cpu().numpy(), s_ref, rtol=tol)
        np.testing.assert_allclose(sec.rot.float().cpu().numpy(), q_ref, rtol=tol, atol=1e-6)
        assert st[0].item() == t


def test_ellipsoid_mapper_reduces_loss(dev):
    """Mapping iterations on an ellipsoid section (render, Eq. 2 L1 + SSIM,
    attribute backward, colour / opacity and shape Adam steps) lower the loss
    and move the scales and rotations."""
    from paper_2506_02741_gb300.mapping import SectionMapper
    K = syn.scaled_intrinsics(160, 120)
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(15)
    keys = [path[i] for i in (0, 5, 10)]
    fr = syn.render_frames(room, K, keys)
    depth = torch.from_numpy(fr.depth).to(dev)
    rgb = torch.from_numpy(fr.rgb).to(dev)
    sec = api.Section.from_rgbd(depth, rgb, K.astuple(), np.stack(keys))
    scale, quat = syn.random_ellipsoids(sec.radius.cpu().numpy(), 2, spread=0.6)
    sec = sec.with_ellipsoids(scale, quat)
    s0, q0 = sec.scale.clone(), sec.rot.clone()
    R = api.Renderer()
    mp = SectionMapper(R, sec, rgb)
    losses = [float(mp.step(i % 3).cpu().sum()) for i in range(30)]
    assert losses[-1] < 0.8 * losses[0], losses
    assert not torch.equal(s0, sec.scale) and not torch.equal(q0, sec.rot)


def test_ellipsoid_fp16_storage_and_invalid_shapes(dev):
    """FP16 storage (both sides read the same rounded attributes, FP32
    arithmetic), with some Gaussians whose scales are zero, negative or NaN
    or whose quaternion is zero: those are not rendered on either side."""
    sec, scale, quat, target, K, W, H = _case("qqvga_2views")
    f16 = lambda a: np.asarray(a, np.float16).astype(np.float64)
    sec = G.quantise(sec, "f16")
    scale, quat = f16(scale), f16(quat)
    rng = np.random.default_rng(12)
    bad = rng.choice(sec.n, 60, replace=False)
    scale[bad[:15], 0] = 0.0
    scale[bad[15:30], 1] = -1e-3
    scale[bad[30:45], 2] = np.nan
    quat[bad[45:]] = 0.0
    dsec = G.to_device(sec, "f16").with_ellipsoids(torch.from_numpy(scale),
                                                   torch.from_numpy(quat))
    R = api.Renderer()
    out = R.render([dsec], api.pose12(target, dev), K, W, H, checked=True)
    torch.cuda.synchronize()
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = _lists_ref(R, sec, scale, quat, target, K, W, H, "ellipsoids_fp16_invalid")
    G.assert_forward_close(out, ref, tol=FWD_TOL)


def test_thin_ellipsoids(dev):
    """Needle- and disc-shaped ellipsoids (axis ratios up to ~30): forward
    and pose gradient against the oracle."""
    sec, _, _, target, K, W, H = _case("tiny")
    rng = np.random.default_rng(13)
    r = sec.radius
    scale = np.stack([r * 3.0, r * 0.1, r * rng.choice([0.1, 3.0], sec.n)], 1)
    quat = _q32(rng.normal(size=(sec.n, 4)))
    scale = _q32(scale)
    R = api.Renderer()
    R.render([_device(sec, scale, quat)], api.pose12(target, dev), K, W, H, checked=True)
    out = R.render([_device(sec, scale, quat)], api.pose12(target, dev), K, W, H)
    ref = _lists_ref(R, sec, scale, quat, target, K, W, H, "thin_ellipsoids", keep=True)
    G.assert_forward_close(out, ref, tol=FWD_TOL)
    gR = rng.normal(0, 1, (3, H, W)).astype(np.float32)
    want = aniso.backward(sec, scale, quat, target, K, W, H, gR, fwd=ref)
    dtw, _ = R.backward(torch.from_numpy(gR).to(dev), None, None, pose_grad=True)
    torch.cuda.synchronize()
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", abs_ref=want["abs_twist"])
