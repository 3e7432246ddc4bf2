"""Loss inputs through the C ABI against the oracle: the visibility check of
Sec. 3.3 (bit-exact masks: both sides decide in FP64 with the same operation
order) and the masked L1 terms of Eq. 1 / Eq. 2 (gradients exact, loss to FP64
summation order)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _room(K, Kv, idx=(0, 10, 20), cur=29):
    """Current frame (intrinsics K) and three section views (intrinsics Kv)
    of the seeded room along the seeded trajectory."""
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(cur + 1)
    fc = syn.render_frames(room, K, [path[cur]])
    fv = syn.render_frames(room, Kv, [path[i] for i in idx])
    views = [(fv.depth[k], Kv.astuple(), path[i]) for k, i in enumerate(idx)]
    return fc.depth[0], path[cur], views


CASES = {
    "tiny_64x48": (syn.TINY, syn.TINY),
    "ragged_37x23_views_50x30": (syn.scaled_intrinsics(37, 23), syn.scaled_intrinsics(50, 30)),
    "vga_640x480": (syn.VGA, syn.VGA),
}


@pytest.mark.parametrize("case", list(CASES))
def test_visibility_bit_exact(dev, case):
    K, Kv = CASES[case]
    depth, pose, views = _room(K, Kv)
    depth = depth.copy()
    depth[0, :3] = 0.0                      # invalid pixels of the current frame
    depth[-1, -1] = np.nan
    views[1][0][2, :] = 0.0                 # an invalid row in one view
    want = oracle.visibility(depth, K.astuple(), pose, views)
    assert 0.02 < want.mean() < 0.999
    gv = [(torch.from_numpy(np.ascontiguousarray(d)).to(dev), k, api.pose12(p, dev))
          for d, k, p in views]
    got = api.visibility(torch.from_numpy(depth).to(dev), K.astuple(), api.pose12(pose, dev), gv)
    assert np.array_equal(got.cpu().numpy().astype(bool), want)
    # one view at a time reproduces each member of the union
    for v, g in zip(views, gv):
        w1 = oracle.visibility(depth, K.astuple(), pose, [v])
        g1 = api.visibility(torch.from_numpy(depth).to(dev), K.astuple(), api.pose12(pose, dev), [g])
        assert np.array_equal(g1.cpu().numpy().astype(bool), w1)


def _images(rng, H, W):
    rgb = rng.random((3, H, W)).astype(np.float32)
    obs = rng.random((3, H, W)).astype(np.float32)
    dep = (0.5 + 3 * rng.random((H, W))).astype(np.float32)
    od = (0.5 + 3 * rng.random((H, W))).astype(np.float32)
    sil = rng.random((H, W)).astype(np.float32)
    sil[rng.random((H, W)) < 0.3] = np.float32(0.99)       # exactly at the threshold
    od[rng.random((H, W)) < 0.05] = 0.0
    od[rng.random((H, W)) < 0.02] = np.nan
    obs[:, 1, 1] = rgb[:, 1, 1]                             # zero residuals
    od[2, 2] = dep[2, 2]
    vis = rng.random((H, W)) < 0.8
    return rgb, dep, sil, obs, od, vis


@pytest.mark.parametrize("H, W", [(23, 37), (480, 640), (1, 1)])
@pytest.mark.parametrize("form", ["eq1_visible", "eq1", "eq2"])
def test_masked_l1_matches_oracle(dev, H, W, form):
    rng = np.random.default_rng(H * 1000 + W)
    if H < 3:
        rgb, dep, sil, obs, od, vis = (a[..., :H, :W] for a in _images(rng, 3, 3))
        rgb, dep, sil, obs, od, vis = (np.ascontiguousarray(a) for a in (rgb, dep, sil, obs, od, vis))
    else:
        rgb, dep, sil, obs, od, vis = _images(rng, H, W)
    kw = {"eq1_visible": dict(w_rgb=0.5, w_depth=0.025, sil_min=0.99, rgb_needs_depth=True),
          "eq1": dict(w_rgb=0.5, w_depth=0.025, sil_min=0.99, rgb_needs_depth=True),
          "eq2": dict(w_rgb=0.8, w_depth=1.0, sil_min=-1.0, rgb_needs_depth=False)}[form]
    v = vis if form == "eq1_visible" else None
    L, gr, gd = oracle.masked_l1(rgb, dep, sil, obs, od, visible=v, **kw)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    R = api.Renderer()
    loss, d_rgb, d_depth = R.masked_l1(t(rgb), t(dep), t(sil) if kw["sil_min"] >= 0 else None,
                                       t(obs), t(od), visible=None if v is None else t(v.astype(np.uint8)),
                                       **kw)
    torch.cuda.synchronize()
    assert np.array_equal(d_rgb.cpu().numpy(), gr.astype(np.float32))
    assert np.array_equal(d_depth.cpu().numpy(), gd.astype(np.float32))
    assert float(loss.item()) == pytest.approx(L, rel=1e-12, abs=1e-300)


def test_loss_inputs_reject_bad_arguments(dev):
    R = api.Renderer()
    z = torch.zeros(4, 5, device=dev)
    z3 = torch.zeros(3, 4, 5, device=dev)
    with pytest.raises(api.L.VTError):
        R.masked_l1(z3, z, None, z3, z, 0.5, 0.025, sil_min=0.99)     # needs the silhouette
    p = api.pose12(syn.identity_pose(), dev)
    with pytest.raises(ValueError):
        api.visibility(z, syn.TINY.astuple(), p, [])
    with pytest.raises(api.L.VTError):
        api.visibility(z, (0.0, 1.0, 2.0, 2.0), p, [(z, syn.TINY.astuple(), p)])


@pytest.mark.parametrize("lr_rot", [4e-4, 0.0])
def test_pose_adam_matches_reference(dev, lr_rot):
    """Five Adam steps on the pose against the float64 reference (lr_rot = 0
    takes the small-angle branch of the exponential); the gradient buffer is
    zeroed after each step."""
    from oracle import optim as op
    rng = np.random.default_rng(11)
    P = syn.perturb_pose(syn.identity_pose(), rng, 0.3, 20.0)
    lr = [2e-3] * 3 + [lr_rot] * 3
    pose = api.pose12(P, dev)
    state = torch.zeros(15, dtype=torch.float64, device=dev)
    d_tw = torch.zeros(6, dtype=torch.float64, device=dev)
    m, v, t = np.zeros(6), np.zeros(6), 0.0
    for _ in range(5):
        g = rng.normal(0, 1, 6) * np.array([1, 10, 0.1, 1, 5, 0.5])
        d_tw.copy_(torch.from_numpy(g))
        api.pose_adam(pose, d_tw, state, lr)
        P, m, v, t = op.adam_pose_step(P, g, m, v, t, lr)
        torch.cuda.synchronize()
        assert not d_tw.any()
        np.testing.assert_allclose(api.matrix_of(pose), P, rtol=1e-12, atol=1e-14)
        st = state.cpu().numpy()
        np.testing.assert_allclose(st[:6], m, rtol=1e-13)
        np.testing.assert_allclose(st[6:12], v, rtol=1e-13)
        assert st[12] == t


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_attr_adam_matches_reference(dev, prec):
    """Three fused Adam steps on a section's attributes against the float64
    reference (FP32 arithmetic: 1e-5 relative on the parameters); storage
    written in the section's precision; gradients zeroed."""
    from oracle import optim as op
    rng = np.random.default_rng(5)
    n = 1000                                    # not a multiple of the block size
    dt = torch.float16 if prec == "f16" else torch.float32
    col = rng.random((n, 3)).astype(np.float32)
    opa = (0.05 + 0.9 * rng.random(n)).astype(np.float32)
    rad = (0.002 + 0.01 * rng.random(n)).astype(np.float32)
    sec = api.Section(poses=torch.zeros(1, 12, dtype=torch.float64, device=dev),
                      depth=torch.ones(1, 1, n, device=dev), K=(1.0, 1.0, 0.0, 0.0),
                      src=torch.arange(n, dtype=torch.int32, device=dev),
                      colour=torch.from_numpy(col).to(dev, dt),
                      opacity=torch.from_numpy(opa).to(dev, dt),
                      radius=torch.from_numpy(rad).to(dev, dt))
    theta = np.stack([col[:, 0], col[:, 1], col[:, 2], np.log(opa / (1 - opa)), np.log(rad)])
    th_d = torch.from_numpy(theta.astype(np.float32)).to(dev)
    m_d, v_d = torch.zeros(5, n, device=dev), torch.zeros(5, n, device=dev)
    st = torch.zeros(3, dtype=torch.float64, device=dev)
    th, m, v, t = theta.astype(np.float32).astype(np.float64), np.zeros((5, n)), np.zeros((5, n)), 0.0
    lr = [0.0025] * 3 + [0.05, 0.005]
    for _ in range(3):
        dc = rng.normal(0, 1e-3, (n, 3)).astype(np.float32)
        do = rng.normal(0, 1e-3, n).astype(np.float32)
        dr = rng.normal(0, 1e-1, n).astype(np.float32)
        gdc, gdo, gdr = (torch.from_numpy(a).to(dev) for a in (dc, do, dr))
        api.attr_adam(sec, th_d, m_d, v_d, st, gdc, gdo, gdr, lr)
        th, m, v, t, c_ref, o_ref, r_ref = op.attr_adam_step(th, m, v, t, dc, do, dr, lr)
        torch.cuda.synchronize()
        assert not gdc.any() and not gdo.any() and not gdr.any()
        np.testing.assert_allclose(th_d.cpu().numpy(), th, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(m_d.cpu().numpy(), m, rtol=1e-4, atol=1e-12)
        np.testing.assert_allclose(v_d.cpu().numpy(), v, rtol=1e-4, atol=1e-16)
        tol = 1e-3 if prec == "f16" else 1e-5
        np.testing.assert_allclose(sec.colour.float().cpu().numpy(), c_ref, rtol=tol, atol=1e-6)
        np.testing.assert_allclose(sec.opacity.float().cpu().numpy(), o_ref, rtol=tol)
        np.testing.assert_allclose(sec.radius.float().cpu().numpy(), r_ref, rtol=tol)
        assert st[0].item() == t


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_adam_init_from_storage(dev, prec):
    """vt_adam_init: theta = (c, logit o, log r) of the stored values (o
    clamped to [1e-4, 1 - 1e-4], so o = 1 and o = 0 stay finite), moments
    and step zeroed; for ellipsoids (log s, q)."""
    rng = np.random.default_rng(8)
    n = 777
    dt = torch.float16 if prec == "f16" else torch.float32
    col = rng.random((n, 3)).astype(np.float32)
    opa = rng.random(n).astype(np.float32)
    opa[:3] = [0.0, 1.0, 0.5]
    rad = (0.002 + 0.01 * rng.random(n)).astype(np.float32)
    sc = rng.uniform(0.002, 0.02, (n, 3)).astype(np.float32)
    qt = rng.normal(size=(n, 4)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    sec = api.Section(poses=torch.zeros(1, 12, dtype=torch.float64, device=dev),
                      depth=torch.ones(1, 1, n, device=dev), K=(1.0, 1.0, 0.0, 0.0),
                      src=torch.arange(n, dtype=torch.int32, device=dev), colour=t(col),
                      opacity=t(opa), radius=t(rad), scale=t(sc), rot=t(qt))
    stored = lambda x: x.float().cpu().numpy().astype(np.float64)
    th, m, v, st = api.adam_init(sec)
    # the clamp bounds and 1 - o in FP32, as the kernel forms them (1 - o is
    # exact there, Sterbenz), the rest in FP64
    o32 = np.clip(sec.opacity.float().cpu().numpy(), np.float32(1e-4), np.float32(1 - 1e-4))
    o = o32.astype(np.float64)
    want = np.stack([*stored(sec.colour).T, np.log(o / (np.float32(1) - o32)),
                     np.log(stored(sec.radius))])
    np.testing.assert_allclose(th.cpu().numpy(), want, rtol=2e-6, atol=2e-6)
    assert not m.any() and not v.any() and not st.any()
    th, m, v, st = api.adam_init(sec, shape=True)
    want = np.concatenate([np.log(stored(sec.scale)).T, stored(sec.rot).T])
    np.testing.assert_allclose(th.cpu().numpy(), want, rtol=2e-6, atol=2e-6)
    assert th.shape == (7, n) and not m.any() and not v.any()


def test_mapper_reduces_loss(dev):
    """A few mapping iterations (render, fused loss, attribute backward, fused
    Adam) on a perturbed section lower the Eq. 2 L1 loss."""
    from paper_2506_02741_gb300.mapping import SectionMapper
    K = syn.scaled_intrinsics(160, 120)
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(15)
    keys = [path[i] for i in (0, 5, 10)]
    fr = syn.render_frames(room, K, keys)
    depth = torch.from_numpy(fr.depth).to(dev)
    rgb = torch.from_numpy(fr.rgb).to(dev)
    sec = api.Section.from_rgbd(depth, rgb, K.astuple(), np.stack(keys))
    g = torch.Generator(device=dev).manual_seed(0)
    sec.colour.copy_((sec.colour + 0.2 * torch.rand(sec.colour.shape, generator=g, device=dev)).clamp(0, 1))
    R = api.Renderer()
    mp = SectionMapper(R, sec, rgb)
    losses = [float(mp.step(i % 3).cpu().sum()) for i in range(30)]
    assert losses[-1] < 0.8 * losses[0]


@pytest.mark.parametrize("K", [syn.scaled_intrinsics(37, 23), syn.VGA, syn.scaled_intrinsics(4, 3)])
def test_ssim_matches_reference(dev, K):
    """SSIM term of Eq. 2 against the float64 reference on a rendered frame
    and its neighbour (smooth texture, edges, borders): loss to 1e-6
    relative; gradient to 1e-4 relative per tensor, and per element within
    1e-4 max(|ref|, 1e-3 max|ref|) + 1e-4 m (m: componentwise magnitude of
    the window sum, the same model as the attribute gradients); the gradient
    accumulates into d_rgb."""
    from oracle import ssim as os_
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(3)
    fr = syn.render_frames(room, K, [path[0], path[2]])
    x, y = fr.rgb[1], fr.rgb[0]
    L, g, mag = os_.ssim_loss(x, y, 0.2, magnitude=True)
    R = api.Renderer()
    xd, yd = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    d = torch.zeros(3, K.H, K.W, device=dev)
    loss, d = R.ssim(xd, yd, 0.2, d_rgb=d)
    torch.cuda.synchronize()
    assert float(loss.item()) == pytest.approx(L, rel=1e-6, abs=1e-9)
    got = d.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - g) <= 1e-4 * np.linalg.norm(g)
    bound = 1e-4 * np.maximum(np.abs(g), 1e-3 * np.abs(g).max()) + 1e-4 * mag
    assert np.all(np.abs(got - g) <= bound)
    R.ssim(xd, yd, 0.2, d_rgb=d)                 # accumulates: twice the gradient
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), (2 * got).astype(np.float32))
