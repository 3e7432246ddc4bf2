"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP32 forward within 1e-5 relative (floor 1 for
colour/silhouette, 4 m for depth); gradients within 1e-4 relative (per-tensor
L2 and per element with a floor of 1e-3 of the largest magnitude).  Integer
and index results (section ids, depth keys, per-pixel counts, list order) are
bit-exact.  Every pixel is checked: the GPU's per-pixel lists of added
Gaussians must be the definition's up to decisions that lie within the
rounding of FP32 of their thresholds (q <= 9, ahat >= 1/255 within 1e-5
relative; T' < 1e-4 within 2e-4), which the oracle verifies; the oracle then
composites along those lists in FP64 and its images and gradients are
compared at every pixel.  The number of pixels with such a decision is
printed per case.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G
from tests import _helpers as h

pytestmark = pytest.mark.gpu

IDENT = syn.identity_pose()


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _render(osecs, target, K, W, H, prec="f32", R=None):
    dsecs = [G.to_device(s, prec) for s in osecs]
    R = R or api.Renderer()
    out = R.render(dsecs, api.pose12(target), K, W, H, checked=True)
    torch.cuda.synchronize()
    return R, dsecs, out


def _upstream(shape, seed, mask):
    H, W = shape
    rng = np.random.default_rng(seed)
    gR = (rng.normal(0, 1, (3, H, W)) * mask).astype(np.float32)
    gD = (rng.normal(0, 1, (H, W)) * mask).astype(np.float32)
    gS = (rng.normal(0, 1, (H, W)) * mask).astype(np.float32)
    return gR, gD, gS


def _cases():
    return {
        "tiny": lambda: (lambda s, t, K: ([G.quantise(s)], t, K.astuple(), K.W, K.H))(*h.tiny_section()),
        "qqvga_2views": lambda: (lambda K: (lambda s, t: ([G.quantise(s)], t, K.astuple(), K.W, K.H))(
            *h.multiview_section(K, n_views=2)))(syn.scaled_intrinsics(160, 120)),
        "ragged_3views": lambda: (lambda K: (lambda s, t: ([G.quantise(s)], t, K.astuple(), 203, 131))(
            *h.multiview_section(K, n_views=3, seed=9)))(syn.scaled_intrinsics(200, 130)),
        # a view seen from its own pose: the back wall gives long runs of equal
        # depth keys, ordered by id (the sort's full-key path)
        "own_view": lambda: (lambda s, t, K: ([G.quantise(s)], IDENT, K.astuple(), K.W, K.H))(
            *h.tiny_section(randomise=False)),
    }


# ---------------------------------------------------------------------------


def test_section_init_bitexact(dev):
    room, fr, _ = syn.tiny_workload()
    K = syn.TINY
    depth = fr.depth.copy()
    depth[0, 3, 4] = 0.0
    depth[0, 10, 11] = np.nan
    depth[0, 20, 21] = -2.0
    ref = oracle.section_init(depth, fr.rgb, K.astuple(), np.stack(fr.poses))
    for prec in ("f32", "f16"):
        s = api.Section.from_rgbd(torch.from_numpy(depth).to(dev), torch.from_numpy(fr.rgb).to(dev),
                                  K.astuple(), np.stack(fr.poses), precision=prec)
        assert s.n == ref.n
        np.testing.assert_array_equal(s.src.cpu().numpy().view(np.uint32), ref.src)
        dt = np.float16 if prec == "f16" else np.float32
        np.testing.assert_array_equal(s.colour.cpu().numpy(), ref.colour.astype(np.float32).astype(dt))
        np.testing.assert_array_equal(s.opacity.cpu().numpy(), np.full(ref.n, 0.9, np.float32).astype(dt))
        r32 = depth.reshape(-1)[ref.src] / np.float32(K.fx)     # IEEE FP32 division
        np.testing.assert_array_equal(s.radius.cpu().numpy(), r32.astype(dt))


def test_section_complement(dev):
    """Complement initialisation against the oracle (bit-exact outputs), and
    the completed section's render against the oracle's render of the same
    Gaussians."""
    K = syn.TINY
    path = syn.trajectory(12)
    room = syn.make_room(syn.SCENE_SEED)
    f0 = syn.render_frames(room, K, [path[0]])
    f1 = syn.render_frames(room, K, [path[11]])
    d1 = f1.depth[0].copy()
    d1[1, 1] = np.nan
    for prec in ("f32", "f16"):
        sec = api.Section.from_rgbd(torch.from_numpy(f0.depth).to(dev),
                                    torch.from_numpy(f0.rgb).to(dev), K.astuple(),
                                    np.stack([path[0]]), precision=prec)
        R = api.Renderer()
        _, _, sil = R.render([sec], api.pose12(path[11], dev), K.astuple(), K.W, K.H, checked=True)
        sil_h = sil.cpu().numpy()
        src, col, op, rad = oracle.section_complement(d1, f1.rgb[0], sil_h, K.astuple(), view=1)
        assert 5 < src.size < K.W * K.H // 2
        both = sec.append_view(torch.from_numpy(d1).to(dev), torch.from_numpy(f1.rgb[0]).to(dev),
                               path[11], sil)
        n0 = sec.n
        dt = np.float16 if prec == "f16" else np.float32
        assert both.n == n0 + src.size and both.n_views == 2
        np.testing.assert_array_equal(both.src[n0:].cpu().numpy().view(np.uint32), src)
        np.testing.assert_array_equal(both.colour[n0:].cpu().numpy(), col.astype(np.float32).astype(dt))
        np.testing.assert_array_equal(both.opacity[n0:].cpu().numpy(), op.astype(np.float32).astype(dt))
        r32 = d1.reshape(-1)[src - K.W * K.H] / np.float32(K.fx)
        np.testing.assert_array_equal(both.radius[n0:].cpu().numpy(), r32.astype(dt))
        if prec == "f32":
            osec = G.quantise(oracle.Section(K.W, K.H, K.astuple(), np.stack([path[0], path[11]]),
                                             np.stack([f0.depth[0], d1]),
                                             both.src.cpu().numpy().view(np.uint32),
                                             both.colour.cpu().numpy().astype(np.float64),
                                             both.opacity.cpu().numpy().astype(np.float64),
                                             both.radius.cpu().numpy().astype(np.float64)))
            # seen from a pose between the views (from the frame's own pose the
            # new Gaussians' neighbours sit exactly at q = 9)
            out = R.render([both], api.pose12(path[10], dev), K.astuple(), K.W, K.H, checked=True)
            ids, cnt = G.gpu_lists(R, K.W, K.H)
            ref = oracle.render_lists([osec], path[10], K.astuple(), K.W, K.H, ids, cnt)
            G.check_decisions(ref, "complement")
            G.assert_forward_close(out, ref)


def test_backproject(dev):
    room = syn.make_room()
    K = syn.scaled_intrinsics(96, 72)
    P = syn.trajectory(9)[8]
    depth, _ = syn.raycast(room, K, P)
    depth[5, 7] = 0.0
    cen_ref, pix_ref = oracle.backproject(depth, K.astuple(), P)
    cen, pix = api.backproject(torch.from_numpy(depth).to(dev), K.astuple(), api.pose12(P))
    np.testing.assert_array_equal(pix.cpu().numpy().view(np.uint32), pix_ref)
    np.testing.assert_allclose(cen.cpu().numpy(), cen_ref, rtol=0, atol=4 * 2.0 ** -24 * 8)


@pytest.mark.parametrize("case", ["tiny", "qqvga_2views", "ragged_3views", "own_view"])
def test_depth_keys_and_tile_order(dev, case):
    osecs, target, K, W, H = _cases()[case]()
    R, dsecs, out = _render(osecs, target, K, W, H)
    z_ref, ok = oracle.zkeys(osecs[0], target, K, W, H)
    z = R.debug(0, osecs[0].n, np.float32)
    # bit-exact depth keys for every Gaussian that survives culling
    np.testing.assert_array_equal(z.view(np.uint32)[ok & (z != 0)], z_ref.view(np.uint32)[ok & (z != 0)])
    assert np.all(z[~ok] == 0)
    tiles_x = (W + 15) // 16
    n_tiles = tiles_x * ((H + 15) // 16)
    off = R.debug(1, n_tiles + 1)
    lists = R.debug(2, int(off[-1]))
    zk = z.view(np.uint32).astype(np.uint64)
    for t in range(n_tiles):
        l = lists[off[t]:off[t + 1]].astype(np.int64)
        if l.size > 1:
            key = (zk[l] << np.uint64(32)) | l.astype(np.uint64)
            assert np.all(key[1:] > key[:-1]), t
    # every pixel's added Gaussians are a subsequence, in order, of its tile
    # list ending at the recorded list end, and they are the definition's
    # decisions (up to decisions at the rounding of their thresholds; seen
    # from its own view every pixel has neighbours at exactly q = 9)
    last = R.debug(3, W * H).reshape(H, W)
    nadd = R.debug(4, W * H).reshape(H, W)
    ids, cnt = G.gpu_lists(R, W, H)
    np.testing.assert_array_equal(cnt, nadd)
    for t in range(n_tiles):
        l = lists[off[t]:off[t + 1]].astype(np.int64)
        where = {g: i for i, g in enumerate(l)}
        ty, tx = divmod(t, tiles_x)
        for y in range(ty * 16, min(H, ty * 16 + 16)):
            for x in range(tx * 16, min(W, tx * 16 + 16)):
                idx = [where.get(int(g), -1) for g in ids[y, x, :cnt[y, x]]]
                assert all(i >= 0 for i in idx) and idx == sorted(idx), (y, x)
                if idx:
                    assert last[y, x] == idx[-1] + 1, (y, x)
    ref = oracle.render_lists(osecs, target, K, W, H, ids, cnt)
    G.check_decisions(ref, "keys_" + case)


@pytest.mark.parametrize("case", ["tiny", "qqvga_2views", "ragged_3views"])
def test_forward_parity(dev, case):
    osecs, target, K, W, H = _cases()[case]()
    R, dsecs, out = _render(osecs, target, K, W, H)
    ids, cnt = G.gpu_lists(R, W, H)
    ref = oracle.render_lists(osecs, target, K, W, H, ids, cnt)
    G.check_decisions(ref, "forward_" + case)
    G.assert_forward_close(out, ref)
    T = R.debug(5, W * H, np.float32).reshape(H, W)
    np.testing.assert_allclose(T, ref["T_final"], rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("case", ["tiny", "qqvga_2views", "ragged_3views"])
def test_backward_parity(dev, case):
    osecs, target, K, W, H = _cases()[case]()
    R, dsecs, out = _render(osecs, target, K, W, H)
    ids, cnt = G.gpu_lists(R, W, H)
    gR, gD, gS = _upstream((H, W), 31, 1.0)
    want = oracle.backward_lists(osecs, target, K, W, H, ids, cnt, g_rgb=gR, g_depth=gD, g_sil=gS)
    grads = [(torch.zeros(s.n, 3, device=dev), torch.zeros(s.n, device=dev),
              torch.zeros(s.n, device=dev)) for s in osecs]
    t = lambda a: torch.from_numpy(a).to(dev)
    dtw, dmat = R.backward(t(gR), t(gD), t(gS), attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    G.assert_grad_close(grads[0][0].cpu().numpy(), want["colour"][0], name="colour",
                        abs_ref=want["abs_colour"][0])
    G.assert_grad_close(grads[0][1].cpu().numpy(), want["opacity"][0], name="opacity",
                        abs_ref=want["abs_opacity"][0])
    G.assert_grad_close(grads[0][2].cpu().numpy(), want["radius"][0], name="radius",
                        abs_ref=want["abs_radius"][0])
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist",
                        noise=want["twist_noise"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", noise=want["mat_noise"])


def test_pose_only_and_attr_only_modes_agree(dev):
    osecs, target, K, W, H = _cases()["tiny"]()
    R, dsecs, out = _render(osecs, target, K, W, H)
    gR, gD, gS = (torch.from_numpy(a).to(dev) for a in _upstream((H, W), 5, 1.0))
    n = osecs[0].n
    g1 = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))]
    g2 = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))]
    R.backward(gR, gD, gS, attr_grads=g1)
    tw1, m1 = R.backward(gR, gD, gS, pose_grad=True)
    tw2, m2 = R.backward(gR, gD, gS, attr_grads=g2, pose_grad=True)
    torch.cuda.synchronize()
    assert torch.equal(tw1, tw2) and torch.equal(m1, m2)     # fixed-order FP64 reduction
    for a, b in zip(g1[0], g2[0]):    # float atomics: summation order only
        torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()))


def test_closed_forms_gpu(dev):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
    W, H, f = 16, 12, 20.0
    K = (f, f, 7.5, 5.5)
    col = np.array([[0.2, 0.5, 0.9]])
    sec = G.quantise(h.hand_section([(IDENT, {(8, 6): 2.0})], W, H, K, colour=col))
    R, _, (rgb, depth, sil) = _render([sec], IDENT, K, W, H)
    for c in gold["single_gaussian"]["cases"]:
        du, dv = c["offset"]
        a = c["alpha"]
        assert sil[6 + dv, 8 + du].item() == pytest.approx(a, rel=2e-6, abs=1e-9)
        np.testing.assert_allclose(rgb[:, 6 + dv, 8 + du].cpu().numpy(), sec.colour[0] * a, rtol=3e-6,
                                   atol=1e-9)
    g = gold["termination"]
    rng = np.random.default_rng(11)
    depths = 1.0 + 0.1 * rng.permutation(g["n"])
    sec = G.quantise(h.hand_section([(IDENT, {(8, 6): float(d)}) for d in depths], W, H, K,
                                    colour=rng.uniform(0, 1, (g["n"], 3)),
                                    opacity=np.full(g["n"], g["opacity"])))
    R, _, (rgb, depth, sil) = _render([sec], IDENT, K, W, H)
    assert R.debug(4, W * H).reshape(H, W)[6, 8] == g["n_added"]
    assert sil[6, 8].item() == g["silhouette"]
    assert R.debug(5, W * H, np.float32).reshape(H, W)[6, 8] == np.float32(g["T_final"])


def test_multi_section_with_frozen(dev):
    K = syn.scaled_intrinsics(128, 96)
    full, target = h.multiview_section(K, n_views=3, seed=12)
    plane = full.W * full.H
    view = full.src // plane
    parts = []
    for k in range(3):
        m = view == k
        parts.append(G.quantise(oracle.Section(full.W, full.H, full.K, full.poses[k:k + 1],
                                               full.depth[k:k + 1],
                                               (full.src[m] - k * plane).astype(np.uint32),
                                               full.colour[m], full.opacity[m], full.radius[m])))
    Kt = K.astuple()
    R, dsecs, out = _render(parts, target, Kt, K.W, K.H)
    ids, cnt = G.gpu_lists(R, K.W, K.H)
    ref = oracle.render_lists(parts, target, Kt, K.W, K.H, ids, cnt)
    G.check_decisions(ref, "three_sections")
    G.assert_forward_close(out, ref)
    gR, gD, gS = _upstream((K.H, K.W), 8, 1.0)
    want = oracle.backward_lists(parts, target, Kt, K.W, K.H, ids, cnt, g_rgb=gR, g_depth=gD,
                                 g_sil=gS)
    grads = [None, (torch.zeros(parts[1].n, 3, device=dev), torch.zeros(parts[1].n, device=dev),
                    torch.zeros(parts[1].n, device=dev)), None]
    t = lambda a: torch.from_numpy(a).to(dev)
    R.backward(t(gR), t(gD), t(gS), attr_grads=grads)
    torch.cuda.synchronize()
    G.assert_grad_close(grads[1][0].cpu().numpy(), want["colour"][1], name="colour",
                        abs_ref=want["abs_colour"][1])
    G.assert_grad_close(grads[1][1].cpu().numpy(), want["opacity"][1], name="opacity",
                        abs_ref=want["abs_opacity"][1])
    G.assert_grad_close(grads[1][2].cpu().numpy(), want["radius"][1], name="radius",
                        abs_ref=want["abs_radius"][1])


def test_fp16_attributes(dev):
    K = syn.scaled_intrinsics(160, 120)
    sec, target = h.multiview_section(K, n_views=2, seed=3)
    q = G.quantise(sec, "f16")
    Kt = K.astuple()
    R, dsecs, out = _render([q], target, Kt, K.W, K.H, prec="f16")
    ids, cnt = G.gpu_lists(R, K.W, K.H)
    ref = oracle.render_lists([q], target, Kt, K.W, K.H, ids, cnt)
    G.check_decisions(ref, "fp16_storage")
    G.assert_forward_close(out, ref)
    # against the FP64 render of the FP32 attributes: colour max-abs <= 2e-3 on
    # pixels whose decisions are farther from their thresholds than the FP16
    # rounding of o and r can move them (relative 2e-3); the 3-sigma cutoff
    # and the 1/255 skip are discontinuous, so the rest may jump by ~0.01 c.
    ref32 = oracle.render([G.quantise(sec)], target, Kt, K.W, K.H)
    stable = (ref32["margin"] > 2e-3) & (ref32["margin_T"] > 2e-3)
    err = np.abs(out[0].cpu().numpy() - ref32["rgb"])
    assert stable.mean() > 0.5
    assert np.max(err[:, stable]) <= 2e-3
    assert np.percentile(err, 99) <= 2e-3
    print("FP16_COLOUR_VS_FP64", dict(pixels=int(err[0].size), max_abs=float(err.max()),
                                       pixels_above_2e_3=int((err.max(0) > 2e-3).sum()),
                                       unstable_pixels=int((~stable).sum())))


def test_empty_and_degenerate(dev):
    K = (20.0, 20.0, 7.5, 5.5)
    # empty section: background everywhere
    sec = G.quantise(h.hand_section([(IDENT, {})], 16, 12, K))
    R, _, (rgb, depth, sil) = _render([sec], IDENT, K, 16, 12)
    assert sec.n == 0 and float(rgb.abs().max()) == 0.0 and float(sil.abs().max()) == 0.0
    # everything behind the camera or closer than z_near: culled
    sec = G.quantise(h.hand_section([(IDENT, {(3, 3): 0.05, (8, 6): 1.0})], 16, 12, K))
    back = np.hstack([np.diag([1.0, 1.0, 1.0]), np.array([[0.0], [0.0], [2.0]])])
    R, _, (rgb, depth, sil) = _render([sec], back, K, 16, 12)
    assert float(sil.abs().max()) == 0.0
    # 1x1 and 17x1 images, one huge Gaussian covering everything
    for W, H in ((1, 1), (17, 1), (33, 47)):
        Kc = (20.0, 20.0, (W - 1) / 2, (H - 1) / 2)
        s = G.quantise(h.hand_section([(IDENT, {(0, 0): 1.0})], 1, 1, (20.0, 20.0, 0.0, 0.0),
                                      radius=[5.0], opacity=[0.5]))
        R, _, out = _render([s], IDENT, Kc, W, H)
        ids, cnt = G.gpu_lists(R, W, H)
        ref = oracle.render_lists([s], IDENT, Kc, W, H, ids, cnt)
        G.check_decisions(ref, f"degenerate_{W}x{H}")
        G.assert_forward_close(out, ref)
        assert float(out[2].min()) > 0.4


def test_capacity_overflow_reported_and_recovered(dev):
    osecs, target, K, W, H = _cases()["qqvga_2views"]()
    dsecs = [G.to_device(s) for s in osecs]
    R = api.Renderer()
    R.reserve(osecs[0].n, W, H, n_instances=1000)
    R.render(dsecs, api.pose12(target), K, W, H)
    from paper_2506_02741_gb300 import _lib as L
    with pytest.raises(L.VTError) as ei:
        R.status()
    assert ei.value.status == L.VT_ERR_CAPACITY
    out = R.render(dsecs, api.pose12(target), K, W, H, checked=True)
    ids, cnt = G.gpu_lists(R, W, H)
    ref = oracle.render_lists(osecs, target, K, W, H, ids, cnt)
    G.check_decisions(ref, "capacity_recovered")
    G.assert_forward_close(out, ref)


def test_determinism(dev):
    osecs, target, K, W, H = _cases()["qqvga_2views"]()
    R, dsecs, a = _render(osecs, target, K, W, H)
    a = [x.clone() for x in a]
    b = R.render(dsecs, api.pose12(target), K, W, H)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    g = torch.ones(3, H, W, device=dev)
    t1, m1 = R.backward(g, None, None, pose_grad=True)
    t2, m2 = R.backward(g, None, None, pose_grad=True)
    assert torch.equal(t1, t2) and torch.equal(m1, m2)


def test_bad_arguments_rejected(dev):
    from paper_2506_02741_gb300 import _lib as L
    osecs, target, K, W, H = _cases()["tiny"]()
    d = G.to_device(osecs[0])
    R = api.Renderer()
    with pytest.raises(L.VTError) as ei:
        R.render([d], api.pose12(target), (0.0, 1.0, 0.0, 0.0), W, H)
    assert ei.value.status == L.VT_ERR_INVALID_ARG
    with pytest.raises(L.VTError) as ei:
        R.render([d], api.pose12(target), K, 0, H)
    assert ei.value.status == L.VT_ERR_INVALID_ARG
    R2 = api.Renderer()
    with pytest.raises(L.VTError) as ei:
        R2.backward(torch.ones(3, H, W, device=dev), pose_grad=True)
    assert ei.value.status == L.VT_ERR_STATE


@pytest.mark.parametrize("cap", [0, 3, 256])
def test_backward_paths_agree(dev, cap):
    """Per-pixel list replay (cap 256), tile replay (cap 0) and the mixed case
    where pixels overflow a tiny list (cap 3) give the oracle's gradients."""
    osecs, target, K, W, H = _cases()["qqvga_2views"]()
    R = api.Renderer()
    R.set_list_capacity(cap)
    R, dsecs, out = _render(osecs, target, K, W, H, R=R)
    assert R.used_lists == (cap > 0)
    ids, cnt = G.decisions(dsecs, api.pose12(target), K, W, H, out=out)
    gR, gD, gS = _upstream((H, W), 77, 1.0)
    want = oracle.backward_lists(osecs, target, K, W, H, ids, cnt, g_rgb=gR, g_depth=gD, g_sil=gS)
    n = osecs[0].n
    grads = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))]
    t = lambda a: torch.from_numpy(a).to(dev)
    dtw, dmat = R.backward(t(gR), t(gD), t(gS), attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    for k, name in enumerate(("colour", "opacity", "radius")):
        G.assert_grad_close(grads[0][k].cpu().numpy(), want[name][0], name=name,
                            abs_ref=want["abs_" + name][0])
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist",
                        noise=want["twist_noise"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", noise=want["mat_noise"])


@pytest.mark.parametrize("cap", [0, 3, 256])
def test_twist_only_backward(dev, cap):
    """A pose backward asked for the twist alone (no matrix gradient: the
    tracking iteration) takes the six-sum form of the list backward: its
    twist agrees with the twelve-sum form's within FP32 rounding and with the
    oracle's, on list tiles, replayed tiles and a mix of both."""
    osecs, target, K, W, H = _cases()["qqvga_2views"]()
    R = api.Renderer()
    R.set_list_capacity(cap)
    R, dsecs, out = _render(osecs, target, K, W, H, R=R)
    ids, cnt = G.decisions(dsecs, api.pose12(target), K, W, H, out=out)
    gR, gD, _ = _upstream((H, W), 78, 1.0)
    want = oracle.backward_lists(osecs, target, K, W, H, ids, cnt, g_rgb=gR, g_depth=gD)
    t = lambda a: torch.from_numpy(a).to(dev)
    tw = torch.zeros(6, dtype=torch.float64, device=dev)
    R.backward(t(gR), t(gD), None, pose_grad=True, d_twist=tw)
    full, _ = R.backward(t(gR), t(gD), None, pose_grad=True)
    torch.cuda.synchronize()
    a, b = tw.cpu().numpy(), full.cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    G.assert_grad_close(a, want["twist"], name="twist", noise=want["twist_noise"])


def test_budget_disables_lists(dev):
    osecs, target, K, W, H = _cases()["tiny"]()
    R = api.Renderer()
    R.set_budget(1)            # nothing fits: lists are dropped, the render still works
    R, dsecs, out = _render(osecs, target, K, W, H, R=R)
    assert not R.used_lists
    ids, cnt = G.decisions(dsecs, api.pose12(target), K, W, H, out=out)
    ref = oracle.render_lists(osecs, target, K, W, H, ids, cnt)
    G.check_decisions(ref, "budget_no_lists")
    G.assert_forward_close(out, ref)


@pytest.mark.parametrize("case", ["qqvga_2views", "ragged_3views"])
def test_view_pose_gradients(dev, case):
    """Source-view pose gradients (head-frame bundle adjustment) against the
    oracle's, per view as twist and matrix: 1e-4 relative per view tensor
    (sums over every pixel of the render, FP32 per pair); each Gaussian's
    depth gradient (movable along its ray) within the gradient tolerance.  Requesting them
    together with the attribute and target-pose gradients leaves those
    unchanged up to the order of float atomics."""
    osecs, target, K, W, H = _cases()[case]()
    R, dsecs, out = _render(osecs, target, K, W, H)
    ids, cnt = G.gpu_lists(R, W, H)
    rng = np.random.default_rng(41)
    gR = rng.normal(0, 1, (3, H, W)).astype(np.float32)
    gD = rng.normal(0, 1, (H, W)).astype(np.float32)
    want = oracle.backward_lists(osecs, target, K, W, H, ids, cnt, g_rgb=gR, g_depth=gD)
    tw_ref, mat_ref = oracle.view_pose_grads(osecs[0], target, want["x"][0])
    V = osecs[0].poses.shape[0]
    vt = torch.zeros(V, 6, dtype=torch.float64, device=dev)
    vm = torch.zeros(V, 12, dtype=torch.float64, device=dev)
    n = osecs[0].n
    vd = torch.zeros(n, device=dev)
    ag = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))]
    dtw, dmat = R.backward(torch.from_numpy(gR).to(dev), torch.from_numpy(gD).to(dev), None,
                           attr_grads=ag, pose_grad=True, view_grads=[(vt, vm, vd)])
    torch.cuda.synchronize()
    dref, dmag = oracle.depth_grads(osecs[0], target, want["x"][0], want["abs_x"][0])
    G.assert_grad_close(vd.cpu().numpy(), dref, name="depth", abs_ref=dmag)
    for k in range(V):
        for got, ref_ in ((vt[k], tw_ref[k]), (vm[k], mat_ref[k])):
            g = got.cpu().numpy()
            assert np.linalg.norm(g - ref_) <= 1e-4 * np.linalg.norm(ref_), (k, g, ref_)
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", noise=want["twist_noise"])
    G.assert_grad_close(ag[0][1].cpu().numpy(), want["opacity"][0], name="opacity",
                        abs_ref=want["abs_opacity"][0])
    # a frozen section gets nothing, views-only mode works alone
    vt2 = torch.zeros_like(vt)
    R.backward(torch.from_numpy(gR).to(dev), torch.from_numpy(gD).to(dev), None,
               view_grads=[(vt2, None)])
    torch.cuda.synchronize()
    np.testing.assert_allclose(vt2.cpu().numpy(), vt.cpu().numpy(), rtol=1e-5,
                               atol=1e-7 * np.abs(tw_ref).max())
    vt3 = torch.zeros_like(vt)
    R.backward(torch.from_numpy(gR).to(dev), None, None, view_grads=[None])
    assert not vt3.any()
