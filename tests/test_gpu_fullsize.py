"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the GPU renders the whole frame, the oracle a crop of it (same camera
with a shifted principal point, so the crop's pixels are the frame's pixels).

* tracking: 640x480, 8 keyframes = 2,457,600 FP32 Gaussians;
* mapping: 1200x680, 10 views = 8,160,000 FP16 Gaussians.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _section(K, n_key, prec):
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(n_key * 5 + 4)
    keys = [path[i * 5] for i in range(n_key)]
    fr = syn.render_frames(room, K, keys)
    osec = oracle.section_init(fr.depth, fr.rgb, K.astuple(), np.stack(keys))
    return G.quantise(osec, prec), path[(n_key - 1) * 5 + 2]


def _crop(K, x0, y0):
    return (K.fx, K.fy, K.cx - x0, K.cy - y0)


@pytest.mark.parametrize("cfg", ["tracking_640x480_fp32", "mapping_1200x680_fp16"])
def test_fullsize_crop_parity(cfg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    if cfg.startswith("tracking"):
        K, n_key, prec = syn.VGA, 8, "f32"
    else:
        K, n_key, prec = syn.REPLICA, 10, "f16"
    osec, target = _section(K, n_key, prec)
    assert osec.n == n_key * K.W * K.H
    sec = G.to_device(osec, prec)
    R = api.Renderer()
    rgb, depth, sil = R.render([sec], api.pose12(target, dev), K.astuple(), K.W, K.H, checked=True)
    cw, ch = 96, 80
    x0, y0 = (K.W - cw) // 2 + 16, (K.H - ch) // 2 - 8
    Kc = _crop(K, x0, y0)
    ids, cnt = G.decisions([sec], api.pose12(target, dev), K.astuple(), K.W, K.H,
                           out=(rgb, depth, sil), box=(x0, y0, cw, ch), cap=1024)
    ref = oracle.render_lists([osec], target, Kc, cw, ch, ids, cnt)
    G.check_decisions(ref, "fullsize_" + cfg)
    sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
    out = (rgb[:, sl[0], sl[1]], depth[sl], sil[sl])
    G.assert_forward_close(out, ref)
    # backward with the upstream gradient on the crop only
    rng = np.random.default_rng(8)
    gR = rng.normal(0, 1, (3, ch, cw)).astype(np.float32)
    gD = rng.normal(0, 1, (ch, cw)).astype(np.float32)
    want = oracle.backward_lists([osec], target, Kc, cw, ch, ids, cnt, g_rgb=gR, g_depth=gD)
    full_gR = torch.zeros(3, K.H, K.W, device=dev)
    full_gD = torch.zeros(K.H, K.W, device=dev)
    full_gR[:, sl[0], sl[1]] = torch.from_numpy(gR).to(dev)
    full_gD[sl] = torch.from_numpy(gD).to(dev)
    n = osec.n
    grads = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))]
    dtw, dmat = R.backward(full_gR, full_gD, None, attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    touched = np.flatnonzero(want["abs_opacity"][0] > 0)
    assert touched.size > 1000
    for k, name in enumerate(("colour", "opacity", "radius")):
        got = grads[0][k].cpu().numpy()
        G.assert_grad_close(got[touched], want[name][0][touched], name=name,
                            abs_ref=want["abs_" + name][0][touched])
        other = np.ones(n, bool)
        other[touched] = False
        assert np.all(got[other] == 0)
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist",
                        noise=want["twist_noise"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", noise=want["mat_noise"])
    # the tracking iteration's form: the twist alone (six-sum list backward)
    tw = torch.zeros(6, dtype=torch.float64, device=dev)
    R.backward(full_gR, full_gD, None, pose_grad=True, d_twist=tw)
    torch.cuda.synchronize()
    G.assert_grad_close(tw.cpu().numpy(), want["twist"], name="twist_only",
                        noise=want["twist_noise"])


def test_4k_render_crop_parity():
    """The 8-keyframe tracking section rendered at 3832x2156 (4K cut so that
    the last tile column and row are ragged; the same field of view: 8.3 M
    pixels, 32,400 tiles, per-pixel lists of 17 GB, so their byte offsets
    pass 2^31): a crop at the bottom edge, through the ragged tiles, against
    the oracle along the GPU's decisions, and the pose gradient of an
    upstream gradient on that crop."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    osec, target = _section(syn.VGA, 8, "f32")
    sec = G.to_device(osec, "f32")
    K = syn.scaled_intrinsics(3832, 2156)
    R = api.Renderer()
    rgb, depth, sil = R.render([sec], api.pose12(target, dev), K.astuple(), K.W, K.H,
                               checked=True)
    assert R.used_lists
    cw, ch = 96, 80
    x0, y0 = (K.W - cw) // 2, K.H - ch       # through the ragged last tile row
    Kc = _crop(K, x0, y0)
    ids, cnt = G.decisions([sec], api.pose12(target, dev), K.astuple(), K.W, K.H,
                           out=(rgb, depth, sil), box=(x0, y0, cw, ch))
    ref = oracle.render_lists([osec], target, Kc, cw, ch, ids, cnt)
    G.check_decisions(ref, "render_3832x2156")
    assert float(ref["sil"].mean()) > 0.5        # the crop sees the scene
    sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
    G.assert_forward_close((rgb[:, sl[0], sl[1]], depth[sl], sil[sl]), ref)
    gR = np.random.default_rng(9).normal(0, 1, (3, ch, cw)).astype(np.float32)
    want = oracle.backward_lists([osec], target, Kc, cw, ch, ids, cnt, g_rgb=gR)
    full_gR = torch.zeros(3, K.H, K.W, device=dev)
    full_gR[:, sl[0], sl[1]] = torch.from_numpy(gR).to(dev)
    dtw, dmat = R.backward(full_gR, None, None, pose_grad=True)
    torch.cuda.synchronize()
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist",
                        noise=want["twist_noise"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", noise=want["mat_noise"])


def _tile_lists_sorted(R, n, W, H):
    z = R.debug(0, n, np.float32)
    tiles_x = (W + 15) // 16
    n_tiles = tiles_x * ((H + 15) // 16)
    off = R.debug(1, n_tiles + 1).astype(np.int64)
    lists = R.debug(2, int(off[-1])).astype(np.int64)
    zk = z.view(np.uint32).astype(np.uint64)
    key = (zk[lists] << np.uint64(32)) | lists.astype(np.uint64)
    tile_of = np.searchsorted(off, np.arange(lists.size), side="right") - 1
    same_tile = tile_of[1:] == tile_of[:-1]
    assert np.all((key[1:] > key[:-1])[same_tile])
    return np.diff(off)


def test_tile_sort_every_size_class():
    """Every tile list is ordered by (depth key, id) at the tracking size
    (tiles of every shared-memory size class, including the few longest sorted
    on the auxiliary stream) and in a crafted case whose lists exceed the
    shared-memory sort (global-memory path); the latter also matches the
    oracle's render."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    K = syn.VGA
    osec, target = _section(K, 8, "f32")
    sec = G.to_device(osec, "f32")
    R = api.Renderer()
    R.render([sec], api.pose12(target, dev), K.astuple(), K.W, K.H, checked=True)
    lens = _tile_lists_sorted(R, osec.n, K.W, K.H)
    for lo, hi in ((1, 1536), (1536, 3584), (3584, 6000), (6000, 13312)):
        assert np.any((lens > lo) & (lens <= hi)), (lo, hi)
    # 30 views of a 64x48 camera with 3x radii: lists beyond 13312 entries
    Kt = syn.TINY
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(31)
    fr = syn.render_frames(room, Kt, path[:30])
    big = oracle.section_init(fr.depth, fr.rgb, Kt.astuple(), np.stack(path[:30]))
    big.radius = big.radius * 3.0
    big = G.quantise(big, "f32")
    bsec = G.to_device(big, "f32")
    R2 = api.Renderer()
    R2.reserve(big.n, Kt.W, Kt.H, 40 * big.n)
    out = R2.render([bsec], api.pose12(path[30], dev), Kt.astuple(), Kt.W, Kt.H, checked=True)
    lens = _tile_lists_sorted(R2, big.n, Kt.W, Kt.H)
    assert lens.max() > 13312
    ids, cnt = G.decisions([bsec], api.pose12(path[30], dev), Kt.astuple(), Kt.W, Kt.H, out=out,
                           cap=4096)
    ref = oracle.render_lists([big], path[30], Kt.astuple(), Kt.W, Kt.H, ids, cnt)
    G.check_decisions(ref, "sort_global_memory_30layers")
    G.assert_forward_close(out, ref)


def test_fullsize_ellipsoid_crop_parity():
    """The ellipsoid path at the full tracking size (640x480, 8 keyframes,
    2,457,600 Gaussians, scales radius * exp(N(0, 0.35)), random rotations):
    forward and gradients of a 96x80 crop against the anisotropic oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import aniso
    dev = torch.device("cuda:0")
    K = syn.VGA
    osec, target = _section(K, 8, "f32")
    q32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    scale, quat = (q32(a) for a in syn.random_ellipsoids(osec.radius, 17))
    sec = G.to_device(osec).with_ellipsoids(torch.from_numpy(scale), torch.from_numpy(quat))
    R = api.Renderer()
    rgb, depth, sil = R.render([sec], api.pose12(target, dev), K.astuple(), K.W, K.H, checked=True)
    cw, ch = 96, 80
    x0, y0 = (K.W - cw) // 2 + 16, (K.H - ch) // 2 - 8
    Kc = _crop(K, x0, y0)
    ids, cnt = G.decisions([sec], api.pose12(target, dev), K.astuple(), K.W, K.H,
                           out=(rgb, depth, sil), box=(x0, y0, cw, ch), cap=1024)
    ref = aniso.render_lists(osec, scale, quat, target, Kc, cw, ch, ids, cnt, keep=True)
    G.check_decisions(ref, "fullsize_ellipsoids")
    sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
    G.assert_forward_close((rgb[:, sl[0], sl[1]], depth[sl], sil[sl]), ref, tol=2e-5)
    rng = np.random.default_rng(8)
    gR = rng.normal(0, 1, (3, ch, cw)).astype(np.float32)
    gD = rng.normal(0, 1, (ch, cw)).astype(np.float32)
    want = aniso.backward(osec, scale, quat, target, Kc, cw, ch, gR, gD, fwd=ref)
    full_gR = torch.zeros(3, K.H, K.W, device=dev)
    full_gD = torch.zeros(K.H, K.W, device=dev)
    full_gR[:, sl[0], sl[1]] = torch.from_numpy(gR).to(dev)
    full_gD[sl] = torch.from_numpy(gD).to(dev)
    n = osec.n
    z = lambda *s: torch.zeros(*s, device=dev)
    grads = [(z(n, 3), z(n), None, z(n, 3), z(n, 4))]
    dtw, dmat = R.backward(full_gR, full_gD, None, attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    touched = np.flatnonzero(want["abs_opacity"] > 0)
    assert touched.size > 1000
    for k, name in ((0, "colour"), (1, "opacity"), (3, "scale"), (4, "quat")):
        got = grads[0][k].cpu().numpy()
        G.assert_grad_close(got[touched], want[name][touched], name=name,
                            abs_ref=want["abs_" + name][touched])
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", abs_ref=want["abs_twist"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", abs_ref=want["abs_mat"])


def _large_sections(n_sec=7, per=14):
    """Seven adjacent sections of 14 keyframes each (every other frame of the
    path) at 640x480: 30,105,600 Gaussians, rendered together (the
    multi-section render)."""
    K = syn.VGA
    path = syn.trajectory(n_sec * per * 2 + 5)
    room = syn.make_room(syn.SCENE_SEED)
    out = []
    for s in range(n_sec):
        keys = [path[2 * (s * per + j)] for j in range(per)]
        fr = syn.render_frames(room, K, keys)
        out.append((fr, np.stack(keys)))
    return K, out, path[n_sec * per + 1]   # between keyframes (odd path index)


def _crop_subset(osec, target, K, box, slack=3.0):
    """The Gaussians of an oracle section whose 3-sigma disc can reach the
    crop box (x0, y0, w, h), as a section of their own: ids keep their
    relative order, so (z_key, id) orders them as in the whole render."""
    import dataclasses
    x0, y0, w, h = box
    P = np.asarray(target, np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    plane = osec.W * osec.H
    src = osec.src.astype(np.int64)
    view = src // plane
    pix = src - view * plane
    u, v = (pix % osec.W).astype(np.float64), (pix // osec.W).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(k)) for k in osec.K)
    D = osec.depth.reshape(-1)[src].astype(np.float64)
    Xc = np.stack([D * (u - cx) / fx, D * (v - cy) / fy, D], 1)
    mu = np.einsum("nab,nb->na", osec.poses[view][:, :, :3], Xc) + osec.poses[view][:, :, 3]
    x = (mu - t) @ R
    z = x[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        uc = K.fx * x[:, 0] / z + K.cx
        vc = K.fy * x[:, 1] / z + K.cy
        e = 3.0 * max(K.fx, K.fy) * osec.radius / z + slack
        keep = (z > 0.05) & (uc + e >= x0) & (uc - e <= x0 + w - 1) & (vc + e >= y0) & \
               (vc - e <= y0 + h - 1)
    return dataclasses.replace(osec, src=osec.src[keep], colour=osec.colour[keep],
                               opacity=osec.opacity[keep], radius=osec.radius[keep]), keep


def test_large_multisection_render():
    """30.1 M Gaussians of seven sections rendered together at 640x480 (about
    1,500 Gaussians over each pixel, so many per-pixel lists overflow and
    their tiles take the replay backward), and again under a workspace
    budget that keeps no lists at all: a 96x80 crop and the pose gradient of
    an upstream gradient on that crop against the oracle, which renders the
    Gaussians that can reach the crop; both backward forms agree."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    K, frames, target = _large_sections()
    dsecs, osecs = [], []
    for fr, keys in frames:
        dsecs.append(api.Section.from_rgbd(torch.from_numpy(fr.depth).to(dev),
                                           torch.from_numpy(fr.rgb).to(dev), K.astuple(), keys))
        osecs.append(G.quantise(oracle.section_init(fr.depth, fr.rgb, K.astuple(), keys)))
    assert sum(s.n for s in dsecs) == 30_105_600
    cw, ch = 96, 80
    x0, y0 = (K.W - cw) // 2 + 40, (K.H - ch) // 2 + 24
    Kc = _crop(K, x0, y0)
    subs, keeps = zip(*[_crop_subset(s, target, K, (x0, y0, cw, ch)) for s in osecs])
    # the GPU's decisions on the crop, from a render that keeps lists long
    # enough for every pixel (about 1,500 Gaussians lie over each)
    ids, cnt = G.decisions(dsecs, api.pose12(target, dev), K.astuple(), K.W, K.H,
                           box=(x0, y0, cw, ch), id_map=G.subset_map(list(keeps)), cap=4096)
    ref = oracle.render_lists(list(subs), target, Kc, cw, ch, ids, cnt)
    G.check_decisions(ref, "large_multisection_30M")
    rng = np.random.default_rng(5)
    gR = rng.normal(0, 1, (3, ch, cw)).astype(np.float32)
    want = oracle.backward_lists(list(subs), target, Kc, cw, ch, ids, cnt, g_rgb=gR)
    sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
    full_gR = torch.zeros(3, K.H, K.W, device=dev)
    full_gR[:, sl[0], sl[1]] = torch.from_numpy(gR).to(dev)
    results = []
    for budget in (None, 1):
        R = api.Renderer()
        if budget is not None:
            R.set_budget(budget)
        rgb, depth, sil = R.render(dsecs, api.pose12(target, dev), K.astuple(), K.W, K.H,
                                   checked=True)
        assert R.used_lists == (budget is None)
        G.assert_forward_close((rgb[:, sl[0], sl[1]], depth[sl], sil[sl]), ref)
        dtw, dmat = R.backward(full_gR, None, None, pose_grad=True)
        torch.cuda.synchronize()
        G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist",
                            noise=want["twist_noise"])
        results.append((rgb, dtw))
        del R
    assert torch.equal(results[0][0], results[1][0])
    torch.testing.assert_close(results[0][1], results[1][1], rtol=1e-6,
                               atol=1e-9 * float(results[1][1].abs().max()))


def _multiroom_sections(dev, n_sec=6, per=16, every=5):
    """Six adjacent sections of 16 keyframes (every 5th frame from frame 200)
    of the 2000-frame path through five rooms, 640x480: 29,491,200
    Gaussians; the target pose lies inside the middle section."""
    K = syn.VGA
    rooms = syn.make_rooms(5)
    path = syn.multi_room_trajectory(2000, 5)
    idx = [200 + every * j for j in range(n_sec * per)]
    fr = syn.render_multi(rooms, K, [path[i] for i in idx])
    dsecs, osecs = [], []
    for s in range(n_sec):
        sl = slice(s * per, (s + 1) * per)
        keys = np.stack([path[i] for i in idx[sl]])
        dsecs.append(api.Section.from_rgbd(torch.from_numpy(fr.depth[sl]).to(dev),
                                           torch.from_numpy(fr.rgb[sl]).to(dev), K.astuple(),
                                           keys))
        osecs.append(G.quantise(oracle.section_init(fr.depth[sl], fr.rgb[sl], K.astuple(), keys)))
    return K, dsecs, osecs, path[200 + every * (n_sec * per // 2) + 2]


def test_multiroom_large_scene_finite_differences():
    """The large end of the multi-room workload (29.5 M Gaussians of six
    sections rendered together): a 96x80 crop and its pose gradient against
    the oracle along the GPU's decisions (given the Gaussians that can reach
    the crop), and central differences of the GPU forward in the opacity of
    64 sampled Gaussians against the oracle's opacity gradient: the GPU's
    render at that scale changes as the oracle's gradient says.  The
    difference quotients take the upstream gradient on the pixels whose
    termination decision is more than 5% from its threshold (there a step of
    2e-3 in o moves the transmittance by under 2% and no walk stops
    elsewhere; o = 0.9 puts the 1/255 cut outside the 3-sigma disc, so no
    inclusion decision moves either)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    K, dsecs, osecs, target = _multiroom_sections(dev)
    assert sum(s.n for s in dsecs) == 29_491_200
    pose = api.pose12(target, dev)
    R = api.Renderer()
    rgb, depth, sil = R.render(dsecs, pose, K.astuple(), K.W, K.H, checked=True)
    cw, ch = 96, 80
    x0, y0 = (K.W - cw) // 2 + 24, (K.H - ch) // 2 - 16
    Kc = _crop(K, x0, y0)
    subs, keeps = zip(*[_crop_subset(s, target, K, (x0, y0, cw, ch)) for s in osecs])
    ids, cnt = G.decisions(dsecs, pose, K.astuple(), K.W, K.H, out=(rgb, depth, sil),
                           box=(x0, y0, cw, ch), id_map=G.subset_map(list(keeps)), cap=4096)
    ref = oracle.render_lists(list(subs), target, Kc, cw, ch, ids, cnt)
    G.check_decisions(ref, "multiroom_29.5M")
    sl = (slice(y0, y0 + ch), slice(x0, x0 + cw))
    G.assert_forward_close((rgb[:, sl[0], sl[1]], depth[sl], sil[sl]), ref)
    rng = np.random.default_rng(21)
    gR = rng.normal(0, 1, (3, ch, cw)).astype(np.float32)
    want = oracle.backward_lists(list(subs), target, Kc, cw, ch, ids, cnt, g_rgb=gR)
    full_gR = torch.zeros(3, K.H, K.W, device=dev)
    full_gR[:, sl[0], sl[1]] = torch.from_numpy(gR).to(dev)
    dtw, _ = R.backward(full_gR, None, None, pose_grad=True)
    torch.cuda.synchronize()
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", noise=want["twist_noise"])
    # 64 Gaussians with the largest opacity terms under the upstream gradient
    # of the pixels far from their termination threshold
    far = oracle.render(list(subs), target, Kc, cw, ch)["margin_T"] > 0.05
    assert far.sum() > 500
    gF = (gR * far).astype(np.float32)
    wantF = oracle.backward_lists(list(subs), target, Kc, cw, ch, ids, cnt, g_rgb=gF)
    # (a Gaussian's opacity gradient sums terms of both signs over its
    # pixels and the pixels behind it; the FP32 difference quotient resolves
    # the sum where it does not cancel to far below its terms' magnitude,
    # so the sample is the Gaussians with the largest gradients among those
    # whose gradient keeps a tenth of that magnitude)
    cand = []
    for s, (k, a, v) in enumerate(zip(keeps, wantF["abs_opacity"], wantF["opacity"])):
        full = np.flatnonzero(k)
        ok_ = np.abs(v) > 0.1 * a
        for j in np.flatnonzero(ok_)[np.argsort(-np.abs(v[ok_]))][:64]:
            cand.append((abs(v[j]), s, int(full[j]), float(v[j]), float(a[j])))
    cand.sort(reverse=True)
    assert len(cand) >= 64
    g_crop = torch.from_numpy(gF.astype(np.float64)).to(dev)

    def loss():
        out, _, _ = R.render(dsecs, pose, K.astuple(), K.W, K.H)
        return float((out[:, sl[0], sl[1]].double() * g_crop).sum())

    e = 2e-3
    ok = 0
    for _, s, li, g_want, mag in cand[:64]:
        o = dsecs[s].opacity
        v = float(o[li])
        o[li] = v + e
        lp = loss()
        o[li] = v - e
        lm = loss()
        o[li] = v
        fd = (lp - lm) / (2 * e)
        ok += abs(fd - g_want) <= 1e-2 * abs(g_want) + 1e-3 * mag
    # allow a few of the 64: where the step +-e moves a decision of the
    # forward (the 1/255 cut or the termination point depend on o), the
    # difference quotient is not the derivative
    assert ok >= 60, ok
