"""Batched work items (vt_batch_*) through the C ABI: each item's images and
tracking results against the single-request calls (vt_render, vt_masked_l1,
vt_render_backward), alone and in a mix of sections, resolutions and kinds;
a crop of every item against the oracle along the GPU's decisions; replay of
a captured launch; the capacity and argument errors."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import _lib as L
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G

pytestmark = pytest.mark.gpu

W_RGB, W_DEPTH, SIL_MIN = 0.5, 0.025, 0.99


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def scene(dev):
    """Three sections of the seeded room (1, 2 and 3 keyframes of a 160x120
    camera, the middle one stored in FP16), poses along the path and the
    observed frames the tracking items are fitted to."""
    K = syn.scaled_intrinsics(160, 120)
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(40)
    osecs, dsecs = [], []
    for s, (views, prec) in enumerate((((0,), "f32"), ((5, 10), "f16"), ((15, 20, 25), "f32"))):
        keys = [path[i] for i in views]
        fr = syn.render_frames(room, K, keys)
        o = G.quantise(oracle.section_init(fr.depth, fr.rgb, K.astuple(), np.stack(keys)), prec)
        osecs.append(o)
        dsecs.append(G.to_device(o, prec))
    return dict(K=K, room=room, path=path, osecs=osecs, dsecs=dsecs)


# (section, track, W, H, path index of the camera)
MIX = [(0, True, 160, 120, 2), (1, False, 203, 131, 7), (2, True, 96, 80, 22),
       (1, True, 160, 120, 12), (2, False, 64, 48, 27), (0, True, 33, 17, 1)]


def _items(sc, dev, mix):
    items = []
    for sec, track, W, H, pi in mix:
        K = syn.scaled_intrinsics(W, H).astuple()
        pose = sc["path"][pi]
        it = api.BatchItem(sec, track, W, H, K, api.pose12(pose, dev),
                           torch.full((5, H, W), -7.0, device=dev))
        if track:
            # observed frame: the room seen from a nearby pose
            fr = syn.render_frames(sc["room"], syn.scaled_intrinsics(W, H), [sc["path"][pi + 1]])
            obs = np.concatenate([fr.rgb[0], fr.depth[0][None]]).astype(np.float32)
            it.obs = torch.from_numpy(obs).to(dev)
            it.result = torch.full((19,), np.nan, dtype=torch.float64, device=dev)
        items.append(it)
    return items


def _runner(sc, list_cap=None):
    return api.BatchRunner(max_gaussians=4_000_000, max_pixels=400_000, max_tiles=4000,
                           max_instances=12_000_000, max_views=64, max_table_rows=64 * 400,
                           list_cap=list_cap)


def _single(sc, it, dev, list_cap=None):
    """The same item through the single-request calls (same per-pixel list
    capacity, so that the same tiles take the list and the replay
    backward)."""
    R = api.Renderer()
    if list_cap is not None:
        R.set_list_capacity(list_cap)
    rgb, depth, sil = R.render([sc["dsecs"][it.section]], it.pose, it.K, it.W, it.H,
                               checked=True)
    out = dict(R=R, image=torch.cat([rgb, depth[None], sil[None]]))
    if it.track:
        g_rgb = torch.zeros(3, it.H, it.W, device=dev)
        g_depth = torch.zeros(it.H, it.W, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        R.masked_l1(rgb, depth, sil, it.obs[:3], it.obs[3], W_RGB, W_DEPTH, sil_min=SIL_MIN,
                    rgb_needs_depth=True, d_rgb=g_rgb, d_depth=g_depth, loss=loss)
        tw, mat = R.backward(g_rgb, g_depth, None, pose_grad=True)
        out.update(loss=loss, twist=tw, mat=mat)
    torch.cuda.synchronize()
    return out


def _check_item(it, ref, bit_exact_loss=False):
    assert torch.equal(it.image, ref["image"]), "image differs from vt_render"
    if it.track:
        r = it.result.cpu().numpy()
        if bit_exact_loss:
            assert r[0] == ref["loss"].item()
        else:   # another fixed order of the same FP64 block sums
            assert r[0] == pytest.approx(ref["loss"].item(), rel=1e-13, abs=1e-300)
        # the same per-pixel terms summed in the same order; the compiler may
        # contract a product and a sum differently in the two instantiations
        # of the backward body, so FP32 rounding may differ by an ulp here and
        # there (the images, evaluated with explicit rounding, are identical)
        for got, want in ((r[1:7], ref["twist"]), (r[7:19], ref["mat"])):
            want = want.cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-7 * np.abs(want).max())


@pytest.mark.parametrize("list_cap", [None, 0, 3])
def test_batch_matches_single_requests(dev, scene, list_cap):
    """Images bit-identical to vt_render; pose gradients within FP32 rounding
    of the single backward (the same per-pixel terms, tiles and order); the
    loss within FP64 rounding of vt_masked_l1.  With list capacity 0
    every tracking tile is replayed, with 3 most are (lists overflow)."""
    items = _items(scene, dev, MIX)
    B = _runner(scene, list_cap)
    B.set(scene["dsecs"], items, W_RGB, W_DEPTH, SIL_MIN, True)
    B.launch()
    torch.cuda.synchronize()
    B.status()
    for it in items:
        _check_item(it, _single(scene, it, dev, list_cap))


def test_each_item_alone_equals_the_mix(dev, scene):
    """Every item gives the same bits as a one-item batch as in the mix."""
    items = _items(scene, dev, MIX)
    B = _runner(scene)
    B.set(scene["dsecs"], items)
    B.launch()
    torch.cuda.synchronize()
    mixed = [(it.image.clone(), None if it.result is None else it.result.clone()) for it in items]
    for it, (img, res) in zip(items, mixed):
        it.image.fill_(-1.0)
        if it.result is not None:
            it.result.fill_(np.nan)
        B.set(scene["dsecs"], [it])
        B.launch()
        torch.cuda.synchronize()
        assert torch.equal(it.image, img)
        if res is not None:
            assert torch.equal(it.result, res)


def test_batch_items_against_the_oracle(dev, scene):
    """Every item's images, and every tracking item's loss and pose gradient,
    against the oracle composited and differentiated along the GPU's own
    decisions (the Eq. 1 loss and its image gradient by the oracle from the
    item's rendered images)."""
    items = _items(scene, dev, MIX)
    B = _runner(scene)
    B.set(scene["dsecs"], items)
    B.launch()
    torch.cuda.synchronize()
    for k, it in enumerate(items):
        osec = scene["osecs"][it.section]
        P = api.matrix_of(it.pose)
        ids, cnt = G.decisions([scene["dsecs"][it.section]], it.pose, it.K, it.W, it.H)
        ref = oracle.render_lists([osec], P, it.K, it.W, it.H, ids, cnt)
        G.check_decisions(ref, f"batch_item_{k}")
        img = it.image
        G.assert_forward_close((img[:3], img[3], img[4]), ref)
        if not it.track:
            continue
        im = img.cpu().numpy()
        ob = it.obs.cpu().numpy()
        loss, d_rgb, d_depth = oracle.masked_l1(im[:3], im[3], im[4], ob[:3], ob[3], W_RGB,
                                                W_DEPTH, sil_min=SIL_MIN, rgb_needs_depth=True)
        r = it.result.cpu().numpy()
        assert r[0] == pytest.approx(loss, rel=1e-12)
        want = oracle.backward_lists([osec], P, it.K, it.W, it.H, ids, cnt, g_rgb=d_rgb,
                                     g_depth=d_depth)
        G.assert_grad_close(r[1:7], want["twist"], name="twist", noise=want["twist_noise"])
        G.assert_grad_close(r[7:19], want["mat"], name="mat", noise=want["mat_noise"])


def test_captured_launch_replays_other_batches(dev, scene):
    """The launch sequence captured once in a CUDA graph serves later
    batches of other compositions: each replay after vt_batch_set gives the
    eager results."""
    B = _runner(scene)
    first = _items(scene, dev, MIX[:2])
    B.set(scene["dsecs"], first)
    B.launch()                      # warm-up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.launch(stream=s)
    for mix in (MIX[2:], MIX[::-1], MIX[1:4]):
        items = _items(scene, dev, mix)
        B.set(scene["dsecs"], items)
        g.replay()
        torch.cuda.synchronize()
        B.status()
        for it in items:
            _check_item(it, _single(scene, it, dev), bit_exact_loss=False)


def test_batch_errors(dev, scene):
    B = _runner(scene)
    items = _items(scene, dev, MIX[:1])
    with pytest.raises(L.VTError) as e:
        B.set(scene["dsecs"], [api.BatchItem(5, False, 16, 16, (10.0, 10.0, 8.0, 8.0),
                                             items[0].pose, torch.zeros(5, 16, 16, device=dev))])
    assert e.value.status == L.VT_ERR_INVALID_ARG
    # an empty batch and more items than a table holds
    for bad in ([], items * 65):
        with pytest.raises(L.VTError) as e:
            B.set(scene["dsecs"], bad)
        assert e.value.status == L.VT_ERR_INVALID_ARG, len(bad)
    # an empty image: refused by the binding's shape check before the call
    with pytest.raises(ValueError):
        B.set(scene["dsecs"], [api.BatchItem(0, False, 0, 16, items[0].K, items[0].pose,
                                             torch.zeros(5, 16, 1, device=dev))])
    small = api.BatchRunner(max_gaussians=1000, max_pixels=1000, max_tiles=10,
                            max_instances=1000, max_views=4, max_table_rows=1000)
    with pytest.raises(L.VTError) as e:
        small.set(scene["dsecs"], items)
    assert e.value.status == L.VT_ERR_CAPACITY
    # instances beyond the reserve are found on the device and reported
    tight = api.BatchRunner(max_gaussians=4_000_000, max_pixels=400_000, max_tiles=4000,
                            max_instances=1000, max_views=64, max_table_rows=64 * 400)
    tight.set(scene["dsecs"], items)
    tight.launch()
    with pytest.raises(L.VTError) as e:
        tight.status()
    assert e.value.status == L.VT_ERR_CAPACITY
    fresh = api.BatchRunner(max_gaussians=1000, max_pixels=1000, max_tiles=10,
                            max_instances=1000, max_views=4, max_table_rows=1000)
    with pytest.raises(L.VTError) as e:
        fresh.launch()
    assert e.value.status == L.VT_ERR_STATE
