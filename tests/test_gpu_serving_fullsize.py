"""Serving at the benchmark's full sizes: the largest section size of the
serving workload (28 views of 640x480, 8.6 M Gaussians in FP16) served at
1920x1080 together with small requests, through the batch server in the
launch configuration bench.py times.  The served colour image of a
1920x1080 render request is checked against the oracle on a crop (along the
GPU's decisions, given the Gaussians that can reach the crop); the served
loss and pose gradient of a 1920x1080 track request against the
single-request calls, which the full-size tests check against the oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import serving
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G
from tests.test_gpu_fullsize import _crop, _crop_subset

pytestmark = pytest.mark.gpu

BIG, SMALL = (1920, 1080), (320, 240)
N_VIEWS = 28


def _workload(dev):
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(200)
    keys = [path[4 * j] for j in range(N_VIEWS)]
    fr = syn.render_frames(room, syn.VGA, keys)
    osec = G.quantise(oracle.section_init(fr.depth, fr.rgb, syn.VGA.astuple(), np.stack(keys)),
                      "f16")
    dsec = G.to_device(osec, "f16", dev)
    poses = [syn.perturb_pose(keys[-1], np.random.default_rng(50 + j)) for j in range(3)]
    obs = {}
    for b, (W, H) in enumerate((BIG, SMALL)):
        d, c = syn.raycast(room, syn.scaled_intrinsics(W, H), path[4 * N_VIEWS - 2])
        obs[b] = torch.from_numpy(np.concatenate([c, d[None]]).astype(np.float32)).pin_memory()
    return osec, dsec, poses, obs


def test_served_fullsize_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    osec, dsec, poses, obs = _workload(dev)
    Req = serving.Request
    reqs = [Req(0, "render", 0, poses[0], 0), Req(1, "track", 0, poses[1], 0, obs=obs[0]),
            Req(2, "render", 0, poses[2], 1), Req(3, "track", 0, poses[0], 1, obs=obs[1]),
            Req(4, "render", 0, poses[1], 0)]
    server = serving.BatchServer([dsec], [BIG, SMALL])
    server.warm(reqs)
    done = {r.rid: r for r in server.run(reqs)}
    assert sorted(done) == [0, 1, 2, 3, 4]
    W, H = BIG
    K = syn.scaled_intrinsics(W, H)
    Kt = K.astuple()

    # render request: bit-identical to vt_render, and a crop against the oracle
    R = api.Renderer()
    rgb, _, _ = R.render([dsec], api.pose12(poses[0], dev), Kt, W, H, checked=True)
    assert torch.equal(done[0].result, rgb.cpu())
    cw, ch = 96, 80
    x0, y0 = (W - cw) // 2 + 40, (H - ch) // 2 + 24
    sub, keep = _crop_subset(osec, poses[0], K, (x0, y0, cw, ch))
    ids, cnt = G.decisions([dsec], api.pose12(poses[0], dev), Kt, W, H, box=(x0, y0, cw, ch),
                           id_map=G.subset_map([keep]), cap=1024)
    ref = oracle.render_lists([sub], poses[0], _crop(K, x0, y0), cw, ch, ids, cnt)
    G.check_decisions(ref, "served_1920x1080_render")
    got = done[0].result[:, y0:y0 + ch, x0:x0 + cw].numpy().astype(np.float64)
    bound = 1e-5 * np.maximum(np.abs(ref["rgb"]), 1.0)
    err = np.abs(got - ref["rgb"])
    print("PARITY_ERROR", dict(case="served_1920x1080_render", tensor="rgb",
                               ratio=float((err / bound).max())))
    assert (err <= bound).all(), float((err / bound).max())

    # track request: the single-request calls' loss and pose gradient
    R = api.Renderer()
    rgb, depth, sil = R.render([dsec], api.pose12(poses[1], dev), Kt, W, H, checked=True)
    ob = obs[0].to(dev)
    g_rgb = torch.zeros(3, H, W, device=dev)
    g_depth = torch.zeros(H, W, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    R.masked_l1(rgb, depth, sil, ob[:3], ob[3], 0.5, 0.025, sil_min=0.99, rgb_needs_depth=True,
                d_rgb=g_rgb, d_depth=g_depth, loss=loss)
    tw, mat = R.backward(g_rgb, g_depth, None, pose_grad=True)
    torch.cuda.synchronize()
    r = done[1].result.numpy()
    assert r[0] == pytest.approx(loss.item(), rel=1e-12)
    for g, w in ((r[1:7], tw.cpu().numpy()), (r[7:19], mat.cpu().numpy())):
        np.testing.assert_allclose(g, w, rtol=1e-5, atol=1e-6 * np.abs(w).max())
