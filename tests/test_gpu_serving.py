"""Serving loops: every request's result is the same alone and in the mix
(render images and tracking results bit-identical: the kernels are
deterministic for these outputs), with and without CUDA graphs, for the
batched server and the slot server; served results against the oracle on a
sample; admission under a small memory budget."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import serving
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G

pytestmark = pytest.mark.gpu

RES = [(160, 120), (320, 240), (96, 72)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def setup(dev):
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(30)
    sections, osecs, poses = [], [], []
    for k, (W, H, nv) in enumerate(((160, 120, 2), (96, 72, 3), (200, 150, 1))):
        K = syn.scaled_intrinsics(W, H)
        keys = [path[5 * k + 3 * j] for j in range(nv)]
        fr = syn.render_frames(room, K, keys)
        osec = G.quantise(oracle.section_init(fr.depth, fr.rgb, K.astuple(), np.stack(keys)), "f16")
        osecs.append(osec)
        sections.append(G.to_device(osec, "f16"))
        poses.append([syn.perturb_pose(keys[0], np.random.default_rng(k + 10 * j)) for j in range(3)])
    frames = []
    for W, H in RES:
        fb = []
        for i in (7, 9):
            d, c = syn.raycast(room, syn.scaled_intrinsics(W, H), path[i])
            fb.append(torch.from_numpy(np.concatenate([c, d[None]]).astype(np.float32)).pin_memory())
        frames.append(fb)
    return sections, osecs, poses, frames


def _requests(setup, n=40, seed=5, rate=4000.0):
    sections, _, poses, frames = setup
    return serving.poisson_requests(n, rate, len(sections), len(RES), poses, seed=seed,
                                    frames=frames)


def _solo(r):
    return serving.Request(r.rid, r.kind, r.section, r.pose, r.bucket, arrival=0.0, obs=r.obs)


@pytest.mark.parametrize("graphs", [True, False])
def test_batched_alone_equals_in_mix(dev, setup, graphs):
    """Batched launches only: a request gives the same bits as a one-item
    batch as inside a mix."""
    reqs = _requests(setup)
    server = serving.BatchServer(setup[0], RES, n_contexts=2, graphs=graphs,
                                 memory_budget=8 << 30, solo=False)
    server.warm(reqs)
    done = server.run(reqs)
    assert len(done) == len(reqs) and all(r.done >= r.arrival for r in done)
    assert server.n_solo == 0 and server.n_batched == len(reqs)
    by_id = {r.rid: r for r in done}
    for r in reqs[:12]:
        (out,) = server.run([_solo(r)])
        assert torch.equal(out.result, by_id[r.rid].result), (r.rid, r.kind)
    s = serving.latency_summary(done, RES)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def _close_track(a, b):
    """Tracking results of the single-request kernels against the batched
    ones: the loss within FP64 rounding of another fixed order of the same
    block sums, the pose gradient within FP32 rounding (the same terms in the
    same order; the compiler may contract a product and a sum differently in
    the two instantiations)."""
    a, b = a.numpy(), b.numpy()
    assert a[0] == pytest.approx(b[0], rel=1e-13, abs=1e-300)
    np.testing.assert_allclose(a[1:7], b[1:7], rtol=1e-6, atol=1e-7 * np.abs(b[1:7]).max())
    np.testing.assert_allclose(a[7:], b[7:], rtol=1e-6, atol=1e-7 * np.abs(b[7:]).max())


@pytest.mark.parametrize("graphs", [True, False])
def test_lone_requests_take_the_single_request_path(dev, setup, graphs):
    """With the single-request renderers a request served alone takes them;
    its colour image equals the batched one bit for bit, its tracking result
    agrees within rounding."""
    reqs = _requests(setup)
    batched = serving.BatchServer(setup[0], RES, n_contexts=2, graphs=graphs,
                                  memory_budget=8 << 30, solo=False)
    batched.warm(reqs)
    server = serving.BatchServer(setup[0], RES, n_contexts=2, graphs=graphs,
                                 memory_budget=8 << 30)
    server.warm(reqs)
    done = server.run(reqs)
    assert len(done) == len(reqs)
    for r in reqs[:12]:
        (a,) = server.run([_solo(r)])
        (b,) = batched.run([_solo(r)])
        if r.kind == "render":
            assert torch.equal(a.result, b.result), r.rid
        else:
            _close_track(a.result, b.result)
    assert server.n_solo >= 12


def test_warm_up_prepares_every_combination(dev, setup):
    """Warm-up with requests of one section and bucket: time estimates and
    single-request graphs exist for every (section, bucket, kind), so a
    request of another combination served alone captures nothing; its
    result equals the batched path's."""
    reqs = [r for r in _requests(setup) if r.section == 0 and r.bucket == 0]
    assert reqs
    server = serving.BatchServer(setup[0], RES, n_contexts=2, memory_budget=8 << 30)
    server.warm(reqs)
    every = {(s, b, k) for s in range(len(setup[0])) for b in range(len(RES))
             for k in ("render", "track")}
    assert set(server.ms_est) == every
    for ctx in server.ctxs:
        assert set(ctx.solo.works) == every
        assert all(w.graph is not None for w in ctx.solo.works.values())
    sections, _, poses, frames = setup
    other = serving.Request(0, "render", 2, poses[2][1], 1)
    graphs_before = [id(w.graph) for c in server.ctxs for w in c.solo.works.values()]
    (a,) = server.run([other])
    assert [id(w.graph) for c in server.ctxs for w in c.solo.works.values()] == graphs_before
    batched = serving.BatchServer(setup[0], RES, n_contexts=1, memory_budget=8 << 30, solo=False)
    batched.warm(reqs)
    (b,) = batched.run([serving.Request(0, "render", 2, poses[2][1], 1)])
    assert torch.equal(a.result, b.result)


@pytest.mark.parametrize("graphs", [True, False])
def test_slot_server_alone_equals_in_mix(dev, setup, graphs):
    reqs = _requests(setup, n=30)
    mix = serving.SlotServer(setup[0], RES, n_slots=3, graphs=graphs)
    mix.warm(reqs)
    done = mix.run(reqs)
    alone = serving.SlotServer(setup[0], RES, n_slots=1, graphs=graphs)
    alone.warm(reqs)
    by_id = {r.rid: r for r in done}
    for r in reqs[:10]:
        (out,) = alone.run([_solo(r)])
        assert torch.equal(out.result, by_id[r.rid].result), (r.rid, r.kind)


def test_served_results_against_the_oracle(dev, setup):
    """A sample of served results: render requests' colour images and
    tracking requests' loss and pose gradient against the oracle along the
    GPU's decisions (the loss and its image gradient by the oracle from the
    request's rendered images)."""
    sections, osecs, _, _ = setup
    reqs = _requests(setup, n=24, seed=9)
    server = serving.BatchServer(sections, RES, n_contexts=2, graphs=True, memory_budget=8 << 30)
    server.warm(reqs)
    done = server.run(reqs)
    checked = {"render": 0, "track": 0}
    for r in done:
        if checked[r.kind] >= 3:
            continue
        checked[r.kind] += 1
        W, H = RES[r.bucket]
        K = server.intrinsics[r.bucket]
        pose = api.pose12(r.pose, dev)
        R = api.Renderer()
        rgb, depth, sil = R.render([sections[r.section]], pose, K, W, H, checked=True)
        ids, cnt = G.gpu_lists(R, W, H)
        ref = oracle.render_lists([osecs[r.section]], r.pose, K, W, H, ids, cnt)
        G.check_decisions(ref, f"served_{r.kind}_{r.rid}")
        if r.kind == "render":
            assert torch.equal(r.result, rgb.cpu())
            G.assert_forward_close((r.result, depth, sil), ref)
            continue
        ob = r.obs.numpy()
        loss, d_rgb, d_depth = oracle.masked_l1(rgb.cpu().numpy(), depth.cpu().numpy(),
                                                sil.cpu().numpy(), ob[:3], ob[3], 0.5, 0.025,
                                                sil_min=0.99, rgb_needs_depth=True)
        got = r.result.numpy()
        assert got[0] == pytest.approx(loss, rel=1e-12)
        want = oracle.backward_lists([osecs[r.section]], r.pose, K, W, H, ids, cnt, g_rgb=d_rgb,
                                     g_depth=d_depth)
        G.assert_grad_close(got[1:7], want["twist"], name="twist", noise=want["twist_noise"])
    assert checked["render"] > 0 and checked["track"] > 0


def test_admission_under_a_small_budget(dev, setup):
    """With capacity for about one request per context the server still
    serves every request (the rest wait for room); a request that can never
    fit a context is refused before anything runs."""
    sections = setup[0]
    reqs = _requests(setup, n=20, seed=11, rate=1e6)
    server = serving.BatchServer(sections, RES, n_contexts=2, graphs=False,
                                 memory_budget=600 << 20, solo=False)
    server.warm(reqs)
    cap = server.ctxs[0].cap
    done = server.run(reqs)
    assert len(done) == len(reqs)
    small = [r for r in reqs if r.bucket != 1]
    tiny = serving.BatchServer(sections, RES[:1] + [(2000, 2000)] + RES[2:], n_contexts=1,
                               graphs=False, memory_budget=100 << 20, solo=False)
    tiny.warm(small)
    big = serving.Request(999, "render", 0, small[0].pose, 1, arrival=0.0)
    with pytest.raises(ValueError):
        tiny.run([big])
    assert cap["pixels"] >= max(W * H for W, H in RES)
