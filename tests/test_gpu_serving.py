"""Serving loop: every request's result is the same alone and in the mix
(render images and pose gradients bit-identical: the kernels are
deterministic for these outputs), with and without CUDA graphs."""

import numpy as np
import pytest
import torch

from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import serving
from paper_2506_02741_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _setup(dev, prec="f16"):
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(30)
    sections, poses = [], []
    for k, (W, H, nv) in enumerate(((160, 120, 2), (96, 72, 3), (200, 150, 1))):
        K = syn.scaled_intrinsics(W, H)
        keys = [path[5 * k + 3 * j] for j in range(nv)]
        fr = syn.render_frames(room, K, keys)
        sections.append(api.Section.from_rgbd(torch.from_numpy(fr.depth).to(dev),
                                              torch.from_numpy(fr.rgb).to(dev), K.astuple(),
                                              np.stack(keys), precision=prec))
        poses.append([syn.perturb_pose(keys[0], np.random.default_rng(k + 10 * j)) for j in range(3)])
    resolutions = [(160, 120), (320, 240)]
    obs = []
    for W, H in resolutions:
        d, c = syn.raycast(room, syn.scaled_intrinsics(W, H), path[7])
        obs.append((torch.from_numpy(c).to(dev), torch.from_numpy(d).to(dev)))
    return sections, poses, resolutions, obs


@pytest.mark.parametrize("graphs", [True, False])
def test_alone_equals_in_mix(graphs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    sections, poses, res, obs = _setup(dev)
    reqs = serving.poisson_requests(40, 4000.0, len(sections), len(res), poses, seed=5)
    mix = serving.Server(sections, res, obs, n_slots=3, graphs=graphs)
    mix.warm(reqs)
    done = mix.run(reqs)
    assert len(done) == len(reqs) and all(r.done >= r.arrival for r in done)
    alone = serving.Server(sections, res, obs, n_slots=1, graphs=graphs)
    alone.warm(reqs)
    by_id = {r.rid: r for r in done}
    for r in reqs[:15]:
        solo = serving.Request(r.rid, r.kind, r.section, r.pose, r.bucket, arrival=0.0)
        (out,) = alone.run([solo])
        assert torch.equal(out.result, by_id[r.rid].result), (r.rid, r.kind)
    s = serving.latency_summary(done, res)
    assert s["p99_ms"] >= s["p50_ms"] > 0
