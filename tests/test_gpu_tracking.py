"""Camera tracking (Sec. 3.3, Eq. 1) through the CUDA path: the pose
converges towards the ground truth, and the CUDA-graph replay of a step is
bit-identical to the eager step (the pose reduction has a fixed order)."""

import numpy as np
import pytest
import torch

from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from paper_2506_02741_gb300.tracking import PoseTracker, pose_error

pytestmark = pytest.mark.gpu


def _setup(dev, n_key=4):
    K = syn.scaled_intrinsics(160, 120)
    room, section, target, gt, start = syn.tracking_workload(K, n_keyframes=n_key)
    sec = api.Section.from_rgbd(torch.from_numpy(section.depth).to(dev),
                                torch.from_numpy(section.rgb).to(dev), K.astuple(),
                                np.stack(section.poses))
    R = api.Renderer()
    tr = PoseTracker(R, [sec], K.astuple(), K.W, K.H, start, lr_rot=2e-3, lr_trans=2e-3,
                     device=dev)
    tr.set_target(torch.from_numpy(target.rgb[0]).to(dev), torch.from_numpy(target.depth[0]).to(dev))
    R.render([sec], tr.pose, K.astuple(), K.W, K.H, checked=True)
    R.reserve(sec.n, K.W, K.H, int(R.status() * 2) + 65536)
    return K, sec, R, tr, gt, start


def test_tracking_reduces_pose_error():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    K, sec, R, tr, gt, start = _setup(dev)
    e0 = pose_error(start, gt)
    losses = []
    for _ in range(150):
        losses.append(float(tr.step()))
    e1 = pose_error(api.matrix_of(tr.pose), gt)
    # Eq. 1 decreases and the translation error with it (at 160x120 the
    # rotation is only weakly observed: it may trade against translation)
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    assert e1[0] < e0[0] and e1[1] < 1.0, (e0, e1)


def test_graph_replay_matches_eager():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    K, sec, R, tr, gt, start = _setup(dev, n_key=2)
    p0 = api.pose12(start, dev)
    tr.capture(warmup=2)
    # eager
    tr.pose.copy_(p0)
    tr.reset_optimiser()
    for _ in range(5):
        tr.step()
    eager = tr.pose.clone()
    # replayed
    tr.pose.copy_(p0)
    tr.reset_optimiser()
    for _ in range(5):
        tr.replay()
    torch.cuda.synchronize()
    assert torch.equal(eager, tr.pose)


def test_host_pipeline_matches_synchronous_steps():
    """HostPipeline (frame uploads on a copy stream, results read one step
    late) returns, step by step, exactly the pose and loss of synchronous
    replays, across a change of the observed frame."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_02741_gb300.tracking import HostPipeline
    dev = torch.device("cuda:0")
    K, sec, R, tr, gt, start = _setup(dev, n_key=2)
    p0 = api.pose12(start, dev)
    tr.capture(warmup=2)
    obs_rgb0, obs_d0 = tr.obs_rgb.cpu(), tr.obs_depth.cpu()
    frames = [(obs_rgb0, obs_d0), (obs_rgb0.flip(-1).contiguous(), obs_d0.flip(-1).contiguous())]
    order = [0, 0, 0, 1, 1, 0, 1]
    # synchronous reference
    tr.pose.copy_(p0)
    tr.reset_optimiser()
    want = []
    for f in order:
        tr.set_target(frames[f][0].to(dev), frames[f][1].to(dev))
        loss = tr.replay()
        torch.cuda.synchronize()
        want.append(np.concatenate([tr.pose.cpu().numpy(), loss.cpu().numpy()]))
    # pipelined from pinned host memory
    pinned = [(a.pin_memory(), b.pin_memory()) for a, b in frames]
    tr.pose.copy_(p0)
    tr.reset_optimiser()
    pipe = HostPipeline(tr)
    got = []
    for f in order:
        r = pipe.step(*pinned[f])
        if r is not None:
            got.append(r)
    got.append(pipe.flush())
    assert pipe.flush() is None
    assert len(got) == len(want)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
