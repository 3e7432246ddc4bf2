"""Overlap-section selection (Sec. 3.3) through the CUDA path: per-view
visibility counts against the oracle (exact integers), the candidate rule,
and pre-tracking."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api, overlap
from paper_2506_02741_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _sections(dev, K, n_secs=4, per=5):
    room = syn.make_room(syn.SCENE_SEED)
    path = syn.trajectory(n_secs * per + 3)
    fr = syn.render_frames(room, K, path[: n_secs * per + 3])
    secs = []
    for s in range(n_secs):
        sl = slice(s * per, (s + 1) * per)
        secs.append(api.Section.from_rgbd(torch.from_numpy(fr.depth[sl]).to(dev),
                                          torch.from_numpy(fr.rgb[sl]).to(dev), K.astuple(),
                                          np.stack(path[sl])))
    head = n_secs * per + 2
    return secs, fr, path, head


def test_counts_and_selection(dev):
    K = syn.TINY
    secs, fr, path, head = _sections(dev, K)
    d = fr.depth[head]
    start = syn.perturb_pose(path[head], np.random.default_rng(2))
    cands = overlap.candidate_views(secs, every=2)          # 10 candidates: two launches
    assert len(cands) == 10
    views = [(secs[s].depth[k], K.astuple(), secs[s].poses[k]) for s, k in cands]
    counts, n_valid = api.visibility_counts(torch.from_numpy(d).to(dev), K.astuple(),
                                            api.pose12(start, dev), views)
    want = [int(oracle.visibility(d, K.astuple(), start,
                                  [(fr.depth[5 * s + k], K.astuple(), path[5 * s + k])]).sum())
            for s, k in cands]
    np.testing.assert_array_equal(counts, want)
    assert n_valid == int((np.isfinite(d) & (d > 0)).sum())
    frac = np.array(want) / n_valid
    gammas = (0.0, float(np.median(frac)), float(frac.max()) + 1e-3)
    for gamma in gammas:
        chosen, per = overlap.select_candidates(torch.from_numpy(d).to(dev), start, K.astuple(),
                                                secs, gamma=gamma, every=2)
        rule = sorted({s for (s, _), f in zip(cands, frac) if f > gamma})[:3]
        assert chosen == rule
        assert len(chosen) == {gammas[0]: 3, gammas[2]: 0}.get(gamma, len(chosen))


def test_pretrack_picks_the_smallest_loss(dev):
    """The candidates tracked together as one batched workload give the
    poses and losses of tracking them one after the other (the same pose
    gradients up to FP32 rounding, the same Adam steps); the section with
    the smallest loss is picked."""
    K = syn.TINY
    secs, fr, path, head = _sections(dev, K)
    start = syn.perturb_pose(path[head], np.random.default_rng(4))
    args = (secs, [1, 2, 3], torch.from_numpy(fr.rgb[head]).to(dev),
            torch.from_numpy(fr.depth[head]).to(dev), start, K.astuple(), K.W, K.H)
    best, res = overlap.pretrack(*args, iters=10, batched=True)
    best1, res1 = overlap.pretrack(*args, iters=10, batched=False)
    assert set(res) == set(res1) == {1, 2, 3}
    assert best == min(res, key=lambda s: res[s][0]) == best1
    for s in res:
        np.testing.assert_allclose(res[s][1], res1[s][1], rtol=0, atol=1e-7)
        assert res[s][0] == pytest.approx(res1[s][0], rel=1e-6)
    assert all(np.isfinite(v[0]) for v in res.values())
