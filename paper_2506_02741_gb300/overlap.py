"""Overlap-section selection for a head frame (Sec. 3.3).

A head frame starting a new section is tracked against an earlier,
overlapping section S^o.  Candidates are every N1-th frame of the sequence
(N1 = 5); the head frame's depth, back-projected with its initial pose, is
checked against each candidate view (vt_visibility_counts), the views that
see more than gamma of the valid points are kept, and the three most front
sections (the earliest, which carry the least accumulated drift) holding one
of them go to pre-tracking: each is tracked for a few iterations and the one
with the smallest rendering error becomes S^o.

Readings: gamma is a fraction of the head frame's valid depth pixels (the
supplementary's 0.24 - 0.26); "rendering error" is the Eq. 1 loss after the
pre-tracking iterations.
"""

from __future__ import annotations

import torch

from . import api
from .tracking import PoseTracker


def candidate_views(sections, every: int = 5, first_frame: int = 0):
    """(section index, view index) of every ``every``-th frame, the sections
    holding consecutive frames in order starting at ``first_frame``."""
    out, f = [], first_frame
    for s, sec in enumerate(sections):
        for k in range(sec.n_views):
            if f % every == 0:
                out.append((s, k))
            f += 1
    return out


def select_candidates(head_depth, head_pose, K, sections, gamma: float = 0.25, every: int = 5,
                      n_pick: int = 3, rel_tol: float = 0.01):
    """The (up to n_pick) earliest sections holding a candidate view that sees
    more than gamma of the head frame's valid points.  Returns (section
    indices, per-candidate (section, view, fraction))."""
    cands = candidate_views(sections, every)
    views = [(sections[s].depth[k], sections[s].K, sections[s].poses[k]) for s, k in cands]
    counts, n_valid = api.visibility_counts(head_depth, K, head_pose, views, rel_tol)
    frac = counts / max(n_valid, 1)
    chosen = sorted({s for (s, _), f in zip(cands, frac) if f > gamma})
    return chosen[:n_pick], [(s, k, float(f)) for (s, k), f in zip(cands, frac)]


def pretrack(sections, chosen, head_rgb, head_depth, pose0, K, W: int, H: int, iters: int = 20,
             lr_rot: float = 4e-4, lr_trans: float = 2e-3, batched: bool = True):
    """Track the head frame against each chosen section for ``iters``
    iterations; returns (index of the section with the smallest final Eq. 1
    loss, {section index: (loss, pose (12,))}).

    batched: the candidates are tracked together as one workload -- every
    iteration is one batch of tracking items (vt_batch_launch: one launch per
    stage for all candidates) followed by each candidate's Adam step; the
    pose gradients are those of the one-at-a-time form up to FP32 rounding.
    batched=False tracks one candidate after the other."""
    if not chosen:
        return None, {}
    if not batched:
        results = {}
        for s in chosen:
            R = api.Renderer()
            tr = PoseTracker(R, [sections[s]], K, W, H, pose0, lr_rot=lr_rot, lr_trans=lr_trans,
                             device=head_depth.device)
            tr.set_target(head_rgb, head_depth)
            for _ in range(iters):
                loss = tr.step()
            results[s] = (float(loss.item()), tr.pose.detach().cpu().numpy().copy())
            R.close()
        best = min(results, key=lambda s: results[s][0])
        return best, results
    dev = head_depth.device
    secs = [sections[s] for s in chosen]
    n = len(secs)
    obs = torch.cat([head_rgb, head_depth[None]]).contiguous()
    poses = api.pose12(pose0, dev).repeat(n, 1).contiguous()
    state = torch.zeros(n, 15, dtype=torch.float64, device=dev)
    result = torch.zeros(n, 19, dtype=torch.float64, device=dev)
    image = torch.empty(n, 5, H, W, device=dev)
    items = [api.BatchItem(i, True, W, H, tuple(K), poses[i], image[i], obs, result[i])
             for i in range(n)]
    g = sum((s.n + 255) // 256 * 256 for s in secs)
    tiles = n * ((W + 15) // 16) * ((H + 15) // 16)
    views = sum(s.n_views for s in secs)
    rows = sum(s.n_views * (s.depth.shape[-1] + s.depth.shape[-2]) for s in secs)
    inst = 8 * g + 65536
    lr = [float(lr_trans)] * 3 + [float(lr_rot)] * 3
    while True:
        runner = api.BatchRunner(g, n * ((W * H + 255) // 256 * 256), tiles, inst, views, rows)
        runner.set(secs, items)
        runner.launch()
        need = runner.needed_instances()
        if need <= inst:
            break
        inst = int(1.25 * need) + 65536        # the first launch told the size: again
    for it in range(iters):
        if it:
            runner.launch()
        for i in range(n):                     # Adam step and retraction per candidate
            api.pose_adam(poses[i], result[i, 1:7], state[i], lr, renderer=runner)
    out = result[:, 0].cpu().numpy()
    pp = poses.cpu().numpy()
    results = {s: (float(out[i]), pp[i].copy()) for i, s in enumerate(chosen)}
    runner.close()
    best = min(results, key=lambda s: results[s][0])
    return best, results
