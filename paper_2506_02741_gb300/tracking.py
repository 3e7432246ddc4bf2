"""Camera tracking loop (Sec. 3.3): optimise the pose of the latest frame
against fixed Gaussians by minimising Eq. 1,

    alpha * W |V - V'|_1 + beta * W |D - D'|_1,

with W masking pixels without depth, not covered by the render (here:
silhouette > 0.99) or, when a visibility mask is given (head frames tracked
against an overlapping section, Sec. 3.3), invisible to that section.  Every
step of an iteration runs in the vtsplat kernels on the device, with no host
synchronisation: render, the masked L1 loss and its image gradient
(vt_masked_l1), the pose backward and the Adam step with the retraction
(vt_pose_adam).

The L1 norms are averaged over the pixels (a reading: the paper writes
||.||_1 without a normaliser).  Pose updates are right-multiplicative,
P <- P Exp(-step), matching the twist gradient of vt_render_backward.
"""

from __future__ import annotations

import numpy as np
import torch

from . import api


class PoseTracker:
    """Adam on the pose twist (learning rates per rotation / translation,
    supplementary: lr_rot, lr_trans)."""

    def __init__(self, renderer: api.Renderer, sections, K, W: int, H: int, pose0,
                 lr_rot: float = 4e-4, lr_trans: float = 2e-3, alpha: float = 0.5,
                 beta: float = 0.025, device="cuda"):
        self.R = renderer
        self.sections = sections
        self.K, self.W, self.H = tuple(K), int(W), int(H)
        self.pose = api.pose12(pose0, device)
        self.alpha, self.beta = float(alpha), float(beta)
        self.lr = [float(lr_trans)] * 3 + [float(lr_rot)] * 3
        self.state = torch.zeros(15, dtype=torch.float64, device=device)   # Adam m, v, t, b^t
        self.d_twist = torch.zeros(6, dtype=torch.float64, device=device)
        self.rgb = torch.empty(3, H, W, device=device)
        self.depth = torch.empty(H, W, device=device)
        self.sil = torch.empty(H, W, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.g_rgb = torch.zeros(3, H, W, device=device)
        self.g_depth = torch.zeros(H, W, device=device)
        self.obs_rgb = torch.zeros(3, H, W, device=device)
        self.obs_depth = torch.zeros(H, W, device=device)
        self.visible = None
        self.graph = None

    def set_target(self, rgb: torch.Tensor, depth: torch.Tensor, visible=None):
        """Copy the observed frame (and optionally a visibility mask (H, W)
        uint8 from api.visibility) into the tracker's fixed buffers.  Whether
        a mask is used is fixed by the first call before capture()."""
        self.obs_rgb.copy_(rgb, non_blocking=True)
        self.obs_depth.copy_(depth, non_blocking=True)
        if visible is not None:
            if self.visible is None:
                self.visible = torch.empty_like(visible)
            self.visible.copy_(visible, non_blocking=True)

    def reset_optimiser(self):
        self.state.zero_()

    def step(self):
        """One tracking iteration: render, Eq. 1 loss and its image gradient,
        pose backward, Adam step and retraction.  All on the device."""
        self.R.render(self.sections, self.pose, self.K, self.W, self.H, self.rgb, self.depth,
                      self.sil)
        self.R.masked_l1(self.rgb, self.depth, self.sil, self.obs_rgb, self.obs_depth,
                         self.alpha, self.beta, sil_min=0.99, rgb_needs_depth=True,
                         visible=self.visible, d_rgb=self.g_rgb, d_depth=self.g_depth,
                         loss=self.loss)
        # d_twist was zeroed by the previous Adam step (and at construction)
        self.R.backward(self.g_rgb, self.g_depth, None, pose_grad=True, d_twist=self.d_twist)
        api.pose_adam(self.pose, self.d_twist, self.state, self.lr, renderer=self.R)
        return self.loss

    def capture(self, warmup: int = 3):
        """Record one step() in a CUDA graph (the renderer's workspace must be
        reserved first: a captured render allocates nothing).  Afterwards
        replay() runs the step with one launch; the pose, optimiser state and
        observation buffers are updated in place."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.loss


class HostPipeline:
    """Tracking iterations fed from pinned host memory, with each iteration's
    pose and loss read back on the host, and the copies overlapped with the
    compute of the neighbouring iterations.

    step(rgb, depth) uploads the observed frame on a copy stream into one of
    two device staging buffers (while the previous iteration still runs) and
    replays the CUDA graph of that buffer: the copy of the staged frame into
    the tracker's observation buffers, the tracking iteration and the copy of
    (pose, loss) to a result buffer; the read-back of that buffer to pinned
    memory follows.  It then waits for the previous iteration's read-back and
    returns that iteration's 13 values (12 pose entries, loss) as a float64
    NumPy array: results arrive one step late, so the host issues iteration
    i + 1 while the device computes iteration i.  flush() returns the last
    one.  The tracker must have been captured once (PoseTracker.capture: it
    warms the step up and shows that it is capture-safe)."""

    def __init__(self, tracker: PoseTracker):
        if tracker.graph is None:
            raise RuntimeError("HostPipeline needs a captured tracker (call capture() first)")
        self.tr = tracker
        dev = tracker.obs_rgb.device
        self.copy_stream = torch.cuda.Stream(dev)
        self.stage = [(torch.empty_like(tracker.obs_rgb), torch.empty_like(tracker.obs_depth))
                      for _ in range(2)]
        self.res = [torch.empty(13, dtype=torch.float64, device=dev) for _ in range(2)]
        self.host = [torch.empty(13, dtype=torch.float64).pin_memory() for _ in range(2)]
        self.staged = [torch.cuda.Event() for _ in range(2)]     # upload into stage k done
        self.consumed = [torch.cuda.Event() for _ in range(2)]   # graph k done with stage k
        self.ready = [torch.cuda.Event() for _ in range(2)]      # read-back k done
        self.used = [False, False]
        self.graphs = []
        for k in range(2):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                tracker.obs_rgb.copy_(self.stage[k][0])
                tracker.obs_depth.copy_(self.stage[k][1])
                loss = tracker.step()
                self.res[k][:12].copy_(tracker.pose)
                self.res[k][12:].copy_(loss)
            self.graphs.append(g)
        self.pending = None
        self.i = 0

    def step(self, rgb: torch.Tensor, depth: torch.Tensor):
        k = self.i & 1
        main = torch.cuda.current_stream()
        cs = self.copy_stream
        if self.used[k]:
            cs.wait_event(self.consumed[k])
        with torch.cuda.stream(cs):
            self.stage[k][0].copy_(rgb, non_blocking=True)
            self.stage[k][1].copy_(depth, non_blocking=True)
            self.staged[k].record(cs)
        main.wait_event(self.staged[k])
        self.graphs[k].replay()
        self.consumed[k].record(main)
        self.used[k] = True
        self.host[k].copy_(self.res[k], non_blocking=True)
        self.ready[k].record(main)
        out = self._collect()
        self.pending = k
        self.i += 1
        return out

    def _collect(self):
        if self.pending is None:
            return None
        j = self.pending
        self.ready[j].synchronize()
        self.pending = None
        return self.host[j].numpy().copy()

    def flush(self):
        """Result of the last step() (None if there is none pending)."""
        return self._collect()


def pose_error(P, Q):
    """(translation error m, rotation error deg) between two (3,4) poses."""
    P = api.matrix_of(P) if not isinstance(P, np.ndarray) or P.shape == (12,) else P
    Q = api.matrix_of(Q) if not isinstance(Q, np.ndarray) or Q.shape == (12,) else Q
    dt = float(np.linalg.norm(P[:, 3] - Q[:, 3]))
    dR = P[:, :3].T @ Q[:, :3]
    ang = float(np.degrees(np.arccos(np.clip((np.trace(dR) - 1) / 2, -1, 1))))
    return dt, ang
