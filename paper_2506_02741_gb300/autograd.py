"""torch.autograd wrapper of the vtsplat render.

``splat(sections, pose, K, W, H)`` returns (rgb, depth, silhouette) and
differentiates them with respect to the camera pose (the 12 entries of the
camera-to-world matrix, as Sec. 3.3 tracking needs) and to each section's
colour / opacity / radius tensors that require grad (Sec. 3.4 mapping: only
the learnable section does, the others stay frozen).

Each forward holds one render context (its workspace keeps the tile lists
and per-pixel lists for the backward) until its backward runs.  With
``recompute=True`` the forward keeps nothing: the backward renders again
(projection, binning and sort included) into a shared context and then runs
the backward, trading time for the memory of the kept workspaces.  The
render is deterministic, so both give the same gradients.
"""

from __future__ import annotations

import threading

import torch

from . import api


class RendererPool:
    """Render contexts handed out to outstanding forwards."""

    def __init__(self):
        self._free = []
        self._lock = threading.Lock()
        self.shared = None

    def acquire(self) -> api.Renderer:
        with self._lock:
            return self._free.pop() if self._free else api.Renderer()

    def release(self, r: api.Renderer):
        with self._lock:
            self._free.append(r)

    def shared_renderer(self) -> api.Renderer:
        with self._lock:
            if self.shared is None:
                self.shared = api.Renderer()
            return self.shared


_default_pool = RendererPool()


class VTSplatFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pool, sections, K, W, H, recompute, pose12, *attrs):
        R = pool.shared_renderer() if recompute else pool.acquire()
        rgb, depth, sil = R.render(sections, pose12.detach(), K, W, H, checked=True)
        ctx.pool, ctx.sections, ctx.geom = pool, sections, (tuple(K), int(W), int(H))
        ctx.recompute = recompute
        ctx.R = None if recompute else R
        ctx.save_for_backward(pose12, *attrs)
        return rgb, depth, sil

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_sil):
        pose12, *attrs = ctx.saved_tensors
        K, W, H = ctx.geom
        if ctx.recompute:
            R = ctx.pool.shared_renderer()
            R.render(ctx.sections, pose12.detach(), K, W, H, checked=True)
        else:
            R = ctx.R
        need_pose = ctx.needs_input_grad[6]
        need_attr = ctx.needs_input_grad[7:]
        grads = []
        any_attr = False
        for s, sec in enumerate(ctx.sections):
            if any(need_attr[3 * s: 3 * s + 3]):
                any_attr = True
                dev = sec.colour.device
                grads.append((torch.zeros(sec.n, 3, device=dev), torch.zeros(sec.n, device=dev),
                              torch.zeros(sec.n, device=dev)))
            else:
                grads.append(None)
        c = lambda g: None if g is None else g.contiguous()
        d_mat = None
        if need_pose or any_attr:
            _, d_mat = R.backward(c(g_rgb), c(g_depth), c(g_sil),
                                  attr_grads=grads if any_attr else None, pose_grad=need_pose)
        if not ctx.recompute:
            ctx.pool.release(R)
            ctx.R = None
        out = []
        for s, sec in enumerate(ctx.sections):
            g = grads[s]
            for k, t in enumerate((sec.colour, sec.opacity, sec.radius)):
                out.append(g[k].to(t.dtype) if g is not None and need_attr[3 * s + k] else None)
        d_pose = d_mat.to(pose12.dtype) if need_pose else None
        return (None, None, None, None, None, None, d_pose, *out)


def splat(sections, pose12: torch.Tensor, K, W: int, H: int, recompute: bool = False,
          pool: RendererPool | None = None):
    """Differentiable render of ``sections`` (a Section or a list of them)
    from ``pose12`` ((12,) float64: R row-major, then t).  Returns (rgb
    (3,H,W), depth (H,W), silhouette (H,W)) float32."""
    if isinstance(sections, api.Section):
        sections = [sections]
    attrs = []
    for s in sections:
        attrs += [s.colour, s.opacity, s.radius]
    return VTSplatFunction.apply(pool or _default_pool, list(sections), tuple(K), int(W), int(H),
                                 bool(recompute), pose12, *attrs)
