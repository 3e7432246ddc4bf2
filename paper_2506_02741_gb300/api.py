"""PyTorch-facing binding of the vtsplat C ABI.

Argument marshalling only: tensors are checked for device, dtype and shape
and their pointers are handed to the CUDA library on the current torch
stream.  Every step of the splatting path runs in the library's kernels.
"""

from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _intr(K) -> L.Intrinsics:
    fx, fy, cx, cy = (float(np.float32(k)) for k in K)
    return L.Intrinsics(fx, fy, cx, cy)


def _cuda(t: torch.Tensor, dtype, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def pose12(P, device="cuda") -> torch.Tensor:
    """(3, 4) or (V, 3, 4) camera-to-world pose(s) -> (12,) / (V, 12) float64
    on the device: R row-major, then t."""
    if isinstance(P, torch.Tensor):
        P = P.detach().to("cpu", torch.float64).numpy()
    p = np.asarray(P, np.float64)
    single = p.ndim == 2
    p = p.reshape(-1, 3, 4)
    flat = np.concatenate([p[:, :, :3].reshape(-1, 9), p[:, :, 3]], axis=1)
    t = torch.from_numpy(np.ascontiguousarray(flat)).to(device)
    return t[0].contiguous() if single else t.contiguous()


def matrix_of(p12) -> np.ndarray:
    """(12,) pose vector -> (3, 4) numpy matrix."""
    v = p12.detach().cpu().numpy() if isinstance(p12, torch.Tensor) else np.asarray(p12)
    return np.hstack([v[:9].reshape(3, 3), v[9:12].reshape(3, 1)])


@dataclasses.dataclass
class Section:
    """A device-resident section (Sec. 3.2): the Gaussians tied to the valid
    depth pixels of ``n_views`` views of one camera.

    poses (V, 12) float64, depth (V, H, W) float32, src (n,) int32 holding
    the uint32 source index (view*H + v)*W + u in increasing order,
    colour (n, 3), opacity (n,), radius (n,) in float32 or float16.  With
    scale (n, 3) and rot (n, 4) (same dtype) the Gaussians are ellipsoids
    (the anisotropic variant of the attribute ablation, Sec. 4): axis
    standard deviations and quaternions (w, x, y, z) in the source view's
    camera frame; the radius is then not used."""
    poses: torch.Tensor
    depth: torch.Tensor
    K: tuple
    src: torch.Tensor
    colour: torch.Tensor
    opacity: torch.Tensor
    radius: torch.Tensor
    scale: torch.Tensor | None = None
    rot: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_views(self) -> int:
        return int(self.depth.shape[0])

    @property
    def prec(self) -> int:
        return L.VT_F16 if self.colour.dtype == torch.float16 else L.VT_F32

    def validate(self):
        V, H, W = self.depth.shape
        _cuda(self.poses, torch.float64, "poses", (V, 12))
        _cuda(self.depth, torch.float32, "depth")
        _cuda(self.src, torch.int32, "src", (self.n,))
        dt = self.colour.dtype
        if dt not in (torch.float32, torch.float16):
            raise TypeError("attributes must be float32 or float16")
        _cuda(self.colour, dt, "colour", (self.n, 3))
        _cuda(self.opacity, dt, "opacity", (self.n,))
        _cuda(self.radius, dt, "radius", (self.n,))
        if (self.scale is None) != (self.rot is None):
            raise ValueError("scale and rot come together")
        if self.scale is not None:
            _cuda(self.scale, dt, "scale", (self.n, 3))
            _cuda(self.rot, dt, "rot", (self.n, 4))

    @property
    def ellipsoids(self) -> bool:
        return self.scale is not None

    def with_ellipsoids(self, scale, rot) -> "Section":
        """The same Gaussians as ellipsoids with the given axis scales (n, 3)
        and quaternions (n, 4), converted to the section's dtype and device
        (the other arrays are shared)."""
        dt, dev = self.colour.dtype, self.colour.device
        as_t = lambda a: (a if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a)))
        return dataclasses.replace(self, scale=as_t(scale).to(dev, dt).contiguous(),
                                   rot=as_t(rot).to(dev, dt).contiguous())

    def c_struct(self) -> L.SectionC:
        self.validate()
        V, H, W = self.depth.shape
        return L.SectionC(V, W, H, _intr(self.K), _ptr(self.poses), _ptr(self.depth), self.n,
                          _ptr(self.src), self.prec, _ptr(self.colour), _ptr(self.opacity),
                          _ptr(self.radius), _ptr(self.scale), _ptr(self.rot))

    @staticmethod
    def from_rgbd(depth: torch.Tensor, rgb: torch.Tensor, K, poses, precision: str = "f32",
                  stream=None) -> "Section":
        """Initialise a section on the device (one Gaussian per valid depth
        pixel, colour = V(u,v), opacity 0.9, radius D/fx).  Synchronises once
        to learn the count."""
        depth = _cuda(depth, torch.float32, "depth")
        V, H, W = depth.shape
        rgb = _cuda(rgb, torch.float32, "rgb", (V, 3, H, W))
        P = poses if isinstance(poses, torch.Tensor) and poses.dtype == torch.float64 and \
            poses.is_cuda else pose12(poses, depth.device)
        P = P.reshape(V, 12).contiguous()
        dt = torch.float16 if precision == "f16" else torch.float32
        cap = V * H * W
        dev = depth.device
        src = torch.empty(cap, dtype=torch.int32, device=dev)
        col = torch.empty(cap, 3, dtype=dt, device=dev)
        op = torch.empty(cap, dtype=dt, device=dev)
        rad = torch.empty(cap, dtype=dt, device=dev)
        n_out = torch.zeros(1, dtype=torch.int64, device=dev)
        L.check(L.lib().vt_section_init(_ptr(depth), _ptr(rgb), V, W, H, _intr(K),
                                        L.VT_F16 if dt == torch.float16 else L.VT_F32,
                                        _ptr(src), _ptr(col), _ptr(op), _ptr(rad), cap,
                                        _ptr(n_out), _stream(stream)), "vt_section_init")
        n = int(n_out.item())
        return Section(P, depth, tuple(float(np.float32(k)) for k in K), src[:n].contiguous(),
                       col[:n].contiguous(), op[:n].contiguous(), rad[:n].contiguous())

    def append_view(self, depth: torch.Tensor, rgb: torch.Tensor, pose, silhouette: torch.Tensor,
                    sil_max: float = 0.5, stream=None) -> "Section":
        """Complement initialisation of a regular frame (Sec. 3.4): a new
        section with the frame as its last view and one Gaussian per pixel
        with valid depth that ``silhouette`` (this section rendered from the
        frame's pose) leaves uncovered (< sil_max).  depth (H, W), rgb
        (3, H, W) float32 device; the frame's intrinsics are the section's.
        Synchronises once to learn the count."""
        V, H, W = self.depth.shape
        depth = _cuda(depth, torch.float32, "depth", (H, W))
        rgb = _cuda(rgb, torch.float32, "rgb", (3, H, W))
        silhouette = _cuda(silhouette, torch.float32, "silhouette", (H, W))
        dev = depth.device
        p = pose if isinstance(pose, torch.Tensor) else pose12(pose, dev)
        p = _cuda(p, torch.float64, "pose", (12,))
        dt = self.colour.dtype
        cap = H * W
        src = torch.empty(cap, dtype=torch.int32, device=dev)
        col = torch.empty(cap, 3, dtype=dt, device=dev)
        op = torch.empty(cap, dtype=dt, device=dev)
        rad = torch.empty(cap, dtype=dt, device=dev)
        n_out = torch.zeros(1, dtype=torch.int64, device=dev)
        L.check(L.lib().vt_section_complement(_ptr(depth), _ptr(rgb), _ptr(silhouette), W, H,
                                              _intr(self.K), float(sil_max), V, self.prec,
                                              _ptr(src), _ptr(col), _ptr(op), _ptr(rad), cap,
                                              _ptr(n_out), _stream(stream)),
                "vt_section_complement")
        n = int(n_out.item())
        cat = lambda a, b: torch.cat([a, b[:n]]).contiguous()
        return Section(torch.cat([self.poses, p[None]]).contiguous(),
                       torch.cat([self.depth, depth[None]]).contiguous(), self.K,
                       cat(self.src, src), cat(self.colour, col), cat(self.opacity, op),
                       cat(self.radius, rad))


def backproject(depth: torch.Tensor, K, pose, stream=None):
    """World centres (n, 3) float32 and raster pixel indices (n,) of the valid
    pixels of one depth map (synchronises once to learn n)."""
    depth = _cuda(depth, torch.float32, "depth")
    H, W = depth.shape
    P = pose if isinstance(pose, torch.Tensor) else pose12(pose, depth.device)
    cap = H * W
    cen = torch.empty(cap, 3, dtype=torch.float32, device=depth.device)
    pix = torch.empty(cap, dtype=torch.int32, device=depth.device)
    n_out = torch.zeros(1, dtype=torch.int64, device=depth.device)
    L.check(L.lib().vt_backproject(_ptr(depth), W, H, _intr(K), _ptr(P), _ptr(cen), _ptr(pix),
                                   cap, _ptr(n_out), _stream(stream)), "vt_backproject")
    n = int(n_out.item())
    return cen[:n], pix[:n]


def visibility(depth: torch.Tensor, K, pose, views, rel_tol: float = 0.01, out=None,
               stream=None) -> torch.Tensor:
    """Visibility check of Sec. 3.3: (H, W) uint8 mask of the valid pixels of
    ``depth`` (seen with intrinsics K from ``pose``, (12,) float64 device or a
    (3, 4) matrix) whose depth in one of ``views`` lies within rel_tol of that
    view's interpolated depth map.  views: list of (depth (h, w) float32
    device, K, pose (12,) float64 device), at most 8 (the paper uses a
    section's head, middle and last frames)."""
    depth = _cuda(depth, torch.float32, "depth")
    H, W = depth.shape
    P = pose if isinstance(pose, torch.Tensor) else pose12(pose, depth.device)
    P = _cuda(P, torch.float64, "pose", (12,))
    if not 1 <= len(views) <= L.MAX_VIS_VIEWS:
        raise ValueError(f"visibility takes 1..{L.MAX_VIS_VIEWS} views")
    vs = []
    for d, k, p in views:
        d = _cuda(d, torch.float32, "view depth")
        p = _cuda(p, torch.float64, "view pose", (12,))
        vs.append(L.ViewC(_ptr(d), d.shape[1], d.shape[0], _intr(k), _ptr(p)))
    arr = (L.ViewC * len(vs))(*vs)
    if out is None:
        out = torch.empty(H, W, dtype=torch.uint8, device=depth.device)
    out = _cuda(out, torch.uint8, "out", (H, W))
    L.check(L.lib().vt_visibility(_ptr(depth), W, H, _intr(K), _ptr(P), arr, len(vs),
                                  float(rel_tol), _ptr(out), _stream(stream)), "vt_visibility")
    return out


def visibility_counts(depth: torch.Tensor, K, pose, views, rel_tol: float = 0.01, stream=None):
    """Per view, the number of valid pixels of ``depth`` (seen from ``pose``)
    visible to it (views as in visibility(); any number, 8 per launch), and
    the number of valid pixels.  Returns (counts (len(views),) int64 numpy,
    n_valid); synchronises once."""
    depth = _cuda(depth, torch.float32, "depth")
    H, W = depth.shape
    dev = depth.device
    P = pose if isinstance(pose, torch.Tensor) else pose12(pose, dev)
    P = _cuda(P, torch.float64, "pose", (12,))
    counts = torch.zeros(max(len(views), 1), dtype=torch.int32, device=dev)
    n_valid = torch.zeros(1, dtype=torch.int32, device=dev)
    keep = []
    for b in range(0, len(views), L.MAX_VIS_VIEWS):
        vs = []
        for d, k, p in views[b:b + L.MAX_VIS_VIEWS]:
            d = _cuda(d, torch.float32, "view depth")
            p = _cuda(p, torch.float64, "view pose", (12,))
            keep += [d, p]
            vs.append(L.ViewC(_ptr(d), d.shape[1], d.shape[0], _intr(k), _ptr(p)))
        arr = (L.ViewC * len(vs))(*vs)
        L.check(L.lib().vt_visibility_counts(_ptr(depth), W, H, _intr(K), _ptr(P), arr, len(vs),
                                             float(rel_tol), C.c_void_p(counts.data_ptr() + 4 * b),
                                             _ptr(n_valid), _stream(stream)),
                "vt_visibility_counts")
    return counts[:len(views)].cpu().numpy().astype(np.int64), int(n_valid.item())


def pose_adam(pose: torch.Tensor, d_twist: torch.Tensor, state: torch.Tensor, lr,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15, renderer=None,
              stream=None):
    """One Adam step on the pose (12,) float64 from the twist gradient (6,)
    float64 (zeroed afterwards), state (15,) float64 = (m, v, t, b1^t, b2^t),
    zero-initialised; lr: six
    rates (rho then phi).  renderer (optional) records the launch."""
    _cuda(pose, torch.float64, "pose", (12,))
    _cuda(d_twist, torch.float64, "d_twist", (6,))
    _cuda(state, torch.float64, "state", (15,))
    rates = (C.c_double * 6)(*[float(x) for x in lr])
    ctx = renderer._ctx if renderer is not None else None
    L.check(L.lib().vt_pose_adam(ctx, _ptr(pose), _ptr(d_twist), _ptr(state), rates,
                                 float(beta1), float(beta2), float(eps), _stream(stream)),
            "vt_pose_adam")


def attr_adam(section, theta: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
              step: torch.Tensor, d_colour: torch.Tensor, d_opacity: torch.Tensor,
              d_radius: torch.Tensor, lr, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, renderer=None, stream=None):
    """One Adam step on the section's attributes in the parametrisation
    theta = (c0, c1, c2, logit o, log r) ((5, n) float32; m, v alike; step
    (3,) float64 zero-initialised); the section's colour / opacity / radius
    storage is overwritten with the activated values and the gradients
    (d_colour (n, 3), d_opacity, d_radius float32) are zeroed.  lr: five
    rates (one per parameter plane)."""
    n = section.n
    for name, t in (("theta", theta), ("m", m), ("v", v)):
        _cuda(t, torch.float32, name, (5, n))
    _cuda(step, torch.float64, "step", (3,))
    _cuda(d_colour, torch.float32, "d_colour", (n, 3))
    _cuda(d_opacity, torch.float32, "d_opacity", (n,))
    _cuda(d_radius, torch.float32, "d_radius", (n,))
    p = L.AdamParamsC((C.c_float * 5)(*[float(x) for x in lr]), float(beta1), float(beta2),
                      float(eps))
    ctx = renderer._ctx if renderer is not None else None
    L.check(L.lib().vt_attr_adam(ctx, n, _ptr(theta), _ptr(m), _ptr(v), _ptr(step),
                                 _ptr(d_colour), _ptr(d_opacity), _ptr(d_radius), section.prec,
                                 _ptr(section.colour), _ptr(section.opacity),
                                 _ptr(section.radius), p, _stream(stream)), "vt_attr_adam")


def adam_init(section, shape: bool = False, renderer=None, stream=None):
    """Optimiser state of a section from its storage (vt_adam_init): returns
    (theta, m, v, step) for vt_attr_adam (theta planes c0, c1, c2, logit o,
    log r) or, with shape, for vt_shape_adam (log s0..2, q0..3)."""
    n = section.n
    dev = section.colour.device
    planes = 7 if shape else 5
    theta = torch.empty(planes, n, device=dev)
    m = torch.empty(planes, n, device=dev)
    v = torch.empty(planes, n, device=dev)
    step = torch.empty(3, dtype=torch.float64, device=dev)
    ctx = renderer._ctx if renderer is not None else None
    sc = _ptr(section.scale) if shape else None
    rt = _ptr(section.rot) if shape else None
    L.check(L.lib().vt_adam_init(ctx, n, section.prec, None if shape else _ptr(section.colour),
                                 None if shape else _ptr(section.opacity),
                                 None if shape else _ptr(section.radius), sc, rt, _ptr(theta),
                                 _ptr(m), _ptr(v), _ptr(step), _stream(stream)), "vt_adam_init")
    return theta, m, v, step


def shape_adam(section, theta: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
               step: torch.Tensor, d_scale: torch.Tensor, d_rot: torch.Tensor,
               lr_scale: float = 0.005, lr_rot: float = 0.001, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8, renderer=None, stream=None):
    """One Adam step on an ellipsoid section's shape in the parametrisation
    theta = (log s0, log s1, log s2, q0, q1, q2, q3) ((7, n) float32; m, v
    alike; step (3,) float64 zero-initialised, its own counter); the
    section's scale / rot storage is overwritten (exp of the log scales, the
    quaternion as stored) and d_scale (n, 3), d_rot (n, 4) are zeroed."""
    n = section.n
    if section.scale is None:
        raise ValueError("shape_adam needs an ellipsoid section")
    for name, t in (("theta", theta), ("m", m), ("v", v)):
        _cuda(t, torch.float32, name, (7, n))
    _cuda(step, torch.float64, "step", (3,))
    _cuda(d_scale, torch.float32, "d_scale", (n, 3))
    _cuda(d_rot, torch.float32, "d_rot", (n, 4))
    p = L.ShapeAdamParamsC(float(lr_scale), float(lr_rot), float(beta1), float(beta2),
                           float(eps))
    ctx = renderer._ctx if renderer is not None else None
    L.check(L.lib().vt_shape_adam(ctx, n, _ptr(theta), _ptr(m), _ptr(v), _ptr(step),
                                  _ptr(d_scale), _ptr(d_rot), section.prec, _ptr(section.scale),
                                  _ptr(section.rot), p, _stream(stream)), "vt_shape_adam")


# Contexts released while a CUDA graph was being captured on the current
# stream: destroying one then would synchronise and free device memory in the
# middle of the capture, so they wait for the next context operation outside
# a capture.
_deferred = []


def _capturing() -> bool:
    try:
        return torch.cuda.is_available() and torch.cuda.is_current_stream_capturing()
    except Exception:
        return False


def _flush_deferred(lib):
    while _deferred and not _capturing():
        lib.vt_ctx_destroy(_deferred.pop())


class Renderer:
    """Owns one vt_ctx (the library's render workspace) on the current device."""

    def __init__(self):
        self._lib = L.lib()
        _flush_deferred(self._lib)
        h = C.c_void_p()
        L.check(self._lib.vt_ctx_create(C.byref(h)), "vt_ctx_create")
        self._ctx = h
        self.last = None

    def close(self):
        if getattr(self, "_ctx", None):
            if _capturing():
                _deferred.append(self._ctx)
            else:
                self._lib.vt_ctx_destroy(self._ctx)
                _flush_deferred(self._lib)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- workspace ---------------------------------------------------------
    def reserve(self, n_gaussians: int, W: int, H: int, n_instances: int = 0, stream=None):
        L.check(self._lib.vt_ctx_reserve(self._ctx, int(n_gaussians), int(W), int(H),
                                         int(n_instances), _stream(stream)), "vt_ctx_reserve")

    def set_list_capacity(self, cap: int):
        """Per-pixel list capacity for the backward (0 = always replay tiles)."""
        L.check(self._lib.vt_ctx_set_list_capacity(self._ctx, int(cap)), "set_list_capacity")

    def set_budget(self, nbytes: int):
        """Workspace budget in bytes (0 = unbounded)."""
        L.check(self._lib.vt_ctx_set_workspace_budget(self._ctx, int(nbytes)), "set_budget")

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.vt_ctx_workspace_bytes(self._ctx))

    @property
    def used_lists(self) -> bool:
        return bool(self._lib.vt_ctx_used_lists(self._ctx))

    def status(self, stream=None) -> int:
        """Synchronise and return the tile-instance count of the last render;
        raises VTError(VT_ERR_CAPACITY) if the workspace was too small."""
        need = C.c_int64(0)
        L.check(self._lib.vt_ctx_sync_status(self._ctx, _stream(stream), C.byref(need)),
                "render status")
        return int(need.value)

    # -- render --------------------------------------------------------------
    def needed_instances(self, stream=None) -> int:
        """Synchronises and returns the tile instances the last render (or
        batch) needed (vt_ctx_sync_status)."""
        need = C.c_int64(0)
        self._lib.vt_ctx_sync_status(self._ctx, _stream(stream), C.byref(need))
        return int(need.value)

    def render(self, sections, pose, K, W: int, H: int, rgb=None, depth=None, sil=None,
               stream=None, checked: bool = False):
        """Render (the concatenation of) ``sections`` from ``pose`` ((12,)
        float64 device tensor).  Returns (rgb (3,H,W), depth (H,W),
        silhouette (H,W)) float32.  With ``checked`` the call synchronises,
        grows the workspace if the instance capacity was short and renders
        again."""
        if isinstance(sections, Section):
            sections = [sections]
        pose = _cuda(pose, torch.float64, "pose", (12,))
        dev = pose.device
        rgb = torch.empty(3, H, W, device=dev) if rgb is None else _cuda(rgb, torch.float32, "rgb", (3, H, W))
        depth = torch.empty(H, W, device=dev) if depth is None else _cuda(depth, torch.float32, "depth", (H, W))
        sil = torch.empty(H, W, device=dev) if sil is None else _cuda(sil, torch.float32, "sil", (H, W))
        arr = (L.SectionC * max(1, len(sections)))(*[s.c_struct() for s in sections])
        args = (self._ctx, arr, len(sections), _ptr(pose), _intr(K), int(W), int(H), _ptr(rgb),
                _ptr(depth), _ptr(sil), _stream(stream))
        L.check(self._lib.vt_render(*args), "vt_render")
        self.last = (sections, pose, tuple(K), W, H)
        if checked:
            try:
                self.status(stream)
            except L.VTError as e:
                if e.status != L.VT_ERR_CAPACITY:
                    raise
                need = C.c_int64(0)
                self._lib.vt_ctx_sync_status(self._ctx, _stream(stream), C.byref(need))
                n = sum(s.n for s in sections)
                self.reserve(n, W, H, int(need.value * 1.25) + 1024, stream)
                L.check(self._lib.vt_render(*args), "vt_render")
                self.status(stream)
        return rgb, depth, sil

    def backward(self, d_rgb=None, d_depth=None, d_sil=None, attr_grads=None, pose_grad=False,
                 d_twist=None, d_mat=None, view_grads=None, stream=None):
        """Backward of the last render.  attr_grads: per section a tuple
        (d_colour (n,3), d_opacity (n,), d_radius (n,)) float32 device tensors
        or None (frozen section); for ellipsoid sections (d_colour, d_opacity,
        None, d_scale (n,3), d_rot (n,4)); gradients are accumulated (+=).  With
        pose_grad, d_twist (6,) and d_mat (12,) float64 device tensors are
        accumulated (both created as zeros when neither is given; a missing
        one is not computed when the other is).  view_grads: per section a
        tuple (d_view_twist (V,6), d_view_mat (V,12)) float64 device tensors
        [, d_depth (n,) float32] (any may be None) or None: gradients with
        respect to the section's source-view poses (head-frame bundle
        adjustment) and to each Gaussian's depth along its ray, accumulated.
        Returns (d_twist, d_mat)."""
        mode = 0
        grads = None
        if attr_grads is not None or view_grads is not None:
            n = len(attr_grads) if attr_grads is not None else len(view_grads)
            gl = []
            for s in range(n):
                ag = attr_grads[s] if attr_grads is not None else None
                vg = view_grads[s] if view_grads is not None else None
                ag = tuple(ag) + (None,) * (5 - len(ag)) if ag is not None else (None,) * 5
                dc, do, dr, ds, dq = ag
                vg = tuple(vg) + (None,) * (3 - len(vg)) if vg is not None else (None,) * 3
                vt, vm, vd = vg
                gl.append(L.GradsC(_ptr(dc), _ptr(do), _ptr(dr), _ptr(vt), _ptr(vm), _ptr(vd),
                                   _ptr(ds), _ptr(dq)))
            grads = (L.GradsC * len(gl))(*gl)
            if attr_grads is not None:
                mode |= L.VT_GRAD_ATTR
            if view_grads is not None:
                mode |= L.VT_GRAD_VIEWS
        if pose_grad:
            mode |= L.VT_GRAD_POSE
            dev = self.last[1].device if self.last else "cuda"
            if d_twist is None and d_mat is None:
                d_twist = torch.zeros(6, dtype=torch.float64, device=dev)
                d_mat = torch.zeros(12, dtype=torch.float64, device=dev)
        L.check(self._lib.vt_render_backward(self._ctx, _ptr(d_rgb), _ptr(d_depth), _ptr(d_sil),
                                             mode, grads, _ptr(d_twist), _ptr(d_mat),
                                             _stream(stream)), "vt_render_backward")
        return d_twist, d_mat

    def masked_l1(self, rgb, depth, sil, obs_rgb, obs_depth, w_rgb: float, w_depth: float,
                  sil_min: float = -1.0, rgb_needs_depth: bool = False, visible=None,
                  d_rgb=None, d_depth=None, loss=None, stream=None):
        """Masked L1 terms of Eq. 1 / Eq. 2 and their image gradient in one
        kernel (this context provides the scratch of the loss sum).  Eq. 1:
        (alpha, beta, sil_min=0.99, rgb_needs_depth=True, visible=mask);
        Eq. 2: (rho, sigma).  Returns (loss (1,) float64, d_rgb (3,H,W),
        d_depth (H,W)); given output tensors are overwritten."""
        depth = _cuda(depth, torch.float32, "depth")
        H, W = depth.shape
        dev = depth.device
        _cuda(rgb, torch.float32, "rgb", (3, H, W))
        _cuda(obs_rgb, torch.float32, "obs_rgb", (3, H, W))
        _cuda(obs_depth, torch.float32, "obs_depth", (H, W))
        if sil is not None:
            _cuda(sil, torch.float32, "sil", (H, W))
        if visible is not None:
            _cuda(visible, torch.uint8, "visible", (H, W))
        if d_rgb is None:
            d_rgb = torch.empty(3, H, W, device=dev)
        if d_depth is None:
            d_depth = torch.empty(H, W, device=dev)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=dev)
        w = L.L1WeightsC(float(w_rgb), float(w_depth), float(sil_min), int(bool(rgb_needs_depth)))
        L.check(self._lib.vt_masked_l1(self._ctx, W, H, _ptr(rgb), _ptr(depth), _ptr(sil),
                                       _ptr(obs_rgb), _ptr(obs_depth), _ptr(visible), w,
                                       _ptr(_cuda(d_rgb, torch.float32, "d_rgb", (3, H, W))),
                                       _ptr(_cuda(d_depth, torch.float32, "d_depth", (H, W))),
                                       _ptr(loss), _stream(stream)), "vt_masked_l1")
        return loss, d_rgb, d_depth

    def ssim(self, rgb, obs_rgb, weight: float, d_rgb=None, loss=None, stream=None):
        """SSIM term of Eq. 2: loss (1,) float64 = weight * (1 - mean SSIM);
        d_rgb (3, H, W) float32, when given, is accumulated (+=) with its
        gradient.  Returns (loss, d_rgb)."""
        rgb = _cuda(rgb, torch.float32, "rgb")
        _, H, W = rgb.shape
        _cuda(obs_rgb, torch.float32, "obs_rgb", (3, H, W))
        if d_rgb is not None:
            _cuda(d_rgb, torch.float32, "d_rgb", (3, H, W))
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=rgb.device)
        L.check(self._lib.vt_ssim(self._ctx, W, H, _ptr(rgb), _ptr(obs_rgb), float(weight),
                                  _ptr(d_rgb), _ptr(loss), _stream(stream)), "vt_ssim")
        return loss, d_rgb

    # -- instrumentation -----------------------------------------------------
    def set_timing(self, on: bool = True):
        L.check(self._lib.vt_ctx_set_timing(self._ctx, int(bool(on))), "vt_ctx_set_timing")

    def timing(self, reset: bool = True, stream=None) -> dict:
        n = 64
        names = (C.c_char_p * n)()
        launches = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        k = self._lib.vt_ctx_timing(self._ctx, _stream(stream), names, launches, ms, n,
                                    int(bool(reset)))
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(k)}

    @property
    def launches(self) -> int:
        return int(self._lib.vt_ctx_launch_count(self._ctx))

    def pixel_lists(self, x0: int, y0: int, w: int, h: int, cap: int | None = None,
                    stream=None):
        """Per-pixel lists of the last render for the rectangle (x0, y0, w, h)
        (vt_ctx_debug_pixel_lists): ids (h, w, cap) int64 (-1 beyond each
        pixel's entries), T_front (h, w, cap) float32, counts (h, w) int64 of
        added Gaussians and the context's list capacity."""
        kept = C.c_int32(0)
        counts = np.zeros((h, w), np.uint32)
        probe = np.zeros(1, np.uint32)
        L.check(self._lib.vt_ctx_debug_pixel_lists(
            self._ctx, int(x0), int(y0), int(w), int(h), 0, probe.ctypes.data_as(C.c_void_p),
            None, counts.ctypes.data_as(C.c_void_p), C.byref(kept), _stream(stream)),
            "vt_ctx_debug_pixel_lists")
        if cap is None:
            cap = max(1, min(int(kept.value), int(counts.max()) if counts.size else 1))
        ids = np.full((h, w, cap), 0xFFFFFFFF, np.uint32)
        T = np.zeros((h, w, cap), np.float32)
        L.check(self._lib.vt_ctx_debug_pixel_lists(
            self._ctx, int(x0), int(y0), int(w), int(h), int(cap),
            ids.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
            counts.ctypes.data_as(C.c_void_p), C.byref(kept), _stream(stream)),
            "vt_ctx_debug_pixel_lists")
        out = ids.astype(np.int64)
        out[ids == 0xFFFFFFFF] = -1
        return out, T, counts.astype(np.int64), int(kept.value)

    def debug(self, what: int, count: int, dtype=np.uint32, stream=None) -> np.ndarray:
        out = np.zeros(count, dtype)
        r = self._lib.vt_ctx_debug_copy(self._ctx, int(what), out.ctypes.data_as(C.c_void_p),
                                        out.nbytes, _stream(stream))
        if r < 0:
            raise L.VTError(-r, "vt_ctx_debug_copy")
        return out[: r // out.itemsize]


@dataclasses.dataclass
class BatchItem:
    """One work item of a batch (vt_batch_item): ``section`` indexes the
    batch's section list; ``pose`` (12,) float64, ``image`` (5, H, W)
    float32 (written: rgb planes, depth, silhouette), and for a tracking item
    ``obs`` (4, H, W) float32 (observed rgb planes and depth) and ``result``
    (19,) float64 (written: loss, dL/dtwist, dL/dR, dL/dt), all device
    tensors."""
    section: int
    track: bool
    W: int
    H: int
    K: tuple
    pose: torch.Tensor
    image: torch.Tensor
    obs: torch.Tensor | None = None
    result: torch.Tensor | None = None

    def c_struct(self) -> L.BatchItemC:
        W, H = int(self.W), int(self.H)
        _cuda(self.pose, torch.float64, "pose", (12,))
        _cuda(self.image, torch.float32, "image", (5, H, W))
        if self.track:
            _cuda(self.obs, torch.float32, "obs", (4, H, W))
            _cuda(self.result, torch.float64, "result", (19,))
        return L.BatchItemC(int(self.section), int(bool(self.track)), W, H, _intr(self.K),
                            _ptr(self.pose), _ptr(self.image),
                            _ptr(self.obs) if self.track else None,
                            _ptr(self.result) if self.track else None)


class BatchRunner(Renderer):
    """A context reserved for batched work items (vt_batch_*): every stage
    of all items' renders -- and for tracking items the Eq. 1 loss and the
    pose gradient -- runs as one launch over all items.  ``set`` stages a batch
    (host only), ``launch`` enqueues it (capturable in a CUDA graph: the
    work-item table is uploaded inside the launch sequence)."""

    def __init__(self, max_gaussians: int, max_pixels: int, max_tiles: int, max_instances: int,
                 max_views: int, max_table_rows: int, list_cap: int | None = None, stream=None):
        super().__init__()
        if list_cap is not None:
            self.set_list_capacity(list_cap)
        self.capacity = dict(gaussians=int(max_gaussians), pixels=int(max_pixels),
                             tiles=int(max_tiles), instances=int(max_instances),
                             views=int(max_views), table_rows=int(max_table_rows))
        L.check(self._lib.vt_batch_reserve(self._ctx, int(max_gaussians), int(max_pixels),
                                           int(max_tiles), int(max_instances), int(max_views),
                                           int(max_table_rows), _stream(stream)),
                "vt_batch_reserve")
        self._keep = None

    @staticmethod
    def workspace_bytes_for(max_gaussians, max_pixels, max_tiles, max_instances, max_views,
                            max_table_rows, list_cap=256) -> int:
        return int(L.lib().vt_batch_workspace_bytes(int(max_gaussians), int(max_pixels),
                                                    int(max_tiles), int(max_instances),
                                                    int(max_views), int(max_table_rows),
                                                    int(list_cap)))

    def set(self, sections, items, w_rgb: float = 0.5, w_depth: float = 0.025,
            sil_min: float = 0.99, rgb_needs_depth: bool = True):
        secs = (L.SectionC * len(sections))(*[s.c_struct() for s in sections])
        its = (L.BatchItemC * len(items))(*[it.c_struct() for it in items])
        w = L.L1WeightsC(float(w_rgb), float(w_depth), float(sil_min), int(bool(rgb_needs_depth)))
        L.check(self._lib.vt_batch_set(self._ctx, secs, len(sections), its, len(items), w),
                "vt_batch_set")
        self._keep = (sections, items)

    def launch(self, stream=None, obs_ready=None):
        """Enqueue the staged batch; obs_ready (a torch.cuda.Event, optional)
        marks the tracking items' observations as uploaded: only the loss
        stage waits for it."""
        ev = C.c_void_p(obs_ready.cuda_event) if obs_ready is not None else None
        L.check(self._lib.vt_batch_launch(self._ctx, _stream(stream), ev), "vt_batch_launch")
