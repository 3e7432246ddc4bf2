"""Python face of the FP64 CPU oracle (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.

The arithmetic lives in ``vt_oracle.c`` (rendering and its gradient) and
``vt_oracle_loss.c`` (visibility check and masked L1 loss); this module
compiles them with gcc
(``-O2 -fopenmp -ffp-contract=off``, no fast-math) into ``oracle/_build`` and
marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "vt_oracle.c"), os.path.join(_HERE, "vt_oracle_loss.c"),
        os.path.join(_HERE, "vt_oracle.h")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if its sources are newer than the library."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC[0], _SRC[1], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Section(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("W", C.c_int32), ("H", C.c_int32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("poses", C.c_void_p), ("depth", C.c_void_p), ("n", C.c_int64),
                ("src", C.c_void_p), ("colour", C.c_void_p), ("opacity", C.c_void_p),
                ("radius", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("pose", C.c_double * 12), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("W", C.c_int32), ("H", C.c_int32)]


class _Image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("sil", C.c_void_p),
                ("T_final", C.c_void_p), ("n_added", C.c_void_p), ("margin", C.c_void_p),
                ("margin_T", C.c_void_p), ("margin_clamp", C.c_void_p),
                ("lists", C.c_void_p), ("list_cap", C.c_int32)]


class _Upstream(C.Structure):
    _fields_ = [("g_rgb", C.c_void_p), ("g_depth", C.c_void_p), ("g_sil", C.c_void_p)]


class _Grads(C.Structure):
    _fields_ = [("d_colour", C.c_void_p), ("d_opacity", C.c_void_p), ("d_radius", C.c_void_p),
                ("a_colour", C.c_void_p), ("a_opacity", C.c_void_p), ("a_radius", C.c_void_p),
                ("d_x", C.c_void_p), ("a_x", C.c_void_p), ("twist", C.c_double * 6), ("mat", C.c_double * 12),
                ("twist_noise", C.c_double * 6), ("mat_noise", C.c_double * 12)]


class _Lists(C.Structure):
    _fields_ = [("ids", C.c_void_p), ("count", C.c_void_p), ("cap", C.c_int32)]


class _Verdict(C.Structure):
    _fields_ = [("status", C.c_void_p), ("flips", C.c_void_p), ("flip_margin", C.c_void_p)]


class _View(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("W", C.c_int32), ("H", C.c_int32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("pose", C.c_double * 12)]


class _L1Weights(C.Structure):
    _fields_ = [("w_rgb", C.c_double), ("w_depth", C.c_double), ("sil_min", C.c_double),
                ("rgb_needs_depth", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_render.restype = C.c_int
            L.orc_render.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
            L.orc_backward.restype = C.c_int
            L.orc_backward.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                       C.c_void_p]
            L.orc_render_lists.restype = C.c_int
            L.orc_render_lists.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_double, C.c_double, C.c_void_p, C.c_void_p]
            L.orc_backward_lists.restype = C.c_int
            L.orc_backward_lists.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
            L.orc_zkeys.restype = None
            L.orc_zkeys.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_backproject.restype = C.c_int64
            L.orc_backproject.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_float,
                                          C.c_float, C.c_float, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
            L.orc_section_init.restype = C.c_int64
            L.orc_section_init.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                           C.c_int32, C.c_float, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p]
            L.orc_visibility.restype = None
            L.orc_visibility.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_float,
                                         C.c_float, C.c_float, C.c_void_p, C.c_void_p,
                                         C.c_int32, C.c_double, C.c_void_p]
            L.orc_masked_l1.restype = C.c_double
            L.orc_masked_l1.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, _L1Weights,
                                        C.c_void_p, C.c_void_p]
            L.orc_section_complement.restype = C.c_int64
            L.orc_section_complement.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                                 C.c_int32, C.c_float, C.c_float, C.c_int32,
                                                 C.c_void_p, C.c_void_p, C.c_void_p,
                                                 C.c_void_p]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


@dataclasses.dataclass
class Section:
    """A section as the oracle sees it (all arrays host numpy).

    poses: (V, 3, 4) float64 camera-to-world; depth: (V, H, W) float32;
    src: (n,) uint32 = (view*H + v)*W + u, strictly increasing;
    colour (n, 3), opacity (n,), radius (n,) float64."""
    W: int
    H: int
    K: tuple          # (fx, fy, cx, cy) float32-representable
    poses: np.ndarray
    depth: np.ndarray
    src: np.ndarray
    colour: np.ndarray
    opacity: np.ndarray
    radius: np.ndarray

    @property
    def n(self) -> int:
        return int(self.src.shape[0])

    def _c(self, keep: list) -> _Section:
        arrs = dict(poses=pose12(self.poses),
                    depth=np.ascontiguousarray(self.depth, np.float32),
                    src=np.ascontiguousarray(self.src, np.uint32),
                    colour=np.ascontiguousarray(self.colour, np.float64).reshape(-1, 3),
                    opacity=np.ascontiguousarray(self.opacity, np.float64),
                    radius=np.ascontiguousarray(self.radius, np.float64))
        keep.append(arrs)
        s = _Section()
        s.n_views = int(self.depth.shape[0])
        s.W, s.H = int(self.W), int(self.H)
        s.fx, s.fy, s.cx, s.cy = (float(np.float32(k)) for k in self.K)
        s.poses = _ptr(arrs["poses"])
        s.depth = _ptr(arrs["depth"])
        s.n = self.n
        s.src = _ptr(arrs["src"])
        s.colour = _ptr(arrs["colour"])
        s.opacity = _ptr(arrs["opacity"])
        s.radius = _ptr(arrs["radius"])
        return s


def pose12(poses) -> np.ndarray:
    """(V, 3, 4) camera-to-world poses -> (V, 12): R row-major, then t."""
    p = np.asarray(poses, np.float64).reshape(-1, 3, 4)
    return np.ascontiguousarray(np.concatenate([p[:, :, :3].reshape(-1, 9), p[:, :, 3]], axis=1))


def _camera(pose, K, W, H) -> _Camera:
    c = _Camera()
    flat = pose12(pose)[0]
    for i in range(12):
        c.pose[i] = float(flat[i])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(k)) for k in K)
    c.W, c.H = int(W), int(H)
    return c


def _sections(secs):
    if isinstance(secs, Section):
        secs = [secs]
    keep = []
    arr = (_Section * len(secs))()
    for i, s in enumerate(secs):
        arr[i] = s._c(keep)
    return list(secs), arr, keep


def render(secs, pose, K, W, H, binned=True, list_cap=0):
    """Forward render.  Returns a dict of float64 images (rgb (3,H,W), depth,
    sil, T_final), n_added (int32), the relative decision margins (margin for
    the inclusion tests, margin_T for termination, margin_clamp for the 0.99
    clamp) and, if list_cap > 0, the ids each pixel added front to back
    (H, W, list_cap; -1 padded)."""
    secs, arr, keep = _sections(secs)
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), sil=np.zeros((H, W)),
               T_final=np.zeros((H, W)), n_added=np.zeros((H, W), np.int32),
               margin=np.zeros((H, W)), margin_T=np.zeros((H, W)),
               margin_clamp=np.zeros((H, W)))
    lists = np.full((H, W, list_cap), -1, np.int64) if list_cap > 0 else None
    img = _Image(_ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["sil"]), _ptr(out["T_final"]),
                 _ptr(out["n_added"]), _ptr(out["margin"]), _ptr(out["margin_T"]),
                 _ptr(out["margin_clamp"]), _ptr(lists), int(list_cap))
    cam = _camera(pose, K, W, H)
    rc = lib().orc_render(C.byref(arr), len(secs), C.byref(cam), int(bool(binned)), C.byref(img))
    if rc != 0:
        raise RuntimeError("oracle render failed")
    if lists is not None:
        out["lists"] = lists
    return out


def backward(secs, pose, K, W, H, g_rgb=None, g_depth=None, g_sil=None, binned=True):
    """Gradients of <g_rgb, rgb> + <g_depth, depth> + <g_sil, sil>.

    Returns dict(colour=[(n,3)], opacity=[(n,)], radius=[(n,)] per section,
    twist (6,) and mat (12,) float64, and abs_colour/abs_opacity/abs_radius:
    per element the sum over pixels of the componentwise magnitude of each
    term, i.e. of the absolute values of the products its formula adds;
    twist_noise (6,) and mat_noise (12,): per component
    sqrt(sum over pixels of n_p m_p^2), n_p the pixel's added Gaussians and
    m_p the componentwise magnitude of the pixel's contribution; x: per
    section (n, 3) dL/dx of every centre in the target camera frame, abs_x
    its componentwise term magnitudes)."""
    secs, arr, keep = _sections(secs)
    return _run_backward(secs, arr, pose, K, W, H, g_rgb, g_depth, g_sil,
                         lambda a, cam, up, g: lib().orc_backward(
                             C.byref(a), len(secs), C.byref(cam), int(bool(binned)),
                             C.byref(up), C.byref(g)))


def _run_backward(secs, arr, pose, K, W, H, g_rgb, g_depth, g_sil, call):
    ups = [None if g is None else np.ascontiguousarray(g, np.float64) for g in (g_rgb, g_depth, g_sil)]
    up = _Upstream(*[_ptr(u) for u in ups])
    dcol = [np.zeros((s.n, 3)) for s in secs]
    dop = [np.zeros(s.n) for s in secs]
    drad = [np.zeros(s.n) for s in secs]
    acol = [np.zeros((s.n, 3)) for s in secs]
    aop = [np.zeros(s.n) for s in secs]
    arad = [np.zeros(s.n) for s in secs]
    dx = [np.zeros((s.n, 3)) for s in secs]
    ax = [np.zeros((s.n, 3)) for s in secs]
    arrs = [(C.c_void_p * len(secs))(*[_ptr(a) for a in lst])
            for lst in (dcol, dop, drad, acol, aop, arad, dx, ax)]
    g = _Grads(*[C.cast(a, C.c_void_p) for a in arrs])
    cam = _camera(pose, K, W, H)
    rc = call(arr, cam, up, g)
    if rc != 0:
        raise RuntimeError("oracle backward failed")
    return dict(colour=dcol, opacity=dop, radius=drad, twist=np.array(g.twist[:]),
                mat=np.array(g.mat[:]), abs_colour=acol, abs_opacity=aop, abs_radius=arad,
                twist_noise=np.array(g.twist_noise[:]), mat_noise=np.array(g.mat_noise[:]),
                x=dx, abs_x=ax)


def _lists(ids, count, H, W):
    ids = np.ascontiguousarray(ids, np.int64).reshape(H, W, -1)
    count = np.ascontiguousarray(count, np.int32).reshape(H, W)
    return ids, count, _Lists(_ptr(ids), _ptr(count), int(ids.shape[2]))


def render_lists(secs, pose, K, W, H, ids, count, tau_incl=1e-5, tau_T=2e-4):
    """Composite along given per-pixel lists of added Gaussians (ids (H, W,
    cap) int64, front to back, count (H, W) entries each; ids are positions
    in the concatenation of the sections) and check them against the
    definition.  Returns the images of render() (rgb, depth, sil, T_final,
    n_added) evaluated in FP64 along the lists, and per pixel ``status``
    (0: the definition's list up to decisions within tau_incl / tau_T
    (relative) of their thresholds; 1: not a list of the definition at all;
    2: a decision differs by more than the margins), ``flips`` (decisions
    taken otherwise than in FP64) and ``flip_margin`` (the largest relative
    margin among them)."""
    secs, arr, keep = _sections(secs)
    ids, count, lst = _lists(ids, count, H, W)
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), sil=np.zeros((H, W)),
               T_final=np.zeros((H, W)), n_added=np.zeros((H, W), np.int32),
               status=np.zeros((H, W), np.int32), flips=np.zeros((H, W), np.int32),
               flip_margin=np.zeros((H, W)))
    img = _Image(_ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["sil"]), _ptr(out["T_final"]),
                 _ptr(out["n_added"]), None, None, None, None, 0)
    vd = _Verdict(_ptr(out["status"]), _ptr(out["flips"]), _ptr(out["flip_margin"]))
    cam = _camera(pose, K, W, H)
    rc = lib().orc_render_lists(C.byref(arr), len(secs), C.byref(cam), C.byref(lst),
                                float(tau_incl), float(tau_T), C.byref(img), C.byref(vd))
    if rc != 0:
        raise RuntimeError("oracle render_lists failed")
    return out


def backward_lists(secs, pose, K, W, H, ids, count, g_rgb=None, g_depth=None, g_sil=None):
    """backward() with each pixel's added Gaussians taken from the given
    lists (as render_lists) instead of from the FP64 decisions."""
    secs, arr, keep = _sections(secs)
    ids, count, lst = _lists(ids, count, H, W)
    return _run_backward(secs, arr, pose, K, W, H, g_rgb, g_depth, g_sil,
                         lambda a, cam, up, g: lib().orc_backward_lists(
                             C.byref(a), len(secs), C.byref(cam), C.byref(lst), C.byref(up),
                             C.byref(g)))


def view_pose_grads(sec: Section, pose, d_x):
    """Gradients with respect to the source-view poses P_k = [R_k | t_k] of a
    section (head-frame bundle adjustment, Sec. 3.4) from d_x = dL/dx of its
    centres in the target camera frame: the centre of Gaussian i of view k is
    mu = R_k X_c + t_k, X_c = D ((u - cx)/fx, (v - cy)/fy, 1), and
    x = R^T (mu - t), so dL/dmu = R dL/dx and
        dL/dR_k = sum dL/dmu X_c^T,  dL/dt_k = sum dL/dmu,
        dL/drho_k = R_k^T sum dL/dmu,  dL/dphi_k = sum X_c x (R_k^T dL/dmu)
    for the right perturbation P_k Exp(xi).  Returns (twist (V, 6), mat
    (V, 12)) float64."""
    R = np.asarray(pose, np.float64).reshape(3, 4)[:, :3]
    V = sec.poses.shape[0]
    plane = sec.W * sec.H
    src = sec.src.astype(np.int64)
    view = src // plane
    pix = src - view * plane
    u = (pix % sec.W).astype(np.float64)
    v = (pix // sec.W).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(k)) for k in sec.K)
    D = sec.depth.reshape(-1)[src].astype(np.float64)
    Xc = np.stack([D * (u - cx) / fx, D * (v - cy) / fy, D], axis=1)
    dmu = np.asarray(d_x, np.float64) @ R.T              # rows: R g
    twist = np.zeros((V, 6))
    mat = np.zeros((V, 12))
    for k in range(V):
        sel = view == k
        Rk = sec.poses[k][:, :3]
        mat[k, :9] = (dmu[sel].T @ Xc[sel]).reshape(-1)
        mat[k, 9:] = dmu[sel].sum(0)
        w = dmu[sel] @ Rk                                   # rows: R_k^T dL/dmu
        twist[k, :3] = w.sum(0)
        twist[k, 3:] = np.cross(Xc[sel], w).sum(0)
    return twist, mat


def zkeys(sec: Section, pose, K, W, H):
    """FP32 depth keys and validity of every Gaussian of one section."""
    _, arr, keep = _sections([sec])
    z = np.zeros(sec.n, np.float32)
    ok = np.zeros(sec.n, np.uint8)
    cam = _camera(pose, K, W, H)
    lib().orc_zkeys(C.byref(arr), C.byref(cam), _ptr(z), _ptr(ok))
    return z, ok.astype(bool)


def backproject(depth, K, pose):
    """Centres (n, 3) float64 and raster pixel indices (n,) uint32."""
    depth = np.ascontiguousarray(depth, np.float32)
    H, W = depth.shape
    cen = np.zeros((H * W, 3))
    pix = np.zeros(H * W, np.uint32)
    flat = pose12(pose)[0]
    fx, fy, cx, cy = (float(np.float32(k)) for k in K)
    n = lib().orc_backproject(_ptr(depth), W, H, fx, fy, cx, cy, _ptr(flat), _ptr(cen), _ptr(pix))
    return cen[:n].copy(), pix[:n].copy()


def section_init(depth, rgb, K, poses) -> Section:
    """One Gaussian per valid depth pixel: colour = V(u,v), opacity 0.9,
    radius = D / fx.  depth (V,H,W) f32, rgb (V,3,H,W) f32, poses (V,3,4)."""
    depth = np.ascontiguousarray(depth, np.float32)
    rgb = np.ascontiguousarray(rgb, np.float32)
    V, H, W = depth.shape
    cap = V * H * W
    src = np.zeros(cap, np.uint32)
    col = np.zeros((cap, 3))
    op = np.zeros(cap)
    rad = np.zeros(cap)
    fx = float(np.float32(K[0]))
    n = lib().orc_section_init(_ptr(depth), _ptr(rgb), V, W, H, fx, _ptr(src), _ptr(col),
                               _ptr(op), _ptr(rad))
    return Section(W, H, tuple(float(np.float32(k)) for k in K),
                   np.asarray(poses, np.float64).reshape(V, 3, 4).copy(), depth,
                   src[:n].copy(), col[:n].copy(), op[:n].copy(), rad[:n].copy())


def visibility(depth, K, pose, views, rel_tol=0.01):
    """Visibility mask (H, W) bool of the valid pixels of ``depth`` (seen
    with intrinsics K and camera-to-world ``pose``) to the union of
    ``views``: a list of (depth (h, w) f32, K, pose)."""
    depth = np.ascontiguousarray(depth, np.float32)
    H, W = depth.shape
    keep = [np.ascontiguousarray(d, np.float32) for d, _, _ in views]
    arr = (_View * max(len(views), 1))()
    for i, ((_, k, p), d) in enumerate(zip(views, keep)):
        arr[i] = _View(_ptr(d), d.shape[1], d.shape[0], *(float(np.float32(x)) for x in k),
                       (C.c_double * 12)(*pose12(p)[0]))
    out = np.zeros((H, W), np.uint8)
    fx, fy, cx, cy = (float(np.float32(k)) for k in K)
    flat = pose12(pose)[0]
    lib().orc_visibility(_ptr(depth), W, H, fx, fy, cx, cy, _ptr(flat), arr, len(views),
                         float(rel_tol), _ptr(out))
    return out.astype(bool)


def masked_l1(rgb, depth, sil, obs_rgb, obs_depth, w_rgb, w_depth, sil_min=-1.0,
              rgb_needs_depth=False, visible=None):
    """Masked L1 loss of Eq. 1 / Eq. 2 (value, float64) and its gradient with
    respect to rgb (3, H, W) and depth (H, W), float64."""
    rgb, depth, sil, obs_rgb, obs_depth = (np.ascontiguousarray(a, np.float32) for a in
                                           (rgb, depth, sil, obs_rgb, obs_depth))
    H, W = depth.shape
    vis = None if visible is None else np.ascontiguousarray(visible, np.uint8)
    d_rgb = np.zeros((3, H, W))
    d_depth = np.zeros((H, W))
    # the coverage threshold is the FP32 value the kernel compares against
    w = _L1Weights(float(w_rgb), float(w_depth), float(np.float32(sil_min)),
                   int(bool(rgb_needs_depth)))
    loss = lib().orc_masked_l1(W, H, _ptr(rgb), _ptr(depth), _ptr(sil), _ptr(obs_rgb),
                               _ptr(obs_depth), None if vis is None else _ptr(vis), w,
                               _ptr(d_rgb), _ptr(d_depth))
    return float(loss), d_rgb, d_depth


def section_complement(depth, rgb, sil, K, view, sil_max=0.5):
    """Complement initialisation of one frame: (src, colour (n, 3), opacity,
    radius) of the Gaussians at its valid, uncovered pixels (silhouette <
    sil_max); the frame is view ``view`` of the section."""
    depth = np.ascontiguousarray(depth, np.float32)
    rgb = np.ascontiguousarray(rgb, np.float32)
    sil = np.ascontiguousarray(sil, np.float32)
    H, W = depth.shape
    cap = H * W
    src = np.zeros(cap, np.uint32)
    col = np.zeros((cap, 3))
    op = np.zeros(cap)
    rad = np.zeros(cap)
    n = lib().orc_section_complement(_ptr(depth), _ptr(rgb), _ptr(sil), W, H,
                                     float(np.float32(K[0])), float(np.float32(sil_max)),
                                     int(view), _ptr(src), _ptr(col), _ptr(op), _ptr(rad))
    return src[:n].copy(), col[:n].copy(), op[:n].copy(), rad[:n].copy()


def depth_grads(sec: Section, pose, d_x, abs_x=None):
    """dL/dD of every Gaussian's depth along its pixel's ray (the movable
    Gaussians of the supplementary): mu = R_k D K^-1 [u v 1] + t_k, so
    dL/dD = (R dL/dx) . (R_k X_c / D).  Returns (n,) float64, and with abs_x
    (the componentwise magnitudes of d_x) also the magnitude bound
    sum_ab |R_k^T R|_ab abs_x_b |X_c / D|_a."""
    R = np.asarray(pose, np.float64).reshape(3, 4)[:, :3]
    plane = sec.W * sec.H
    src = sec.src.astype(np.int64)
    view = src // plane
    pix = src - view * plane
    u = (pix % sec.W).astype(np.float64)
    v = (pix // sec.W).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(k)) for k in sec.K)
    ray = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=1)   # X_c / D
    dmu = np.asarray(d_x, np.float64) @ R.T
    Rk = sec.poses[view][:, :, :3]                                            # (n, 3, 3)
    val = np.einsum("na,nab,nb->n", dmu, Rk, ray)
    if abs_x is None:
        return val
    M = np.abs(np.einsum("nca,cb->nab", Rk, R))                               # |R_k^T R|
    return val, np.einsum("nab,nb,na->n", M, np.asarray(abs_x, np.float64), np.abs(ray))
