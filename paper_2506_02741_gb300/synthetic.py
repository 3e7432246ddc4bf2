"""Seeded synthetic RGB-D workloads shaped like the paper's indoor sequences.

This module only *makes inputs*: a procedural room (five planes and three
spheres), ray-cast RGB-D frames, smooth camera trajectories and random pose
perturbations.  It contains none of the splatting method's arithmetic, so both
the CUDA path and the CPU oracle may consume what it produces.  It imports
numpy only.

Conventions shared with the rest of the library:

* A camera pose is a float64 array of shape (3, 4), ``[R | t]``,
  camera-to-world, row-major.  Camera axes: x right, y down, z forward.
* Intrinsics are ``(fx, fy, cx, cy)`` as float32-representable values; pixel
  ``(u, v)`` looks along the camera ray ``((u - cx)/fx, (v - cy)/fy, 1)``.
* Depth is z-depth in metres (float32, shape (H, W)); colour is float32 in
  [0, 1] with shape (3, H, W).

The real datasets of the paper (Replica, TUM-RGBD, ScanNet, ScanNet++, KITTI)
are not available; the shapes below stand in for them (Sec. 4 of the paper
uses 1200x680 Replica frames and 640x480 TUM/ScanNet frames).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# Seeds fixed by the workload recipe.
SCENE_SEED = 0
TRAJECTORY_SEED = 1
POSE_NOISE_SEED = 2
REQUEST_SEED = 3

DEPTH_MIN = 0.5
DEPTH_MAX = 4.0


@dataclasses.dataclass(frozen=True)
class Intrinsics:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float

    def astuple(self):
        return (float(np.float32(self.fx)), float(np.float32(self.fy)),
                float(np.float32(self.cx)), float(np.float32(self.cy)))


# Camera models of the workloads.
TINY = Intrinsics(64, 48, 52.5, 52.5, 31.5, 23.5)              # 64x48
VGA = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5)         # 640x480
REPLICA = Intrinsics(1200, 680, 600.0, 600.0, 599.5, 339.5)    # 1200x680


def scaled_intrinsics(W: int, H: int) -> Intrinsics:
    """A pinhole camera of size W x H with the VGA field of view."""
    f = 525.0 * W / 640.0
    return Intrinsics(W, H, f, f, (W - 1) / 2.0, (H - 1) / 2.0)


# ----------------------------------------------------------------------------
# small rigid-motion helpers (generic geometry, not the splatting method)


def rotvec_to_matrix(w: np.ndarray) -> np.ndarray:
    """Rodrigues' formula: rotation matrix of the rotation vector ``w``."""
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    if th < 1e-300:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(th) * Kx + (1.0 - math.cos(th)) * (Kx @ Kx)


def identity_pose() -> np.ndarray:
    return np.hstack([np.eye(3), np.zeros((3, 1))])


def compose(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Pose product a*b of two (3,4) rigid transforms."""
    R = a[:, :3] @ b[:, :3]
    t = a[:, :3] @ b[:, 3] + a[:, 3]
    return np.hstack([R, t[:, None]])


def perturb_pose(pose: np.ndarray, rng: np.random.Generator,
                 trans_sigma: float = 0.01, rot_sigma_deg: float = 0.5) -> np.ndarray:
    """Right-multiply ``pose`` by a random small motion (N(0, sigma) per axis)."""
    dR = rotvec_to_matrix(rng.normal(0.0, math.radians(rot_sigma_deg), 3))
    dt = rng.normal(0.0, trans_sigma, 3)
    return compose(pose, np.hstack([dR, dt[:, None]]))


# ----------------------------------------------------------------------------
# procedural room


@dataclasses.dataclass
class Room:
    # planes: normal n (pointing into the room) and offset h with n.X = h
    plane_n: np.ndarray      # (P, 3)
    plane_h: np.ndarray      # (P,)
    sphere_c: np.ndarray     # (S, 3)
    sphere_r: np.ndarray     # (S,)
    albedo: np.ndarray       # (P+S, 3)
    tex_k1: np.ndarray       # (P+S, 3)
    tex_k2: np.ndarray       # (P+S, 3)
    tex_ph: np.ndarray       # (P+S, 2)
    light: np.ndarray        # (3,) unit vector towards the light
    backdrop: np.ndarray     # (3,) colour of rays that leave the room
    x_offset: float = 0.0


def make_room(seed: int = SCENE_SEED, x_offset: float = 0.0) -> Room:
    """Five axis-aligned planes (floor, ceiling, three walls) + three spheres."""
    rng = np.random.default_rng(seed)
    hx, hy, zb = 2.0, 1.4, 3.6
    # y points down: the floor is at y=+hy and faces -y.
    plane_n = np.array([[0, -1, 0], [0, 1, 0], [0, 0, -1], [1, 0, 0], [-1, 0, 0]], np.float64)
    plane_h = np.array([-hy, -hy, -zb, -hx + x_offset, -hx - x_offset], np.float64)
    sphere_r = rng.uniform(0.2, 0.5, 3)
    sphere_c = np.stack([
        rng.uniform(-1.2, 1.2, 3) + x_offset,
        rng.uniform(-0.6, 0.9, 3),
        rng.uniform(1.6, 3.0, 3)], axis=1)
    nprim = 5 + 3
    albedo = rng.uniform(0.0, 1.0, (nprim, 3))
    tex_k1 = rng.uniform(-3.0, 3.0, (nprim, 3))
    tex_k2 = rng.uniform(-3.0, 3.0, (nprim, 3))
    tex_ph = rng.uniform(0.0, 2 * math.pi, (nprim, 2))
    light = rng.normal(0.0, 1.0, 3)
    light[1] = -abs(light[1]) - 0.5   # from above
    light /= np.linalg.norm(light)
    backdrop = rng.uniform(0.2, 0.6, 3)
    return Room(plane_n, plane_h, sphere_c, sphere_r, albedo, tex_k1, tex_k2,
                tex_ph, light, backdrop, x_offset)


def raycast(room: Room, K: Intrinsics, pose: np.ndarray):
    """Ray-cast one RGB-D frame.  Returns (depth (H,W) f32, rgb (3,H,W) f32).

    Depth is the camera z of the first hit, clamped to [0.5, 4] m; rays that
    hit nothing get depth 4 m and the backdrop colour.  Colour is
    albedo * texture * max(0, n.l) + 0.1, clipped to [0, 1].
    """
    H, W = K.H, K.W
    fx, fy, cx, cy = K.astuple()
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    dc = np.empty((H, W, 3))
    dc[..., 0] = ((u - cx) / fx)[None, :]
    dc[..., 1] = ((v - cy) / fy)[:, None]
    dc[..., 2] = 1.0
    R = pose[:, :3]
    o = pose[:, 3]
    dw = dc @ R.T                                     # world ray directions
    best = np.full((H, W), np.inf)
    prim = np.full((H, W), -1, np.int64)
    for i in range(len(room.plane_h)):
        n = room.plane_n[i]
        den = dw @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            s = (room.plane_h[i] - n @ o) / den
        ok = (s > 1e-9) & (s < best)
        best = np.where(ok, s, best)
        prim = np.where(ok, i, prim)
    P = len(room.plane_h)
    for j in range(len(room.sphere_r)):
        oc = o - room.sphere_c[j]
        a = np.einsum("hwk,hwk->hw", dw, dw)
        b = 2.0 * (dw @ oc)
        c = oc @ oc - room.sphere_r[j] ** 2
        disc = b * b - 4 * a * c
        sq = np.sqrt(np.maximum(disc, 0.0))
        s = (-b - sq) / (2 * a)
        ok = (disc > 0) & (s > 1e-9) & (s < best)
        best = np.where(ok, s, best)
        prim = np.where(ok, P + j, prim)
    hit = np.isfinite(best)
    s = np.where(hit, best, DEPTH_MAX)
    X = o[None, None, :] + s[..., None] * dw
    normal = np.zeros_like(X)
    for i in range(P):
        normal[prim == i] = room.plane_n[i]
    for j in range(len(room.sphere_r)):
        m = prim == P + j
        nn = X[m] - room.sphere_c[j]
        normal[m] = nn / np.linalg.norm(nn, axis=1, keepdims=True)
    pid = np.maximum(prim, 0)
    k1 = room.tex_k1[pid]
    k2 = room.tex_k2[pid]
    ph = room.tex_ph[pid]
    tex = 0.75 + 0.25 * np.sin(np.einsum("hwk,hwk->hw", k1, X) + ph[..., 0]) * \
        np.sin(np.einsum("hwk,hwk->hw", k2, X) + ph[..., 1])
    lam = np.maximum(0.0, normal @ room.light)
    col = room.albedo[pid] * (tex * lam)[..., None] + 0.1
    col = np.where(hit[..., None], col, room.backdrop[None, None, :])
    col = np.clip(col, 0.0, 1.0)
    depth = np.clip(s, DEPTH_MIN, DEPTH_MAX)
    return depth.astype(np.float32), np.ascontiguousarray(col.transpose(2, 0, 1)).astype(np.float32)


def trajectory(n_frames: int, seed: int = TRAJECTORY_SEED, max_step_m: float = 0.02,
               max_step_deg: float = 1.0, start: np.ndarray | None = None) -> list:
    """Smooth seeded camera path: every frame moves <= max_step_m and turns
    <= max_step_deg relative to the previous one."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.03, 0.06, 6)          # rad / frame
    ph = rng.uniform(0.0, 2 * math.pi, 6)
    # amplitude * omega bounds the per-frame step (split over three axes)
    At = (max_step_m / math.sqrt(3.0)) * 0.95 / w[:3]
    Ar = math.radians(max_step_deg / math.sqrt(3.0)) * 0.95 / w[3:]
    Ar = Ar * np.array([1.0, 1.0, 0.3])     # little roll
    base = identity_pose() if start is None else start
    poses = []
    for f in range(n_frames):
        tr = At * (np.sin(w[:3] * f + ph[:3]) - np.sin(ph[:3]))
        rv = Ar * (np.sin(w[3:] * f + ph[3:]) - np.sin(ph[3:]))
        # rotation vector in (pitch about x, yaw about y, roll about z)
        Rm = rotvec_to_matrix(rv)
        poses.append(compose(base, np.hstack([Rm, tr[:, None]])))
    return poses


@dataclasses.dataclass
class Frames:
    K: Intrinsics
    poses: list           # list of (3,4) float64
    depth: np.ndarray     # (F, H, W) float32
    rgb: np.ndarray       # (F, 3, H, W) float32


def render_frames(room: Room, K: Intrinsics, poses: list) -> Frames:
    ds, cs = [], []
    for p in poses:
        d, c = raycast(room, K, p)
        ds.append(d)
        cs.append(c)
    return Frames(K, list(poses), np.stack(ds), np.stack(cs))


# ----------------------------------------------------------------------------
# multi-room scene: closed rooms side by side along x (room k spans
# x in [4k - 2, 4k + 2] and has its own seeded spheres, colours and light);
# a frame shows the room its camera is in.

ROOM_PITCH = 4.0


def make_rooms(n_rooms: int, seed: int = SCENE_SEED) -> list:
    return [make_room(seed + 101 * k, x_offset=ROOM_PITCH * k) for k in range(n_rooms)]


def room_of(rooms: list, pose: np.ndarray) -> Room:
    k = int(np.clip(np.floor((pose[0, 3] + ROOM_PITCH / 2) / ROOM_PITCH), 0, len(rooms) - 1))
    return rooms[k]


def multi_room_trajectory(n_frames: int, n_rooms: int, seed: int = TRAJECTORY_SEED,
                          max_step_m: float = 0.02, max_step_deg: float = 1.0) -> list:
    """A smooth seeded path through n_rooms rooms: the camera advances along
    x at a constant speed from 0.6 m inside the first room's far wall to 0.6 m
    before the last room's (at most half of max_step_m per frame) and wanders
    by the seeded sinusoids of trajectory() within the other half of the
    per-frame bounds."""
    speed = (ROOM_PITCH * n_rooms - 1.2) / max(n_frames - 1, 1)
    if speed > 0.5 * max_step_m:
        raise ValueError("too few frames for the rooms at this step bound")
    wander = trajectory(n_frames, seed, max_step_m=0.5 * max_step_m, max_step_deg=max_step_deg)
    x0 = -ROOM_PITCH / 2 + 0.6
    out = []
    for f, p in enumerate(wander):
        q = p.copy()
        q[0, 3] += x0 + speed * f
        q[2, 3] += 0.4
        out.append(q)
    return out


def render_multi(rooms: list, K: Intrinsics, poses: list) -> Frames:
    ds, cs = [], []
    for p in poses:
        d, c = raycast(room_of(rooms, p), K, p)
        ds.append(d)
        cs.append(c)
    return Frames(K, list(poses), np.stack(ds), np.stack(cs))


def tiny_workload(seed: int = SCENE_SEED):
    """64x48, one view at the identity pose, target pose perturbed by
    (1 cm, 0.5 deg) noise."""
    room = make_room(seed)
    fr = render_frames(room, TINY, [identity_pose()])
    rng = np.random.default_rng(POSE_NOISE_SEED)
    target = perturb_pose(identity_pose(), rng)
    return room, fr, target


def tracking_workload(K: Intrinsics = VGA, n_keyframes: int = 8, key_every: int = 5,
                      target_frame: int | None = None):
    """A section of ``n_keyframes`` keyframes (every ``key_every``-th frame of
    a smooth path) plus a target frame to track, its ground-truth pose and a
    perturbed starting pose."""
    room = make_room(SCENE_SEED)
    n_frames = n_keyframes * key_every + 1
    path = trajectory(n_frames)
    keys = [path[i * key_every] for i in range(n_keyframes)]
    if target_frame is None:
        target_frame = (n_keyframes - 1) * key_every + 2
    gt = path[target_frame]
    section = render_frames(room, K, keys)
    target = render_frames(room, K, [gt])
    rng = np.random.default_rng(POSE_NOISE_SEED)
    start = perturb_pose(gt, rng)
    return room, section, target, gt, start


def random_attributes(n: int, seed: int, opacity_range=(0.05, 0.98), colour_jitter=0.0):
    """Seeded random per-Gaussian values a test may substitute for the
    initial ones: colours in [0,1], opacities in ``opacity_range`` and a
    positive radius scale factor in [0.6, 1.8]."""
    rng = np.random.default_rng(seed)
    colour = rng.uniform(0.0, 1.0, (n, 3))
    opacity = rng.uniform(opacity_range[0], opacity_range[1], n)
    rscale = rng.uniform(0.6, 1.8, n)
    return colour, opacity, rscale


def random_ellipsoids(radius, seed: int, spread: float = 0.35):
    """Seeded ellipsoid attributes for the anisotropic variant: per Gaussian
    three axis scales radius * exp(N(0, spread)) and a rotation quaternion
    (w, x, y, z) drawn uniformly (a normalised 4-D normal sample, w >= 0)."""
    rng = np.random.default_rng(seed)
    r = np.asarray(radius, np.float64).reshape(-1)
    scale = r[:, None] * np.exp(rng.normal(0.0, spread, (r.size, 3)))
    q = rng.normal(0.0, 1.0, (r.size, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return scale, q
