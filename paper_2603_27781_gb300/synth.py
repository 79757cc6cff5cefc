"""Seeded synthetic workloads for the semantic-splatting rasterizer.

This module only draws numbers: Gaussian fields, pinhole cameras, keyframe
trajectories and RGB-D-semantic target frames.  It contains none of the
splatting method's arithmetic (no projection of Gaussians, no blending, no
loss), so both the CUDA path and the FP64 oracle can be fed from it without
sharing any of the computation they are compared on.

The paper measures on real RGB-D sequences with 2D semantic labels (Replica at
1200x680, ScanNet at 640x480; Sec. 4.1.2).  Those are not available, so these
scenes stand in for their shape: an indoor room with planar walls, floor,
ceiling and box furniture, Gaussians sampled area-proportionally on the
surfaces, and target frames obtained by casting pixel rays against the same
analytic room (depth = camera-frame z of the first hit, colour = a procedural
albedo of the hit surface, label = the surface's class).

All arrays are little-endian numpy; Gaussian parameters are float32 SoA:
means [N,3], quats [N,4] as (w,x,y,z) unnormalised, log_scales [N,3],
opacity_logits [N], rgb [N,3], feat [N,D].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_SCENE = 0
SEED_TARGET = 1
SEED_DECODER = 2
SEED_POSE = 3
SEED_KEYFRAMES = 4
SEED_FD = 5


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class Gaussians:
    means: np.ndarray
    quats: np.ndarray
    log_scales: np.ndarray
    opacity_logits: np.ndarray
    rgb: np.ndarray
    feat: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def feat_dim(self) -> int:
        return int(self.feat.shape[1])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(*(np.ascontiguousarray(a[idx]) for a in dataclasses.astuple(self)))

    def copy(self) -> "Gaussians":
        return Gaussians(*(a.copy() for a in dataclasses.astuple(self)))

    def arrays(self):
        return dataclasses.astuple(self)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_cw: np.ndarray  # 4x4 float64, world -> camera, OpenCV axes (x right, y down, z forward)


@dataclasses.dataclass
class Frame:
    rgb: np.ndarray    # [3,H,W] float32 in [0,1]
    depth: np.ndarray  # [H,W] float32, metres, 0 = no measurement
    label: np.ndarray  # [H,W] uint8 class id, 255 = unlabelled


@dataclasses.dataclass
class Decoder:
    W: np.ndarray  # [K,D] float32
    b: np.ndarray  # [K] float32


# ---------------------------------------------------------------- parameters
def _common_params(g: np.random.Generator, n: int, d: int, log_scale_mu: float,
                   log_scale_sd: float):
    quats = g.standard_normal((n, 4))
    quats /= np.linalg.norm(quats, axis=1, keepdims=True)
    log_scales = g.normal(log_scale_mu, log_scale_sd, (n, 3))
    opacity_logits = g.standard_normal(n)
    rgb = g.random((n, 3))
    feat = g.standard_normal((n, d))
    return quats, log_scales, opacity_logits, rgb, feat


def _pack(means, quats, log_scales, opacity_logits, rgb, feat) -> Gaussians:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Gaussians(f(means), f(quats), f(log_scales), f(opacity_logits), f(rgb), f(feat))


def box_field(n: int, d: int = 16, seed: int = SEED_SCENE) -> Gaussians:
    """Gaussians in a 2x2x2 m box whose near face is 3 m in front of an identity camera.

    Means ~ U([-1,1]^2 x [3,5]); log-scales ~ N(-3, 0.3) per axis; unit quaternions
    from normalised N(0,I4); opacity logits ~ N(0,1); RGB ~ U[0,1]; features ~ N(0,1).
    """
    g = rng(seed)
    means = np.stack([g.uniform(-1, 1, n), g.uniform(-1, 1, n), g.uniform(3, 5, n)], 1)
    return _pack(means, *_common_params(g, n, d, -3.0, 0.3))


# ------------------------------------------------------------------- the room
@dataclasses.dataclass
class Room:
    size: np.ndarray            # (6, 5, 3) metres, world z is up, floor at z=0
    boxes: np.ndarray           # [nb, 2, 3] axis-aligned (lo, hi)
    albedo: np.ndarray          # [n_surfaces, 3] base colour per surface id
    surface_class: np.ndarray   # [n_surfaces] class id per surface


def make_room(seed: int = SEED_SCENE, n_boxes: int = 20, n_classes: int = 8) -> Room:
    g = rng(seed + 1000)
    size = np.array([6.0, 5.0, 3.0])
    boxes = np.zeros((n_boxes, 2, 3))
    for i in range(n_boxes):
        side = g.uniform(0.2, 1.0, 3)
        lo_xy = g.uniform([0.1, 0.1], size[:2] - side[:2] - 0.1)
        boxes[i, 0] = [lo_xy[0], lo_xy[1], 0.0]
        boxes[i, 1] = [lo_xy[0] + side[0], lo_xy[1] + side[1], side[2]]
    n_surf = 6 + n_boxes
    albedo = g.uniform(0.15, 0.9, (n_surf, 3))
    surface_class = np.concatenate([np.arange(6) % n_classes,
                                    6 + g.integers(0, n_classes - 6 if n_classes > 6 else 1, n_boxes)])
    surface_class = (surface_class % n_classes).astype(np.uint8)
    return Room(size, boxes, albedo, surface_class)


def _room_faces(room: Room):
    """Rectangles (origin, edge u, edge v) of the 6 room faces and 5 faces per box."""
    sx, sy, sz = room.size
    o = np.zeros(3)
    faces = [
        (o, np.array([sx, 0, 0]), np.array([0, sy, 0])),               # floor
        (np.array([0, 0, sz]), np.array([sx, 0, 0]), np.array([0, sy, 0])),  # ceiling
        (o, np.array([sx, 0, 0]), np.array([0, 0, sz])),               # wall y=0
        (np.array([0, sy, 0]), np.array([sx, 0, 0]), np.array([0, 0, sz])),  # wall y=sy
        (o, np.array([0, sy, 0]), np.array([0, 0, sz])),               # wall x=0
        (np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, sz])),  # wall x=sx
    ]
    owner = list(range(6))
    for b, (lo, hi) in enumerate(room.boxes):
        e = hi - lo
        ex, ey, ez = np.array([e[0], 0, 0]), np.array([0, e[1], 0]), np.array([0, 0, e[2]])
        faces += [
            (np.array([lo[0], lo[1], hi[2]]), ex, ey),   # top
            (lo, ex, ez), (np.array([lo[0], hi[1], lo[2]]), ex, ez),
            (lo, ey, ez), (np.array([hi[0], lo[1], lo[2]]), ey, ez),
        ]
        owner += [6 + b] * 5
    return faces, np.array(owner)


def room_field(n: int, d: int = 16, seed: int = SEED_SCENE, room: Room | None = None,
               jitter: float = 0.01, log_scale_mu: float = -4.0,
               log_scale_sd: float = 0.5) -> Gaussians:
    """N Gaussians sampled area-proportionally on the room's surfaces, jittered N(0, jitter^2)."""
    room = room or make_room(seed)
    g = rng(seed)
    faces, _ = _room_faces(room)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v in faces])
    which = g.choice(len(faces), size=n, p=areas / areas.sum())
    a, b = g.random(n), g.random(n)
    org = np.array([f[0] for f in faces])[which]
    eu = np.array([f[1] for f in faces])[which]
    ev = np.array([f[2] for f in faces])[which]
    means = org + a[:, None] * eu + b[:, None] * ev + g.normal(0, jitter, (n, 3))
    return _pack(means, *_common_params(g, n, d, log_scale_mu, log_scale_sd))


def jitter_means(gs: Gaussians, sigma: float = 0.01, seed: int = SEED_TARGET) -> Gaussians:
    out = gs.copy()
    out.means = (gs.means + rng(seed).normal(0, sigma, gs.means.shape)).astype(np.float32)
    return out


# ----------------------------------------------------------------- cameras
def look_pose(position, forward, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera 4x4 for a camera at `position` looking along `forward` (OpenCV axes)."""
    f = np.asarray(forward, float)
    f = f / np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, float))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R_wc = np.stack([right, down, f], 1)
    T = np.eye(4)
    T[:3, :3] = R_wc.T
    T[:3, 3] = -R_wc.T @ np.asarray(position, float)
    return T


def axis_angle(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def perturb_pose(T_cw: np.ndarray, deg: float = 2.0, metres: float = 0.05,
                 seed: int = SEED_POSE) -> np.ndarray:
    """Left-multiply T_cw by a rotation of `deg` about a random axis and a random `metres` shift."""
    g = rng(seed)
    axis = g.standard_normal(3)
    shift = g.standard_normal(3)
    D = np.eye(4)
    D[:3, :3] = axis_angle(axis, math.radians(deg))
    D[:3, 3] = metres * shift / np.linalg.norm(shift)
    return D @ T_cw


def camera(width, height, fx, fy=None, cx=None, cy=None, T_cw=None, round_f32=True) -> Camera:
    """Pinhole camera.  By default intrinsics and pose are rounded to float32 values (the
    C ABI's camera is float32), so every consumer sees exactly the same camera."""
    f = (lambda x: float(np.float32(x))) if round_f32 else float
    T = np.eye(4) if T_cw is None else np.asarray(T_cw, float)
    if round_f32:
        T = T.astype(np.float32).astype(np.float64)
    return Camera(int(width), int(height), f(fx), f(fx if fy is None else fy),
                  f(width / 2 if cx is None else cx), f(height / 2 if cy is None else cy), T)


def room_camera(width=1200, height=680, fx=600.0, room: Room | None = None,
                position=(3.0, 2.5, 1.5), forward=(1.0, 0.0, 0.0)) -> Camera:
    return camera(width, height, fx, T_cw=look_pose(position, forward))


def keyframe_loop(n_poses: int = 200, seed: int = SEED_KEYFRAMES, room: Room | None = None):
    """World->camera poses on a closed ellipse through the room, 1.2-1.8 m high,
    yaw along the tangent +- 30 degrees."""
    room = room or make_room()
    g = rng(seed)
    cx, cy = room.size[0] / 2, room.size[1] / 2
    rx, ry = 0.35 * room.size[0], 0.35 * room.size[1]
    poses = []
    for k in range(n_poses):
        th = 2 * math.pi * k / n_poses
        pos = (cx + rx * math.cos(th), cy + ry * math.sin(th), 1.5 + 0.3 * math.sin(3 * th))
        tangent = math.atan2(ry * math.cos(th), -rx * math.sin(th))
        yaw = tangent + math.radians(g.uniform(-30, 30))
        poses.append(look_pose(pos, (math.cos(yaw), math.sin(yaw), g.uniform(-0.15, 0.15))))
    return poses


def smooth_path(n: int, step_deg: float = 0.6, room: Room | None = None):
    """World->camera poses of a camera moving along the loop ellipse without yaw jitter: n
    consecutive frames, each step_deg of the ellipse apart, looking along the tangent."""
    room = room or make_room()
    cx, cy = room.size[0] / 2, room.size[1] / 2
    rx, ry = 0.35 * room.size[0], 0.35 * room.size[1]
    poses = []
    for k in range(n):
        th = math.radians(step_deg * k)
        pos = (cx + rx * math.cos(th), cy + ry * math.sin(th), 1.5)
        tangent = math.atan2(ry * math.cos(th), -rx * math.sin(th))
        poses.append(look_pose(pos, (math.cos(tangent), math.sin(tangent), -0.05)))
    return poses


def draw_keyframes(n: int, n_poses: int = 200, seed: int = SEED_KEYFRAMES):
    """Indices of n keyframes drawn i.i.d. uniformly from the n_poses loop poses."""
    return rng(seed + 7).integers(0, n_poses, n)


def decoder(k: int, d: int, seed: int = SEED_DECODER) -> Decoder:
    g = rng(seed)
    s = 1.0 / math.sqrt(max(d, 1))
    return Decoder(g.normal(0, s, (k, d)).astype(np.float32), g.normal(0, s, k).astype(np.float32))


# ------------------------------------------------------------ target frames
def raycast_room(room: Room, cam: Camera) -> Frame:
    """Sensor frame of the analytic room seen by `cam` (pixel centres at +0.5)."""
    H, W = cam.height, cam.width
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    dc = np.stack([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy,
                   np.ones_like(px)], -1).reshape(-1, 3)          # camera-frame ray, z = 1
    R_cw, t_cw = cam.T_cw[:3, :3], cam.T_cw[:3, 3]
    origin = -R_cw.T @ t_cw
    d = dc @ R_cw                                                # world direction (R_wc @ dc)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        # exit from the room interior
        t_hi = np.where(d > 0, (room.size - origin) * inv, -origin * inv)
        t_hi = np.where(np.isfinite(t_hi), t_hi, np.inf)
        t_room = t_hi.min(1)
        exit_axis = t_hi.argmin(1)
        sign = np.take_along_axis(d, exit_axis[:, None], 1)[:, 0] > 0
        surf = np.choose(exit_axis, [np.where(sign, 5, 4), np.where(sign, 3, 2), np.where(sign, 1, 0)])
        t_best = t_room.copy()
        for b, (lo, hi) in enumerate(room.boxes):
            t0 = (lo - origin) * inv
            t1 = (hi - origin) * inv
            tn = np.nanmax(np.minimum(t0, t1), 1)
            tf = np.nanmin(np.maximum(t0, t1), 1)
            hit = (tn <= tf) & (tn > 1e-6) & (tn < t_best)
            t_best = np.where(hit, tn, t_best)
            surf = np.where(hit, 6 + b, surf)
    hitp = origin + t_best[:, None] * d
    tex = 0.5 + 0.5 * np.sin(7.0 * hitp[:, 0]) * np.sin(5.0 * hitp[:, 1] + 3.0 * hitp[:, 2])
    rgb = np.clip(room.albedo[surf] * (0.6 + 0.4 * tex[:, None]), 0, 1)
    depth = t_best  # camera-frame z of the hit point, since dc has z = 1
    label = room.surface_class[surf]
    return Frame(np.ascontiguousarray(rgb.T.reshape(3, H, W), dtype=np.float32),
                 depth.reshape(H, W).astype(np.float32), label.reshape(H, W).astype(np.uint8))


def random_frame(cam: Camera, k: int, seed: int = SEED_TARGET, depth_range=(2.5, 5.5)) -> Frame:
    """Unstructured target frame (uniform colour/depth, random labels) for small tests."""
    g = rng(seed)
    H, W = cam.height, cam.width
    return Frame(g.random((3, H, W)).astype(np.float32),
                 g.uniform(*depth_range, (H, W)).astype(np.float32),
                 g.integers(0, k, (H, W)).astype(np.uint8))


SEED_SLAM = 6


def rskm_draws(n: int, seed: int = SEED_SLAM) -> np.ndarray:
    """n uniform 32-bit random words for keyframe draws (uint32)."""
    return rng(seed).integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)


def feature_bank(n: int, d: int, seed: int = SEED_SLAM + 1) -> np.ndarray:
    """n rows of N(0, 1) features [n, d] float32 for Gaussians added by expansion."""
    return rng(seed).standard_normal((n, d)).astype(np.float32)
