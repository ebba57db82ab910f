"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras and target images.

This module only draws inputs. It holds none of the rasterizer's arithmetic
(no projection, binning, compositing or gradients), so both the CUDA path and
the CPU oracle may take their inputs from it.

Scene shapes follow the paper's workloads:

* the camera model of the ReplicaMultiagent Plus renders (Sec. VI, "Rendered
  modalities"): 1200x680 pixels with a 90 degree horizontal field of view,
  hence fx = fy = 600, cx = 600, cy = 340; all agents share one camera model;
* Gaussians carry a centre, per-axis scale, rotation, opacity and RGB colour
  (Sec. III-A, Gaussian seeding; Eq. 19 for how scale and rotation act);
* world-to-camera poses (Sec. III-B, the lifting relation, Eq. 15).

The room generator stands in for Replica-style indoor scenes: Gaussians are
sampled on the interior faces of a box room and on axis-aligned furniture
boxes, flattened along the surface normal, and coloured by smooth noise.
All draws use numpy's PCG64 generator, so a seed gives the same arrays on
every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "Camera", "random_cloud", "room_scene", "room_cameras",
    "floor_scene", "floor_cameras", "smooth_image", "uniform_image",
    "concat_scenes", "look_at", "workload",
]


@dataclass
class Scene:
    """Gaussians as float32 structure-of-arrays.

    means [N,3]; log_scales [N,3] (natural log of the per-axis std-dev);
    quats [N,4] as (w, x, y, z), not necessarily unit; opacities [N] in (0,1)
    (already activated); colors [N,3] RGB in [0,1].
    """
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacities: np.ndarray
    colors: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclass
class Camera:
    """Pinhole camera with a world-to-camera pose p_c = R p_w + t.

    Camera axes: x right, y down, z forward (looking direction).
    """
    R: np.ndarray            # [3,3] float32, row-major
    t: np.ndarray            # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_row(self) -> np.ndarray:
        """R(9), t(3), fx, fy, cx, cy as one float32 row of 16."""
        return np.concatenate([self.R.reshape(9), self.t.reshape(3),
                               np.array([self.fx, self.fy, self.cx, self.cy])]).astype(np.float32)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """Unit quaternions (w,x,y,z) of proper rotation matrices R [N,3,3] (Shepperd's method)."""
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    diag = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    k = np.argmax(diag, 1)
    for case in range(4):
        m = k == case
        if not np.any(m):
            continue
        r = R[m]
        if case == 0:
            s = np.sqrt(1.0 + tr[m]) * 2.0
            q[m, 0] = 0.25 * s
            q[m, 1] = (r[:, 2, 1] - r[:, 1, 2]) / s
            q[m, 2] = (r[:, 0, 2] - r[:, 2, 0]) / s
            q[m, 3] = (r[:, 1, 0] - r[:, 0, 1]) / s
        elif case == 1:
            s = np.sqrt(1.0 + r[:, 0, 0] - r[:, 1, 1] - r[:, 2, 2]) * 2.0
            q[m, 0] = (r[:, 2, 1] - r[:, 1, 2]) / s
            q[m, 1] = 0.25 * s
            q[m, 2] = (r[:, 0, 1] + r[:, 1, 0]) / s
            q[m, 3] = (r[:, 0, 2] + r[:, 2, 0]) / s
        elif case == 2:
            s = np.sqrt(1.0 + r[:, 1, 1] - r[:, 0, 0] - r[:, 2, 2]) * 2.0
            q[m, 0] = (r[:, 0, 2] - r[:, 2, 0]) / s
            q[m, 1] = (r[:, 0, 1] + r[:, 1, 0]) / s
            q[m, 2] = 0.25 * s
            q[m, 3] = (r[:, 1, 2] + r[:, 2, 1]) / s
        else:
            s = np.sqrt(1.0 + r[:, 2, 2] - r[:, 0, 0] - r[:, 1, 1]) * 2.0
            q[m, 0] = (r[:, 1, 0] - r[:, 0, 1]) / s
            q[m, 1] = (r[:, 0, 2] + r[:, 2, 0]) / s
            q[m, 2] = (r[:, 1, 2] + r[:, 2, 1]) / s
            q[m, 3] = 0.25 * s
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# --------------------------------------------------------------------------------------
# Config-1 style cloud in front of an identity camera
# --------------------------------------------------------------------------------------

def random_cloud(n: int = 10_000, seed: int = 1, xy: float = 1.0,
                 z_range=(2.0, 6.0), log_scale=(-3.5, 0.5)) -> Scene:
    """Gaussians uniform in a box in front of an identity camera.

    means: x,y ~ U[-xy, xy], z ~ U[z_range]; log-scales ~ N(mean, std) per axis;
    quats = normalise(N(0,1)^4); opacity = sigmoid(N(0,1)); colour ~ U[0,1]^3.
    """
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-xy, xy, n), rng.uniform(-xy, xy, n),
                      rng.uniform(z_range[0], z_range[1], n)], 1)
    ls = rng.normal(log_scale[0], log_scale[1], (n, 3))
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = _sigmoid(rng.normal(0.0, 1.0, n))
    c = rng.uniform(0.0, 1.0, (n, 3))
    return Scene(_f32(means), _f32(ls), _f32(q), _f32(o), _f32(c))


def identity_camera(width=320, height=240, fx=300.0, fy=300.0, cx=None, cy=None) -> Camera:
    return Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), float(fx), float(fy),
                  float(width / 2 if cx is None else cx), float(height / 2 if cy is None else cy),
                  int(width), int(height))


# --------------------------------------------------------------------------------------
# Surfaces, value noise, rooms
# --------------------------------------------------------------------------------------

@dataclass
class _Rect:
    origin: np.ndarray   # corner
    u: np.ndarray        # edge vector 1
    v: np.ndarray        # edge vector 2
    normal: np.ndarray   # unit normal facing the visible side

    @property
    def area(self) -> float:
        return float(np.linalg.norm(np.cross(self.u, self.v)))


def _R(o, u, v, n):
    return _Rect(np.asarray(o, float), np.asarray(u, float), np.asarray(v, float), np.asarray(n, float))


def _box_faces(x0, y0, sx, sy, sz) -> list:
    """Five exposed faces (top and four sides) of a box resting on z=0."""
    return [
        _R((x0, y0, sz), (sx, 0, 0), (0, sy, 0), (0, 0, 1)),
        _R((x0, y0, 0), (0, sy, 0), (0, 0, sz), (-1, 0, 0)),
        _R((x0 + sx, y0, 0), (0, sy, 0), (0, 0, sz), (1, 0, 0)),
        _R((x0, y0, 0), (sx, 0, 0), (0, 0, sz), (0, -1, 0)),
        _R((x0, y0 + sy, 0), (sx, 0, 0), (0, 0, sz), (0, 1, 0)),
    ]


def _room_faces(x0, y0, lx, ly, lz) -> list:
    """Interior faces of an axis-aligned box room (floor, ceiling, four walls)."""
    return [
        _R((x0, y0, 0), (lx, 0, 0), (0, ly, 0), (0, 0, 1)),
        _R((x0, y0, lz), (lx, 0, 0), (0, ly, 0), (0, 0, -1)),
        _R((x0, y0, 0), (0, ly, 0), (0, 0, lz), (1, 0, 0)),
        _R((x0 + lx, y0, 0), (0, ly, 0), (0, 0, lz), (-1, 0, 0)),
        _R((x0, y0, 0), (lx, 0, 0), (0, 0, lz), (0, 1, 0)),
        _R((x0, y0 + ly, 0), (lx, 0, 0), (0, 0, lz), (0, -1, 0)),
    ]


def _value_noise(points: np.ndarray, seed: int, base_cell=0.5, octaves=3) -> np.ndarray:
    """Smooth RGB value noise in [0,1]: random lattice values, trilinear interpolation,
    octaves at cell sizes base_cell / 2^k with weights 2^-k."""
    rng = np.random.default_rng(seed)
    lo = points.min(0) - 1e-3
    out = np.zeros((points.shape[0], 3))
    wsum = 0.0
    for k in range(octaves):
        cell = base_cell / (2 ** k)
        g = (points - lo) / cell
        dims = np.floor(g.max(0)).astype(int) + 2
        lattice = rng.uniform(0.0, 1.0, (dims[0], dims[1], dims[2], 3))
        i0 = np.floor(g).astype(int)
        f = g - i0
        f = f * f * (3 - 2 * f)          # smoothstep weights (C1-continuous)
        acc = np.zeros_like(out)
        for dx in (0, 1):
            wx = f[:, 0] if dx else 1 - f[:, 0]
            for dy in (0, 1):
                wy = f[:, 1] if dy else 1 - f[:, 1]
                for dz in (0, 1):
                    wz = f[:, 2] if dz else 1 - f[:, 2]
                    acc += (wx * wy * wz)[:, None] * lattice[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
        w = 0.5 ** k
        out += w * acc
        wsum += w
    return np.clip(out / wsum, 0.0, 1.0)


def _surface_gaussians(faces: list, n: int, rng, log_scale=(-4.5, 0.4), opacity=(1.0, 1.0)):
    """Sample n Gaussians on the faces, count per face proportional to area.

    The smallest of three N(log_scale) draws goes on the surface normal; the other two
    axes lie in the face plane with a random in-plane rotation.
    """
    areas = np.array([f.area for f in faces])
    face_idx = rng.choice(len(faces), size=n, p=areas / areas.sum())
    a = rng.uniform(0, 1, n)
    b = rng.uniform(0, 1, n)
    O = np.stack([faces[i].origin for i in range(len(faces))])
    U = np.stack([faces[i].u for i in range(len(faces))])
    V = np.stack([faces[i].v for i in range(len(faces))])
    Nrm = np.stack([faces[i].normal for i in range(len(faces))])
    means = O[face_idx] + a[:, None] * U[face_idx] + b[:, None] * V[face_idx]
    nrm = Nrm[face_idx]
    e1 = U[face_idx] / np.linalg.norm(U[face_idx], axis=1, keepdims=True)
    e2 = np.cross(nrm, e1)
    th = rng.uniform(0, 2 * np.pi, n)
    t1 = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
    t2 = np.cross(nrm, t1)
    Rg = np.stack([t1, t2, nrm], 2)          # columns: local x, y, z(=normal)
    quats = _quat_from_matrix(Rg)
    ls = np.sort(rng.normal(log_scale[0], log_scale[1], (n, 3)), axis=1)[:, ::-1]  # big, mid, small
    o = _sigmoid(rng.normal(opacity[0], opacity[1], n))
    return means, ls, quats, o


def _boxes(rng, n_boxes, x0, y0, lx, ly, margin=0.0):
    out = []
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.3, 1.5), rng.uniform(0.3, 1.5), rng.uniform(0.3, 1.2)
        bx = rng.uniform(x0 + margin, x0 + lx - sx - margin)
        by = rng.uniform(y0 + margin, y0 + ly - sy - margin)
        out.append((bx, by, sx, sy, sz))
    return out


def room_scene(n: int = 500_000, seed: int = 10, size=(6.0, 5.0, 3.0), n_boxes: int = 12) -> Scene:
    """Replica-shaped room: Gaussians on the interior faces of a size[0] x size[1] x size[2] m box
    room and on the five exposed faces of n_boxes furniture boxes resting on the floor."""
    rng = np.random.default_rng(seed)
    lx, ly, lz = size
    boxes = _boxes(rng, n_boxes, 0.0, 0.0, lx, ly)
    faces = _room_faces(0.0, 0.0, lx, ly, lz)
    for b in boxes:
        faces += _box_faces(*b)
    means, ls, q, o = _surface_gaussians(faces, n, rng)
    col = _value_noise(means, seed + 7919)
    sc = Scene(_f32(means), _f32(ls), _f32(q), _f32(o), _f32(col))
    sc.boxes = boxes  # type: ignore[attr-defined]
    sc.room = (0.0, 0.0, lx, ly, lz)  # type: ignore[attr-defined]
    return sc


def look_at(center, target, width, height, fx, fy, cx, cy) -> Camera:
    """World-to-camera pose of a camera at `center` looking at `target`, world up = +z."""
    c = np.asarray(center, float)
    f = np.asarray(target, float) - c
    f /= np.linalg.norm(f)
    r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], 0)
    t = -R @ c
    return Camera(_f32(R), _f32(t), float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def _camera_in_room(rng, room, boxes, width, height, fx, fy, cx, cy, shrink=0.5):
    x0, y0, lx, ly, lz = room
    for _ in range(1000):
        c = np.array([rng.uniform(x0 + shrink, x0 + lx - shrink), rng.uniform(y0 + shrink, y0 + ly - shrink),
                      rng.uniform(1.2, 1.8)])
        if all(not (bx - 0.3 <= c[0] <= bx + sx + 0.3 and by - 0.3 <= c[1] <= by + sy + 0.3 and c[2] <= sz + 0.3)
               for (bx, by, sx, sy, sz) in boxes):
            break
    walls = [((x0, y0), (0, ly)), ((x0 + lx, y0), (0, ly)), ((x0, y0), (lx, 0)), ((x0, y0 + ly), (lx, 0))]
    lens = np.array([abs(w[1][0]) + abs(w[1][1]) for w in walls])
    k = rng.choice(4, p=lens / lens.sum())
    (ox, oy), (ux, uy) = walls[k]
    a = rng.uniform(0.05, 0.95)
    tgt = np.array([ox + a * ux, oy + a * uy, rng.uniform(0.3, lz - 0.3)])
    return look_at(c, tgt, width, height, fx, fy, cx, cy)


REPLICA_CAM = dict(width=1200, height=680, fx=600.0, fy=600.0, cx=600.0, cy=340.0)


def room_cameras(scene: Scene, n_views: int, seed: int, **cam) -> list:
    """Cameras inside the room (interior shrunk by 0.5 m, height U[1.2,1.8], clear of furniture),
    each looking at a random wall point."""
    cam = {**REPLICA_CAM, **cam}
    rng = np.random.default_rng(seed)
    return [_camera_in_room(rng, scene.room, scene.boxes, **cam) for _ in range(n_views)]  # type: ignore


def floor_scene(n: int = 4_000_000, seed: int = 500, size=(20.0, 15.0, 3.0), grid=(3, 2),
                boxes_per_room: int = 8, agents=(4, 4), door=(1.0, 2.1), wall=0.1) -> Scene:
    """Multi-room floor: grid[0] x grid[1] rooms of equal size joined by door-sized openings in the
    interior walls, furniture in each room.  Gaussians are grouped into agents[0]*agents[1]
    spatial submaps (contiguous row ranges, `scene.agent_offsets`)."""
    rng = np.random.default_rng(seed)
    LX, LY, LZ = size
    gx, gy = grid
    rx, ry = LX / gx, LY / gy
    faces = []
    rooms = []
    all_boxes = []
    dw, dh = door
    for i in range(gx):
        for j in range(gy):
            x0, y0 = i * rx, j * ry
            rooms.append((x0 + wall / 2, y0 + wall / 2, rx - wall, ry - wall, LZ))
            # floor & ceiling
            faces.append(_R((x0, y0, 0), (rx, 0, 0), (0, ry, 0), (0, 0, 1)))
            faces.append(_R((x0, y0, LZ), (rx, 0, 0), (0, ry, 0), (0, 0, -1)))
            bx = _boxes(rng, boxes_per_room, x0 + wall, y0 + wall, rx - 2 * wall, ry - 2 * wall, margin=0.05)
            all_boxes += bx
            for b in bx:
                faces += _box_faces(*b)
    # walls: for each wall line, faces on each side; interior walls get a centred door per room span
    def wall_faces(p0, along, length, normal, has_door):
        along = np.asarray(along, float)
        up = np.array([0, 0, LZ], float)
        if not has_door:
            return [_R(p0, along * length, up, normal)]
        a = (length - dw) / 2
        p0 = np.asarray(p0, float)
        return [_R(p0, along * a, up, normal),
                _R(p0 + along * (a + dw), along * a, up, normal),
                _R(p0 + along * a + np.array([0, 0, dh]), along * dw, np.array([0, 0, LZ - dh]), normal)]
    ex, ey = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    for i in range(gx + 1):          # walls at x = i*rx, spans over each room row
        for j in range(gy):
            interior = 0 < i < gx
            x = i * rx
            if i > 0:      # face looking -x (belongs to room i-1)
                faces += wall_faces((x - wall / 2 * interior, j * ry, 0), ey, ry, (-1, 0, 0), interior)
            if i < gx:     # face looking +x
                faces += wall_faces((x + wall / 2 * interior, j * ry, 0), ey, ry, (1, 0, 0), interior)
    for j in range(gy + 1):
        for i in range(gx):
            interior = 0 < j < gy
            y = j * ry
            if j > 0:
                faces += wall_faces((i * rx, y - wall / 2 * interior, 0), ex, rx, (0, -1, 0), interior)
            if j < gy:
                faces += wall_faces((i * rx, y + wall / 2 * interior, 0), ex, rx, (0, 1, 0), interior)
    means, ls, q, o = _surface_gaussians(faces, n, rng)
    col = _value_noise(means, seed + 7919)
    ax, ay = agents
    cell = (np.clip((means[:, 0] / (LX / ax)).astype(int), 0, ax - 1) * ay
            + np.clip((means[:, 1] / (LY / ay)).astype(int), 0, ay - 1))
    order = np.argsort(cell, kind="stable")
    counts = np.bincount(cell, minlength=ax * ay)
    sc = Scene(_f32(means[order]), _f32(ls[order]), _f32(q[order]), _f32(o[order]), _f32(col[order]))
    sc.agent_offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)  # type: ignore
    sc.rooms = rooms  # type: ignore
    sc.boxes = all_boxes  # type: ignore
    sc.agents = agents  # type: ignore
    sc.size = size  # type: ignore
    return sc


def floor_cameras(scene: Scene, per_agent: int, seed: int, **cam) -> list:
    """per_agent cameras for each agent, placed in the agent's cell of the floor (inside a room),
    looking at a random wall point of that room."""
    cam = {**REPLICA_CAM, **cam}
    rng = np.random.default_rng(seed)
    LX, LY, _ = scene.size  # type: ignore
    ax, ay = scene.agents  # type: ignore
    out = []
    for a in range(ax * ay):
        cx0, cy0 = (a // ay) * LX / ax, (a % ay) * LY / ay
        ctr = np.array([cx0 + LX / ax / 2, cy0 + LY / ay / 2])
        room = min(scene.rooms, key=lambda r: (np.clip(ctr[0], r[0], r[0] + r[2]) - ctr[0]) ** 2  # type: ignore
                   + (np.clip(ctr[1], r[1], r[1] + r[3]) - ctr[1]) ** 2)
        # restrict the room to the agent's cell where they overlap
        x0 = max(room[0], cx0)
        y0 = max(room[1], cy0)
        x1 = min(room[0] + room[2], cx0 + LX / ax)
        y1 = min(room[1] + room[3], cy0 + LY / ay)
        if x1 - x0 < 1.2 or y1 - y0 < 1.2:
            x0, y0, x1, y1 = room[0], room[1], room[0] + room[2], room[1] + room[3]
        sub = (x0, y0, x1 - x0, y1 - y0, room[4])
        for _ in range(per_agent):
            cm = _camera_in_room(rng, sub, scene.boxes, **cam)  # type: ignore
            out.append(cm)
    return out


def concat_scenes(scenes: list) -> tuple:
    """Concatenate scenes row-wise; returns (Scene, offsets[S+1] int64)."""
    cat = Scene(*[np.ascontiguousarray(np.concatenate([getattr(s, k) for s in scenes], 0))
                  for k in ("means", "log_scales", "quats", "opacities", "colors")])
    offs = np.concatenate([[0], np.cumsum([s.n for s in scenes])]).astype(np.int64)
    return cat, offs


def uniform_image(width, height, seed, channels=3) -> np.ndarray:
    """[channels,H,W] float32 ~ U[0,1]."""
    return _f32(np.random.default_rng(seed).uniform(0.0, 1.0, (channels, height, width)))


def smooth_image(width, height, seed, channels=3, cell=24.0, lo=0.0, hi=1.0) -> np.ndarray:
    """[channels,H,W] float32 smooth value noise in [lo,hi] (2-D, cell in pixels)."""
    ys, xs = np.mgrid[0:height, 0:width].astype(float)
    pts = np.stack([xs.ravel() / cell * 0.5, ys.ravel() / cell * 0.5, np.zeros(xs.size)], 1)
    out = np.empty((channels, height, width))
    for c in range(channels):
        out[c] = _value_noise(pts, seed * 31 + c, base_cell=0.5, octaves=3)[:, 0].reshape(height, width)
    return _f32(lo + (hi - lo) * out)


# --------------------------------------------------------------------------------------
# Named workloads (the five configurations of the rasterizer benchmark)
# --------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    scene: Scene
    scene_offsets: np.ndarray          # [S+1]
    cameras: list                      # V cameras
    scene_of_view: np.ndarray          # [V] int32
    width: int
    height: int
    meta: dict = field(default_factory=dict)


def workload(name: str, scale: float = 1.0) -> Workload:
    """Build one of the named workloads.  `scale` < 1 shrinks Gaussian counts (test sizes).

    cloud10k   : 10k Gaussians, 320x240, identity camera (fx=fy=300).
    room500k   : 500k-Gaussian room, one 1200x680 view.
    agents8x4  : 8 rooms of 50k..400k Gaussians, 4 views each (32 views).
    room1m     : 1M-Gaussian room, 8 views.
    floor4m    : 4M-Gaussian multi-room floor, 16 agent submaps, 64 views.
    """
    def nn(x):
        return max(16, int(round(x * scale)))
    if name == "cloud10k":
        sc = random_cloud(nn(10_000), seed=1)
        cams = [identity_camera(320, 240, 300.0, 300.0, 160.0, 120.0)]
        return Workload(name, sc, np.array([0, sc.n], np.int64), cams, np.zeros(1, np.int32), 320, 240)
    if name == "room500k":
        sc = room_scene(nn(500_000), seed=10)
        cams = room_cameras(sc, 1, seed=11)
        return Workload(name, sc, np.array([0, sc.n], np.int64), cams, np.zeros(1, np.int32), 1200, 680)
    if name == "agents8x4":
        counts = [50_000, 80_000, 120_000, 160_000, 200_000, 260_000, 330_000, 400_000]
        scenes, cams, sov = [], [], []
        for a, c in enumerate(counts):
            s = room_scene(nn(c), seed=100 + a)
            scenes.append(s)
            cams += room_cameras(s, 4, seed=1000 + a)
            sov += [a] * 4
        sc, offs = concat_scenes(scenes)
        return Workload(name, sc, offs, cams, np.array(sov, np.int32), 1200, 680)
    if name == "room1m":
        sc = room_scene(nn(1_000_000), seed=200)
        cams = room_cameras(sc, 8, seed=201)
        return Workload(name, sc, np.array([0, sc.n], np.int64), cams, np.zeros(8, np.int32), 1200, 680)
    if name == "floor4m":
        sc = floor_scene(nn(4_000_000), seed=500)
        cams = floor_cameras(sc, 4, seed=501)
        return Workload(name, sc, np.array([0, sc.n], np.int64), cams, np.zeros(len(cams), np.int32), 1200, 680,
                        meta={"agent_offsets": sc.agent_offsets})  # type: ignore
    raise KeyError(name)
