"""Seeded synthetic scenes and frames for the DISC integration step.

Input plumbing only: a ray caster over boxes/ellipsoids in a box room, masks
from the largest visible objects, and patch tokens drawn as a per-object mean
plus noise.  It contains none of the integration method's arithmetic and is
shared by the oracle, the CUDA path, the tests and the benchmark.

Workloads (stand-ins for the paper's Replica/ScanNet/HM3D trajectories, which
are not available here):
  * ``tiny``:  4x4x3 m room, 4 axis-aligned boxes, 20 orbit frames of 64x48,
    fx = fy = 50, tokens 8x6x512, <= 8 masks, voxel 5 cm.
  * ``room``:  10x8x3 m room, 80 random boxes/ellipsoids (0.2-1.5 m),
    a smooth closed path of 2000 frames at 1.2 m height, 640x480, fx = fy = 525,
    1 % multiplicative depth noise, 40 masks, tokens 24x24x768, voxel 2.5 cm.
  * ``multistory``: 3 floors of 40x30 m (3 m each) split into 8 rooms per floor
    by partition walls along a central corridor, 1000 random objects, a
    serpentine path through every room of every floor (5000 frames at 1.2 m
    above the floor), 640x480, <= 100 masks, tokens 24x24x768, voxel 5 cm,
    valid depth up to 20 m.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdisc_synth.so")


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", _SO, src, "-lm"])
    return _SO


class _Prim(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("id", ctypes.c_int32),
                ("c", ctypes.c_double * 3), ("h", ctypes.c_double * 3)]


class _Scene(ctypes.Structure):
    _fields_ = [("room_lo", ctypes.c_double * 3), ("room_hi", ctypes.c_double * 3),
                ("face_id", ctypes.c_int32 * 6), ("tile", ctypes.c_double),
                ("n_prims", ctypes.c_int32),
                ("prims", ctypes.POINTER(_Prim)),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("depth_noise", ctypes.c_double),
                ("patch_h", ctypes.c_int32), ("patch_w", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("token_noise", ctypes.c_double), ("max_masks", ctypes.c_int32),
                ("max_id", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("grid_nx", ctypes.c_int32), ("grid_ny", ctypes.c_int32),
                ("grid_x0", ctypes.c_double), ("grid_y0", ctypes.c_double), ("grid_cell", ctypes.c_double),
                ("cell_start", ctypes.POINTER(ctypes.c_int32)), ("cell_items", ctypes.POINTER(ctypes.c_int32))]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_render.restype = ctypes.c_int
        _lib.synth_render.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
        _lib.synth_assoc_tokens.restype = ctypes.c_int
        _lib.synth_assoc_tokens.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_void_p]
        _lib.synth_object_mean.restype = None
        _lib.synth_object_mean.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int32, ctypes.c_void_p]
    return _lib


@dataclasses.dataclass
class Scene:
    """A static scene plus a camera trajectory and the frame/token format."""
    name: str
    room_lo: tuple
    room_hi: tuple
    face_ids: tuple            # base id of -x, +x, -y, +y, floor, ceiling
    prims: list                # (kind, id, centre(3), half-extent or radii(3))
    poses: np.ndarray          # [F, 4, 4] camera->world, float64
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    depth_noise: float
    patch_h: int
    patch_w: int
    dim: int
    token_noise: float
    max_masks: int
    voxel_size: float
    z_min: float
    z_max: float
    seed: int
    tile: float = 0.0          # > 0: room faces cut into panels, one id each

    @property
    def num_frames(self) -> int:
        return int(self.poses.shape[0])

    @property
    def max_id(self) -> int:
        ids = [p[1] for p in self.prims] + list(self.face_ids)
        if self.tile > 0:
            ids += [self.face_ids[f] + self._panels(f) - 1 for f in range(6)]
        return int(max(ids))

    def _panels(self, face: int) -> int:
        a = face // 2
        b0, b1 = (1 if a == 0 else 0), (1 if a == 2 else 2)
        ext = [self.room_hi[i] - self.room_lo[i] for i in range(3)]
        return int(np.ceil(ext[b0] / self.tile - 1e-9)) * int(np.ceil(ext[b1] / self.tile - 1e-9))

    def _cscene(self, grid: bool = True):
        prims = (_Prim * max(1, len(self.prims)))()
        for i, (kind, pid, c, h) in enumerate(self.prims):
            prims[i].kind = kind
            prims[i].id = pid
            for a in range(3):
                prims[i].c[a] = c[a]
                prims[i].h[a] = h[a]
        s = _Scene()
        for a in range(3):
            s.room_lo[a] = self.room_lo[a]
            s.room_hi[a] = self.room_hi[a]
        for a in range(6):
            s.face_id[a] = self.face_ids[a]
        s.tile = self.tile
        s.n_prims = len(self.prims)
        s.prims = prims
        s.width, s.height = self.width, self.height
        s.fx, s.fy, s.cx, s.cy = self.fx, self.fy, self.cx, self.cy
        s.depth_noise = self.depth_noise
        s.patch_h, s.patch_w, s.dim = self.patch_h, self.patch_w, self.dim
        s.token_noise = self.token_noise
        s.max_masks = self.max_masks
        s.max_id = self.max_id
        s.seed = self.seed
        keep = [prims]
        if grid and len(self.prims) > 200:
            # a 2 m grid over the floor plan: each ray tests the primitives
            # of the cells it crosses only
            cs = 2.0
            x0, y0 = self.room_lo[0], self.room_lo[1]
            nx = max(1, int(np.ceil((self.room_hi[0] - x0) / cs)))
            ny = max(1, int(np.ceil((self.room_hi[1] - y0) / cs)))
            cells = [[] for _ in range(nx * ny)]
            for i, (_k, _id, c, h) in enumerate(self.prims):
                i0 = max(0, int(np.floor((c[0] - h[0] - x0) / cs)))
                i1 = min(nx - 1, int(np.floor((c[0] + h[0] - x0) / cs)))
                j0 = max(0, int(np.floor((c[1] - h[1] - y0) / cs)))
                j1 = min(ny - 1, int(np.floor((c[1] + h[1] - y0) / cs)))
                for j in range(j0, j1 + 1):
                    for ii in range(i0, i1 + 1):
                        cells[j * nx + ii].append(i)
            start = np.zeros(nx * ny + 1, np.int32)
            start[1:] = np.cumsum([len(c) for c in cells])
            items = np.array([i for c in cells for i in c] or [0], np.int32)
            s.grid_nx, s.grid_ny = nx, ny
            s.grid_x0, s.grid_y0, s.grid_cell = x0, y0, cs
            s.cell_start = start.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            s.cell_items = items.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            keep += [start, items]
        return s, keep

    def render(self, frames, grid: bool = True) -> "Frames":
        """Render the given frame indices (any order, computed in parallel);
        grid=False tests every primitive for every ray (same frames)."""
        frames = np.asarray(list(frames), dtype=np.int64)
        n = len(frames)
        H, W, P, D, M = self.height, self.width, self.patch_h * self.patch_w, self.dim, self.max_masks
        depth = np.zeros((n, H, W), np.float32)
        labels = np.zeros((n, H, W), np.uint16)
        tokens = np.zeros((n, P, D), np.float32)
        mask_ids = np.zeros((n, M), np.int32)
        num_masks = np.zeros((n,), np.int32)
        ids = np.zeros((n, H, W), np.int32)
        poses = np.ascontiguousarray(self.poses[frames].reshape(n, 16), dtype=np.float64)
        s, keep = self._cscene(grid)
        rc = _load().synth_render(ctypes.byref(s), n, poses.ctypes.data, frames.ctypes.data,
                                  depth.ctypes.data, labels.ctypes.data, tokens.ctypes.data,
                                  mask_ids.ctypes.data, num_masks.ctypes.data, ids.ctypes.data)
        del keep
        if rc != 0:
            raise RuntimeError(f"synth_render failed: {rc}")
        return Frames(self, frames, poses.reshape(n, 4, 4), depth, labels, tokens, mask_ids,
                      num_masks, ids)

    def object_mean(self, obj_id: int) -> np.ndarray:
        out = np.zeros((self.dim,), np.float32)
        s, keep = self._cscene()
        _load().synth_object_mean(ctypes.byref(s), int(obj_id), out.ctypes.data)
        del keep
        return out


@dataclasses.dataclass
class Frames:
    scene: Scene
    index: np.ndarray
    poses: np.ndarray      # [n, 4, 4] float64
    depth: np.ndarray      # [n, H, W] float32
    labels: np.ndarray     # [n, H, W] uint16, 1..num_masks
    tokens: np.ndarray     # [n, P, D] float32
    mask_ids: np.ndarray   # [n, max_masks] object id of each mask
    num_masks: np.ndarray  # [n]
    ids: np.ndarray        # [n, H, W] object id per pixel

    def __len__(self):
        return int(self.index.shape[0])

    def assoc_tokens(self, patch_h: int, patch_w: int, dim: int) -> np.ndarray:
        """A second token grid [n, patch_h * patch_w, dim] (the association
        encoder's): per-object means and noise of their own, same recipe."""
        out = np.zeros((len(self), patch_h * patch_w, dim), np.float32)
        s, keep = self.scene._cscene(grid=False)
        ids = np.ascontiguousarray(self.ids, np.int32)
        idx = np.ascontiguousarray(self.index, np.int64)
        rc = _load().synth_assoc_tokens(ctypes.byref(s), len(self), idx.ctypes.data, ids.ctypes.data,
                                        patch_h, patch_w, dim, out.ctypes.data)
        del keep
        if rc != 0:
            raise RuntimeError(f"synth_assoc_tokens failed: {rc}")
        return out


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """camera->world pose with OpenCV axes (x right, y down, z forward)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, z, eye
    return T


def tiny_scene(seed: int = 0, num_frames: int = 20) -> Scene:
    """4x4x3 m room, four axis-aligned boxes with faces off the 5 cm grid,
    20 orbit poses (radius 1.5 m, height 1.2 m) looking at the room centre."""
    off = 0.013
    prims = [
        (0, 1, (1.2 + off, 1.1 + off, 0.30 + off), (0.25, 0.20, 0.30)),
        (0, 2, (2.8 + off, 1.2 + off, 0.20 + off), (0.30, 0.25, 0.20)),
        (0, 3, (2.7 + off, 2.8 + off, 0.35 + off), (0.20, 0.30, 0.35)),
        (0, 4, (1.3 + off, 2.7 + off, 0.25 + off), (0.30, 0.20, 0.25)),
    ]
    poses = []
    for i in range(num_frames):
        a = 2.0 * np.pi * i / num_frames
        eye = (2.0 + 1.5 * np.cos(a), 2.0 + 1.5 * np.sin(a), 1.2)
        poses.append(look_at(eye, (2.0 - 0.3 * np.cos(a), 2.0 - 0.3 * np.sin(a), 0.5)))
    # the room's faces are shifted off the voxel grid as well
    lo = (-0.0113, -0.0137, -0.0071)
    hi = (4.0 + lo[0], 4.0 + lo[1], 3.0 + lo[2])
    return Scene("tiny", lo, hi, (6, 7, 8, 9, 5, 10), prims,
                 np.stack(poses), 64, 48, 50.0, 50.0, 32.0, 24.0, 0.0, 6, 8, 512, 0.1, 8,
                 0.05, 0.1, 10.0, seed)


def _room_path(s: np.ndarray):
    cx, cy = 5.0, 4.0
    x = cx + 3.2 * np.cos(s) + 0.5 * np.cos(3 * s)
    y = cy + 2.4 * np.sin(s) + 0.4 * np.sin(2 * s)
    return x, y


def _polyline(points, n):
    """n samples at equal arc length along the polyline, with the direction
    of travel at each."""
    pts = np.asarray(points, np.float64)
    seg = np.linalg.norm(np.diff(pts, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    s = np.linspace(0.0, cum[-1], n, endpoint=False)
    out, dirs = [], []
    for v in s:
        k = min(int(np.searchsorted(cum, v, side="right")) - 1, len(seg) - 1)
        f = (v - cum[k]) / seg[k]
        out.append(pts[k] + f * (pts[k + 1] - pts[k]))
        dirs.append((pts[k + 1] - pts[k]) / seg[k])
    return np.array(out), np.array(dirs)


def multistory_scene(seed: int = 3, num_frames: int = 5000, n_objects: int = 1000, width: int = 640,
                     height: int = 480, patch: int = 24, dim: int = 768, max_masks: int = 100,
                     voxel: float = 0.05) -> Scene:
    """Three 40x30x3 m floors; partition walls at x = 10, 20, 30 leave a
    corridor at 13 <= y <= 17, so each floor has 8 rooms of 10x13 m; the floor
    slabs and walls are cut into panels with one id each; objects are kept
    0.6 m from the camera path and clear of the walls."""
    rng = np.random.default_rng(seed)
    off = 0.0113  # every face off the 5 cm voxel grid
    prims = []
    oid = 1

    def box(c, h, kind=0):
        nonlocal oid
        prims.append((kind, oid, tuple(float(x) + off for x in c), tuple(float(x) for x in h)))
        oid += 1

    # floor slabs between the storeys, 5 x 5 m panels
    for z in (3.0, 6.0):
        for x in range(0, 40, 5):
            for y in range(0, 30, 5):
                box((x + 2.5, y + 2.5, z), (2.5, 2.5, 0.05))
    # partition walls, 0.1 m thick, in panels of about 3 m
    walls = []
    for f in range(3):
        z0 = 3.0 * f
        for x in (10.0, 20.0, 30.0):
            for ya, yb in ((0.0, 13.0), (17.0, 30.0)):
                for k in range(4):
                    y0 = ya + (yb - ya) * k / 4.0
                    y1 = ya + (yb - ya) * (k + 1) / 4.0
                    c, h = (x, 0.5 * (y0 + y1), z0 + 1.475), (0.05, 0.5 * (y1 - y0), 1.425)
                    box(c, h)
                    walls.append((c, h))
    # the path: for every 10 m column of rooms, into the lower room, back to
    # the corridor, into the upper room, back; one floor after the other
    legs = []
    for f in range(3):
        pts = []
        for x0 in (0.0, 10.0, 20.0, 30.0):
            pts += [(x0 + 2.5, 15.0), (x0 + 2.5, 2.5), (x0 + 7.5, 2.5), (x0 + 7.5, 15.0),
                    (x0 + 7.5, 27.5), (x0 + 2.5, 27.5), (x0 + 2.5, 15.5), (x0 + 9.0, 15.5)]
        legs.append(pts)
    per = [num_frames // 3 + (1 if f < num_frames % 3 else 0) for f in range(3)]
    path_xy = np.concatenate([_polyline(p, 4 * len(p) * 20)[0] for p in legs])
    # objects resting on the floors, inside the rooms, away from path and walls
    tries = 0
    placed = 0
    while placed < n_objects and tries < 200000:
        tries += 1
        f = placed % 3
        size = rng.uniform(0.2, 1.2, 3)
        half = size / 2.0
        c = np.array([rng.uniform(0.3 + half[0], 39.7 - half[0]), rng.uniform(0.3 + half[1], 29.7 - half[1]),
                      3.0 * f + 0.05 + half[2]])
        if 12.6 - half[1] < c[1] < 17.4 + half[1]:
            continue  # corridor
        if any(abs(c[0] - wc[0]) < half[0] + wh[0] + 0.15 and abs(c[1] - wc[1]) < half[1] + wh[1] + 0.15
               for wc, wh in walls[:24]):  # one floor's walls; the plan repeats on every floor
            continue
        if np.min(np.hypot(path_xy[:, 0] - c[0], path_xy[:, 1] - c[1])) < float(np.hypot(half[0], half[1])) + 0.6:
            continue
        box(c, half, kind=int(rng.uniform() < 0.35))
        placed += 1
    poses = []
    for f in range(3):
        xy, dirs = _polyline(legs[f], per[f])
        for (x, y), (dx, dy) in zip(xy, dirs):
            eye = (x, y, 3.0 * f + 1.2)
            poses.append(look_at(eye, (x + 3.0 * dx, y + 3.0 * dy, 3.0 * f + 0.6)))
    faces = []
    tile = 1.0
    ext = (40.0, 30.0, 9.0)
    for fc in range(6):
        a = fc // 2
        b0, b1 = (1 if a == 0 else 0), (1 if a == 2 else 2)
        faces.append(oid)
        oid += int(np.ceil(ext[b0] / tile)) * int(np.ceil(ext[b1] / tile))
    f = 525.0 * width / 640.0
    lo = (-0.0071, -0.0093, -0.0051)
    hi = (40.0 + lo[0], 30.0 + lo[1], 9.0 + lo[2])
    return Scene("multistory", lo, hi, tuple(faces), prims, np.stack(poses), width, height, f, f, width / 2.0,
                 height / 2.0, 0.01, patch, patch, dim, 0.1, max_masks, voxel, 0.1, 20.0, seed, tile)


def room_scene(seed: int = 1, num_frames: int = 2000, n_objects: int = 80,
               width: int = 640, height: int = 480, patch: int = 24, dim: int = 768,
               max_masks: int = 40, voxel: float = 0.025) -> Scene:
    """10x8x3 m room with random boxes/ellipsoids (0.2-1.5 m) kept clear of a
    smooth closed camera path at 1.2 m height; 1 % depth noise."""
    rng = np.random.default_rng(seed)
    ss = np.linspace(0.0, 2.0 * np.pi, 720, endpoint=False)
    px, py = _room_path(ss)
    prims = []
    oid = 1
    tries = 0
    while len(prims) < n_objects and tries < 100000:
        tries += 1
        size = rng.uniform(0.2, 1.5, 3)
        size[2] = min(size[2], 2.6)
        half = size / 2.0
        c = np.array([rng.uniform(0.2 + half[0], 9.8 - half[0]),
                      rng.uniform(0.2 + half[1], 7.8 - half[1]),
                      half[2] + rng.uniform(0.0, 0.3) * (rng.uniform() < 0.3)])
        c[2] = min(c[2], 3.0 - half[2] - 0.05)
        r = float(np.hypot(half[0], half[1]))
        if np.min(np.hypot(px - c[0], py - c[1])) < r + 0.6:
            continue
        kind = int(rng.uniform() < 0.35)
        c = c + 0.0071  # keep faces off the voxel grid
        prims.append((kind, oid, tuple(c), tuple(half)))
        oid += 1
    # walls, floor and ceiling are cut into 1 m panels, each its own id (a
    # segmenter splits large surfaces the same way), so a frame sees ~40 masks
    tile = 1.0
    ext = (10.0, 8.0, 3.0)
    faces = []
    for f in range(6):
        a = f // 2
        b0, b1 = (1 if a == 0 else 0), (1 if a == 2 else 2)
        faces.append(oid)
        oid += int(np.ceil(ext[b0] / tile)) * int(np.ceil(ext[b1] / tile))
    faces = tuple(faces)
    s = np.linspace(0.0, 2.0 * np.pi, num_frames, endpoint=False)
    x, y = _room_path(s)
    poses = []
    for i in range(num_frames):
        tx = 5.0 + 2.2 * np.cos(2.0 * s[i] + 1.0)
        ty = 4.0 + 1.8 * np.sin(3.0 * s[i])
        poses.append(look_at((x[i], y[i], 1.2), (tx, ty, 0.6)))
    f = 525.0 * width / 640.0
    lo = (-0.0071, -0.0093, -0.0051)   # faces off the voxel grid
    hi = (10.0 + lo[0], 8.0 + lo[1], 3.0 + lo[2])
    return Scene("room", lo, hi, faces, prims, np.stack(poses),
                 width, height, f, f, width / 2.0, height / 2.0, 0.01, patch, patch, dim, 0.1,
                 max_masks, voxel, 0.1, 10.0, seed, tile)
