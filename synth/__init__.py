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
                ("max_id", ctypes.c_int32), ("seed", ctypes.c_uint64)]


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

    def _cscene(self):
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
        return s, prims

    def render(self, frames) -> "Frames":
        """Render the given frame indices (any order, computed in parallel)."""
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
        s, keep = self._cscene()
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
