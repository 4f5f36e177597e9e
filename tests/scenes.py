"""Hand-built frames for the oracle pins and the parity tests.

Analytic planar depth maps and label images whose voxel keys, coverage and
view-angle terms have closed forms.  Input construction only: no step of the
integration method is computed here.
"""
import numpy as np


def plane_depth(H, W, fx, fy, cx, cy, z0, theta=0.0):
    """Camera-frame depth of the plane through (0, 0, z0) whose normal is
    rotated by theta about the camera y axis (theta = 0: fronto-parallel)."""
    u = (np.arange(W, dtype=np.float64) + 0.5 - cx) / fx
    v = (np.arange(H, dtype=np.float64) + 0.5 - cy) / fy
    xh = np.broadcast_to(u[None, :], (H, W))
    # plane n . X = z0 cos(theta) with n = (sin theta, 0, cos theta); X = t (xh, yh, 1)
    t = z0 * np.cos(theta) / (np.sin(theta) * xh + np.cos(theta))
    return t.astype(np.float32)


def identity_pose():
    return np.eye(4)


def pose_from(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def rot_z(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def tokens_from_ids(id_img, Ph, Pw, means, noise=0.0, rng=None):
    """Token of patch (i, j) = means[id at the patch-centre pixel] (+ noise)."""
    H, W = id_img.shape
    D = means.shape[1]
    F = np.zeros((Ph * Pw, D), np.float32)
    for i in range(Ph):
        for j in range(Pw):
            vc = ((2 * i + 1) * H) // (2 * Ph)
            uc = ((2 * j + 1) * W) // (2 * Pw)
            F[i * Pw + j] = means[id_img[vc, uc]]
    if noise and rng is not None:
        F = F + noise * rng.standard_normal(F.shape).astype(np.float32)
    return F.astype(np.float32)


def custom_scene(prims, poses, width=64, height=48, f=50.0, dim=64, patch=(6, 8), voxel=0.05,
                 max_masks=8, room=30.0, seed=7, token_noise=0.1, depth_noise=0.0):
    """A synth.Scene with the given primitives inside a room so large that its
    walls lie beyond the valid depth range (their masks carry no voxels)."""
    import synth
    return synth.Scene("custom", (-room, -room, -room), (room, room, room), (901, 902, 903, 904, 905, 906),
                       list(prims), np.stack(poses), width, height, f, f, width / 2.0, height / 2.0,
                       depth_noise, patch[0], patch[1], dim, token_noise, max_masks, voxel, 0.1, 10.0,
                       seed)


def orbit(center, radius, height, n, start=0.0, sweep=2 * np.pi, look_height=None):
    import synth
    out = []
    for i in range(n):
        a = start + sweep * i / max(n - 1, 1) if sweep < 2 * np.pi else start + sweep * i / n
        eye = (center[0] + radius * np.cos(a), center[1] + radius * np.sin(a), height)
        out.append(synth.look_at(eye, (center[0], center[1], center[2] if look_height is None else look_height)))
    return out
