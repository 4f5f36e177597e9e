"""The oracle's stateful steps (a7-a10 of the integration step, Sec. III-B and
III-C) replayed independently in float64 Python.

Each frame's segment voxel sets, pooled embeddings and quality scores come
from the oracle's own report (a1-a6, pinned in test_oracle_pins.py); from
them and the map as the replay holds it, the replay recomputes:
  - the overlap histogram against the map before the frame (Sec. III-B);
  - the association edges: the overlap coefficient ov / min(|V_m|, |V_k|)
    >= num / den as an exact integer test, and the cosine of the pooled
    embedding with the stored one >= tau, here in float64;
  - the components of segments and instances (union-find), each keeping its
    smallest instance id; a segment without an edge opens a new id, in mask
    order; merged ids point at the representative;
  - new voxels labelled with the instance of their lowest-index segment, and
    the voxel counts;
  - the fusion of Sec. III-C: over the existing members by ascending id,
    then the segments by ascending mask, the first highest Q wins (strict >);
  - observations: a component's members' sum plus its segments;
  - optionally the 26-neighbour overlap (an instance counts once per segment
    voxel that it or one of the voxel's 26 neighbours carries) and a second
    token grid (the gate compares association features, which travel with
    the embedding through fusion).
Every frame's representatives and counters, and the final map (voxels, their
instances, parents, counts, Q, embeddings, observations), must equal the
oracle's.  The float64 cosine takes every gate decision the oracle's exact
fp32-rounded cosine takes on these scenes; a frame where the two disagree
fails the test.
"""
import numpy as np
import pytest

import oracle
import synth


class Replay:
    def __init__(self, cfg):
        self.num, self.den = int(cfg["ov_num"]), int(cfg["ov_den"])
        self.tau = float(cfg["tau_cos"])
        # options: the 26-neighbour overlap (reading N1) and a second token
        # grid whose features drive the gate and travel with the embedding
        # through fusion (reading T1)
        self.dilate = bool(cfg.get("overlap_dilation", 0))
        self.assoc = int(cfg.get("assoc_dim", 0)) > 0
        self.vox = {}          # voxel key -> instance id written when it was inserted
        self.at = {}           # voxel coordinates -> voxel key (dilation)
        self.parent, self.count, self.Q, self.E, self.obs, self.A = [], [], [], [], [], []
        self.cos_rejects = 0   # pairs past the overlap gate that the cosine gate stopped

    def root(self, i):
        while self.parent[i] != i:
            i = self.parent[i]
        return i

    @staticmethod
    def cos64(a, b):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        na, nb = np.linalg.norm(a), np.linalg.norm(b)
        return float(a @ b / (na * nb)) if na > 0 and nb > 0 else 0.0

    def frame(self, r, M):
        seg = {}
        for m, k in zip(r["seg_m"].tolist(), r["seg_keys"].tolist()):
            seg.setdefault(m, []).append(k)
        live = sorted(m for m in seg if seg[m])
        nv = {m: len(seg[m]) for m in live}
        # overlap histogram against the map before the frame
        ov = {}
        for m in live:
            for k in seg[m]:
                if self.dilate:
                    c = oracle.unpack_key(k)
                    near = set()
                    for dx in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dz in (-1, 0, 1):
                                kk = self.at.get((c[0] + dx, c[1] + dy, c[2] + dz))
                                if kk is not None:
                                    near.add(self.root(self.vox[kk]))
                else:
                    near = {self.root(self.vox[k])} if k in self.vox else set()
                for i in near:
                    ov[(m, i)] = ov.get((m, i), 0) + 1
        feat = "A" if self.assoc else "E"
        mine = self.A if self.assoc else self.E
        edges = []
        for (m, i), n in sorted(ov.items()):
            if n * self.den >= self.num * min(nv[m], self.count[i]):
                if self.cos64(r[feat][m - 1], mine[i]) >= self.tau:
                    edges.append((m, i))
                else:
                    self.cos_rejects += 1
        # components over segments ('s', m) and instances ('i', id)
        uf = {}

        def find(x):
            while uf.setdefault(x, x) != x:
                x = uf[x]
            return x

        for m, i in edges:
            a, b = find(("s", m)), find(("i", i))
            if a != b:
                uf[a] = b
        comp = {}
        for m, i in edges:
            comp.setdefault(find(("i", i)), [set(), set()])
        for x in list(uf):
            c = find(x)
            if c in comp:
                comp[c][0 if x[0] == "i" else 1].add(x[1])
        rep = {}
        merges = 0
        for insts, segs in comp.values():
            members = sorted(insts)
            g = members[0]
            merges += len(members) - 1
            for i in members:
                for x in range(len(self.parent)):
                    if self.parent[x] == i:
                        self.parent[x] = g
            cands = [(self.Q[i], self.E[i], self.A[i]) for i in members]
            cands += [(float(r["S"][m - 1][4]), r["E"][m - 1].copy(), r["A"][m - 1].copy() if self.assoc else None)
                      for m in sorted(segs)]
            best = 0
            for j in range(1, len(cands)):
                if cands[j][0] > cands[best][0]:
                    best = j
            total = sum(self.count[i] for i in members)
            obs = sum(self.obs[i] for i in members) + len(segs)
            for i in members[1:]:
                self.count[i] = 0
            self.count[g] = total
            self.Q[g], self.E[g], self.A[g] = cands[best]
            self.obs[g] = obs
            for m in segs:
                rep[m] = g
        new_ids = 0
        for m in live:
            if m not in rep:
                g = len(self.parent)
                self.parent.append(g)
                self.count.append(0)
                self.Q.append(float(r["S"][m - 1][4]))
                self.E.append(r["E"][m - 1].copy())
                self.A.append(r["A"][m - 1].copy() if self.assoc else None)
                self.obs.append(1)
                rep[m] = g
                new_ids += 1
        # new voxels: the instance of their lowest-index segment
        owner = {}
        for m in live:
            for k in seg[m]:
                if k not in self.vox and (k not in owner or m < owner[k]):
                    owner[k] = m
        for k, m in owner.items():
            self.vox[k] = rep[m]
            self.count[rep[m]] += 1
            if self.dilate:
                self.at[oracle.unpack_key(k)] = k
        reps = np.array([rep.get(m, -1) for m in range(1, M + 1)], np.int32)
        return dict(rep=reps, nv=nv, live=len(live), new_instances=new_ids, merges=merges,
                    overlap_pairs=len(ov), active=len({i for (_, i) in ov}), new_voxels=len(owner))


def _split_masks(labels, num_masks, max_masks, frame):
    """Over-segmentation: on odd frames the two largest masks are cut into a
    left and a right part (the right part takes a fresh label), so fragments
    open separate instances and later views merge them."""
    out = labels.copy()
    if frame % 2 == 0:
        return out, num_masks
    ids, cnt = np.unique(labels[labels > 0], return_counts=True)
    n = num_masks
    for m in ids[np.argsort(-cnt)][:2]:
        if n >= max_masks:
            break
        vs, us = np.nonzero(labels == m)
        cut = int(np.median(us))
        n += 1
        out[(labels == m) & (np.arange(labels.shape[1])[None, :] > cut)] = n
    return out, n


def _replay(sc, idx, split=False, **kw):
    fr = sc.render(idx)
    cfg = oracle.config_for_scene(sc, **kw)
    om = oracle.OracleMap(**cfg)
    rp = Replay(cfg)
    at = fr.assoc_tokens(cfg["assoc_patch_h"], cfg["assoc_patch_w"], cfg["assoc_dim"]) if rp.assoc else None
    for i in range(len(fr)):
        depth, labels, tokens, pose, intr, M = oracle.frame_args(fr, i)
        if split:
            labels, M = _split_masks(labels, M, sc.max_masks, i)
        r = om.integrate(depth, labels, tokens, pose, intr, M, assoc_tokens=at[i] if rp.assoc else None)
        x = rp.frame(r, M)
        ctx = f"{sc.name} frame {idx[i]}"
        assert np.array_equal(r["rep"], x["rep"]), (ctx, r["rep"], x["rep"])
        for m, n in x["nv"].items():
            assert r["nvox"][m - 1] == n, ctx
        assert r["live_segments"] == x["live"], ctx
        assert r["overlap_pairs"] == x["overlap_pairs"], ctx
        assert r["active_instances"] == x["active"], ctx
        assert r["new_instances"] == x["new_instances"], ctx
        assert r["merges"] == x["merges"], ctx
        assert r["new_voxels"] == x["new_voxels"], ctx
    keys, ids = om.voxels()
    assert sorted(rp.vox) == keys.tolist()
    assert [rp.root(rp.vox[k]) for k in keys.tolist()] == ids.tolist()
    inst = om.instances()
    n = len(rp.parent)
    assert len(inst["parent"]) == n
    assert [rp.root(i) for i in range(n)] == inst["parent"].tolist()
    roots = [i for i in range(n) if rp.parent[i] == i]
    assert [rp.count[i] for i in roots] == inst["count"][roots].tolist()
    assert [rp.obs[i] for i in roots] == inst["n_obs"][roots].tolist()
    for i in roots:
        assert np.float32(rp.Q[i]) == inst["Q"][i]
        assert np.array_equal(np.asarray(rp.E[i], np.float32).view(np.uint32), inst["E"][i].view(np.uint32))
        if rp.assoc:
            assert np.array_equal(np.asarray(rp.A[i], np.float32).view(np.uint32), inst["A"][i].view(np.uint32))
    _replay.last = rp
    return len(roots), sum(1 for i in range(n) if rp.parent[i] != i)


def test_replay_tiny_trajectory():
    live, merged = _replay(synth.tiny_scene(), list(range(20)))
    assert live >= 4


def test_replay_tiny_trajectory_with_split_masks():
    # fragments of one object open separate instances and merge later
    live, merged = _replay(synth.tiny_scene(), list(range(20)), split=True)
    assert merged > 0


@pytest.mark.parametrize("stride", [7])
def test_replay_room_frames(stride):
    sc = synth.room_scene()
    live, merged = _replay(sc, list(range(0, 14 * stride, stride)))
    assert live >= 10


def test_replay_with_neighbourhood_overlap():
    # reading N1: an instance counts once per segment voxel when it labels
    # the voxel or one of its 26 neighbours
    live, merged = _replay(synth.tiny_scene(), list(range(20)), split=True, overlap_dilation=1)
    assert merged > 0
    _replay(synth.room_scene(), list(range(0, 70, 7)), overlap_dilation=1)


def test_replay_with_a_second_token_grid():
    # reading T1: the gate compares the association features, and fusion
    # carries them with the embedding
    _replay(synth.tiny_scene(), list(range(20)), split=True, assoc_dim=48, assoc_patch_h=4, assoc_patch_w=6)


def _random_scene(seed):
    # boxes and ellipsoids in pairs that touch, seen along a noisy orbit with
    # noisy tokens: the cosine gate both passes and stops pairs the overlap
    # gate lets through
    from tests import scenes
    rng = np.random.default_rng(seed)
    prims, pid = [], 1
    for _ in range(3):
        c = rng.uniform([0.2, 0.2, 0.15], [1.8, 1.8, 0.4])
        h = rng.uniform(0.1, 0.25, 3)
        h2 = rng.uniform(0.1, 0.25, 3)
        c2 = c + np.array([h[0] + h2[0] + 0.013, 0.0, 0.0])
        prims.append((int(rng.integers(0, 2)), pid, tuple(c + 0.013), tuple(h)))
        prims.append((0, pid + 1, tuple(c2 + 0.013), tuple(h2)))
        pid += 2
    poses = scenes.orbit((1.0, 1.0, 0.3), 2.2, 1.1, 14, start=float(rng.uniform(0, 6.28)))
    return scenes.custom_scene(prims, poses, width=80, height=60, f=60.0, dim=64, patch=(6, 8), voxel=0.05,
                               max_masks=8, seed=seed, token_noise=0.45, depth_noise=0.01)


@pytest.mark.parametrize("seed", [21, 22, 23, 24])
def test_replay_random_scenes_with_noisy_tokens(seed):
    _replay(_random_scene(seed), list(range(14)), split=(seed % 2 == 1))


def test_random_scenes_exercise_the_cosine_gate():
    total = 0
    for seed in (21, 22, 23, 24):
        _replay(_random_scene(seed), list(range(14)), split=(seed % 2 == 1))
        total += _replay.last.cos_rejects
    assert total > 0
