"""The oracle's end-of-trajectory step (Sec. III-B, last paragraph; reading
F1) replayed independently in float64 Python on the states real
trajectories leave, not only on hand-built ones.

From the exported voxels and instance table the replay computes:
  - contact(a, b): voxels of a or b with a face neighbour (one of the 6
    voxels sharing a face) in the other;
  - a merge of a and b when contact * den >= num * min(|a|, |b|) and the
    cosine of their embeddings >= tau (float64 here), on the state at the
    start; merges are transitive and the smallest id represents a component,
    which takes the Q and embedding of its member with the highest Q (ties:
    the smallest id) and the sums of the voxel and observation counts;
  - then every live instance with 0 < count < min_voxels is dropped: its
    voxels report -1, and its count, observations and Q become 0.
The report (pairs in contact, merged, removed, removed voxels) and the final
map must equal the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_replay import _split_masks


def _state(sc, idx, split):
    fr = sc.render(idx)
    cfg = oracle.config_for_scene(sc)
    om = oracle.OracleMap(**cfg)
    for i in range(len(fr)):
        depth, labels, tokens, pose, intr, M = oracle.frame_args(fr, i)
        if split:
            labels, M = _split_masks(labels, M, sc.max_masks, i)
        om.integrate(depth, labels, tokens, pose, intr, M)
    return om, cfg


def replay_finalize(keys, ids, inst, min_voxels, num, den, tau):
    coord = [tuple(oracle.unpack_key(k)) for k in keys.tolist()]
    owner = dict(zip(coord, ids.tolist()))
    parent = inst["parent"].tolist()
    count = inst["count"].astype(np.int64).tolist()
    Q = inst["Q"].tolist()
    E = inst["E"]
    obs = inst["n_obs"].tolist()
    n = len(parent)
    # contact: each voxel counts once for every other instance it touches
    touch = {}
    for c, a in owner.items():
        if a < 0:
            continue
        seen = set()
        for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            b = owner.get((c[0] + d[0], c[1] + d[1], c[2] + d[2]), -1)
            if b >= 0 and b != a and b not in seen:
                seen.add(b)
                key = (min(a, b), max(a, b))
                touch[key] = touch.get(key, 0) + 1
    uf = list(range(n))

    def find(x):
        while uf[x] != x:
            x = uf[x]
        return x

    for (a, b), ct in sorted(touch.items()):
        Ea, Eb = E[a].astype(np.float64), E[b].astype(np.float64)
        cos = float(Ea @ Eb / (np.linalg.norm(Ea) * np.linalg.norm(Eb)))
        if ct * den >= num * min(count[a], count[b]) and cos >= tau:
            ra, rb = find(a), find(b)
            if ra != rb:
                uf[max(ra, rb)] = min(ra, rb)
    comps = {}
    for i in range(n):
        if parent[i] == i and count[i] > 0:
            comps.setdefault(find(i), []).append(i)
    newQ, newE, newc, newo, newp = list(Q), E.copy(), list(count), list(obs), list(parent)
    merged = 0
    for g, mem in comps.items():
        mem.sort()
        best = mem[0]
        for i in mem[1:]:
            if Q[i] > Q[best]:
                best = i
        newQ[g], newE[g] = Q[best], E[best]
        newc[g] = sum(count[i] for i in mem)
        newo[g] = sum(obs[i] for i in mem)
        for i in mem:
            if i != g:
                newc[i] = 0  # a merged id holds no voxels; its other fields are not read
                merged += 1
        for x in range(n):
            if newp[x] in mem:
                newp[x] = g
    removed, removed_vox = 0, 0
    drop = set()
    for i in range(n):
        if newp[i] == i and 0 < newc[i] < min_voxels:
            drop.add(i)
            removed += 1
            removed_vox += newc[i]
            newc[i] = 0
            newo[i] = 0
            newQ[i] = 0.0
    final_ids = []
    for k in ids.tolist():
        r = newp[k] if k >= 0 else -1
        final_ids.append(-1 if r in drop else r)
    rep = dict(contact_pairs=len(touch), merged=merged, removed=removed, removed_voxels=removed_vox)
    return rep, np.array(final_ids, np.int32), dict(parent=newp, count=newc, Q=newQ, E=newE, n_obs=newo)


@pytest.mark.parametrize("scene,idx,split,min_voxels", [
    ("tiny", list(range(20)), True, 40),
    ("tiny", list(range(0, 20, 3)), False, 200),
    ("room", list(range(0, 84, 7)), False, 400),
])
def test_finalize_replay(scene, idx, split, min_voxels):
    sc = synth.tiny_scene() if scene == "tiny" else synth.room_scene()
    om, cfg = _state(sc, idx, split)
    keys, ids = om.voxels()
    inst = om.instances()
    num, den, tau = 1, 5, float(cfg["tau_cos"])
    rep_x, ids_x, inst_x = replay_finalize(keys, ids, inst, min_voxels, num, den, tau)
    rep = om.finalize(min_voxels, num, den, tau)
    assert rep == rep_x
    keys2, ids2 = om.voxels()
    assert np.array_equal(keys2, keys)
    assert np.array_equal(ids2, ids_x)
    got = om.instances()
    assert got["parent"].tolist() == inst_x["parent"]
    assert got["count"].tolist() == inst_x["count"]
    # a root's fields carry the instance (a merged id's are not read)
    roots = [i for i, p in enumerate(inst_x["parent"]) if p == i]
    assert got["n_obs"][roots].tolist() == [inst_x["n_obs"][i] for i in roots]
    assert np.array_equal(got["Q"][roots], np.asarray([inst_x["Q"][i] for i in roots], np.float32))
    assert np.array_equal(got["E"][roots].view(np.uint32),
                          np.asarray(inst_x["E"][roots], np.float32).view(np.uint32))
    # the states exercise the rules: contacts and removals in every case,
    # merges in the Tiny subsample and the Room frames
    assert rep["contact_pairs"] > 0 and rep["removed"] > 0
    if not split:
        assert rep["merged"] > 0
