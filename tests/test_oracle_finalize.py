"""Pins of the oracle's end-of-trajectory step (Sec. III-B, last paragraph):
orphan merge by face contact and embedding similarity, then the voxel-count
filter.  Each case builds an exact map state and checks the outcome the
stated reading fixes by hand.
"""
import numpy as np
import pytest

import oracle
import synth

D = 8
S = 0.05


def _cfg():
    return dict(voxel_size=S, z_min=0.1, z_max=10.0, eps=1e-6, tau_cos=0.75, lambda_size=3.3, ov_num=1,
                ov_den=5, embed_dim=D, patch_h=2, patch_w=2, min_mask_pixels=1)


def _key(kx, ky, kz):
    k = oracle.point_key((kx + 0.5) * S, (ky + 0.5) * S, (kz + 0.5) * S, S)
    assert k is not None
    return k


def _vec(seed, base=None, noise=0.0):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(D).astype(np.float32)
    if base is not None:
        v = base + noise * v
    return v.astype(np.float32)


def _build(instances, parent=None, Q=None, n_obs=None):
    """instances: list of (voxel list, embedding); every voxel labelled with
    its instance id."""
    keys, labels = [], []
    for i, (vox, _) in enumerate(instances):
        for v in vox:
            keys.append(_key(*v))
            labels.append(i)
    n = len(instances)
    parent = np.arange(n, dtype=np.int32) if parent is None else np.asarray(parent, np.int32)
    count = np.zeros(n, np.int64)
    for i, (vox, _) in enumerate(instances):
        count[parent[i]] += len(vox)
    for i in range(n):
        if parent[i] != i:
            count[i] = 0
    Q = np.linspace(0.5, 0.9, n).astype(np.float32) if Q is None else np.asarray(Q, np.float32)
    n_obs = np.ones(n, np.int32) if n_obs is None else np.asarray(n_obs, np.int32)
    E = np.stack([e for _, e in instances]).astype(np.float32)
    m = oracle.OracleMap(**_cfg())
    m.set_state(np.array(keys, np.uint64), np.array(labels, np.int32), parent, count, Q, E, n_obs)
    return m


def _plate(x0, x1, y0, y1, z=0):
    return [(x, y, z) for x in range(x0, x1) for y in range(y0, y1)]


def _ids(m):
    k, i = m.voxels()
    return dict(zip(k.tolist(), i.tolist()))


def test_touching_similar_fragment_merges_into_smallest_id():
    base = _vec(1)
    m = _build([(_plate(0, 6, 0, 6), base), (_plate(6, 8, 0, 1), _vec(2, base, 0.05))])
    r = m.finalize(min_voxels=1)
    # contact: voxel (5,0) of instance 0 and voxel (6,0) of instance 1
    assert r == {"contact_pairs": 1, "merged": 1, "removed": 0, "removed_voxels": 0}
    inst = m.instances()
    assert inst["parent"].tolist() == [0, 0] and inst["count"].tolist() == [38, 0]
    assert set(_ids(m).values()) == {0}
    # Q[1] > Q[0]: the component keeps instance 1's embedding and Q
    assert inst["Q"][0] == np.float32(0.9)
    assert np.array_equal(inst["E"][0], _vec(2, base, 0.05))
    assert inst["n_obs"][0] == 2


def test_dissimilar_or_separated_fragments_stay():
    base = _vec(1)
    far = -base  # cosine -1
    m = _build([(_plate(0, 6, 0, 6), base), (_plate(6, 8, 0, 1), far)])
    r = m.finalize(min_voxels=1)
    assert r["contact_pairs"] == 1 and r["merged"] == 0
    m = _build([(_plate(0, 6, 0, 6), base), (_plate(7, 9, 0, 1), base)])  # one empty voxel between
    r = m.finalize(min_voxels=1)
    assert r["contact_pairs"] == 0 and r["merged"] == 0
    # edge or corner neighbours are not face neighbours
    m = _build([(_plate(0, 6, 0, 6), base), ([(6, 6, 0), (7, 7, 0)], base)])
    assert m.finalize(min_voxels=1)["contact_pairs"] == 0


def test_contact_ratio_is_an_exact_rational_test():
    base = _vec(1)
    # a 1 x 10 line along x = 6 touching the 6 x 6 plate on y = 0..5:
    # 6 plate voxels + 6 line voxels in contact, min(|a|, |b|) = 10
    line = [(6, y, 0) for y in range(10)]
    for num, den, merged in ((6, 5, 1), (7, 5, 0), (12, 10, 1), (13, 10, 0)):
        m = _build([(_plate(0, 6, 0, 6), base), (line, base)])
        r = m.finalize(min_voxels=1, contact_num=num, contact_den=den)
        assert r["merged"] == merged, (num, den)


def test_merges_are_transitive_and_counts_add_up():
    base = _vec(3)
    a, b, c = _plate(0, 4, 0, 4), _plate(4, 5, 0, 4), _plate(5, 9, 0, 4)
    m = _build([(a, base), (b, _vec(4, base, 0.05)), (c, _vec(5, base, 0.05))], Q=[0.3, 0.3, 0.3])
    r = m.finalize(min_voxels=1)
    assert r["contact_pairs"] == 2 and r["merged"] == 2
    inst = m.instances()
    assert inst["parent"].tolist() == [0, 0, 0] and inst["count"].tolist() == [36, 0, 0]
    # equal Q: the smallest id's embedding stays
    assert np.array_equal(inst["E"][0], base)
    assert inst["n_obs"][0] == 3


def test_small_instances_are_dropped_after_merging():
    base = _vec(6)
    lone = _vec(7)  # dissimilar, isolated, 2 voxels
    frag = _vec(8, base, 0.05)  # 2 voxels touching the plate: merged, so it survives
    m = _build([(_plate(0, 6, 0, 6), base), ([(20, 0, 0), (21, 0, 0)], lone), (_plate(6, 7, 0, 2), frag)])
    r = m.finalize(min_voxels=3)
    assert r == {"contact_pairs": 1, "merged": 1, "removed": 1, "removed_voxels": 2}
    inst = m.instances()
    assert inst["count"].tolist() == [38, 0, 0] and inst["Q"][1] == 0.0 and inst["n_obs"][1] == 0
    ids = _ids(m)
    assert ids[_key(20, 0, 0)] == -1 and ids[_key(21, 0, 0)] == -1
    assert sum(1 for v in ids.values() if v == 0) == 38


def test_voxels_of_merged_ids_resolve_through_two_levels():
    base = _vec(9)
    # id 2 was merged into 1 earlier (parent[2] = 1); its voxels keep label 2
    m = _build([(_plate(0, 4, 0, 4), base), (_plate(4, 5, 0, 4), base), (_plate(5, 6, 0, 4), base)],
               parent=[0, 1, 1])
    r = m.finalize(min_voxels=1)
    assert r["merged"] == 1
    assert set(_ids(m).values()) == {0}
    assert m.instances()["parent"].tolist() == [0, 0, 0]


def test_integration_after_finalisation_is_refused():
    sc = synth.tiny_scene()
    fr = sc.render(range(2))
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    m.integrate(*oracle.frame_args(fr, 0))
    m.finalize(min_voxels=5)
    with pytest.raises(Exception):
        m.integrate(*oracle.frame_args(fr, 1))


def test_trajectory_invariants_after_finalisation():
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    for i in range(20):
        m.integrate(*oracle.frame_args(fr, i), report=False)
    n_before = len(m.voxels()[0])
    r = m.finalize(min_voxels=40, contact_num=1, contact_den=10, tau_cos=0.5)
    keys, ids = m.voxels()
    inst = m.instances()
    live = (inst["parent"] == np.arange(len(inst["parent"]))) & (inst["count"] > 0)
    assert len(keys) == n_before
    assert int((ids == -1).sum()) == r["removed_voxels"]
    assert all(live[i] for i in ids[ids >= 0])
    assert int(inst["count"][live].sum()) == int((ids >= 0).sum())
    assert not np.any((inst["count"] > 0) & (inst["count"] < 40))
