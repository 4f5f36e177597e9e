"""The constants the paper prints for the per-frame step
(tests/golden/paper_constants.txt, each with its passage) against the oracle:
its default lambda, the plateau and slope of S_size, the affine form of
S_dist, and Q as the product of the four terms on rendered frames."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _constants():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_constants.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


C = _constants()


def test_default_lambda_is_the_papers():
    assert oracle.default_config(8, 2, 2, 0.05)["lambda_size"] == pytest.approx(C["lambda_size"])


def test_s_size_plateau_and_slope():
    # a mask of a fraction a of the frame: S_size = min(lambda a, 1)
    H, W, Ph, Pw, D = 60, 80, 4, 4, 8
    rng = np.random.default_rng(5)
    F = rng.standard_normal((Ph * Pw, D)).astype(np.float32)
    depth = np.full((H, W), 2.0, np.float32)
    for a in (0.05, 0.1, 0.2, 1 / C["lambda_size"], 0.5):
        n = int(round(a * H * W))
        lab = np.zeros(H * W, np.uint16)
        lab[:n] = 1
        m = oracle.OracleMap(**oracle.default_config(D, Ph, Pw, 0.05, min_mask_pixels=1))
        r = m.integrate(depth, lab.reshape(H, W), F, np.eye(4), (100.0, 100.0, W / 2, H / 2), 1)
        assert r["S"][0, 0] == pytest.approx(min(C["lambda_size"] * n / (H * W), 1.0), rel=1e-6)


def test_s_dist_and_q_on_rendered_frames():
    sc = synth.tiny_scene()
    fr = sc.render(range(0, 20, 5))
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    for i in range(len(fr)):
        r = m.integrate(*oracle.frame_args(fr, i))
        for k in range(int(fr.num_masks[i])):
            if r["nvox"][k] == 0:
                continue
            S = r["S"][k].astype(np.float64)
            # S_dist from the mask's coverage-weighted mean distinctiveness
            c = r["cov"][k].astype(np.float64)
            dbar = float(c @ r["Dp"].astype(np.float64)) / c.sum()
            assert S[3] == pytest.approx(C["s_dist_offset"] + C["s_dist_slope"] * dbar, abs=1e-6)
            # Q is the product of the four terms
            assert int(C["q_factors"]) == 4
            assert S[4] == pytest.approx(S[0] * S[1] * S[2] * S[3], rel=1e-6)
