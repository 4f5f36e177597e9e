"""The allocation-free token-statistics entry point (disc_token_stats_static).

It serves callers that cannot call cudaMalloc; its scratch lives in a static
device array.  Through the C ABI, two calls in a row must each reproduce,
bit for bit, the distinctiveness map and token cosines that the map-based
entry point (disc_integrate_frame) reports for the same tokens.  This file is
collected last so a failure here does not hide the other tests.
"""
import numpy as np
import pytest

import synth
from tests import common

pytestmark = pytest.mark.gpu


def test_static_token_stats_match_the_map_path_twice():
    import torch
    from paper_2603_03935_gb300 import DiscMap, _build, device_frame, token_stats_static
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    sc = synth.tiny_scene()
    fr = sc.render([0, 5])
    gmap = DiscMap(**common.disc_cfg(sc))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    for i in range(2):
        d = torch.from_numpy(fr.depth[i]).to(dev)
        l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
        t = torch.from_numpy(fr.tokens[i]).to(dev)
        gmap.integrate(device_frame(d, l, t, fr.poses[i], intr, fr.num_masks[i]))
        ref = gmap.last_frame()
        Dp, cosg = token_stats_static(t, eps=float(gmap.cfg["eps"]))
        torch.cuda.synchronize()
        assert np.array_equal(Dp.cpu().numpy().view(np.uint32), ref["Dp"].view(np.uint32)), f"call {i}: Dp"
        assert np.array_equal(cosg.cpu().numpy().view(np.uint32), ref["cosg"].view(np.uint32)), f"call {i}: cosg"
    gmap.close()


def test_static_token_stats_reject_sizes_beyond_the_limit():
    import torch
    from paper_2603_03935_gb300 import DiscError, _build, token_stats_static
    _build.build()
    t = torch.zeros((16385, 8), dtype=torch.float32, device="cuda:0")
    with pytest.raises(DiscError):
        token_stats_static(t)
