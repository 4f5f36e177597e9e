"""The synthetic input generator (plumbing shared by both sides): the grid
traversal of many-primitive scenes gives exactly the frames of testing every
primitive."""
import numpy as np

import synth


def test_grid_traversal_equals_testing_every_primitive():
    sc = synth.multistory_scene(width=160, height=120)
    assert len(sc.prims) > 200
    idx = [0, 900, 1800, 2600, 3500, 4400]
    a = sc.render(idx)
    b = sc.render(idx, grid=False)
    assert np.array_equal(a.ids, b.ids)
    assert np.array_equal(a.depth.view(np.uint32), b.depth.view(np.uint32))
    assert np.array_equal(a.labels, b.labels) and np.array_equal(a.tokens, b.tokens)
    assert (a.num_masks > 10).all()
