"""The seeded synthetic workloads keep the recipes the measurements are
quoted on: panel counts by kind, conductor counts and determinism (panels by
the oracle's brute-force enumeration, Sec. II.A-B)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

# name -> (generator, grid [z, y, x], panels, conductor panels, dielectric panels, conductors)
RECIPES = {
    "cube4": (lambda: W.cube(4), (4, 4, 4), 96, 96, 0, 1),
    "plates": (W.plates, (16, 32, 32), 3072, 2688, 384, 2),
    "bus_crossing": (W.bus_crossing, (64, 128, 128), 110848, 12544, 98304, 8),
    "pillars": (lambda: W.pillars_field()[0], (64, 64, 64), 781952, 3328, 778624, 2),
    "meanders": (W.meanders, (64, 512, 512), 1410624, 755264, 655360, 2),
    "meanders256": (lambda: W.meanders(256, 256, 64, 16), (64, 256, 256), 377408, 180800, 196608, 2),
}


@pytest.mark.parametrize("name", list(RECIPES))
def test_workload_recipe(name):
    gen, shape, n, nc, nd, m = RECIPES[name]
    w = gen()
    assert w.labels.shape == shape
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    assert (ps.n, ps.n_cond, ps.n_diel, ps.n_conductors) == (n, nc, nd, m)
    again = gen()
    assert np.array_equal(w.labels, again.labels) and np.array_equal(w.eps_r, again.eps_r)


def test_small_boxes_are_sixteen_seeded_one_conductor_grids():
    boxes = W.small_boxes()
    assert len(boxes) == 16
    for w, v in zip(boxes, W.small_boxes()):
        assert w.labels.shape == (16, 16, 16) and np.array_equal(w.labels, v.labels)
        ps = O.panels(w.labels, w.conductor_id, w.eps_r)
        assert ps.n_conductors == 1 and ps.n_cond > 0
    assert len({w.labels.tobytes() for w in boxes}) == 16          # distinct seeds, distinct grids
