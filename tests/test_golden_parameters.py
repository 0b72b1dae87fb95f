"""The synthetic workloads use the shapes and definitions the paper prints
(tests/golden/paper_parameters.json, each value with its section)."""
import json
import math
import os

from paper_1508_07077_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_parameters.json")))


def test_reservoir_packing_fraction_definition():
    # phi_p^r = (pi/6) q^3 z_p  (colloid diameter 1)
    for eta, q in [(0.2, 0.2), (0.4, 0.15), (0.3, 0.1)]:
        zp = W.fugacity(eta, q)
        assert math.isclose(math.pi / 6.0 * q ** 3 * zp, eta, rel_tol=1e-14)


def test_discoid_is_the_printed_spheroid():
    a, b, c = GOLD["discoid"]["semi_axes"]
    assert a == b == W.SHAPE_PARAMS[W.SPHEROID][0]
    assert c == W.SHAPE_PARAMS[W.SPHEROID][1]
    L = W.box_length(1000, 0.3, W.SPHEROID)
    assert math.isclose(1000 * 4.0 / 3.0 * math.pi * a * b * c / L ** 3, 0.3)


def test_hemisphere_is_half_a_unit_sphere():
    d = GOLD["hemisphere"]["diameter"]
    L = W.box_length(512, 0.25, W.HEMISPHERE)
    assert math.isclose(512 * math.pi / 12.0 * d ** 3 / L ** 3, 0.25)
