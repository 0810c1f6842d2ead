"""Host-side logic that needs no GPU: the seeded input generators (geometry nets are data only and
must describe the same maps the oracle builds from their definitions), the warm-start features
and parameter sets, and the binding's argument checks that run before any library call."""
import math

import numpy as np
import pytest

from oracle import nurbs
from paper_2011_13861_gb300 import inputs


def as_map(net):
    return nurbs.NURBSMap(net["deg"], net["knots"], net["ctrl"], net["weights"])


@pytest.mark.parametrize("dim", [2, 3])
def test_nets_describe_the_oracle_maps(dim):
    x = np.random.default_rng(dim).uniform(0, 1, (40, dim))
    pairs = [(inputs.quarter_annulus_net(1.0, 2.0, 1.0, dim), nurbs.quarter_annulus(1.0, 2.0, 1.0, dim)),
             (inputs.two_patch_annulus_net(1.0, 2.0, 1.0, dim, 1.0 / 3.0),
              nurbs.two_patch_annulus(1.0, 2.0, 1.0, dim, 1.0 / 3.0)),
             (inputs.two_patch_bar_net(0.6, 1.0 / 3.0, dim), nurbs.two_patch_bar(0.6, 1.0 / 3.0, dim))]
    for net, ref in pairs:
        F = as_map(net)
        assert np.abs(F(x) - ref(x)).max() < 1e-14
        assert np.abs(F.detDF(x) - ref.detDF(x)).max() < 1e-12 * np.abs(ref.detDF(x)).max()


def test_two_patch_nets_are_c0_with_a_jump_in_det_df():
    net = inputs.two_patch_annulus_net(dim=2, split=1.0 / 3.0)
    F = as_map(net)
    x = np.array([[0.5, 1.0 / 3.0]])
    assert np.abs(F(x, np.array([[0, -1]])) - F(x)).max() < 1e-15
    jl, jr = F.detDF(x, np.array([[0, -1]]))[0], F.detDF(x)[0]
    assert abs(jl / jr - 2.0) < 1e-12          # parametric lengths 1/3 and 2/3


def test_warmstart_parameters_are_seeded_and_in_range():
    a = inputs.warmstart_params(200, seed=5)
    b = inputs.warmstart_params(200, seed=5)
    c = inputs.warmstart_params(200, seed=6)
    assert a == b and a != c
    L = np.array([q["L"] for q in a])
    assert L.min() >= 0.1 and L.max() <= 2.0
    assert all(0.8 <= q["r_in"] <= 1.2 and 1.8 <= q["r_out"] <= 2.2 for q in a)
    kinds = {q["kernel"] for q in a}
    assert kinds == {"exp", "gauss"}


def test_warmstart_features():
    pytest.importorskip("torch")
    from paper_2011_13861_gb300 import warmstart
    f = warmstart.features({"kernel": "gauss", "L": 1.0, "r_in": 1.1, "r_out": 1.9})
    assert len(f) == warmstart.N_FEATURES
    assert f[0] == 0.0 and f[1] == -1.0
    assert abs(f[2] - 0.5) < 1e-12 and abs(f[3] + 0.5) < 1e-12
    g = warmstart.features({"kernel": "exp", "L": math.e, "r_in": 1.0, "r_out": 2.0})
    assert g == [1.0, 1.0, 0.0, 0.0]
