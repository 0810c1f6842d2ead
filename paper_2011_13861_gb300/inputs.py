"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

Holds none of the method's arithmetic: only random blocks and the workload definitions
(geometry, spaces, kernels) of the synthetic configurations.
"""
import numpy as np


def random_block(n, nvec, seed):
    """n x nvec float64 block, entries uniform in [-1, 1), from numpy's PCG64 with the given seed."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, nvec))


# Synthetic workloads shaped like the configurations the method is measured on.
# Each entry: dim, degree, elements per direction, kernel, sigma, L, k, box.
WORKLOADS = {
    "square-p2-20x20-expsep": dict(dim=2, p=2, ne=20, kernel="exp_sep", sigma=1.0, L=1.0, k=10),
    "cube-p2-32^3-exp-L0.5": dict(dim=3, p=2, ne=32, kernel="exp", sigma=1.0, L=0.5, k=20),
    "cube-p3-48^3-gauss-L0.3": dict(dim=3, p=3, ne=48, kernel="gauss", sigma=1.0, L=0.3, k=20),
    # reduced meshes of the two cube workloads, sized for the dense oracle
    "cube-p2-16^3-exp-L0.5": dict(dim=3, p=2, ne=16, kernel="exp", sigma=1.0, L=0.5, k=20),
    "cube-p3-16^3-gauss-L0.3": dict(dim=3, p=3, ne=16, kernel="gauss", sigma=1.0, L=0.3, k=20),
}


def quarter_annulus_net(r_in=1.0, r_out=2.0, height=1.0, dim=3):
    """Control net of the quarter-annulus geometry (radius r_in..r_out, angle 0..pi/2, extruded
    to height for dim = 3): degree 2 per direction, one element, equally spaced radii and
    heights, the three angular control directions (1,0), (1,1), (0,1) with weights 1, sqrt(1/2),
    1.  Geometry data only (the input both sides evaluate): dict(deg, knots, ctrl, weights) with
    ctrl of shape (n_d, ..., n_1, dim), direction 1 (radius) fastest."""
    knots = [np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]) for _ in range(dim)]
    radii = [r_in, 0.5 * (r_in + r_out), r_out]
    dirs = [(1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    wang = [1.0, float(np.sqrt(0.5)), 1.0]
    zs = [0.0, 0.5 * height, height]
    shape = (3,) * dim
    ctrl = np.zeros(shape + (dim,))
    wts = np.zeros(shape)
    for idx in np.ndindex(*shape):
        i, j = idx[-1], idx[-2]              # radius (direction 1), angle (direction 2)
        pt = [radii[i] * dirs[j][0], radii[i] * dirs[j][1]]
        if dim == 3:
            pt.append(zs[idx[0]])
        ctrl[idx] = pt
        wts[idx] = wang[j]
    return {"deg": [2] * dim, "knots": knots, "ctrl": ctrl, "weights": wts}


def batched_instances(count=64, seed=2011, ne_range=(8, 40), degrees=(2, 3), L_range=(0.1, 2.0)):
    """Seeded instances of the batched workload: quarter annulus (radius 1..2, height 1, the net
    of quarter_annulus_net), elements per direction uniform on ne_range, degree uniform on
    `degrees` (same in every direction), kernels alternating exponential / Gaussian, L
    log-uniform on L_range, sigma 1.  Returns dicts with dim, p, ne, kernel, L, sigma."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ne = [int(x) for x in rng.integers(ne_range[0], ne_range[1] + 1, size=3)]
        p = int(rng.choice(degrees))
        L = float(np.exp(rng.uniform(np.log(L_range[0]), np.log(L_range[1]))))
        out.append({"dim": 3, "p": p, "ne": ne, "kernel": "exp" if i % 2 == 0 else "gauss", "L": L, "sigma": 1.0})
    return out


def warmstart_params(count, seed, L_range=(0.1, 2.0), r_in_range=(0.8, 1.2), r_out_range=(1.8, 2.2)):
    """Seeded parameter sets of the learned-warm-start workload (quarter annulus of height 1):
    kernel exponential or Gaussian with probability 1/2 each, L log-uniform on L_range, inner
    and outer radius uniform on their ranges, sigma 1.  Returns dicts with kernel, L, r_in, r_out."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kern = "exp" if rng.random() < 0.5 else "gauss"
        L = float(np.exp(rng.uniform(np.log(L_range[0]), np.log(L_range[1]))))
        r_in = float(rng.uniform(*r_in_range))
        r_out = float(rng.uniform(*r_out_range))
        out.append({"kernel": kern, "L": L, "r_in": r_in, "r_out": r_out})
    return out


def two_patch_annulus_net(r_in=1.0, r_out=2.0, height=1.0, dim=3, split=1.0 / 3.0):
    """Control net of a half annulus (radius r_in..r_out, angle 0..pi, extruded to height for
    dim = 3) made of two quarter-annulus patches joined with C^0 continuity at the angular
    parameter `split`: degree 2 per direction, angular knots (0,0,0,split,split,1,1,1), the
    angular control directions (1,0), (1,1), (0,1), (-1,1), (-1,0) with weights 1, sqrt(1/2), 1,
    sqrt(1/2), 1.  Geometry data only: dict(deg, knots, ctrl, weights), direction 1 (radius)
    fastest."""
    kl = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    ka = np.array([0.0, 0.0, 0.0, split, split, 1.0, 1.0, 1.0])
    knots = [kl, ka] + ([kl] if dim == 3 else [])
    radii = [r_in, 0.5 * (r_in + r_out), r_out]
    dirs = [(1.0, 0.0), (1.0, 1.0), (0.0, 1.0), (-1.0, 1.0), (-1.0, 0.0)]
    wang = [1.0, float(np.sqrt(0.5)), 1.0, float(np.sqrt(0.5)), 1.0]
    zs = [0.0, 0.5 * height, height]
    shape = ((3,) if dim == 3 else ()) + (5, 3)
    ctrl = np.zeros(shape + (dim,))
    wts = np.zeros(shape)
    for idx in np.ndindex(*shape):
        i, j = idx[-1], idx[-2]
        pt = [radii[i] * dirs[j][0], radii[i] * dirs[j][1]]
        if dim == 3:
            pt.append(zs[idx[0]])
        ctrl[idx] = pt
        wts[idx] = wang[j]
    return {"deg": [2] * dim, "knots": knots, "ctrl": ctrl, "weights": wts}


def two_patch_bar_net(a=0.6, split=1.0 / 3.0, dim=2):
    """Control net of a piecewise affine map of [0,1]^dim: direction 1 degree 1 with knots
    (0,0,split,1,1) and control abscissae 0, a, 1 (two affine patches joined with C^0 continuity),
    the other directions the identity (degree 1, one element).  Geometry data only."""
    k1 = np.array([0.0, 0.0, split, 1.0, 1.0])
    kid = np.array([0.0, 0.0, 1.0, 1.0])
    xs = [0.0, a, 1.0]
    shape = (2,) * (dim - 1) + (3,)
    ctrl = np.zeros(shape + (dim,))
    for idx in np.ndindex(*shape):
        pt = [xs[idx[-1]]] + [float(idx[-2 - k]) for k in range(dim - 1)]
        ctrl[idx] = pt
    return {"deg": [1] * dim, "knots": [k1] + [kid] * (dim - 1), "ctrl": ctrl, "weights": np.ones(shape)}
