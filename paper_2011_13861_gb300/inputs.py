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
