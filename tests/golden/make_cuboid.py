"""Writes cuboid_n*_np*.json: the oracle's interior densities for the cuboid
verification of Sec. 4.1 (Eq. RhoNeumann source on the x = 0 side, r = 1 on
every wall, mu = eta omega / (2c) = 0.4 pi for eta = 0.004, omega = 200 pi,
c = 1) on seeded Kuhn cuboids, and their relative mean error against the exact
ray solution of Eq. ExactSol.  Calls only the oracle and the seeded input
generators.

    python tests/golden/make_cuboid.py N NP   (cells per unit length, order)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1608_04607_gb300 import inputs as I  # noqa: E402

MU = 0.4 * np.pi
LENGTH = 2.0
JITTER, SEED = 0.2, 0


def exact_ray_density(x, mu=MU, length=LENGTH):
    """Eq. ExactSol with unit source density: forward and returning beams summed."""
    return (np.exp(-mu * x) + np.exp(-mu * (2 * length - x))) / (1 - np.exp(-2 * mu * length))


def _digits(v):
    """12 significant digits: far below every tolerance the tests apply."""
    return [float(f"{x:.12g}") for x in v]


def main(n, Np):
    m = I.kuhn_cuboid_mesh(n, length=LENGTH, jitter=JITTER, seed=SEED)
    mu = np.full(m.n_tets, MU)
    op = O.assemble(m.verts, m.tets, mu, 1.0, Np, nthreads=os.cpu_count())
    rho0 = O.source_directed(m.verts, m.tets, I.cuboid_rows_x0(m), Np, combine=True)
    rho, _ = O.solve_gmres(op, rho0, tol=1e-12, restart=200, nthreads=os.cpu_count())
    # the interior density functional: adaptive cubature (the accurate value)
    # and the fixed 32- and 64-point collapsed Gauss rules the GPU offers
    dens = O.tet_density(m.verts, m.tets, mu, Np, rho, nq=None, rtol=1e-11, nthreads=os.cpu_count())
    d32 = O.tet_density(m.verts, m.tets, mu, Np, rho, nq=32)
    d64 = O.tet_density(m.verts, m.tets, mu, Np, rho, nq=64)
    ex = exact_ray_density(O.centroids(m.verts, m.tets)[:, 0])
    err = float(np.mean(np.abs(dens - ex)) / np.mean(ex))
    out = dict(section="Sec. 4.1 (Eqs. RhoNeumann, IntDens, ExactSol)", n=n, Np=Np, length=LENGTH, mu=MU,
               refl=1.0, jitter=JITTER, seed=SEED, n_tets=m.n_tets, rel_mean_err=err,
               rel_mean_err_nq32=float(np.mean(np.abs(d32 - ex)) / np.mean(ex)),
               nq32_max_dev=float(np.abs(d32 - dens).max() / np.abs(dens).max()),
               nq64_max_dev=float(np.abs(d64 - dens).max() / np.abs(dens).max()),
               density=_digits(dens), density_nq32=_digits(d32), density_nq64=_digits(d64))
    with open(os.path.join(HERE, f"cuboid_n{n}_np{Np}.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(f"n={n} Np={Np}: {m.n_tets} tets, relative mean error {err:.5f} (32-point rule "
          f"{out['rel_mean_err_nq32']:.5f}; largest deviation of the 32/64-point rules "
          f"{out['nq32_max_dev']:.2e} / {out['nq64_max_dev']:.2e} of the maximum density)")


if __name__ == "__main__":
    main(int(sys.argv[1]), int(sys.argv[2]))
