"""Writes the training pairs of the learned surrogate with the oracle only.

    python -m oracle.make_surrogate_data [n_per_degree]

For p = 7 and p = 3 (the curvilinear workloads' smoothed degrees) it draws
interior elements from `surrogate.training_elements` (seed 20261202 + 100 + p),
fits the Kronecker-sum coefficients to each element block and stores
float32 inputs X [n, 24], targets Y [n, 6] and the geometric coefficients in
tests/golden/surrogate_fits_p{p}.npz.  Elements whose fitted coefficients are
not all positive are dropped (they have no valid surrogate).
"""
import os
import sys

import numpy as np

from . import surrogate as su

MU_STAR = 10.0
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "tests", "golden")


def make(p, n, seed):
    rng = np.random.default_rng(seed)
    corners = su.training_elements(n, rng)
    lv = dict(p=p, corners=corners, nbr=np.zeros((n, 6), np.int32))
    g_fit, g_geo = su.fit_coefficients(lv, MU_STAR)
    ok = np.all(g_fit > 0, axis=1)
    X = su.mlp_inputs(corners[ok])
    Y = su.mlp_targets(corners[ok], g_fit[ok])
    return X.astype(np.float32), Y.astype(np.float32), g_geo[ok], g_fit[ok]


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 6000
    for p in (7, 3):
        X, Y, g_geo, g_fit = make(p, n, 20261202 + 100 + p)
        path = os.path.join(OUT, f"surrogate_fits_p{p}.npz")
        np.savez_compressed(path, X=X, Y=Y, g_geo=g_geo.astype(np.float32),
                            g_fit=g_fit.astype(np.float32), mu_star=MU_STAR, p=p)
        print(path, X.shape)


if __name__ == "__main__":
    main()
