"""Writes the training targets of the learned surrogate with the oracle only.

    python -m oracle.make_surrogate_data [n] [workers]

For p = 7 and p = 3 (the curvilinear workloads' smoothed degrees) it takes
the n seeded training elements of `workloads.surrogate_training_set(n, p)`
(half from the graded +-0.25 distribution, half from the uniform +-0.15 one),
fits the Kronecker-sum coefficients to each element block
(`surrogate.fit_coefficients`) and stores in
tests/golden/surrogate_fits_p{p}_n{n}.npz:

  ok  bool [n]         elements with all fitted coefficients positive (the
                       others have no valid surrogate and are dropped)
  Y   float32 [n_ok,6] targets (log(dx_i^geo / V^(1/3)), log(g_i^fit / g_i^geo))
  g_fit float32 [n_ok,3]

The inputs are not stored: they are the elements' normalized corners,
regenerated from the seed (`surrogate.mlp_inputs` on the oracle side, the
library's own input kernel on the CUDA side).  The fits of disjoint chunks
run in worker processes (spawned, not forked).
"""
import os
import sys

import numpy as np

from . import surrogate as su

MU_STAR = 10.0
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "tests", "golden")


def _fit_chunk(args):
    p, corners = args
    lv = dict(p=p, corners=corners, nbr=np.zeros((len(corners), 6), np.int32))
    g_fit, _ = su.fit_coefficients(lv, MU_STAR)
    return g_fit


def fit_all(p, corners, workers=1, chunk=500):
    parts = [(p, corners[i:i + chunk]) for i in range(0, len(corners), chunk)]
    if workers <= 1:
        return np.concatenate([_fit_chunk(a) for a in parts], 0)
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.concatenate(pool.map(_fit_chunk, parts), 0)


def make(p, n, workers=1):
    from paper_2608_14123_b300.workloads import surrogate_training_set
    corners = surrogate_training_set(n, p)
    g_fit = fit_all(p, corners, workers)
    ok = np.all(g_fit > 0, axis=1)
    Y = su.mlp_targets(corners[ok], g_fit[ok])
    return ok, Y.astype(np.float32), g_fit[ok].astype(np.float32)


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 100000
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    for p in (7, 3):
        ok, Y, g_fit = make(p, n, workers)
        path = os.path.join(OUT, f"surrogate_fits_p{p}_n{n}.npz")
        np.savez_compressed(path, ok=ok, Y=Y, g_fit=g_fit, mu_star=MU_STAR, p=p, n=n)
        print(path, int(ok.sum()), "of", n)


if __name__ == "__main__":
    main()
