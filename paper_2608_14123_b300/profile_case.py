"""Small cases for kernel profiling (ncu): one kernel of the hot path on a
mesh whose vectors exceed the 126 MB L2, so DRAM counters mean something,
with a few GB on the device at most.

    python -m paper_2608_14123_b300.profile_case apply_fp64 [reps]
    python -m paper_2608_14123_b300.profile_case apply_fp32 [reps]
    python -m paper_2608_14123_b300.profile_case scg_bf16 [reps]

apply_fp64: the FP64 curvilinear operator on 16^3 trilinear elements
(+-0.15h perturbation, p = 7, 2.1M DoF, about 0.25 GB of vectors and
geometry), `reps` applications inside the NVTX range "profiled" (the set-up's
own operator launches, on the root, stay outside it).  apply_fp32: the
smoothers' FP32 operator (g - A u, metric recomputed from the trilinear map)
on 32^3 such elements (16.8M DoF; its FP32 vectors and face data, about
0.6 GB, exceed L2 as well).  scg_bf16: the top-level SCG steps of the
mixed-precision smoother (BF16 tensor-core Schwarz sweep) on the 32^3 mesh
(the weighted patches alone take 0.23 GB).
"""
import sys

import numpy as np


def main():
    import torch

    from . import dgfas, workloads as wl
    case = sys.argv[1] if len(sys.argv) > 1 else "apply_fp64"
    reps = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    rng = np.random.default_rng(wl.SEED_BASE + 5)
    V = wl.perturbed_vertices(16 if case == "apply_fp64" else 32, 0.15, rng)
    levels = wl.hierarchy(V, [7, 3, 1], h_root=4)
    prec = dgfas.DGFAS_FP64 if case == "apply_fp64" else dgfas.DGFAS_BF16
    S = dgfas.Solver(levels, 5.0, 0.08, 2, 2, 4, precision=prec, smoother=dgfas.DGFAS_SCG)
    n = S.ndof(-1)
    u = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    g = torch.from_numpy(rng.standard_normal(n)).cuda()
    out = torch.empty_like(u)
    u32 = u.float()
    out32 = torch.empty_like(u32)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profiled")
    for _ in range(reps):
        if case == "apply_fp64":
            S.dgfas_apply_op(-1, u, g, out)
        elif case == "apply_fp32":
            S.dgfas_apply_op32(-1, u32, g, out32)
        else:
            S.dgfas_schwarz_smooth(-1, u, g, 1)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    S.close()
    print(f"{case}: {reps} launches on {n} DoF")


if __name__ == "__main__":
    main()
