"""Adaptive refinement loop of the steep-front problem (Sec. 6.4) on the CUDA
path: solve on the current multilevel mesh, element error indicators
eps_e . (A eps)_e of the error against the exact solution on every level
(`dgfas_element_energy`), marking of the leaves above a fraction of the
largest indicator (plus the elements cut by the front), admissibility closure
and rebuild of the refinement levels.  The marking and the rebuild are host
logic on integer cell sets; every numerical step runs in the library.
"""
import numpy as np

from . import dgfas
from . import workloads as wl


def cut_cells(spec, n, cells):
    """Cells (integer coordinates on grid n) that the front passes through."""
    arr = np.array(sorted(cells), dtype=np.int64).reshape(-1, 3)
    h = 1.0 / n
    d = wl._cell_front_distance(spec, arr * h, h)
    return {tuple(int(v) for v in c) for c, dd in zip(arr, d) if dd <= 0.0}


def level_rhs(S, spec):
    """Per-level right-hand sides, assembled on the GPU from the exact f and
    u_D, root first; the ones below the top are also handed to the library
    (their leaf rows use them)."""
    import torch
    L = S.n_levels - 1
    out = []
    for l in range(S.n_levels):
        xyz = S.node_coords(l).cpu().numpy()
        fn = torch.from_numpy(wl.eval_front_f(spec, xyz)).cuda()
        un = torch.from_numpy(wl.eval_front_u(spec, xyz)).cuda()
        b = torch.empty_like(fn)
        S.dgfas_assemble_rhs_level(l, fn, un, b)
        if l < L:
            S.dgfas_set_level_rhs(l, b)
        out.append(b)
    return out


def indicators(S, spec, u_top):
    """Element indicators of every level from the composite solution: the
    top's u_top and the level solutions kept by the solve, whose last
    composite residual left the twigs with the projection of the finer level."""
    import torch
    out = []
    for l in range(S.n_levels):
        if l == S.n_levels - 1:
            ul = u_top
        else:
            ul = torch.empty(S.ndof(l), dtype=torch.float64, device="cuda")
            S.dgfas_get_level_solution(l, ul)
        xyz = S.node_coords(l).cpu().numpy()
        eps = ul - torch.from_numpy(wl.eval_front_u(spec, xyz)).cuda()
        ne = S.levels[l]["corners"].shape[0]
        ind = torch.empty(ne, dtype=torch.float64, device="cuda")
        S.dgfas_element_energy(l, eps, ind)
        out.append(ind.cpu().numpy())
    return out


def new_marks(levels, marks, ind, base, max_ref, spec, n_base, frac=0.7):
    """Refined cell sets of the next mesh: the current ones, the leaves of the
    adaptive levels (base and up, below the last allowed) whose indicator
    exceeds frac times the largest leaf indicator, and the leaves cut by the
    front."""
    marks = [set(m) for m in marks]
    leaf = [np.asarray(lv["cls"]) == wl.LEAF for lv in levels]
    top = max(float(np.max(np.where(lf, x, -np.inf))) for x, lf in zip(ind[base:], leaf[base:]))
    for k in range(max_ref):
        l = base + k
        if l >= len(levels):
            break
        lv = levels[l]
        cells = [tuple(int(v) for v in c) for c in lv["ijk"]]
        big = {c for c, x, lf in zip(cells, ind[l], leaf[l]) if lf and x > frac * top}
        cut = cut_cells(spec, n_base << k, [c for c, lf in zip(cells, leaf[l]) if lf])
        while len(marks) <= k:
            marks.append(set())
        marks[k] |= big | cut
    return marks


def run(spec, n_base=4, p=3, n_root=2, max_ref=2, rounds=3, cycles=2, mu_star=5.0,
        delta=0.08, s=(2, 2, 2), precision=dgfas.DGFAS_FP64, smoother=dgfas.DGFAS_SCG,
        start="fmg"):
    """The loop; returns one record per round (closed marks, leaf elements per
    level, composite energy norm of the error) and the final marks.  Each
    round solves as the paper's loop does: the full multigrid startup (Alg. 4)
    and `cycles` = 2 FAS V-cycles with the SCG(2, 2, 2) smoother (start =
    "zero": the cycles from u = 0 instead)."""
    import torch
    marks = [cut_cells(spec, n_base, {(x, y, z) for z in range(n_base) for y in range(n_base)
                                       for x in range(n_base)})]
    hist = []
    for _ in range(rounds):
        marks = wl.close_marks(marks, n_base)
        levels = wl.hierarchy_from_marks(marks, n_base=n_base, p=p, n_root=n_root)
        base = len(levels) - 1 - len(marks)
        S = dgfas.Solver(levels, mu_star, delta, *s, precision=precision, smoother=smoother)
        try:
            f = level_rhs(S, spec)
            u = torch.zeros_like(f[-1])
            if start == "fmg":
                S.dgfas_fmg(f, u, 1)
            S.dgfas_solve(u, f[-1], 1e-300, cycles, raise_on_fail=False)   # exactly `cycles` cycles
            ind = indicators(S, spec, u)
        finally:
            S.close()
        leaf = [np.asarray(lv["cls"]) == wl.LEAF for lv in levels]
        err = float(np.sqrt(sum(x[lf].sum() for x, lf in zip(ind, leaf))))
        hist.append(dict(marks=[sorted(m) for m in marks], leaves=[int(lf.sum()) for lf in leaf],
                         energy_error=err))
        marks = new_marks(levels, marks, ind, base, max_ref, spec, n_base)
    return hist, marks
