"""The adaptive loop of the front problem (Sec. 6.4) on the CUDA path against
the same loop on the oracle: each round solves with the full multigrid
startup and two FAS V-cycles with the SCG(2, 2, 2) smoother, as the paper's
loop; per round the closed refined-cell sets, the leaf elements per level and
the composite energy norm of the error are compared (the marking is each
side's own; the cell-set closure and rebuild are shared topology)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import adaptive, dgfas
from paper_2608_14123_b300 import workloads as wl

pytestmark = pytest.mark.gpu

N_BASE, P, N_ROOT, MAX_REF, ROUNDS, CYCLES = 4, 3, 2, 2, 2, 2
MU, DELTA, S = 5.0, 0.08, (2, 2, 2)


def _cut(spec, n, cells):
    arr = np.array(sorted(cells), dtype=np.int64).reshape(-1, 3)
    d = wl._cell_front_distance(spec, arr / n, 1.0 / n)
    return {tuple(int(v) for v in c) for c, dd in zip(arr, d) if dd <= 0.0}


def _oracle_loop(spec):
    from oracle import fas, sip
    marks = [_cut(spec, N_BASE, {(x, y, z) for z in range(N_BASE) for y in range(N_BASE)
                                 for x in range(N_BASE)})]
    hist = []
    for _ in range(ROUNDS):
        marks = wl.close_marks(marks, N_BASE)
        levels = wl.hierarchy_from_marks(marks, n_base=N_BASE, p=P, n_root=N_ROOT)
        base = len(levels) - 1 - len(marks)
        H = fas.LocalHierarchy(levels, MU, DELTA, *S, smoother="scg")
        f, uex = [], []
        for op in H.ops:
            X = op.geo["x"]
            f.append(sip.rhs(op, wl.eval_front_f(spec, X), wl.eval_front_u(spec, X)).reshape(-1))
            uex.append(wl.eval_front_u(spec, X).reshape(-1))
        u, _ = H.solve_local(H.fmg_local(f, 1), f, rtol=1e-300, max_cycles=CYCLES)
        # the composite solution: twigs take the projection of the finer level
        # (as the library's last composite residual evaluation leaves them)
        for l in range(len(levels) - 1, 0, -1):
            u[l - 1], _ = H.tr[l].project_active(u[l], u[l - 1], H.cls[l])
        ind = [H.element_energy(l, u[l] - uex[l]) for l in range(len(levels))]
        leaf = [np.asarray(lv["cls"]) == wl.LEAF for lv in levels]
        err = float(np.sqrt(sum(x[lf].sum() for x, lf in zip(ind, leaf))))
        hist.append(dict(marks=[sorted(m) for m in marks], leaves=[int(lf.sum()) for lf in leaf],
                         energy_error=err))
        big = fas.LocalHierarchy.mark_for_refinement(ind[base:], leaf[base:], 0.7)
        marks = [set(m) for m in marks]
        for k in range(MAX_REF):
            l = base + k
            if l >= len(levels):
                break
            cells = [tuple(int(v) for v in c) for c in levels[l]["ijk"]]
            sel = {c for c, b in zip(cells, big[k]) if b}
            cut = _cut(spec, N_BASE << k, [c for c, lf in zip(cells, leaf[l]) if lf])
            while len(marks) <= k:
                marks.append(set())
            marks[k] |= sel | cut
    return hist


def test_adaptive_loop_matches_oracle():
    spec = wl.front_spec(np.random.default_rng(wl.SEED_BASE + 4))
    hist_g, _ = adaptive.run(spec, n_base=N_BASE, p=P, n_root=N_ROOT, max_ref=MAX_REF,
                             rounds=ROUNDS, cycles=CYCLES, mu_star=MU, delta=DELTA, s=S,
                             precision=dgfas.DGFAS_FP64)
    hist_o = _oracle_loop(spec)
    for hg, ho in zip(hist_g, hist_o):
        assert hg["marks"] == ho["marks"]
        assert hg["leaves"] == ho["leaves"]
        assert abs(hg["energy_error"] - ho["energy_error"]) <= 1e-9 * ho["energy_error"]
    # the loop refines: the second mesh has more leaf elements
    assert sum(hist_g[1]["leaves"]) > sum(hist_g[0]["leaves"])
