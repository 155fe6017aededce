"""Multigrid cycles (Sec. 4.1-4.2, Algs. 1, 2, 5, 6), FP64.

Hierarchy: a list of levels (root first) with global refinement, so every
element of a non-top level is a twig and the top level holds the leaves.

* `was` is Alg. 5 (residual, then u += weighted Schwarz correction).
* `fas_vcycle` is Alg. 2; the projected solution P u_l of the down leg is kept
  and reused for the correction u_l += I (u_{l-1} - P u_l) of the up leg
  (u_l does not change in between).
* `cs_vcycle` is Alg. 1 (used to pin the FAS cycle: for a linear operator the
  FAS correction u_{l-1} - P u_l equals the CS correction, so both produce
  the same iterates up to round-off).
* `solve` runs V-cycles with crossover smoothing (Sec. 6.1 naming
  X-Y-S(n_s1,n_s2,n_sc)): n_s1 top sweeps before the first cycle and n_sc top
  sweeps between consecutive cycles in place of n_s2 + n_s1; the residual of
  the first down-leg step of each cycle is the stopping test
  r_2 <= rtol * r_2^0 (Euclidean norm over the leaf DoF, Sec. 6.1).
* The root problem is solved exactly (dense Cholesky of the assembled root
  matrix), or by SCG from the projected solution (coarse = "scg").
* `scg` is Alg. 6.
"""
import numpy as np
import scipy.linalg as sla

from .sip import LevelOps, apply, assemble
from .schwarz import Schwarz
from .transfer import Transfer


class Hierarchy:
    def __init__(self, levels, mu_star, delta, s1=2, s2=2, sc=4, nu=1.0, kappa=0.0,
                 gcoefs=None, smoother="was", scg_first="z", coarse="dense", root_rtol=1e-3,
                 root_steps=64, projection="interp"):
        self.levels = levels
        self.smoother = smoother
        self.scg_first = scg_first
        self.coarse = coarse
        self.root_rtol, self.root_steps = root_rtol, root_steps
        self.s1, self.s2, self.sc = s1, s2, sc
        self.ops = [LevelOps(lv, mu_star, nu, kappa) for lv in levels]
        self.sw = [Schwarz(lv, delta, mu_star, nu, kappa,
                           None if gcoefs is None else gcoefs[l])
                   if (l > 0 or coarse == "scg") else None
                   for l, lv in enumerate(levels)]
        self.tr = [None] + [Transfer(levels[l - 1], levels[l], projection)
                            for l in range(1, len(levels))]
        self.cls = [np.asarray(lv["cls"]) for lv in levels]
        self.active = [c != 2 for c in self.cls]
        self.local = any(np.any(c == 2) for c in self.cls) or any(
            np.any(c == 0) for c in self.cls[:-1])
        if coarse == "scg":
            self.nullspace = False
            self.root_chol = None
            return
        A0 = assemble(self.ops[0]).toarray()
        # kappa = 0 without Dirichlet faces (periodic or pure Neumann): A is
        # semidefinite with the constants as null space (remark on IPCG for
        # semidefinite systems).  The root is solved in the complement: for a
        # consistent g (1^T g = 0) the solution x of (A0 + c 1 1^T) x = g has
        # 1^T x = 0 and A0 x = g.
        self.nullspace = kappa == 0.0 and not np.any(np.asarray(levels[0]["nbr"]) == -1)
        if self.nullspace:
            n = A0.shape[0]
            A0 = A0 + (np.trace(A0) / n / n) * np.ones((n, n))
        self.root_chol = sla.cho_factor(A0)

    @property
    def L(self):
        return len(self.levels) - 1

    def A(self, l, u):
        """A_l u with frozen rows set to zero (Eq. (4d): r^f = 0)."""
        return apply(self.ops[l], u, rows_mask=self.active[l]).reshape(-1)

    def residual(self, l, u, g):
        return g - self.A(l, u)

    def smooth(self, l, u, g, n):
        """The level smoother: WAS (Alg. 5) or SCG (Alg. 6) with n steps."""
        if self.smoother == "scg":
            return self.scg(l, u, g, n, 0.0)
        return self.was(l, u, g, n)

    def was(self, l, u, g, n):
        """Alg. 5."""
        for _ in range(n):
            r = self.residual(l, u, g)
            u = u + self.sw[l].correction(r)
        return u

    def root_solve(self, g, u0=None):
        """The root problem A_0 u = g: exactly (dense Cholesky), or with
        coarse = "scg" by Alg. 6 as the coarse solver (Sec. 4.3.2): from u0
        (the projected solution in a V-cycle; zero if None) at most
        root_steps steps, leaving as soon as |r| <= root_rtol |r_start|."""
        if self.coarse != "scg":
            return sla.cho_solve(self.root_chol, g)
        u = np.zeros(self.ops[0].ndof) if u0 is None else u0
        r_max = self.root_rtol * np.linalg.norm(g - self.A(0, u))
        return self.scg(0, u, g, self.root_steps, r_max)

    def _down_up(self, u, f, r_top, top=None):
        """Alg. 2 below the top pre-smoothing: given the top residual r_top of
        u[L], project, form the parent right-hand sides, solve the root,
        prolongate the corrections and smooth on levels L-1..1 (top-level
        smoothing is left to the caller).  `top` makes a lower level act as
        the top (the sub-hierarchy cycles of the full multigrid startup)."""
        L = self.L if top is None else top
        u = list(u)
        g = [None] * (L + 1)
        g[L] = f
        ubar = [None] * (L + 1)
        r = r_top
        for l in range(L, 0, -1):
            if l < L:
                u[l] = self.smooth(l, u[l], g[l], self.s1)
                r = self.residual(l, u[l], g[l])
            u[l - 1] = self.tr[l].project(u[l])
            ubar[l - 1] = u[l - 1].copy()
            g[l - 1] = self.A(l - 1, u[l - 1]) + self.tr[l].restrict(r)
        u[0] = self.root_solve(g[0], u[0])
        for l in range(1, L + 1):
            u[l] = u[l] + self.tr[l].interpolate(u[l - 1] - ubar[l - 1])
            if l < L:
                u[l] = self.smooth(l, u[l], g[l], self.s2)
        return u

    def fas_vcycle(self, u, f):
        """Alg. 2 on the list u (one vector per level, root first); f is the top
        RHS.  Returns (u, |r_top|) with r_top the top residual after pre-smoothing."""
        L = self.L
        u = [x.copy() for x in u]
        u[L] = self.smooth(L, u[L], f, self.s1)
        r = self.residual(L, u[L], f)
        u = self._down_up(u, f, r)
        u[L] = self.smooth(L, u[L], f, self.s2)
        return u, np.linalg.norm(r)

    def fmg(self, f_levels, cycles=1):
        """Alg. 4 (FAS-FMG startup).  f_levels: each level's own right-hand
        side, root first.  Level 1 of the paper's loop is the root, whose
        V-cycle is its exact solve; then for l = 1 .. L-1 (root = 0) the
        solution is interpolated, u_l = I_l u_{l-1}, and improved by `cycles`
        FAS V-cycles (Alg. 2) on levels 0..l with f_l on top; the returned
        top start value is I_L u_{L-1}."""
        L = self.L
        u = [np.zeros(o.ndof) for o in self.ops]
        u[0] = self.root_solve(f_levels[0])
        for l in range(1, L):
            u[l] = self.tr[l].interpolate(u[l - 1])
            for _ in range(cycles):
                u[l] = self.smooth(l, u[l], f_levels[l], self.s1)
                r = self.residual(l, u[l], f_levels[l])
                u[:l + 1] = self._down_up(u[:l + 1], f_levels[l], r, top=l)
                u[l] = self.smooth(l, u[l], f_levels[l], self.s2)
        return self.tr[L].interpolate(u[L - 1])

    def cmg(self, f_levels, sc=None):
        """Alg. 3 (FAS-CMG, the cascadic startup).  f_levels: each level's own
        right-hand side, root first.  The root is solved for its right-hand
        side; then for l = 1 .. L-1 (root = 0) the solution is interpolated,
        u_l = I_l u_{l-1} (the whole level, frozen elements included), and
        improved by n_sc smoothing steps (`sc`, default the hierarchy's n_sc)
        with f_l; the top receives I_L u_{L-1} (the same end as Alg. 4).
        Returns the list of level vectors, root first, the top's last."""
        n = self.sc if sc is None else sc
        L = self.L
        u = [np.zeros(o.ndof) for o in self.ops]
        u[0] = self.root_solve(f_levels[0])
        for l in range(1, L):
            u[l] = self.smooth(l, self.tr[l].interpolate(u[l - 1]), f_levels[l], n)
        u[L] = self.tr[L].interpolate(u[L - 1])
        return u

    def cs_vcycle(self, u_top, f_top):
        """Alg. 1."""
        s1, s2 = self.s1, self.s2
        L = self.L
        u = [None] * (L + 1)
        f = [None] * (L + 1)
        u[L], f[L] = u_top.copy(), f_top
        for l in range(L, 0, -1):
            u[l] = self.smooth(l, u[l], f[l], s1)
            u[l - 1] = np.zeros(self.ops[l - 1].ndof)
            f[l - 1] = self.tr[l].restrict(f[l] - self.A(l, u[l]))
        u[0] = self.root_solve(f[0])
        for l in range(1, L + 1):
            u[l] = u[l] + self.tr[l].interpolate(u[l - 1])
            u[l] = self.smooth(l, u[l], f[l], s2)
        return u[L]

    def zero_levels(self, u_top):
        return [np.zeros(o.ndof) for o in self.ops[:-1]] + [u_top.copy()]

    def solve(self, u_top, f, rtol=1e-10, max_cycles=50):
        """V-cycles with crossover smoothing; returns (u_top, history of r_2).

        n_s1 top sweeps, then per cycle: top residual r (the stopping test
        |r| <= rtol |r^0|), the down/up legs, and n_sc top sweeps."""
        L = self.L
        u = self.zero_levels(u_top)
        hist = [np.linalg.norm(self.residual(L, u[L], f))]
        u[L] = self.smooth(L, u[L], f, self.s1)
        for k in range(max_cycles + 1):
            r = self.residual(L, u[L], f)
            if k > 0:
                hist.append(np.linalg.norm(r))
                if hist[-1] <= rtol * hist[0] or k == max_cycles:
                    break
            u = self._down_up(u, f, r)
            u[L] = self.smooth(L, u[L], f, self.sc)
        return u[L], hist

    def scg(self, l, u, f, n, r_max, precond=None, first=None):
        """Alg. 6: inexact preconditioned CG with one Schwarz sweep z = M r as
        the preconditioner, n steps or until |r| <= r_max.

        The first search direction is a reading (`first`, default the
        hierarchy's `scg_first`): "z" takes p = z in the first step, as in the
        inexact PCG the algorithm adopts (Golub and Ye), so that the step
        length gamma / p.q = z.r / z.A z is the exact line minimum along p;
        "r" takes the algorithm's printed initialization p = r unchanged in
        step 1.  `precond` replaces the Schwarz sweep (pins: identity ->
        textbook CG, exact inverse -> one step)."""
        first = self.scg_first if first is None else first
        M = self.sw[l].correction if precond is None else precond
        r = f - self.A(l, u)
        p = r.copy()
        r0 = None
        gamma = None
        for i in range(1, n + 1):
            z = M(r)
            if i > 1:
                beta = z @ (r - r0) / gamma
                p = beta * p + z
            elif first == "z":
                p = z.copy()
            q = self.A(l, p)
            gamma = z @ r
            alpha = gamma / (p @ q)
            r0 = r.copy()
            r = r - alpha * q
            u = u + alpha * p
            if np.linalg.norm(r) <= r_max:
                break
        return u


class LocalHierarchy(Hierarchy):
    """FAS for locally refined multilevel meshes (Sec. 3.1, 3.3, Alg. 2):
    twigs, leaves and frozen elements on every level; f is a list of per-level
    right-hand sides (used on leaves), u a list of per-level vectors."""

    def leaf_mask(self, l):
        N3 = self.ops[l].N ** 3
        return np.repeat(self.cls[l] == 0, N3)

    def element_energy(self, l, eps):
        """Element error indicators of the adaptive loop (Sec. 6.4): the
        operator applied to the complete error vector eps of level l (active
        and frozen columns), restricted to element e and weighted with the
        element's error coefficients, eps_e . (A_l eps)_e, for every element."""
        N3 = self.ops[l].N ** 3
        Ae = apply(self.ops[l], eps).reshape(-1, N3)
        return np.einsum("en,en->e", np.asarray(eps).reshape(-1, N3), Ae)

    def energy_error(self, eps_levels):
        """Energy norm of the error on the composite mesh (Sec. 6.1):
        (sum_l sum over the leaf elements of level l of eps_e . (A_l eps)_e)^(1/2)."""
        tot = 0.0
        for l, eps in enumerate(eps_levels):
            ind = self.element_energy(l, eps)
            tot += ind[self.cls[l] == 0].sum()
        return np.sqrt(tot)

    @staticmethod
    def mark_for_refinement(indicators, leaf, frac=0.7):
        """Leaf elements whose indicator exceeds frac times the largest one over
        all levels (Sec. 6.4); indicators and leaf are per-level arrays."""
        top = max(float(np.max(np.where(lf, ind, -np.inf))) for ind, lf in zip(indicators, leaf))
        return [lf & (ind > frac * top) for ind, lf in zip(indicators, leaf)]

    def composite_residual(self, u, f):
        """r_2 of Sec. 6.1: Euclidean norm of the leaf residuals of all levels,
        evaluated on the composite solution: the twigs of each level first take
        the projection of the finer level (top down, Eq. (6b)), the frozen
        elements keep their interpolated values."""
        u = list(u)
        for l in range(self.L, 0, -1):
            u[l - 1], _ = self.tr[l].project_active(u[l], u[l - 1], self.cls[l])
        s = 0.0
        for l in range(self.L + 1):
            m = self.leaf_mask(l)
            if np.any(m):
                r = f[l] - self.A(l, u[l])
                s += np.sum(r[m] ** 2)
        return np.sqrt(s)

    def _down_up_local(self, u, f, r_top, top=None):
        L = self.L if top is None else top
        u = list(u)
        g = [None] * (L + 1)
        g[L] = f[L]
        ubar = [None] * (L + 1)
        r = r_top
        for l in range(L, 0, -1):
            if l < L:
                u[l] = self.smooth(l, u[l], g[l], self.s1)
                r = self.residual(l, u[l], g[l])
            u[l - 1], _ = self.tr[l].project_active(u[l], u[l - 1], self.cls[l])
            ubar[l - 1] = u[l - 1].copy()
            t = self.tr[l].restrict_active(r, self.cls[l])
            gl = self.A(l - 1, u[l - 1]) + t
            leaf = self.leaf_mask(l - 1)
            gl[leaf] = f[l - 1][leaf]
            g[l - 1] = gl
        u[0] = self.root_solve(g[0], u[0])
        for l in range(1, L + 1):
            u[l] = self.tr[l].prolong_fas(u[l], u[l - 1], ubar[l - 1], self.cls[l])
            if l < L:
                u[l] = self.smooth(l, u[l], g[l], self.s2)
        return u

    def fmg_local(self, f, cycles=1):
        """Alg. 4 on a locally refined hierarchy: the root solved for its own
        right-hand side, then for l = 1 .. L-1 the interpolation of the whole
        level u_l = I_l u_{l-1} (frozen elements included) and `cycles` FAS
        V-cycles with level l as the top (all its active rows use f_l; below
        it the leaves keep their own f).  Returns the list of level vectors
        with the top's I_L u_{L-1}: the start of the composite solve."""
        L = self.L
        u = [np.zeros(o.ndof) for o in self.ops]
        u[0] = self.root_solve(f[0])
        for l in range(1, L):
            u[l] = self.tr[l].interpolate(u[l - 1])
            for _ in range(cycles):
                u[l] = self.smooth(l, u[l], f[l], self.s1)
                r = self.residual(l, u[l], f[l])
                u[:l + 1] = self._down_up_local(u[:l + 1], f[:l + 1], r, top=l)
                u[l] = self.smooth(l, u[l], f[l], self.s2)
        u[L] = self.tr[L].interpolate(u[L - 1])
        return u

    def fas_vcycle_local(self, u, f):
        """Alg. 2 on all levels of a locally refined hierarchy; returns (u, |r_top|)."""
        L = self.L
        u = [x.copy() for x in u]
        u[L] = self.smooth(L, u[L], f[L], self.s1)
        r = self.residual(L, u[L], f[L])
        u = self._down_up_local(u, f, r)
        u[L] = self.smooth(L, u[L], f[L], self.s2)
        return u, np.linalg.norm(r)

    def solve_local(self, u, f, rtol=1e-10, max_cycles=50):
        """Crossover solve on the composite problem; returns (u, history of r_2)."""
        L = self.L
        u = [x.copy() for x in u]
        hist = [self.composite_residual(u, f)]
        u[L] = self.smooth(L, u[L], f[L], self.s1)
        for k in range(max_cycles):
            r = self.residual(L, u[L], f[L])
            u = self._down_up_local(u, f, r)
            u[L] = self.smooth(L, u[L], f[L], self.sc)
            hist.append(self.composite_residual(u, f))
            if hist[-1] <= rtol * hist[0]:
                break
        return u, hist
