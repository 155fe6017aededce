"""Transfer operators between consecutive levels (Sec. 3.2), FP64.

* I (prolongation): embedded interpolation, the coarse polynomial evaluated at
  the fine nodes.  p-refinement: same element; h-refinement: child octant
  (c1,c2,c3) takes the parent reference coordinate (xi + (2c-1))/2.
* R = I^T (restriction, the transpose of I, Sec. 3.2).
* P (solution projection), two variants (Sec. 3.2):
  - embedded interpolation ("interp"): the fine polynomial evaluated at the
    coarse nodes; for h-refinement each parent node takes the value of the
    child that contains it, and parent nodes on a child interface (only for
    even p, the middle GLL node) average the children that share them;
  - L2 projection ("l2"), reading: the projection onto the coarse polynomials
    in the reference coordinates with the inner product of the fine level's
    GLL quadrature, P = (I^T W I)^-1 I^T W per direction.  For h-refinement
    the two half-cells of a direction each carry half of the parent's
    reference width: P_s = M^-1 (1/2) I_s^T W with M = (1/2) sum_s I_s^T W I_s,
    and a parent sums the contributions of its children (no averaging).  On
    affine elements this is the physical L2 projection.

Pins (tests/test_oracle_transfer.py): P I = identity; I reproduces coarse
polynomials at the fine nodes' physical positions; R equals the transpose of
the assembled I; averaging happens only for even p.
"""
import numpy as np

from .gll import gll, interp_matrix


def _mode(A1, A2, A3, u):
    """(A3 x A2 x A1) applied to u [ne, k, j, i]."""
    y = np.einsum("ai,ekji->ekja", A1, u)
    y = np.einsum("bj,ekja->ekba", A2, y)
    return np.einsum("ck,ekba->ecba", A3, y)


class Transfer:
    """Transfers between coarse level `lc` and fine level `lf` (fine['parent'])."""

    def __init__(self, lc, lf, projection="interp"):
        self.projection = projection
        self.pc, self.pf = lc["p"], lf["p"]
        self.Nc, self.Nf = self.pc + 1, self.pf + 1
        self.nec, self.nef = lc["nbr"].shape[0], lf["nbr"].shape[0]
        self.parent = lf["parent"]
        self.octant = lf["octant"]
        self.h = bool(np.all(self.octant >= 0))
        xf, _ = gll(self.pf)
        xc, _ = gll(self.pc)
        if not self.h:
            self.I1 = [interp_matrix(self.pc, xf)]          # [Nf, Nc]
            self.P1 = [interp_matrix(self.pf, xc)]          # [Nc, Nf]
        else:
            assert self.pc == self.pf
            self.I1 = [interp_matrix(self.pc, (xf + s) / 2.0) for s in (-1.0, 1.0)]
            self.P1 = []
            for s, inside in ((-1.0, xc <= 0.0), (1.0, xc >= 0.0)):
                wgt = np.where(inside, np.where(xc == 0.0, 0.5, 1.0), 0.0)
                xchild = np.clip(2.0 * xc - s, -1.0, 1.0)
                self.P1.append(wgt[:, None] * interp_matrix(self.pf, xchild))
        if projection == "l2":
            _, wf = gll(self.pf)
            W = np.diag(wf)
            if not self.h:
                I1 = self.I1[0]
                self.P1 = [np.linalg.solve(I1.T @ W @ I1, I1.T @ W)]
            else:
                M = 0.5 * sum(I.T @ W @ I for I in self.I1)
                self.P1 = [np.linalg.solve(M, 0.5 * I.T @ W) for I in self.I1]
        elif projection != "interp":
            raise ValueError(f"unknown projection {projection}")

    def _oct(self, e):
        o = self.octant[e]
        return (0, 0, 0) if o < 0 else (o & 1, (o >> 1) & 1, (o >> 2) & 1)

    def active_children(self, lf_cls):
        """Mask of fine elements that take part in P and R (active children)."""
        return np.asarray(lf_cls) != 2

    def project_active(self, uf, uc_old, fine_cls):
        """u_c^t = P^{t,a} u_f^a: only active children contribute and only their
        parents (twigs) receive a result; other coarse entries keep uc_old."""
        act = self.active_children(fine_cls)
        uf = np.asarray(uf).reshape(self.nef, self.Nf, self.Nf, self.Nf)
        out = np.asarray(uc_old).reshape(self.nec, self.Nc, self.Nc, self.Nc).copy()
        recv = np.zeros(self.nec, bool)
        recv[self.parent[act]] = True
        out[recv] = 0.0
        for e in np.nonzero(act)[0]:
            o = self._oct(e)
            A = [self.P1[o[d]] for d in range(3)] if self.h else [self.P1[0]] * 3
            out[self.parent[e]] += _mode(A[0], A[1], A[2], uf[e][None])[0]
        return out.reshape(-1), recv

    def restrict_active(self, rf, fine_cls):
        """R^{t,a} r_f^a: only active children contribute."""
        act = self.active_children(fine_cls)
        rf = np.asarray(rf).reshape(self.nef, self.Nf, self.Nf, self.Nf).copy()
        rf[~act] = 0.0
        return self.restrict(rf)

    def prolong_fas(self, uf, uc, ubar, fine_cls):
        """Frozen update u_f^f = I u_c (parents are leaves) and correction
        prolongation u_f^a += I (u_c - ubar) on active children (Alg. 2)."""
        fr = np.asarray(fine_cls) == 2
        uf = np.asarray(uf).reshape(self.nef, self.Nf, self.Nf, self.Nf).copy()
        full = self.interpolate(uc).reshape(uf.shape)
        corr = self.interpolate(np.asarray(uc) - np.asarray(ubar)).reshape(uf.shape)
        uf[fr] = full[fr]
        uf[~fr] += corr[~fr]
        return uf.reshape(-1)

    def interpolate(self, uc):
        """u_f = I u_c on every fine element."""
        uc = np.asarray(uc).reshape(self.nec, self.Nc, self.Nc, self.Nc)
        uf = np.zeros((self.nef, self.Nf, self.Nf, self.Nf))
        for e in range(self.nef):
            o = self._oct(e)
            A = [self.I1[o[d]] for d in range(3)] if self.h else [self.I1[0]] * 3
            uf[e] = _mode(A[0], A[1], A[2], uc[self.parent[e]][None])[0]
        return uf.reshape(-1)

    def restrict(self, rf):
        """r_c = R r_f = I^T r_f."""
        rf = np.asarray(rf).reshape(self.nef, self.Nf, self.Nf, self.Nf)
        rc = np.zeros((self.nec, self.Nc, self.Nc, self.Nc))
        for e in range(self.nef):
            o = self._oct(e)
            A = [self.I1[o[d]] for d in range(3)] if self.h else [self.I1[0]] * 3
            rc[self.parent[e]] += _mode(A[0].T, A[1].T, A[2].T, rf[e][None])[0]
        return rc.reshape(-1)

    def project(self, uf):
        """u_c = P u_f (embedded interpolation with averaging at shared nodes)."""
        uf = np.asarray(uf).reshape(self.nef, self.Nf, self.Nf, self.Nf)
        uc = np.zeros((self.nec, self.Nc, self.Nc, self.Nc))
        for e in range(self.nef):
            o = self._oct(e)
            A = [self.P1[o[d]] for d in range(3)] if self.h else [self.P1[0]] * 3
            uc[self.parent[e]] += _mode(A[0], A[1], A[2], uf[e][None])[0]
        return uc.reshape(-1)
