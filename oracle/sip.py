"""Symmetric interior penalty DG-SEM operator (Sec. 2.2, Eq. (2)), FP64.

Three independent forms of the same operator A of Eq. (3):

* `brute_force_matrix`: the bilinear form of Eq. (2) evaluated entry by entry
  from physical points: basis values/gradients from the Lagrange product
  formula at each quadrature point, face normals from the cross product of the
  face tangents, and the neighbour's reference coordinates of every face point
  found by Newton inversion of the neighbour's map.  Tiny meshes only.
* `assemble`: element-block assembly with dense per-element reference gradient
  operators (Kronecker products of the 1D derivative matrix) and trace /
  normal-flux operators per face.  Small meshes.
* `apply`: matrix-free sum-factorized application, vectorized over elements
  (used by the V-cycle and the CPU baseline).

With GLL collocation (the remark of Sec. 2.2) the lumped mass and the volume
and face integrals all use the nodal quadrature.  Constant nu and kappa.

Pins (tests/test_oracle_sip.py): brute force == assembly to 1e-12; apply ==
assembly; symmetry; positive definiteness with Dirichlet faces; A 1 = 0 with
all-Neumann faces and kappa = 0; on uniform Cartesian meshes A equals the
Kronecker sum of the separately assembled global 1D SIP matrices; discrete
consistency A I(u) = b for polynomials u in Q_p; convergence of order p+1 to a
manufactured solution.
"""
import numpy as np
import scipy.sparse as sp

from .gll import gll, diff_matrix, lagrange_eval, lagrange_deriv_eval
from .geometry import (node_geometry, volume_metric, face_factors, face_node_index,
                       h_perp, penalties, map_and_jacobian)


class LevelOps:
    """All per-level data the oracle needs: geometry, metric, face factors, penalty."""

    def __init__(self, level, mu_star, nu=1.0, kappa=0.0):
        self.level = level
        self.p = level["p"]
        self.N = self.p + 1
        self.nu, self.kappa, self.mu_star = nu, kappa, mu_star
        self.nbr = level["nbr"]
        self.ne = self.nbr.shape[0]
        self.geo = node_geometry(level["corners"], self.p)
        self.G = volume_metric(self.geo, nu)
        self.W, self.c = face_factors(self.geo, nu)
        self.hp = h_perp(self.geo, self.W)
        self.mu = penalties(level, self.hp, mu_star)
        self.D = diff_matrix(self.p)
        self.mass = self.geo["W3"] * self.geo["detJ"]  # lumped GLL mass

    @property
    def ndof(self):
        return self.ne * self.N ** 3


# ------------------------------------------------------------------ matrix-free
def ref_grad(D, u):
    """du/dxi_t for t = 1,2,3 on node arrays u [ne, k, j, i]."""
    d1 = np.einsum("il,ekjl->ekji", D, u)
    d2 = np.einsum("jl,ekli->ekji", D, u)
    d3 = np.einsum("kl,elji->ekji", D, u)
    return np.stack([d1, d2, d3], axis=-1)


def ref_grad_T(D, F):
    """Transpose of ref_grad: sum_t B_t^T F_t."""
    r = np.einsum("li,ekjl->ekji", D, F[..., 0])
    r += np.einsum("lj,ekli->ekji", D, F[..., 1])
    r += np.einsum("lk,elji->ekji", D, F[..., 2])
    return r


def apply(ops, u, rows_mask=None):
    """A u, matrix-free (Eq. (2) with GLL collocation).  u [ne, N, N, N] or flat.

    rows_mask (bool [ne]) optionally zeroes rows of elements not in the mask
    (frozen rows, Eq. (4d))."""
    N, ne = ops.N, ops.ne
    u = np.asarray(u, dtype=np.float64).reshape(ne, N, N, N)
    du = ref_grad(ops.D, u)
    F = np.einsum("ekjidf,ekjif->ekjid", ops.G, du)
    R = ops.kappa * ops.mass * u
    for f in range(6):
        K, J, I = face_node_index(N, f)
        nb = ops.nbr[:, f]
        um = u[:, K, J, I]
        qm = np.einsum("ebat,ebat->eba", ops.c[:, f], du[:, K, J, I, :])
        W, c, mu = ops.W[:, f], ops.c[:, f], ops.mu[:, f][:, None, None]
        interior = nb >= 0
        dirichlet = nb == -1
        jump = np.zeros_like(um)
        flux = np.zeros_like(um)
        if np.any(interior):
            nbi = nb[interior]
            g = f ^ 1
            Kg, Jg, Ig = face_node_index(N, g)
            up = u[nbi][:, Kg, Jg, Ig]
            dup = du[nbi][:, Kg, Jg, Ig, :]
            qp = np.einsum("ebat,ebat->eba", ops.c[nbi, g], dup)
            jump[interior] = um[interior] - up
            # penalty mu*nu*[[v]].[[u]] and -[[v]].{{nu grad u}} = -v (q- - q+)/2
            flux[interior] = mu[interior] * W[interior] * jump[interior] * ops.nu \
                - 0.5 * (qm[interior] - qp)
        # -{{nu grad v}}.[[u]]: lifted into the volume flux, -c_t [[u]]/2 per node
        lift = -0.5 * jump
        if np.any(dirichlet):
            ud = um[dirichlet]
            flux[dirichlet] = 2.0 * mu[dirichlet] * ops.nu * W[dirichlet] * ud - qm[dirichlet]
            lift[dirichlet] = -ud
        R[:, K, J, I] += flux
        F[:, K, J, I, :] += c * lift[..., None]
    R += ref_grad_T(ops.D, F)
    if rows_mask is not None:
        R[~rows_mask] = 0.0
    return R


def rhs(ops, f_nodal, uD_nodal=None):
    """Right-hand side of Eq. (2): int v f + Dirichlet terms, GLL quadrature.
    f_nodal, uD_nodal: node values [ne, N, N, N] (uD only read at Dirichlet faces)."""
    N, ne = ops.N, ops.ne
    b = ops.mass * np.asarray(f_nodal).reshape(ne, N, N, N)
    if uD_nodal is None:
        return b
    uD = np.asarray(uD_nodal).reshape(ne, N, N, N)
    F = np.zeros((ne, N, N, N, 3))
    for f in range(6):
        K, J, I = face_node_index(N, f)
        dirichlet = ops.nbr[:, f] == -1
        if not np.any(dirichlet):
            continue
        ud = np.where(dirichlet[:, None, None], uD[:, K, J, I], 0.0)
        mu = ops.mu[:, f][:, None, None]
        b[:, K, J, I] += 2.0 * mu * ops.nu * ops.W[:, f] * ud
        F[:, K, J, I, :] += -ops.c[:, f] * ud[..., None]
    return b + ref_grad_T(ops.D, F)


# ------------------------------------------------------------------ assembly
def _kron3(A3, A2, A1):
    return np.kron(A3, np.kron(A2, A1))


def assemble(ops, fmt="csr"):
    """Element-block assembly of A (sparse), rows/cols e*N^3 + (k N + j) N + i."""
    N, ne = ops.N, ops.ne
    n3 = N ** 3
    I_ = np.eye(N)
    B = [_kron3(I_, I_, ops.D), _kron3(I_, ops.D, I_), _kron3(ops.D, I_, I_)]
    rows, cols, vals = [], [], []

    def add(ei, ej, M):
        r, c = np.nonzero(np.abs(M) > 0)
        rows.append(ei * n3 + r)
        cols.append(ej * n3 + c)
        vals.append(M[r, c])

    def trace(f):
        K, J, I = face_node_index(N, f)
        T = np.zeros((N * N, n3))
        T[np.arange(N * N), (K * N * N + J * N + I).reshape(-1)] = 1.0
        return T

    Ts = [trace(f) for f in range(6)]
    for e in range(ne):
        G = ops.G[e].reshape(n3, 3, 3)
        Ke = ops.kappa * np.diag(ops.mass[e].reshape(-1))
        for d in range(3):
            for g in range(3):
                Ke += B[d].T @ (G[:, d, g][:, None] * B[g])
        add(e, e, Ke)
        for f in range(6):
            nb = ops.nbr[e, f]
            if nb == -2:
                continue
            T = Ts[f]
            W = ops.W[e, f].reshape(-1)
            Q = sum(ops.c[e, f, :, :, t].reshape(-1)[:, None] * (T @ B[t]) for t in range(3))
            mu = ops.mu[e, f]
            if nb == -1:
                add(e, e, 2.0 * mu * ops.nu * T.T @ (W[:, None] * T) - Q.T @ T - T.T @ Q)
                continue
            g = f ^ 1
            Tp = Ts[g]
            Qp = sum(ops.c[nb, g, :, :, t].reshape(-1)[:, None] * (Tp @ B[t]) for t in range(3))
            # rows of e only; columns of e and nb
            add(e, e, mu * ops.nu * T.T @ (W[:, None] * T) - 0.5 * Q.T @ T - 0.5 * T.T @ Q)
            add(e, nb, -mu * ops.nu * T.T @ (W[:, None] * Tp) + 0.5 * Q.T @ Tp + 0.5 * T.T @ Qp)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ne * n3, ne * n3))
    return A.asformat(fmt)


# ------------------------------------------------------------------ brute force
def _invert_map(corners, x, guess=(0.0, 0.0, 0.0)):
    xi = np.array(guess, dtype=np.float64)
    for _ in range(60):
        xx, J = map_and_jacobian(corners, xi[0], xi[1], xi[2])
        dx = np.linalg.solve(J, x - xx)
        xi += dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    return xi


def _basis_at(p, corners, xi):
    """Values [n3] and physical gradients [n3, 3] of the 3D nodal basis at xi."""
    nodes, _ = gll(p)
    L = [lagrange_eval(nodes, xi[d])[0] for d in range(3)]
    dL = [lagrange_deriv_eval(nodes, xi[d])[0] for d in range(3)]
    val = np.einsum("k,j,i->kji", L[2], L[1], L[0]).reshape(-1)
    g1 = np.einsum("k,j,i->kji", L[2], L[1], dL[0]).reshape(-1)
    g2 = np.einsum("k,j,i->kji", L[2], dL[1], L[0]).reshape(-1)
    g3 = np.einsum("k,j,i->kji", dL[2], L[1], L[0]).reshape(-1)
    _, J = map_and_jacobian(corners, xi[0], xi[1], xi[2])
    Jinv = np.linalg.inv(J)  # [b, a] = dxi_b / dx_a
    gref = np.stack([g1, g2, g3], axis=1)  # [n3, b]
    return val, gref @ Jinv


def brute_force_matrix(level, mu_star, nu=1.0, kappa=0.0):
    """Dense A with A[i, j] = a(psi_j, psi_i) from Eq. (2), computed point by point."""
    p = level["p"]
    N = p + 1
    n3 = N ** 3
    corners = level["corners"]
    nbr = level["nbr"]
    ne = nbr.shape[0]
    nodes, w = gll(p)
    A = np.zeros((ne * n3, ne * n3))

    # element volumes and face areas from the same physical quadrature
    def face_points(e, f):
        d, side = f // 2, f % 2
        t = [q for q in range(3) if q != d]
        pts = []
        for b in range(N):
            for a in range(N):
                xi = np.zeros(3)
                xi[d] = 1.0 if side else -1.0
                xi[t[0]], xi[t[1]] = nodes[a], nodes[b]
                x, J = map_and_jacobian(corners[e], *xi)
                ta, tb = J[:, t[0]], J[:, t[1]]
                nrm = np.cross(ta, tb)
                dS = np.linalg.norm(nrm)
                n = nrm / dS
                # outward: away from the element centre
                xc, _ = map_and_jacobian(corners[e], 0.0, 0.0, 0.0)
                if np.dot(n, x - xc) < 0:
                    n = -n
                # local extent perpendicular to the face: the height of the
                # image of the reference cell's half-width along n (2 n . dx/dxi_d)
                pts.append((xi.copy(), x, n, w[a] * w[b] * dS, 2.0 * abs(np.dot(n, J[:, d]))))
        return pts

    # penalty length: the smallest local perpendicular extent over the face
    hperp = np.array([[min(q[4] for q in face_points(e, f)) for f in range(6)] for e in range(ne)])
    own = p * (p + 1) / (2.0 * hperp)

    for e in range(ne):
        sl = slice(e * n3, (e + 1) * n3)
        for k in range(N):
            for j in range(N):
                for i in range(N):
                    xi = np.array([nodes[i], nodes[j], nodes[k]])
                    val, grad = _basis_at(p, corners[e], xi)
                    _, J = map_and_jacobian(corners[e], *xi)
                    wq = w[i] * w[j] * w[k] * np.linalg.det(J)
                    A[sl, sl] += wq * (nu * grad @ grad.T + kappa * np.outer(val, val))
        for f in range(6):
            nb = nbr[e, f]
            if nb == -2:
                continue
            if nb >= 0 and nb < e:
                continue  # each interior face once
            mu = mu_star * (0.5 * (own[e, f] + own[nb, f ^ 1]) if nb >= 0 else own[e, f])
            for xi, x, n, wq, _ in face_points(e, f):
                vm, gm = _basis_at(p, corners[e], xi)
                if nb == -1:
                    dn = gm @ n
                    A[sl, sl] += wq * (2.0 * mu * nu * np.outer(vm, vm)
                                       - nu * np.outer(dn, vm) - nu * np.outer(vm, dn))
                    continue
                xi_p = _invert_map(corners[nb], x, guess=-xi)
                vp, gp = _basis_at(p, corners[nb], xi_p)
                idx = np.r_[np.arange(e * n3, (e + 1) * n3), np.arange(nb * n3, (nb + 1) * n3)]
                jmp = np.r_[vm, -vp]                    # [[v]] . n^-
                avg = 0.5 * np.r_[gm @ n, gp @ n]       # {{grad v}} . n^-
                blk = mu * nu * np.outer(jmp, jmp) - nu * np.outer(avg, jmp) - nu * np.outer(jmp, avg)
                A[np.ix_(idx, idx)] += wq * blk
    return A
