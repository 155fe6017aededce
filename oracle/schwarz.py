"""Weighted additive Schwarz smoother with fast diagonalization (Sec. 4.3.1,
Eqs. (9)-(11), Alg. 5), FP64.

Readings of the paper taken here (the paper leaves these open):
* Overlap layers: m = #{GLL nodes xi_j with (1 + xi_j)/2 <= delta}, counted
  from the shared face (the face node always counts).
* 1D surrogate matrices: the 1D SIP matrix on three standard cells [-1,1]
  (penalty mu_star p(p+1)/4, i.e. h_perp = 2) with the central cell's side
  conditions, restricted to the central N nodes plus m nodes of each interior
  neighbour cell; M is the lumped GLL mass.  The far faces of the neighbour
  cells do not reach this block because m < N.
* Surrogate widths: Legendre P1 coefficients a_i = 1/8 sum_c s_i(c) x_c of the
  trilinear map give the parallelepiped; cuboid edges 2|a_i| are scaled by one
  common factor so that the cuboid has the exact volume of the element.
* Weights: the quintic weighting function of the cited earlier work is not
  printed in the paper.  Reading: across each interior side a symmetric
  quintic blend phi(t) = s(clip((delta - t)/(2 delta), 0, 1)),
  s(x) = 6x^5 - 15x^4 + 10x^3, with t the signed normalized distance of the
  node beyond that side (negative inside the own element); factor 1 at
  boundary sides; W = W3 x W2 x W1.  The weights themselves are not printed,
  so entry by entry they are pinned only by the partition of unity
  sum_e R_s^T W^e R_s 1 = 1; as a whole the reading is pinned by the cycle
  counts the paper prints for its uniform Cartesian study, which the CUDA
  path (equal to this module to 1e-12 on the same periodic meshes)
  reproduces exactly for h-multigrid at p = 4
  (tests/test_gpu_paper_cartesian.py).

Pins (tests/test_oracle_schwarz.py): S^T M S = I and S^T L S = Lambda; the FD
inverse equals the dense inverse of the Kronecker surrogate; on uniform
Cartesian meshes R_s A R_s^T equals the surrogate exactly, so one FD solve
equals the dense solve of the true subdomain problem, for interior and boundary
subdomains; partition of unity; the overlap-layer table for delta in
{0.04, 0.08, 0.16} and p in {4, 8, 16}.
"""
import numpy as np

from .gll import gll, diff_matrix

SIDE = {-1: "d", -2: "n"}
VARIANTS = ("ii", "id", "in", "di", "dd", "dn", "ni", "nd", "nn")
# with local refinement a fourth side type appears: "f", an interior face
# whose neighbour is frozen (its values are fixed, so the subdomain takes no
# layers from it; the face's own-side terms stay in the local operator)
SIDES4 = ("i", "d", "n", "f")
VARIANTS16 = tuple(a + b for a in SIDES4 for b in SIDES4)


def overlap_layers(p, delta):
    x, _ = gll(p)
    return int(np.sum((1.0 + x) / 2.0 <= delta + 1e-14))


def side_of(nb, cls=None):
    if nb >= 0:
        return "f" if cls is not None and cls[nb] == 2 else "i"
    return SIDE[int(nb)]


def sip_1d_three_cells(p, mu_star, left, right):
    """1D SIP matrix (Eq. (2) in 1D, reference cells of width 2) on the cells
    (left neighbour, centre, right neighbour).  `left`/`right` in {'i','d','n'}
    are the centre's side conditions; absent cells keep empty rows.
    Returns L [3N, 3N], mass [3N]."""
    N = p + 1
    x, w = gll(p)
    D = diff_matrix(p)
    mu = mu_star * p * (p + 1) / 4.0
    L = np.zeros((3 * N, 3 * N))
    mass = np.zeros(3 * N)
    cells = [0 if left in "if" else None, 1, 2 if right in "if" else None]
    for c in cells:
        if c is None:
            continue
        s = slice(c * N, (c + 1) * N)
        L[s, s] += D.T @ np.diag(w) @ D
        mass[s] = w

    def e(c, i):
        v = np.zeros(3 * N)
        v[c * N + i] = 1.0
        return v

    def dn(c, i, n):  # n * d/dx at node i of cell c (row vector)
        v = np.zeros(3 * N)
        v[c * N:(c + 1) * N] = n * D[i, :]
        return v

    # interior faces: between cells (0,1) and (1,2) when present
    for a, b in ((0, 1), (1, 2)):
        if cells[a] is None or cells[b] is None:
            continue
        T = e(a, N - 1) - e(b, 0)                     # [[v]] . n^a
        Q = 0.5 * (dn(a, N - 1, 1.0) - dn(b, 0, -1.0))  # {{v'}} . n^a
        L += mu * np.outer(T, T) - np.outer(Q, T) - np.outer(T, Q)
    # Dirichlet sides of the centre
    if left == "d":
        T, Q = e(1, 0), dn(1, 0, -1.0)
        L += 2.0 * mu * np.outer(T, T) - np.outer(Q, T) - np.outer(T, Q)
    if right == "d":
        T, Q = e(1, N - 1), dn(1, N - 1, 1.0)
        L += 2.0 * mu * np.outer(T, T) - np.outer(Q, T) - np.outer(T, Q)
    return L, mass


def subdomain_1d(p, m, mu_star, left, right):
    """Selected 1D block (M, L) of the surrogate for one direction."""
    N = p + 1
    L3, mass3 = sip_1d_three_cells(p, mu_star, left, right)
    sel = []
    if left == "i":
        sel += list(range(N - m, N))
    sel += list(range(N, 2 * N))
    if right == "i":
        sel += list(range(2 * N, 2 * N + m))
    sel = np.array(sel)
    return np.diag(mass3[sel]), L3[np.ix_(sel, sel)]


def fd_eigen(M, L):
    """Generalized eigenpairs L s = lambda M s with S^T M S = I, S^T L S = Lambda."""
    d = np.sqrt(np.diag(M))
    C = L / d[:, None] / d[None, :]
    lam, Q = np.linalg.eigh(0.5 * (C + C.T))
    S = Q / d[:, None]
    return S, lam


def quintic(x):
    return x * x * x * (10.0 - 15.0 * x + 6.0 * x * x)


def weights_1d(p, m, delta, left, right):
    """Weight vector over the subdomain nodes of one direction (reading above)."""
    x, _ = gll(p)
    pos = []  # (distance beyond left face, distance beyond right face), normalized
    if left == "i":
        for j in range(p + 1 - m, p + 1):          # left neighbour's last m nodes
            pos.append(((1.0 - x[j]) / 2.0, -1.0 - (1.0 - x[j]) / 2.0))
    for i in range(p + 1):
        pos.append((-(1.0 + x[i]) / 2.0, -(1.0 - x[i]) / 2.0))
    if right == "i":
        for j in range(m):                          # right neighbour's first m nodes
            pos.append((-1.0 - (1.0 + x[j]) / 2.0, (1.0 + x[j]) / 2.0))

    def phi(t):
        return quintic(np.clip((delta - t) / (2.0 * delta), 0.0, 1.0))

    w = []
    for tl, tr in pos:
        fl = phi(tl) if left == "i" else 1.0
        fr = phi(tr) if right == "i" else 1.0
        w.append(fl * fr)
    return np.array(w)


class FDTables:
    """S, Lambda, W for the nine side variants of one (p, m, mu_star, delta)."""

    def __init__(self, p, delta, mu_star):
        self.p, self.delta, self.mu_star = p, delta, mu_star
        self.m = overlap_layers(p, delta)
        self.tab = {}
        for v in VARIANTS16:
            M, L = subdomain_1d(p, self.m, mu_star, v[0], v[1])
            S, lam = fd_eigen(M, L)
            W = weights_1d(p, self.m, delta, v[0], v[1])
            self.tab[v] = dict(M=M, L=L, S=S, lam=lam, W=W)


def element_volume_exact(corners):
    """Exact volume of a trilinear element (2-point Gauss per direction; det J has
    degree <= 2 in each reference coordinate)."""
    from .geometry import map_and_jacobian
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    vol = 0.0
    for a in g:
        for b in g:
            for c in g:
                _, J = map_and_jacobian(corners, a, b, c)
                vol += np.linalg.det(J)
    return vol


def surrogate_widths(corners):
    """Cuboid widths Delta x_i of the Cartesian surrogate (Sec. 4.3.1, four steps)."""
    a = np.zeros((3, 3))
    for c in range(8):
        for i in range(3):
            s = 1.0 if (c >> i) & 1 else -1.0
            a[i] += s * corners[c] / 8.0
    ell = 2.0 * np.linalg.norm(a, axis=1)
    vol = element_volume_exact(corners)
    return ell * (vol / np.prod(ell)) ** (1.0 / 3.0)


def surrogate_coeffs(dx, nu=1.0, kappa=0.0):
    """g0..g3 of Eq. (10)."""
    g0 = kappa * dx[0] * dx[1] * dx[2] / 8.0
    g = [nu * dx[(i + 1) % 3] * dx[(i + 2) % 3] / (2.0 * dx[i]) for i in range(3)]
    return np.array([g0] + g)


class Schwarz:
    """Subdomain restriction, FD solve and weighted combination on one level."""

    def __init__(self, level, delta, mu_star, nu=1.0, kappa=0.0, gcoef=None):
        self.level = level
        self.p = level["p"]
        self.N = self.p + 1
        self.tables = FDTables(self.p, delta, mu_star)
        self.m = self.tables.m
        nbr = level["nbr"]
        self.ne = nbr.shape[0]
        cls = level["cls"]
        self.var = [[side_of(nbr[e, 2 * d], cls) + side_of(nbr[e, 2 * d + 1], cls)
                     for d in range(3)] for e in range(self.ne)]
        if gcoef is None:
            gcoef = np.array([surrogate_coeffs(surrogate_widths(level["corners"][e]), nu, kappa)
                              for e in range(self.ne)])
        self.g = gcoef
        self.active = level["cls"] != 2

    def index_1d(self, v):
        """(offset, local node) of each subdomain node in one direction."""
        N, m = self.N, self.m
        out = []
        if v[0] == "i":
            out += [(-1, i) for i in range(N - m, N)]
        out += [(0, i) for i in range(N)]
        if v[1] == "i":
            out += [(1, i) for i in range(m)]
        return out

    def restriction(self, e):
        """Global flat indices (or -1 = zero fill) of the subdomain nodes,
        array [n3, n2, n1] (direction 1 fastest)."""
        N = self.N
        ix = [self.index_1d(self.var[e][d]) for d in range(3)]
        out = np.full((len(ix[2]), len(ix[1]), len(ix[0])), -1, dtype=np.int64)
        nb27 = self.level["nbr27"][e]
        for c, (oz, k) in enumerate(ix[2]):
            for b, (oy, j) in enumerate(ix[1]):
                for a, (ox, i) in enumerate(ix[0]):
                    n = nb27[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)]
                    if n >= 0:
                        out[c, b, a] = ((n * N + k) * N + j) * N + i
        return out

    def surrogate_matrix(self, e):
        """Dense A~ of Eq. (10) for element e."""
        T = [self.tables.tab[self.var[e][d]] for d in range(3)]
        g = self.g[e]
        M1, M2, M3 = (T[d]["M"] for d in range(3))
        L1, L2, L3 = (T[d]["L"] for d in range(3))
        k = lambda A3, A2, A1: np.kron(A3, np.kron(A2, A1))
        return g[0] * k(M3, M2, M1) + g[1] * k(M3, M2, L1) + g[2] * k(M3, L2, M1) + g[3] * k(L3, M2, M1)

    def fd_solve(self, e, rs):
        """(S3 x S2 x S1) D^-1 (S3^T x S2^T x S1^T) rs, rs [n3, n2, n1]."""
        T = [self.tables.tab[self.var[e][d]] for d in range(3)]
        S1, S2, S3 = T[0]["S"], T[1]["S"], T[2]["S"]
        l1, l2, l3 = T[0]["lam"], T[1]["lam"], T[2]["lam"]
        g = self.g[e]
        y = np.einsum("ai,cba->cbi", S1, rs)
        y = np.einsum("bj,cbi->cji", S2, y)
        y = np.einsum("ck,cji->kji", S3, y)
        Dg = g[0] + g[1] * l1[None, None, :] + g[2] * l2[None, :, None] + g[3] * l3[:, None, None]
        y = y / Dg
        y = np.einsum("ai,kji->kja", S1, y)
        y = np.einsum("bj,kja->kba", S2, y)
        y = np.einsum("ck,kba->cba", S3, y)
        return y

    def weights(self, e):
        T = [self.tables.tab[self.var[e][d]] for d in range(3)]
        return T[2]["W"][:, None, None] * T[1]["W"][None, :, None] * T[0]["W"][None, None, :]

    def correction(self, r):
        """Delta u = sum_e R_s^T W^e A~^-1 R_s r (Eq. (11)); frozen rows of r are
        taken as zero and frozen entries of the result are not updated."""
        r = np.asarray(r, dtype=np.float64).reshape(-1)
        N3 = self.N ** 3
        rz = r.copy().reshape(self.ne, N3)
        rz[~self.active] = 0.0
        rz = rz.reshape(-1)
        du = np.zeros_like(rz)
        for e in range(self.ne):
            if not self.active[e]:
                continue
            idx = self.restriction(e)
            rs = np.where(idx >= 0, rz[np.maximum(idx, 0)], 0.0)
            ys = self.weights(e) * self.fd_solve(e, rs)
            ok = idx >= 0
            np.add.at(du, idx[ok], ys[ok])
        du = du.reshape(self.ne, N3)
        du[~self.active] = 0.0
        return du.reshape(-1)
