"""Best-fit Kronecker-sum surrogates of the element operator and the training
data of the learned surrogate (FP64).

The tensor-product surrogate of Eq. (10) has, for kappa = 0, three free
coefficients g_1..g_3 per element.  The geometric surrogate (Sec. 4.3.1) takes
them from the cuboid widths; here they are fitted to the element's own
operator instead:

* Target A^ee: the element block of Eq. (2) with the element's geometry
  (volume term plus the own-side face terms; an interior face uses the
  penalty of a congruent neighbour, mu = mu_star p(p+1)/(2 h_perp_own); a
  Dirichlet face the 2 mu of Eq. (2); a Neumann face nothing).
* Basis K_i: the Kronecker products M x M x L_i with L_i the central N x N
  block of the 1D three-cell SIP matrix of the element's side variant in
  direction i (the same matrices the fast-diagonalization tables use).
* Fit: minimise || M^-1/2 (A^ee - sum_i g_i K_i) M^-1/2 ||_F (3x3 normal
  equations), M = W x W x W.  Only the direction-i line entries of A^ee meet
  K_i, so `line_entries` evaluates them in closed form from the metric and
  face factors instead of forming the dense block.

MLP training pairs (reading of the learned surrogate; the paper has no
learned part): inputs are the 24 corner coordinates minus the centroid,
divided by V^(1/3); targets are (log(dx_i^geo / V^(1/3)), log(g_i^fit /
g_i^geo)) for i = 1..3.

Pins (tests/test_oracle_surrogate.py): line entries equal the dense element
block; on axis-aligned boxes the fit reproduces the geometric surrogate
exactly; the normal-equation solution equals lstsq on the dense vectorised
matrices; the fit is invariant under translation and scales like h.
"""
import numpy as np

from .gll import gll, diff_matrix
from .geometry import node_geometry, volume_metric, face_factors, h_perp
from .schwarz import sip_1d_three_cells, surrogate_widths, surrogate_coeffs, side_of


def _sym(G, a, b):
    return G[..., a, b]


def line_entries(G, c, W, mu, D, w, sides, d):
    """Direction-d line entries E[e, k, j, i, i'] of A^ee in the node order
    rotated so that direction d is the fastest index.

    G [e,k,j,i,3,3] volume metric, c [e,6,b,a,3] and W [e,6,b,a] face factors,
    mu [e,6] penalties, sides [e,6] in {'i','d','n'}."""
    # rotate the node axes and the metric components so that d becomes axis x
    perm = {0: (0, 1, 2), 1: (1, 0, 2), 2: (2, 1, 0)}[d]   # new (x,y,z) <- old dirs
    ax = {0: (1, 2, 3), 1: (1, 3, 2), 2: (3, 2, 1)}[d]      # node axes (k,j,i) order
    Gr = np.transpose(G, (0,) + ax + (4, 5))
    Gr = Gr[..., list(perm), :][..., :, list(perm)]
    ne, N = G.shape[0], G.shape[1]
    E = np.zeros((ne, N, N, N, N))
    # volume (derivation: B_1 = I x I x D etc. restricted to equal (k, j))
    E += np.einsum("li,ekjl,lm->ekjim", D, Gr[..., 0, 0], D)
    dd = np.diag(D)
    diag = (np.einsum("lj,ekli->ekji", D * D, Gr[..., 1, 1])
            + np.einsum("lk,elji->ekji", D * D, Gr[..., 2, 2])
            + 2.0 * dd[None, None, :, None] * dd[None, :, None, None] * Gr[..., 1, 2])
    idx = np.arange(N)
    E[:, :, :, idx, idx] += diag
    # cross terms x-y and x-z: D[i',i] D_jj G12(k,j,i') + D_jj G12(k,j,i) D[i,i']
    for t, dj in ((1, dd[None, None, :, None]), (2, dd[None, :, None, None])):
        Gt = Gr[..., 0, t] * dj                     # [e,k,j,i]
        E += np.einsum("mi,ekjm->ekjim", D, Gt)     # D[i',i] Gt(k,j,i')
        E += np.einsum("ekji,im->ekjim", Gt, D)     # Gt(k,j,i) D[i,i']
    # faces: rotate face indices the same way
    fmap = {0: [0, 1, 2, 3, 4, 5], 1: [2, 3, 0, 1, 4, 5], 2: [4, 5, 2, 3, 0, 1]}[d]
    for fn in range(6):           # face in the rotated frame
        fo = fmap[fn]             # original face index
        dn, side = fn // 2, fn % 2
        end = N - 1 if side else 0
        cf, Wf, muf = c[:, fo], W[:, fo], mu[:, fo]
        sd = sides[:, fo]
        scale_pen = np.where(sd == "d", 2.0, np.where(sd == "i", 1.0, 0.0))
        scale_flux = np.where(sd == "d", 1.0, np.where(sd == "i", 0.5, 0.0))
        # the face arrays [e, b, a] are in the original face-local order; map
        # to the rotated node axes (k, j, i)
        cr = _face_to_rotated(cf, d, fo, N)          # [e, ., ., 3] in original t order
        Wr = _face_to_rotated(Wf[..., None], d, fo, N)[..., 0]
        cr = cr[..., list(perm)]                     # t components in rotated order
        if dn == 0:   # face i = end: nodes (k, j, end), face-local (k, j)
            E[:, :, :, end, end] += (scale_pen * muf)[:, None, None] * Wr
            q1 = cr[..., 0]                          # [e, k, j]
            cjk = cr[..., 1] * dd[None, None, :] + cr[..., 2] * dd[None, :, None]
            # Q^T T: row (k,j,i), col (k,j,end): c1 D[end][i] + (c2 D_jj + c3 D_kk) d_i,end
            QT = np.einsum("ekj,i->ekji", q1, D[end])
            QT[:, :, :, end] += cjk
            s = scale_flux[:, None, None, None]
            E[:, :, :, :, end] -= s * QT
            E[:, :, :, end, :] -= s * QT
        else:
            # faces with normal y or z: face nodes (k, end, i) / (end, j, i);
            # the x-line couplings: diagonal penalty + c1 D[i'][i] + diagonal
            q = cr                                     # [e, k, i, 3] or [e, j, i, 3]
            Wq = Wr
            if dn == 1:
                kk = slice(None)
                sel = (slice(None), slice(None), end)      # E[:, k, end, i, i']
                dn_d = dd[end]
                other = dd[None, :, None] * q[..., 2]      # c3 D_kk  [e,k,i]
            else:
                sel = (slice(None), end, slice(None))      # E[:, end, j, i, i']
                dn_d = dd[end]
                other = dd[None, :, None] * q[..., 1]      # c2 D_jj  [e,j,i]
            Ef = E[sel]                                    # [e, X, i, i'] view
            s = scale_flux[:, None, None]
            pen = (scale_pen * muf)[:, None, None] * Wq     # [e, X, i]
            Ef[:, :, idx, idx] += pen
            # Q^T T entry (X, i),(X, i'): c1(X,i') D[i'][i] + (c_n D_end,end + other) d_ii'
            QT = np.einsum("exm,mi->exim", q[..., 0], D)   # [e,X,i,i'] = c1(X,i') D[i'][i]
            QT[:, :, idx, idx] += (q[..., dn] * dn_d + other)
            Ef -= s[..., None] * QT
            Ef -= s[..., None] * np.swapaxes(QT, 2, 3)
            E[sel] = Ef
    return E


def _face_to_rotated(arr, d, fo, N):
    """Face array [e, b, a, X] (original face-local order of face fo) to the
    rotated frame's face-local order (the two tangential rotated axes, slower
    first)."""
    # original face-local axes (b, a) = tangential directions in increasing
    # order, slower first: face dir 0 -> (z, y), 1 -> (z, x), 2 -> (y, x)
    fd = fo // 2
    orig = {0: (2, 1), 1: (2, 0), 2: (1, 0)}[fd]
    # rotated frame: perm maps new axis -> old dir
    perm = {0: (0, 1, 2), 1: (1, 0, 2), 2: (2, 1, 0)}[d]
    inv = {old: new for new, old in enumerate(perm)}
    new_dirs = (inv[orig[0]], inv[orig[1]])       # tangential dirs in the rotated frame
    # rotated face-local order: slower = larger rotated axis index
    if new_dirs[0] > new_dirs[1]:
        return arr
    return np.swapaxes(arr, 1, 2)


def central_blocks(p, mu_star, sides_e):
    """Central N x N blocks of the 1D three-cell SIP matrices per direction."""
    N = p + 1
    out = []
    for d in range(3):
        L3, _ = sip_1d_three_cells(p, mu_star, sides_e[2 * d], sides_e[2 * d + 1])
        out.append(L3[N:2 * N, N:2 * N])
    return out


def fit_coefficients(level, mu_star, nu=1.0):
    """g_1..g_3 of the best-fit Kronecker sum for every element of `level`
    (kappa = 0), and the geometric ones, as arrays [ne, 3]."""
    p = level["p"]
    N = p + 1
    geo = node_geometry(level["corners"], p)
    G = volume_metric(geo, nu)
    W, c = face_factors(geo, nu)
    hp = h_perp(geo, W)
    mu = mu_star * p * (p + 1) / (2.0 * hp)   # congruent neighbour: own h_perp only
    W = W * nu
    D = diff_matrix(p)
    _, w = gll(p)
    nbr = level["nbr"]
    ne = nbr.shape[0]
    sides = np.array([[side_of(nbr[e, f]) for f in range(6)] for e in range(ne)])
    Es = [line_entries(G, c, W, mu, D, w, sides, d) for d in range(3)]
    inv = 1.0 / w
    g_fit = np.zeros((ne, 3))
    g_geo = np.zeros((ne, 3))
    for e in range(ne):
        Lc = central_blocks(p, mu_star, sides[e])
        # scaled Gram matrix and right-hand side
        wk = inv[:, None, None, None] * inv[None, :, None, None]
        Gm = np.zeros((3, 3))
        rhs = np.zeros(3)
        for a in range(3):
            La = Lc[a] * inv[:, None] * inv[None, :]
            rhs[a] = np.sum(Es[a][e] * wk * La[None, None])
            for b in range(3):
                Gm[a, b] = _gram(Lc, w, a, b)
        g_fit[e] = np.linalg.solve(Gm, rhs)
        g_geo[e] = surrogate_coeffs(surrogate_widths(level["corners"][e]), nu)[1:]
    return g_fit, g_geo


def _gram(Lc, w, a, b):
    """< M x M x L_a , M x M x L_b >_scaled (directions a, b) in closed form."""
    N = len(w)
    La = Lc[a] / np.sqrt(w)[:, None] / np.sqrt(w)[None, :]
    Lb = Lc[b] / np.sqrt(w)[:, None] / np.sqrt(w)[None, :]
    if a == b:
        return N * N * np.sum(La * La)
    # only diagonal entries overlap
    return N * np.sum(np.diag(La)) * np.sum(np.diag(Lb))


def mlp_inputs(corners):
    """24 normalized corner coordinates per element: (x_c - centroid) / V^(1/3)."""
    cen = corners.mean(axis=1, keepdims=True)
    vol = np.array([_vol(cr) for cr in corners])
    return ((corners - cen) / np.cbrt(vol)[:, None, None]).reshape(len(corners), 24)


def _vol(cr):
    from .schwarz import element_volume_exact
    return element_volume_exact(cr)


def mlp_targets(corners, g_fit, nu=1.0):
    dx = np.array([surrogate_widths(cr) for cr in corners])
    vol = np.array([_vol(cr) for cr in corners])
    g_geo = np.array([surrogate_coeffs(x, nu)[1:] for x in dx])
    return np.concatenate([np.log(dx / np.cbrt(vol)[:, None]), np.log(g_fit / g_geo)], axis=1)


def coeffs_from_outputs(y, vol, nu=1.0):
    """g_1..g_3 from MLP outputs (log widths over V^(1/3), log scalings)."""
    dx = np.exp(y[:, :3]) * np.cbrt(vol)[:, None]
    s = np.exp(y[:, 3:])
    g = np.stack([nu * dx[:, (i + 1) % 3] * dx[:, (i + 2) % 3] / (2.0 * dx[:, i]) for i in range(3)], 1)
    return s * g


def training_elements(n, rng, ar_max=16.0, amp=0.25):
    """Single interior elements of the curvilinear workloads' distribution
    (the seeded input generator shared with the CUDA path)."""
    from paper_2608_14123_b300.workloads import surrogate_training_corners
    return surrogate_training_corners(n, rng, ar_max, amp)


def element_block_dense(level, e, mu_star, nu=1.0):
    """Dense A^ee of element e (definition above), by the element-block
    assembly of the SIP operator: volume B_d^T G_df B_f plus the own-side face
    blocks.  Small p only (used to pin `line_entries`)."""
    from .sip import _kron3
    from .geometry import face_node_index
    p = level["p"]
    N = p + 1
    n3 = N ** 3
    corners = level["corners"][e:e + 1]
    geo = node_geometry(corners, p)
    G = volume_metric(geo, nu)[0].reshape(n3, 3, 3)
    W, c = face_factors(geo, nu)
    hp = h_perp(geo, W)[0]
    W = W[0] * nu
    c = c[0]
    D = diff_matrix(p)
    I_ = np.eye(N)
    B = [_kron3(I_, I_, D), _kron3(I_, D, I_), _kron3(D, I_, I_)]
    A = np.zeros((n3, n3))
    for a in range(3):
        for b in range(3):
            A += B[a].T @ (G[:, a, b][:, None] * B[b])
    for f in range(6):
        sd = side_of(level["nbr"][e, f])
        if sd == "n":
            continue
        K, J, I = face_node_index(N, f)
        T = np.zeros((N * N, n3))
        T[np.arange(N * N), (K * N * N + J * N + I).reshape(-1)] = 1.0
        Q = sum(c[f, :, :, t].reshape(-1)[:, None] * (T @ B[t]) for t in range(3))
        mu = mu_star * p * (p + 1) / (2.0 * hp[f])
        Wf = W[f].reshape(-1)
        if sd == "d":
            A += 2.0 * mu * T.T @ (Wf[:, None] * T) - Q.T @ T - T.T @ Q
        else:
            A += mu * T.T @ (Wf[:, None] * T) - 0.5 * Q.T @ T - 0.5 * T.T @ Q
    return A
