"""Element geometry for the SIP form (Sec. 2.2).

Each element is the image of the standard element [-1,1]^3 under the trilinear
map x(xi) = sum_c N_c(xi) x_c through its 8 corners (c = cx + 2cy + 4cz,
N_c = prod_d (1 + s_cd xi_d)/2, s = -1 for bit 0 and +1 for bit 1).  The
Jacobian is evaluated analytically from that formula at the GLL nodes.

Conventions (node arrays are [..., k, j, i], i fastest; xi_1 <-> i):
  jac[e,k,j,i,a,b]  = d x_a / d xi_b
  ginv[e,k,j,i,b,a] = d xi_b / d x_a
  detJ[e,k,j,i]
Faces f = 0..5 are (-xi1, +xi1, -xi2, +xi2, -xi3, +xi3).

Pins (tests/test_oracle_sip.py): on axis-aligned boxes all factors reduce to the
closed forms of a box of widths (dx,dy,dz); outward normals computed here from
grad(xi_d) agree with the cross product of the face tangents; volumes and face
areas sum to the exact values of polyhedra with planar faces.
"""
import numpy as np

from .gll import gll


def _sgn(c, d):
    return 1.0 if (c >> d) & 1 else -1.0


def map_and_jacobian(corners, xi1, xi2, xi3):
    """Trilinear map and Jacobian at points (xi1, xi2, xi3) (broadcast arrays).

    corners [8, 3].  Returns x [..., 3] and jac [..., 3, 3] (jac[a, b] = dx_a/dxi_b).
    """
    xi = np.broadcast_arrays(np.asarray(xi1, float), np.asarray(xi2, float), np.asarray(xi3, float))
    shape = xi[0].shape
    x = np.zeros(shape + (3,))
    jac = np.zeros(shape + (3, 3))
    for c in range(8):
        s = [_sgn(c, d) for d in range(3)]
        f = [(1.0 + s[d] * xi[d]) / 2.0 for d in range(3)]
        Nc = f[0] * f[1] * f[2]
        dN = [s[0] / 2.0 * f[1] * f[2], f[0] * s[1] / 2.0 * f[2], f[0] * f[1] * s[2] / 2.0]
        for a in range(3):
            x[..., a] += Nc * corners[c, a]
            for b in range(3):
                jac[..., a, b] += dN[b] * corners[c, a]
    return x, jac


def node_geometry(corners_all, p):
    """Node coordinates, Jacobians, det J and inverse Jacobians at the GLL nodes.

    corners_all [ne, 8, 3] -> dict of arrays with node axes [k, j, i].
    """
    xi, w = gll(p)
    X3, X2, X1 = np.meshgrid(xi, xi, xi, indexing="ij")  # [k, j, i]
    ne = corners_all.shape[0]
    N = p + 1
    X = np.zeros((ne, N, N, N, 3))
    jac = np.zeros((ne, N, N, N, 3, 3))
    for e in range(ne):
        X[e], jac[e] = map_and_jacobian(corners_all[e], X1, X2, X3)
    detJ = np.linalg.det(jac)
    ginv = np.linalg.inv(jac)  # [.., b, a] = dxi_b/dx_a
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return dict(x=X, jac=jac, detJ=detJ, ginv=ginv, w=w, xi=xi, W3=W3)


def volume_metric(geo, nu=1.0):
    """G[e,k,j,i,d,f] = nu * w_ijk * detJ * grad(xi_d) . grad(xi_f), the factor of
    the volume stiffness term  int nu grad v . grad u  under GLL collocation."""
    gi = geo["ginv"]
    G = np.einsum("...da,...fa->...df", gi, gi)
    return nu * (geo["W3"] * geo["detJ"])[..., None, None] * G


def face_node_index(N, f):
    """(k, j, i) index arrays [N, N] of the face-f nodes, face-local axes (b, a)
    where (a, b) are the two tangential directions in increasing order."""
    d, side = f // 2, f % 2
    end = N - 1 if side else 0
    B, A = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    if d == 0:
        return B, A, np.full_like(A, end)          # k=b, j=a, i=end
    if d == 1:
        return B, np.full_like(A, end), A          # k=b, j=end, i=a
    return np.full_like(A, end), B, A              # k=end, j=b, i=a


def face_factors(geo, nu=1.0):
    """Per element, per face, per face node (axes [e, f, b, a]):
      W    surface quadrature weight  w_a w_b detJ |grad xi_d|   (Nanson)
      c[.., t] = W * n . grad(xi_t) * nu, with n the outward unit normal
               = s * nu * w_a w_b detJ grad(xi_d) . grad(xi_t)
    so that  nu * n . grad u = sum_t c_t du/dxi_t / W  at the face node.
    """
    ginv, detJ, w = geo["ginv"], geo["detJ"], geo["w"]
    ne, N = detJ.shape[0], detJ.shape[1]
    W = np.zeros((ne, 6, N, N))
    c = np.zeros((ne, 6, N, N, 3))
    wab = w[:, None] * w[None, :]  # [b, a]
    for f in range(6):
        d, s = f // 2, (1.0 if f % 2 else -1.0)
        K, J, I = face_node_index(N, f)
        gd = ginv[:, K, J, I, d, :]         # grad xi_d  [ne, N, N, 3]
        dj = detJ[:, K, J, I]
        W[:, f] = wab * dj * np.linalg.norm(gd, axis=-1)
        for t in range(3):
            gt = ginv[:, K, J, I, t, :]
            c[:, f, :, :, t] = s * nu * wab * dj * np.sum(gd * gt, axis=-1)
    return W, c


def h_perp(geo, W):
    """Element extent normal to each face (Sec. 2.2, "the element extension
    perpendicular to the interface"), reading for curved elements: the
    smallest local extent over the face's GLL nodes, 2 / |grad xi_d| (the
    reference width 2 over the rate of change of the face-normal reference
    coordinate), exactly h on a cube.  This is the quantity the discrete
    trace bound needs node by node: at a face node the face quadrature weight
    over the volume weight of the same node is |grad xi_d| / w_end, so a
    penalty built from the face's mean extent |Omega| / |face| leaves faces
    next to a nearly folded corner uncontrolled (indefinite operator)."""
    N = geo["detJ"].shape[1]
    out = np.zeros((geo["detJ"].shape[0], 6))
    for f in range(6):
        d = f // 2
        K, J, I = face_node_index(N, f)
        gd = geo["ginv"][:, K, J, I, d, :]
        out[:, f] = np.min(2.0 / np.linalg.norm(gd, axis=-1), axis=(1, 2))
    return out


def penalties(level, geo_h, mu_star):
    """Face penalty mu per element face (Sec. 2.2):
    interior: mu = mu_star * avg(p(p+1)/(2 h_perp)) of both sides,
    boundary: mu = mu_star * p(p+1)/(2 h_perp) of the own side (the Dirichlet
    term of Eq. (2) multiplies it by 2)."""
    p = level["p"]
    hp = geo_h
    nbr = level["nbr"]
    ne = nbr.shape[0]
    own = p * (p + 1) / (2.0 * hp)
    mu = np.zeros((ne, 6))
    for e in range(ne):
        for f in range(6):
            n = nbr[e, f]
            if n >= 0:
                mu[e, f] = mu_star * 0.5 * (own[e, f] + own[n, f ^ 1])
            else:
                mu[e, f] = mu_star * own[e, f]
    return mu
