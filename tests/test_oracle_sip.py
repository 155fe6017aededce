"""Oracle pins for the SIP operator (Sec. 2.2, Eq. (2))."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2608_14123_b300 import workloads as wl
from oracle import sip
from oracle.gll import gll


def _level(kind, n, p, seed=1):
    if kind == "cart":
        V = wl.uniform_vertices(n)
    elif kind == "box":
        V = wl.uniform_vertices(n, hi=(1.0, 0.5, 2.0))
    else:
        V = wl.perturbed_vertices(n, 0.2, np.random.default_rng(seed))
    return wl.level_from_vertices(V, p)


@pytest.mark.parametrize("kind", ["cart", "box", "pert"])
@pytest.mark.parametrize("p", [1, 2])
def test_brute_force_equals_assembly(kind, p):
    lev = _level(kind, 2, p)
    ops = sip.LevelOps(lev, 2.0)
    A = sip.assemble(ops).toarray()
    B = sip.brute_force_matrix(lev, 2.0)
    assert np.abs(A - B).max() <= 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("kind", ["cart", "pert"])
@pytest.mark.parametrize("p", [1, 3])
def test_apply_equals_assembly_symmetric_spd(kind, p):
    lev = _level(kind, 3, p)
    ops = sip.LevelOps(lev, 5.0)
    A = sip.assemble(ops).toarray()
    u = np.random.default_rng(0).standard_normal(ops.ndof)
    Au = sip.apply(ops, u).reshape(-1)
    assert np.abs(A @ u - Au).max() <= 1e-13 * np.abs(Au).max()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A)[0] > 0


def test_kappa_mass_term():
    lev = _level("pert", 2, 2)
    ops0 = sip.LevelOps(lev, 5.0, kappa=0.0)
    ops1 = sip.LevelOps(lev, 5.0, kappa=3.0)
    u = np.random.default_rng(2).standard_normal(ops0.ndof)
    d = sip.apply(ops1, u) - sip.apply(ops0, u)
    np.testing.assert_allclose(d, 3.0 * ops0.mass * u.reshape(d.shape), rtol=1e-12, atol=1e-14)


def test_neumann_constants_in_kernel():
    V = wl.perturbed_vertices(3, 0.2, np.random.default_rng(3))
    lev = wl.level_from_vertices(V, 2, boundary=-2)
    ops = sip.LevelOps(lev, 5.0)
    r = sip.apply(ops, np.ones(ops.ndof))
    assert np.abs(r).max() < 1e-12


def _sip_1d_global(n, p, h, mu_star):
    """Global 1D SIP matrix on n equal cells of width h with Dirichlet ends,
    written out from the 1D form of Eq. (2) independently of the 3D code."""
    from oracle.gll import diff_matrix
    x, w = gll(p)
    N = p + 1
    D = diff_matrix(p) * 2.0 / h
    wq = w * h / 2.0
    mu = mu_star * p * (p + 1) / (2.0 * h)
    L = np.zeros((n * N, n * N))
    for c in range(n):
        s = slice(c * N, (c + 1) * N)
        L[s, s] += D.T @ np.diag(wq) @ D
    for c in range(n + 1):
        T = np.zeros(n * N)
        Q = np.zeros(n * N)
        if 0 < c < n:   # interior face between cell c-1 and c
            T[(c - 1) * N + N - 1], T[c * N] = 1.0, -1.0
            Q[(c - 1) * N:c * N] += 0.5 * D[N - 1]
            Q[c * N:(c + 1) * N] += 0.5 * D[0]
            L += mu * np.outer(T, T) - np.outer(Q, T) - np.outer(T, Q)
        else:           # Dirichlet end
            i = 0 if c == 0 else n * N - 1
            nrm = -1.0 if c == 0 else 1.0
            T[i] = 1.0
            cc = 0 if c == 0 else n - 1
            Q[cc * N:(cc + 1) * N] = nrm * (D[0] if c == 0 else D[N - 1])
            L += 2.0 * mu * np.outer(T, T) - np.outer(Q, T) - np.outer(T, Q)
    M = np.diag(np.tile(wq, n))
    return L, M


@pytest.mark.parametrize("p", [1, 2, 4])
def test_uniform_cartesian_is_kronecker_sum(p):
    n = 3
    lev = _level("cart", n, p)
    ops = sip.LevelOps(lev, 2.0)
    A = sip.assemble(ops).toarray()
    L, M = _sip_1d_global(n, p, 1.0 / n, 2.0)
    # global (x,y,z) ordering -> element-major ordering of the 3D code
    N = p + 1
    g = np.arange(n * N)
    perm = []
    for ez in range(n):
        for ey in range(n):
            for ex in range(n):
                for k in range(N):
                    for j in range(N):
                        for i in range(N):
                            perm.append(((ez * N + k) * n * N + ey * N + j) * n * N + ex * N + i)
    perm = np.array(perm)
    K = lambda a, b, c: np.kron(a, np.kron(b, c))
    Ak = K(M, M, L) + K(M, L, M) + K(L, M, M)
    Ak = Ak[np.ix_(perm, perm)]
    assert np.abs(A - Ak).max() <= 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("p", [2, 3])
def test_discrete_consistency_polynomial(p):
    """A I(u) = b(f = -lap u, u_D = u) exactly for u in Q_p on affine boxes."""
    V = wl.uniform_vertices(2, hi=(1.0, 0.7, 1.3))
    lev = wl.level_from_vertices(V, p)
    ops = sip.LevelOps(lev, 3.0)
    X = ops.geo["x"]
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    u = x ** p * y ** (p - 1) + z ** p * x + y * z
    lap = (p * (p - 1) * x ** (p - 2) * y ** (p - 1) + x ** p * (p - 1) * (p - 2) * y ** max(p - 3, 0)
           + p * (p - 1) * z ** (p - 2) * x)
    b = sip.rhs(ops, -lap, u)
    Au = sip.apply(ops, u)
    assert np.abs(Au - b).max() <= 1e-11 * np.abs(b).max()


def test_convergence_order_p_plus_1():
    spec = wl.sine_rhs_spec()
    for p in (1, 2):
        errs = []
        for n in (2, 4, 8):
            lev = wl.level_from_vertices(wl.uniform_vertices(n), p)
            ops = sip.LevelOps(lev, 2.0)
            A = sip.assemble(ops).tocsc()
            X = ops.geo["x"]
            b = sip.rhs(ops, wl.eval_f(spec, X), np.zeros(X.shape[:-1])).reshape(-1)
            u = spla.spsolve(A, b)
            e = u - wl.eval_u(spec, X).reshape(-1)
            errs.append(np.sqrt(np.sum(ops.mass.reshape(-1) * e * e)))
        rate = np.log2(errs[1] / errs[2])
        assert rate > p + 1 - 0.3, (p, errs, rate)
