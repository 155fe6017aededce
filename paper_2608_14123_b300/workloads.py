"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds mesh *topology and coordinates* and the manufactured
right-hand-side functions only.  It contains none of the method's arithmetic
(no basis, quadrature, operator, smoother or transfer): both the oracle and the
CUDA library derive every discrete quantity from these inputs on their own.

Meshes are multilevel hexahedral meshes in the sense of Sec. 3.1: a list of
levels from the root (index 0) to the top, each level a conforming hex mesh
with one polynomial degree.  Consecutive levels are related either by
p-refinement (same elements, higher degree) or by regular h-refinement (each
element split into 8 children).

Per level (all numpy arrays, element index e in lexicographic x-fastest order):
  p        polynomial degree of the level
  corners  float64 [ne, 8, 3]   corner c = cx + 2*cy + 4*cz of the trilinear map
  nbr      int32   [ne, 6]      face f in (-x,+x,-y,+y,-z,+z): neighbour element,
                                or -1 = Dirichlet boundary, -2 = Neumann boundary
  nbr27    int32   [ne, 27]     element at offset (ox,oy,oz) in {-1,0,1}^3,
                                slot (ox+1) + 3*(oy+1) + 9*(oz+1); -1 = none
  parent   int32   [ne]         element of the next coarser level (-1 on the root)
  octant   int32   [ne]         child octant cx+2cy+4cz for h-refinement, -1 for
                                p-refinement (parent is the same element)
  cls      int8    [ne]         0 = leaf, 1 = twig, 2 = frozen (Sec. 3.1)
All neighbouring elements share aligned local axes (structured topology).
"""
import numpy as np

SEED_BASE = 20261202
# smallest corner-Jacobian ratio of a cell of the graded, strongly perturbed
# workload (the worst cell of the +-0.15h uniform workload has 0.21)
MIN_JACOBIAN_RATIO = 0.2

LEAF, TWIG, FROZEN = 0, 1, 2

_FACE_OFF = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def uniform_vertices(nx, ny=None, nz=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Vertex grid [nx+1, ny+1, nz+1, 3] of an axis-aligned box."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    V = np.zeros((nx + 1, ny + 1, nz + 1, 3))
    V[..., 0] = xs[:, None, None]
    V[..., 1] = ys[None, :, None]
    V[..., 2] = zs[None, None, :]
    return V


def corner_jacobians_positive(V):
    """Input validation: the triple product of the three edges at every corner of
    every cell of the vertex grid is positive (no folded cells)."""
    ok = True
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                sx, sy, sz = 1 - 2 * cx, 1 - 2 * cy, 1 - 2 * cz
                def at(dx, dy, dz):
                    return V[cx + dx: V.shape[0] - 1 + cx + dx,
                             cy + dy: V.shape[1] - 1 + cy + dy,
                             cz + dz: V.shape[2] - 1 + cz + dz]
                o = at(0, 0, 0)
                ex = (at(sx, 0, 0) - o) * sx
                ey = (at(0, sy, 0) - o) * sy
                ez = (at(0, 0, sz) - o) * sz
                trip = np.einsum("...a,...a->...", ex, np.cross(ey, ez))
                ok = ok and bool(np.all(trip > 0))
    return ok


def corner_jacobian_ratio(V):
    """Shape measure of every cell of the vertex grid: the smallest over the
    largest of the eight corner triple products (1 for a parallelepiped,
    <= 0 for a folded cell).  Array [nx, ny, nz]."""
    dets = []
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                sx, sy, sz = 1 - 2 * cx, 1 - 2 * cy, 1 - 2 * cz

                def at(dx, dy, dz):
                    return V[cx + dx: V.shape[0] - 1 + cx + dx,
                             cy + dy: V.shape[1] - 1 + cy + dy,
                             cz + dz: V.shape[2] - 1 + cz + dz]
                o = at(0, 0, 0)
                ex = (at(sx, 0, 0) - o) * sx
                ey = (at(0, sy, 0) - o) * sy
                ez = (at(0, 0, sz) - o) * sz
                dets.append(np.einsum("...a,...a->...", ex, np.cross(ey, ez)))
    d = np.stack(dets, -1)
    return d.min(-1) / d.max(-1)


def perturbed_vertices(n, amp, rng, graded_ratio_z=None, max_draws=100, min_ratio=None):
    """As `_perturbed_vertices_once`, redrawn until every cell is unfolded.

    min_ratio: additionally, the perturbations of the vertices of every cell
    whose corner-Jacobian ratio (`corner_jacobian_ratio`) is below min_ratio
    are drawn again (same distribution, same generator) until no such cell
    is left: independent uniform perturbations of +-0.25 cells occasionally
    bring a corner close to folding (det J at that corner near 0), which no
    penalty of the method's form keeps coercive."""
    for _ in range(max_draws):
        eps = _perturbation(n, amp, rng)
        if min_ratio is not None:
            for _ in range(1000):
                bad = corner_jacobian_ratio(_vertices(n, eps, graded_ratio_z)) < min_ratio
                if not bad.any():
                    break
                touch = np.zeros((n + 1,) * 3, dtype=bool)
                for c in range(8):
                    ox, oy, oz = c & 1, (c >> 1) & 1, (c >> 2) & 1
                    touch[ox:n + ox, oy:n + oy, oz:n + oz] |= bad
                touch[[0, -1], :, :] = touch[:, [0, -1], :] = touch[:, :, [0, -1]] = False
                new = _perturbation(n, amp, rng)
                eps[touch] = new[touch]
            else:
                continue
        V = _vertices(n, eps, graded_ratio_z)
        if corner_jacobians_positive(V):
            return V
    raise RuntimeError("no valid perturbed mesh drawn")


def _perturbation(n, amp, rng):
    """Logical displacements U(-amp, amp) of every vertex, zero on the boundary."""
    eps = rng.uniform(-amp, amp, size=(n + 1, n + 1, n + 1, 3))
    interior = np.zeros((n + 1, n + 1, n + 1), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    return eps * interior[..., None]


def _vertices(n, eps, graded_ratio_z=None):
    """Vertex grid of [0,1]^3 from logical displacements eps; the logical z
    coordinate s is graded by Z(s) = (r^s - 1) / (r^n - 1) if r is given."""
    idx = np.arange(n + 1, dtype=np.float64)
    L = np.zeros((n + 1, n + 1, n + 1, 3))
    L[..., 0] = idx[:, None, None]
    L[..., 1] = idx[None, :, None]
    L[..., 2] = idx[None, None, :]
    L = L + eps
    V = L / n
    if graded_ratio_z is not None:
        r = graded_ratio_z
        V[..., 2] = (r ** L[..., 2] - 1.0) / (r ** n - 1.0)
    return V


def _perturbed_vertices_once(n, amp, rng, graded_ratio_z=None):
    """Vertex grid of [0,1]^3 with n^3 cells; interior vertices are moved by
    U(-amp, amp) cells per coordinate in logical space, boundary vertices stay
    on the cube faces.  If graded_ratio_z is given, the logical z coordinate s
    is mapped by the geometric grading Z(s) = (r^s - 1) / (r^n - 1)."""
    return _vertices(n, _perturbation(n, amp, rng), graded_ratio_z)


def grading_ratio(n, total_over_min):
    """Ratio r with sum_{k<n} r^k = total_over_min (bisection)."""
    lo, hi = 1.0 + 1e-12, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = (mid ** n - 1.0) / (mid - 1.0)
        if s < total_over_min:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def level_from_vertices(V, p, boundary=-1, periodic=False):
    """Conforming structured level from a vertex grid V [nx+1, ny+1, nz+1, 3];
    `periodic`: the faces of the box are identified (neighbours wrap around)."""
    nx, ny, nz = V.shape[0] - 1, V.shape[1] - 1, V.shape[2] - 1
    ne = nx * ny * nz
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # lexicographic, x fastest
    x = x.transpose(2, 1, 0).reshape(-1)
    y = y.transpose(2, 1, 0).reshape(-1)
    z = z.transpose(2, 1, 0).reshape(-1)
    corners = np.zeros((ne, 8, 3))
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        corners[:, c, :] = V[x + cx, y + cy, z + cz]

    def eid(ix, iy, iz):
        if periodic:
            ix, iy, iz = ix % nx, iy % ny, iz % nz
        ok = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny) & (iz >= 0) & (iz < nz)
        return np.where(ok, ix + nx * (iy + ny * iz), -1), ok

    nbr = np.zeros((ne, 6), dtype=np.int32)
    for f, (ox, oy, oz) in enumerate(_FACE_OFF):
        idn, ok = eid(x + ox, y + oy, z + oz)
        nbr[:, f] = np.where(ok, idn, boundary)
    nbr27 = np.zeros((ne, 27), dtype=np.int32)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                idn, _ = eid(x + ox, y + oy, z + oz)
                nbr27[:, (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] = idn
    return dict(p=int(p), shape=(nx, ny, nz), corners=corners, nbr=nbr, nbr27=nbr27,
                parent=np.full(ne, -1, np.int32), octant=np.full(ne, -1, np.int32),
                cls=np.full(ne, LEAF, np.int8), ijk=np.stack([x, y, z], 1).astype(np.int32))


def hierarchy(V_top, p_levels, h_root=None, boundary=-1, periodic=False):
    """Multilevel mesh with global refinement (all non-top elements are twigs).

    p_levels: degrees of the p-levels on the top mesh, finest first, e.g. [8,4,2,1].
    h_root:   if given, the last p-level mesh is h-coarsened (every other
              vertex kept) down to h_root cells per direction.
    Returns the list of levels, root first.
    """
    levels_fine_first = []
    for p in p_levels:
        levels_fine_first.append(level_from_vertices(V_top, p, boundary, periodic))
    V = V_top
    if h_root is not None:
        n = V.shape[0] - 1
        while n > h_root:
            assert n % 2 == 0 and all(s - 1 == n for s in V.shape[:3])
            V = V[::2, ::2, ::2]
            n //= 2
            levels_fine_first.append(level_from_vertices(V, p_levels[-1], boundary, periodic))
    levels = levels_fine_first[::-1]
    for l in range(1, len(levels)):
        fine, coarse = levels[l], levels[l - 1]
        ne = fine["corners"].shape[0]
        if fine["shape"] == coarse["shape"]:
            fine["parent"] = np.arange(ne, dtype=np.int32)
            fine["octant"] = np.full(ne, -1, np.int32)
        else:
            ijk = fine["ijk"]
            cnx, cny, _ = coarse["shape"]
            pi = ijk // 2
            fine["parent"] = (pi[:, 0] + cnx * (pi[:, 1] + cny * pi[:, 2])).astype(np.int32)
            o = ijk % 2
            fine["octant"] = (o[:, 0] + 2 * o[:, 1] + 4 * o[:, 2]).astype(np.int32)
    for l in range(len(levels) - 1):
        levels[l]["cls"] = np.full(levels[l]["corners"].shape[0], TWIG, np.int8)
    return levels


# ---------------------------------------------------------------- right-hand sides
def sine_rhs_spec(k=1.0):
    """u = sin(k pi x) sin(k pi y) sin(k pi z), -lap u = 3 (k pi)^2 u."""
    return dict(kind="sine", k=float(k))


def modes_rhs_spec(rng, n_modes=16, kmax=8):
    """f = sum_m a_m prod_d sin(k_md pi x_d); exact u = sum_m a_m prod sin / (pi^2 |k_m|^2)."""
    k = rng.integers(1, kmax + 1, size=(n_modes, 3))
    a = rng.standard_normal(n_modes)
    return dict(kind="modes", k=k.astype(np.float64), a=a)


def eval_f(spec, xyz):
    """Source f(x) at points xyz [..., 3] (the manufactured input)."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    if spec["kind"] == "sine":
        kp = spec["k"] * np.pi
        return 3.0 * kp * kp * np.sin(kp * x) * np.sin(kp * y) * np.sin(kp * z)
    if spec["kind"] == "psine":
        return 3.0 * np.sin(x) * np.sin(y) * np.sin(z)
    out = np.zeros_like(x)
    for (kx, ky, kz), a in zip(spec["k"], spec["a"]):
        out += a * np.sin(kx * np.pi * x) * np.sin(ky * np.pi * y) * np.sin(kz * np.pi * z)
    return out


def eval_u(spec, xyz):
    """Exact solution u(x) at points xyz [..., 3]."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    if spec["kind"] == "sine":
        kp = spec["k"] * np.pi
        return np.sin(kp * x) * np.sin(kp * y) * np.sin(kp * z)
    if spec["kind"] == "psine":
        return np.sin(x) * np.sin(y) * np.sin(z)
    out = np.zeros_like(x)
    for (kx, ky, kz), a in zip(spec["k"], spec["a"]):
        out += (a / (np.pi ** 2 * (kx * kx + ky * ky + kz * kz))
                * np.sin(kx * np.pi * x) * np.sin(ky * np.pi * y) * np.sin(kz * np.pi * z))
    return out


def periodic_sine_spec():
    """u = sin x sin y sin z on the periodic box [0, 2 pi)^3, -lap u = 3 u
    (zero mean: the right-hand side is consistent with the constant null space)."""
    return dict(kind="psine")


def paper_cartesian_periodic(p, kind, n=None, seed=6):
    """The uniform Cartesian study of the paper (Sec. 6.2, uniform Cartesian):
    [0, 2 pi)^3 with periodic conditions, (128/p)^3 elements (or n^3), mu_star =
    2, delta = 0.08.  kind 'h': h-multigrid at degree p with the paper's L = 4
    levels (root n/8 cells per direction); kind 'p': p-multigrid p, p/2, ...,
    1, then h down to a 2^3 root."""
    n = 128 // p if n is None else n
    V = uniform_vertices(n, hi=(2 * np.pi,) * 3)
    if kind == "h":
        p_levels = [p]
    else:
        p_levels = []
        q = p
        while q >= 1:
            p_levels.append(q)
            q //= 2
    levels = hierarchy(V, p_levels, h_root=max(2, n // 8) if kind == "h" else 2, periodic=True)
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    ndof = levels[-1]["corners"].shape[0] * (p + 1) ** 3
    return dict(levels=levels, rhs=periodic_sine_spec(),
                params=dict(mu_star=2.0, delta=0.08, s1=1, s2=1, sc=2),
                u0=random_start(rng, ndof))


def surrogate_training_corners(n, rng, ar_max=16.0, amp=0.25):
    """Single elements drawn like the interior elements of the curvilinear
    workloads (the learned surrogate's training inputs): a box of widths
    (1, 1, 1/AR) with AR ~ U[1, ar_max], each corner moved by U(-amp, amp) of
    the box width per coordinate.  Returns corners [n, 8, 3]."""
    ar = rng.uniform(1.0, ar_max, size=n)
    h = np.stack([np.ones(n), np.ones(n), 1.0 / ar], 1)
    corners = np.zeros((n, 8, 3))
    for cc in range(8):
        for d in range(3):
            corners[:, cc, d] = ((cc >> d) & 1) * h[:, d]
    corners += rng.uniform(-amp, amp, size=corners.shape) * h[:, None, :]
    return corners


SURROGATE_SET_SEED = SEED_BASE + 200


def surrogate_training_set(n, p):
    """The learned surrogate's training elements at degree p: the first half
    from the distribution of the graded, strongly perturbed workload (AR ~
    U[1, 16], corners moved by +-0.25 widths), the second half from that of
    the large uniform workload (AR 1, +-0.15); seeded by p."""
    rng = np.random.default_rng(SURROGATE_SET_SEED + p)
    a = surrogate_training_corners(n // 2, rng, 16.0, 0.25)
    b = surrogate_training_corners(n - n // 2, rng, 1.0, 0.15)
    return np.concatenate([a, b], 0)


def random_start(rng, n):
    """Start vector uniform in [-1, 1] (Sec. 6.1)."""
    return rng.uniform(-1.0, 1.0, size=n)


# ---------------------------------------------------------------- the configurations
def config(cid, small=False, root=None):
    """Workload `cid` in 1, 2, 3, 5 (config 4: `config4`).

    Returns dict(levels, rhs, u0, params) with params the solver parameters
    (mu_star, delta, s1, s2, sc, and for an SCG root coarse / root_rtol /
    root_steps).  `small` shrinks configs 2/3/5 to a mesh the oracle handles
    in seconds while keeping the structure (degree, hierarchy shape,
    perturbation, grading).  `root` chooses the bottom of the curvilinear
    hierarchies (configs 3, 5): "p1" ends at the p = 1 level of the fine mesh,
    solved by SCG (p-multigrid 7 -> 3 -> 1); "h" continues with h-coarsening
    at p = 1 down to a 4^3 root solved exactly.
    """
    rng = np.random.default_rng(SEED_BASE + cid)
    if cid == 1:
        V = uniform_vertices(4)
        levels = hierarchy(V, [4, 2, 1])
        rhs = sine_rhs_spec()
        prm = dict(mu_star=2.0, delta=0.08, s1=2, s2=2, sc=4)
    elif cid == 2:
        n = 4 if small else 32
        V = uniform_vertices(n)
        levels = hierarchy(V, [8, 4, 2, 1], h_root=min(4, n))
        rhs = modes_rhs_spec(rng)
        prm = dict(mu_star=5.0, delta=0.08, s1=2, s2=2, sc=4)
    elif cid == 3:
        # small: 4^3 cells, grading to aspect ratio 4 (AR 16 on four cells folds)
        n = 4 if small else 16
        r = grading_ratio(n, (4.0 if small else 16.0) * n)
        V = perturbed_vertices(n, 0.25, rng, graded_ratio_z=r, min_ratio=MIN_JACOBIAN_RATIO)
        levels = hierarchy(V, [7, 3, 1], h_root=None if root == "p1" else min(4, n))
        rhs = modes_rhs_spec(rng)
        # aspect ratios up to 16 with strongly sheared thin cells: the paper's
        # robust setting for high aspect ratios, SCG with (12, 4, 8) steps
        prm = dict(mu_star=5.0, delta=0.08, s1=12, s2=4, sc=8)
    elif cid == 5:
        n = 8 if small else 64
        V = perturbed_vertices(n, 0.15, rng)
        levels = hierarchy(V, [7, 3, 1], h_root=None if root == "p1" else 4)
        rhs = modes_rhs_spec(rng)
        prm = dict(mu_star=5.0, delta=0.08, s1=2, s2=2, sc=4)
    else:
        raise ValueError(f"unknown config {cid}")
    if root == "p1":
        prm.update(coarse="scg", root_rtol=1e-3, root_steps=64)
    top = levels[-1]
    N = top["p"] + 1
    ndof = top["corners"].shape[0] * N ** 3
    u0 = random_start(rng, ndof)
    return dict(levels=levels, rhs=rhs, u0=u0, params=prm, cid=cid)


# ---------------------------------------------------------------- local refinement
def front_spec(rng, alpha=50.0):
    """Steep spherical front u = atan(alpha (|x - x0| - r0)): x0 = -U(0.05, 0.25)^3
    (outside the domain), r0 uniform in the middle 60% between the nearest and
    the farthest point of [0,1]^3 from x0."""
    x0 = -rng.uniform(0.05, 0.25, size=3)
    near = np.linalg.norm(x0)                   # nearest point is the origin corner
    far = np.linalg.norm(1.0 - x0)
    r0 = near + (far - near) * rng.uniform(0.2, 0.8)
    return dict(kind="front", alpha=float(alpha), x0=x0, r0=float(r0))


def _front_parts(spec, xyz):
    d = xyz - spec["x0"]
    rho = np.linalg.norm(d, axis=-1)
    return rho, spec["alpha"] * (rho - spec["r0"])


def eval_front_u(spec, xyz):
    _, s = _front_parts(spec, xyz)
    return np.arctan(s)


def eval_front_f(spec, xyz):
    """f = -lap u = -(u'' + 2 u' / rho) for u = atan(alpha (rho - r0))."""
    rho, s = _front_parts(spec, xyz)
    a = spec["alpha"]
    up = a / (1.0 + s * s)
    upp = -2.0 * a * a * s / (1.0 + s * s) ** 2
    return -(upp + 2.0 * up / rho)


def _cell_front_distance(spec, lo, h):
    """Distance from the axis-aligned cells [lo, lo+h] to the sphere |x-x0| = r0."""
    x0, r0 = spec["x0"], spec["r0"]
    near = np.linalg.norm(np.clip(x0, lo, lo + h) - x0, axis=-1)
    far = np.linalg.norm(np.maximum(np.abs(lo - x0), np.abs(lo + h - x0)), axis=-1)
    return np.where(r0 < near, near - r0, np.where(r0 > far, r0 - far, 0.0))


def refined_hierarchy(spec, n_base=8, p=3, n_ref=3, n_root=4, buffer=2.0):
    """Multilevel mesh with local refinement towards the front (Sec. 3.1).

    Levels: h-coarsened p=1 levels down to n_root^3 (root), the base n_base^3
    at p=1 and at degree p (global), then n_ref refinement levels at degree p.
    A cell of grid n (size h = 1/n) is marked for regular refinement when its
    distance to the front is <= buffer * h; with buffer >= 2 every neighbour of
    a marked cell lies in the active zone of its level, so marked cells are
    nested and every frozen child has a leaf parent.  Level k+1 holds the
    children of the marked cells of level k (active) and of their unmarked
    face/edge/vertex neighbours (frozen).  Faces of frozen elements that leave
    the level's zone are Neumann (-2); frozen rows are never evaluated.
    """
    levels = []
    # global part: p=1 from n_root to n_base, then degree p on n_base
    V = uniform_vertices(n_base)
    glob = hierarchy(V, [p, 1], h_root=n_root)          # root first, ends at (n_base, p)
    glob_shapes = [lv["shape"] for lv in glob]
    assert glob_shapes[-1] == (n_base,) * 3
    # cells (integer coordinates) per level from the base up
    def mark(n, cells):
        h = 1.0 / n
        lo = cells * h
        return _cell_front_distance(spec, lo, h) <= buffer * h

    base_cells = glob[-1]["ijk"].astype(np.int64)
    marked = mark(n_base, base_cells)
    glob[-1]["cls"] = np.where(marked, TWIG, LEAF).astype(np.int8)
    levels = glob
    n = n_base
    prev_cells, prev_marked = base_cells, marked
    prev_index = {tuple(c): i for i, c in enumerate(base_cells)}
    for k in range(n_ref):
        n2 = 2 * n
        mset = {tuple(c) for c in prev_cells[prev_marked]}
        # unmarked neighbours of marked cells on the parent grid
        nbrs = set()
        for c in mset:
            for oz in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    for ox in (-1, 0, 1):
                        q = (c[0] + ox, c[1] + oy, c[2] + oz)
                        if q in mset or min(q) < 0 or max(q) >= n:
                            continue
                        nbrs.add(q)
        assert all(q in prev_index for q in nbrs), "frozen parent outside the active zone"
        children, cls_list, parent, octant = [], [], [], []
        for group, cl in ((sorted(mset), None), (sorted(nbrs), FROZEN)):
            for c in group:
                for o in range(8):
                    ox, oy, oz = o & 1, (o >> 1) & 1, (o >> 2) & 1
                    children.append((2 * c[0] + ox, 2 * c[1] + oy, 2 * c[2] + oz))
                    cls_list.append(cl)
                    parent.append(prev_index[c])
                    octant.append(o)
        cells = np.array(children, dtype=np.int64)
        ne = len(cells)
        index = {tuple(c): i for i, c in enumerate(cells)}
        last = k == n_ref - 1
        m2 = np.zeros(ne, bool) if last else mark(n2, cells)
        cls = np.array([FROZEN if cl == FROZEN else (TWIG if m2[i] else LEAF)
                        for i, cl in enumerate(cls_list)], dtype=np.int8)
        m2 &= cls != FROZEN
        h2 = 1.0 / n2
        corners = np.zeros((ne, 8, 3))
        for cc in range(8):
            off = np.array([cc & 1, (cc >> 1) & 1, (cc >> 2) & 1])
            corners[:, cc, :] = (cells + off) * h2
        nbr = np.zeros((ne, 6), np.int32)
        for f, (ox, oy, oz) in enumerate(_FACE_OFF):
            for i, c in enumerate(cells):
                q = (c[0] + ox, c[1] + oy, c[2] + oz)
                if min(q) < 0 or max(q) >= n2:
                    nbr[i, f] = -1
                else:
                    nbr[i, f] = index.get(q, -2)
        nbr27 = np.full((ne, 27), -1, np.int32)
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    s = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)
                    for i, c in enumerate(cells):
                        nbr27[i, s] = index.get((c[0] + ox, c[1] + oy, c[2] + oz), -1)
        levels.append(dict(p=int(p), shape=(n2, n2, n2), corners=corners, nbr=nbr, nbr27=nbr27,
                           parent=np.array(parent, np.int32), octant=np.array(octant, np.int32),
                           cls=cls, ijk=cells.astype(np.int32)))
        n, prev_cells, prev_marked, prev_index = n2, cells, m2, index
    return levels


def geometric_marks(spec, n_base=8, n_ref=3, buffer=2.0):
    """The refined cell sets of `refined_hierarchy`, level by level from the
    base (grid n_base 2^k at refinement level k): cells within buffer * h of
    the front among the active cells of the level."""
    marks = []
    n = n_base
    cells = [(x, y, z) for z in range(n) for y in range(n) for x in range(n)]
    for k in range(n_ref):
        arr = np.array(cells, dtype=np.int64)
        h = 1.0 / n
        m = _cell_front_distance(spec, arr * h, h) <= buffer * h
        mk = {c for c, f in zip(cells, m) if f}
        marks.append(mk)
        cells = sorted({(2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2))
                        for c in mk for o in range(8)})
        n *= 2
    return marks


def close_marks(marks, n_base):
    """Admissible refinement: adds to `marks` (refined cell sets per level,
    base first, each a set of integer cells of grid n_base 2^k) what is needed
    so that every face / edge / vertex neighbour of a refined cell inside the
    domain is an element of its level (then the neighbours' children can be
    frozen with a leaf parent).  A missing neighbour position is covered by a
    leaf of a coarser level, which gets refined, down the levels until
    nothing changes.  Returns the closed sets (new objects)."""
    marks = [set(m) for m in marks]
    changed = True
    while changed:
        changed = False
        for k in range(len(marks)):
            n = n_base << k
            active = None if k == 0 else {
                (2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2))
                for c in marks[k - 1] for o in range(8)}
            for c in list(marks[k]):
                for oz in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for ox in (-1, 0, 1):
                            q = (c[0] + ox, c[1] + oy, c[2] + oz)
                            if min(q) < 0 or max(q) >= n or active is None or q in active:
                                continue
                            # q is covered by a coarser leaf: refine its parent at k-1
                            par = (q[0] // 2, q[1] // 2, q[2] // 2)
                            if par not in marks[k - 1]:
                                marks[k - 1].add(par)
                                changed = True
    return marks


def hierarchy_from_marks(marks, n_base=8, p=3, n_root=4):
    """Multilevel mesh with local refinement from refined cell sets (as
    `refined_hierarchy`, whose geometric marking `geometric_marks` returns):
    the global part up to the base n_base^3 at degree p, then one level per
    set, holding the children of the refined cells of the level below
    (active) and of their unmarked neighbours (frozen).  The sets must be
    admissible (`close_marks`)."""
    V = uniform_vertices(n_base)
    levels = hierarchy(V, [p, 1], h_root=n_root)
    base_cells = levels[-1]["ijk"].astype(np.int64)
    prev_index = {tuple(int(v) for v in c): i for i, c in enumerate(base_cells)}
    m0 = marks[0] if marks else set()
    levels[-1]["cls"] = np.array([TWIG if tuple(int(v) for v in c) in m0 else LEAF
                                  for c in base_cells], np.int8)
    n = n_base
    active = set(prev_index)   # the active (non-frozen) elements of the level
    for k, mset in enumerate(marks):
        n2 = 2 * n
        assert all(c in active for c in mset), "refined cell is not an active element of its level"
        nbrs = set()
        for c in mset:
            for oz in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    for ox in (-1, 0, 1):
                        q = (c[0] + ox, c[1] + oy, c[2] + oz)
                        if q in mset or min(q) < 0 or max(q) >= n:
                            continue
                        nbrs.add(q)
        assert all(q in active for q in nbrs), "marks not admissible (close_marks)"
        nxt = marks[k + 1] if k + 1 < len(marks) else set()
        children, cls_list, parent, octant = [], [], [], []
        for group, frozen in ((sorted(mset), False), (sorted(nbrs), True)):
            for c in group:
                for o in range(8):
                    ch = (2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2))
                    children.append(ch)
                    cls_list.append(FROZEN if frozen else (TWIG if ch in nxt else LEAF))
                    parent.append(prev_index[c])
                    octant.append(o)
        cells = np.array(children, dtype=np.int64)
        ne = len(cells)
        index = {c: i for i, c in enumerate(children)}
        h2 = 1.0 / n2
        corners = np.zeros((ne, 8, 3))
        for cc in range(8):
            off = np.array([cc & 1, (cc >> 1) & 1, (cc >> 2) & 1])
            corners[:, cc, :] = (cells + off) * h2
        nbr = np.zeros((ne, 6), np.int32)
        for f, (ox, oy, oz) in enumerate(_FACE_OFF):
            for i, c in enumerate(children):
                q = (c[0] + ox, c[1] + oy, c[2] + oz)
                nbr[i, f] = -1 if (min(q) < 0 or max(q) >= n2) else index.get(q, -2)
        nbr27 = np.full((ne, 27), -1, np.int32)
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    sl = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)
                    for i, c in enumerate(children):
                        nbr27[i, sl] = index.get((c[0] + ox, c[1] + oy, c[2] + oz), -1)
        levels.append(dict(p=int(p), shape=(n2, n2, n2), corners=corners, nbr=nbr, nbr27=nbr27,
                           parent=np.array(parent, np.int32), octant=np.array(octant, np.int32),
                           cls=np.array(cls_list, np.int8), ijk=cells.astype(np.int32)))
        n, prev_index = n2, index
        active = {c for c, cl in zip(children, cls_list) if cl != FROZEN}
    return levels


def _cell_dist_to_front(spec, cells, n):
    """Distance of the cells (integer coordinates on grid n) to the front."""
    h = 1.0 / n
    return _cell_front_distance(spec, np.asarray(cells, dtype=np.float64) * h, h)


def add_p_levels(levels, spec, p_levels, p_buffers):
    """Local p-refinement levels on top of a locally refined hierarchy (Sec.
    3.1: p-refinement elevates the degree in selected elements; every level
    keeps one degree).  Level k raises to degree p_levels[k] the active cells
    of the level below whose distance to the front is <= p_buffers[k] cell
    widths and whose 26 neighbours inside the domain are all active there
    (so that each frozen child has an active parent); their unmarked
    neighbours become frozen p-children.  Children keep the geometry; parent
    = the same cell one level down, octant -1 (p-refinement)."""
    for pk, bk in zip(p_levels, p_buffers):
        prev = levels[-1]
        n = prev["shape"][0]
        cells = [tuple(int(v) for v in c) for c in prev["ijk"]]
        index = {c: i for i, c in enumerate(cells)}
        active = {c for c, cl in zip(cells, prev["cls"]) if cl != FROZEN}
        dist = _cell_dist_to_front(spec, cells, n)
        h = 1.0 / n

        def nbrs(c):
            for oz in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    for ox in (-1, 0, 1):
                        q = (c[0] + ox, c[1] + oy, c[2] + oz)
                        if q != c and min(q) >= 0 and max(q) < n:
                            yield q
        marked = {c for c, d in zip(cells, dist)
                  if c in active and d <= bk * h and all(q in active for q in nbrs(c))}
        if not marked:
            raise ValueError(f"no cell qualifies for p-refinement to p = {pk}")
        frozen = {q for c in marked for q in nbrs(c) if q not in marked}
        new_cells = sorted(marked) + sorted(frozen)
        # the previous level's marked cells become twigs there
        prev["cls"] = np.array([TWIG if c in marked else cl for c, cl in zip(cells, prev["cls"])],
                               np.int8)
        ne = len(new_cells)
        new_index = {c: i for i, c in enumerate(new_cells)}
        corners = np.stack([prev["corners"][index[c]] for c in new_cells], 0)
        nbr = np.zeros((ne, 6), np.int32)
        for f, (ox, oy, oz) in enumerate(_FACE_OFF):
            for i, c in enumerate(new_cells):
                q = (c[0] + ox, c[1] + oy, c[2] + oz)
                nbr[i, f] = -1 if (min(q) < 0 or max(q) >= n) else new_index.get(q, -2)
        nbr27 = np.full((ne, 27), -1, np.int32)
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    sl = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)
                    for i, c in enumerate(new_cells):
                        nbr27[i, sl] = new_index.get((c[0] + ox, c[1] + oy, c[2] + oz), -1)
        cls = np.array([LEAF] * len(marked) + [FROZEN] * len(frozen), np.int8)
        levels.append(dict(p=int(pk), shape=prev["shape"], corners=corners, nbr=nbr, nbr27=nbr27,
                           parent=np.array([index[c] for c in new_cells], np.int32),
                           octant=np.full(ne, -1, np.int32), cls=cls,
                           ijk=np.array(new_cells, np.int32).reshape(-1, 3)))
    return levels


def leaf_dofs(levels):
    """Leaf degrees of freedom per degree over the composite mesh."""
    out = {}
    for lv in levels:
        nl = int(np.sum(np.asarray(lv["cls"]) == LEAF))
        out[lv["p"]] = out.get(lv["p"], 0) + nl * (lv["p"] + 1) ** 3
    return out


# degrees and distance bands (cell widths of the finest h-level) of the local
# p-refinement levels of the front workload
HP_DEGREES = (5, 7, 10)
HP_BUFFERS = (2.5, 1.75, 0.0)


def config4(small=False, hp=True):
    """Config 4: steep front (alpha = 50) on [0,1]^3, base 8^3 at p = 3 with up
    to 3 levels of local h-refinement towards the front (p = 3), then, with
    hp, local p-refinement levels raising the elements closest to the front
    to p = 5, 7, 10 (HP_DEGREES / HP_BUFFERS): the composite leaves carry
    degrees 3, 5, 7 and 10, each level one degree.  small: base 4^3, one
    h-level, p-levels 5 and 7."""
    rng = np.random.default_rng(SEED_BASE + 4)
    spec = front_spec(rng)
    levels = refined_hierarchy(spec, n_base=4 if small else 8, n_ref=1 if small else 3,
                               n_root=2 if small else 4)
    if hp:
        if small:
            levels = add_p_levels(levels, spec, (5, 7), (1.5, 0.0))
        else:
            levels = add_p_levels(levels, spec, HP_DEGREES, HP_BUFFERS)
    top = levels[-1]
    ndof = top["corners"].shape[0] * (top["p"] + 1) ** 3
    u0 = random_start(rng, ndof)
    return dict(levels=levels, rhs=spec, u0=u0, cid=4,
                params=dict(mu_star=5.0, delta=0.08, s1=2, s2=2, sc=4))
