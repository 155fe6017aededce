"""Edge cases and full-size sampled parity of the CUDA path against the oracle:
maximum degree (p = 10, N = 11; FP64 and the FP32 smoother operator), a
ragged 3 x 5 x 2 mesh, a single element,
invalid arguments, and the full 32^3, p = 8 workload (the bench's launch
configuration) checked on sampled elements."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import rel, torch_cuda

pytestmark = pytest.mark.gpu


def _pair(levels, mu=5.0):
    from oracle import fas
    S = dgfas.Solver(levels, mu, 0.08, 2, 2, 4, precision=dgfas.DGFAS_FP64)
    H = fas.Hierarchy(levels, mu, 0.08, 2, 2, 4)
    return S, H


def _apply_and_sweep(S, H, seed=1):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    for l in range(S.n_levels):
        n = S.ndof(l)
        u, g = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        out = torch.empty_like(ud)
        S.dgfas_apply_op(l, ud, gd, out)
        Au = H.A(l, u)
        assert rel(out.cpu().numpy(), g - Au) < 1e-12, l
        # the smoothers' FP32 operator on the FP32-rounded u (curvilinear
        # levels: metric recomputed from the trilinear map), 3e-5 of max |A u|
        u32 = u.astype(np.float32)
        Au32 = H.A(l, u32.astype(np.float64))
        o32 = torch.empty(n, dtype=torch.float32, device="cuda")
        S.dgfas_apply_op32(l, torch.from_numpy(u32).cuda(), gd, o32)
        assert np.abs(o32.cpu().numpy() - (g - Au32)).max() <= 3e-5 * (np.abs(Au32).max() + 1.0), l
        if l > 0:
            S.dgfas_schwarz_smooth(l, ud, gd, 1)
            ref = H.was(l, u, g, 1)
            assert rel(ud.cpu().numpy() - u, ref - u) < 1e-10, l


def test_maximum_degree_p10():
    V = wl.perturbed_vertices(2, 0.1, np.random.default_rng(2))
    levels = wl.hierarchy(V, [10, 5, 1])
    S, H = _pair(levels)
    _apply_and_sweep(S, H)


def test_ragged_mesh_and_box_widths():
    V = wl.uniform_vertices(3, 5, 2, hi=(0.6, 1.0, 0.3))
    levels = wl.hierarchy(V, [4, 2, 1])
    S, H = _pair(levels)
    _apply_and_sweep(S, H)


def test_single_element():
    V = wl.uniform_vertices(1)
    levels = wl.hierarchy(V, [3, 1])
    S, H = _pair(levels)
    _apply_and_sweep(S, H)


def test_invalid_arguments_return_codes():
    torch = torch_cuda()
    lib = dgfas.load()
    with pytest.raises(dgfas.DgfasError) as e:          # p > 10
        dgfas.Solver(wl.hierarchy(wl.uniform_vertices(1), [11, 1]), 5.0, 0.08)
    assert e.value.code == -7
    with pytest.raises(dgfas.DgfasError) as e:          # delta outside (0, 0.5)
        dgfas.Solver(wl.hierarchy(wl.uniform_vertices(2), [2, 1]), 5.0, 0.7)
    assert e.value.code == -1
    S = dgfas.Solver(wl.hierarchy(wl.uniform_vertices(2), [2, 1]), 5.0, 0.08)
    u = torch.zeros(S.ndof(-1), dtype=torch.float64, device="cuda")
    assert lib.dgfas_apply_op(S.ctx, 5, dgfas._ptr(u), None, dgfas._ptr(u.clone())) == -1
    assert lib.dgfas_apply_op(S.ctx, 1, dgfas._ptr(u), None, dgfas._ptr(u)) == -1   # aliasing
    assert lib.dgfas_schwarz_smooth(S.ctx, 0, dgfas._ptr(u), dgfas._ptr(u), 1) == -1  # root
    assert lib.dgfas_fas_vcycle(None, dgfas._ptr(u), dgfas._ptr(u), None) == -1


def _patch_level(level, centre, rings):
    """Sub-level of the elements within `rings` (Chebyshev distance in the
    element grid) of `centre`; faces leaving the patch become Neumann.  Rows
    of elements at distance < rings - 1 equal the full level's rows."""
    ijk = level["ijk"]
    c = ijk[centre]
    sel = np.nonzero(np.max(np.abs(ijk - c), axis=1) <= rings)[0]
    remap = -np.ones(ijk.shape[0], np.int64)
    remap[sel] = np.arange(len(sel))
    nbr = level["nbr"][sel].copy()
    inside = nbr >= 0
    nbr[inside] = remap[nbr[inside]]
    nbr[inside & (nbr < 0)] = -2
    nb27 = level["nbr27"][sel].copy()
    ok = nb27 >= 0
    nb27[ok] = remap[nb27[ok]]
    sub = dict(level, corners=level["corners"][sel], nbr=nbr.astype(np.int32),
               nbr27=nb27.astype(np.int32), cls=level["cls"][sel], ijk=ijk[sel],
               parent=np.full(len(sel), -1, np.int32), octant=np.full(len(sel), -1, np.int32))
    return sub, sel


def test_full_size_config2_sampled_parity():
    """The bench's 32^3, p = 8 top level: apply and one FP64 sweep on the GPU at
    full size, compared on sampled elements with the oracle evaluated on a
    patch around each sample."""
    torch = torch_cuda()
    from oracle import schwarz, sip
    cfg = wl.config(2)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                     precision=dgfas.DGFAS_FP64)
    top = cfg["levels"][-1]
    L = S.n_levels - 1
    N3 = 9 ** 3
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, S.ndof(L))
    g = rng.uniform(-1, 1, S.ndof(L))
    ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
    out = torch.empty_like(ud)
    S.dgfas_apply_op(L, ud, gd, out)
    us = ud.clone()
    S.dgfas_schwarz_smooth(L, us, gd, 1)
    out, du = out.cpu().numpy(), (us - ud).cpu().numpy()
    samples = [0, 31, 1023, 16 * 1024 + 16 * 32 + 16, 32767]   # corner, edge, face, interior
    for e in samples:
        sub, sel = _patch_level(top, e, 3)
        k = int(np.nonzero(sel == e)[0][0])
        ops = sip.LevelOps(sub, pr["mu_star"])
        us_ = u.reshape(-1, N3)[sel].reshape(-1)
        gs_ = g.reshape(-1, N3)[sel].reshape(-1)
        r = gs_ - sip.apply(ops, us_).reshape(-1)
        got = out.reshape(-1, N3)[e]
        assert rel(got, r.reshape(-1, N3)[k]) < 1e-12, e
        sw = schwarz.Schwarz(sub, pr["delta"], pr["mu_star"])
        ref = sw.correction(r).reshape(-1, N3)[k]
        assert rel(du.reshape(-1, N3)[e], ref) < 1e-10, e


def test_full_size_config5_sampled_parity():
    """The bench's headline level, 64^3 curvilinear elements at p = 7 (134M
    DoF): the FP64 residual (two-pass operator), the FP32 operator of the
    smoothers (metric recomputed from the trilinear map) and one FP64 Schwarz
    sweep on the GPU at full size, compared on sampled elements (corner, edge,
    face, interior) with the oracle evaluated on the 7^3-element patch around
    each sample."""
    torch = torch_cuda()
    from oracle import schwarz, sip
    cfg = wl.config(5)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                     precision=dgfas.DGFAS_FP64)
    top = cfg["levels"][-1]
    L = S.n_levels - 1
    N3 = 8 ** 3
    rng = np.random.default_rng(6)
    n = S.ndof(L)
    u = rng.uniform(-1, 1, n)
    g = rng.uniform(-1, 1, n)
    u32 = u.astype(np.float32)
    ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
    out = torch.empty_like(ud)
    S.dgfas_apply_op(L, ud, gd, out)
    o32 = torch.empty(n, dtype=torch.float32, device="cuda")
    S.dgfas_apply_op32(L, torch.from_numpy(u32).cuda(), gd, o32)
    us = ud.clone()
    S.dgfas_schwarz_smooth(L, us, gd, 1)
    out, o32, du = out.cpu().numpy(), o32.cpu().numpy(), (us - ud).cpu().numpy()
    S.close()
    samples = [0, 63, 64 * 64 * 32 + 31, 64 * 64 * 32 + 64 * 32 + 32, 64 ** 3 - 1]
    for e in samples:
        sub, sel = _patch_level(top, e, 3)
        k = int(np.nonzero(sel == e)[0][0])
        ops = sip.LevelOps(sub, pr["mu_star"])
        gs_ = g.reshape(-1, N3)[sel].reshape(-1)
        r = gs_ - sip.apply(ops, u.reshape(-1, N3)[sel].reshape(-1)).reshape(-1)
        assert rel(out.reshape(-1, N3)[e], r.reshape(-1, N3)[k]) < 1e-12, e
        Au32 = sip.apply(ops, u32.astype(np.float64).reshape(-1, N3)[sel].reshape(-1))
        ref32 = (gs_ - Au32.reshape(-1)).reshape(-1, N3)[k]
        scale = np.abs(Au32.reshape(-1, N3)[k]).max() + 1.0
        assert np.abs(o32.reshape(-1, N3)[e] - ref32).max() <= 3e-5 * scale, e
        sw = schwarz.Schwarz(sub, pr["delta"], pr["mu_star"])
        ref = sw.correction(r).reshape(-1, N3)[k]
        assert rel(du.reshape(-1, N3)[e], ref) < 1e-10, e
