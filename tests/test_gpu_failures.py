"""Failure reporting through the C ABI, made on the host side (no GPU fault,
trap or hang): an inverted element is refused at set-up (DGFAS_ERR_MESH, by
the host-side face check or the Jacobian test), a
NaN in the right-hand side ends the solve with DGFAS_ERR_DIVERGED, a cycle
cap below the cycles the solve needs returns DGFAS_ERR_NOT_CONVERGED, and
the context stays usable after each of them."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_oracle, make_solver, rhs_both, torch_cuda

pytestmark = pytest.mark.gpu


def test_inverted_element_is_refused_at_setup():
    torch_cuda()
    cfg = wl.config(1)
    levels = [dict(lv) for lv in cfg["levels"]]
    top = dict(levels[-1])
    corners = top["corners"].copy()
    # mirror element 5 through its own centre plane x: corners swap left and
    # right, the trilinear map is orientation-reversing (det J < 0)
    c = corners[5].copy()
    xm = c[:, 0].mean()
    corners[5, :, 0] = 2 * xm - c[:, 0]
    top["corners"] = corners
    levels[-1] = top
    pr = cfg["params"]
    with pytest.raises(dgfas.DgfasError) as ex:
        dgfas.Solver(levels, pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    assert ex.value.code == -4
    # refused by the host-side face check (the mirrored element's faces no
    # longer meet its neighbours' corner by corner) or, if it passes that, by
    # the Jacobian test at the GLL nodes; either names the element
    msg = dgfas.load().dgfas_last_error()
    assert (b"Jacobian" in msg or b"aligned local axes" in msg) and b"5" in msg


def test_nan_in_rhs_reports_divergence_and_context_survives():
    torch = torch_cuda()
    cfg = wl.config(1)
    S, H = make_solver(cfg), make_oracle(cfg)
    b, _ = rhs_both(cfg, S, H)
    bad = b.clone()
    bad[17] = float("nan")
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, bad, 1e-10, 10, raise_on_fail=False)
    assert info["code"] == -6
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 20)
    assert info["code"] == 0 and info["r_final"] <= 1e-10 * info["r0"]


def test_cycle_cap_reports_not_converged():
    torch = torch_cuda()
    cfg = wl.config(1)
    S, H = make_solver(cfg), make_oracle(cfg)
    b, _ = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 1, raise_on_fail=False)
    assert info["code"] == -5 and info["cycles"] == 1
    with pytest.raises(dgfas.DgfasError) as ex:
        S.dgfas_solve(torch.from_numpy(cfg["u0"].copy()).cuda(), b, 1e-10, 1)
    assert ex.value.code == -5
