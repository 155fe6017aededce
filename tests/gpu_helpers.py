"""Shared helpers of the GPU parity tests: build the CUDA-path solver and the
oracle hierarchy for one workload, both from the same seeded inputs."""
import numpy as np

from paper_2608_14123_b300 import workloads as wl


def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


SOLVER_KW = ("coarse", "root_rtol", "root_steps", "projection")


def make_solver(cfg, precision=0, smoother=0, **over):
    """CUDA-path solver of workload cfg; `over` replaces solver parameters
    (mu_star, delta, s1, s2, sc, coarse, root_rtol, root_steps, projection;
    coarse and projection by the oracle's names "dense" / "scg", "interp" /
    "l2")."""
    from paper_2608_14123_b300 import dgfas
    pr = dict(cfg["params"])
    pr.update(over)
    kw = {k: pr[k] for k in SOLVER_KW if k in pr}
    if "coarse" in kw:
        kw["coarse"] = {"dense": dgfas.DGFAS_COARSE_DENSE, "scg": dgfas.DGFAS_COARSE_SCG}[kw["coarse"]]
    if "projection" in kw:
        kw["projection"] = {"interp": dgfas.DGFAS_P_INTERP, "l2": dgfas.DGFAS_P_L2}[kw["projection"]]
    return dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                        precision=precision, smoother=smoother, **kw)


def make_oracle(cfg, smoother="was", **over):
    """Oracle hierarchy of the same workload and parameters."""
    from oracle import fas
    pr = dict(cfg["params"])
    pr.update(over)
    kw = {k: pr[k] for k in SOLVER_KW if k in pr}
    return fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                         smoother=smoother, **kw)


def rhs_both(cfg, S, H):
    """Top-level RHS from f sampled at each side's own node coordinates."""
    torch = torch_cuda()
    from oracle import sip
    top = H.ops[-1]
    X = top.geo["x"]
    b_or = sip.rhs(top, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1)
    xyz = S.node_coords(-1)
    f = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz.cpu().numpy())).cuda()
    b = torch.empty_like(f)
    S.dgfas_assemble_rhs(f, None, b)
    torch.cuda.synchronize()
    return b, b_or


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
