"""GPU element error indicators of the adaptive loop (Sec. 6.4) against the
oracle on the locally refined config 4 (small): eps_e . (A eps)_e per element
for every level (frozen rows are 0 on the GPU and not compared), and the
composite energy norm over the leaves (Sec. 6.1)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import rel, torch_cuda

pytestmark = pytest.mark.gpu


def test_element_energy_matches_oracle():
    torch = torch_cuda()
    from oracle import fas
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    H = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    rng = np.random.default_rng(9)
    eps_all, tot = [], 0.0
    for l in range(S.n_levels):
        eps = rng.uniform(-1, 1, S.ndof(l))
        eps_all.append(eps)
        out = torch.empty(cfg["levels"][l]["corners"].shape[0], dtype=torch.float64, device="cuda")
        S.dgfas_element_energy(l, torch.from_numpy(eps).cuda(), out)
        g = out.cpu().numpy()
        o = H.element_energy(l, eps)
        act = np.asarray(cfg["levels"][l]["cls"]) != wl.FROZEN
        assert rel(g[act], o[act]) < 1e-12, l
        assert np.all(g[~act] == 0.0)
        tot += g[np.asarray(cfg["levels"][l]["cls"]) == wl.LEAF].sum()
    assert abs(np.sqrt(tot) - H.energy_error(eps_all)) <= 1e-12 * H.energy_error(eps_all)
