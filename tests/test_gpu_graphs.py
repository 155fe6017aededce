"""CUDA-graph replay of the cycle body: one captured graph per (u, f) buffer
pair, four kept (least recently used replaced).  Replays on alternating and
evicted buffer pairs give the same bits as the uncaptured cycle."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [dgfas.DGFAS_FP64, dgfas.DGFAS_BF16])
def test_graph_cache_over_buffer_pairs(prec):
    from tests.gpu_helpers import make_solver, torch_cuda
    torch = torch_cuda()
    cfg = wl.config(2, small=True)
    S = make_solver(cfg, precision=prec)
    rng = np.random.default_rng(5)
    n = S.ndof(-1)
    u0 = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    # reference: the cycle without graphs
    S.dgfas_use_graph(False)
    ref = u0.clone()
    S.dgfas_fas_vcycle(ref, b)
    ref = ref.cpu().numpy()
    S.dgfas_use_graph(True)
    pairs = [(torch.empty_like(u0), b.clone()) for _ in range(5)]   # one more than kept
    order = [0, 1, 0, 2, 3, 1, 4, 0, 4, 2]
    for i in order:
        u, f = pairs[i]
        u.copy_(u0)
        S.dgfas_fas_vcycle(u, f)
        np.testing.assert_array_equal(u.cpu().numpy(), ref, err_msg=f"pair {i}")
