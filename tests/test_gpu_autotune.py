"""Launch-shape autotuner (batching / tile tuning of the hot path): every
candidate launch shape of every tunable kernel gives bit-identical V-cycles,
the tuner keeps one of the candidates, and invalid shapes are rejected."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _vcycle(S, u0, b):
    u = u0.clone()
    S.dgfas_fas_vcycle(u, b)
    return u.cpu().numpy()


def _setup(cid, prec):
    from tests.gpu_helpers import make_solver, torch_cuda
    torch = torch_cuda()
    cfg = wl.config(cid, small=True)
    S = make_solver(cfg, precision=prec)
    rng = np.random.default_rng(11)
    n = S.ndof(-1)
    u0 = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    return S, u0, b


@pytest.mark.parametrize("cid,prec", [(2, dgfas.DGFAS_BF16), (2, dgfas.DGFAS_FP64),
                                      (1, dgfas.DGFAS_FP32), (3, dgfas.DGFAS_FP32)])
def test_every_candidate_shape_is_bit_identical(cid, prec):
    S, u0, b = _setup(cid, prec)
    ref = _vcycle(S, u0, b)
    tried = 0
    for level in range(S.n_levels):
        for kernel in range(4):
            cur, cands = S.dgfas_get_tuning(level, kernel)
            assert cur == 0
            for v in cands:
                S.dgfas_set_tuning(level, kernel, v)
                np.testing.assert_array_equal(_vcycle(S, u0, b), ref,
                                              err_msg=f"level {level} kernel {kernel} value {v}")
                tried += 1
            S.dgfas_set_tuning(level, kernel, 0)
    assert tried > 0


def test_autotune_keeps_a_candidate_and_results():
    S, u0, b = _setup(2, dgfas.DGFAS_BF16)
    ref = _vcycle(S, u0, b)
    rep = S.dgfas_autotune(reps=3)
    kinds = {r["kernel"] for r in rep}
    # the top level runs the FP64 and BF16-mode operators and the tensor-core FD;
    # the p = 4 level the narrow-subdomain FD
    assert {"apply_fp64_elements_per_cta", "apply_smoother_elements_per_cta",
            "fd_tensorcore_ctas_per_sm", "fd_elements_per_cta"} <= kinds
    for r in rep:
        k = S.TUNE_KERNELS.index(r["kernel"])
        cur, cands = S.dgfas_get_tuning(r["level"], k)
        assert cur == r["value"] and (cur == 0 or cur in cands)
        assert 0 < r["ms"] <= r["default_ms"] * 1.0000001
    np.testing.assert_array_equal(_vcycle(S, u0, b), ref)


def test_invalid_shape_is_rejected():
    S, _, _ = _setup(2, dgfas.DGFAS_BF16)
    with pytest.raises(dgfas.DgfasError) as e:
        S.dgfas_set_tuning(S.n_levels - 1, 0, 1000)
    assert e.value.code == -1   # DGFAS_ERR_INVALID
    with pytest.raises(dgfas.DgfasError):
        S.dgfas_set_tuning(0, 7, 1)
