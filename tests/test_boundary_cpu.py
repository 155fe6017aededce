"""CPU checks of the C-ABI library: it loads, exports every symbol declared in
include/dgfas.h, and its host-side setup (fast-diagonalization tables of
Sec. 4.3.1) agrees with the oracle.  No device work."""
import os
import re

import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from oracle import schwarz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"\b(dgfas_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = dgfas.load()
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(dgfas.SYMBOLS)


def test_strerror_codes():
    lib = dgfas.load()
    for code in range(-7, 1):
        assert lib.dgfas_strerror(code)
    assert lib.dgfas_strerror(-5) == b"not converged within max_cycles"


@pytest.mark.parametrize("p,delta", [(1, .08), (2, .08), (4, .08), (7, .08), (8, .08), (8, .16), (10, .08)])
def test_host_fd_tables_match_oracle(p, delta):
    mu = 5.0
    T = schwarz.FDTables(p, delta, mu)
    rng = np.random.default_rng(p)
    for v, name in enumerate(schwarz.VARIANTS16):
        S, lam, W = dgfas.dgfas_host_fd_variant(p, delta, mu, v)
        t = T.tab[name]
        assert S.shape == t["S"].shape
        np.testing.assert_allclose(np.sort(lam), np.sort(t["lam"]), rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(W, t["W"], rtol=0, atol=1e-15)
        # the FD inverse S diag(1/(g0 + g lam)) S^T is unique (eigenvector signs drop out)
        g0, g1 = 0.3, 1.7
        A = S @ np.diag(1.0 / (g0 + g1 * lam)) @ S.T
        B = t["S"] @ np.diag(1.0 / (g0 + g1 * t["lam"])) @ t["S"].T
        np.testing.assert_allclose(A, B, rtol=1e-10, atol=1e-12 * np.abs(B).max())


def test_host_fd_rejects_bad_arguments():
    with pytest.raises(dgfas.DgfasError):
        dgfas.dgfas_host_fd_variant(11, 0.08, 5.0, 0)
    with pytest.raises(dgfas.DgfasError):
        dgfas.dgfas_host_fd_variant(4, 0.08, 5.0, 16)
    with pytest.raises(dgfas.DgfasError):
        dgfas.dgfas_host_fd_variant(4, 0.6, 5.0, 0)


def test_binding_rejects_wrong_dtype_and_short_vectors_before_any_launch():
    """The binding checks element type and length of every vector argument on
    the host: a float32 or short tensor where the kernels expect FP64 of the
    level's size raises before the library is called."""
    import torch
    with pytest.raises(TypeError):
        dgfas._ptr(torch.zeros(16, dtype=torch.float32), 16)
    with pytest.raises(ValueError):
        dgfas._ptr(torch.zeros(8, dtype=torch.float64), 16)
    with pytest.raises(TypeError):
        dgfas._ptr(torch.zeros(16, dtype=torch.float64), 16, "float32")
    with pytest.raises(ValueError):   # right type and size, but host memory
        dgfas._ptr(torch.zeros(16, dtype=torch.float64), 16)
    assert dgfas._ptr(None, 16) is None
