"""GPU checks of the learned surrogate: the CUDA MLP kernels against the FP64
oracle network, training on the oracle's Kronecker-sum fits, and the effect of
the learned coefficients on the multigrid convergence."""
import os

import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import mlp as omlp
from tests.gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


N_SET = 100000


def _targets(p):
    """The oracle's fits of the seeded training set (written by
    oracle/make_surrogate_data.py): validity mask and targets."""
    d = np.load(os.path.join(GOLD, f"surrogate_fits_p{p}_n{N_SET}.npz"))
    return d["ok"], d["Y"]


def _corners(p):
    ok, _ = _targets(p)
    return wl.surrogate_training_set(N_SET, p)[ok]


def _data(p, n=None):
    """Inputs (computed by the library from the regenerated corners) and
    targets of the first n valid training elements (all if None)."""
    from paper_2608_14123_b300 import learned
    ok, Y = _targets(p)
    cr = _corners(p)[:n]
    X = learned.inputs(cr).cpu().numpy()
    return X, Y[:len(cr)]


def _oracle_data(p, n):
    from oracle import surrogate as su
    _, Y = _targets(p)
    return su.mlp_inputs(_corners(p)[:n]).astype(np.float32), Y[:n]


def test_library_inputs_match_oracle():
    """The library's input kernel (normalized corners) against the oracle's."""
    X, _ = _data(7, 512)
    Xo, _ = _oracle_data(7, 512)
    assert np.abs(X - Xo).max() <= 1e-6 * max(1.0, np.abs(Xo).max())


def test_forward_and_gradient_match_oracle():
    torch = torch_cuda()
    from paper_2608_14123_b300 import learned
    X, Y = _oracle_data(7, 512)
    th = learned.init_params(3)
    thd, Xd, Yd = (torch.from_numpy(a).cuda() for a in (th, X, Y))
    out = learned.forward(thd, Xd).cpu().numpy()
    ref, _ = omlp.forward(th.astype(np.float64), X.astype(np.float64))
    assert np.abs(out - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    g = learned.grad(thd, Xd, Yd).cpu().numpy()
    gr = omlp.grad(th.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    # per layer relative error (FP32 kernels vs FP64 oracle)
    sizes = omlp.SIZES
    o = 0
    for i in range(len(sizes) - 1):
        n = sizes[i + 1] * sizes[i] + sizes[i + 1]
        a, b = g[o:o + n], gr[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), i
        o += n


def test_one_adam_step_matches_oracle():
    torch = torch_cuda()
    from paper_2608_14123_b300 import learned
    X, Y = _oracle_data(7, 256)
    th = learned.init_params(5)
    thd = torch.from_numpy(th).cuda()
    th1, _ = learned.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=1,
                           batch=256, lr=1e-3, seed=7, params=thd)
    g = omlp.grad(th.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    ref, _, _ = omlp.adam_step(th.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1)
    # first Adam step moves every weight by ~lr * sign(g); FP32 sums may flip tiny gradients
    d = np.abs(th1.cpu().numpy() - ref)
    assert np.mean(d < 1e-5) > 0.98 and d.max() <= 2.1e-3


def test_training_fits_the_oracle_targets():
    """Training on 9 10^4 of the 10^5 oracle fits: on the held-out 10^4 (the
    near-cubic elements of the uniform workload's distribution, whose fitted
    scalings are close to the geometric ones) the predicted log scalings have
    a clearly smaller mean squared error than the geometric surrogate's
    log s = 0 (measured on the B300: 0.56 of it)."""
    torch = torch_cuda()
    from paper_2608_14123_b300 import learned
    X, Y = _data(7)
    n_tr = len(X) - 10000
    Xd, Yd = torch.from_numpy(X[:n_tr]).cuda(), torch.from_numpy(Y[:n_tr]).cuda()
    th, loss = learned.train(Xd, Yd, epochs=80, batch=256, lr=2e-3, seed=11)
    assert loss[-1] < 0.25 * loss[0]
    # held-out samples: the predicted log scalings beat the geometric surrogate (log s = 0)
    out = learned.forward(th, torch.from_numpy(X[n_tr:]).cuda()).cpu().numpy()
    err_learned = np.mean((out[:, 3:] - Y[n_tr:, 3:]) ** 2)
    err_geo = np.mean(Y[n_tr:, 3:] ** 2)
    assert err_learned < 0.7 * err_geo


def test_learned_surrogate_improves_multigrid_convergence():
    """Perturbed 4^3 mesh (vertices moved by up to 0.25 h) at p = 3: with the
    geometric surrogate the V-cycle with the Schwarz smoother diverges there,
    with the learned surrogate it converges."""
    torch = torch_cuda()
    from paper_2608_14123_b300 import dgfas, learned
    X, Y = _data(3)
    th, _ = learned.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=40,
                          batch=256, lr=2e-3, seed=11)
    V = wl.perturbed_vertices(4, 0.25, np.random.default_rng(1))
    levels = wl.hierarchy(V, [3, 1])
    rates = {}
    for mode in ("geometric", "learned"):
        S = dgfas.Solver(levels, 10.0, 0.08, 2, 2, 4, precision=dgfas.DGFAS_FP64)
        if mode == "learned":
            nf = S.dgfas_learned_surrogate(-1, th)
            assert nf < S.ndof(-1) // 64 // 4       # few fallbacks
        rng = np.random.default_rng(2)
        b = torch.from_numpy(rng.standard_normal(S.ndof(-1))).cuda()
        u = torch.from_numpy(rng.uniform(-1, 1, S.ndof(-1))).cuda()
        info = S.dgfas_solve(u, b, 1e-8, 12, raise_on_fail=False)
        h = info["history"]
        rates[mode] = (h[-1] / h[0]) ** (1.0 / max(1, len(h) - 1))
    assert rates["geometric"] > 1.0
    assert rates["learned"] < 0.9
