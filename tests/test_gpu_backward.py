"""GPU parity of the coordinate adjoint (Sec. IV-C) through the C ABI and autograd:
against the oracle gradient, against FP64 central finite differences with frozen
support, for every cutoff/boundary mode and grad dtype, and sampled at full size on the
differentiation workload (loss <W, G>, W ~ N(0,1))."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import GRAD_TOL, grad_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api
    return api


def _grad(pg, wl, W, batch=None, dtype=torch.float32):
    batch = wl.batch if batch is None else batch
    db = pg.DeviceBatch.from_numpy(batch)
    g = pg.voxelize_backward(db, pg.Grid.from_workload(wl),
                             torch.as_tensor(W, device="cuda").to(dtype))
    assert pg.sync_status() == 0
    return g.cpu().numpy()


@pytest.mark.parametrize("cutoff,periodic", [("sphere", False), ("box", False),
                                             ("none", False), ("sphere", True),
                                             ("box", True), ("none", True)])
def test_gradient_matches_oracle(pg, cutoff, periodic):
    wl = synth.differentiation(n_mol=12)
    wl.cutoff, wl.periodic = cutoff, periodic
    if periodic:
        wl.cutoff_k = 2.5
    W = synth.loss_weights(wl)
    prob = oracle.Problem.from_workload(wl)
    g_ref = oracle.gradient(prob, W)
    grad_check(_grad(pg, wl, W), g_ref, wl.batch.mol_off)
    fd = oracle.fd_gradient_frozen(prob, W, 1e-4)
    # oracle pinned to FD at 1e-6; the GPU result then sits within 1e-4 of FD too
    grad_check(_grad(pg, wl, W), fd, wl.batch.mol_off, rel_tol=GRAD_TOL + 1e-6)


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_half_precision_upstream_gradient(pg, dtype):
    wl = synth.differentiation(n_mol=6)
    W = synth.loss_weights(wl)
    Wq = torch.as_tensor(W).to(dtype).float().numpy()  # oracle sees the rounded weights
    g_ref = oracle.gradient(oracle.Problem.from_workload(wl), Wq)
    grad_check(_grad(pg, wl, W, dtype=dtype), g_ref, wl.batch.mol_off)


def test_autograd_function_matches_direct_call_and_loss(pg):
    wl = synth.differentiation(n_mol=8)
    W = torch.as_tensor(synth.loss_weights(wl), device="cuda")
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    x = db.coords.clone().requires_grad_(True)
    G = pg.voxelize_autograd(x, db, grid)
    loss = (W * G).sum()
    loss.backward()
    loss64 = float((W.double() * G.detach().double()).sum())
    direct = pg.voxelize_backward(db, grid, W)
    torch.cuda.synchronize()
    assert torch.equal(x.grad, direct)
    prob = oracle.Problem.from_workload(wl)
    assert loss64 == pytest.approx(oracle.loss(prob, W.cpu().numpy()), rel=1e-5)


def test_gradient_deterministic_and_stray_atoms_zeroed(pg):
    wl = synth.differentiation(n_mol=10)
    W = synth.loss_weights(wl)
    a = _grad(pg, wl, W)
    b = _grad(pg, wl, W)
    assert np.array_equal(a, b)
    # Atoms past the last molecule's range get a zero gradient.
    bt = wl.batch
    extra = synth.Batch(np.concatenate([bt.coords, bt.coords[:3]]),
                        np.concatenate([bt.elem, bt.elem[:3]]), bt.mol_off, bt.origin,
                        bt.spacing)
    g = _grad(pg, wl, W, batch=extra)
    assert np.all(g[-3:] == 0.0)
    np.testing.assert_array_equal(g[:-3], a)


def test_differentiation_full_size_sampled(pg):
    wl = synth.differentiation()
    n = wl.batch.n_mol
    W = torch.as_tensor(synth.loss_weights(wl), device="cuda")
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    x = db.coords.clone().requires_grad_(True)
    G = pg.voxelize_autograd(x, db, grid)
    (W * G).sum().backward()
    torch.cuda.synchronize()
    assert pg.sync_status() == 0
    idx = np.sort(np.random.default_rng(15).choice(n, 32, replace=False))
    sub = wl.batch.subset(idx)
    prob = oracle.Problem.from_workload(wl, batch=sub)
    Ws = W[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    rows = np.concatenate([np.arange(wl.batch.mol_off[i], wl.batch.mol_off[i + 1]) for i in idx])
    g_gpu = x.grad[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    grad_check(g_gpu, oracle.gradient(prob, Ws), sub.mol_off)
    grad_check(g_gpu, oracle.fd_gradient_frozen(prob, Ws, 1e-4), sub.mol_off,
               rel_tol=GRAD_TOL + 1e-6)
