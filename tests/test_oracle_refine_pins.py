"""Pins for the oracle's grid reversal by gradient descent (Sec. IV-A steps 2-5, Sec. IV-C).

The true coordinates are the global minimiser of L = ||F(x) - T||^2 when T is their own grid,
so descent from a perturbed start must converge to them.  That checks the sign of the
update, the factor 2 and the residual's orientation.  Starting at the truth must give loss 0
and no step.  The loss must fall monotonically for a small step size.  One step must equal
x - lr * gradient(W = 2 (F - T)) built from the separately pinned forward and gradient.
Molecules are independent, and the early stop at eps is honoured.
"""
import numpy as np
import pytest

import oracle
import synth


def problem(n_mol=4, form="point", seed=3, noise=0.1):
    wl = synth.plain_small(n_mol=n_mol)
    wl.form = form
    truth = oracle.Problem.from_workload(wl)
    T = oracle.voxelize(truth)
    start = wl.batch.coords.astype(np.float64) + np.random.default_rng(seed).normal(
        0.0, noise, wl.batch.coords.shape)
    return wl, truth, T, oracle.Problem.from_workload(wl, coords=start)


def test_starting_at_the_truth_gives_zero_loss_and_no_step(oracle_lib):
    wl, truth, T, _ = problem()
    x, loss, steps = oracle.refine(truth, T, iters=10, lr=0.02, eps=1e-30)
    assert np.all(loss == 0.0) and np.all(steps == 0)
    assert np.array_equal(x, truth.coords)


@pytest.mark.parametrize("form,lr,iters", [("point", 0.02, 400), ("integral", 5.0, 1200)])
def test_descent_recovers_the_true_coordinates(oracle_lib, form, lr, iters):
    # The erf form's values are smaller (peak ~ h^3 / (2 pi sigma^2)^{3/2}), so its stable
    # step is larger and its convergence slower.
    wl, truth, T, start = problem(form=form)
    x, loss, steps = oracle.refine(start, T, iters=iters, lr=lr)
    assert np.all(steps == iters)
    # Converged to the truth: the noise was 0.1 A, the residual error is below 1e-5 A (two
    # close atoms of one channel make the slowest mode).
    assert np.max(np.abs(x - truth.coords)) < 1e-5
    assert np.all(loss < 1e-10)


def test_loss_falls_monotonically(oracle_lib):
    wl, truth, T, start = problem(n_mol=2)
    losses = [oracle.refine(start, T, iters=t, lr=0.02)[1] for t in range(8)]
    L = np.array(losses)
    assert np.all(np.diff(L, axis=0) < 0.0)


def test_one_step_is_minus_lr_times_the_gradient_of_the_squared_error(oracle_lib):
    wl, truth, T, start = problem(n_mol=3)
    F = oracle.voxelize(start)
    g = oracle.gradient(start, 2.0 * (F - T))
    x1, loss0, steps = oracle.refine(start, T, iters=1, lr=0.02)
    assert np.all(steps == 1)
    assert np.allclose(x1, start.coords - 0.02 * g, rtol=0, atol=1e-14)


def test_molecules_are_independent_and_eps_stops_early(oracle_lib):
    wl, truth, T, start = problem(n_mol=4)
    x_all, loss_all, _ = oracle.refine(start, T, iters=20, lr=0.02)
    for b in range(4):
        sub = wl.batch.subset([b])
        s = wl.batch.atoms_of(b)
        pb = oracle.Problem.from_workload(wl, batch=sub, coords=start.coords[s])
        xb, lb, _ = oracle.refine(pb, T[b:b + 1], iters=20, lr=0.02)
        assert np.array_equal(xb, x_all[s]) and lb[0] == loss_all[b]
    eps = float(np.median(loss_all)) * 10.0
    x_eps, loss_eps, steps = oracle.refine(start, T, iters=20, lr=0.02, eps=eps)
    assert np.all((steps == 20) | (loss_eps < eps))
    assert np.any(steps < 20)
