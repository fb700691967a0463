"""CUDA-graph execution: parareal as one graph with a device-driven while loop
(conditional node) must give the same iterates, iteration counts and increment
logs as the host loop -- the kernels are the same and deterministic -- and the
uniform serial solver, captured once per handle, must replay to the oracle's
result."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu


def _solve(wl, prec, graph, tol, mlp=None):
    with psl1.Problem(wl, precision=prec) as pr:
        if mlp is not None:
            pr.set_coarse(mlp)
        pr.set_graph(graph)
        pr.solve_parareal(tol=tol, allow_not_converged=True)
        U = pr.get_coeffs("parareal", flat=True)
        its = pr.get_iterations()
        logs = [pr.get_errlog(b) for b in range(wl.B)]
        st = pr.stats()
        # a second solve on the same handle replays the graph
        pr.solve_parareal(tol=tol, allow_not_converged=True)
        U2 = pr.get_coeffs("parareal", flat=True)
    return U, its, logs, st, U2


@pytest.mark.parametrize("case", ["1d-mixed", "1d-fp64", "2d-mixed"])
def test_graph_parareal_equals_host_loop(case):
    wl = workloads.small_batch_2d() if case.startswith("2d") else workloads.small_batch()
    prec = case.split("-")[1]
    Uh, ih, lh, sh, _ = _solve(wl, prec, False, 1e-11)
    Ug, ig, lg, sg, Ug2 = _solve(wl, prec, True, 1e-11)
    assert np.array_equal(ih, ig)
    assert np.array_equal(Uh, Ug)          # bitwise: same kernels, same order
    assert np.array_equal(Ug, Ug2)
    for a, b in zip(lh, lg):
        assert np.array_equal(a, b)
    assert sg["fine_steps"] == sh["fine_steps"]
    assert sg["flop_fine"] == pytest.approx(sh["flop_fine"], rel=1e-12)


def test_graph_parareal_rebuilt_after_coarse_propagator_change():
    wl = workloads.cfg1(K=12, N=48, P=6, alpha=0.45)
    with psl1.MLP(12, 4, 16, 12, seed=5) as mlp:
        rng = np.random.default_rng(3)
        mlp.set_params((0.3 * rng.standard_normal(mlp.nparams)).astype(np.float32),
                       (1e-2 * (1 + rng.random(mlp.nout))).astype(np.float32))
        Uh, ih, _, _, _ = _solve(wl, "fp64", False, 1e-12, mlp)
        with psl1.Problem(wl) as pr:
            pr.set_graph(True)
            pr.solve_parareal(tol=1e-12)
            plain = pr.get_coeffs("parareal", flat=True)
            pr.set_coarse(mlp)                      # invalidates the graph's kernel arguments
            pr.solve_parareal(tol=1e-12)
            learned = pr.get_coeffs("parareal", flat=True)
            its = pr.get_iterations()
    assert np.array_equal(learned, Uh) and np.array_equal(its, ih)
    assert rel(plain, learned) < 1e-10 and not np.array_equal(plain, learned)


def test_graph_parareal_respects_max_iter_and_keep_iterates():
    wl = workloads.cfg1(K=16, N=48, P=6)
    with psl1.Problem(wl) as pr:
        pr.set_graph(True)
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.solve_parareal(tol=1e-15, max_iter=2)
        assert ei.value.status == -6 and pr.get_iterations()[0] == 2
        pr.keep_iterates(True)                       # falls back to the host loop
        k = pr.solve_parareal(tol=0.0)
        assert k == wl.P and rel(pr.get_iterate(k)[0], pr.get_coeffs("parareal")[0]) == 0.0


@pytest.mark.parametrize("wl", [workloads.cfg1(K=24, N=96, P=8), workloads.small_batch_2d()],
                         ids=["1d", "2d"])
def test_uniform_solver_graph_replays(wl):
    with psl1.Problem(wl, precision="fp64") as pr:
        pr.solve_serial("uniform")
        W1 = pr.get_coeffs("serial")
        assert pr.stats()["kernel_launches"] == 2 * max(s.nsteps for s in wl.specs)
        pr.solve_serial("uniform")
        W2 = pr.get_coeffs("serial")
    for b, spec in enumerate(wl.specs):
        op = oracle_prob(spec, wl.P)
        assert np.array_equal(W1[b], W2[b])
        assert rel(W1[b], O.serial_uni(op, wl.u0[b])[:: op.m]) < 1e-10
