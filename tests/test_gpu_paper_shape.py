"""The paper's model problem shape (Sec. 4.2): D = 1 + u, f = sin(pi x) e^{-t},
u0 = x^4 (1-x)^4 (projected), alpha = 0.5, 2^4 modes, P = 2^8 slices, m = 2^5
fine steps per slice (N = 8192).  GPU serial solvers and parareal against the
CPU oracle, both precisions; parareal must converge to the serial hybrid
solution (its fixed point, Eq. PararealConvergence)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_paper_model_problem_shape(prec):
    wl = workloads.e1()
    spec, u0 = wl.specs[0], wl.u0[0]
    op = oracle_prob(spec, wl.P)
    S_or = O.serial_hyb(op, u0)
    W_or = O.serial_uni(op, u0)[:: op.m]
    with psl1.Problem(wl, precision=prec) as pr:
        pr.set_graph(True)
        k = pr.solve_parareal(tol=1e-10)
        U = pr.get_coeffs("parareal")[0]
        log = pr.get_errlog(0)
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        pr.solve_serial("uniform")
        W = pr.get_coeffs("serial")[0]
    assert rel(S, S_or) < 1e-10
    assert rel(W, W_or) < 1e-10
    assert rel(U, S) < 1e-9
    assert 1 <= k < wl.P and log[-1] <= 1e-10
    # increments decrease geometrically once parareal is in its convergence regime
    assert log[-1] < 1e-3 * log[0]
