"""The learned coarse correction on the GPU: network forward, gradients and Adam
against the FP64 CPU oracle (evaluated with the same BF16-rounded weights),
the learned coarse sweep against the oracle's, and parareal's finite
termination with a learned G.  Tolerances: forward 1e-4, gradients 1e-3
(FP32 activations vs FP64), Adam 1e-5, learned coarse sweep 1e-10 relative
(the in-sweep inference accumulates in double-float)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu


def bf16_round(x):
    import torch
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def oracle_params(mlp: psl1.MLP, p32):
    """The device's effective parameters: BF16 weights, FP32 biases."""
    p = p32.astype(np.float64).copy()
    din = [mlp.nin, mlp.width, mlp.width, mlp.width]
    dout = [mlp.width, mlp.width, mlp.width, mlp.nout]
    o = 0
    for l in range(4):
        nw = din[l] * dout[l]
        p[o:o + nw] = bf16_round(p32[o:o + nw])
        o += nw + dout[l]
    return p


def randomise(mlp: psl1.MLP, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = (scale * rng.standard_normal(mlp.nparams)).astype(np.float32)
    s = (1e-2 * (1 + rng.random(mlp.nout))).astype(np.float32)
    mlp.set_params(p, s)
    return p, s


@pytest.mark.parametrize("dims", [(12, 4, 16, 12), (128, 32, 512, 128)])
def test_forward_and_gradients_match_oracle(dims):
    nU, nH, W, nout = dims
    with psl1.MLP(nU, nH, W, nout, seed=3) as mlp:
        p32, _ = randomise(mlp, 7, scale=1.0 / np.sqrt(W))
        po = oracle_params(mlp, p32)
        rng = np.random.default_rng(1)
        z = rng.standard_normal((5, mlp.nin)).astype(np.float32)
        t = rng.standard_normal((5, nout)).astype(np.float32)
        y = mlp.forward(z)
        yo = O.mlp_forward(po, mlp.nin, W, nout, z.astype(np.float64))
        assert rel(y, yo) < 1e-4
        g, loss = mlp.loss_grad(z, t)
        go, lo = O.mlp_backward(po, mlp.nin, W, nout, z.astype(np.float64), t.astype(np.float64))
        assert abs(loss - lo) < 1e-4 * abs(lo)
        assert rel(g, go) < 1e-3


def test_adam_step_matches_oracle():
    with psl1.MLP(6, 2, 8, 5, seed=1) as mlp:
        p0, _ = mlp.get_params()
        rng = np.random.default_rng(2)
        g1 = rng.standard_normal(mlp.nparams).astype(np.float32)
        g2 = rng.standard_normal(mlp.nparams).astype(np.float32)
        mlp.adam_step(g1, 1e-2)
        mlp.adam_step(g2, 5e-3)
        p, _ = mlp.get_params()
        po = p0.astype(np.float64)
        m, v = np.zeros_like(po), np.zeros_like(po)
        O.adam_step(po, g1.astype(np.float64), m, v, 1, lr=1e-2)
        O.adam_step(po, g2.astype(np.float64), m, v, 2, lr=5e-3)
        assert np.abs(p - po).max() < 1e-5 * max(1.0, np.abs(po).max())


def _mlp_dict(mlp, po, s):
    return {"params": po, "oscale": s.astype(np.float64), "nU": mlp.nU, "nH": mlp.nH, "width": mlp.width,
            "nout": mlp.nout}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("K", [12, 8, 20])   # K = nU, K < nU (zero features), K > nout
def test_learned_coarse_sweep_matches_oracle(prec, K):
    wl = workloads.cfg1(K=K, N=24, P=6, alpha=0.45)
    op = oracle_prob(wl.specs[0], wl.P)
    with psl1.MLP(12, 4, 16, 12, seed=5) as mlp, psl1.Problem(wl, precision=prec) as pr:
        p32, s = randomise(mlp, 11)
        pr.set_coarse(mlp)
        pr.solve_serial("coarse")
        G = pr.get_coeffs("serial")[0]
        Go = O.coarse_sweep(op, wl.u0[0], mlp=_mlp_dict(mlp, oracle_params(mlp, p32), s))
        plain = O.coarse_sweep(op, wl.u0[0])
        assert rel(Go, plain) > 1e-4          # the correction is active
        assert rel(G, Go) < 1e-10
        pr.set_coarse(None)
        pr.solve_serial("coarse")
        assert rel(pr.get_coeffs("serial")[0], plain) < 1e-10


def test_parareal_with_learned_g_terminates_at_serial_solution():
    wl = workloads.cfg1(K=16, N=48, P=6, alpha=0.6)
    with psl1.MLP(16, 4, 16, 16, seed=9) as mlp, psl1.Problem(wl, precision="fp64") as pr:
        randomise(mlp, 13)
        pr.set_coarse(mlp)
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=0.0)
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        for j in range(k + 1):
            Uj = pr.get_iterate(j)[0]
            assert np.abs(Uj[: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j


def test_trained_network_gains_over_plain_l1_coarse_propagator():
    # what the learned correction buys: trained on the (z(U^k_{0:n}), F - G) pairs of six
    # parareal iterations on 96 training instances, it lowers the parareal error after a
    # fixed number of iterations on 8 held-out instances (same PDE family, new u0, alpha).
    K, N, P = 64, 1024, 32
    tr = workloads.cfg4_trajectories(96, seed=20251013, K=K, N=N, P=P)
    ho = workloads.cfg4_trajectories(8, seed=20251014, K=K, N=N, P=P)
    with psl1.Problem(tr, precision="mixed") as data, psl1.MLP(K, 32, 256, K, seed=1) as mlp:
        mlp.dataset(data, iterates=6)
        log = mlp.train(data, epochs=60, batch=512, lr=1e-3, seed=2)
        assert log[-1] < 0.2 * log[0]
        with psl1.Problem(ho, precision="mixed") as pr:
            pr.solve_serial("hybrid")
            S = pr.get_coeffs("serial")
            errs = {}
            for name, m in (("L1", None), ("learned", mlp)):
                pr.set_coarse(m)
                pr.keep_iterates(True)
                pr.solve_parareal(tol=0.0, max_iter=5, allow_not_converged=True)
                errs[name] = [max(float(np.sqrt(((u - s) ** 2).sum(1)).max() / np.sqrt((s ** 2).sum(1)).max())
                                  for u, s in zip(pr.get_iterate(k), S)) for k in range(6)]
    print("parareal error per iteration", errs)
    assert errs["learned"][4] < 0.5 * errs["L1"][4]
    assert errs["learned"][5] < 0.5 * errs["L1"][5]
