"""The F-stage autotuner (psl1_autotune), through the C ABI: it picks the
inner CG tolerance per K bucket and the persistent grid by timing F stages,
writes its choices to a JSON-lines cache, and a second handle with the same
batch takes them from the cache without timing.  A tuned solve still reaches
the sequential solution at the mixed path's tolerance (1e-10)."""
import json

import numpy as np
import pytest

from paper_2510_11023_gb300 import psl1, workloads
from helpers import rel

pytestmark = pytest.mark.gpu


def test_autotune_writes_and_reuses_cache(tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    wl = workloads.cfg2(B=12, seed=5, P=8, kmin=24, kmax=200, mmin=4, mmax=8)
    with psl1.Problem(wl, precision="mixed") as pr:
        assert pr.autotune(cache) is False
        first = [pr.tuning(b) for b in range(wl.B)]
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.set_graph(True)
        pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U[b], S[b]) < 1e-10, b
        assert first[b]["inner_rtol"] in (np.float32(1e-7), np.float32(1e-5), np.float32(3e-4))
    lines = [json.loads(l) for l in open(cache)]
    keys = [l["key"] for l in lines]
    assert any("fstage_ctas_per_sm" in k for k in keys) and any("inner_rtol" in k for k in keys)
    with psl1.Problem(wl, precision="mixed") as pr:
        assert pr.autotune(cache) is True
        assert [pr.tuning(b) for b in range(wl.B)] == first
    assert len(open(cache).readlines()) == len(lines)   # nothing new appended
