"""The uneven batch at full size: 64 seeded jobs, N in {256, 384, 512, 768},
M = 1.5 N angles, N bins, S ~ U{1..32}, noisy ellipse phantoms, 20 CGLS
iterations in one batched call (mixed precision, binary16 storage).  Each
job equals, bit for bit, the plain solver on its geometry's concatenated
slices; one N = 256 job is checked against the FP64 oracle over the stable
phase (4 iterations)."""
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


@pytest.fixture(scope="module")
def batch():
    jobs = inputs.batch_jobs()
    with ProcessPoolExecutor(max_workers=8, mp_context=get_context("spawn")) as ex:
        sinos = list(ex.map(inputs.job_sinograms, jobs))
    return jobs, [s.astype(np.float32) for s in sinos]


def test_full_batch(xct, batch):
    jobs, sinos = batch
    K = inputs.BATCH["iters"]
    sizes = sorted({j["n"] for j in jobs})
    assert sizes == [256, 384, 512, 768]
    plans = {n: xct.Plan(n, 3 * n // 2, n, "f16", cos_sin=inputs.angle_table(3 * n // 2)) for n in sizes}
    try:
        ys = [torch.tensor(s, device="cuda") for s in sinos]
        xs = [torch.empty((j["slices"], j["n"], j["n"]), device="cuda") for j in jobs]
        x4 = [torch.empty_like(x) for x in xs]
        xct.xct_cgls_batch([(plans[j["n"]].handle, ys[i], xs[i], j["slices"]) for i, j in enumerate(jobs)], K)
        xct.xct_cgls_batch([(plans[j["n"]].handle, ys[i], x4[i], j["slices"]) for i, j in enumerate(jobs)], 4)
        for n in (256, 768):
            idx = [i for i, j in enumerate(jobs) if j["n"] == n]
            xg = plans[n].cgls(torch.cat([ys[i] for i in idx]), K)
            o = 0
            for i in idx:
                S = jobs[i]["slices"]
                assert torch.equal(xs[i], xg[o:o + S]), (n, i)
                o += S
        assert all(bool(torch.isfinite(x).all()) for x in xs)
        i = next(i for i, j in enumerate(jobs) if j["n"] == 256)
        j = jobs[i]
        pick = list(range(min(2, j["slices"])))
        g = oracle.Geometry(n=j["n"], m=j["m"], nd=j["nd"], cos_sin=inputs.angle_table(j["m"]))
        a = oracle.siddon_csr(g)
        at = oracle.transpose(a)
        xo, _ = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y),
                            sinos[i].reshape(j["slices"], -1)[pick].astype(np.float64), 4)
        got = x4[i].reshape(j["slices"], -1)[pick].double().cpu().numpy()
        assert np.linalg.norm(got - xo) / np.linalg.norm(xo) <= 2e-3
    finally:
        for p in plans.values():
            p.close()
