"""Batched solve of uneven jobs (xct_cgls_batch): jobs of three geometries and
uneven slice counts, where geometries with the same slice-tile width share
one persistent launch per product phase.  Each job's result must equal, bit for bit, the plain solver
run on its geometry group's concatenated slices (same slice-tile width, so
the same arithmetic in the same order); the stable phase is also checked
against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu

GEOMS = {"A": (64, 96, 64, 0.0), "B": (48, 72, 50, 0.3), "C": (80, 120, 80, 0.0)}
JOBS = [("A", 3), ("B", 1), ("A", 17), ("C", 64), ("B", 40), ("A", 9)]


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


def _sinos(key, S, seed):
    n, m, nd, off = GEOMS[key]
    cs = inputs.angle_table(m)
    ells = inputs.random_ellipsoids(np.random.default_rng(seed), 12)
    out = np.stack([inputs.line_integrals(inputs.cut_ellipsoids(ells, inputs.slice_z(s, S)), n, cs, nd,
                                          offset=off) for s in range(S)])
    for s in range(S):
        out[s] = inputs.poisson_noise(np.random.default_rng(seed * 100 + s), out[s], n, 1e4)
    return out.astype(np.float32)


@pytest.mark.parametrize("kind", ["f16", "f32", "f16-paired"])
def test_batch_equals_grouped_solves(xct, kind):
    """f16-paired: binary16 plans with paired layouts; groups B and C run
    64-slice tiles on them, in one launch per product phase."""
    iters = 12
    storage, paired = kind.split("-")[0], kind.endswith("-paired")
    plans = {k: xct.Plan(n, m, nd, storage, cos_sin=inputs.angle_table(m), det_offset=off,
                         paired_rows=paired)
             for k, (n, m, nd, off) in GEOMS.items()}
    try:
        ys = [torch.tensor(_sinos(k, S, 10 + i), device="cuda") for i, (k, S) in enumerate(JOBS)]
        xs = [torch.full((S, GEOMS[k][0], GEOMS[k][0]), float("nan"), device="cuda") for k, S in JOBS]
        logs = [torch.zeros((iters + 1, S, 2), dtype=torch.float64, device="cuda") for _, S in JOBS]
        xct.xct_cgls_batch([(plans[k].handle, ys[i], xs[i], S, logs[i]) for i, (k, S) in enumerate(JOBS)],
                           iters)
        torch.cuda.synchronize()
        for key in GEOMS:
            idx = [i for i, (k, _) in enumerate(JOBS) if k == key]
            yg = torch.cat([ys[i] for i in idx])
            xg, lg = plans[key].cgls(yg, iters, resid=True)
            o = 0
            for i in idx:
                S = JOBS[i][1]
                assert torch.equal(xs[i], xg[o:o + S]), (key, i)
                assert torch.equal(logs[i], lg[:, o:o + S]), (key, i)
                o += S
    finally:
        for p in plans.values():
            p.close()


def test_batch_stable_phase_vs_oracle(xct):
    key, S = "B", 5
    n, m, nd, off = GEOMS[key]
    cs = inputs.angle_table(m)
    y = _sinos(key, S, 3)
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs, det_offset=off)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    xr, _ = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y),
                        y.reshape(S, -1).astype(np.float64), 4)
    with xct.Plan(n, m, nd, "f32", cos_sin=cs, det_offset=off) as p32, \
            xct.Plan(n, m, nd, "f16", cos_sin=cs, det_offset=off) as p16:
        yt = torch.tensor(y, device="cuda")
        x32 = torch.empty((S, n, n), device="cuda")
        x16 = torch.empty((S, n, n), device="cuda")
        xct.xct_cgls_batch([(p32.handle, yt, x32, S), (p16.handle, yt, x16, S)], 4)
    for x, tol in ((x32, 2e-5), (x16, 2e-3)):
        got = x.cpu().numpy().reshape(S, -1)
        assert np.linalg.norm(got - xr) / np.linalg.norm(xr) <= tol


def test_batch_autotune_and_graphless(xct):
    key, S = "A", 24
    n, m, nd, off = GEOMS[key]
    y = torch.tensor(_sinos(key, S, 4), device="cuda")
    with xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m)) as p:
        x1 = torch.empty((S, n, n), device="cuda")
        x2 = torch.empty((S, n, n), device="cuda")
        xct.xct_cgls_batch([(p.handle, y, x1, S)], 6, xct.XCT_BATCH_AUTOTUNE)
        xct.xct_cgls_batch([(p.handle, y, x2, S)], 6, xct.XCT_BATCH_AUTOTUNE | xct.XCT_CGLS_NO_GRAPH)
        assert torch.isfinite(x1).all()
        assert torch.equal(x1, x2)          # same cached tile width, graph or not
    with pytest.raises(xct.XctError):
        xct.xct_cgls_batch([(0, y, x1, S)], 3)
