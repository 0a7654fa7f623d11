"""GPU projection / back projection vs the oracle, element by element.

FP32 storage: relative L2 error <= 1e-5 against the FP64 oracle, and each
output within 1e-5 of the sum of |a_e x_e| over its row (FP32 accumulation
over at most 2n+2 terms).  Mixed storage: against the oracle's model of the
16-bit semantics (same rounding of matrix and inputs, exact sums), same
bounds, plus the error against FP64 reported and bounded by the 16-bit unit
roundoff.  Sizes span several thread blocks and stages with ragged tails;
slice counts span several slice tiles with a ragged last tile."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_07226_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct as x
    return x


_cache = {}


def _setup(n, m, nd, off=0.0, sp=1.0):
    key = (n, m, nd, off, sp)
    if key not in _cache:
        g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=inputs.angle_table(m), det_offset=off,
                            det_spacing=sp)
        a = oracle.siddon_csr(g)
        at = oracle.transpose(a)
        absa = oracle.CSR(a.nrow, a.ncol, a.rowptr, a.col, np.abs(a.val))
        absat = oracle.CSR(at.nrow, at.ncol, at.rowptr, at.col, np.abs(at.val))
        _cache[key] = (g, a, at, absa, absat)
    return _cache[key]


def _check(got, want, bound, rel_l2=1e-5):
    got = np.asarray(got, dtype=np.float64).reshape(want.shape)
    nrm = np.linalg.norm(want)
    if nrm > 0:
        assert np.linalg.norm(got - want) / nrm <= rel_l2
    assert np.all(np.abs(got - want) <= 1e-5 * bound + 1e-30)


CASES = [
    # n, m, nd, S, off, spacing
    (8, 8, 8, 1, 0.0, 1.0),
    (32, 45, 32, 3, 0.13, 1.0),
    (37, 23, 41, 5, -0.4, 0.9),
    (64, 96, 64, 17, 0.0, 1.0),
    (128, 180, 128, 1, 0.0, 1.0),
    (128, 180, 128, 33, 0.0, 1.0),
    (96, 64, 100, 64, 0.25, 1.0),
    (96, 64, 100, 65, 0.25, 1.0),
    (1, 1, 1, 2, 0.0, 1.0),
    (9, 7, 30, 4, 0.5, 1.0),
]


@pytest.mark.parametrize("n,m,nd,S,off,sp", CASES)
def test_f32_products_vs_oracle(xct, n, m, nd, S, off, sp):
    g, a, at, absa, absat = _setup(n, m, nd, off, sp)
    rng = np.random.default_rng(n * 1000 + S)
    x = rng.uniform(-1, 1, size=(S, n * n))
    y = rng.uniform(-1, 1, size=(S, m * nd))
    dev = torch.device("cuda")
    with xct.Plan(n, m, nd, "f32", cos_sin=g.table(), det_offset=off, det_spacing=sp) as p:
        xt = torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device=dev)
        yt = torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device=dev)
        yo = torch.full((S, m, nd), float("nan"), device=dev)   # poisoned outputs
        xo = torch.full((S, n, n), float("nan"), device=dev)
        p.project(xt, out=yo)
        p.backproject(yt, out=xo)
        torch.cuda.synchronize()
        x32 = x.astype(np.float32).astype(np.float64)
        y32 = y.astype(np.float32).astype(np.float64)
        _check(yo.cpu().numpy(), oracle.project(a, x32), oracle.project(absa, np.abs(x32)))
        _check(xo.cpu().numpy(), oracle.backproject(at, y32), oracle.backproject(absat, np.abs(y32)))


@pytest.mark.parametrize("kind", ["f16", "bf16", "f16a", "bf16a"])
@pytest.mark.parametrize("n,m,nd,S,off,sp", [CASES[1], CASES[2], CASES[3], CASES[6], CASES[7], CASES[9]])
def test_mixed_products_vs_oracle_model(xct, kind, n, m, nd, S, off, sp):
    g, a, at, absa, absat = _setup(n, m, nd, off, sp)
    rng = np.random.default_rng(7 * n + S)
    # slices of very different magnitudes exercise the per-slice normalisation
    mag = 10.0 ** rng.uniform(-3, 3, size=(S, 1))
    x = rng.uniform(-1, 1, size=(S, n * n)) * mag
    y = rng.uniform(-1, 1, size=(S, m * nd)) * mag
    dev = torch.device("cuda")
    with xct.Plan(n, m, nd, kind, cos_sin=g.table(), det_offset=off, det_spacing=sp) as p:
        yo = p.project(torch.tensor(x.reshape(S, n, n), dtype=torch.float32, device=dev))
        xo = p.backproject(torch.tensor(y.reshape(S, m, nd), dtype=torch.float32, device=dev))
        torch.cuda.synchronize()
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    for got, mat, absm, v in ((yo, a, absa, x32), (xo, at, absat, y32)):
        got = got.cpu().numpy().reshape(S, -1)
        # f16a / bf16a: only the matrix is 16-bit, the slices stay FP32
        model = (oracle.mixed_project(mat, v, kind) if kind in ("f16", "bf16")
                 else oracle.matrix16_project(mat, v, kind[:-1]))
        _check(got, model, oracle.project(absm, np.abs(v)))
        # against FP64: per slice, within the 16-bit unit roundoff
        exact = oracle.project(mat, v)
        u = 2.0 ** -11 if kind.startswith("f16") else 2.0 ** -8
        for s in range(S):
            nrm = np.linalg.norm(exact[s])
            if nrm > 0:
                assert np.linalg.norm(got[s] - exact[s]) / nrm < u


def test_host_pointers_match_device(xct):
    n, m, nd, S = 48, 40, 50, 6
    g, a, *_ = _setup(n, m, nd)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=(S, n, n)).astype(np.float32)
    with xct.Plan(n, m, nd, "f16", cos_sin=g.table()) as p:
        y_host = np.zeros((S, m, nd), dtype=np.float32)
        xct.xct_project(p.handle, x, y_host, S)            # pageable host memory
        pinned_x = torch.tensor(x).pin_memory()
        pinned_y = torch.zeros((S, m, nd)).pin_memory()
        xct.xct_project(p.handle, pinned_x, pinned_y, S)   # pinned host memory
        y_dev = p.project(torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.array_equal(y_host, y_dev)
    assert np.array_equal(pinned_y.numpy(), y_dev)


def test_runs_are_deterministic(xct):
    n, m, nd, S = 64, 96, 64, 40
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.uniform(0, 1, size=(S, n, n)), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.uniform(0, 1, size=(S, m, nd)), dtype=torch.float32, device="cuda")
    for kind in ("f32", "f16", "bf16"):
        with xct.Plan(n, m, nd, kind) as p:
            r1, r2 = p.project(x), p.project(x)
            b1, b2 = p.backproject(y), p.backproject(y)
        assert torch.equal(r1, r2) and torch.equal(b1, b2)
        with xct.Plan(n, m, nd, kind) as p2:      # a rebuilt plan gives the same bits
            assert torch.equal(p2.project(x), r1)


def test_zero_slices_and_empty_matrix(xct):
    with xct.Plan(8, 5, 4, "f32", det_offset=100.0) as p:   # every ray misses
        assert p.stats()["nnz"] == 0
        x = torch.rand((3, 8, 8), device="cuda")
        y = torch.full((3, 5, 4), float("nan"), device="cuda")
        p.project(x, out=y)
        assert torch.all(y == 0)
        xb = torch.full((3, 8, 8), float("nan"), device="cuda")
        p.backproject(torch.rand((3, 5, 4), device="cuda"), out=xb)
        assert torch.all(xb == 0)
        xct.xct_project(p.handle, x, y, 0)                   # S = 0: no-op


def test_adjoint_identity_on_gpu(xct):
    """<A x, y> = <x, A^T y> with the GPU's two stored matrices (FP32)."""
    n, m, nd, S = 100, 120, 110, 4
    rng = np.random.default_rng(8)
    x = torch.tensor(rng.standard_normal((S, n, n)), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.standard_normal((S, m, nd)), dtype=torch.float32, device="cuda")
    with xct.Plan(n, m, nd, "f32", det_offset=0.3) as p:
        ax = p.project(x).double()
        aty = p.backproject(y).double()
    lhs = (ax * y.double()).sum(dim=(1, 2))
    rhs = (x.double() * aty).sum(dim=(1, 2))
    scale = ax.norm(dim=(1, 2)) * y.double().norm(dim=(1, 2))
    assert torch.all((lhs - rhs).abs() <= 1e-6 * scale)
