"""The rounding envelope of mixed-precision CGLS, computed with the oracle
only (test infrastructure shared by the CPU pin and the GPU tracking test).

The workload is the batched noisy 3D case of the GPU CGLS tests: 64^2 grid,
96 angles, 64 bins, 8 slices of a 20-ellipsoid phantom, Poisson noise at
1e4 photons.

Model of the mixed-precision solve (Sec. III-C): the oracle's CGLS
recurrence with every product replaced by the oracle's mixed-precision
product (16-bit matrix values and normalised 16-bit input slices, products
summed exactly) rounded to FP32, the precision in which the GPU keeps its
vectors.

A CGLS trajectory on noisy data is chaotic after a few iterations (loss of
conjugacy): a rounding difference at the unit roundoff changes ||r_k|| by
percents.  The GPU's mixed solve rounds like the model until its trajectory
departs from the model's, and independently from then on.  So the model is
one sample of the rounding process; more samples come from the standard
probabilistic model of rounding errors (each computed value carries an
independent relative error of at most the unit roundoff u): every product of
the model multiplied elementwise by (1 + delta), delta ~ U(-u, u), u = 2^-11
(binary16) or 2^-8 (bfloat16), seeded.  The envelope is the largest
deviation of ||r_k|| from the FP32 solve's over the model and these samples.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2009_07226_gb300 import inputs

UNIT_ROUNDOFF = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


def noisy_batch():
    """(n, m, nd, S, cos_sin, sinogram [S, m, nd] float64, A, A^T)."""
    n, m, nd, S = 64, 96, 64, 8
    cs = inputs.angle_table(m)
    rng = np.random.default_rng(2)
    ells = inputs.random_ellipsoids(rng, 20)
    sino = np.stack([inputs.line_integrals(inputs.cut_ellipsoids(ells, inputs.slice_z(s, S)), n, cs, nd)
                     for s in range(S)])
    for s in range(S):
        sino[s] = inputs.poisson_noise(np.random.default_rng(100 + s), sino[s], n, 1e4)
    g = oracle.Geometry(n=n, m=m, nd=nd, cos_sin=cs)
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    return n, m, nd, S, cs, sino, a, at


def _to_f32(Y):
    return np.asarray(Y).astype(np.float32).astype(np.float64)


def fp32_ops(a, at):
    """The FP64 oracle products rounded to FP32."""
    return (lambda X: _to_f32(oracle.project(a, X))), (lambda Y: _to_f32(oracle.backproject(at, Y)))


def mixed_ops(a, at, kind, seed=None, u=None):
    """The mixed-precision products rounded to FP32; with a seed, each
    output element also multiplied by (1 + delta), delta ~ U(-u, u) (u the
    unit roundoff of `kind` unless given)."""
    if u is None:
        u = UNIT_ROUNDOFF[kind]
    rng = np.random.default_rng(seed) if seed is not None else None

    def op(mat):
        def f(X):
            Y = oracle.mixed_project(mat, X, kind)
            if rng is not None:
                Y = Y * (1.0 + rng.uniform(-u, u, size=Y.shape))
            return _to_f32(Y)
        return f

    return op(a), op(at)


def residual_deviation(log, ref):
    """|‖r_k‖ / ‖r_k‖_ref - 1| per iteration and slice."""
    return np.abs(np.asarray(log)[:, :, 0] / np.asarray(ref)[:, :, 0] - 1.0)


def envelope(a, at, b, kind, iters, seeds=range(6)):
    """Largest transient and final deviation of ||r_k|| from the FP32
    solve's, over the model ("model") and the perturbed samples
    ("samples": one (max, final) pair per seed)."""
    b = _to_f32(b)
    _, l32 = oracle.cgls(*fp32_ops(a, at), b, iters)
    _, lm = oracle.cgls(*mixed_ops(a, at, kind), b, iters)
    dm = residual_deviation(lm, l32)
    out = {"model": (float(dm.max()), float(dm[-1].max())), "samples": []}
    for sd in seeds:
        _, lp = oracle.cgls(*mixed_ops(a, at, kind, seed=1000 + sd), b, iters)
        d = residual_deviation(lp, l32)
        out["samples"].append((float(d.max()), float(d[-1].max())))
    allp = [out["model"]] + out["samples"]
    out["max"] = max(p[0] for p in allp)
    out["final"] = max(p[1] for p in allp)
    return out
