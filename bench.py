"""Benchmark: batched parallel-beam CGLS on the 512^2 x 768-angle x 512-bin
geometry with 64 slices per GPU, 50 iterations per solve (one step = one
solve of one batch on a memoized operator).

Prints one JSON line: value = projection + back-projection GFLOP/s of the
mixed-precision (binary16) solve (2 * nnz * S flops per product, 50
projections + 51 back projections per step), with the FP32 solve, CGLS
iterations per second, algorithmic HBM GB/s, the mixed-vs-FP32 error, the
per-launch roofline of the dominant kernel (the sparse product), the
clocks seen during the timed region, an end-to-end figure through host
buffers, and the CPU oracle as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own 64 consecutive slices of a
volume of 64 * N slices (weak scaling; no data exchange) and rank 0 prints
the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch3d_512"
METRIC = "proj+backproj GFLOP/s, HBM GB/s, CGLS iter/s: mixed vs FP32 at <=1e-3 rel err"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d
    except Exception:
        return 6800.0, "fallback", {}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[4 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _kernel_sources_hash() -> str:
    """Hash of the sources that determine the product kernel and its layout."""
    import hashlib
    h = hashlib.sha256()
    for f in ("spmm_pipe.cu", "spmm.cu", "plan.cu", "xct_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2009_07226_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(key: str):
    """DRAM bytes per launch recorded under profiles/ from an ncu capture of
    the current kernel sources (None if absent or captured from other ones)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and parts[0] == key and parts[1] == _kernel_sources_hash():
                    return int(parts[2])
    except OSError:
        pass
    return None


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------
# reference arm: the CPU FP64 oracle
# --------------------------------------------------------------------------

def _oracle_setup(w):
    import oracle
    g = oracle.Geometry(n=w["n"], m=w["m"], nd=w["nd"], cos_sin=w["cos_sin"])
    a = oracle.siddon_csr(g)
    at = oracle.transpose(a)
    return a, at


def _oracle_step(a, at, b, iters):
    import oracle
    oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y), b, iters)


def _config(n, m, nd, S, K, nnz, world):
    """The workload of the JSON line (both arms)."""
    return {"workload": WORKLOAD, "n": n, "angles": m, "bins": nd, "slices_per_gpu": S,
            "iters": K, "nnz": nnz, "l2": "inputs larger than L2 (packed A 1.2 GB per product)",
            "parallelism": f"slice-sharded x{world}, no collective"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2009_07226_gb300 import inputs
    w = inputs.make_workload(WORKLOAD, slices=1, with_images=False)
    a, at = _oracle_setup(w)
    nnz = a.nnz
    b = w["sino"].reshape(1, -1)
    iters = 2                       # bounded sample: 1 slice, 2 iterations per step
    for _ in range(args.warmup):
        _oracle_step(a, at, b, iters)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(a, at, b, iters)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    flops = (2 * iters + 1) * 2.0 * nnz * 1
    gf = flops / dt / 1e9
    import oracle
    cores = oracle.set_threads(0)
    sample = f"1 of 64 slices, {iters} CGLS iterations per step (FP64, CSR oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gf, "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w["n"], w["m"], w["nd"], inputs.WORKLOADS[WORKLOAD]["slices"],
                          inputs.WORKLOADS[WORKLOAD]["iters"], nnz, world),
        "cpu_baseline": {"value": gf, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gf, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def _cgls2d_vs_oracle(c1):
    """The plain 2D workload's GPU solves against the FP64 oracle's CGLS of
    the same (FP32-rounded) sinogram, projected by the oracle itself (30
    iterations), and the oracle's own time."""
    import oracle
    xs, w = c1
    a, at = _oracle_setup(w)
    # the same consistent sinogram, from the oracle's own projector
    b = oracle.project(a, w["images"].reshape(1, -1)).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    xo, _ = oracle.cgls(lambda X: oracle.project(a, X), lambda Y: oracle.backproject(at, Y), b, w["iters"])
    dt = time.perf_counter() - t0
    out = {"oracle_ms_per_solve": dt * 1e3}
    for kind, x in xs.items():
        out[f"rel_err_{kind}_vs_oracle"] = float(np.linalg.norm(x - xo) / np.linalg.norm(xo))
    ph = w["images"].reshape(1, -1)
    out["phantom_rel_err"] = {"oracle": float(np.linalg.norm(xo - ph) / np.linalg.norm(ph)),
                              **{k: float(np.linalg.norm(x - ph) / np.linalg.norm(ph)) for k, x in xs.items()}}
    return out


def cpu_baseline(w, c1=None):
    """The oracle, as it stands, on this host's cores: one slice, a few
    iterations (a bounded sample of the same workload); with c1, also the
    plain 2D workload's solve checked against the oracle's."""
    import oracle
    a, at = _oracle_setup(w)
    b = w["sino"][:1].reshape(1, -1)
    iters = 2
    _oracle_step(a, at, b, 1)
    t0 = time.perf_counter()
    _oracle_step(a, at, b, iters)
    dt = time.perf_counter() - t0
    nprod = 2 * iters + 1
    gf = nprod * 2.0 * a.nnz / dt / 1e9
    # the same on one core (one iteration: 3 products)
    prev = oracle.set_threads(1)
    t1 = time.perf_counter()
    _oracle_step(a, at, b, 1)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(prev)
    return {"value": gf, "unit": "GFLOP/s", "cores": prev, "kind": "oracle",
            "sample": f"1 of 64 slices, {iters} CGLS iterations, FP64 CSR products (OpenMP)",
            "ms_per_product": dt / nprod * 1e3, "ms_per_iteration": dt / iters * 1e3,
            "single_core": {"value": 3 * 2.0 * a.nnz / dt1 / 1e9, "unit": "GFLOP/s",
                            "ms_per_product": dt1 / 3 * 1e3},
            "cpu": _cpu_model(),
            **({"cgls2d_128": _cgls2d_vs_oracle(c1)} if c1 else {})}


def _cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86 model name, or the Arm
    implementer / part codes), with the logical core count."""
    name = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model name"):
            hits = [l.split(":", 1)[1].strip() for l in info if l.startswith(key)]
            if hits:
                name = hits[0]
                break
        if name is None:
            imp = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
            part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
            if imp and part:
                name = f"Arm implementer {imp[0]} part {part[0]}"
    except OSError:
        pass
    return f"{name or platform.machine()}, {os.cpu_count()} logical cores"


ROOF_KINDS = {0: "gather16_mixed_fma", 1: "mixed_fma", 2: "fp32_fma", 3: "gather16", 4: "gather16_fp32x2_fma"}


def _measure_roof(stream, iters=20000, ctas_per_sm=2):
    """The product kernel's core roofs measured on this GPU by the library's
    roof probe (xct_roof_probe): rates of the product's inner step -- a
    16-byte shared-memory gather by 8 lanes of one 128-byte row, feeding 8
    mixed-precision FMAs -- and of its parts.  Returns per kind: operations
    per second (FMAs, or 16-byte loads for the gathers alone) and the
    derived flop rate (2 per FMA)."""
    import torch
    from paper_2009_07226_gb300 import xct
    out = {}
    for kind, name in ROOF_KINDS.items():
        xct.xct_roof_probe(kind, iters // 10, ctas_per_sm, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ops = xct.xct_roof_probe(kind, iters, ctas_per_sm, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        rate = ops / sec
        out[name] = {"ms": sec * 1e3, "ops_per_s": rate,
                     **({"tflops": 2.0 * rate / 1e12} if kind != 3 else {"tb_per_s": 16.0 * rate / 1e12})}
    return out


def _hbm_regime(xct, plan, y, n, m, nd, nnz, peak_hbm, stream, slices=(1, 2, 4, 8)):
    """The product kernel where few slices share the matrix, so the matrix
    stream from HBM is the lowest roof: per slice count, the projection and
    back-projection launches of a short binary16 CGLS solve timed with CUDA
    events on the launching stream (XCT_CGLS_TIMING), and the algorithmic
    bytes per launch -- nnz x 4 B of packed entries + (rows + 1) x 8 B + S x
    input rows x 2 B + S x output rows x 4 B -- over that time, against the
    measured HBM bandwidth."""
    import torch
    out = {}
    rows_a, cols_a = m * nd, n * n
    for S in slices:
        x = torch.empty((S, n, n), dtype=torch.float32, device=y.device)
        for _ in range(2):
            xct.xct_cgls(plan.handle, y[:S].contiguous(), x, S, 5, xct.XCT_CGLS_TIMING, None, stream)
        torch.cuda.synchronize()
        st = plan.stats()
        tp = st["t_project_ms"] / max(st["n_project"], 1)
        tb = st["t_backproject_ms"] / max(st["n_backproject"], 1)
        alg_p = nnz * 4 + (rows_a + 1) * 8 + S * cols_a * 2 + S * rows_a * 4
        alg_b = nnz * 4 + (cols_a + 1) * 8 + S * rows_a * 2 + S * cols_a * 4
        gp, gb = alg_p / (tp * 1e-3) / 1e9, alg_b / (tb * 1e-3) / 1e9
        out[S] = {"project_ms": tp, "backproject_ms": tb, "alg_bytes_project": alg_p,
                  "alg_bytes_backproject": alg_b, "project_gbs": gp, "backproject_gbs": gb,
                  "project_frac_hbm": gp / peak_hbm, "backproject_frac_hbm": gb / peak_hbm,
                  "project_tflops": 2.0 * nnz * S / (tp * 1e-3) / 1e12}
    return out


def _accuracy(xct, plans, p64, w, first, count, volume, S, n, K, y, y64, err_vs_phantom, stream, dev):
    """The accuracy target (relative reconstruction error vs FP64) measured
    where it is well posed.

    noiseless: consistent data, where CGLS converges: the sinogram is the
    FP64 projection of the rasterised phantom with the FP64 matrix
    (xct_project_f64); each form's relative distance to the phantom after
    K iterations and to the FP64 iterate, and |err_form - err_FP64|.

    noisy: on the measured (Poisson) sinogram CGLS semi-converges: the
    distance to the phantom falls to a minimum and then grows as the solve
    fits the noise.  Each form's phantom error at 5, 10, 20 and K
    iterations and at its best iteration (binary16 and FP32 every
    iteration, through checkpoint / resume one iteration at a time; FP64 at
    those counts and at the FP32 form's best iteration)."""
    import torch
    from paper_2009_07226_gb300 import inputs
    phantom = torch.tensor(w["images"], dtype=torch.float64, device=dev)
    yc64 = p64.project_f64(phantom, stream=stream)
    yc = yc64.float()
    del phantom
    xc = {}
    for kind in ("f16", "f32"):
        xc[kind] = torch.empty((S, n, n), dtype=torch.float32, device=dev)
        xct.xct_cgls(plans[kind].handle, yc, xc[kind], S, K, 0, None, stream)
    xc["f64"] = torch.empty((S, n, n), dtype=torch.float64, device=dev)
    xct.xct_cgls_f64(p64.handle, yc64, xc["f64"], S, K, 0, None, stream)
    e_c = {k: err_vs_phantom(v) for k, v in xc.items()}
    noiseless = {
        "iters": K, "phantom_rel_err": e_c,
        "rel_err_vs_fp64_iterate": {k: float(torch.linalg.norm(xc[k].double() - xc["f64"]) /
                                             torch.linalg.norm(xc["f64"])) for k in ("f16", "f32")},
        "abs_diff_phantom_err_vs_fp64": {k: abs(e_c[k] - e_c["f64"]) for k in ("f16", "f32")},
    }
    del xc, yc, yc64

    def curve(kind):
        plan = plans[kind]
        state = torch.empty(xct.xct_cgls_state_bytes(plan.handle, S), dtype=torch.uint8, device=dev)
        x = torch.empty((S, n, n), dtype=torch.float32, device=dev)
        errs = []
        for k in range(1, K + 1):
            fl = xct.XCT_CGLS_SAVE | xct.XCT_CGLS_NO_GRAPH | (xct.XCT_CGLS_RESUME if k > 1 else 0)
            xct.xct_cgls_state(plan.handle, y if k == 1 else None, x, S, 1, fl, state, None, stream)
            errs.append(err_vs_phantom(x))
        return errs

    marks = sorted({5, 10, 20, K})
    noisy = {"phantom_rel_err_by_iteration": {}, "best": {}}
    curves = {k: curve(k) for k in ("f16", "f32")}
    for kind, c in curves.items():
        kb = int(np.argmin(c)) + 1
        noisy["phantom_rel_err_by_iteration"][kind] = {k: c[k - 1] for k in marks}
        noisy["best"][kind] = {"iteration": kb, "phantom_rel_err": c[kb - 1]}
    kb32 = noisy["best"]["f32"]["iteration"]
    e64 = {}
    for k in sorted(set(marks) | {kb32}):
        x64k = torch.empty((S, n, n), dtype=torch.float64, device=dev)
        xct.xct_cgls_f64(p64.handle, y64, x64k, S, k, 0, None, stream)
        e64[k] = err_vs_phantom(x64k)
    noisy["phantom_rel_err_by_iteration"]["f64"] = {k: e64[k] for k in marks}
    kb64 = min(e64, key=e64.get)
    noisy["best"]["f64"] = {"iteration": kb64, "phantom_rel_err": e64[kb64],
                            "note": "FP64 evaluated at 5, 10, 20, K and the FP32 best iteration"}
    noisy["best_abs_diff_vs_fp64"] = {k: abs(noisy["best"][k]["phantom_rel_err"] - e64[kb64])
                                      for k in ("f16", "f32")}
    return {"noiseless": noiseless, "noisy": noisy}


def _measure_cgls2d(steps):
    """The plain 2D workload: one 128^2 slice, 180 angles, 128 bins, 10
    random ellipses, noiseless sinogram (the rasterised phantom projected
    with the FP64 matrix, xct_project_f64), 30 CGLS iterations from zero;
    FP32 (the configuration's form) and binary16.
    A (28 MB in FP32) and every vector fit in the 129 MB L2, so the byte
    rate is reported against L2-resident data, not HBM."""
    import torch
    from paper_2009_07226_gb300 import inputs, xct
    w = inputs.make_workload("cgls2d_128")
    n, m, nd, S, K = w["n"], w["m"], w["nd"], w["slices"], w["iters"]
    stream = torch.cuda.current_stream()
    with xct.Plan(n, m, nd, "f32", cos_sin=w["cos_sin"], keep_f64=True) as p64:
        y = p64.project_f64(torch.tensor(w["images"], dtype=torch.float64, device="cuda")).float()
    out = {"n": n, "angles": m, "bins": nd, "slices": S, "iters": K, "l2_resident": True}
    xs = {}
    for kind in ("f32", "f16"):
        with xct.Plan(n, m, nd, kind, cos_sin=w["cos_sin"]) as p:
            st = p.stats()
            x = torch.empty((S, n, n), device="cuda")
            for _ in range(3):
                xct.xct_cgls(p.handle, y, x, S, K, 0, None, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                xct.xct_cgls(p.handle, y, x, S, K, 0, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            nnz = st["nnz"]
            ebytes = 8 if kind == "f32" else 4
            alg = nnz * ebytes + (m * nd + n * n + 2) * 8 + S * (m * nd + n * n) * 8
            out[kind] = {"ms_per_solve": ms, "cgls_iter_per_s": K / (ms * 1e-3),
                         "gflops": (2 * K + 1) * 2.0 * nnz * S / (ms * 1e-3) / 1e9,
                         "alg_gbs": (2 * K + 1) * alg / (ms * 1e-3) / 1e9, "nnz": nnz}
            xs[kind] = x.cpu().numpy().reshape(S, -1).astype(np.float64)
    out["note"] = ("whole solves (graph path) including one natural <-> internal conversion; "
                   "error against the FP64 oracle's solve is in cpu_baseline.cgls2d_128")
    return out, xs, w


def _workloads(args):
    """The other configurations, each measured once in this process with
    reduced repetition (stated per entry); their full-length runs are the
    --mode batch / tv / large lines."""
    import torch
    res = {}
    c1 = None
    jobs = (("cgls2d_128", lambda: _measure_cgls2d(10)),
            ("large3d_1536", lambda: _measure_large(2, 1)),
            ("tv3d_1024", lambda: _measure_tv(1, with_autograd=False)),
            ("batch_uneven_64", lambda: _measure_batch(1, 1, combos=("batched_mixed", "per_job_fp32"))))
    reps = {"cgls2d_128": "3 warm-up + 10 timed solves", "large3d_1536": "1 warm-up + 2 timed solves per form",
            "tv3d_1024": "1 warm-up + 1 timed 200-step run (native loop)",
            "batch_uneven_64": "1 warm-up + 1 timed batch per form"}
    for name, fn in jobs:
        t0 = time.perf_counter()
        try:
            r = fn()
            if name == "cgls2d_128":
                r, xs, w1 = r
                c1 = (xs, w1)
            res[name] = {**r, "repetition": reps[name], "wall_s": time.perf_counter() - t0}
        except Exception as e:      # keep the line: record the failure
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res, c1


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, shard, xct

    per_rank = inputs.WORKLOADS[WORKLOAD]["slices"]
    first, count = shard.weak_range(per_rank, rank)
    w = inputs.make_workload(WORKLOAD, slices=count, slice_offset=first, with_images=True,
                             volume_slices=per_rank * world)
    n, m, nd, S, K = w["n"], w["m"], w["nd"], w["slices"], w["iters"]
    y = torch.tensor(w["sino"], dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # the FP32 plan also keeps the FP64 matrices for the double-precision yardstick
    # the binary16 plan also builds the paired layouts its 64-slice tiles run on
    # (XCT_PLAN_PAIRED_ROWS); "f16u" is the same storage on the plain layouts,
    # timed for comparison
    plans = {k: xct.Plan(n, m, nd, "f16" if k == "f16u" else k, cos_sin=w["cos_sin"],
                         keep_f64=(k == "f32"), paired_rows=(k == "f16"))
             for k in ("f16", "f32", "f16a", "f16u")}
    nnz = plans["f16"].stats()["nnz"]
    flops_step = (2 * K + 1) * 2.0 * nnz * S
    xs = {k: torch.empty((S, n, n), dtype=torch.float32, device=dev) for k in plans}

    def step(kind, flags=xct.XCT_CGLS_TIMING):
        xct.xct_cgls(plans[kind].handle, y, xs[kind], S, K, flags, None, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(kind, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tp = tb = to = 0.0
        parts = {"stage": 0.0, "vector": 0.0, "scalar": 0.0}
        npj = nbp = 0
        barrier()
        launches0 = xct.xct_launch_count()
        ev0.record(stream)
        for _ in range(steps):
            step(kind)
            st = plans[kind].stats()
            tp += st["t_project_ms"]
            tb += st["t_backproject_ms"]
            to += st["t_other_ms"]
            for k in parts:
                parts[k] += st[f"t_{k}_ms"]
            npj += st["n_project"]
            nbp += st["n_backproject"]
        ev1.record(stream)
        barrier()
        launches = xct.xct_launch_count() - launches0
        ms = shard.max_over_ranks(ev0.elapsed_time(ev1) / steps, dev)
        timed.parts[kind] = {k: v / steps for k, v in parts.items()}
        return ms, tp / max(npj, 1), tb / max(nbp, 1), to / steps, launches

    timed.parts = {}
    for kind in ("f16", "f32", "f16a", "f16u"):
        for _ in range(args.warmup):
            step(kind)
    torch.cuda.synchronize()

    peak_hbm, peak_kind, peaks = _peaks()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    ms16, proj16, back16, other16, launches = timed("f16", args.steps)
    ms32, proj32, back32, other32, _ = timed("f32", args.steps)
    msa, proja, backa, othera, _ = timed("f16a", args.steps)
    msu, proju, backu, otheru, _ = timed("f16u", args.steps)
    clocks = sampler.stop() if sampler else None

    # graph path (the default call) for reference, untimed by the roofline
    barrier()
    g0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        step("f16", 0)
    torch.cuda.synchronize()
    graph_ms = shard.max_over_ranks((time.perf_counter() - g0) / max(1, args.steps // 2) * 1e3, dev)

    # end to end through host buffers (pinned), H2D + solve + D2H every step
    yh = torch.tensor(w["sino"], dtype=torch.float32).pin_memory()
    xh = torch.empty((S, n, n), dtype=torch.float32).pin_memory()
    barrier()
    e0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 2)
    for _ in range(e2e_steps):
        xct.xct_cgls(plans["f16"].handle, yh, xh, S, K, 0, None, stream)
    torch.cuda.synchronize()
    e2e_ms = shard.max_over_ranks((time.perf_counter() - e0) / e2e_steps * 1e3, dev)

    rel = float(torch.linalg.norm(xs["f16"] - xs["f32"]) / torch.linalg.norm(xs["f32"]))
    # residual curves of the two solves (||y - A x_k|| per slice and
    # iteration, as the solver logs them) and the error of one mixed
    # projection against the FP32 one, on the FP32 iterate
    logs = {}
    for kind in plans:
        lg = torch.zeros((K + 1, S, 2), dtype=torch.float64, device=dev)
        xct.xct_cgls(plans[kind].handle, y, xs[kind], S, K, 0, lg, stream)
        logs[kind] = lg[:, :, 0]
    track = (logs["f16"] / logs["f32"] - 1.0).abs()
    track_a = (logs["f16a"] / logs["f32"] - 1.0).abs()
    rel_a = float(torch.linalg.norm(xs["f16a"] - xs["f32"]) / torch.linalg.norm(xs["f32"]))
    q16, q32 = plans["f16"].project(xs["f32"]), plans["f32"].project(xs["f32"])
    proj_err = float(torch.linalg.norm((q16 - q32).double()) / torch.linalg.norm(q32.double()))
    track_max, track_final = float(track.max()), float(track[-1].max())

    # double-precision yardstick (Sec. V compares double, single and 16-bit
    # forms): one FP64 solve on the unrounded sinogram, one FP64 projection;
    # every form's iterate and residual curve against it
    p64 = plans["f32"]
    y64 = torch.tensor(w["sino"], dtype=torch.float64, device=dev)
    p64.project_f64(xs["f32"].double())                # warm-up of the FP64 kernels
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    barrier()
    ev[0].record(stream)
    x64p = p64.project_f64(xs["f32"].double(), stream=stream)
    ev[1].record(stream)
    log64 = torch.zeros((K + 1, S, 2), dtype=torch.float64, device=dev)
    x64 = torch.empty((S, n, n), dtype=torch.float64, device=dev)
    xct.xct_cgls_f64(p64.handle, y64, x64, S, K, 0, log64, stream)
    ev[2].record(stream)
    barrier()
    proj64_ms, ms64 = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    proj_err64 = {k: float(torch.linalg.norm(q.double() - x64p) / torch.linalg.norm(x64p))
                  for k, q in (("f16", q16), ("f32", q32))}
    phantom = torch.tensor(w["images"], dtype=torch.float64, device=dev)

    def err_vs_phantom(x):
        return float(torch.linalg.norm(x.double() - phantom) / torch.linalg.norm(phantom))

    vs64 = {"phantom_rel_err": {"f64": err_vs_phantom(x64)}}
    for kind in plans:
        vs64["phantom_rel_err"][kind] = err_vs_phantom(xs[kind])
    for kind in plans:
        dev_k = (logs[kind] / log64[:, :, 0] - 1.0).abs()
        vs64[kind] = {"rel_err": float(torch.linalg.norm(xs[kind].double() - x64) / torch.linalg.norm(x64)),
                      "residual_curve_max_rel_dev": float(dev_k.max()),
                      "residual_curve_final_rel_dev": float(dev_k[-1].max())}
    # the same against FP64 after fewer iterations: where the iterates
    # still agree (rounding differences grow once CGLS loses conjugacy)
    vs64["rel_err_by_iteration"] = {"f16": {}, "f32": {}}
    for k in (5, 10, 20):
        x64k = torch.empty((S, n, n), dtype=torch.float64, device=dev)
        xct.xct_cgls_f64(p64.handle, y64, x64k, S, k, 0, None, stream)
        for kind in ("f16", "f32"):
            xk = torch.empty((S, n, n), dtype=torch.float32, device=dev)
            xct.xct_cgls(plans[kind].handle, y, xk, S, k, 0, None, stream)
            vs64["rel_err_by_iteration"][kind][k] = float(torch.linalg.norm(xk.double() - x64k) /
                                                          torch.linalg.norm(x64k))
    vs64["rel_err_by_iteration"]["f16"][K] = vs64["f16"]["rel_err"]
    vs64["rel_err_by_iteration"]["f32"][K] = vs64["f32"]["rel_err"]
    del x64p
    accuracy = _accuracy(xct, plans, p64, w, first, count, per_rank * world, S, n, K, y, y64,
                         err_vs_phantom, stream, dev)
    hbm_regime = _hbm_regime(xct, plans["f16"], y, n, m, nd, nnz, _peaks()[0], stream)
    with xct.Plan(n, m, nd, "f16", cos_sin=w["cos_sin"], few_slices=True) as pw:
        hbm_regime_wide = _hbm_regime(xct, pw, y, n, m, nd, nnz, _peaks()[0], stream)

    if rank != 0:
        return
    st16 = plans["f16"].stats()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else peaks.get("sm_max_mhz", 2070.0)
    # dominant kernel: the product (projection launch of the mixed solve),
    # per-launch duration from CUDA events on its stream
    flops_launch = 2.0 * nnz * S
    achieved = flops_launch / (proj16 * 1e-3) / 1e12
    clk = sm_mhz * 1e6
    # three roofs of the 16-bit product (per launch):
    #  FP32 FMA pipe: nsm x 128 FMA/clk x 2 flop
    #  16-bit operands: every FMA also issues one 16->32-bit conversion, and
    #    reads 2 bytes of a staged row from shared memory (128 B/clk/SM):
    #    both give nsm x 64 FMA/clk x 2 flop
    #  HBM: 2 flop per matrix entry and slice over the algorithmic bytes
    fma_peak_derived = 128 * 2 * nsm * clk / 1e12
    op16_peak_derived = 64 * 2 * nsm * clk / 1e12
    # the roofs derived from the unit counts and the clock: every FMA reads
    # 2 bytes of a staged row from shared memory (128 B/clk/SM), and FP32
    # FMAs (128/clk/SM); the library's roof probe times the product's inner
    # step alone on this GPU as a check of the first
    roof = _measure_roof(stream)
    fma_peak = fma_peak_derived
    # the paired layouts read one staged row per distinct column of a pair of
    # rows (gathers_a_paired of them per tile) instead of one per entry: their
    # operand roof is the plain one scaled by nnz / gathers
    gathers = st16["gathers_a_paired"] or nnz
    op16_peak_plain = op16_peak_derived
    op16_peak = op16_peak_derived * nnz / gathers
    rows_a, cols_a = m * nd, n * n
    alg_bytes = nnz * 4 + (rows_a + 1) * 8 + S * cols_a * 2 + S * rows_a * 4
    alg_bytes_bp = nnz * 4 + (cols_a + 1) * 8 + S * rows_a * 2 + S * cols_a * 4
    hbm_roof = flops_launch / (alg_bytes / (peak_hbm * 1e9)) / 1e12
    gather_bytes = gathers * S * 2
    smem_peak = 128.0 * nsm * clk / 1e9
    traffic = _profiled_traffic("spmm_pipe_f16_projection")
    value = flops_step / (ms16 * 1e-3) / 1e9
    peak = min(fma_peak, op16_peak, hbm_roof)
    out = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms16,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded ellipsoid phantom, exact line integrals, Poisson 1e4)",
        "config": _config(n, m, nd, S, K, nnz, world),
        "fp32": {"value": flops_step / (ms32 * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms32,
                 "cgls_iter_per_s": K / (ms32 * 1e-3)},
        "speedup_mixed_vs_fp32": ms32 / ms16,
        "cgls_iter_per_s": K / (ms16 * 1e-3),
        "hbm_gbs_alg": (alg_bytes * K + alg_bytes_bp * (K + 1)) / (ms16 * 1e-3) / 1e9,
        "rel_err_mixed_vs_fp32": rel,
        "residual_curve_mixed_vs_fp32": {"max_rel_dev": track_max, "final_rel_dev": track_final},
        "mixed_fp32_vectors": {"storage": "f16a (binary16 matrix, FP32 slices)",
                               "value": flops_step / (msa * 1e-3) / 1e9, "unit": "GFLOP/s",
                               "ms_per_step": msa, "speedup_vs_fp32": ms32 / msa,
                               "project_ms": proja, "backproject_ms": backa,
                               "residual_curve_vs_fp32": {"max_rel_dev": float(track_a.max()),
                                                          "final_rel_dev": float(track_a[-1].max())},
                               "rel_err_vs_fp32": rel_a},
        "rel_err_projection_mixed_vs_fp32": proj_err,
        "fp64": {"ms_per_step": ms64, "value": flops_step / (ms64 * 1e-3) / 1e9, "unit": "GFLOP/s",
                 "project_ms": proj64_ms,
                 "project_tflops": 2.0 * nnz * S / (proj64_ms * 1e-3) / 1e12,
                 "project_frac_of_fp64_nominal": 2.0 * nnz * S / (proj64_ms * 1e-3) / 1e12 / 1.25,
                 "note": "one solve, kept FP64 CSR, FP64 FMAs (nominal GB300 FP64 rate 1.25 TFLOP/s); "
                         "FP32 and binary16 forms use the FP32-rounded sinogram"},
        "vs_fp64": vs64,
        "accuracy_vs_fp64": accuracy,
        "hbm_regime": {"storage": "f16", "note": "few slices: the packed matrix stream (nnz x 4 B) "
                       "sets the roof; slice counts below 8 run as an 8-slice tile (on wide stages only its 2 or 4 "
                       "live slices are read and multiplied when the rest are padding); by_slices: the "
                       "plan's own layouts, by_slices_wide: a plan built with XCT_PLAN_FEW_SLICES "
                       "(wide stages, entries streamed from device memory)", "by_slices": hbm_regime,
                       "by_slices_wide": hbm_regime_wide,
                       "peak_gbs": _peaks()[0], "peak_source": _peaks()[1]},
        "rel_err_projection_vs_fp64": proj_err64,
        "graph_ms_per_step": graph_ms,
        "other_f16_ms_per_step": timed.parts["f16"],
        "kernel_ms": {"project_f16": proj16, "backproject_f16": back16, "other_f16_per_step": other16,
                      "project_f32": proj32, "backproject_f32": back32, "other_f32_per_step": other32},
        "roofline": {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "spmm_pipe_kernel<__half,__half,64,false,true> (projection on the paired layout, "
                      "2*nnz*S flops per launch)",
            "peak_source": (f"derived at the median SM clock {sm_mhz:.0f} MHz, the least of three roofs: "
                            f"the 16-bit operand roof of the paired layout {op16_peak:.1f} (one 128-byte "
                            f"staged row read from shared memory at 128 B/clk/SM per distinct column of a "
                            f"pair of rows, {gathers / nnz:.3f} reads per entry; the plain layouts' "
                            f"{op16_peak_plain:.1f} at one read per entry, {nsm} SMs x 64 FMA/clk x 2 flop, "
                            f"which the library's roof probe reaches to "
                            f"{roof['gather16_mixed_fma']['tflops'] / op16_peak_plain:.0%} with the plain "
                            f"layouts' inner step alone, {roof['gather16_mixed_fma']['tflops']:.1f} measured); "
                            f"the FP32 FMA roof {fma_peak:.1f} ({nsm} x 128 FMA/clk x 2 flop); the HBM roof "
                            f"{hbm_roof:.1f} (2*nnz*S flop over the algorithmic bytes at the measured "
                            f"{peak_hbm:.0f} GB/s)"),
            "plain_layout": {"operand_roof": op16_peak_plain,
                             "frac_of_plain_operand_roof": achieved / op16_peak_plain,
                             "project_ms": proju, "backproject_ms": backu, "ms_per_step": msu,
                             "value": flops_step / (msu * 1e-3) / 1e9,
                             "achieved": flops_launch / (proju * 1e-3) / 1e12,
                             "frac": flops_launch / (proju * 1e-3) / 1e12 / min(fma_peak, op16_peak_plain, hbm_roof),
                             "note": "the same binary16 solve on a plan without XCT_PLAN_PAIRED_ROWS "
                                     "(one staged-row read per entry)"},
            "roof_probe": {k: {**v, "fma_per_clk_per_sm": (v["ops_per_s"] / (nsm * clk)
                                                           if "tflops" in v else None)}
                           for k, v in roof.items()},
            "fp32_fma": {"peak": fma_peak, "frac": achieved / fma_peak},
            "hbm": {"achieved_gbs": alg_bytes / (proj16 * 1e-3) / 1e9, "peak_gbs": peak_hbm,
                    "frac": alg_bytes / (proj16 * 1e-3) / 1e9 / peak_hbm, "peak_source": peak_kind,
                    "alg_bytes_per_launch": alg_bytes,
                    "traffic_over_alg": (traffic / alg_bytes) if traffic else None},
            "smem_gather": {"achieved_gbs": gather_bytes / (proj16 * 1e-3) / 1e9, "peak_gbs": smem_peak,
                            "frac": gather_bytes / (proj16 * 1e-3) / 1e9 / smem_peak},
        },
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": flops_step / (e2e_ms * 1e-3) / 1e9, "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(S * m * nd * 4), "d2h_bytes_per_step": int(S * n * n * 4)},
        "plan_ms": {"f16": st16["plan_ms"], "f32": plans["f32"].stats()["plan_ms"]},
        "plan_flags": {"f16": "XCT_PLAN_PAIRED_ROWS", "f32": "XCT_PLAN_KEEP_F64", "f16a": "",
                       "f16u": ""},
    }
    c1 = None
    if world == 1 and not args.no_workloads:
        for pl in plans.values():
            pl.close()
        del xs, logs, q16, q32
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["workloads"], c1 = _workloads(args)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, c1)
    print(json.dumps(out))


def run_roof(args):
    """The roof probe alone: the product kernel's core roofs on this GPU."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sampler = ClockSampler(0)
    sampler.start()
    res = {c: _measure_roof(torch.cuda.current_stream(), iters=args.steps * 4000, ctas_per_sm=c)
           for c in (1, 2, 3)}
    clocks = sampler.stop()
    clk = (clocks.get("sm_mhz") or 2070.0) * 1e6
    for c, r in res.items():
        for v in r.values():
            v["per_clk_per_sm"] = v["ops_per_s"] / (nsm * clk)
    print(json.dumps({"mode": "roof", "sms": nsm, "ctas_per_sm": res, "clocks": clocks}))


def run_products(args):
    """Projection and back projection alone (S = 64 slices of the workload's
    geometry unless --slices says otherwise, one storage type): for
    profiling the product kernels."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, xct
    wl = inputs.WORKLOADS[WORKLOAD]
    n, m, nd = wl["n"], wl["m"], wl["nd"]
    S = args.slices or wl["slices"]
    plan = xct.Plan(n, m, nd, args.storage, cos_sin=inputs.angle_table(m), few_slices=args.few_slices,
                    paired_rows=args.paired_rows, narrow_tiles=args.narrow_tiles)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((S, n, n), device="cuda", generator=g)
    y = torch.rand((S, m, nd), device="cuda", generator=g)
    yo, xo = torch.empty_like(y), torch.empty_like(x)
    for _ in range(args.warmup):
        plan.project(x, out=yo)
        plan.backproject(y, out=xo)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(args.steps):
        plan.project(x, out=yo)
    e[1].record()
    for _ in range(args.steps):
        plan.backproject(y, out=xo)
    e[2].record()
    torch.cuda.synchronize()
    nnz = plan.stats()["nnz"]
    tp, tb = e[0].elapsed_time(e[1]) / args.steps, e[1].elapsed_time(e[2]) / args.steps
    st = plan.stats()
    print(json.dumps({"mode": "products", "storage": args.storage, "nnz": nnz, "slices": S,
                      "few_slices": args.few_slices, "paired_rows": args.paired_rows,
                      "narrow_tiles": args.narrow_tiles,
                      "stages_a": st["stages_a"], "stages_at": st["stages_at"],
                      "slots_a": st["slots_a"], "slots_at": st["slots_at"],
                      "bytes_a": st["bytes_a"], "bytes_at": st["bytes_at"],
                      "project_ms": tp, "backproject_ms": tb,
                      "project_gflops": 2.0 * nnz * S / tp / 1e6,
                      "backproject_gflops": 2.0 * nnz * S / tb / 1e6}))


def run_pipeline(args):
    """Products with pinned host vectors over several slice tiles (256
    slices of the workload's geometry): the library's slice-tile pipeline
    (copies on a second stream overlapping the tiles' products) against the
    same work done serially (copy in, product, copy out) and against the
    device-resident product alone."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, xct
    wl = inputs.WORKLOADS[WORKLOAD]
    n, m, nd, S = wl["n"], wl["m"], wl["nd"], 4 * wl["slices"]
    plan = xct.Plan(n, m, nd, args.storage, cos_sin=inputs.angle_table(m))
    nnz = plan.stats()["nnz"]
    g = torch.Generator(device="cuda").manual_seed(0)
    xd = torch.rand((S, n, n), device="cuda", generator=g)
    yd = torch.empty((S, m, nd), device="cuda")
    xh, yh = xd.cpu().pin_memory(), torch.empty((S, m, nd)).pin_memory()
    xd2 = torch.empty_like(xd)
    stream = torch.cuda.current_stream()

    def device_only():
        xct.xct_project(plan.handle, xd, yd, S, stream)

    def serial():
        xd2.copy_(xh, non_blocking=True)
        xct.xct_project(plan.handle, xd2, yd, S, stream)
        yh.copy_(yd, non_blocking=True)

    def pipelined():
        xct.xct_project(plan.handle, xh, yh, S, stream)

    res = {}
    for name, fn in (("device", device_only), ("serial", serial), ("pipelined", pipelined)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / args.steps * 1e3
        res[name] = {"ms": ms, "gflops": 2.0 * nnz * S / (ms * 1e-3) / 1e9}
    ref = yd.cpu()
    pipelined()
    same = bool(torch.equal(yh, ref))
    print(json.dumps({"mode": "pipeline", "storage": args.storage, "slices": S, "nnz": nnz,
                      "h2d_bytes": S * n * n * 4, "d2h_bytes": S * m * nd * 4,
                      "pipelined_equals_device": same, **res,
                      "pipelined_speedup_vs_serial": res["serial"]["ms"] / res["pipelined"]["ms"]}))


def _job_sinos(jobs):
    """Sinograms of the uneven batch, generated on the host cores (spawned
    workers, before any GPU work)."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context

    from paper_2009_07226_gb300 import inputs
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=get_context("spawn")) as ex:
        return list(ex.map(inputs.job_sinograms, jobs))


def _measure_batch(steps, warmup, combos=None):
    """The uneven batch: 64 seeded jobs, N in {256, 384, 512, 768}, M = 1.5 N,
    S ~ U{1..32}, 20 CGLS iterations each.  Mixed precision (binary16) in one
    batched, graph-captured, autotuned call per step, against per-job FP32
    calls (and the two other combinations, to separate batching from
    precision)."""
    from paper_2009_07226_gb300 import inputs
    jobs = inputs.batch_jobs()
    sinos = _job_sinos(jobs)
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct
    K = inputs.BATCH["iters"]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sizes = sorted({j["n"] for j in jobs})
    # binary16 plans with paired layouts for their 64-slice tiles
    plans = {(n, k): xct.Plan(n, 3 * n // 2, n, k, cos_sin=inputs.angle_table(3 * n // 2),
                              paired_rows=(k == "f16"))
             for n in sizes for k in ("f16", "f32")}
    nnz = {n: plans[(n, "f32")].stats()["nnz"] for n in sizes}
    ys = [torch.tensor(s, dtype=torch.float32, device=dev) for s in sinos]
    xs = {k: [torch.empty((j["slices"], j["n"], j["n"]), device=dev) for j in jobs] for k in ("f16", "f32")}
    flops = sum((2 * K + 1) * 2.0 * nnz[j["n"]] * j["slices"] for j in jobs)

    def batched(kind):
        xct.xct_cgls_batch([(plans[(j["n"], kind)].handle, ys[i], xs[kind][i], j["slices"])
                            for i, j in enumerate(jobs)], K, xct.XCT_BATCH_AUTOTUNE, stream)

    def per_job(kind):
        for i, j in enumerate(jobs):
            xct.xct_cgls(plans[(j["n"], kind)].handle, ys[i], xs[kind][i], j["slices"], K, 0, None, stream)

    def timed(fn, kind):
        for _ in range(warmup):
            fn(kind)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = xct.xct_launch_count()
        e0.record(stream)
        for _ in range(steps):
            fn(kind)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, (xct.xct_launch_count() - l0) // steps

    res = {}
    all_combos = (("batched_mixed", batched, "f16"), ("per_job_fp32", per_job, "f32"),
                  ("per_job_mixed", per_job, "f16"), ("batched_fp32", batched, "f32"))
    for name, fn, kind in all_combos:
        if combos and name not in combos:
            continue
        ms, launches = timed(fn, kind)
        res[name] = {"ms_per_step": ms, "gflops": flops / (ms * 1e-3) / 1e9, "gpu_launches": launches}
    batched("f16")
    per_job("f32")
    torch.cuda.synchronize()
    rel = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(xs["f16"], xs["f32"]))
    for p in plans.values():
        p.close()
    return {
        "metric": "proj+backproj GFLOP/s of the uneven batch (2*nnz*S per product)",
        "jobs": len(jobs), "slices": sum(j["slices"] for j in jobs), "iters": K,
        "slices_per_size": {n: sum(j["slices"] for j in jobs if j["n"] == n) for n in sizes},
        "nnz": nnz, "flops_per_step": flops, "plan_flags": {"f16": "XCT_PLAN_PAIRED_ROWS", "f32": ""}, **res,
        "speedup_batched_mixed_vs_per_job_fp32": res["per_job_fp32"]["ms_per_step"] /
                                                  res["batched_mixed"]["ms_per_step"],
        "max_rel_diff_mixed_vs_fp32": rel}


def run_batch(args):
    sampler = ClockSampler(0)
    sampler.start()
    out = _measure_batch(args.steps, args.warmup)
    clocks = sampler.stop()
    print(json.dumps({"mode": "batch", **out, "clocks": clocks}))


def _measure_tv(reps, with_autograd=True):
    """The regularised reconstruction: 1024^2 grid, 720 angles, 1024 bins,
    16 slices, BF16 storage, 200 Adam steps on 0.5 ||A x - y||^2 +
    1e-3 TV_eps (eps 1e-3, lr 1e-2), through the fused native loop and
    through the autograd Functions (PyTorch loop around the same kernels)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import autograd as ag
    from paper_2009_07226_gb300 import inputs, xct
    w = inputs.make_workload("tv3d_1024", with_images=False)
    n, m, nd, S, steps = w["n"], w["m"], w["nd"], w["slices"], w["iters"]
    lam, eps, lr = 1e-3, 1e-3, 1e-2
    stream = torch.cuda.current_stream()
    # 16-slice tiles: the plan orders each 4-row group's entries for them
    plan = xct.Plan(n, m, nd, "bf16", cos_sin=w["cos_sin"], narrow_tiles=True)
    nnz = plan.stats()["nnz"]
    y = torch.tensor(w["sino"], dtype=torch.float32, device="cuda")
    x = torch.empty((S, n, n), device="cuda")
    loss = torch.zeros(steps, dtype=torch.float64, device="cuda")

    def native():
        xct.xct_tv_reconstruct(plan.handle, y, x, S, steps, lr, lam, eps, 0, loss, stream)

    def autograd_loop():
        ag.tv_reconstruct(plan, y, steps=steps, lr=lr, lam=lam, eps=eps)

    res = {}
    runs = [("native", native, reps)] + ([("autograd", autograd_loop, 1)] if with_autograd else [])
    for name, fn, r in runs:
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = xct.xct_launch_count()
        e0.record(stream)
        for _ in range(r):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / r
        res[name] = {"ms_per_run": ms, "ms_per_adam_step": ms / steps,
                     "gflops": steps * 2 * 2.0 * nnz * S / (ms * 1e-3) / 1e9,
                     "gpu_launches_per_run": (xct.xct_launch_count() - l0) // r}
    native()
    lh = loss.cpu().numpy()
    plan.close()
    return {"metric": "Adam steps/s and product GFLOP/s (2 products of 2*nnz*S flops per step)",
            "n": n, "angles": m, "bins": nd, "slices": S, "steps": steps, "storage": "bf16",
            "plan_flags": "XCT_PLAN_NARROW_TILES", "nnz": nnz, **res, "cost_first": float(lh[0]), "cost_last": float(lh[-1])}


def run_tv(args):
    sampler = ClockSampler(0)
    sampler.start()
    out = _measure_tv(args.steps)
    clocks = sampler.stop()
    print(json.dumps({"mode": "tv", **out, "clocks": clocks}))


def _measure_large(steps, warmup):
    """The large geometry: 1536^2 grid, 1024 angles, 1536 bins (A with about
    2.9e9 entries), 32 slices, 30 CGLS iterations, binary16 storage against
    FP32."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context

    from paper_2009_07226_gb300 import inputs
    wl = inputs.WORKLOADS["large3d_1536"]
    S = wl["slices"]
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=get_context("spawn")) as ex:
        parts = list(ex.map(_large_slices, [(s0, min(4, S - s0)) for s0 in range(0, S, 4)]))
    sino = np.concatenate(parts)
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import xct
    n, m, nd, K = wl["n"], wl["m"], wl["nd"], wl["iters"]
    stream = torch.cuda.current_stream()
    y = torch.tensor(sino, dtype=torch.float32, device="cuda")
    res = {}
    xs = {}
    for kind in ("f16", "f32"):
        # 32-slice tiles: the binary16 plan orders each 4-row group's entries
        # for them (XCT_PLAN_NARROW_TILES needs a 16-bit matrix)
        plan = xct.Plan(n, m, nd, kind, cos_sin=inputs.angle_table(m), narrow_tiles=(kind == "f16"))
        st = plan.stats()
        x = torch.empty((S, n, n), device="cuda")
        for _ in range(warmup):
            xct.xct_cgls(plan.handle, y, x, S, K, xct.XCT_CGLS_TIMING, None, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tp = tb = 0.0
        e0.record(stream)
        for _ in range(steps):
            xct.xct_cgls(plan.handle, y, x, S, K, xct.XCT_CGLS_TIMING, None, stream)
            ps = plan.stats()
            tp += ps["t_project_ms"] / max(ps["n_project"], 1)
            tb += ps["t_backproject_ms"] / max(ps["n_backproject"], 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        flops = (2 * K + 1) * 2.0 * st["nnz"] * S
        res[kind] = {"ms_per_solve": ms, "gflops": flops / (ms * 1e-3) / 1e9,
                     "plan_flags": "XCT_PLAN_NARROW_TILES" if kind == "f16" else "",
                     "project_ms": tp / steps, "backproject_ms": tb / steps,
                     "plan_ms": st["plan_ms"], "bytes_a": st["bytes_a"], "bytes_at": st["bytes_at"]}
        xs[kind] = x
        plan.close()
        torch.cuda.empty_cache()
    rel = float(torch.linalg.norm(xs["f16"] - xs["f32"]) / torch.linalg.norm(xs["f32"]))
    return {"n": n, "angles": m, "bins": nd, "slices": S, "iters": K,
            "nnz": st["nnz"], **res, "speedup_mixed_vs_fp32": res["f32"]["ms_per_solve"] /
            res["f16"]["ms_per_solve"], "rel_diff_mixed_vs_fp32": rel}


def run_large(args):
    sampler = ClockSampler(0)
    sampler.start()
    out = _measure_large(args.steps, args.warmup)
    clocks = sampler.stop()
    print(json.dumps({"mode": "large", **out, "clocks": clocks}))


def run_cusparse(args):
    """Comparison point: cuSPARSE SpMM (through torch.sparse, FP32 CSR times
    a dense [columns, S] block) on the same A and A^T as the library's FP32
    and binary16 products, 512^2 x 768 x 512, 64 slices."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, xct
    wl = inputs.WORKLOADS[WORKLOAD]
    n, m, nd, S = wl["n"], wl["m"], wl["nd"], wl["slices"]
    cs = inputs.angle_table(m)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"mode": "cusparse", "n": n, "angles": m, "bins": nd, "slices": S}
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((S, n, n), device="cuda", generator=g)
    y = torch.rand((S, m, nd), device="cuda", generator=g)
    with xct.Plan(n, m, nd, "f32", cos_sin=cs) as p32:
        nnz = p32.stats()["nnz"]
        mats = {}
        for name, what in (("A", xct.XCT_EXPORT_A_STORED), ("At", xct.XCT_EXPORT_AT_STORED)):
            rp, col, val = xct.xct_plan_export(p32.handle, what)
            mats[name] = torch.sparse_csr_tensor(torch.from_numpy(rp), torch.from_numpy(col.astype(np.int64)),
                                                 torch.from_numpy(val.astype(np.float32)),
                                                 size=(len(rp) - 1, m * nd if name == "At" else n * n)).cuda()
        xb = x.reshape(S, -1).t().contiguous()          # [pixels, S]
        yb = y.reshape(S, -1).t().contiguous()          # [rays, S]
        out["cusparse_project_ms"] = timed(lambda: torch.sparse.mm(mats["A"], xb), 10)
        out["cusparse_backproject_ms"] = timed(lambda: torch.sparse.mm(mats["At"], yb), 10)
        q = torch.sparse.mm(mats["A"], xb).t().reshape(S, m, nd)
        yo = torch.empty_like(y)
        out["xct_f32_project_ms"] = timed(lambda: p32.project(x, out=yo), 10)
        out["max_rel_diff_f32_vs_cusparse"] = float((yo - q).abs().max() / q.abs().max())
        xo = torch.empty_like(x)
        out["xct_f32_backproject_ms"] = timed(lambda: p32.backproject(y, out=xo), 10)
    with xct.Plan(n, m, nd, "f16", cos_sin=cs) as p16:
        yo = torch.empty_like(y)
        xo = torch.empty_like(x)
        out["xct_f16_project_ms"] = timed(lambda: p16.project(x, out=yo), 10)
        out["xct_f16_backproject_ms"] = timed(lambda: p16.backproject(y, out=xo), 10)
    for k in ("cusparse_project_ms", "xct_f32_project_ms", "xct_f16_project_ms"):
        out[k.replace("_ms", "_gflops")] = 2.0 * nnz * S / (out[k] * 1e-3) / 1e9
    out["note"] = ("library products include the natural <-> internal layout conversions (and the "
                   "16-bit staging); cuSPARSE is given the dense block already transposed")
    print(json.dumps(out))


def run_matfree(args):
    """Memoized against matrix-free projection and back projection (Sec.
    II-B's argument for memoizing A), 512^2 x 768 x 512, FP32 and binary16
    plans."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_07226_gb300 import inputs, xct
    wl = inputs.WORKLOADS[WORKLOAD]
    n, m, nd = wl["n"], wl["m"], wl["nd"]
    out = {"mode": "matfree", "n": n, "angles": m, "bins": nd}
    with xct.Plan(n, m, nd, "f32", cos_sin=inputs.angle_table(m)) as p32, \
            xct.Plan(n, m, nd, "f16", cos_sin=inputs.angle_table(m)) as p16:
        nnz = p32.stats()["nnz"]
        out["nnz"] = nnz
        for S in (8, 64):
            g = torch.Generator(device="cuda").manual_seed(0)
            x = torch.rand((S, n, n), device="cuda", generator=g)
            y = torch.empty((S, m, nd), device="cuda")

            def timed(fn, reps):
                fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                return e0.elapsed_time(e1) / reps

            t_mf = timed(lambda: xct.xct_project_matfree(p32.handle, x, y, S), max(1, args.steps // 3))
            t32 = timed(lambda: p32.project(x, out=y), args.steps)
            t16 = timed(lambda: p16.project(x, out=y), args.steps)
            # back projection: pixel by pixel without the matrix
            t_bmf = timed(lambda: xct.xct_backproject_matfree(p32.handle, y, x, S),
                          max(1, args.steps // 3))
            tb32 = timed(lambda: p32.backproject(y, out=x), args.steps)
            tb16 = timed(lambda: p16.backproject(y, out=x), args.steps)
            out[f"S{S}"] = {"matfree_ms": t_mf, "memoized_f32_ms": t32, "memoized_f16_ms": t16,
                            "matfree_gflops": 2.0 * nnz * S / (t_mf * 1e-3) / 1e9,
                            "speedup_memoized_f32": t_mf / t32, "speedup_memoized_f16": t_mf / t16,
                            "back_matfree_ms": t_bmf, "back_memoized_f32_ms": tb32,
                            "back_memoized_f16_ms": tb16,
                            "back_matfree_gflops": 2.0 * nnz * S / (t_bmf * 1e-3) / 1e9,
                            "back_speedup_memoized_f16": t_bmf / tb16}
        # CGLS without the stored matrix: 8 slices, 3 iterations (7 products)
        S, K = 8, 3
        g = torch.Generator(device="cuda").manual_seed(1)
        y8 = torch.rand((S, m, nd), device="cuda", generator=g)
        x8 = torch.empty((S, n, n), device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        xct.xct_cgls_matfree(p32.handle, y8, x8, S, K)
        ev[1].record()
        xct.xct_cgls(p16.handle, y8, x8, S, K, 0, None)
        ev[2].record()
        torch.cuda.synchronize()
        out["cgls_S8_3iters"] = {"matfree_ms": ev[0].elapsed_time(ev[1]),
                                 "memoized_f16_ms": ev[1].elapsed_time(ev[2])}
    print(json.dumps(out))


def _large_slices(arg):
    s0, count = arg
    from paper_2009_07226_gb300 import inputs
    return inputs.make_workload("large3d_1536", slices=count, slice_offset=s0, with_images=False)["sino"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other configurations' compact measurements in the default line")
    ap.add_argument("--mode", default="cgls", choices=["cgls", "products", "batch", "tv", "large", "cusparse", "matfree",
                             "pipeline", "roof"])
    ap.add_argument("--storage", default="f16", choices=["f32", "f16", "bf16", "f16a", "bf16a"])
    ap.add_argument("--slices", type=int, default=0,
                    help="--mode products: slices per product (default: the workload's 64)")
    ap.add_argument("--few-slices", action="store_true",
                    help="--mode products: build the plan with XCT_PLAN_FEW_SLICES (wide-stage layouts)")
    ap.add_argument("--paired-rows", action="store_true",
                    help="--mode products: build the plan with XCT_PLAN_PAIRED_ROWS (paired layouts, 64-slice tiles)")
    ap.add_argument("--narrow-tiles", action="store_true",
                    help="--mode products: build the plan with XCT_PLAN_NARROW_TILES")
    args = ap.parse_args()
    if args.mode == "products":
        run_products(args)
    elif args.mode == "roof":
        run_roof(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "tv":
        run_tv(args)
    elif args.mode == "large":
        run_large(args)
    elif args.mode == "cusparse":
        run_cusparse(args)
    elif args.mode == "matfree":
        run_matfree(args)
    elif args.mode == "pipeline":
        run_pipeline(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
