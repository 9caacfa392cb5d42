"""Throughput benchmark of the fused non-ideal LBM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload tgv256|tgv256-fp64|tgv256-fp16dev|riemann|shockdrop2d|column2d|
                                shockdrop3d|batched|shocktube3d|shocktube3d-mlp|strongshock3d|...]

Prints one JSON line (rank 0).  A step is one full time step of the method
(stream, moments, EOS, correction terms, collide, boundary fill) over the
whole lattice.  ``value`` is MLUPS (million lattice-node updates per second)
with the state resident in HBM; ``e2e`` is the same metric through the C
interface with host buffers: lbm_init from pinned host fields, K calls of
lbm_step(h, 1) (each reads the 4-byte status word back), lbm_moments to host.
With N GPUs (torchrun) every rank runs an independent replica of the
workload (the solver is single-GPU); the value is the sum over ranks of the
updates divided by the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle (the only other place this
file runs oracle code) on a bounded sample of the workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (builder kwargs, precision, description)
    "tgv256": ("tgv", dict(N=256), "fp32", "D3Q27 compressible Taylor-Green vortex 256^3, vdW dense vapour, FP32"),
    "tgv128": ("tgv", dict(N=128), "fp32", "D3Q27 Taylor-Green 128^3, FP32 (small profiling case)"),
    "tgv256-fp64": ("tgv", dict(N=256), "fp64", "D3Q27 compressible Taylor-Green vortex 256^3, FP64"),
    "tgv256-pr": ("tgv", dict(N=256, scenario_name="tgv_pr_d3q27"), "fp32",
                  "D3Q27 compressible Taylor-Green vortex 256^3 in a Peng-Robinson fluid (nitrogen-like; temperature "
                  "from the caloric relation, inverted per node), FP32"),
    "tgv256-fp16dev": ("tgv", dict(N=256), "fp16dev", "D3Q27 Taylor-Green 256^3, FP16-deviation storage"),
    "riemann": ("riemann", dict(), "fp64", "D2Q9 non-ideal Riemann problem 1000x4, FP64"),
    "shockdrop2d": ("shock_column", dict(D=2, shape=(4096, 2048), radius=128), "fp32",
                    "D2Q9 shock-drop 4096x2048: liquid column radius 128, tanh width 3, Ma 1.47 shock; the paper's "
                    "saturated liquid/vapour at T_r 0.9 (U^2 = 35), shock capturing C_mu = C_k = 0.3, FP32"),
    "column2d": ("shock_column", dict(D=2, shape=(800, 800), radius=65), "fp32",
                 "D2Q9 shock-liquid column 800x800 (radius 65, Ma 1.47, saturated at T_r 0.9): the paper's case, "
                 "shock capturing C_mu = C_k = 0.3, FP32"),
    "shockdrop3d": ("shock_column", dict(D=3, shape=(512, 256, 256), radius=32), "fp32",
                    "D3Q27 shock-drop 512x256x256: saturated liquid sphere radius 32 at T_r 0.9, Ma 1.47 shock "
                    "(U^2 = 35), shock capturing C_mu = C_k = 0.3, FP32"),
    "batched": ("batch", dict(), "fp32",
                "256 uneven D2Q9 shock tubes (128x64 .. 1024x512, Ma 1.1-1.3), one persistent launch per step, FP32"),
    "batched-drops": ("batch_columns", dict(), "fp32",
                      "256 uneven D2Q9 instances (128x64 .. 1024x512), about half with a liquid column (radius 9-64), "
                      "Ma 1.1-1.5 shocks, saturated liquid/vapour at T_r 0.9 (U^2 = 35), shock capturing C_mu = C_k "
                      "= 0.3 in the batched step, one graph launch per step, FP32"),
    "shockdrop3d-mlp": ("shock_column", dict(D=3, shape=(512, 256, 256), radius=32), "fp32",
                        "D3Q27 shock-drop 512x256x256: saturated liquid sphere radius 32 at T_r 0.9, Ma 1.47 shock "
                        "(U^2 = 35), shock capturing C_mu = C_k = 0.3, learned closure (2-64-64-3 BF16 MLP trained on "
                        "column and tube states of this fluid), FP32"),
    "shocktube3d-mlp": ("shock_tube_3d", dict(shape=(512, 256, 256), Ma=1.15, seed=21), "fp32",
                        "D3Q27 shock tube 512x256x256 (Ma 1.15), learned closure (2-64-64-3 BF16 MLP), FP32"),
    "shocktube3d": ("shock_tube_3d", dict(shape=(512, 256, 256), Ma=1.15, seed=21), "fp32",
                    "D3Q27 shock tube 512x256x256 (Ma 1.15), exact closure, FP32"),
    "strongshock3d": ("strong_shock", dict(D=3, shape=(512, 256, 256), seed=21), "fp32",
                      "D3Q27 shock tube 512x256x256 at the workloads' Ma 1.47 (U^2 = 16), shock capturing "
                      "C_mu = C_k = 0.3, FP32"),
    "strongshock3d-mlp": ("strong_shock", dict(D=3, shape=(512, 256, 256), seed=21), "fp32",
                          "D3Q27 shock tube 512x256x256 at Ma 1.47 (U^2 = 16), shock capturing C_mu = C_k = 0.3, "
                          "learned closure (2-64-64-3 BF16 MLP), FP32"),
    "shocktube3d-mlp-small": ("shock_tube_3d", dict(shape=(256, 128, 128), Ma=1.15, seed=21), "fp32",
                              "D3Q27 shock tube 256x128x128 (Ma 1.15), learned closure, FP32 (profiling case)"),
}
# workloads whose step uses the learned closure, trained before the timed region
# learned-closure workloads: training-run table, largest Mach number, scenario of the units,
# number of 2-D shock-liquid column runs among the training runs
MLP_WORKLOADS = {"shocktube3d-mlp": ("batch_d2q9", 1.25, "shock_drop_d3q27", 0),
                 "shocktube3d-mlp-small": ("batch_d2q9", 1.25, "shock_drop_d3q27", 0),
                 "strongshock3d-mlp": ("strong_posts_d2q9", 1.5, "strong_shock_d3q27", 0),
                 "shockdrop3d-mlp": ("batch_columns_d2q9", 1.5, "column_d3q27", 3)}
# workloads that run with shock capturing (C_mu, C_eta, C_k)
SC_WORKLOADS = {"strongshock3d": (0.3, 0.0, 0.3), "strongshock3d-mlp": (0.3, 0.0, 0.3),
                "shockdrop2d": (0.3, 0.0, 0.3), "column2d": (0.3, 0.0, 0.3), "shockdrop3d": (0.3, 0.0, 0.3),
                "batched-drops": (0.3, 0.0, 0.3), "shockdrop3d-mlp": (0.3, 0.0, 0.3)}
MLP_TRAIN = dict(snapshots=50, every=20, batch=8192, steps=60000, lr0=3e-3, lr1=1e-6, seed=5, net_seed=11)
BYTES = {"fp64": 8, "fp32": 4, "fp16dev": 2}
# Longest run from the initial state that stays finite, per (builder, precision):
# the Ma 0.5 Taylor-Green vortex at 256^3 develops a blow-up after ~250 steps in
# FP32 (~150 in FP16-deviation) without extra dissipation, so timed steps are
# taken in chunks from the initial state (re-initialised outside the timing).
# The shock-column runs stay finite to about t / t0 = 0.85 (1860 steps on the 4096 x
# 2048 grid: the rarefaction reflected at the column's rear drives the liquid to
# negative pressure), so they too are timed in chunks.
# In the batched shock-drop table the smallest columns (128 x 64, radius 14, Ma ~1.5)
# reach their outflow face within 500-750 steps, where the zero-gradient outflow
# fails.
MAX_CHUNK = {("tgv", "fp32"): 200, ("tgv", "fp16dev"): 100, ("tgv", "fp64"): 400, ("strong_shock", "fp32"): 500,
             ("shock_column", "fp32"): 1500, ("batch_columns", "fp32"): 400}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16dev": "f16-storage/f32"}


def build_case(name):
    import inputs
    builder, kw, prec, desc = WORKLOADS[name]
    return getattr(inputs, builder)(**kw), prec, desc


def kernel_sources():
    """Every file the library is built from: all of csrc/, the public headers and the build script."""
    pkg = os.path.join(ROOT, "paper_2510_14712_gb300")
    src = os.path.join(pkg, "csrc")
    inc = os.path.join(ROOT, "include")
    files = [os.path.join(src, f) for f in sorted(os.listdir(src))]
    files += [os.path.join(inc, f) for f in sorted(os.listdir(inc))]
    return files + [os.path.join(pkg, "build.py")]


def kernel_hash():
    """Hash of the sources and build flags of the library (traffic counters in
    profiles/traffic.json are used only while it matches)."""
    h = hashlib.sha256()
    for p in kernel_sources():
        if os.path.isfile(p):
            h.update(os.path.basename(p).encode())
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(workload):
    """ncu DRAM bytes per step from profiles/traffic.json, if taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_step")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.path = os.path.join("/tmp", "lbm_clocks_%d.csv" % os.getpid())
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, device=None):
    """The largest value of x over all ranks (x itself on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(nodes, steps, world, seconds):
    """Whole-job throughput of `world` replicas, each updating `nodes` nodes `steps`
    times, timed by the slowest rank (weak scaling)."""
    return nodes * steps * world / seconds / 1e6


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def cpu_model():
    """CPU model name of the host (lscpu / /proc/cpuinfo), or the machine type."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _run_children(codes, timeout=600):
    procs = [subprocess.Popen([sys.executable, "-c", c], cwd=ROOT, env=_oracle_env(), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for c in codes]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        if p.returncode != 0:
            return None, (e.strip().splitlines()[-1] if e else "oracle leg failed")
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return outs, None


def cpu_oracle_leg(workload, seconds=12.0, steps=None, warmup=1, save=None, all_cores=True):
    """Time the FP64 oracle on a bounded sample of the workload in child processes.

    One process on one core (as many steps as fit in ``seconds``, or ``steps``),
    saving its final fields to ``save`` when given; then, with ``all_cores``, one
    process per host core, each stepping its own copy of the sample the same
    number of steps from a common start time.  ``value`` is the all-core
    figure: the node updates of every process over the common wall time.
    """
    code = ("import bench, json; print(json.dumps(bench._oracle_sample(%r, %r, %r, %r, save=%r)))"
            % (workload, seconds, steps, warmup, save))
    outs, err = _run_children([code])
    if err:
        return {"error": err}
    one = outs[0]
    res = {"value": one["value"], "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": one["sample"],
           "model": cpu_model(), "single_core": {"value": one["value"], "sample": one["sample"]}}
    if not all_cores:
        return res
    n = host_cores()
    k = one["steps"]
    t_start = time.time() + 3.0 + 0.05 * n          # every child has imported and built its case by then
    codes = ["import bench, json; print(json.dumps(bench._oracle_sample(%r, None, %r, %r, start_at=%r)))"
             % (workload, k, warmup, t_start) for _ in range(n)]
    outs, err = _run_children(codes)
    if err:
        res["all_cores_error"] = err
        return res
    wall = max(o["t_end"] for o in outs) - t_start
    late = max(o["t_begin"] for o in outs) - t_start
    updates = sum(o["nodes"] * o["steps"] for o in outs)
    res.update(value=updates / wall / 1e6, cores=n,
               sample="%s; %d processes (one per core, %s), %d steps each, common wall time %.1f s "
                      "(last start %.2f s after the common start)" % (one["sample_case"], n, res["model"], k, wall,
                                                                        late))
    return res


def _sample_case(workload):
    """The bounded oracle sample of a workload: (case, description)."""
    import inputs
    builder, kw, prec, _ = WORKLOADS[workload]
    if builder == "tgv":
        case = inputs.tgv(shape=(48, 48, 48), scenario_name=kw.get("scenario_name", "tgv_d3q27"))
        sample = "D3Q27 Taylor-Green 48^3 box (same state, k scaled%s), FP64 oracle" % (
            ", Peng-Robinson fluid, Newton temperature" if "scenario_name" in kw else "")
    elif builder == "riemann":
        case = inputs.riemann()
        sample = "D2Q9 Riemann 1000x4 (the full workload), FP64 oracle"
    elif builder == "batch":
        case = inputs.batch(1)[0]
        sample = "D2Q9 shock tube %dx%d (instance 0 of the batch), FP64 oracle" % case.shape
    elif builder == "batch_columns":
        tab = inputs.scenario("batch_columns_d2q9")["instances"]
        k = min((d["Nx"] * d["Ny"], k) for k, d in enumerate(tab) if d["radius"] > 0)[1]
        case = inputs.batch_columns(k + 1)[k]
        sample = ("D2Q9 shock-liquid column %dx%d (instance %d of the batch, the smallest with a column) with shock "
                  "capturing, FP64 oracle" % (case.shape + (k,)))
    elif builder == "shock_tube_3d":
        case = inputs.shock_tube_3d(shape=(128, 8, 8), Ma=kw["Ma"], seed=kw["seed"])
        sample = "D3Q27 shock tube 128x8x8 down-scale, exact closure, FP64 oracle"
    elif builder == "strong_shock":
        case = inputs.strong_shock(3, (128, 8, 8), seed=kw["seed"])
        sample = "D3Q27 Ma 1.47 shock tube 128x8x8 down-scale with shock capturing, FP64 oracle"
    elif builder == "shock_column" and kw["D"] == 2:
        case = inputs.shock_column(2, (512, 256), radius=16, center=(128, 128), shock_x=64)
        sample = "D2Q9 shock-liquid column 512x256 down-scale (radius 16) with shock capturing, FP64 oracle"
    else:
        case = inputs.shock_column(3, (128, 64, 64), radius=8, center=(32, 32, 32), shock_x=16)
        sample = "D3Q27 shock-liquid sphere 128x64x64 down-scale (radius 8) with shock capturing, FP64 oracle"
    return case, sample


def _oracle_sample(workload, seconds, steps=None, warmup=1, save=None, start_at=None):
    """Oracle MLUPS on a sub-box of the workload: same physics, fewer nodes, few steps.

    With ``steps`` given, exactly that many timed steps after ``warmup``;
    otherwise as many as fit in ``seconds`` (at most 1000).  ``start_at``: a
    time.time() to wait for before the timed steps.  ``save``: an .npz path for
    the final rho, u, T (and the total step count).
    """
    import numpy as np
    from oracle import lbm as olbm
    case, sample = _sample_case(workload)
    m = olbm.Model(case.D, case.shape, case.eos, case.tau, case.Pr, case.cv, case.x_low, case.x_high)
    m.shock_capturing = SC_WORKLOADS.get(workload)
    s = olbm.Sim(m, case.rho, case.u, case.T)
    s.step(warmup)
    if start_at is not None:
        time.sleep(max(0.0, start_at - time.time()))
    done, t_begin = 0, time.time()
    t0 = time.perf_counter()
    while True:
        s.step(1)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and (el > seconds or done >= 1000)):
            break
    t_end = time.time()
    n = int(np.prod(case.shape))
    if save:
        F = s.fields()
        np.savez(save, rho=F["rho"], u=np.stack(F["u"]), T=F["T"], steps=warmup + done)
    return {"value": n * done / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle", "nodes": n, "steps": done,
            "t_begin": t_begin, "t_end": t_end, "sample_case": sample,
            "sample": "%s, %d steps, %.1f s, 1 thread" % (sample, done, el)}


def l2_vs_oracle(P, workload, prec, path, t64=False):
    """Relative L2 error of the GPU path against the oracle's final fields of the CPU
    leg (same sample box, same steps, the line's precision)."""
    import numpy as np
    if not path or not os.path.exists(path):
        return None
    ref = np.load(path)
    steps = int(ref["steps"])
    case, sample = _sample_case(workload)
    s = P.Solver(case, precision=prec, t_fp64=t64)
    try:
        sc = SC_WORKLOADS.get(workload)
        if sc:
            P.lbm_set_shock_capturing(s.h, *sc)
        s.init().step(steps)
        got = s.fields()
    finally:
        s.close()
    err = {}
    for k in ("rho", "u", "T"):
        a, b = np.asarray(got[k]), np.asarray(ref[k])
        err[k] = float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
    err.update(steps=steps, box="x".join(str(v) for v in case.shape), against="FP64 CPU oracle",
               closure="exact", sample=sample.replace(", FP64 oracle", ""))
    return err


def run_reference(args):
    """The FP64 oracle on all host cores: W warm-up and K timed steps of the bounded sample per core."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    desc = WORKLOADS[args.workload][3]
    r = cpu_oracle_leg(args.workload, steps=args.steps, warmup=args.warmup)
    if "error" in r:
        print(json.dumps({"impl": "reference", "unavailable": r["error"]}))
        return 0
    v = r["value"]
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "impl": "FP64 CPU oracle (numpy), bounded sample, one process per host core"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"], "model": r.get("model"), "single_core": r.get("single_core")},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """The batched form: all instances advance per step in one graph of two launches."""
    import numpy as np
    import torch
    import inputs
    from paper_2510_14712_gb300 import build
    build.build()
    import paper_2510_14712_gb300 as P
    rank, world, local = dist_env()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    builder = WORKLOADS[args.workload][0]
    cases = getattr(inputs, builder)()
    prec = args.precision or "fp32"
    b = P.Batch(cases, precision=prec)
    P._bcheck(P.load().lbm_batch_set_stream(b.b, ctypes_void_p(stream.cuda_stream)))
    sc_coef = SC_WORKLOADS.get(args.workload)
    if sc_coef:
        b.set_shock_capturing(*sc_coef)
    b.init()
    tile = b.autotune(3)
    N = b.nodes()
    # chunks of at most `chunk` steps from the initial state (re-initialised outside the timing)
    chunk = MAX_CHUNK.get((builder, prec), 1 << 30)
    b.step(min(args.warmup, chunk))
    torch.cuda.synchronize(dev)
    ms, done, launches, nchunks = 0.0, 0, 0, 0
    while done < args.steps:
        k = min(chunk, args.steps - done)
        if nchunks > 0 or min(args.warmup, chunk) + k > chunk:
            b.init()
            torch.cuda.synchronize(dev)
        l0 = b.launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.step_async(k)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        b.sync()
        ms += ev0.elapsed_time(ev1)
        launches += b.launches() - l0
        done += k
        nchunks += 1
    alg = sum(4 * c.lattice * BYTES[prec] * c.nodes for c in cases)
    achieved = alg / (ms * 1e-3 / args.steps) / 1e9
    peak, peak_kind = measured_peaks()
    b.close()
    line = {"metric": "MLUPS", "value": N * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][3], "nodes": N, "instances": len(cases),
                       "tile_shape": tile[0], "graph_captured": True, "shock_capturing": sc_coef,
                       "timed_chunk_steps": min(chunk, args.steps)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "batched step (persistent fused kernel + ghost fill%s)"
                         % (" + batched shock-capturing stencils" if sc_coef else ""),
                         "algorithmic_bytes_per_step": alg, "peak_source": peak_kind},
            "e2e": None, "gpu_launches": launches}
    if not args.no_cpu:
        import tempfile
        path = os.path.join(tempfile.gettempdir(), "lbm_oracle_%d.npz" % os.getpid())
        line["cpu_baseline"] = cpu_oracle_leg(args.workload, save=path)
        try:
            line["l2_error"] = l2_vs_oracle(P, args.workload, prec, path)
        finally:
            if os.path.exists(path):
                os.unlink(path)
    print(json.dumps(line))
    return 0


def ctypes_void_p(v):
    import ctypes
    return ctypes.c_void_p(v)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2510_14712_gb300 import build
    build.build()
    import paper_2510_14712_gb300 as P

    case, prec, desc = build_case(args.workload)
    if args.precision:
        prec = args.precision
    N = case.nodes
    stream = torch.cuda.current_stream(dev)
    sk = P.LBM_STEP_MULTIPASS if args.step_kernel == "multipass" else P.LBM_STEP_FUSED
    t64 = args.t64
    solver = P.Solver(case, precision=prec, stream=stream.cuda_stream, step_kernel=sk, t_fp64=t64)
    sc_coef = SC_WORKLOADS.get(args.workload)
    if sc_coef:
        P.lbm_set_shock_capturing(solver.h, *sc_coef)
    rho = torch.from_numpy(np.ascontiguousarray(case.rho, dtype=np.float64)).to(dev)
    u = torch.from_numpy(np.ascontiguousarray(np.stack(case.u), dtype=np.float64)).to(dev)
    T = torch.from_numpy(np.ascontiguousarray(case.T, dtype=np.float64)).to(dev)
    P.lbm_init_device(solver.h, rho, u, T)
    closure_info, net = None, None
    if args.workload in MLP_WORKLOADS:
        # same case with the exact closure first: tuned, then timed like the main loop
        net, closure_info = train_closure(P, dev, args.workload, args.train_mma)
        if not args.no_autotune:
            P.lbm_autotune(solver.h, 3)
        P.lbm_step(solver.h, args.warmup)
        ne = min(args.steps, 100)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        P.lbm_step_async(solver.h, ne)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        P.lbm_sync(solver.h)
        closure_info["exact_closure_ms_per_step"] = e0.elapsed_time(e1) / ne
        P.lbm_init_device(solver.h, rho, u, T)
        net.attach(solver)
    tile, tile_ms = None, None
    if sk == P.LBM_STEP_FUSED and not args.no_autotune:
        tile = P.lbm_autotune(solver.h, 3)
        tile_ms = P.lbm_autotune_times(solver.h)

    if args.graphs:
        P.lbm_set_graphs(solver.h, True)
    # warm-up
    builder = WORKLOADS[args.workload][0]
    chunk = MAX_CHUNK.get((builder, prec), 1 << 30)
    P.lbm_step(solver.h, min(args.warmup, chunk))
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()

    # timed region: device events around every step on the solver's stream;
    # chunks of at most `chunk` steps start from the initial state
    cvd = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    phys = cvd[dev.index] if dev.index < len(cvd) and cvd[dev.index].isdigit() else str(dev.index)
    clocks = ClockSampler(phys)
    time.sleep(0.4)
    launches0 = P.lbm_launch_count(solver.h)
    step_ms, done, nchunks = [], 0, 0
    while done < args.steps:
        k = min(chunk, args.steps - done)
        P.lbm_init_device(solver.h, rho, u, T)             # back to the initial state, not timed
        torch.cuda.synchronize(dev)
        if args.graphs:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.lbm_step_async(solver.h, k)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            P.lbm_sync(solver.h)
            step_ms += [e0.elapsed_time(e1) / k] * k
        else:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
            ev[0].record(stream)
            for j in range(k):
                P.lbm_step_async(solver.h, 1)
                ev[j + 1].record(stream)
            torch.cuda.synchronize(dev)
            P.lbm_sync(solver.h)
            step_ms += [ev[j].elapsed_time(ev[j + 1]) for j in range(k)]
        done += k
        nchunks += 1
    launches = P.lbm_launch_count(solver.h) - launches0
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = replica_mlups(N, args.steps, world, total_ms * 1e-3)

    # roofline of the step kernel(s): algorithmic 4 Q s bytes per node update
    Q = case.lattice
    alg_bytes = 4 * Q * BYTES[prec] * N
    avg_step_s = statistics.mean(step_ms) * 1e-3
    achieved = alg_bytes / avg_step_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profile_traffic(args.workload + ":" + prec)
    flags = P.lbm_get_flags(solver.h)
    solver.close()

    # end to end through the C interface with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        h_rho = torch.from_numpy(np.ascontiguousarray(case.rho, dtype=np.float64)).pin_memory()
        h_u = torch.from_numpy(np.ascontiguousarray(np.stack(case.u), dtype=np.float64)).pin_memory()
        h_T = torch.from_numpy(np.ascontiguousarray(case.T, dtype=np.float64)).pin_memory()
        o_rho, o_u, o_T = torch.empty_like(h_rho).pin_memory(), torch.empty_like(h_u).pin_memory(), \
            torch.empty_like(h_T).pin_memory()
        tot = np.empty(case.D + 2)
        s2 = P.Solver(case, precision=prec, stream=stream.cuda_stream, step_kernel=sk, t_fp64=t64)
        if sc_coef:
            P.lbm_set_shock_capturing(s2.h, *sc_coef)
        if net is not None:
            net.attach(s2)
        lib = P.load()
        import ctypes
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        done2, inits = 0, 0
        while done2 < args.steps:
            k = min(chunk, args.steps - done2)
            P._check(lib.lbm_init(s2.h, vp(h_rho), vp(h_u), vp(h_T)))
            inits += 1
            for _ in range(k):
                P._check(lib.lbm_step(s2.h, 1))
            done2 += k
        P._check(lib.lbm_moments(s2.h, vp(o_rho), vp(o_u), vp(o_T), tot.ctypes.data_as(ctypes.c_void_p)))
        el = max_over_ranks(time.perf_counter() - t0, dev)
        s2.close()
        fb = N * (case.D + 2) * 8
        e2e = {"value": replica_mlups(N, args.steps, world, el), "unit": "MLUPS",
               "h2d_bytes_per_step": fb * inits / args.steps,
               "d2h_bytes_per_step": 4 + (fb + 8 * (case.D + 2)) / args.steps}

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": desc, "nodes": N, "lattice": "D%dQ%d" % (case.D, Q), "precision": prec,
                       "parallelism": "replicas" if world > 1 else "single-gpu",
                       "tile_shape": tile[0] if tile else None, "tile_candidates_ms": tile_ms,
                       "timed_chunk_steps": min(chunk, args.steps), "cuda_graphs": bool(args.graphs),
                       "shock_capturing": list(sc_coef) if sc_coef else None,
                       "temperature_inversion": ("fp64" if t64 else "fp32") if prec != "fp64" else "fp64",
                       "l2": "state %.1f GB >> 129 MB L2 (no flush needed)" % (2 * Q * BYTES[prec] * N / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "step (%s: all launches of one time step)" % args.step_kernel,
                         "algorithmic_bytes_per_step": alg_bytes, "peak_source": peak_kind},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "status_flags": flags,
        }
        if closure_info is not None:
            em = closure_info["exact_closure_ms_per_step"]
            closure_info["exact_closure_mlups"] = N / (em * 1e-3) / 1e6
            closure_info["gain_vs_exact"] = value / world / closure_info["exact_closure_mlups"]
            closure_info["accuracy"] = closure_accuracy(P, net, args.workload)
            line["closure"] = closure_info
        if not args.no_cpu:
            # the oracle on the host cores; its single-core run's final fields give the
            # line's stated error: the same sample box on the GPU, same steps, the line's precision
            import tempfile
            path = os.path.join(tempfile.gettempdir(), "lbm_oracle_%d.npz" % os.getpid())
            line["cpu_baseline"] = cpu_oracle_leg(args.workload, save=path)
            try:
                line["l2_error"] = l2_vs_oracle(P, args.workload, prec, path, t64)
            finally:
                if os.path.exists(path):
                    os.unlink(path)
        print(json.dumps(line))
    if net is not None:
        net.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


CLOSURE_ACCURACY_STEPS = 400


def closure_accuracy(P, net, workload):
    """Density error of the learned closure in FP32, beside that of the exact closure in FP32, against the exact
    closure in FP64 (relative L2 after CLOSURE_ACCURACY_STEPS steps), on the workload at half its size in every
    direction (the same fluid, shock and shock capturing); outside the timed region."""
    import numpy as np
    import inputs
    builder, kw, _, _ = WORKLOADS[workload]
    kw = dict(kw)
    kw["shape"] = tuple(n // 2 for n in kw["shape"])
    if "radius" in kw:
        kw["radius"] = kw["radius"] // 2
    case = getattr(inputs, builder)(**kw)
    sc = SC_WORKLOADS.get(workload)

    def density(prec, learned):
        s = P.Solver(case, precision=prec)
        if sc:
            P.lbm_set_shock_capturing(s.h, *sc)
        s.init()
        if learned:
            net.attach(s)
        s.step(CLOSURE_ACCURACY_STEPS)
        rho = np.asarray(s.fields()["rho"], dtype=np.float64)
        s.close()
        return rho

    ref = density("fp64", False)

    def rel(a):
        return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    return {"case": "x".join(str(n) for n in kw["shape"]) + (", radius %d" % kw["radius"] if "radius" in kw else ""),
            "steps": CLOSURE_ACCURACY_STEPS, "reference": "exact closure, FP64",
            "rho_rel_l2_learned_fp32": rel(density("fp32", True)),
            "rho_rel_l2_exact_fp32": rel(density("fp32", False)), "bar": 1e-3}


def train_closure(P, dev, workload, mma="tcgen05"):
    """Train the learned closure on solver states (GPU), outside the timed region; returns (net, info).
    The AdamW steps are timed with CUDA events on the network's stream (the current stream)."""
    import numpy as np
    import torch
    import inputs
    t0 = time.perf_counter()
    table, Ma_max, units, columns = MLP_WORKLOADS[workload]
    sc = inputs.scenario(units)
    net = P.Closure(sc["eos"]["a"], sc["eos"]["b"], sc["eos"]["R"], sc["cv"], seed=MLP_TRAIN["net_seed"],
                    stream=torch.cuda.current_stream(dev).cuda_stream)
    net.mma = P.LBM_MLP_MMA_TCGEN05 if mma == "tcgen05" else P.LBM_MLP_MMA_WARP
    runs = inputs.closure_training_runs(table=table, Ma_max=Ma_max, columns=columns)
    rho, e = net.collect_runs(runs, MLP_TRAIN["snapshots"],
                              MLP_TRAIN["every"], precision="fp32", shock_capturing=SC_WORKLOADS.get(workload))
    net.fit_scaling(rho, e)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    losses = net.train(rho, e, batch=MLP_TRAIN["batch"], steps=MLP_TRAIN["steps"], lr0=MLP_TRAIN["lr0"],
                       lr1=MLP_TRAIN["lr1"], seed=MLP_TRAIN["seed"])
    e1.record()
    torch.cuda.synchronize(dev)
    train_ms = e0.elapsed_time(e1)
    info = {"kind": "mlp 2-64-64-3, bf16 weights, fp32 accumulate, range-gated exact fallback",
            "train_samples": int(rho.numel()), "train_steps": MLP_TRAIN["steps"], "batch": MLP_TRAIN["batch"],
            "final_loss": float(np.mean(losses[-100:])), "train_and_collect_s": time.perf_counter() - t0,
            "train_contraction": mma, "train_s": train_ms / 1e3,
            "train_us_per_step": 1e3 * train_ms / max(1, MLP_TRAIN["steps"])}
    del rho, e
    return net, info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32", "fp16dev"])
    ap.add_argument("--step-kernel", default="fused", choices=["fused", "multipass"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--t64", action="store_true",
                    help="FP64 temperature inversion in the FP32 / FP16-deviation kernels "
                         "(lbm_set_temperature_fp64; default: the whole step in FP32)")
    ap.add_argument("--graphs", action="store_true",
                    help="replay captured CUDA graphs (lbm_set_graphs); each chunk is timed as a whole")
    ap.add_argument("--train-steps", type=int, default=None,
                    help="AdamW steps of the learned closure (learned-closure workloads)")
    ap.add_argument("--train-mma", default="tcgen05", choices=["tcgen05", "warp"],
                    help="contraction path of the closure training (lbm_mlp_set_mma)")
    args = ap.parse_args()
    if args.train_steps is not None:
        MLP_TRAIN["steps"] = args.train_steps
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload][0] in ("batch", "batch_columns"):
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
