#!/usr/bin/env python3
"""Benchmark of the GB300 LDDMM library: GN Hessian-vector products per second.

One step = one whole inexact Gauss-Newton-Krylov solve of the hot path from
v0 = 0: 10 GN iterations, each a gradient (forward shoot, transport, adjoint
Jacobi sweep), 20 PCG iterations (one GN Hessian-vector product each) and an
Armijo line search.  Default workload: the 160x192x160 brain phantom, band
32^3, Nt = 10, FP32 with FP64 reductions and tcgen05 3xTF32 transforms (the
largest single-GPU configuration); ``--workload 3d_64_ellipsoids`` runs the
64^3 ellipsoid phantom, band 16^3.  ``value`` = Hessian-vector products per
second over the timed steps, summed over ranks (each rank registers its own
pair: weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores: one
Hessian-vector product per step at a fixed linearisation point, the steps
spread over worker processes on all host cores.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GN Hessian-vector products/sec and GN solve time at 1e-5 rel. error vs FP64 oracle"
UNIT = "hessvec/s"
ALPHA, S, SIGMA = 0.0025, 2, 0.03
N_PCG = 20
N_GN_CONFIG = 10
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="3d_160x192x160_brain")
    ap.add_argument("--probe", default="auto", help="kernel class timed for the roofline (auto: dominant)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--state", default="image", choices=["image", "deformation"],
                    help="constraint: image state equation (Section 3.2) or band-limited deformation "
                         "state equation (Section 3.3)")
    ap.add_argument("--tensor-cores", default="auto", choices=["auto", "on", "off"],
                    help="image-grid band-to-grid transforms on tcgen05 (3xTF32): auto = grids >= 2^20 voxels")
    ap.add_argument("--persistent", default="auto", choices=["auto", "on", "off"],
                    help="band-limited sweeps as one persistent kernel: auto = padded grids up to 32^3")
    ap.add_argument("--precision", default=None, choices=["fp32", "3xtf32", "bf16x3", "fp64"],
                    help="fp32: tensor cores per --tensor-cores (3xTF32); 3xtf32 / bf16x3: every contraction "
                         "with a tensor-core kernel for its sizes on tcgen05 with that operand split; fp64; "
                         "default: the workload's (fp64 for 2d_64_blobs, else fp32)")
    ap.add_argument("--grid", default=None,
                    help="override the workload's image grid, e.g. 64,64,64 (a smaller case of the same "
                         "phantom and band, for kernel captures)")
    ap.add_argument("--band", default=None, help="override the workload's band, e.g. 32,32,32")
    return ap.parse_args()


SIZE_OVERRIDE = {}
# GN iterations x PCG iterations of a workload's solve, and its default precision
SOLVE_SHAPE = {"2d_64_blobs": (5, 10)}
DEFAULT_PRECISION = {"2d_64_blobs": "fp64"}


def solve_shape(name):
    return SOLVE_SHAPE.get(name, (N_GN_CONFIG, N_PCG))


def workload(name):
    from paper_1807_11560_gb300 import inputs
    kind, Ns, Ks, Nt, seed = inputs.WORKLOADS[name]
    Ns = SIZE_OVERRIDE.get("grid", Ns)
    Ks = SIZE_OVERRIDE.get("band", Ks)
    return kind, Ns, Ks, Nt, seed


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
        flat = {}

        def walk(d):
            for k, v in d.items():
                if isinstance(v, dict):
                    walk(v)
                elif isinstance(v, (int, float)):
                    flat.setdefault(k, float(v))
        walk(data)
        if "hbm_gbs" in flat:
            return flat, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# --------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, device_uuid=None):
        self.path = tempfile.mktemp(suffix=".csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd[1:1] = ["-i", device_uuid]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
                if len(parts) > 9:
                    try:
                        util.append(float(parts[9]))
                    except ValueError:
                        pass
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                # share of each sample period with a kernel running (host round trips show here)
                "gpu_util_pct_median": statistics.median(util) if util else None}


# --------------------------------------------------------------------------- oracle
# The FP64 oracle as it stands (single-threaded numpy/pocketfft), timed on the
# host cores.  "All cores" runs independent copies of the same bounded sample in
# worker processes (spawned: no CUDA state is inherited), one per core, and
# counts the products all of them finish per second of wall time.
ORACLE_MAX_WORKERS = 16


def _oracle_problem(spec, state, quant):
    """The oracle problem of a workload (kind, grid, band, Nt, seed), with the
    seeded v0 and direction p; quant: the inputs rounded to FP32 first, as the
    FP32 library receives them."""
    import numpy as np
    from oracle import deformation, objective
    from paper_1807_11560_gb300 import inputs
    kind, Ns, Ks, Nt, seed = spec
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    v0 = inputs.random_bl(Ks, len(Ns), seed + 1, 2.0, Ns)
    p = inputs.random_bl(Ks, len(Ns), seed + 2, 1.0, Ns)
    if quant:
        I0, I1 = (np.asarray(x, np.float32).astype(np.float64) for x in (I0, I1))
        v0, p = (np.asarray(x, np.complex64).astype(np.complex128) for x in (v0, p))
    cls = deformation.DeformationProblem if state == "deformation" else objective.Problem
    P = cls(I0, I1, Ks, ALPHA, S, SIGMA, Nt)
    return P, v0, p


def _oracle_worker(spec, state, quant, keep, jobs, barrier, results):
    """Linearise once (untimed, the worker's warm-up), wait for every worker,
    then take Hessian-vector products from the shared job counter; with keep,
    also return (E, g, H p) of the last product."""
    P, v0, p = _oracle_problem(spec, state, quant)
    lin = P.gradient(v0)
    barrier.wait()
    times = []
    Hp = None
    while True:
        with jobs.get_lock():
            if jobs.value <= 0:
                break
            jobs.value -= 1
        t0 = time.perf_counter()
        Hp = P.hessvec(lin, p)
        times.append(time.perf_counter() - t0)
    results.put((times, (lin.E, lin.g, Hp) if keep and Hp is not None else None))


def oracle_hessvec_rate(name, n_hv, state="image", workers=1, keep=False, quant=False):
    """FP64 oracle Hessian-vector products at a fixed linearisation point:
    n_hv products shared by `workers` processes.  Returns (products per second
    of wall time, per-product times, wall seconds, (E, g, H p) of one product
    when keep, else None)."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "MKL_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ[var] = "1"
    spec = workload(name)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    jobs = ctx.Value("i", n_hv)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(spec, state, quant, keep, jobs, barrier, results))
             for _ in range(workers)]
    for q in procs:
        q.start()
    barrier.wait()
    t0 = time.perf_counter()
    times, ref = [], None
    for _ in procs:
        t, r = results.get()
        times += t
        ref = ref if ref is not None else r
    wall = time.perf_counter() - t0
    for q in procs:
        q.join()
    return len(times) / wall, times, wall, ref


def oracle_parity(ctx, ref, Ns, Ks, seed, CT):
    """Energy, gradient and GN Hessian-vector product of the library at the
    oracle's seeded point (v0, p) against the oracle's (E, g, H p) from the CPU
    leg: relative errors, each the larger of the l2 and the element-wise
    (max |a - b| / max |b|) measure."""
    import numpy as np
    import torch

    from paper_1807_11560_gb300 import inputs
    if ref is None:
        return None
    E_ref, g_ref, H_ref = ref
    d = len(Ns)
    v0 = torch.as_tensor(inputs.random_bl(Ks, d, seed + 1, 2.0, Ns), dtype=CT, device="cuda")
    pv = torch.as_tensor(inputs.random_bl(Ks, d, seed + 2, 1.0, Ns), dtype=CT, device="cuda")
    g = torch.empty_like(v0)
    E = ctx.gradient(v0, g)
    Hp = torch.empty_like(v0)
    ctx.hessvec(pv, Hp)

    def rel(a, b):
        a = a.detach().cpu().numpy().astype(np.complex128)
        return float(max(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()),
                         np.abs(a - b).max() / np.abs(b).max()))
    return {"energy_rel_err": abs(E - E_ref) / abs(E_ref), "gradient_rel_err": rel(g, g_ref),
            "hessvec_rel_err": rel(Hp, H_ref), "target": 1e-5,
            "point": "the oracle CPU leg's seeded v0 and direction p (inputs rounded to the "
                     "library's precision), one gradient and one GN product"}


def oracle_workers(n):
    return max(1, min(n, os.cpu_count() or 1, ORACLE_MAX_WORKERS))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    kind, Ns, Ks, Nt, seed = workload(name)
    workers = oracle_workers(args.steps)
    value, times, wall, _ = oracle_hessvec_rate(name, args.steps, state=args.state, workers=workers)
    sample = (f"{len(times)} GN Hessian-vector products of the FP64 NumPy oracle at a fixed "
              f"linearisation point ({name}), one per step, spread over {workers} worker processes "
              "(one host core each; each worker's untimed linearisation is its warm-up)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name if not SIZE_OVERRIDE else f"{name} resized", "grid": list(Ns),
                   "band": list(Ks), "Nt": Nt, "gn_iters": solve_shape(name)[0],
                   "pcg_per_gn": solve_shape(name)[1], "state": args.state, "l2": "oracle on host cores",
                   "step": "one bounded sample: one GN Hessian-vector product at a fixed linearisation point"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count(),
                         "seconds_per_product_median": statistics.median(times)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- ranks
def rank_seed(seed, rank):
    """Each rank registers its own pair (replicas, no data-path collective)."""
    return seed + 1000 * rank


def combine_ranks(t_sec, n_hv, world, device):
    """Whole-job figures: the slowest rank's time and the products of all ranks."""
    if world == 1:
        return float(t_sec), float(n_hv)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_sec)], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_hv)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


# --------------------------------------------------------------------------- GPU arm
def kernel_sources_hash():
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1807_11560_gb300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload_name, cls):
    """DRAM bytes per launch of a kernel class from the committed ncu summary, or
    None when there is none or the CUDA sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    if data.get("kernel_sources_sha256_16") != kernel_sources_hash():
        return None
    entry = data.get(workload_name, {}).get(cls)
    return None if entry is None else float(entry["bytes"])


PROBE_CLASSES = ("sweep", "iota_ab", "cpw", "pi_ba", "inc_step", "transport", "iota_full", "pi_full", "deform")
HBM_CLASSES = ("inc_step", "transport")
FP32_LANES = 128
NOMINAL_FP64_TFLOPS = 1.25
# nominal dense tensor rates of the GB300 (PFLOP/s): TF32 takes the measured
# BF16 peak times their ratio, and the 3xTF32 split issues three TF32 MMAs per
# product, so its peak in algorithmic flops is a third of that
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
# kernel classes whose contractions run on tcgen05 (3xTF32) in the per-evaluation
# launches of padded grids above 32^3 points (the default tensor-core setting):
# iota A+B, C / bracket products / C', pi B'+A'
TENSOR_CLASSES = ("iota_ab", "cpw", "pi_ba")


def tensor_chain(args, Ks):
    """True when the bracket evaluations run as per-evaluation tcgen05 kernels."""
    import numpy as np
    mvol = int(np.prod([(3 * k + 1) // 2 for k in Ks]))
    persistent = args.persistent == "on" or (args.persistent == "auto" and mvol <= 32768)
    if persistent or args.tensor_cores == "off":
        return False
    if args.precision == "fp64":
        return False
    return args.tensor_cores == "on" or args.precision in ("3xtf32", "bf16x3") or mvol > 32768


def pick_dominant(ctx, v, n_pcg):
    """Probe every kernel class over one GN iteration (untimed); return the class
    with the largest total device time and the per-class totals (ms)."""
    totals = {}
    for cls in PROBE_CLASSES:
        ctx.probe(cls)
        w = v.clone()
        ctx.gn_solve(w, 1, n_pcg)
        totals[cls] = ctx.probe_read()[0]
    ctx.probe(None)
    return max(totals, key=totals.get), totals


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1807_11560_gb300 import Context, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    name = args.workload
    kind, Ns, Ks, Nt, seed = workload(name)
    d = len(Ns)
    n_gn, n_pcg = solve_shape(name)
    fp64 = args.precision == "fp64"
    RT = torch.float64 if fp64 else torch.float32
    CT = torch.complex128 if fp64 else torch.complex64
    I0, I1 = inputs.make_pair(kind, Ns, rank_seed(seed, rank))
    I0d = torch.as_tensor(I0, dtype=RT, device=dev)
    I1d = torch.as_tensor(I1, dtype=RT, device=dev)
    ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision=args.precision,
                  tensor_cores={"auto": "auto", "on": True, "off": False}[args.tensor_cores], state=args.state,
                  persistent={"auto": "auto", "on": True, "off": False}[args.persistent])
    ctx.set_images(I0d, I1d)
    v = torch.zeros((d,) + tuple(Ks), dtype=CT, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    class_ms = None
    probe_cls = args.probe
    if probe_cls == "auto":
        probe_cls, class_ms = pick_dominant(ctx, v, n_pcg)

    # a step is one whole GN-Krylov solve from v0 = 0 (n_gn GN iterations
    # x n_pcg PCG products, the workload's configuration), as a user runs it:
    # its time is the GN solve time
    for _ in range(args.warmup):
        ctx.gn_solve(v.clone(), n_gn, n_pcg)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    hv = 0
    k0 = ctx.kernel_count
    barrier()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                             # L2 flush between steps (untimed)
        w = v.clone()
        starts[k].record()
        rep_t = ctx.gn_solve(w, n_gn, n_pcg)
        ends[k].record()
        hv += rep_t["pcg_iters"]
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = ctx.kernel_count - k0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_dev = sum(step_ms) / 1e3
    # roofline pass: the same K steps again with CUDA events around every
    # launch of the dominant kernel class (events perturb the step time, so
    # the headline value above is taken without them)
    ctx.probe(probe_cls)
    ctx.gn_solve(v.clone(), 1, n_pcg)                     # builds the probed graph
    ctx.probe_read()
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ctx.gn_solve(v.clone(), n_gn, n_pcg)
    barrier()
    probe_ms, probe_n, probe_work = ctx.probe_read()
    ctx.probe(None)

    t_dev, hv_all = combine_ranks(t_dev, hv, world, dev)
    value = hv_all / t_dev

    # pure Hessian-vector rate at a fixed linearisation point (context figure)
    g = torch.empty_like(v)
    ctx.gradient(v, g)
    p = torch.as_tensor(inputs.random_bl(Ks, d, seed + 2, 1.0, Ns), dtype=CT, device=dev)
    out = torch.empty_like(p)
    for _ in range(3):
        ctx.hessvec(p, out)
    n_fix = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(n_fix):
        ctx.hessvec(p, out)
    e1.record()
    torch.cuda.synchronize()
    hv_fixed = n_fix / (e0.elapsed_time(e1) / 1e3)


    # end to end through the C interface with host buffers
    I0h = torch.as_tensor(I0, dtype=RT).pin_memory()
    I1h = torch.as_tensor(I1, dtype=RT).pin_memory()
    vh = torch.zeros((d,) + tuple(Ks), dtype=CT).pin_memory()
    hv_e2e = 0
    barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        vh.zero_()
        ctx.set_images(I0h, I1h)
        rep = ctx.gn_solve(vh, n_gn, n_pcg)
        hv_e2e += rep["pcg_iters"]
    barrier()
    te = time.perf_counter() - te0
    te, hv_e2e = combine_ranks(te, hv_e2e, world, dev)
    e2e_value = hv_e2e / te

    if rank == 0:
        peaks, src = load_peaks()
        avg_s = (probe_ms / 1e3) / max(probe_n, 1)
        work = probe_work / max(probe_n, 1)
        if probe_cls in HBM_CLASSES:
            achieved = work / avg_s / 1e9
            peak = peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
            roof = {"bound": "hbm", "unit": "GB/s", "peak_source": f"{src} HBM copy bandwidth (of {src})"}
            wunit = "B"
        else:
            mhz = clk.get("sm_mhz") or 2070.0
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            achieved = work / avg_s / 1e12
            tf32 = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]) * NOMINAL_TF32_OVER_BF16
            tensor = {"peak": tf32 / 3.0, "frac": achieved / (tf32 / 3.0),
                      "peak_source": f"{src} BF16 dense peak x 1.1/2.25 (nominal TF32/BF16) / 3 "
                                     f"(3xTF32: three TF32 MMAs per product; of {src})"}
            if probe_cls in TENSOR_CLASSES and tensor_chain(args, Ks):
                peak = tensor["peak"]
                roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": tensor["peak_source"]}
            else:
                if fp64:
                    peak = NOMINAL_FP64_TFLOPS
                    roof = {"bound": "alu", "unit": "TFLOP/s",
                            "peak_source": f"nominal GB300 FP64 rate ({NOMINAL_FP64_TFLOPS} TFLOP/s); FP64 SIMT "
                                           "contraction"}
                else:
                    peak = sms * FP32_LANES * 2 * mhz * 1e6 / 1e12
                    roof = {"bound": "alu", "unit": "TFLOP/s",
                            "peak_source": f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz "
                                           "(median sampled SM clock); FP32 SIMT contraction",
                            "vs_tensor_3xtf32": tensor}
            wunit = "flop"
        roof.update({"kernel": probe_cls, "achieved": achieved, "peak": peak, "frac": achieved / peak,
                     "traffic": measured_traffic(name, probe_cls), "traffic_unit": "B per launch (ncu)",
                     "launches_timed": probe_n, "avg_launch_us": avg_s * 1e6,
                     "algorithmic_per_launch": work, "algorithmic_unit": wunit,
                     "measured": f"CUDA events around each launch over a second pass of the {args.steps} "
                                 "timed steps"})
        if class_ms:
            roof["class_ms_one_gn_iteration"] = class_ms
        cpu = None
        parity = None
        if not args.no_cpu_baseline:
            one, t1, _, ref = oracle_hessvec_rate(name, 1, state=args.state, workers=1, keep=True,
                                                  quant=not fp64)
            nw = oracle_workers(os.cpu_count() or 1)
            allc, tall, _, _ = oracle_hessvec_rate(name, nw, state=args.state, workers=nw)
            parity = oracle_parity(ctx, ref, Ns, Ks, seed, CT)
            cpu = {"value": allc, "unit": UNIT, "cores": nw, "kind": "oracle",
                   "sample": f"{nw} GN Hessian-vector products of the FP64 NumPy oracle on {name} at a "
                             f"fixed linearisation point, one per worker process on {nw} host cores "
                             "(single-threaded numpy/pocketfft each; linearisation untimed)",
                   "host_cores": os.cpu_count(),
                   "single_core": {"value": one, "cores": 1, "seconds_per_product": t1[0],
                                   "sample": "one product in one process"}}
        nvox, nband = int(np.prod(Ns)), d * int(np.prod(Ks))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": {"workload": name if not SIZE_OVERRIDE else f"{name} resized", "grid": list(Ns),
                       "band": list(Ks), "Nt": Nt,
                       "gn_iters": n_gn, "pcg_per_gn": n_pcg, "state": args.state,
                       "step": f"one GN-Krylov solve from v0 = 0: {n_gn} GN iterations (gradient, "
                               f"{n_pcg} PCG Hessvecs, Armijo)",
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"replicas x{world}",
                       "precision": args.precision,
                       "tensor_cores": f"{args.tensor_cores} (tcgen05 3xTF32: image-grid iota on grids of at "
                                       "least 2^20 voxels, bracket evaluations launched per evaluation)",
                       "tiles": dict(zip(("iota_ab_twiddles", "cpw_pencils", "pi_rows"), ctx.tiles))},
            "gn_solve_s": 1e-3 * statistics.mean(step_ms),
            "gn_solve_note": f"mean timed step: one lddmm_gn_solve call ({rep_t['gn_iters']} GN iterations and "
                             f"{rep_t['pcg_iters']} products ran, E {rep_t['E_initial']:.6g} -> "
                             f"{rep_t['E_final']:.6g}, line-search steps {rep_t['eps']})",
            "hessvec_per_s_fixed_point": hv_fixed,
            "wall_s": t_wall,
            "roofline": roof,
            "cpu_baseline": cpu,
            "oracle_parity": parity,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 2 * nvox * 4 + nband * 8, "d2h_bytes_per_step": nband * 8},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_population(args):
    """The batched population workload (32 brain pairs of uneven grids and bands):
    one step = one GN iteration with 20 PCG Hessian-vector products on every pair,
    all pairs at once through lddmm_batch_gn_solve (one CUDA stream and one host
    thread per context).  The work spans 32 streams, so steps are timed by the host
    clock between device synchronisations.  Also reported: the same contexts solved
    one after another, and the population with plain FP32 SIMT transforms instead of
    the tcgen05 3xTF32 split."""
    import collections

    import numpy as np
    import torch

    from paper_1807_11560_gb300 import Context, batch_gn_solve, inputs

    if int(os.environ.get("RANK", "0")) != 0:
        return
    pop = inputs.population()

    def make(tc):
        made = []
        for kind, Ns, Ks, Nt, seed in pop:
            I0, I1 = inputs.make_pair(kind, Ns, seed)
            st = torch.cuda.Stream()
            ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32", stream=st.cuda_stream,
                          tensor_cores=tc, persistent=False)
            I0d = torch.as_tensor(I0, dtype=torch.float32, device="cuda")
            I1d = torch.as_tensor(I1, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            ctx.set_images(I0d, I1d)
            made.append((ctx, st, np.zeros((3,) + tuple(Ks), np.complex64)))
        return made

    def timed(made, steps, threads):
        ctxs = [m[0] for m in made]
        hv, t = 0, 0.0
        for _ in range(steps):
            v0s = [np.zeros_like(m[2]) for m in made]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = batch_gn_solve(ctxs, v0s, 1, N_PCG, threads=threads)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            hv += sum(r["pcg_iters"] for r in reps)
        return hv / t, t / steps, v0s

    # one pair of each grid and band: gradient and GN product at the pair's seeded
    # point, for the split-precision against the plain FP32 comparison
    picked, seen = [], set()
    for i, (_, Ns, Ks, _, _) in enumerate(pop):
        if (tuple(Ns), tuple(Ks)) not in seen:
            seen.add((tuple(Ns), tuple(Ks)))
            picked.append(i)

    def products(made):
        out = {}
        for i in picked:
            _, Ns, Ks, _, seed = pop[i]
            v0 = inputs.random_bl(Ks, 3, seed + 1, 2.0, Ns).astype(np.complex64)
            pv = inputs.random_bl(Ks, 3, seed + 2, 1.0, Ns).astype(np.complex64)
            g, Hp = np.empty_like(v0), np.empty_like(v0)
            made[i][0].gradient(v0, g)
            made[i][0].hessvec(pv, Hp)
            out[i] = (g.astype(np.complex128), Hp.astype(np.complex128))
        return out

    def rel(a, b):
        return float(max(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()),
                         np.abs(a - b).max() / np.abs(b).max()))

    made = make("auto")
    timed(made, args.warmup, 0)
    clocks = Clocks()
    value, step_s, v_tc = timed(made, args.steps, 0)
    clk = clocks.stop()
    seq_value, _, _ = timed(made, 1, 1)
    prod_tc = products(made)
    held = sum(m[0].device_bytes for m in made)
    for m in made:
        m[0].close()
    del made
    made = make(False)
    timed(made, 1, 0)
    plain_value, _, v_plain = timed(made, args.steps, 0)
    prod_plain = products(made)
    for m in made:
        m[0].close()
    # one GN step from v0 = 0 on the same images: the two precisions' updates
    diffs = [float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)) for a, b in zip(v_tc, v_plain)]
    hist = collections.Counter(f"{'x'.join(map(str, g))}/K{k[0]}" for _, g, k, _, _ in pop)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "population_32", "pairs": len(pop), "grids_bands": dict(hist), "Nt": 10,
                   "pcg_per_gn": N_PCG, "step": "one GN iteration on every pair",
                   "timer": "host clock between device synchronisations (32 streams)",
                   "tensor_cores": "auto (grids of at least 2^20 voxels)"},
        "sequential_value": seq_value,
        "plain_fp32_value": plain_value,
        "split_vs_plain_rel_update_diff_max": max(diffs),
        "split_vs_plain_product_rel_diff_max": {
            "gradient": max(rel(prod_tc[i][0], prod_plain[i][0]) for i in picked),
            "hessvec": max(rel(prod_tc[i][1], prod_plain[i][1]) for i in picked),
            "pairs": len(picked), "measure": "larger of l2 and element-wise, one pair per grid and band"},
        "device_bytes_held": held,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


BAND_SWEEP = (16, 32, 40, 48, 56, 64)


def run_band_sweep(args):
    """Band-size sweep on the 160x192x160 brain phantom (a synthetic analogue of the
    paper's band-size tables): for each K^3 band, a GN-Krylov solve from v0 = 0
    (``--steps`` GN iterations x 10 PCG), reporting MSE_rel = 100 ||m(1) - I1||^2 /
    ||I0 - I1||^2, the relative infinity norm of the gradient, the device memory the
    context holds and the solve time (host clock between device synchronisations)."""
    import numpy as np
    import torch

    from paper_1807_11560_gb300 import Context, inputs

    if int(os.environ.get("RANK", "0")) != 0:
        return
    kind, Ns, _, Nt, seed = workload("3d_160x192x160_brain")
    I0, I1 = inputs.make_pair(kind, Ns, seed)
    I0d = torch.as_tensor(I0, dtype=torch.float32, device="cuda")
    I1d = torch.as_tensor(I1, dtype=torch.float32, device="cuda")
    d01 = float(torch.sum((I0d - I1d) ** 2))
    rows = []
    for k in BAND_SWEEP:
        Ks = (k, k, k)
        ctx = Context(Ns, Ks, ALPHA, S, SIGMA, Nt, precision="fp32")
        ctx.set_images(I0d, I1d)
        v = torch.zeros((3,) + Ks, dtype=torch.complex64, device="cuda")
        g = torch.empty_like(v)
        ctx.gradient(v, g)
        g0 = float(g.abs().max())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.gn_solve(v, args.steps, 10)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        m1 = torch.empty_like(I0d)
        ctx.transport(v, m1)
        ctx.gradient(v, g)
        rows.append({"K": k, "mse_rel_pct": 100.0 * float(torch.sum((m1 - I1d) ** 2)) / d01,
                     "grad_inf_rel": float(g.abs().max()) / g0, "device_gib": ctx.device_bytes / 2**30,
                     "solve_s": t, "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters"],
                     "hessvec_per_s": rep["pcg_iters"] / t, "tiles": ctx.tiles})
        ctx.close()
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"workload": "band_sweep_160x192x160", "Nt": Nt, "gn": args.steps, "pcg_per_gn": 10,
                      "rows": rows}), flush=True)


def main():
    args = parse()
    if args.precision is None:
        args.precision = DEFAULT_PRECISION.get(args.workload, "fp32")
    if args.grid:
        SIZE_OVERRIDE["grid"] = tuple(int(x) for x in args.grid.split(","))
    if args.band:
        SIZE_OVERRIDE["band"] = tuple(int(x) for x in args.band.split(","))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "population_32":
        run_population(args)
    elif args.workload == "band_sweep":
        run_band_sweep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
