"""Throughput benchmark of the DG-LES hot path on B300.

Metric: DG node-stage updates per second (one node advanced through one
LSRK(5,4) stage: a full right-hand-side evaluation plus the stage update) on
the throughput box (160 x 160 x 80 elements, N = 4, 256M nodes), and the HBM
roofline fraction of the dominant kernel.  A step is one LSRK(5,4) step
(5 stages) over the whole box; inputs are resident in HBM and much larger than
L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cmles|reference]

--impl reference times the FP64 CPU oracle (the method's plain reference
implementation) on a bounded sub-box of the same workload on the host cores.
With N > 1 (torchrun) each rank runs an independent replica of the box on its
own GPU (weak scaling, no data-path collective); rank 0 prints the line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_00853_b300 import inputs as I  # noqa: E402

WORKLOAD = "c5"
STAGES = {"lsrk54": 5, "lsrk144": 14, "ark2_hevi": 3}
METRIC = "DG node-stage updates/s at 1 B300 and HBM roofline %, FP32+learned vs FP64 plain"
# algorithmic bytes per node for each kernel launch (compulsory traffic),
# averaged over the S stages of a step (S = 5 for LSRK(5,4)):
#   gradient pass: read the state (Q or the FP32 shadow S) and its h_tot,
#     theta_v (2 words), write F2 (15 words)
#   flux/update pass, FP64 path: read Q, F2, p - p_r and c; write dQ, Q_out
#     and Q_out's four thermodynamic fields; read dQ except in the first stage
#     (A_1 = 0): ((S - 1) * 45 + 39) words / S
#   flux/update pass, FP32 path (FP32 shadow S, FP32 register dQ and step
#     increment D, FP64 state Q64): read S, F2, p' and c (23 words) in every
#     stage; every stage writes the new state's thermodynamic fields (+4);
#     stage 1 writes dQ, D, S (+18); the middle stages read dQ, D and write dQ,
#     D, S (+30); the last stage reads dQ, D, reads and writes Q64 and writes S
#     (+12 + 24 FP32 words for Q64): (45 + (S - 2) * 57 + 69) words / S, 57
#     words for S = 5
#   flux pass of the HEVI stages: the tendency alone, read Q (S), F2, aux (p',
#     c) and write R (FP64)
def alg_bytes(prec, kind, stages=5, integrator="lsrk54"):
    if kind == "grad":
        return (6 + 15 + 2) * (8 if prec == "fp64" else 4)
    if integrator == "ark2_hevi":
        return 29 * 8 if prec == "fp64" else 23 * 4 + 6 * 8
    if prec == "fp64":
        return ((stages - 1) * 45 + 39) * 8 / stages
    return (45 + (stages - 2) * 57 + 69) * 4 / stages


# name: (precision, closure, numerical flux of F1, integrator); the first
# three are the default run, the others are reported when asked for with
# --variants
VARIANTS = {"fp32acc64_mlp": ("fp32", "mlp", "rusanov", "lsrk54"), "fp32acc64_sl": ("fp32", "sl", "rusanov", "lsrk54"),
            "fp64_sl": ("fp64", "sl", "rusanov", "lsrk54"),
            "fp32acc64_vreman": ("fp32", "vreman", "rusanov", "lsrk54"),
            "fp32acc64_mlp_hllc": ("fp32", "mlp", "hllc", "lsrk54"),
            "fp32acc64_mlp_roe": ("fp32", "mlp", "roe", "lsrk54"),
            "fp32acc64_mlp_lsrk144": ("fp32", "mlp", "rusanov", "lsrk144"),
            "fp64_sl_lsrk144": ("fp64", "sl", "rusanov", "lsrk144"),
            "fp64_sl_hevi": ("fp64", "sl", "rusanov", "ark2_hevi"),
            "fp32acc64_mlp_hevi": ("fp32", "mlp", "rusanov", "ark2_hevi"),
            # the flow over the Gaussian ridge at its configured size: 128 x 16 x 64
            # warped elements (16.4M nodes), curvilinear FP32 kernels
            "c3_fp32acc64_sl": ("fp32", "sl", "rusanov", "lsrk54"),
            "c3_fp32acc64_mlp": ("fp32", "mlp", "rusanov", "lsrk54")}
# the workload of a variant: the throughput box unless its name says otherwise
def variant_workload(name):
    return "c3" if name.startswith("c3_") else WORKLOAD
DTYPE = {"fp32": "f32", "fp64": "f64"}
# What bounds each dominant kernel, from its ncu capture (profiles/): the
# roofline above is HBM's, the metric's; the gradient passes are limited by
# instruction issue and the FP64 passes by the FP64 pipe.
LIMITER = {("fp32acc64_mlp", "grad"): "issue (SiLU epilogue of the tensor-core network)",
           ("fp32acc64_sl", "grad"): "issue", ("fp32acc64_sl", "rhs"): "latency and LSU",
           ("fp32acc64_mlp", "rhs"): "latency and LSU", ("fp64_sl", "rhs"): "FP64 pipe",
           ("fp64_sl", "grad"): "FP64 pipe"}
# The tendency's parity bound against the FP64 oracle (tests/): the FP32 path's
# 1e-5 relative L2 holds with Smagorinsky-Lilly; with the learned closure the
# BF16 activations (defined by the oracle's BF16 network, rounded sums on the
# GPU) hold 1e-4.
PARITY = {"fp32acc64_mlp": "1e-4 rel L2 per variable vs the FP64 oracle with its BF16 network",
          "fp32acc64_sl": "1e-5 rel L2 per variable vs the FP64 oracle",
          "fp64_sl": "1e-12 rel L2 per variable vs the FP64 oracle"}
# ncu counters of the dominant kernels are not constants of this script: they
# come from profiles/ncu_counters_c5.txt, written from one ncu capture (its
# command is in that file), one line per kernel:
#   <variant> <kernel> dram_B_per_node=<x> warp_inst_per_element=<y> sources=<sha>
# where sha is the SHA-256 (first 16 hex digits) of the kernel's source files
# at capture time.  A line whose kernel sources have changed since is stale and
# is not used (traffic and issue then read null).
COUNTERS = os.path.join(ROOT, "profiles", "ncu_counters_c5.txt")
KERNEL_SOURCES = {
    "grad": ["dg_fp32.cu", "dg32_parts.cuh", "mlp.cuh", "tc.cuh", "common.cuh", "thermo32.cuh"],
    "rhs": ["dg_fp32.cu", "dg32_parts.cuh", "common.cuh", "thermo32.cuh"],
    "grad64": ["dg_fp64.cu", "common.cuh", "thermo.cuh"],
    "rhs64": ["dg_fp64.cu", "common.cuh", "thermo.cuh"],
}


def kernel_sources_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2110_00853_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_counters(variant, kind, prec):
    """(DRAM bytes per node, warp instructions per element) of one launch from
    the committed ncu capture, or (None, None) when absent or stale."""
    key = kind if prec == "fp32" else kind + "64"
    try:
        lines = open(COUNTERS).read().splitlines()
    except OSError:
        return None, None
    for ln in lines:
        parts = ln.split()
        if len(parts) < 3 or parts[0] != variant or parts[1] != kind:
            continue
        kv = dict(p.split("=", 1) for p in parts[2:] if "=" in p)
        if kv.get("sources") != kernel_sources_sha(key):
            return None, None
        return float(kv["dram_B_per_node"]), float(kv.get("warp_inst_per_element", "nan"))
    return None, None


def issue_peak():
    """warp instructions per second the SMs can issue at the maximum SM clock
    (MEASURED_PEAKS.json's sm_max_mhz, else B300's 2032 MHz)"""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = json.load(f).get("sm_max_mhz", 2032.0)
    except Exception:
        mhz = 2032.0
    return 148 * 4 * mhz * 1e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, world, torch, device):
    """the slowest rank's time (every rank gets it); a no-op for one rank"""
    if world <= 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank, world, steps, ms, stages=5):
    """node-stage updates per second of all ranks together over the slowest
    rank's time (replicas: every rank advances its own box)"""
    return nodes_per_rank * world * stages * steps / (ms / 1e3)


def fp64_peak(torch, n=8192, reps=5):
    """FP64 GEMM rate of the GPU (cuBLAS DGEMM, 2 n^3 flops, best of reps
    after a warm-up): the measured ceiling of FP64 arithmetic the FP64 path
    is compared with."""
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    torch.matmul(a, b)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return {"fp64_gemm_tflops": 2.0 * n ** 3 / (best / 1e3) / 1e12, "n": n, "ms": best}


def closure_weights():
    """Seeded network of the closure's architecture (13 -> 64 -> 64 -> 2); the
    throughput does not depend on the weight values.  Input scales match the
    magnitudes of the box's gradients, output scales give nu_t, D_t of a few
    m^2/s."""
    from paper_2110_00853_b300 import closure
    return closure.init_params(seed=0, in_scale=[100.0] * 9 + [300.0] * 3 + [0.02], out_scale=(5.0, 10.0),
                               b3=(0.5, 0.5))


def workload_mesh(sub, workload=WORKLOAD):
    """the workload's mesh, or a sub-box of it with the same element size
    (used for small profiling cases)"""
    return I.mesh(workload) if sub is None else I.sub_mesh(workload, *sub)


def run_variant(name, precision, closure, flux, integrator, steps, warmup, world, rank, torch, sub=None):
    from paper_2110_00853_b300 import cmles
    wl = variant_workload(name)
    mesh, phys, case = workload_mesh(sub, wl), I.physics(wl, closure=closure), I.case(wl)
    phys["flux"] = flux
    phys["integrator"] = integrator
    G = cmles.Solver(mesh, phys, precision=precision)
    G.init_case(case)
    if closure == "mlp":
        G.set_closure_weights(closure_weights())
    G.step(warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = G.launch_count()
    G.enable_timing(True)
    G.kernel_times()  # reset counters
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    torch.cuda.synchronize()
    e0.record(s)
    G.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    kt = G.kernel_times()
    launches = G.launch_count() - launches0
    G.enable_timing(False)
    diag = G.diagnostics(raise_on_error=False)
    nodes = G.E * G.Np
    G.close()
    del G
    torch.cuda.empty_cache()
    ms = max_over_ranks(ms, world, torch, "cuda")
    return dict(name=name, ms=ms, kt=kt, launches=launches, nodes=nodes, clocks=clocks,
                finite=not diag["nonfinite"], satadj_failures=diag["satadj_failures"])


def run_e2e(precision, closure, flux, integrator, steps, torch):
    """Same metric through the C ABI with host buffers, as a host-resident
    application would use it: every step starts from the state in pinned host
    memory, advances it (cmles_step) and brings the advanced state back to
    pinned host memory, which becomes the next step's input; each step's
    budget diagnostics are read too.  Two host buffers alternate as input and
    output.  The copies cannot overlap the step (each step's input is the
    previous step's output), but the two directions overlap each other: the
    download runs in chunks (cmles_fetch_state_host) and the upload of the
    same buffer (cmles_stage_state_host, then cmles_commit_staged_state)
    sends each chunk as soon as it has arrived."""
    from paper_2110_00853_b300 import cmles
    mesh, phys, case = I.mesh(WORKLOAD), I.physics(WORKLOAD, closure=closure), I.case(WORKLOAD)
    phys["flux"] = flux
    phys["integrator"] = integrator
    G = cmles.Solver(mesh, phys, precision=precision)
    G.init_case(case)
    if closure == "mlp":
        G.set_closure_weights(closure_weights())
    bufs = [G.get_state_host(), G.get_state_host()]
    G.step(1)
    G.get_state_host(out=bufs[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        G.stage_state_host(bufs[k % 2])
        G.commit_staged_state()
        G.step(1)
        # the budgets' small read-back goes before the download, which would
        # otherwise hold it back on the device-to-host copy engine
        G.diagnostics(raise_on_error=False)
        G.fetch_state_host(bufs[(k + 1) % 2])
    G.wait_fetch()
    t1 = time.perf_counter()
    nodes = G.E * G.Np
    state_bytes = nodes * 6 * 8
    G.close()
    del bufs, G
    torch.cuda.empty_cache()
    sec = (t1 - t0) / steps
    return dict(value=nodes * STAGES[integrator] / sec, unit="node-stage/s", h2d_bytes_per_step=state_bytes,
                d2h_bytes_per_step=state_bytes + 7 * 8 + 16 * 4, ms_per_step=sec * 1e3,
                note="host state in, one step, host state out; the next step starts from that host state; "
                     "download and upload overlap chunk by chunk")


def _omp_threads(n):
    """Set the OpenMP thread count of the oracle (libgomp) at run time."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return True
    except OSError:
        return False


def _cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(max_seconds=20.0, threads=None):
    """The FP64 CPU oracle, as it stands, on a sub-box of the throughput
    workload (same element size and physics, fewer elements), with OpenMP
    over elements on `threads` host threads (default all)."""
    from oracle import oracle as O
    nproc = os.cpu_count() or 1
    threads = threads or int(os.environ.get("OMP_NUM_THREADS", nproc))
    n = (20, 20, 16) if threads > 1 else (8, 8, 8)
    m = I.sub_mesh(WORKLOAD, *n)
    c = I.case(WORKLOAD)
    c["modes"] = I.velocity_modes(m["Lx"], m["Ly"], m["Lz"], nmodes=200, seed=5)
    S, Q, rr, pr, _ = O.from_inputs(m, I.physics(WORKLOAD), c)
    _omp_threads(threads)
    try:
        S.lsrk54(Q, 1, 0.02)   # warm-up
        t0 = time.perf_counter()
        steps = 0
        while True:
            Q, _ = S.lsrk54(Q, 1, 0.02)
            steps += 1
            if time.perf_counter() - t0 > max_seconds / 2 or steps >= 4:
                break
        sec = time.perf_counter() - t0
    finally:
        _omp_threads(nproc)
    nodes = S.E * S.Np
    return dict(value=nodes * STAGES["lsrk54"] * steps / sec, unit="node-stage/s", cores=threads, kind="oracle",
                nproc=nproc, cpu=_cpu_model(),
                sample=f"{n[0]}x{n[1]}x{n[2]}-element sub-box of the {WORKLOAD} workload (same element size, "
                       f"moist SL physics, {nodes} nodes), {steps} LSRK(5,4) step(s) after 1 warm-up step, "
                       f"{threads} OpenMP thread(s)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cmles", choices=["cmles", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sub", default=None, help="nex,ney,nez: run a sub-box of the workload (profiling cases)")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="print the FP64 GEMM rate of this GPU (the FP64 path's roofline) and exit")
    ap.add_argument("--variants", default="fp32acc64_mlp,fp32acc64_sl,fp64_sl",
                    help="comma list; the first is the headline value")
    args = ap.parse_args()
    sub = tuple(int(x) for x in args.sub.split(",")) if args.sub else None
    world, rank, local = dist_setup()

    if args.fp64_peak:
        import torch
        print(json.dumps(fp64_peak(torch)))
        return 0

    if args.impl == "reference":
        if rank != 0:
            return 0
        cb = cpu_baseline()
        line = dict(impl="reference", metric=METRIC, value=cb["value"], unit=cb["unit"], n_gpus=args.gpus,
                    steps=args.steps, warmup=args.warmup, ms_per_step=None, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                    config={"workload": f"{WORKLOAD}: 160x160x80 elements, N=4, moist, SL closure (CPU oracle on a "
                                        "bounded sub-box)"},
                    cpu_baseline=cb, e2e={"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0})
        print(json.dumps(line))
        return 0

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    hbm, peak_kind = measured_peaks()
    variants = [(n,) + VARIANTS[n] for n in args.variants.split(",")]
    results = {}
    for name, prec, clo, flux, integ in variants:
        results[name] = run_variant(name, prec, clo, flux, integ, args.steps, args.warmup, world, rank, torch, sub)
    head = results[variants[0][0]]
    prec = variants[0][1]
    hstages = STAGES[variants[0][4]]
    value = whole_job_rate(head["nodes"], world, args.steps, head["ms"], hstages)
    kt = head["kt"]
    kinds = ["grad", "rhs"]
    dom = max(range(2), key=lambda k: kt["ms"][k])
    avg_ms = kt["ms"][dom] / max(kt["count"][dom], 1)
    achieved = head["nodes"] * alg_bytes(prec, kinds[dom], hstages, variants[0][4]) / (avg_ms / 1e3) / 1e9
    tb, wi = ncu_counters(variants[0][0], kinds[dom], prec)
    traffic = tb * head["nodes"] if tb is not None else None
    limiter = LIMITER.get((variants[0][0], kinds[dom]), "unmeasured")
    hbm_view = {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"{peak_kind} hbm_gbs"}
    if wi is not None and wi == wi and limiter.startswith("issue"):
        # an instruction-issue-bound kernel: its roofline is the SMs' issue
        # rate (148 SMs x 4 schedulers x one warp instruction per clock at the
        # maximum SM clock), its achieved rate the ncu instruction count per
        # element times the elements of one launch over the launch's CUDA-event
        # time; the HBM view stays beside it
        ipk = issue_peak()
        ach = wi * (head["nodes"] // 125) / (avg_ms / 1e3)
        roofline = {"bound": "alu", "kernel": kinds[dom], "achieved": ach, "peak": ipk, "unit": "warp-inst/s",
                    "frac": ach / ipk, "traffic": traffic, "warp_inst_per_element": wi,
                    "peak_source": "148 SMs x 4 schedulers x 1 warp instruction/clock x maximum SM clock",
                    "limiter": limiter, "hbm": hbm_view}
    else:
        roofline = dict({"bound": "hbm", "kernel": kinds[dom], "traffic": traffic, "limiter": limiter}, **hbm_view)
    out_variants = {}
    for (name, vprec, _, _, vint), r in zip(variants, results.values()):
        v = whole_job_rate(r["nodes"], world, args.steps, r["ms"], STAGES[vint])
        per = {}
        for k in range(2):
            a = r["kt"]["ms"][k] / max(r["kt"]["count"][k], 1)
            gbs = r["nodes"] * alg_bytes(vprec, kinds[k], STAGES[vint], vint) / (a / 1e3) / 1e9
            per[kinds[k]] = dict(avg_ms=a, launches=r["kt"]["count"][k], gbs=gbs, hbm_frac=gbs / hbm)
        out_variants[name] = dict(value=v, ms_per_step=r["ms"] / args.steps, kernels=per, finite=r["finite"],
                                  satadj_failures=r["satadj_failures"], workload=variant_workload(name),
                                  nodes=r["nodes"])
        if variant_workload(name) == "c3":
            out_variants[name]["bytes_note"] = ("GB/s from the flat-mesh byte counts; the curvilinear kernels "
                                                "also read per-node metric terms and reference tables")
    e2e = None
    if not args.no_e2e and rank == 0 and sub is None:
        e2e = run_e2e(variants[0][1], variants[0][2], variants[0][3], variants[0][4], max(2, min(args.steps, 4)),
                      torch)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and sub is None:
        cb = cpu_baseline()
        cb["single_thread"] = cpu_baseline(threads=1)
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="node-stage/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=head["ms"] / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype=DTYPE[prec], data="synthetic",
                    config={"workload": f"{WORKLOAD}: 160x160x80 hexahedral elements, N=4 (256M nodes), moist, "
                                        + {"lsrk54": "LSRK(5,4)", "lsrk144": "LSRK(14,4)",
                                           "ark2_hevi": "ARK2 HEVI"}[variants[0][4]],
                            "variant": variants[0][0],
                            "closure": {"mlp": "learned (BF16 tensor-core MLP 13-64-64-2, seeded weights)",
                                        "sl": "Smagorinsky-Lilly + Richardson",
                                        "vreman": "Vreman + Richardson"}[variants[0][2]],
                            "flux": variants[0][3], "integrator": variants[0][4],
                            "elements": head["nodes"] // 125, "nodes_per_gpu": head["nodes"],
                            "l2": "inputs larger than L2 (state alone 12 GB)", "parallelism": f"replicas{world}"},
                    roofline=roofline,
                    parity=PARITY[variants[0][0]] if variants[0][0] in PARITY else None,
                    cpu_baseline=cb, e2e=e2e, gpu_launches=head["launches"], clocks=head["clocks"],
                    variants=out_variants)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
