"""Benchmark: PCDM1 (tau-nice, LASSO) solved to a relative duality gap on one GB300 per rank.

One step = one complete solve of the scale workload from x = 0:
  reset (x = 0, g = -b), then Algorithm 1 iterations in chunks of one epoch
  (ceil(n / tau) iterations, one persistent kernel launch each), each chunk
  followed by an FP64 residual refresh and an FP64 duality-gap check, until
  gap / primal <= tol.
The default workload is the square scale instance: m = n = 4e6, every row with
exactly omega = 16 nonzeros at uniform columns (nnz = 6.4e7), N(0,1) values,
x* 1%-dense +-U[1,2], b = A x* + N(0, 1e-4), lambda = 0.05 ||A^T b||_inf,
tau = 65536, FP64 values and iterates, tolerance 1e-6.

value     coordinate updates per second over the timed steps (inputs resident in HBM)
e2e       the same metric through the public API from pinned host buffers: create
          (host-to-device copy of A and b, validation, L and omega), solve, read x back
roofline  the fused iteration kernel: algorithmic bytes per launch / CUDA-event time
cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of the same solve

--impl reference times the oracle itself (one bounded sample of iterations per step).
Under torchrun every rank solves its own replica (no collective on the data path).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coord updates/s & HBM GB/s vs peak; time to rel. duality gap 1e-6, plain vs batched"
UNIT = "coord updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["pcdm", "reference"], default="pcdm")
    p.add_argument("--n", type=int, default=4_000_000)
    p.add_argument("--omega", type=int, default=16)
    p.add_argument("--tau", type=int, default=65536)
    p.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64")
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--check-every", type=int, default=0)
    p.add_argument("--refresh-every", type=int, default=-1, help="-1: 0 for f64, 64 otherwise")
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--unfused", action="store_true")
    p.add_argument("--max-iters", type=int, default=200_000)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    p.add_argument("--quiet", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the batched regularisation-path measurement")
    p.add_argument("--path-len", type=int, default=32, help="lambdas on the batched regularisation path")
    p.add_argument("--no-grad", action="store_true", help="skip the differentiation measurement")
    p.add_argument("--no-svm", action="store_true", help="skip the SVM-dual measurement (Sec. 8.3 workload)")
    p.add_argument("--no-logistic", action="store_true", help="skip the logistic-regression measurement (Sec. 8.4)")
    p.add_argument("--no-tvr", action="store_true", help="skip the theory-versus-reality experiment")
    p.add_argument("--no-async", action="store_true", help="skip the asynchronous-mode measurement")
    p.add_argument("--no-multi", action="store_true", help="skip the many-small-problems measurement")
    p.add_argument("--no-tune", action="store_true", help="keep the built-in kernel choice (no pcdm_autotune)")
    p.add_argument("--no-l2-persist", action="store_true",
                   help="FP64: leave the context's L2 persisting-lines limit as it is (no opts.l2_persist)")
    p.add_argument("--tuning", default=None,
                   help="kernel,lanes_per_col,threads_per_block,heads[,zero_cert] set by hand (pcdm_set_tuning) instead of "
                        "pcdm_autotune, e.g. 0,1,448,1 for the pipelined kernel with 448-thread blocks")
    p.add_argument("--no-omega128", action="store_true", help="skip the omega = 128 FP64 solve (5.12e8 nonzeros)")
    p.add_argument("--no-precisions", action="store_true",
                   help="skip the other precision pairs and the errors against the oracle")
    p.add_argument("--no-gather-ceiling", action="store_true",
                   help="skip the random-gather ceiling measured beside the roofline")
    p.add_argument("--sweep", action="store_true", help="print the omega x tau x dtype table of the scale workload")
    p.add_argument("--sweep-omega", default="2,16,128", help="the omega values of --sweep (comma-separated)")
    p.add_argument("--huge", action="store_true", help="time the 4e9-nonzero configuration (about 140 GB of HBM)")
    p.add_argument("--huge-m", type=int, default=1_000_000_000, help="rows of the huge configuration (scaled runs)")
    p.add_argument("--huge-n", type=int, default=500_000_000, help="columns of the huge configuration")
    return p.parse_args()


# ----------------------------------------------------------------------------- distributed plumbing
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(local_units, local_seconds, world):
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    if world == 1:
        return local_units / local_seconds, local_seconds, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if (dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- helpers
def workload_name(a):
    return ("square scale LASSO: m=n=%d, omega=%d per row (nnz=%d), tau=%d, %s values, solve from x=0 "
            "to rel. duality gap %g" % (a.n, a.omega, a.n * a.omega, a.tau, a.dtype, a.tol))


def make_instance(a):
    from paper_1212_0873_gb300 import instances
    return instances.row_omega_instance(a.n, a.n, a.omega, density=0.01, noise=0.01, lam_frac=0.05,
                                        val_dtype=a.dtype, seed=1002)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1212_0873_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_per_update(a, tuning):
    """(DRAM bytes per coordinate update, the tuning they were taken at) of the
    iteration kernel from the committed ncu summary, when it was taken on the
    current kernel sources, this workload and this kernel (same kernel, lanes per
    column and column-head choice; the block size may differ), else (None, None)."""
    path = os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, None
    if d.get("src_hash") != kernel_source_hash():
        return None, None
    key = "%s/omega%d/tau%d" % (a.dtype, a.omega, a.tau)
    ent = d.get("workloads", {}).get(key)
    if ent is None or tuning is None:
        return None, None
    if any(ent.get("tuning", {}).get(f, 0) != tuning.get(f, 0) for f in ("kernel", "lanes_per_col", "heads")):
        return None, None
    # the zero-step certificate changes the kernel's loads (taken without it unless recorded; the
    # warp-cooperative kernel's -1 is its adaptive rule)
    want = int(tuning.get("zero_cert", 0))
    if tuning.get("kernel") != 5 and want < 0:
        want = 0
    if int(ent.get("tuning", {}).get("zero_cert", 0)) != want:
        return None, None
    return float(ent["dram_bytes_per_update"]), ent["tuning"]


def gather_ceiling(m, elem_bytes, kernel_gathers_per_s):
    """Random-gather rates of this GPU as a second ceiling for the iteration
    kernel, whose time goes to scattered gathers of g: pcdm_gather_rate (a full
    grid of independent coherent loads at hashed positions) from a vector of m
    entries (the size of one residual buffer, L2-resident) and from a 4 GiB one
    (every gather a DRAM access), beside the kernel's own rate of gathered
    nonzeros per second."""
    import torch
    from paper_1212_0873_gb300 import _binding as B
    dt = torch.float64 if elem_bytes == 8 else torch.float32
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, size in (("l2_resident", int(m)), ("hbm", (4 << 30) // elem_bytes)):
        src = torch.ones(size, dtype=dt, device="cuda")
        out["gathers_per_s_" + name] = B.pcdm_gather_rate(src.data_ptr(), size, elem_bytes, st)
        del src
    torch.cuda.empty_cache()
    out["kernel_gathers_per_s"] = kernel_gathers_per_s
    if kernel_gathers_per_s is not None:
        out["kernel_frac_of_l2_resident"] = kernel_gathers_per_s / out["gathers_per_s_l2_resident"]
        out["kernel_frac_of_hbm"] = kernel_gathers_per_s / out["gathers_per_s_hbm"]
    out["how"] = ("pcdm_gather_rate: 2 x 1024 threads per SM, rounds of 16 independent %d-byte coherent loads at "
                  "hashed positions, from a vector of %d entries (one residual buffer) and from a 4 GiB vector; "
                  "kernel: gathered nonzeros per second of the iteration kernel's launches" % (elem_bytes, int(m)))
    return out


class ClockSampler:
    """nvidia-smi samples during the timed region (never changes any setting)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.file = None
        self.gpu = gpu_index
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
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
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- the oracle arm
def host_threads():
    """Host cores this process may run on (the CPU baseline's thread count)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return max(1, os.cpu_count() or 1)


def oracle_sample(inst, tau, seconds, max_iters, threads=1, refresh_every=0):
    """Time the FP64 oracle on the first iterations of the same solve: its
    threaded timing mode on `threads` host threads (equal to the single-threaded
    run bit for bit)."""
    import oracle
    st = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)
    done, t_used = 0, 0.0
    chunk = 1
    while t_used < seconds and done < max_iters:
        t0 = time.perf_counter()
        st.run_threads(tau, chunk, 0, threads, refresh_every=refresh_every)
        t_used += time.perf_counter() - t0
        done += chunk
        chunk = min(chunk * 2, max_iters - done) if done < max_iters else chunk
        if chunk <= 0:
            break
    return done * tau / t_used, done, t_used


def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import oracle
    inst = make_instance(a)
    st = oracle.State(oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64), inst.b, inst.lam)
    threads = host_threads()
    iters_per_step = 4
    for _ in range(a.warmup):
        st.run_threads(a.tau, iters_per_step, 0, threads)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        st.run_threads(a.tau, iters_per_step, 0, threads)
    dt = time.perf_counter() - t0
    value = a.steps * iters_per_step * a.tau / dt
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "m": inst.m, "n": inst.n, "nnz": inst.nnz, "omega": a.omega,
                   "tau": a.tau, "parallelism": "host, %d threads" % threads},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d iterations of %d updates per step, continuing one PCDM1 run from x=0, the "
                                   "oracle's threaded timing mode (FP64, bit-identical to its serial run) on %d "
                                   "threads" % (iters_per_step, a.tau, threads)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched vs plain
def run_batched_path(a):
    """The batched regularisation path: one A (4e6 x 2e6, 15 nonzeros per column,
    BF16 values), 16 right-hand sides, path-len lambdas geometric from lambda_max
    to 1e-3 lambda_max with warm starts, every problem to relative gap 1e-6 at
    each lambda; FP32 residuals, FP64 x, FP64 refresh every 64 iterations.  The
    plain form solves the same 16 paths one problem at a time in FP64 (values
    promoted exactly from the stored BF16), also with warm starts.  Both timed
    with CUDA events on the solver's stream."""
    import numpy as np
    import torch
    from paper_1212_0873_gb300 import BatchLasso, Lasso, instances

    inst, B, lmax = instances.batched_path_instance()
    nrhs = B.shape[0]
    path = np.geomspace(1.0, 1e-3, a.path_len)
    tau, tol = 65536, 1e-6

    def batched_once(bt):
        bt.reset()
        iters = 0
        worst = 0.0
        for f in path:
            bt.set_lambda([v * f for v in lmax])
            ok, it, rel = bt.solve(tau, 0, tol, 10**6)
            if not ok:
                raise RuntimeError("batched path did not converge at lambda factor %g" % f)
            iters += it
            worst = max(worst, float(rel.max()))
        return iters, worst

    with BatchLasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val, B, [v * path[0] for v in lmax],
                    refresh_every=64) as bt:
        batched_tuning = bt.autotune(tau, 20)             # the grid of the batched kernel (untimed)
        batched_once(bt)                                  # warm-up
        bt.reset_stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        iters, worst = batched_once(bt)
        e1.record()
        e1.synchronize()
        t_batched = e0.elapsed_time(e1) / 1e3
        st = bt.stats()

    def plain_path(s, l):
        s.reset()
        its = 0
        for f in path:
            s.set_lambda(lmax[l] * f)
            ok, it, rel = s.solve(tau, 0, tol, 10**6)
            if not ok:
                raise RuntimeError("plain path did not converge")
            its += it
        return its

    # the plain arm as the headline FP64 solve runs: the persisting-L2 window over its
    # residual buffers and the kernel pcdm_autotune picks (tuned once on this A and tau,
    # outside the timed region, and set on every later handle)
    plain_iters = 0
    t_plain = 0.0
    with Lasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64, B[0].copy(), lmax[0], l2_persist=True) as s:
        plain_tuning = s.autotune(tau, 20)
        s.reset()
        plain_path(s, 0)                                  # warm-up
    for l in range(nrhs):
        with Lasso(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64, B[l].copy(), lmax[l],
                   l2_persist=True) as s:
            s.set_tuning(plain_tuning["kernel"], plain_tuning["lanes_per_col"], plain_tuning["threads_per_block"],
                         plain_tuning["heads"], plain_tuning["zero_cert"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plain_iters += plain_path(s, l)
            e1.record()
            e1.synchronize()
            t_plain += e0.elapsed_time(e1) / 1e3
    return {
        "workload": "regularisation path: A %d x %d, 15 nonzeros per column, bf16 values; %d right-hand sides; "
                    "%d lambdas geometric from lambda_max to 1e-3 lambda_max with warm starts; tau=%d; every "
                    "problem to rel. duality gap %g at every lambda; fp32 residuals, fp64 x, fp64 refresh every "
                    "64 iterations" % (inst.m, inst.n, nrhs, a.path_len, tau, tol),
        "time_s": t_batched,
        "problem_updates_per_s": st["updates"] / t_batched,
        "iterations": iters,
        "gap_checks": st["gaps"],
        "max_rel_gap": worst,
        "plain_f64_time_s": t_plain,
        "plain_f64_iterations": plain_iters,
        "plain": "the same 16 paths solved one problem at a time by the plain FP64 form, values promoted "
                 "exactly from the stored bf16, with the persisting-L2 window and the autotuner's kernel",
        "plain_tuning": plain_tuning,
        "batched_tuning": batched_tuning,
        "batched_scatter": "fp32 residuals: one red.global.add.v4.f32 per row for four right-hand sides",
        "speedup_vs_plain_f64": t_plain / t_batched,
    }


# ----------------------------------------------------------------------------- many small problems
def run_multi():
    """256 independent problems (n log-uniform in [1e3, 1e5], m = 2n, 8 nonzeros
    per column, bf16 values, fp32 residuals, fp64 refresh + gap every 64
    iterations, tau = min(256, n)), one thread block each, to relative gap 1e-6;
    against the plain FP64 form solving them one after another."""
    import torch
    from paper_1212_0873_gb300 import Lasso, MultiLasso, instances

    insts = instances.small_instances()
    tol = 1e-6

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        out = fn()
        torch.cuda.synchronize()
        e1.record(torch.cuda.current_stream())
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    with MultiLasso([(i.m, i.n, i.col_ptr, i.row_idx, i.val, i.b, i.lam) for i in insts]) as ml:
        def once():
            ml.reset()
            ok, it, rel = ml.solve(tau=256, seed=0, tol=tol, max_iters=10**7, iters_per_check=64)
            if not ok:
                raise RuntimeError("multi-problem solve did not converge")
            return it
        once()
        ml_stats0 = ml.stats()
        t_multi, iters = timed(once)
        st = ml.stats()
    plain = [Lasso(i.m, i.n, i.col_ptr, i.row_idx, i.val64, i.b, i.lam) for i in insts]
    try:
        def seq():
            its = 0
            for s_, i in zip(plain, insts):
                s_.reset()
                ok, it, rel = s_.solve(min(256, i.n), 0, tol, 10**7)
                if not ok:
                    raise RuntimeError("plain solve did not converge")
                its += it
            return its
        seq()
        t_plain, plain_iters = timed(seq)
    finally:
        for s_ in plain:
            s_.close()
    updates = st["updates"] - ml_stats0["updates"]
    return {"workload": "256 independent problems, n log-uniform in [1e3, 1e5], m = 2n, 8 nonzeros per column, "
                        "bf16 values, fp32 residuals, fp64 refresh and gap every 64 iterations, tau = min(256, n), "
                        "each to rel. duality gap 1e-6",
            "time_s": t_multi, "problem_updates_per_s": updates / t_multi, "max_iterations": int(iters.max()),
            "total_n": int(sum(i.n for i in insts)),
            "plain_f64_time_s": t_plain, "plain_f64_iterations": plain_iters,
            "plain": "the same problems solved one after another by the plain FP64 form (pcdm_solve, same tau)",
            "speedup_vs_plain_f64": t_plain / t_multi}


# ----------------------------------------------------------------------------- differentiation
def _timed_cuda(fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def run_svm():
    """The SVM-dual workload of Sec. 8.3 on rcv1-shaped synthetic data: n =
    677,399 examples, d = 47,236 features, 73 feature draws per example with
    popularity proportional to (r+1)^-0.64 (so the most common feature is in
    about 43% of the examples: omega / n near the paper's 291,516 / 677,399),
    unit-norm nonnegative values, lambda = 1e-5.  Each tau solves from x = 0 to
    relative duality gap 1e-2 (the paper: a gap near 0.01 suffices for
    training).  Reported per tau: beta, iterations, epochs, time, and the
    speedup in iterations over tau = 1 beside the theory's tau / beta."""
    import numpy as np
    from paper_1212_0873_gb300 import LabeledProblem, instances

    t0 = time.perf_counter()
    inst = instances.svm_instance(47_236, 677_399, 73, lam=1e-5, zipf=0.64, val_dtype="f64", seed=1010)
    t_gen = time.perf_counter() - t0
    rows = []
    with LabeledProblem.from_instance(inst, check_every=0) as s:
        for tau in (1, 16, 256):
            s.reset()
            tuning = s.autotune(tau, 200)
            s.solve(tau, 0, 0.5, 10**7)                      # warm-up: the kernel of this tau, column heads
            s.reset()
            t, (ok, it, rel) = _timed_cuda(lambda: s.solve(tau, 0, 1e-2, 10**8))
            x = s.x()
            rows.append({"tau": tau, "beta": s.beta(tau), "tuning": tuning, "converged": ok, "iterations": it,
                         "epochs": it * tau / inst.n, "seconds": t, "rel_gap": rel,
                         "updates_per_s": it * tau / t, "at_upper_bound": float(np.mean(x == 1.0)),
                         "at_zero": float(np.mean(x == 0.0))})
        omega = s.omega
    base = rows[0]["iterations"]
    for r in rows:
        r["iteration_speedup"] = base / r["iterations"]
        r["theory_tau_over_beta"] = r["tau"] / r["beta"]
        r["time_speedup"] = rows[0]["seconds"] / r["seconds"]
    return {"workload": "SVM dual (Sec. 8.3), rcv1-shaped synthetic: n=677399 examples, d=47236 features, %d "
                        "nonzeros (about 72 per example), omega=%d, lambda=1e-5, fp64; from x=0 to relative duality "
                        "gap 1e-2" % (inst.nnz, omega),
            "generate_s": t_gen, "omega": omega, "rows": rows}


def run_logistic(a):
    """L2-regularised logistic regression (Sec. 8.4) on KDDB-shaped synthetic
    data at a smaller scale: m = 2e6 examples (rows) with exactly 29 features each
    (KDDB's mean; so omega = 29) out of n = 3e6, N(0,1)/sqrt(29) values, labels
    from a logistic model, lambda = 1 as in the paper.  tau = 65536 from x = 0 to
    relative duality gap 1e-6, once with FP64 values and margins and once with
    BF16 values and FP32 margins (FP64 x and steps, FP64 refresh every 64
    iterations); the time of one epoch and F(x_0)/F(x_k) after it (the ratio the
    paper's table reports)."""
    from paper_1212_0873_gb300 import LabeledProblem, instances

    tau = 65536
    rows = []
    cpu = None
    for val_dtype in ("f64", "bf16"):
        t0 = time.perf_counter()
        inst = instances.logistic_instance(2_000_000, 3_000_000, 29, lam=1.0, val_dtype=val_dtype, seed=1011)
        t_gen = time.perf_counter() - t0
        refresh = 0 if val_dtype == "f64" else 64
        with LabeledProblem.from_instance(inst, profile=True, refresh_every=refresh) as s:
            tuning = s.autotune(tau, 20)
            s.reset()
            s.solve(tau, 0, 1e-6, 10**6)                      # warm-up
            s.reset()
            F0 = s.gap()["primal"]
            epoch_iters = (inst.n + tau - 1) // tau
            s.reset()
            t_epoch, _ = _timed_cuda(lambda: s.step(tau, epoch_iters, 0))
            F1 = s.gap()["primal"]
            s.reset()
            s.reset_stats()
            t_solve, (ok, it, rel) = _timed_cuda(lambda: s.solve(tau, 0, 1e-6, 10**6))
            st = s.stats()
            beta = s.beta(tau)
        # algorithmic bytes as for LASSO: per gathered nonzero value + index + margin, per update
        # x read and write, 1/L and the descriptor, per scattered nonzero value + index + margin read/write
        sv, sg = st["val_bytes"], st["xg_bytes"]
        alg = st["gathered_nnz"] * (sv + 4 + sg) + st["updates"] * (16 + sg + 8) + st["scattered_nnz"] * (sv + 4 + 2 * sg)
        kernel_s = st["iter_kernel_ms"] / 1e3
        rows.append({"values": val_dtype, "margins": "f64" if val_dtype == "f64" else "f32", "generate_s": t_gen,
                     "beta": beta, "tuning": tuning, "epoch_s": t_epoch, "epoch_iterations": epoch_iters,
                     "F0_over_F1epoch": F0 / F1, "solve_s": t_solve, "converged": ok, "iterations": it,
                     "rel_gap": rel, "updates_per_s": it * tau / t_solve,
                     "us_per_iteration_kernel": 1e6 * kernel_s / max(st["iterations"], 1),
                     "alg_GB_per_s": alg / kernel_s / 1e9 if kernel_s > 0 else None})
        if val_dtype == "f64" and not a.no_cpu_baseline:
            import oracle
            A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
            ost = oracle.GlmState(oracle.LOGISTIC, A, inst.y, inst.lam)
            c0 = time.perf_counter()
            ost.run(tau, 4, 0)
            c1 = time.perf_counter() - c0
            cpu = {"value": 4 * tau / c1, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "first 4 iterations (tau=%d) of the FP64 run, single-threaded FP64 oracle, %.1f s"
                             % (tau, c1)}
        del inst
    return {"workload": "L2-regularised logistic regression (Sec. 8.4), KDDB-shaped synthetic at 1/10 scale: "
                        "m=2e6 examples x n=3e6 features, 29 nonzeros per example (omega=29), lambda=1; "
                        "tau=65536 from x=0 to relative duality gap 1e-6",
            "note": "every gathered nonzero costs one exp (the logistic gradient map): an FP64 exp in the FP64 "
                    "form, an FP32 one in the BF16/FP32 form",
            "rows": rows, "cpu_baseline": cpu}


def run_grad():
    """Forward (solve to relative gap 1e-6, then the FP64 polish on the support)
    and backward (pcdm_backward: dL/db and dL/dlambda for L = 1/2 ||x - x*||^2)
    on the differentiation workload: A 1e6 x 5e5, 12 FP32 nonzeros per column,
    x* 1% dense, b = A x* + N(0, 1e-4), lambda = 0.1 ||A^T b||_inf."""
    import numpy as np
    import torch
    from paper_1212_0873_gb300 import Lasso, instances

    inst = instances.per_col_instance(1_000_000, 500_000, 12, density=0.01, noise=0.01, lam_frac=0.1,
                                      val_dtype="f32", seed=1005)
    tau = 4096
    with Lasso.from_instance(inst, refresh_every=64) as s:
        def forward():
            s.reset()
            ok, it, rel = s.solve(tau, 0, 1e-6, 10**6)
            ok2, it2, res2 = s.polish(1e-14)
            if not (ok and ok2):
                raise RuntimeError("differentiation forward failed")
            return it, it2

        def timed(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3, out

        forward()                                            # warm-up
        t_fwd, (it, it2) = timed(forward)
        x = s.x()
        dx = torch.from_numpy(x - inst.x_star).cuda()
        db = torch.empty(inst.m, dtype=torch.float64, device="cuda")
        s.backward(dx, tol=1e-13, db_out=db)                 # warm-up
        t_bwd, (db, dlam, ok, itb, res) = timed(lambda: s.backward(dx, tol=1e-13, db_out=db))
        support = s.support_size()
    return {"workload": "A 1e6 x 5e5, 12 fp32 nonzeros per column; L = 1/2 ||x(b, lambda) - x*||^2; forward "
                        "= solve to rel. gap 1e-6 (tau=%d) + fp64 polish on the support to 1e-14; backward = "
                        "dL/db (1e6) and dL/dlambda to relative residual 1e-13" % tau,
            "forward_s": t_fwd, "forward_iterations": it, "polish_iterations": it2,
            "backward_s": t_bwd, "backward_iterations": itb, "backward_rel_residual": res,
            "support": support}


# ----------------------------------------------------------------------------- asynchronous mode
def run_async(a, inst):
    """The asynchronous mode (pcdm_solve_async: every GPU thread applies
    updates with atomics, no barrier) on the bench workload, to the same
    relative gap; device-timed solves after one warm-up."""
    import torch
    from paper_1212_0873_gb300 import Lasso

    out = {}
    with Lasso.from_instance(inst, profile=False) as s:
        def once():
            s.reset()
            ok, upd, rel = s.solve_async(seed=0, tol=a.tol, max_updates=10**12)
            if not ok:
                raise RuntimeError("asynchronous solve did not converge")
            return upd, rel
        once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        upd, rel = once()
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
    out.update({"workload": "the bench workload, asynchronous updates (all resident GPU threads, atomics on x and "
                            "g, no barrier), from x = 0 to the same relative gap",
                "time_to_gap_s": t, "updates": upd, "updates_per_s": upd / t, "rel_gap": rel})
    return out


# ----------------------------------------------------------------------------- theory vs reality
def run_theory_vs_reality():
    """Sec. 8.2: iteration speedup of tau-nice PCDM1 against tau / beta on least
    squares with 3000 x 1000 equal-valued rows of omega nonzeros, eps = 1e-6."""
    import time
    from paper_1212_0873_gb300 import experiments
    t0 = time.perf_counter()
    rows = experiments.theory_vs_reality()
    dev = max(abs(r["empirical"] / r["theory"] - 1.0) for r in rows)
    return {"workload": "min 1/2 ||Ax - b||^2, A 3000 x 1000 with omega in {5, 10, 50, 100} equal nonzeros per row, "
                        "tau in 1 .. 1000, iterations until F - F* <= 1e-6",
            "max_relative_deviation_from_tau_over_beta": dev, "seconds": time.perf_counter() - t0,
            "rows": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in rows]}


# ----------------------------------------------------------------------------- the CUDA arm
def kernel_name(a, tuning):
    if a.unfused or (tuning and tuning["kernel"] == 2):
        return "k_gather + k_scatter (two-kernel PCDM1 iterations)"
    if tuning and tuning["kernel"] == 1:
        return "k_fused (persistent PCDM1 iterations, %d lanes per column)" % tuning["lanes_per_col"]
    if tuning and tuning["kernel"] == 3:
        return "k_fused_pipe_rounds (persistent PCDM1 iterations, several positions per thread)"
    if tuning and tuning["kernel"] == 4:
        return "k_fused_stream (persistent PCDM1 iterations, columns streamed by TMA)"
    if tuning and tuning["kernel"] == 5:
        return "k_fused_warp (persistent PCDM1 iterations, a warp per column)"
    return "k_fused_pipe_wide (persistent PCDM1 iterations, pipelined, wide slots)"


def kernel_roofline(a, st, tuning, dtype):
    """Roofline of the iteration kernel from a handle's counters: algorithmic
    bytes per launch (per gathered nonzero value + row index + g_r; per update
    x_i read and write (FP64), 1/L_i and the column's start and length; per
    scattered nonzero value + row index + read and write of g_r) over its
    CUDA-event-timed average launch."""
    sv, sg, sx = st["val_bytes"], st["xg_bytes"], 8
    sidx, sL = 4, sg
    alg_bytes = (st["gathered_nnz"] * (sv + sidx + sg) + st["updates"] * (2 * sx + sL + 8)
                 + st["scattered_nnz"] * (sv + sidx + 2 * sg))
    launches = max(st["iter_launches"], 1)
    avg_launch_s = st["iter_kernel_ms"] / launches / 1e3
    achieved = alg_bytes / launches / avg_launch_s / 1e9 if avg_launch_s > 0 else None
    peak, peak_kind = measured_peaks()
    b = argparse.Namespace(**dict(vars(a), dtype=dtype))
    tpu, tpu_tuning = traffic_per_update(b, tuning)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (tpu * st["updates"] / launches) if tpu is not None else None,
                "kernel": kernel_name(a, tuning), "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes / launches, "avg_launch_ms": avg_launch_s * 1e3,
                "launches": st["iter_launches"], "traffic_taken_at": tpu_tuning}
    return roofline, avg_launch_s, launches


def rel_err(a_, b_):
    b_ = np.asarray(b_, dtype=np.float64)
    return float(np.max(np.abs(np.asarray(a_, dtype=np.float64) - b_))) / max(float(np.max(np.abs(b_))), 1e-300)


def error_vs_oracle(a, inst, solver, refresh, x_final, gpu_rel_gap, threads, K=64):
    """The result's error against the FP64 oracle: x and g after K iterations
    from x = 0 (same seed and samples on both sides), and the final x of the
    timed solve judged by the oracle's own residual and duality gap."""
    import oracle
    solver.reset()
    solver.step(a.tau, K, 0)
    xg, gg = solver.x(), solver.residual()
    A = oracle.Csc(inst.m, inst.n, inst.col_ptr, inst.row_idx, inst.val64)
    ref = oracle.State(A, inst.b, inst.lam)
    ref.run_threads(a.tau, K, 0, threads, refresh_every=refresh)
    r = oracle.residual(A, inst.b, x_final)
    rec = oracle.gap(A, inst.b, x_final, r, inst.lam)
    return {"iterations": K, "x_rel_err_after_K": rel_err(xg, ref.x), "g_rel_err_after_K": rel_err(gg, ref.g),
            "final_rel_gap_by_oracle": rec["gap"] / max(rec["primal"], 1e-300), "final_rel_gap_by_gpu": gpu_rel_gap,
            "how": "max|v - v_oracle| / max|v_oracle| after K iterations of tau=%d from x=0 (seed 0, the same S_k; "
                   "the oracle in FP64 on the stored values); the oracle's residual and duality gap of the timed "
                   "solve's final x" % a.tau}


def run_other_precision(a, dtype, threads, steps=5, warmup=3):
    """The same workload with values stored in `dtype` (FP32 residual, FP64 x,
    FP64 refresh every 64 iterations and FP64 gap): time to relative gap tol,
    updates/s, the iteration kernel's roofline and the error against the oracle."""
    import torch
    from paper_1212_0873_gb300 import Lasso
    b = argparse.Namespace(**dict(vars(a), dtype=dtype))
    inst = make_instance(b)
    refresh = 64
    solver = Lasso.from_instance(inst, profile=True, refresh_every=refresh, check_every=a.check_every)
    try:
        tuning = solver.autotune(a.tau, 30) if not a.no_tune else None
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for _ in range(warmup):
            solver.reset()
            solver.solve(a.tau, 0, a.tol, a.max_iters)
        solver.reset_stats()
        ms, its, rel = [], [], None
        for _ in range(steps):
            flush.zero_()
            solver.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ok, it, rel = solver.solve(a.tau, 0, a.tol, a.max_iters)
            e1.record()
            e1.synchronize()
            if not ok:
                raise RuntimeError("%s solve did not converge" % dtype)
            ms.append(e0.elapsed_time(e1))
            its.append(it)
        st = solver.stats()
        x_final = solver.x()
        roof, _, _ = kernel_roofline(b, st, tuning, dtype)
        err = error_vs_oracle(b, inst, solver, refresh, x_final, rel, threads)
    finally:
        solver.close()
    return {"values": dtype, "residual": "f32", "refresh_every": refresh, "tuning": tuning,
            "updates_per_s": st["updates"] / (sum(ms) / 1e3), "time_to_gap_s": sum(ms) / len(ms) / 1e3,
            "iterations": its[-1], "us_per_iteration": 1e3 * st["iter_kernel_ms"] / max(st["iterations"], 1),
            "roofline": roof, "error_vs_oracle": err, "steps": steps}


def run_omega128(a, steps=3):
    """The long-column end of the scale workload: m = n = 4e6 with omega = 128 nonzeros per row
    (nnz = 5.12e8), FP64, tau = 65536, solved from x = 0 to relative gap tol; the kernel picked by
    pcdm_autotune, with the persisting-L2 window, as the headline.  The autotuner times its
    candidates from the state of a solve taken to relative gap 1e-2 (reached after about half
    of the solve's iterations; from there on the per-iteration time stays flat, while from
    x = 0, where most coordinates still move, the kernels rank differently), then the timed
    solves start from x = 0."""
    import torch
    from paper_1212_0873_gb300 import Lasso
    b = argparse.Namespace(**dict(vars(a), omega=128, dtype="f64"))
    t0 = time.perf_counter()
    inst = make_instance(b)
    t_gen = time.perf_counter() - t0
    with Lasso.from_instance(inst, profile=True, refresh_every=0, l2_persist=True) as s:
        tuning = None
        if not a.no_tune:
            s.solve(a.tau, 0, 1e-2, a.max_iters)
            tuning = s.autotune(a.tau, 20)
        s.reset()
        s.solve(a.tau, 0, a.tol, a.max_iters)              # warm-up
        s.reset_stats()
        ms, its = [], []
        for _ in range(steps):
            s.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ok, it, rel = s.solve(a.tau, 0, a.tol, a.max_iters)
            e1.record()
            e1.synchronize()
            if not ok:
                raise RuntimeError("omega = 128 solve did not converge")
            ms.append(e0.elapsed_time(e1))
            its.append(it)
        st = s.stats()
    roof, _, _ = kernel_roofline(b, st, tuning, "f64")
    return {"workload": "square scale LASSO: m=n=%d, omega=128 per row (nnz=%d), tau=%d, f64 values, solve from x=0 "
                        "to rel. duality gap %g" % (a.n, inst.nnz, a.tau, a.tol),
            "updates_per_s": st["updates"] / (sum(ms) / 1e3), "time_to_gap_s": sum(ms) / len(ms) / 1e3,
            "iterations": its[-1], "us_per_iteration": 1e3 * st["iter_kernel_ms"] / max(st["iterations"], 1),
            "tuning": tuning,
            "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                              "alg_bytes_per_launch", "avg_launch_ms", "traffic_taken_at")},
            "steps": steps, "instance_gen_s": t_gen}


def run_pcdm(a, rank, local, world):
    import torch
    from paper_1212_0873_gb300 import Lasso

    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    inst = make_instance(a)
    t_gen = time.perf_counter() - t_gen
    refresh = a.refresh_every if a.refresh_every >= 0 else (0 if a.dtype == "f64" else 64)
    # FP64: the double-buffered FP64 residual (2 x 8m bytes) only stays in L2 next to the
    # streamed columns with the largest persisting-lines set-aside (opts.l2_persist)
    l2p = a.dtype == "f64" and not a.no_l2_persist
    kw = dict(fused=not a.unfused, refresh_every=refresh, check_every=a.check_every, lanes_per_col=a.lanes,
              l2_persist=l2p)
    seed = rank
    solver = Lasso.from_instance(inst, profile=True, **kw)
    omega = solver.omega
    if a.tuning:
        f = [int(v) for v in a.tuning.split(",")]
        k, w, t, hd = f[:4]
        zc = f[4] if len(f) > 4 else -1
        solver.set_tuning(k, w, t, hd, zc)
        tuning = {"kernel": k, "lanes_per_col": w, "threads_per_block": t, "heads": hd, "zero_cert": zc,
                  "set_by_hand": True}
    else:
        tuning = solver.autotune(a.tau, 30) if (not a.unfused and not a.no_tune) else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def one_solve():
        solver.reset()
        return solver.solve(a.tau, seed, a.tol, a.max_iters)

    for _ in range(a.warmup):
        ok, it, rel = one_solve()
        if not ok:
            raise RuntimeError("warm-up solve did not converge (%d iterations, rel gap %g)" % (it, rel))
    solver.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_ms, iters = [], []
    for _ in range(a.steps):
        flush.zero_()                                   # L2 flush, outside the timed events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ok, it, rel = one_solve()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters.append(it)
        if not ok:
            raise RuntimeError("solve did not converge")
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    st = solver.stats()
    local_seconds = sum(step_ms) / 1e3
    local_updates = st["updates"]
    value, max_seconds, _ = aggregate(local_updates, local_seconds, world)

    roofline, avg_launch_s, launches = kernel_roofline(a, st, tuning, a.dtype)
    sg = st["xg_bytes"]
    if avg_launch_s > 0 and not a.no_gather_ceiling:
        roofline["gather_ceiling"] = gather_ceiling(a.n, sg, st["gathered_nnz"] / launches / avg_launch_s)

    # end to end through the public API from pinned host memory
    e2e = None
    if not a.no_e2e:
        pin = {}
        for name in ("col_ptr", "row_idx", "val", "b"):
            arr = getattr(inst, name)
            t = torch.empty(arr.shape, dtype=getattr(torch, {"float64": "float64", "float32": "float32",
                                                              "int64": "int64", "int32": "int32",
                                                              "uint16": "int16"}[str(arr.dtype)]),
                            pin_memory=True)
            t.numpy().view(arr.dtype)[...] = arr
            pin[name] = t.numpy().view(arr.dtype)
        h2d = sum(v.nbytes for v in pin.values())
        e2e_s, e2e_updates, d2h = [], 0, 0
        phases = [0.0, 0.0, 0.0]
        for q in range(a.warmup + a.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # a one-shot handle: no persisting-L2 set-aside (changing the context limit costs
            # about 14 ms at create and destroy, more than it saves in one solve)
            s2 = Lasso(inst.m, inst.n, pin["col_ptr"], pin["row_idx"], pin["val"], pin["b"], inst.lam,
                       **dict(kw, l2_persist=False))
            t1 = time.perf_counter()
            ok, it, rel = s2.solve(a.tau, seed, a.tol, a.max_iters)
            t2 = time.perf_counter()
            x = s2.x()
            gaps = s2.stats()["gaps"]
            s2.close()
            torch.cuda.synchronize()
            if q >= a.warmup:
                t3 = time.perf_counter()
                e2e_s.append(t3 - t0)
                for j, d in enumerate((t1 - t0, t2 - t1, t3 - t2)):
                    phases[j] += d
                e2e_updates += it * a.tau
                d2h = x.nbytes + gaps * 9 * 8
        e2e_value, _, _ = aggregate(e2e_updates, sum(e2e_s), world)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * sum(e2e_s) / len(e2e_s),
               "ms_create_solve_finish": [round(1e3 * p / len(e2e_s), 2) for p in phases], "l2_persist": False}

    cpu = None
    threads = host_threads()
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, done, used = oracle_sample(inst, a.tau, a.cpu_seconds, max(1, iters[-1]), threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "first %d iterations (tau=%d, %d updates; the GPU's solve takes %d) of the same solve from "
                         "x=0, the FP64 oracle's "
                         "threaded timing mode (bit-identical to its serial run) on %d host threads, %.1f s"
                         % (done, a.tau, done * a.tau, iters[-1], threads, used)}

    # every precision pair on the same workload, each with its error against the oracle
    precisions = None
    if rank == 0 and world == 1 and not a.no_precisions:
        x_final = solver.x()
        head = {"values": a.dtype, "residual": "f64" if a.dtype == "f64" else "f32", "refresh_every": refresh,
                "tuning": tuning, "updates_per_s": value, "time_to_gap_s": max_seconds / a.steps,
                "iterations": iters[-1], "us_per_iteration": 1e3 * st["iter_kernel_ms"] / max(st["iterations"], 1),
                "roofline": {k: roofline[k] for k in ("achieved", "peak", "frac", "traffic", "kernel")},
                "error_vs_oracle": error_vs_oracle(a, inst, solver, refresh, x_final, rel, threads),
                "steps": a.steps}
        precisions = {a.dtype: head}
        for dt in ("f64", "f32", "bf16"):
            if dt != a.dtype:
                precisions[dt] = run_other_precision(a, dt, threads)

    omega128 = None
    if rank == 0 and world == 1 and not a.no_omega128:
        omega128 = run_omega128(a)
    asyn = None
    if rank == 0 and world == 1 and not a.no_async:
        asyn = run_async(a, inst)
    batched = None
    if rank == 0 and world == 1 and not a.no_batched:
        batched = run_batched_path(a)
    multi = None
    if rank == 0 and world == 1 and not a.no_multi:
        multi = run_multi()
    grad = None
    if rank == 0 and world == 1 and not a.no_grad:
        grad = run_grad()
    svm = None
    if rank == 0 and world == 1 and not a.no_svm:
        svm = run_svm()
    logistic = None
    if rank == 0 and world == 1 and not a.no_logistic:
        logistic = run_logistic(a)
    tvr = None
    if rank == 0 and world == 1 and not a.no_tvr:
        tvr = run_theory_vs_reality()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": max_seconds / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
            "config": {"workload": workload_name(a), "m": inst.m, "n": inst.n, "nnz": inst.nnz, "omega": omega,
                       "tau": a.tau, "tol": a.tol, "lambda": inst.lam, "fused": not a.unfused,
                       "refresh_every": refresh, "check_every": a.check_every or math.ceil(a.n / a.tau),
                       "iters_per_solve": iters[-1], "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "256 MB buffer written between timed steps (outside the events); A is %.2f GB"
                             % ((inst.col_ptr.nbytes + inst.row_idx.nbytes + inst.val.nbytes) / 1e9),
                       "l2_persist": l2p},
            "time_to_gap_s": max_seconds / a.steps,
            "tuning": tuning,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": st["kernel_launches"],
            "clocks": clk,
            "precisions": precisions,
            "omega128": omega128,
            "batched": batched,
            "batched_time_s": batched["time_s"] if batched else None,
            "plain_f64_time_s": batched["plain_f64_time_s"] if batched else None,
            "batched_speedup_vs_plain_f64": batched["speedup_vs_plain_f64"] if batched else None,
            "asynchronous": asyn,
            "many_small_problems": multi,
            "differentiation": grad,
            "svm_dual": svm,
            "logistic": logistic,
            "theory_vs_reality": tvr,
            "extras": {"nonzero_update_frac": st["nonzero_updates"] / max(st["updates"], 1),
                       "mean_col_nnz_gathered": st["gathered_nnz"] / max(st["updates"], 1),
                       "us_per_iteration_kernel": 1e3 * st["iter_kernel_ms"] / max(st["iterations"], 1),
                       "gap_checks": st["gaps"], "instance_gen_s": t_gen,
                       "step_ms": [round(v, 3) for v in step_ms]},
        }
        print(json.dumps(out), flush=True)
    solver.close()
    return 0


def run_huge(a):
    """The huge mixed-precision configuration: A 1e9 x 5e8 with 8 BF16 nonzeros
    per column (4e9 nonzeros, generated on the device by libpcdm_gen), b FP32,
    x* 1e-4 dense, lambda = 0.1 ||A^T b||_inf, tau = 2^20, FP32 residuals with an
    FP64 refresh every 32 iterations, solved from x = 0 to relative gap 1e-5.
    One JSON line.  Not part of the default run (about 140 GB of HBM)."""
    import time
    import torch
    from paper_1212_0873_gb300 import Lasso, device_instances
    torch.cuda.set_device(0)
    m, n, per_col, tau, tol = a.huge_m, a.huge_n, 8, 1 << 20, 1e-5
    t0 = time.perf_counter()
    gen = device_instances.per_col_on_device(m, n, per_col, seed=1008, val_dtype="bf16", x_density=1e-4,
                                             noise_sd=1e-2, b_dtype="f32")
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    lam = 0.1 * gen["lambda_max"]
    t0 = time.perf_counter()
    s = Lasso(m, n, gen["col_ptr"], gen["row_idx"], gen["val"], gen["b"], lam, refresh_every=32, profile=True)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    del gen
    torch.cuda.empty_cache()
    if a.tuning:
        f = [int(v) for v in a.tuning.split(",")]
        s.set_tuning(*f)
        tuning = {"kernel": f[0], "lanes_per_col": f[1], "threads_per_block": f[2], "heads": f[3], "set_by_hand": True}
    else:
        tuning = s.autotune(tau, 10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.reset_stats()
    e0.record()
    ok, it, rel = s.solve(tau, 0, tol, 10**6)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    st = s.stats()
    sv, sg, sx = st["val_bytes"], st["xg_bytes"], 8
    alg = (st["gathered_nnz"] * (sv + 4 + sg) + st["updates"] * (2 * sx + sg + 8)
           + st["scattered_nnz"] * (sv + 4 + 2 * sg))
    peak, kind = measured_peaks()
    ach = alg / (st["iter_kernel_ms"] / 1e3) / 1e9
    kernel_gathers = st["gathered_nnz"] / (st["iter_kernel_ms"] / 1e3)
    s.close()
    # the residual (1e9 FP32 entries, 4 GB) is far beyond L2: every gather is a DRAM access
    ceiling = gather_ceiling(m, 4, kernel_gathers)
    print(json.dumps({"workload": "huge: A %d x %d, 8 bf16 nonzeros per column (%d nonzeros), b fp32, tau = 2^20, "
                                  "fp32 residuals, fp64 refresh every 32, from x = 0 to rel. gap 1e-5"
                                  % (m, n, n * per_col),
                      "converged": ok, "iterations": it, "rel_gap": rel, "time_to_gap_s": t,
                      "updates_per_s": it * tau / t, "us_per_iteration": 1e3 * st["iter_kernel_ms"] / it,
                      "tuning": tuning, "generate_s": t_gen, "create_s": t_create,
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                   "peak_source": kind, "kernel": kernel_name(a, tuning),
                                   "gather_ceiling": ceiling,
                                   "kernel_frac_of_random_gather_ceiling": ceiling.get("kernel_frac_of_hbm")}}),
          flush=True)
    return 0


def run_sweep(a):
    """The scale configurations (m = n = 4e6, omega in {2, 16, 128}, tau in {1,
    256, 4096, 65536}, FP64 and FP32): time to relative gap 1e-6 where it takes
    less than about a minute (tau >= 256), updates/s otherwise; one JSON line per
    point.  Not part of the default run."""
    import torch
    from paper_1212_0873_gb300 import Lasso, instances
    torch.cuda.set_device(0)
    for omega in [int(v) for v in a.sweep_omega.split(",")]:
        for dtype in ("f64", "f32"):
            inst = instances.row_omega_instance(a.n, a.n, omega, density=0.01, noise=0.01, lam_frac=0.05,
                                                val_dtype=dtype, seed=1002)
            for tau in (1, 256, 4096, 65536):
                with Lasso.from_instance(inst, profile=True, refresh_every=0 if dtype == "f64" else 64) as s:
                    tuning = s.autotune(tau, 20)
                    rec = {"omega": omega, "dtype": dtype, "tau": tau, "tuning": tuning, "beta": s.beta(tau)}
                    if tau == 1:
                        s.step(tau, 2000, 0)
                        s.reset_stats()
                        s.step(tau, 20000, 0)
                        st = s.stats()
                        rec["updates_per_s"] = st["updates"] / (st["iter_kernel_ms"] / 1e3)
                        rec["us_per_iteration"] = 1e3 * st["iter_kernel_ms"] / st["iterations"]
                    else:
                        s.reset()
                        torch.cuda.synchronize()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        ok, it, rel = s.solve(tau, 0, a.tol, 10**7)
                        e1.record()
                        e1.synchronize()
                        t = e0.elapsed_time(e1) / 1e3
                        st = s.stats()
                        rec.update({"converged": ok, "iterations": it, "rel_gap": rel, "time_to_gap_s": t,
                                    "updates_per_s": it * tau / t,
                                    "us_per_iteration": 1e3 * st["iter_kernel_ms"] / max(st["iterations"], 1)})
                    print(json.dumps(rec), flush=True)
            del inst
    return 0


def main():
    a = parse()
    if a.sweep:
        return run_sweep(a)
    if a.huge:
        return run_huge(a)
    rank, local, world = dist_setup()
    if a.impl == "reference":
        rc = run_reference(a, rank, world)
    else:
        rc = run_pcdm(a, rank, local, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
