"""Benchmark of the overlap-fermion hot path on GB300.

Workload (precision workload): 16^4 lattice, a = r = M0 = 1, m = 0.05,
g = 0.3, phi Gaussian sigma 0.5 (seed 0), 12 complex-Gaussian right-hand
sides (seed 1).  One step = solve (M^dagger M) x = b for all 12 right-hand
sides by the library's CG, FP32 iteration with FP64 reliable updates, to an
FP64 true relative residual <= 1e-10.

value = M^dagger M applies per second over the timed steps, with
applies = sum over right-hand sides of the CG iterations (one FP32 M^dagger M
each) plus the FP64 M^dagger M applies of the reliable updates.  The inputs
are resident on the device; L2 is flushed (256 MB write) before every step.

Extra keys (all on the same GPU, after the timed steps):
  fp64            the same solve in FP64 throughout, also against the measured
                  FP64 FMA throughput (fma_peak_TFLOP_s, the project's microkernel)
  kernels         every kernel class of one solve, probed one launch at a time
                  (CUDA events per launch, algorithmic bytes of the same launches);
                  roofline = the class with the most time per solve
  solve_roofline  the whole CG iteration against HBM (592 B per site-RHS)
  solve_32x4      the mixed solve at 32^4 x 4 RHS, a working set far beyond L2
  apply_sweep     M^dag M applies at L = 8, 16, 32, FP32 and FP64, L2 flushed
                  before every repetition, with the zt and xy passes probed
  hmc             trajectories/s of the 16^4 differentiation workload: one
                  lattice and a batch of independent replicas, mixed and FP64,
                  from thermalised configurations (acceptance, dH, HBM fraction)
  batch           the 64-lattice batching workload (16 each of 4^4..16^4)
  large           the 32^4 workload: an Omelyan trajectory with 4 pseudofermions
                  (2 of its 40 steps by default) and the measurements of the new
                  configuration (<F~>, Ward identity, supercurrent correlators)
  rhmc, one_loop, paper_solver_table, paper_fft_table
                  rational heatbath, RHMC trajectory, one-loop sums, the
                  solver-table runs and M applies on the FFT table's lattices,
                  each beside the paper's printed numbers
  e2e             the headline through the C ABI with host buffers
  cpu_baseline    the FP64 CPU oracle on a bounded sample
  clocks          SM clocks and throttle reasons sampled during the timed steps

--impl reference times the FP64 CPU oracle (the plain definitions) on the
host cores with the same metric.  Under torchrun every rank runs its own
independent replica (the path does not shard a single lattice); rank 0
prints one JSON line with the aggregate over ranks.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1005_3276_gb300 import synth  # noqa: E402

METRIC = "M^dag M applies/s and HMC traj/s at 16^4, mixed vs FP64 GPU @1e-10 residual"


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


PEAK_HBM = measured_peaks().get("hbm_gbs")


def mdagm_flops_per_site(V):
    """Algorithmic flops of one M^dag M apply per site: two M applies, each two
    4D FFTs of 4 spin components at the paper's 5 N log2 N convention plus ~96
    flops of site terms (the survey's count: 1472 at V = 16^4)."""
    return 2.0 * (2.0 * 4.0 * 5.0 * np.log2(V) + 96.0)
UNIT = "M^dag M applies/s"


def solve_gflops(applies, V, seconds):
    """Gflop/s of a solve at the paper's counting (5 N log2 N per FFT, two M
    applies per CG iteration), the convention of its solver-table Gflop/s."""
    return applies * mdagm_flops_per_site(V) * V / seconds / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wz", choices=["wz", "reference"])
    ap.add_argument("--probe", default="auto",
                    help="kernel class for the roofline, e.g. zt_fp32 (auto: the one with the most time per solve)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end solve")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--oracle-sample", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-hmc", action="store_true", help="skip the HMC trajectory timing")
    ap.add_argument("--hmc-traj", type=int, default=2, help="timed mixed trajectories (FP64: half, batched: 1)")
    ap.add_argument("--hmc-replicas", type=int, default=8, help="independent 16^4 replicas of the batched HMC")
    ap.add_argument("--hmc-batch-traj", type=int, default=7,
                    help="timed mixed trajectories of the batch (x replicas: 56 by default, the workload's 50)")
    ap.add_argument("--hmc-therm", type=int, default=4, help="thermalisation trajectories of the HMC start")
    ap.add_argument("--no-sweep", action="store_true", help="skip the L = 8, 16, 32 apply sweep")
    ap.add_argument("--no-solve32", action="store_true", help="skip the 32^4 x 4 RHS mixed solve")
    ap.add_argument("--no-invtab", action="store_true", help="skip the solver-table shaped L^3 x T solves")
    ap.add_argument("--invtab-full", action="store_true",
                    help="also the unpreconditioned FP64 solve of the 32^3 x 64 solver-table row")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-lattice batched workload")
    ap.add_argument("--no-ffttab", action="store_true", help="skip the FFT-table shaped M applies")
    ap.add_argument("--no-rhmc", action="store_true", help="skip the rational heatbath / RHMC timings")
    ap.add_argument("--no-oneloop", action="store_true", help="skip the one-loop lattice sums (Sec. 5 tables)")
    ap.add_argument("--no-large", action="store_true", help="skip the 32^4 Omelyan trajectory and measurements")
    ap.add_argument("--large-steps", type=int, default=2,
                    help="Omelyan steps of the 32^4 trajectory at eps = 1/40 (40: the whole trajectory)")
    ap.add_argument("--rhmc-fp64", action="store_true", help="also time the RHMC trajectory with FP64 solves")
    return ap.parse_args()


def workload_config(w):
    return {
        "workload": f"{w.name}: 16^4 lattice (T=Z=Y=X=16), m={w.m}, g={w.g}, phi Gaussian sigma {w.sigma}, "
                    f"{w.nrhs} complex-Gaussian RHS, CG on M^dag M to {w.tol:g} FP64 true residual",
        "lattice": "16^4",
        "nrhs": w.nrhs,
        "tol": w.tol,
        "solver": "CG, FP32 iteration + FP64 reliable updates (delta 0.1)",
        "l2": "flushed before every step (256 MB write); solver working set ~330 MB > L2",
    }


# ----------------------------------------------------------------------------- CPU oracle


def oracle_applies_per_s(w, seconds):
    """FP64 oracle CG iterations (one M^dag M each) on RHS 0 for ~seconds."""
    import oracle
    P = oracle.Params(dims=w.dims, m=w.m, g=w.g)
    phi = synth.scalar_field(w.dims, w.sigma, 0)
    b = synth.spinor_rhs(1, w.dims, 1)[0]
    A = lambda v: oracle.fftops.apply_MdagM(P, phi, v)  # noqa: E731
    A(b)  # warm caches
    t0 = time.perf_counter()
    c0 = time.process_time()
    n = 0
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    while time.perf_counter() - t0 < seconds:
        Ap = A(p)
        alpha = rr / np.vdot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        n += 1
    dt = time.perf_counter() - t0
    oracle_applies_per_s.cores = max(1, round((time.process_time() - c0) / dt))
    return n / dt, n, dt


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "cg_passes_fp32_16x4_12rhs.traffic.txt")
TRAFFIC_SOURCES = ("wz_kernels.cuh", "wz_cg.cuh", "wz_fft.cuh", "wz_tma.cuh", "launch_impl.cuh", "twiddles.h")

# kernel classes of one mixed solve: FP32 iteration passes and the FP64
# reliable-update passes (zt runs in both precisions)
PROBE_CLASSES = (("zt", 4), ("cg_p1", 4), ("cg_p3", 4), ("cg_p5", 4), ("zt", 8), ("ru_p1", 8), ("cg_p3", 8),
                 ("ru_p5", 8))


def kernel_table(probes):
    """Per kernel class: launches, timed launches, the average event time of a
    timed launch, the algorithmic bytes of a timed launch, the achieved rate
    (bytes / time over the same launches), the time per solve extrapolated to
    every launch, and that time's share of the summed classes."""
    out = {}
    for k, v in probes.items():
        timed = v["timed_launches"]
        if timed <= 0 or v["total_ms"] <= 0:
            out[k] = {"launches": v["launches"], "timed_launches": timed, "avg_launch_us": None,
                      "algorithmic_bytes_per_launch": None, "achieved_GB_s": None, "ms_per_solve": 0.0}
            continue
        avg_ms = v["total_ms"] / timed
        out[k] = {"launches": v["launches"], "timed_launches": timed, "avg_launch_us": 1000.0 * avg_ms,
                  "algorithmic_bytes_per_launch": v["bytes"] / timed,
                  "achieved_GB_s": v["bytes"] / (v["total_ms"] / 1000.0) / 1e9,
                  "ms_per_solve": avg_ms * v["launches"]}
    tot = sum(x["ms_per_solve"] for x in out.values())
    for x in out.values():
        x["share_of_probed_time"] = x["ms_per_solve"] / tot if tot > 0 else None
    return out


def dominant_class(kernels):
    """The class with the largest extrapolated time per solve."""
    return max(kernels, key=lambda k: kernels[k]["ms_per_solve"])


def recorded_traffic(cls, probe, alg_bytes_per_launch):
    """DRAM bytes per launch of an FP32 kernel class from the committed ncu
    record, scaled to the launch's algorithmic bytes, or None if the record is
    for other kernel sources or another class."""
    if not cls.endswith("_fp32") or alg_bytes_per_launch is None:
        return None
    kind = cls[:-len("_fp32")]
    try:
        rec = dict(line.split(":", 1) for line in open(TRAFFIC_FILE) if ":" in line and not line.startswith("#"))
    except OSError:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1005_3276_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != rec.get("source_sha256_16", "").strip() or kind not in rec:
        return None
    per_rhs, alg_per_rhs = (float(v) for v in rec[kind].split())
    return per_rhs * alg_bytes_per_launch / alg_per_rhs


def oracle_sample_one_thread(seconds):
    """The same oracle sample in a child process whose BLAS / OpenMP pools are
    limited to one thread: (applies/s, applies, seconds, threads used)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        return None
    return json.loads(p.stdout.strip().splitlines()[-1])


def cpu_threads():
    """Threads the oracle sample actually kept busy: process CPU time / wall time."""
    return getattr(oracle_applies_per_s, "cores", 1)


def combine_ranks(dist, total_ms, total_applies, device):
    """Whole-job numbers of the replicas: the slowest rank's time and the work of
    all ranks (identity without a process group)."""
    if dist is None:
        return total_ms, total_applies
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    a = torch.tensor([float(total_applies)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), int(a.item())


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    secs = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_applies_per_s(w, secs / 4)
    vals, total_n, total_t = [], 0, 0.0
    for _ in range(args.steps):
        v, n, dt = oracle_applies_per_s(w, secs)
        vals.append(v)
        total_n += n
        total_t += dt
    value = total_n / total_t
    sample = f"FP64 oracle CG iterations on RHS 0 of {w.name}, {total_n} M^dag M applies in {total_t:.1f} s"
    cores = cpu_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(workload_config(w), parallelism="replicas x1"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU arm


def main():
    args = parse()
    w = synth.PRECISION_16
    if args.oracle_sample > 0:
        v, n, dt = oracle_applies_per_s(w, args.oracle_sample)
        print(json.dumps({"value": v, "applies": n, "seconds": dt, "cores": cpu_threads()}))
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1005_3276_gb300 import binding as wz

    stream = torch.cuda.current_stream()
    phi = synth.scalar_field(w.dims, w.sigma, 0)
    b = synth.spinor_rhs(w.nrhs, w.dims, 1)
    lat = wz.Lattice(w.dims, m=w.m, g=w.g, stream=stream.cuda_stream)
    lat.set_phi(torch.from_numpy(phi).cuda())
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    def solve(mixed=True):
        rc, st, _ = lat.solve(bd, xd, tol=w.tol, mixed=mixed)
        assert st["converged"] == w.nrhs and st["max_true_residual"] <= w.tol, st
        return st["total_iterations"] + st["reliable_updates"], st

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    # FMA throughput of this GPU (the project's microkernel): the ALU roofline
    # of the FP64 passes
    fp64_peak, _ = wz.wz_fma_peak(8, 20000)
    fp32_peak, _ = wz.wz_fma_peak(4, 1000000)

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = wz.wz_kernel_launches()
    total_ms, total_applies, stats = 0.0, 0, []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n, st = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        total_ms += e0.elapsed_time(e1)
        total_applies += n
        stats.append(st)
    launches = wz.wz_kernel_launches() - launches0
    clk = clocks.stop()

    # Roofline of the dominant kernel: one more solve of the same workload per
    # kernel class with the library's probe armed (CUDA events around every
    # launch of the class on its launching stream; the probe makes the solver
    # launch its kernels one by one on one stream instead of replaying its
    # graph -- the kernels are the same).
    probes = {}
    for kind, rb in PROBE_CLASSES:
        flush.zero_()
        torch.cuda.synchronize()
        wz.wz_probe_begin(kind, rb)
        solve()
        probes[f"{kind}_fp{8 * rb}"] = wz.wz_probe_end()
    # the same kernels with one launch per pass covering all right-hand sides
    # (the group size forced to nrhs): per-kernel efficiency at full launch size
    probes_full = {}
    saved = {k: os.environ.get(k) for k in ("WZ_RHS_GROUP", "WZ_RHS_BRANCHES")}
    os.environ["WZ_RHS_GROUP"], os.environ["WZ_RHS_BRANCHES"] = str(w.nrhs), "1"
    for kind, rb in PROBE_CLASSES[:4]:
        flush.zero_()
        torch.cuda.synchronize()
        wz.wz_probe_begin(kind, rb)
        solve()
        probes_full[f"{kind}_fp{8 * rb}"] = wz.wz_probe_end()
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v

    t_max, applies_all = combine_ranks(dist, total_ms, total_applies, "cuda")
    value = applies_all / (t_max / 1000.0)

    # FP64 throughout, same workload: one untimed solve (its tuner and graph
    # capture), then one timed solve
    fp64 = None
    if not args.no_fp64:
        solve(mixed=False)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n64, st64 = solve(mixed=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        tf64 = n64 * mdagm_flops_per_site(int(np.prod(w.dims))) * int(np.prod(w.dims)) / (ms64 / 1000.0) / 1e12
        fp64 = {"value": n64 / (ms64 / 1000.0), "unit": UNIT, "ms_per_solve": ms64,
                "alu_TFLOP_s": tf64, "fp64_fma_peak_TFLOP_s": fp64_peak, "frac_of_fp64_peak": tf64 / fp64_peak,
                "roofline_note": "FP64 passes are arithmetic-bound on this GPU: M^dag M flops at the paper's "
                                 "5 N log2 N FFT convention (1472 per site at 16^4) against the measured FP64 "
                                 "FMA throughput",
                "iterations": st64["iterations"], "max_true_residual": st64["max_true_residual"],
                "mixed_speedup_per_solve": ms64 / (total_ms / args.steps)}

    # HMC trajectories/s on the differentiation workload (16^4, m = 0.1, g = 0.5,
    # one pseudofermion, tau = 1, 20 leapfrog steps, CG to 1e-10), mixed and
    # FP64 solves, one lattice and a batch of R independent replicas (one
    # context, the replicas as members; each trajectory of the batch is one
    # CUDA graph).  All start from the same configurations, thermalised by
    # args.hmc_therm shorter trajectories (tau 0.5, 10 steps) of the batch.
    hmc = None
    if not args.no_hmc:
        hw = synth.FORCE_16
        V = int(np.prod(hw.dims))
        R = args.hmc_replicas
        kw = dict(tau=hw.extra["tau"], nsteps=hw.extra["nsteps"], npf=1, tol=1e-10)
        hmc = {"workload": f"{hw.name}: 16^4, m={hw.m}, g={hw.g}, 1 pseudofermion, tau={hw.extra['tau']}, "
                           f"{hw.extra['nsteps']} leapfrog steps, CG to 1e-10; start: {R} configurations drawn "
                           f"with sigma {hw.sigma}, then {args.hmc_therm} trajectories of tau 0.5, 10 steps",
               "bytes_per_site_cg_iteration": {"mixed": 18 * 32 + 2 * 8, "fp64": 18 * 64 + 2 * 16},
               "bytes_per_site_mdagm": {"mixed": 440, "fp64": 880}}
        bt = wz.Batch([dict(dims=hw.dims, m=hw.m, g=hw.g)] * R)
        for i in range(R):
            bt.set_phi(i, torch.from_numpy(synth.scalar_field(hw.dims, hw.sigma, 300 + i)).cuda())
        therm = []
        for t in range(args.hmc_therm):
            sts = bt.trajectory(tau=0.5, nsteps=10, npf=1, tol=1e-10, seed=555, traj_index=t)
            therm.append([round(x["dH"], 3) for x in sts])
        hmc["thermalisation_dH"] = therm
        phis = []
        for i in range(R):
            p = torch.zeros(hw.dims, dtype=torch.complex128, device="cuda")
            bt.get_phi(i, p)
            phis.append(p)

        def fractions(d, label, ms, iters):
            d["cg_GB_s"] = iters * hmc["bytes_per_site_cg_iteration"][label] * V / (ms / 1000.0) / 1e9
            d["cg_frac_of_hbm"] = d["cg_GB_s"] / (PEAK_HBM or 6800.0)
            d["mdagm_frac_of_hbm"] = (iters * hmc["bytes_per_site_mdagm"][label] * V / (ms / 1000.0) / 1e9
                                      / (PEAK_HBM or 6800.0))

        hlat = wz.Lattice(hw.dims, m=hw.m, g=hw.g, stream=stream.cuda_stream)
        for label, flags in (("mixed", 0), ("fp64", wz.WZ_HMC_FP64_SOLVES)):
            n = args.hmc_traj if label == "mixed" else max(1, args.hmc_traj // 2)
            hlat.set_phi(phis[0])
            hlat.trajectory(traj_index=1000, seed=2024, flags=flags, **kw)  # warm-up (graph capture)
            hlat.set_phi(phis[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = [hlat.trajectory(traj_index=t, seed=2024, flags=flags, **kw) for t in range(n)]
            torch.cuda.synchronize()
            ms = 1000.0 * (time.perf_counter() - t0)
            iters = float(sum(x["cg_iterations"] for x in sts))
            d = {"traj_per_s": n / (ms / 1000.0), "ms_per_traj": ms / n, "trajectories": n,
                 "cg_iterations_per_traj": iters / n, "dH": [round(x["dH"], 4) for x in sts],
                 "accepted": int(sum(x["accept"] for x in sts))}
            fractions(d, label, ms, iters)
            hmc["single_" + label] = d
        hlat.close()
        for label, flags in (("mixed", 0), ("fp64", wz.WZ_HMC_FP64_SOLVES)):
            n = args.hmc_batch_traj if label == "mixed" else 1
            for i in range(R):
                bt.set_phi(i, phis[i])
            bt.trajectory(traj_index=1000, seed=2024, flags=flags, **kw)  # warm-up (graph capture)
            for i in range(R):
                bt.set_phi(i, phis[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = [bt.trajectory(traj_index=t, seed=2024, flags=flags, **kw) for t in range(n)]
            torch.cuda.synchronize()
            ms = 1000.0 * (time.perf_counter() - t0)
            iters = float(sum(x[0]["cg_iterations"] for x in sts))  # all members of the group together
            d = {"replicas": R, "traj_per_s": R * n / (ms / 1000.0), "ms_per_batch_traj": ms / n,
                 "trajectories_per_replica": n, "cg_iterations_per_batch_traj": iters / n,
                 "dH": [[round(x["dH"], 4) for x in st] for st in sts],
                 "accepted": int(sum(x["accept"] for st in sts for x in st)), "of": R * n}
            fractions(d, label, ms, iters)
            hmc[f"batch{R}_" + label] = d
        bt.close()
        hmc["batched_mixed_over_single_fp64"] = hmc[f"batch{R}_mixed"]["traj_per_s"] / hmc["single_fp64"]["traj_per_s"]
        hmc["batched_mixed_over_batched_fp64"] = (hmc[f"batch{R}_mixed"]["traj_per_s"]
                                                  / hmc[f"batch{R}_fp64"]["traj_per_s"])
        hmc["single_mixed_over_single_fp64"] = hmc["single_mixed"]["traj_per_s"] / hmc["single_fp64"]["traj_per_s"]

    # rational heatbath eta = (M^dag M)^1/8 R of the paper's heatbath table: L^3 x 32,
    # m = 1, g = 0.1, degree 20, poles beta <= 100 preconditioned by M0^-1; the
    # interval is the free spectrum widened by 2 on both ends.  Then RHMC
    # trajectories (r_a ~ x^-1/4, r_h ~ x^1/8, degree 20) on the HMC workload.
    rhmc = None
    if not args.no_rhmc:
        rhmc = {"heatbath": [], "paper_gtx285": {"8^3x32": {"single_s": 0.93, "single_iters": 360, "double_s": 3.5,
                                                           "double_iters": 700, "single_gflops": 15,
                                                           "double_gflops": 7.5},
                                                "16^3x32": {"single_s": 4.8, "single_iters": 370, "double_s": 20,
                                                            "double_iters": 730, "single_gflops": 28,
                                                            "double_gflops": 13}}}
        for L in (8, 16):
            dims = (32, L, L, L)
            rl = wz.Lattice(dims, m=1.0, g=0.1, stream=stream.cuda_stream)
            rl.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
            lo, hi = rl.spectral_bounds()
            rh = wz.wz_rational_minimax(0.125, 0.5 * lo, 2.0 * hi, 20)
            R = torch.from_numpy(synth.spinor_rhs(1, dims, 1)).cuda()
            eta = torch.empty_like(R)
            row = {"lattice": f"{L}^3x32", "degree": 20, "interval": [0.5 * lo, 2.0 * hi], "approx_err": rh.err}
            for label, mixed, tol, pc in (("mixed_1e-6_pc", True, 1e-6, True), ("mixed_1e-10_pc", True, 1e-10, True),
                                          ("fp64_1e-12_pc", False, 1e-12, True), ("mixed_1e-10_nopc", True, 1e-10, False)):
                rl.rational_apply(rh, R, eta, tol=tol, mixed=mixed, pc=pc)  # warm-up (graphs, tuner)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = rl.rational_apply(rh, R, eta, tol=tol, mixed=mixed, pc=pc)
                e1.record(stream)
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) / 1000.0
                row[label] = {"seconds": sec, "total_iterations": st["total_iterations"],
                              "max_iterations": st["iterations"], "reliable_updates": st["reliable_updates"],
                              "gflops": solve_gflops(st["total_iterations"] + st["reliable_updates"],
                                                     L ** 3 * 32, sec)}
            rhmc["heatbath"].append(row)
            rl.close()
        hw = synth.FORCE_16
        tl = wz.Lattice(hw.dims, m=hw.m, g=hw.g, stream=stream.cuda_stream)
        lo, hi = tl.spectral_bounds()
        ra = wz.wz_rational_minimax(-0.25, 0.5 * lo, 2.0 * hi, 20)
        rh = wz.wz_rational_minimax(0.125, 0.5 * lo, 2.0 * hi, 20)
        rhmc["trajectory"] = {"workload": f"{hw.name}: 16^4, m={hw.m}, g={hw.g}, 1 pseudofermion, degree 20 "
                                          f"(action err {ra.err:.2e}, heatbath err {rh.err:.2e}), "
                                          f"tau={hw.extra['tau']}, {hw.extra['nsteps']} leapfrog steps, CG to 1e-10"}
        for label, flags in (("mixed", 0),) + ((("fp64", wz.WZ_HMC_FP64_SOLVES),) if args.rhmc_fp64 else ()):
            tl.set_phi(torch.from_numpy(synth.scalar_field(hw.dims, hw.sigma, 0)).cuda())
            kw = dict(tau=hw.extra["tau"], nsteps=hw.extra["nsteps"], npf=1, tol=1e-10, seed=2024, flags=flags)
            tl.rhmc_trajectory(ra, rh, traj_index=0, **kw)  # warm-up (graph capture)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sts = []
            e0.record(stream)
            for t in range(args.hmc_traj):
                sts.append(tl.rhmc_trajectory(ra, rh, traj_index=1 + t, **kw))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rhmc["trajectory"][label] = {"ms_per_traj": ms / args.hmc_traj,
                                         "cg_iterations_per_traj": float(np.mean([x["cg_iterations"] for x in sts])),
                                         "dH": [round(x["dH"], 5) for x in sts],
                                         "accept": [x["accept"] for x in sts]}
        tl.close()

    # CG solves shaped like the paper's solver table (Sec. 7.4): L^3 x 32, m = 1,
    # g = 0.2, one Gaussian right-hand side; unpreconditioned and M0^-1
    # preconditioned; FP32 iteration to 1e-6 and FP64 to 1e-12 (true residual).
    # Printed beside the paper's GTX 285 seconds and iterations (context only).
    invtab = None
    if not args.no_invtab:
        paper = {"8^3x32": {"single": (1.3, 830, 0.038, 8), "double": (4.9, 1600, 0.13, 15)},
                 "16^3x32": {"single": (7.1, 870, 0.20, 8), "double": (31, 1800, 0.74, 15)},
                 "32^3x64": {"single": (420, 1600, 6.8, 8), "double": (2200, 3900, 25, 15)}}
        # the same table's Gflop/s columns (no PC, PC)
        paper_gflops = {"8^3x32": {"single": (14, 17), "double": (7.2, 8.1)},
                        "16^3x32": {"single": (25, 31), "double": (12, 13)},
                        "32^3x64": {"single": (14, 15), "double": (6.5, 7.0)}}
        invtab = {"workload": "L^3 x T (8^3 x 32, 16^3 x 32, 32^3 x 64), m = 1, g = 0.2, phi sigma 0.5, "
                              "1 complex-Gaussian RHS; "
                              "'single' = FP32 iteration with FP64 reliable updates to 1e-6, "
                              "'double' = FP64 to 1e-12 (true residuals)", "rows": []}
        for L, T in ((8, 32), (16, 32), (32, 64)):
            dims = (T, L, L, L)
            il = wz.Lattice(dims, m=1.0, g=0.2, stream=stream.cuda_stream)
            il.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
            bi = torch.from_numpy(synth.spinor_rhs(1, dims, 1)).cuda()
            xi = torch.zeros_like(bi)
            row = {"lattice": f"{L}^3x{T}", "paper_gtx285": paper[f"{L}^3x{T}"],
                   "paper_gtx285_gflops": paper_gflops[f"{L}^3x{T}"]}
            for prec, mixed, tol in (("single", True, 1e-6), ("double", False, 1e-12)):
                for pc in (False, True):
                    if T == 64 and prec == "double" and not pc and not args.invtab_full:
                        continue  # thousands of FP64 iterations at 2M sites: --invtab-full
                    il.solve(bi, xi, tol=tol, mixed=mixed, pc=pc)  # warm-up (graph, tuner)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    rc, st, _ = il.solve(bi, xi, tol=tol, mixed=mixed, pc=pc)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    sec = e0.elapsed_time(e1) / 1000.0
                    row[f"{prec}_{'pc' if pc else 'npc'}"] = {
                        "seconds": sec, "iterations": st["iterations"],
                        "reliable_updates": st["reliable_updates"], "true_residual": st["max_true_residual"],
                        "gflops": solve_gflops(st["total_iterations"] + st["reliable_updates"], L ** 3 * T, sec)}
            invtab["rows"].append(row)
            il.close()

    # The paper's 4D FFT table (one spinor field, Gflop/s at 5 N log2 N) beside
    # one M apply on the same lattices: the apply's two 4D FFTs of the 4 spin
    # components are counted, its momentum multiply and site terms are not (a
    # lower bound on the work done).  One right-hand side, L2 flushed before
    # every repetition, median of 10.
    ffttab = None
    if not args.no_ffttab:
        paper = {"8^3x32": {"single": {"cpu": 1.1, "cufft": 6.9, "own": 24}, "double": {"cpu": 0.94, "cufft": 4.4, "own": 11}},
                 "16^3x32": {"single": {"cpu": 0.88, "cufft": 14, "own": 71}, "double": {"cpu": 0.69, "cufft": 10, "own": 35}},
                 "32^3x64": {"single": {"cpu": 0.11, "cufft": 20, "own": None}, "double": {"cpu": 0.085, "cufft": 10, "own": None}}}
        ffttab = {"workload": "M applied to one complex-Gaussian spinor field on L^3 x T, m = 1, g = 0.2; Gflop/s "
                              "counts the apply's two 4D FFTs (4 spin components, 5 N log2 N each) only", "rows": []}
        for L, T in ((8, 32), (16, 32), (32, 64)):
            dims = (T, L, L, L)
            V = L ** 3 * T
            fl = wz.Lattice(dims, m=1.0, g=0.2, stream=stream.cuda_stream)
            fl.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
            row = {"lattice": f"{L}^3x{T}", "paper_gtx285_gflops": paper[f"{L}^3x{T}"]}
            for name, dt in (("single", torch.complex64), ("double", torch.complex128)):
                x = torch.from_numpy(synth.spinor_rhs(1, dims, 1)).to(dt).cuda()
                y = torch.empty_like(x)
                for _ in range(3):
                    fl.apply("M", x, y, 1)
                times = []
                for _ in range(10):
                    flush.zero_()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fl.apply("M", x, y, 1)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = float(np.median(times))
                row[name] = {"ms_per_apply": ms, "fft_gflops": 2 * 4 * 5.0 * V * np.log2(V) / (ms / 1000.0) / 1e9}
            ffttab["rows"].append(row)
            fl.close()

    # one-loop counterterms of Tables sse, fse, ase at mL = 8 (N = 8 / ma up to 1024),
    # FP64 on the device, beside the paper's printed mL = 8 columns
    oneloop = None
    if not args.no_oneloop:
        paper = {0.5: (-0.006355, -0.004027, 0.082542), 0.25: (-0.009532, -0.006973, 0.088658),
                 0.125: (-0.013358, -0.011406, 0.095266), 0.0625: (-0.017541, -0.015632, 0.105719),
                 0.03125: (-0.021837, -0.019965, 0.11255), 0.015625: (-0.026205, -0.024336, 0.13276),
                 0.0078125: (-0.030583, -0.028720, 0.140261)}
        oneloop = {"workload": "Z - 1 over |g|^2 at p = (0,0,0,2 pi/N), N = 8/ma, FP64", "rows": []}
        for ma, ref in paper.items():
            N = int(round(8.0 / ma))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            z = wz.wz_one_loop(N, ma)
            dt = time.perf_counter() - t0
            oneloop["rows"].append({"ma": ma, "N": N, "Z_phi": z[0], "Z_chi": z[1], "Z_F": z[2],
                                    "paper_mL8": ref, "seconds": dt,
                                    "terms_per_s": N ** 4 / 48.0 / dt})

    # large single lattice: 32^4, m = 0.02, g = 1.0, hot start sigma 1, 4
    # pseudofermions, mixed CG to 1e-10.  One Omelyan 2MN trajectory at the
    # workload's step size eps = tau / 40 = 0.025, over args.large_steps steps
    # (40 = the whole trajectory of length 1; the default 2 steps is a
    # trajectory of length 0.05 at the same step size), then the measurements
    # of the new configuration: <F~>, both sides of the Ward identity and the
    # supercurrent correlators on one Gaussian noise source.
    large = None
    if not args.no_large:
        lw = synth.LARGE_32
        ll = wz.Lattice(lw.dims, m=lw.m, g=lw.g, stream=stream.cuda_stream)
        ll.set_phi(torch.from_numpy(synth.scalar_field(lw.dims, lw.sigma, 0)).cuda())
        nst = args.large_steps
        eps = lw.extra["tau"] / lw.extra["nsteps"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tst = ll.trajectory(tau=eps * nst, nsteps=nst, npf=lw.nrhs, integrator="omelyan", tol=1e-10, seed=9,
                            traj_index=0)
        torch.cuda.synchronize()
        t_traj = time.perf_counter() - t0
        t0 = time.perf_counter()
        F = ll.aux_vev()
        t_aux = time.perf_counter() - t0
        t0 = time.perf_counter()
        WR, WL, wst = ll.ward_identity(tol=1e-10, mixed=True)
        t_ward = time.perf_counter() - t0
        # supercurrent correlators on one Gaussian noise source, E[w w^*] = 1 per site
        wsrc = torch.from_numpy(synth.scalar_field(lw.dims, np.sqrt(0.5), 2)).cuda()
        t0 = time.perf_counter()
        Rsc, sst = ll.supercurrent(wsrc, tol=1e-10, mixed=True)
        t_sc = time.perf_counter() - t0
        V32 = int(np.prod(lw.dims))
        gbs = tst["cg_iterations"] * 592.0 * V32 / t_traj / 1e9
        large = {"workload": f"{lw.name}: 32^4, m={lw.m}, g={lw.g}, hot start phi sigma {lw.sigma}, {lw.nrhs} "
                             f"pseudofermions, Omelyan 2MN at eps = {eps:g}, mixed CG to 1e-10",
                 "md_steps": nst, "tau": eps * nst, "full_trajectory": nst == lw.extra["nsteps"],
                 "trajectory_s": t_traj, "force_evals": tst["force_evals"], "cg_iterations": tst["cg_iterations"],
                 "dH": tst["dH"], "accept": tst["accept"],
                 "cg_GB_s": gbs, "cg_frac_of_hbm": gbs / (PEAK_HBM or 6800.0),
                 "est_full_trajectory_s": t_traj * (2 * lw.extra["nsteps"] + 1) / max(1, tst["force_evals"]),
                 "aux_vev": [F.real, F.imag], "aux_s": t_aux,
                 "ward_s": t_ward, "ward_cg_iterations_max": wst["iterations"],
                 # the [0][1] element of both sides (C has a zero diagonal, so tr W_L vanishes)
                 "ward_R_01": [float(WR[0, 1].real), float(WR[0, 1].imag)],
                 "ward_L_01": [float(WL[0, 1].real), float(WL[0, 1].imag)],
                 "supercurrent_s": t_sc, "supercurrent_cg_iterations_max": sst["iterations"],
                 "supercurrent_R0_mu0_dx1_dy0_trace": [float(np.trace(Rsc[0, 0, 1, 0]).real),
                                                       float(np.trace(Rsc[0, 0, 1, 0]).imag)]}
        ll.close()

    # apply-throughput sweep: (M^dag M) on L^4, FP32 vs FP64 fields.  Every
    # repetition starts from a flushed L2 (256 MB write, outside its events),
    # so inputs and outputs come from HBM; the pass intermediates of one apply
    # stay wherever the hardware keeps them.  The zt and xy passes of the FP32
    # apply are then probed one launch at a time (CUDA events per launch).
    sweep = None
    if not args.no_sweep:
        sweep = []
        for L, nr in ((8, 256), (16, 16), (16, 3), (32, 1), (32, 4)):
            dims = (L, L, L, L)
            slat = wz.Lattice(dims, m=w.m, g=w.g, stream=stream.cuda_stream)
            slat.set_phi(torch.from_numpy(synth.scalar_field(dims, w.sigma, 0)).cuda())
            row = {"L": L, "nrhs": nr}
            for name, dt, S in (("fp32", torch.complex64, 32), ("fp64", torch.complex128, 64)):
                if name == "fp64" and nr == 3:
                    continue
                x = torch.from_numpy(synth.spinor_rhs(nr, dims, 1)).to(dt).cuda()
                y = torch.empty_like(x)
                for _ in range(3):
                    slat.apply("MdagM", x, y, nr)
                reps = 10
                times = []
                for _ in range(reps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    slat.apply("MdagM", x, y, nr)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = float(np.median(times))
                # five passes: 13 spinor fields + 2 phi per site-RHS
                gbs = (13 * S + 2 * S // 4) * L ** 4 * nr / (ms / 1000.0) / 1e9
                row[name] = {"applies_per_s": nr / (ms / 1000.0), "ms": ms, "GB_s": gbs,
                             "frac_of_hbm": gbs / (PEAK_HBM or 6800.0)}
                tf = mdagm_flops_per_site(L ** 4) * L ** 4 * nr / (ms / 1000.0) / 1e12
                row[name]["alu_TFLOP_s"] = tf
                row[name]["frac_of_fma_peak"] = tf / (fp64_peak if name == "fp64" else fp32_peak)
                if name == "fp32":
                    kk = {}
                    for kind in ("zt", "xy"):
                        flush.zero_()
                        torch.cuda.synchronize()
                        wz.wz_probe_begin(kind, 4)
                        slat.apply("MdagM", x, y, nr)
                        kk[kind] = wz.wz_probe_end()
                    for kind, v in kernel_table(kk).items():
                        row[name][kind + "_per_launch"] = {
                            "launches": v["launches"], "avg_launch_us": v["avg_launch_us"],
                            "algorithmic_bytes_per_launch": v["algorithmic_bytes_per_launch"],
                            "GB_s": v["achieved_GB_s"],
                            "frac_of_hbm": v["achieved_GB_s"] / (PEAK_HBM or 6800.0) if v["achieved_GB_s"] else None}
            if "fp64" in row:
                row["fp32_over_fp64"] = row["fp32"]["applies_per_s"] / row["fp64"]["applies_per_s"]
            sweep.append(row)
            slat.close()

    # the mixed solve on a lattice whose working set is far beyond L2: 32^4,
    # 4 right-hand sides (5 FP32 fields of 128 MB plus the FP64 vectors), the
    # same couplings and tolerance as the 16^4 headline
    solve32 = None
    if not args.no_solve32:
        dims = (32, 32, 32, 32)
        l32 = wz.Lattice(dims, m=w.m, g=w.g, stream=stream.cuda_stream)
        l32.set_phi(torch.from_numpy(synth.scalar_field(dims, w.sigma, 0)).cuda())
        b32 = torch.from_numpy(synth.spinor_rhs(4, dims, 1)).cuda()
        x32 = torch.zeros_like(b32)
        l32.solve(b32, x32, tol=w.tol, mixed=True)  # warm-up: tuner and graph
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, st32, _ = l32.solve(b32, x32, tol=w.tol, mixed=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        n32 = st32["total_iterations"] + st32["reliable_updates"]
        gbs = n32 * 592.0 * 32 ** 4 / (ms / 1000.0) / 1e9
        solve32 = {"workload": f"32^4, m={w.m}, g={w.g}, phi sigma {w.sigma}, 4 complex-Gaussian RHS, mixed CG to "
                               f"{w.tol:g}", "ms_per_solve": ms, "applies_per_s": n32 / (ms / 1000.0),
                   "iterations_max": st32["iterations"], "max_true_residual": st32["max_true_residual"],
                   "cg_GB_s": gbs, "cg_frac_of_hbm": gbs / (PEAK_HBM or 6800.0),
                   "note": "592 B per site-RHS per CG iteration (18 FP32 spinor fields + 2 phi); working set "
                           "~0.9 GB, far beyond the 129 MB L2"}
        l32.close()

    # batched workload: 64 lattices (16 each of 4^4, 8^4, 12^4, 16^4), (m, g)
    # on an 8 x 8 grid, 8 right-hand sides each, one mixed solve to 1e-10
    batch = None
    if not args.no_batch:
        ws = synth.batch_workloads()
        bt = wz.Batch([dict(dims=x.dims, m=x.m, g=x.g) for x in ws])
        bs, xs = [], []
        for i, x in enumerate(ws):
            bt.set_phi(i, torch.from_numpy(synth.scalar_field(x.dims, x.sigma, 100 + i)).cuda())
            bs.append(torch.from_numpy(synth.spinor_rhs(x.nrhs, x.dims, 200 + i)).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        bt.solve(bs, xs, ws[0].nrhs, tol=1e-10)  # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bst = bt.solve(bs, xs, ws[0].nrhs, tol=1e-10)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        applies = bst["total_iterations"] + bst["reliable_updates"]
        site_rhs = sum(int(np.prod(x.dims)) * x.nrhs for x in ws)
        gbs = bst["site_applies"] * 592.0 / dt / 1e9
        batch = {"workload": "64 lattices: 16 each of 4^4, 8^4, 12^4, 16^4; m in linspace(0.02, 0.2, 8), "
                             "g in linspace(0.1, 1.0, 8); 8 RHS each; mixed CG to 1e-10",
                 "groups": bt.groups, "seconds": dt, "applies": applies, "applies_per_s": applies / dt,
                 "site_rhs_applies_per_s": bst["site_applies"] / dt,
                 "cg_GB_s": gbs, "cg_frac_of_hbm": gbs / (PEAK_HBM or 6800.0),
                 "max_iterations": bst["iterations"],
                 "max_true_residual": bst["max_true_residual"], "site_rhs": site_rhs}
        t0 = time.perf_counter()
        tst = bt.trajectory(tau=0.1, nsteps=2, npf=8, tol=1e-10, seed=7, traj_index=0)
        torch.cuda.synchronize()
        batch["short_trajectory"] = {"tau": 0.1, "nsteps": 2, "npf": 8, "seconds": time.perf_counter() - t0,
                                     "accepted": int(sum(x["accept"] for x in tst)),
                                     "cg_iterations": int(tst[0]["cg_iterations"])}
        bt.close()

    # end to end through the C ABI with pinned host buffers
    hb = torch.from_numpy(b).pin_memory()
    hx = torch.zeros_like(hb).pin_memory()
    e2e_t, e2e_n = 0.0, 0
    if not args.no_e2e:
        lat.solve(hb, hx, tol=w.tol, mixed=True)  # untimed: the context's staging buffer grows here once
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st, _ = lat.solve(hb, hx, tol=w.tol, mixed=True)
        e2e_t += time.perf_counter() - t0
        e2e_n += st["total_iterations"] + st["reliable_updates"]
    e2e = {"value": e2e_n / e2e_t if e2e_t > 0 else None, "unit": UNIT, "h2d_bytes_per_step": int(hb.numel() * hb.element_size()),
           "d2h_bytes_per_step": int(hx.numel() * hx.element_size())}

    peak = PEAK_HBM
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    kernels = kernel_table(probes)
    dom = args.probe if args.probe != "auto" else dominant_class(kernels)
    k = kernels[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": k["achieved_GB_s"], "peak": peak, "unit": "GB/s",
                "frac": k["achieved_GB_s"] / peak if k["achieved_GB_s"] else None, "peak_source": peak_src,
                "traffic": recorded_traffic(dom, probes[dom], k["algorithmic_bytes_per_launch"]),
                "launches": k["launches"], "timed_launches": k["timed_launches"],
                "avg_launch_us": k["avg_launch_us"],
                "algorithmic_bytes_per_launch": k["algorithmic_bytes_per_launch"],
                "note": "eager single-stream launches of one solve, CUDA events per launch; achieved = "
                        "algorithmic bytes / event time over the same (timed) launches"}
    kernels_full = kernel_table(probes_full)
    kf = kernels_full[dom] if dom in kernels_full else None
    roofline_full = None if kf is None else {
        "bound": "hbm", "kernel": dom, "achieved": kf["achieved_GB_s"], "peak": peak, "unit": "GB/s",
        "frac": kf["achieved_GB_s"] / peak if kf["achieved_GB_s"] else None,
        "avg_launch_us": kf["avg_launch_us"], "algorithmic_bytes_per_launch": kf["algorithmic_bytes_per_launch"],
        "note": f"the dominant class with one launch per pass covering all {w.nrhs} right-hand sides"}

    # the whole CG iteration against the same peak: per M^dag M apply of one RHS
    # the five passes move 18 FP32 spinor fields (P1 6, zt 2 + 2, P3 4, P5 4)
    # and phi twice (P3, P5), 18 * 32 + 2 * 8 = 592 B per site (tables not counted)
    it_bytes = 592.0 * int(np.prod(w.dims))
    solve_roofline = {"bound": "hbm", "bytes_per_apply": it_bytes, "achieved": value * it_bytes / 1e9,
                      "peak": peak, "unit": "GB/s", "frac": value * it_bytes / 1e9 / peak,
                      "note": "mixed solve, reliable updates included in the time, not in the bytes"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, n, dt = oracle_applies_per_s(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"FP64 oracle CG iterations on RHS 0 of {w.name}: {n} M^dag M applies in {dt:.1f} s"}
        one = oracle_sample_one_thread(args.cpu_seconds / 2)
        if one is not None:
            cpu["one_thread"] = {"value": one["value"], "cores": one["cores"],
                                 "sample": f"the same, BLAS/OpenMP limited to one thread: {one['applies']} "
                                           f"applies in {one['seconds']:.1f} s"}

    if rank == 0:
        it = [s["iterations"] for s in stats]
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config(w), parallelism=f"replicas x{world}"),
            "solve": {"iterations_max": max(it), "applies_per_step": total_applies / args.steps,
                      "max_true_residual": max(s["max_true_residual"] for s in stats)},
            "fp64": fp64, "hmc": hmc, "rhmc": rhmc, "one_loop": oneloop, "large": large, "apply_sweep": sweep, "solve_32x4": solve32, "paper_solver_table": invtab, "paper_fft_table": ffttab,
            "fma_peak_TFLOP_s": {"fp64": fp64_peak, "fp32": fp32_peak}, "batch": batch, "kernels": kernels, "kernels_full_launch": kernels_full, "e2e": e2e, "roofline": roofline,
            "roofline_full_launch": roofline_full, "solve_roofline": solve_roofline, "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": int(launches),
            "hmc_traj_per_s": None if hmc is None else {
                "single_mixed": hmc["single_mixed"]["traj_per_s"], "single_fp64": hmc["single_fp64"]["traj_per_s"],
                f"batch{args.hmc_replicas}_mixed": hmc[f"batch{args.hmc_replicas}_mixed"]["traj_per_s"],
                f"batch{args.hmc_replicas}_fp64": hmc[f"batch{args.hmc_replicas}_fp64"]["traj_per_s"],
                "batched_mixed_over_single_fp64": hmc["batched_mixed_over_single_fp64"],
                "batched_mixed_cg_frac_of_hbm": hmc[f"batch{args.hmc_replicas}_mixed"]["cg_frac_of_hbm"],
                "single_mixed_cg_frac_of_hbm": hmc["single_mixed"]["cg_frac_of_hbm"],
                "workload": hmc["workload"]},
        }))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
