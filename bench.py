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

Extra keys: the same solve in FP64 throughout (the baseline the mixed path
must beat), "e2e" through the C ABI with host buffers, a roofline of the
dominant kernel from the library's event probe, the FP64 CPU oracle timed on
a bounded sample, SM clocks sampled during the timed region, and the count of
library kernels launched in the timed region.

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
UNIT = "M^dag M applies/s"


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
    ap.add_argument("--no-hmc", action="store_true", help="skip the HMC trajectory timing")
    ap.add_argument("--hmc-traj", type=int, default=2, help="timed trajectories per precision")
    ap.add_argument("--no-sweep", action="store_true", help="skip the L = 8, 16, 32 apply sweep")
    ap.add_argument("--batch", action="store_true", help="also time the 64-lattice batched workload")
    ap.add_argument("--no-rhmc", action="store_true", help="skip the rational heatbath / RHMC timings")
    ap.add_argument("--no-oneloop", action="store_true", help="skip the one-loop lattice sums (Sec. 5 tables)")
    ap.add_argument("--large", action="store_true",
                    help="also time the 32^4 large-lattice pieces (force evaluation, Ward identity, <F>, "
                         "supercurrent correlators)")
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
PROBE_CLASSES = (("zt", 4), ("cg_p1", 4), ("cg_p3", 4), ("cg_p5", 4), ("zt", 8), ("ru_p1", 8), ("ru_p5", 8))


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
        "data": "synthetic", "config": workload_config(w),
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

    t_max, applies_all = combine_ranks(dist, total_ms, total_applies, "cuda")
    value = applies_all / (t_max / 1000.0)

    # FP64 throughout, same workload (one solve)
    fp64 = None
    if not args.no_fp64:
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n64, st64 = solve(mixed=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": n64 / (ms64 / 1000.0), "unit": UNIT, "ms_per_solve": ms64,
                "iterations": st64["iterations"], "max_true_residual": st64["max_true_residual"],
                "mixed_speedup_per_solve": ms64 / (total_ms / args.steps)}

    # HMC trajectories/s on the differentiation workload (16^4, m = 0.1, g = 0.5,
    # one pseudofermion, tau = 1, 20 leapfrog steps), mixed and FP64 solves
    hmc = None
    if not args.no_hmc:
        hw = synth.FORCE_16
        hlat = wz.Lattice(hw.dims, m=hw.m, g=hw.g, stream=stream.cuda_stream)
        hmc = {"workload": f"{hw.name}: 16^4, m={hw.m}, g={hw.g}, phi sigma {hw.sigma}, 1 pseudofermion, "
                           f"tau={hw.extra['tau']}, {hw.extra['nsteps']} leapfrog steps, CG to 1e-10"}
        for label, flags in (("mixed", 0), ("fp64", wz.WZ_HMC_FP64_SOLVES)):
            hlat.set_phi(torch.from_numpy(synth.scalar_field(hw.dims, hw.sigma, 0)).cuda())
            kw = dict(tau=hw.extra["tau"], nsteps=hw.extra["nsteps"], npf=1, tol=1e-10, seed=2024, flags=flags)
            hlat.trajectory(traj_index=0, **kw)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sts = []
            e0.record(stream)
            for t in range(args.hmc_traj):
                sts.append(hlat.trajectory(traj_index=1 + t, **kw))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            hmc[label] = {"traj_per_s": args.hmc_traj / (ms / 1000.0), "ms_per_traj": ms / args.hmc_traj,
                          "cg_iterations_per_traj": float(np.mean([x["cg_iterations"] for x in sts])),
                          "dH": [round(x["dH"], 5) for x in sts], "accept": [x["accept"] for x in sts]}
        hmc["mixed_speedup"] = hmc["fp64"]["ms_per_traj"] / hmc["mixed"]["ms_per_traj"]
        # the CG iterations of a trajectory as a whole-iteration HBM figure: one
        # FP32 (FP64) iteration moves 18 spinor fields and phi twice per site
        V = int(np.prod(hw.dims))
        for label, bps in (("mixed", 18 * 32 + 2 * 8), ("fp64", 18 * 64 + 2 * 16)):
            h = hmc[label]
            h["cg_bytes_per_site_iteration"] = bps
            h["cg_GB_s"] = h["cg_iterations_per_traj"] * bps * V / (h["ms_per_traj"] / 1000.0) / 1e9
        hlat.close()

    # rational heatbath eta = (M^dag M)^1/8 R of the paper's heatbath table: L^3 x 32,
    # m = 1, g = 0.1, degree 20, poles beta <= 100 preconditioned by M0^-1; the
    # interval is the free spectrum widened by 2 on both ends.  Then RHMC
    # trajectories (r_a ~ x^-1/4, r_h ~ x^1/8, degree 20) on the HMC workload.
    rhmc = None
    if not args.no_rhmc:
        rhmc = {"heatbath": [], "paper_gtx285": {"8^3x32": {"single_s": 0.93, "single_iters": 360, "double_s": 3.5,
                                                           "double_iters": 700},
                                                "16^3x32": {"single_s": 4.8, "single_iters": 370, "double_s": 20,
                                                            "double_iters": 730}}}
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
                row[label] = {"seconds": e0.elapsed_time(e1) / 1000.0, "total_iterations": st["total_iterations"],
                              "max_iterations": st["iterations"], "reliable_updates": st["reliable_updates"]}
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

    # large single lattice: 32^4, m = 0.02, g = 1.0, hot start sigma 1, 4 pseudofermions.
    # A whole trajectory (Omelyan, 40 steps = 81 force evaluations) is minutes; the
    # pieces of one are timed: a force evaluation with its 4-RHS mixed solve, the
    # Ward-identity measurement (4 uniform-source solves), <F> and the supercurrent
    # correlators on a Gaussian noise source (4 solves).
    large = None
    if args.large:
        lw = synth.LARGE_32
        ll = wz.Lattice(lw.dims, m=lw.m, g=lw.g, stream=stream.cuda_stream)
        ll.set_phi(torch.from_numpy(synth.scalar_field(lw.dims, lw.sigma, 0)).cuda())
        eta = torch.from_numpy(synth.spinor_rhs(lw.nrhs, lw.dims, 1)).cuda()
        G = torch.zeros(lw.dims, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sb, spf, fst = ll.force(eta, G, tol=1e-10)
        torch.cuda.synchronize()
        t_force = time.perf_counter() - t0
        t0 = time.perf_counter()
        WR, WL, wst = ll.ward_identity(tol=1e-10, mixed=True)
        t_ward = time.perf_counter() - t0
        t0 = time.perf_counter()
        F = ll.aux_vev()
        t_aux = time.perf_counter() - t0
        # supercurrent correlators on one Gaussian noise source, E[w w^*] = 1 per site
        wsrc = torch.from_numpy(synth.scalar_field(lw.dims, np.sqrt(0.5), 2)).cuda()
        t0 = time.perf_counter()
        Rsc, sst = ll.supercurrent(wsrc, tol=1e-10, mixed=True)
        t_sc = time.perf_counter() - t0
        large = {"workload": f"{lw.name}: 32^4, m={lw.m}, g={lw.g}, phi sigma {lw.sigma}, {lw.nrhs} pseudofermions, "
                             "mixed CG to 1e-10",
                 "force_eval_s": t_force, "force_cg_iterations_max": fst["iterations"],
                 "force_cg_iterations_total": fst["total_iterations"],
                 "ward_s": t_ward, "ward_cg_iterations_max": wst["iterations"],
                 "ward_R_trace": [float(np.trace(WR).real), float(np.trace(WR).imag)],
                 "ward_L_00_01": [float(WL[0, 1].real), float(WL[0, 1].imag)],
                 "aux_vev": [F.real, F.imag], "aux_s": t_aux,
                 "supercurrent_s": t_sc, "supercurrent_cg_iterations_max": sst["iterations"],
                 "supercurrent_R0_mu0_dx1_dy0_trace": [float(np.trace(Rsc[0, 0, 1, 0]).real),
                                                       float(np.trace(Rsc[0, 0, 1, 0]).imag)]}
        ll.close()

    # apply-throughput sweep: (M^dag M) on L^4, FP32 vs FP64 fields, about 1M
    # site-RHS per launch sequence (256 / 16 / 1 right-hand sides at L = 8/16/32)
    sweep = None
    if not args.no_sweep:
        sweep = []
        for L in (8, 16, 32):
            dims = (L, L, L, L)
            nr = max(1, (1 << 20) // (L ** 4))
            slat = wz.Lattice(dims, m=w.m, g=w.g, stream=stream.cuda_stream)
            slat.set_phi(torch.from_numpy(synth.scalar_field(dims, w.sigma, 0)).cuda())
            row = {"L": L, "nrhs": nr}
            for name, dt, S in (("fp32", torch.complex64, 32), ("fp64", torch.complex128, 64)):
                x = torch.from_numpy(synth.spinor_rhs(nr, dims, 1)).to(dt).cuda()
                y = torch.empty_like(x)
                for _ in range(3):
                    slat.apply("MdagM", x, y, nr)
                reps = 10
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    slat.apply("MdagM", x, y, nr)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                # five passes: 13 spinor fields + 2 phi per site-RHS
                gbs = (13 * S + 2 * S // 4) * L ** 4 * nr / (ms / 1000.0) / 1e9
                row[name] = {"applies_per_s": nr / (ms / 1000.0), "ms": ms, "GB_s": gbs}
            row["fp32_over_fp64"] = row["fp32"]["applies_per_s"] / row["fp64"]["applies_per_s"]
            sweep.append(row)
            slat.close()

    # batched workload: 64 lattices (16 each of 4^4, 8^4, 12^4, 16^4), (m, g)
    # on an 8 x 8 grid, 8 right-hand sides each, one mixed solve to 1e-10
    batch = None
    if args.batch:
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
        batch = {"workload": "64 lattices: 16 each of 4^4, 8^4, 12^4, 16^4; m in linspace(0.02, 0.2, 8), "
                             "g in linspace(0.1, 1.0, 8); 8 RHS each; mixed CG to 1e-10",
                 "groups": bt.groups, "seconds": dt, "applies": applies, "applies_per_s": applies / dt,
                 "site_rhs_applies_per_s": None, "max_iterations": bst["iterations"],
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
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st, _ = lat.solve(hb, hx, tol=w.tol, mixed=True)
        e2e_t += time.perf_counter() - t0
        e2e_n += st["total_iterations"] + st["reliable_updates"]
    e2e = {"value": e2e_n / e2e_t if e2e_t > 0 else None, "unit": UNIT, "h2d_bytes_per_step": int(hb.numel() * hb.element_size()),
           "d2h_bytes_per_step": int(hx.numel() * hx.element_size())}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
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

    if rank == 0:
        it = [s["iterations"] for s in stats]
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config(w), parallelism=f"replicas x{world}"),
            "solve": {"iterations_max": max(it), "applies_per_step": total_applies / args.steps,
                      "max_true_residual": max(s["max_true_residual"] for s in stats)},
            "fp64": fp64, "hmc": hmc, "rhmc": rhmc, "one_loop": oneloop, "large": large, "apply_sweep": sweep, "batch": batch, "kernels": kernels, "e2e": e2e, "roofline": roofline, "solve_roofline": solve_roofline, "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": int(launches),
            "hmc_traj_per_s": None if hmc is None else {
                "mixed": hmc["mixed"]["traj_per_s"], "fp64": hmc["fp64"]["traj_per_s"],
                "mixed_over_fp64": hmc["mixed_speedup"],
                "mixed_cg_frac_of_hbm": hmc["mixed"]["cg_GB_s"] / peak, "workload": hmc["workload"]},
        }))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
