"""Apply one operator of the library repeatedly, or run a bounded mixed CG
solve, for profiling a pass in isolation.

Usage (a CUDA device and the built libwz.so are required):

    python -m paper_1005_3276_gb300.profile_apply --dims 16 16 16 16 --nrhs 16 --op MdagM --dtype c64 --reps 3
    WZ_NO_GRAPHS=1 python -m paper_1005_3276_gb300.profile_apply --nrhs 12 --solve-iters 24

With --solve-iters N the script runs one mixed-precision solve of (M^dag M) x = b
for the right-hand sides, stopped after N iterations (the CG passes of the
solver; WZ_NO_GRAPHS=1 makes them separate launches a profiler can capture).

Fields are seeded synthetic inputs (phi Gaussian sigma 0.5, right-hand sides
unit complex Gaussian), m = 0.05, g = 0.3.  Each repetition is one call of the
operator through the C ABI; the script prints the mean event time per call.
Run it under a profiler with a kernel filter (e.g. ncu -k regex:zt_pass) to
capture single launches of one pass.
"""

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16], help="T Z Y X")
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--op", default="MdagM")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--solve-iters", type=int, default=0, help="run a mixed CG solve stopped after N iterations")
    args = ap.parse_args()

    import torch

    from . import binding as wz
    from . import synth

    dims = tuple(args.dims)
    dt = torch.complex64 if args.dtype == "c64" else torch.complex128
    lat = wz.Lattice(dims, m=0.05, g=0.3)
    lat.set_phi(torch.from_numpy(synth.scalar_field(dims, 0.5, 0)).cuda())
    if args.solve_iters > 0:
        b = torch.from_numpy(synth.spinor_rhs(args.nrhs, dims, 1)).cuda()
        xs = torch.zeros_like(b)
        stream = torch.cuda.current_stream()
        times = []
        for _ in range(max(1, args.reps)):
            xs.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, st, _ = lat.solve(b, xs, tol=1e-10, maxiter=args.solve_iters, mixed=True,
                                  raise_on_nonconvergence=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        n = st["total_iterations"] + st["reliable_updates"]
        print(f"solve {dims} x {args.nrhs}: {st['iterations']} iterations, status {rc}, "
              f"{min(times):.2f} ms (best of {len(times)}), {n / (min(times) / 1000.0):.0f} applies/s")
        lat.close()
        return
    x = torch.from_numpy(synth.spinor_rhs(args.nrhs, dims, 1)).to(dt).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    lat.apply(args.op, x, y, args.nrhs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        lat.apply(args.op, x, y, args.nrhs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    finite = bool(torch.isfinite(torch.view_as_real(y)).all())
    print(f"{args.op} {dims} x {args.nrhs} {args.dtype}: {ms:.4f} ms per call, finite={finite}")
    lat.close()
    if not finite:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
