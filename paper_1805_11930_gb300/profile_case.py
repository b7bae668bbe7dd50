"""Small, fixed launch sequence of one kernel family, for ncu captures.

python -m paper_1805_11930_gb300.profile_case --what apply|block|smooth --prec fp64|fp32 [--n 48] [--p 4]
    [--inner pcg|gmres|direct] [--wpb-apply W] [--wpb-smooth W] [--layout auto|line|element|plane]
    [--advection]

Sets up the log-normal diffusion workload on an n^3 mesh (48^3 at p = 4 is
13.8 M dofs, 110 MB per FP64 vector: larger than L2, a few hundred MB in
total), runs two warm-up launches and then `--reps` launches of the chosen
operation through the C ABI.  Prints the median CUDA-event time per launch.
--inner direct times the smoother with the stored block inverses (built
before the warm-up); --wpb-* set the launch shapes (warps per block) so that
a capture can use the shapes the benchmark's autotuning picked; --layout
sets the work layout of both kernels.  --advection takes the convection
workload instead (rotating b, kappa = 1e-3, Dirichlet) on the same mesh;
its smoother wants --inner gmres.
"""
import argparse
import statistics
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", default="apply", choices=["apply", "block", "smooth"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--inner", default="pcg", choices=["pcg", "gmres", "direct"])
    ap.add_argument("--wpb-apply", type=int, default=0)
    ap.add_argument("--wpb-smooth", type=int, default=0)
    ap.add_argument("--layout", default="auto", choices=["auto", "line", "element", "plane"])
    ap.add_argument("--advection", action="store_true")
    args = ap.parse_args()

    import torch

    from . import dgmg, inputs
    w = inputs.convection(args.n, args.p) if args.advection else inputs.lognormal(args.n, args.p)
    ctx = dgmg.Context(0)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    nd = ctx.sizes()["ndof"]
    prec = dgmg.FP64 if args.prec == "fp64" else dgmg.FP32
    ctx.set_launch_shape(prec, args.wpb_apply, args.wpb_smooth)
    lay = {"auto": dgmg.LAYOUT_AUTO, "line": dgmg.LAYOUT_LINE, "element": dgmg.LAYOUT_ELEMENT,
           "plane": dgmg.LAYOUT_PLANE}[args.layout]
    ctx.set_layout(prec, lay, lay)
    inner = {"pcg": dgmg.INNER_PCG, "gmres": dgmg.INNER_GMRES, "direct": dgmg.INNER_DIRECT}[args.inner]
    if inner == dgmg.INNER_DIRECT:
        ctx.block_inverse(prec)
    dt = torch.float64 if args.prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(1805)
    x = torch.rand(nd, dtype=dt, device="cuda", generator=g)
    y = torch.rand(nd, dtype=dt, device="cuda", generator=g)
    stream = torch.cuda.current_stream()

    def op():
        if args.what == "apply":
            ctx.apply(x, y)
        elif args.what == "block":
            ctx.block_apply(x, y)
        else:
            ctx.block_smooth(x, y, nsweep=1, omega=0.8, eps=1e-2, inner=inner)

    for _ in range(2):
        op()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    print(f"{args.what} {args.prec} {args.inner} {args.layout} n={args.n} p={args.p} ndof={nd}: median {statistics.median(ms):.4f} ms "
          f"({nd / statistics.median(ms) / 1e6:.3f} GDOF/s)")
    sys.stdout.flush()


if __name__ == "__main__":
    main()
