"""Operator-apply throughput over the polynomial degree.

python -m paper_1805_11930_gb300.apply_sweep [--degrees 2,3,4,5,6] [--advection]
    [--layout auto|line|element|plane]

Meshes sized to 30-300 MB per FP64 vector: 64^3 cells for p <= 3, 40^3 for
p = 4..6 (log-normal K, Dirichlet).  For each p and precision: median
CUDA-event time of dgmg_apply over 20 launches (an L2-sized buffer is
written between launches), GDOF/s, the rate of the flops the kernel issues
(flops.kernel_apply_full for the work layout the operator ran in: the
element layout's factored or Gauss-point form, or the line form; the
automatic choice unless --layout names one) as a fraction of the FP64 pipe peak
(4 flop/clk/SM x 152 SMs x 2070 MHz; for df64, FP64 vectors in double-float
arithmetic, as well) or of the measured FP32 FMA rate (75.6 TFLOP/s), the
same for the algorithmic count (32 n^4 + 120 n^3 flop per cell), and the HBM
rate of the compulsory traffic (read u, write v) as a fraction of the
measured copy bandwidth.  One JSON line per (p, precision).

--advection: the advection-on variant (the rotating field b of the
convection workload, kappa = 1e-3), whose volume term carries the value
terms (algorithmic 36 n^4 + 120 n^3 per cell), in FP64 and FP32 (the
double-float kernels cover b = 0 only).
"""
import argparse
import json
import statistics

FP64_PEAK = 152 * 4 * 2070e6
FP32_PEAK = 75.6e12
HBM_GBS = 6686.8


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--degrees", default="2,3,4,5,6")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--advection", action="store_true")
    ap.add_argument("--layout", default="auto", choices=["auto", "line", "element", "plane"])
    args = ap.parse_args()
    import torch

    from . import dgmg, flops, inputs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for p in [int(x) for x in args.degrees.split(",")]:
        n = 64 if p <= 3 else 40
        w = inputs.convection(n, p) if args.advection else inputs.lognormal(n, p)
        ctx = dgmg.Context(0)
        ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
        ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
        s = ctx.sizes()
        variants = [(torch.float64, "fp64", FP64_PEAK, dgmg.FP64), (torch.float32, "fp32", FP32_PEAK, dgmg.FP32),
                    (torch.float64, "df64", FP64_PEAK, dgmg.DF64)]
        for dt, name, peak, prec in variants:
            if args.advection and prec == dgmg.DF64:
                continue
            if args.layout != "auto":
                lay = getattr(dgmg, "LAYOUT_" + args.layout.upper())
                try:
                    ctx.set_layout(prec, lay, lay)
                except dgmg.DgmgError:
                    continue
            layout = dgmg.LAYOUT_NAMES[ctx.get_layout(prec)[0]]
            x = torch.rand(s["ndof"], dtype=dt, device="cuda")
            y = torch.empty_like(x)
            df = name == "df64"
            for _ in range(3):
                ctx.apply(x, y, df64=df)
            ms = []
            for _ in range(args.reps):
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                ctx.apply(x, y, df64=df)
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms) / 1e3
            fl = flops.algorithmic_apply(p + 1, value_terms=args.advection) * s["ncell"] / t
            kfl = flops.kernel_apply_full(p + 1, advection=args.advection,
                                          element=layout == "element") * s["ncell"] / t
            by = flops.hbm_bytes_apply(p + 1, s["ncell"], 4 if name == "fp32" else 8) / t
            print(json.dumps({"p": p, "mesh": n, "ndof": s["ndof"], "prec": name, "advection": args.advection,
                              "layout": layout,
                              "ms": round(t * 1e3, 4),
                              "gdofs": round(s["ndof"] / t / 1e9, 3), "tflops": round(kfl / 1e12, 3),
                              "alu_frac": round(kfl / peak, 3), "alu_frac_generic_count": round(fl / peak, 3),
                              "hbm_gbs": round(by / 1e9, 1),
                              "hbm_frac": round(by / 1e9 / HBM_GBS, 4)}), flush=True)
        ctx.close()


if __name__ == "__main__":
    main()
