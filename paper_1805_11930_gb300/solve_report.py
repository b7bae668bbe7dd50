"""Time-to-solution report for the synthetic workloads.

python -m paper_1805_11930_gb300.solve_report [--workloads poisson,lognormal,lognormal_p6,convection,reservoir,convection_pe2000,variable_k] [--repeat 3]

For each workload: set-up time (coefficients, diag(D_T), Q1 matrix, AMG),
then the solve to a 1e-8 relative residual from u = 0: in FP64; with the
mixed-precision V-cycle (FP32 smoother, inner solves and residual; FP64 outer
Krylov, dots, coarse solve and final residual check); and with the V-cycle and
the outer operator in double-float arithmetic on FP64 vectors (the final
residual check stays FP64); also with exact block solves by the stored block
inverses (inner = DIRECT, FP64 and mixed; the inverse set-up time is
reported separately; lognormal_p6 runs them at p = 6); the reservoir workload also with the P0 coarse
space (the paper's choice for SPE10); the grid-Peclet-2000 convection
workload (Sec. 4.3) with the paper's set-up: FGMRES preconditioned by two
multicolour block-SSOR sweeps and no coarse correction, inner GMRES with the
tridiagonal (Thomas) preconditioner; the inhomogeneous test of Sec. 4.2 with
K(x), c(x) at the quadrature points in the outer operator and cell-centre
values in the V-cycle.  Reports the median
solve time over --repeat runs (CUDA events, inputs resident), outer
iterations, mean / max inner iterations, the recomputed FP64 residual, the
difference between the mixed and FP64 solutions and, where the workload has
an exact solution, the max nodal error.  One JSON line per workload.
"""
import argparse
import json
import statistics
import time


def run(name, repeat):
    import numpy as np
    import torch

    from . import dgmg, inputs
    extra = {}
    if name == "poisson":
        w, kry, inner = inputs.poisson_sine(8, 2), dgmg.KRYLOV_CG, dgmg.INNER_PCG
    elif name == "lognormal":
        w, kry, inner = inputs.lognormal(32, 4), dgmg.KRYLOV_CG, dgmg.INNER_PCG
    elif name == "lognormal_p6":
        # the paper's highest order in its set-up table (App. B): stored
        # inverses of 343 x 343 blocks by the panel-blocked elimination
        w, kry, inner = inputs.lognormal(12, 6), dgmg.KRYLOV_CG, dgmg.INNER_PCG
    elif name == "convection":
        # block-SSOR smoother (the paper's choice for convection) + AMG
        w, kry, inner = inputs.convection(64, 3), dgmg.KRYLOV_FGMRES, dgmg.INNER_GMRES
        extra = dict(smoother=dgmg.SMOOTHER_SSOR)
    elif name == "reservoir":
        # high-contrast anisotropic K: three AMG cycles per coarse correction
        w, kry, inner = inputs.reservoir(), dgmg.KRYLOV_CG, dgmg.INNER_PCG
        extra = dict(coarse_cycles=3)
    elif name == "variable_k":
        # K(x), c(x) at the quadrature points in the outer operator, cell-centre values in the V-cycle
        w, kry, inner = inputs.variable_k(32, 3), dgmg.KRYLOV_CG, dgmg.INNER_PCG
    elif name == "convection_pe2000":
        w, kry, inner = inputs.convection_pe(32, 3), dgmg.KRYLOV_FGMRES, dgmg.INNER_GMRES_TRIDIAG
        extra = dict(smoother=dgmg.SMOOTHER_SSOR, coarse=dgmg.COARSE_NONE)
    else:
        raise ValueError(name)
    t0 = time.perf_counter()
    ctx = dgmg.Context(0)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    if "vark" in w:
        vk = w["vark"]
        ctx.set_variable_coefficients(vk["basis"], vk["p0"], vk["p2"], vk["gamma"])
    else:
        ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    vol, face = ctx.quadrature_points()
    s = ctx.sizes()
    f = torch.empty(s["ndof"], dtype=torch.float64, device="cuda")
    ctx.assemble_rhs(inputs.evaluate(w["f"], vol), f, g_qp=inputs.evaluate(w["g"], face),
                     j_qp=inputs.evaluate(w["j"], face))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = {"workload": w["name"], "ndof": s["ndof"], "setup_s": round(setup_s, 3)}
    flex = dgmg.KRYLOV_FCG if kry == dgmg.KRYLOV_CG else kry
    sols = {}
    variants = [("fp64", dgmg.default_opts(krylov=kry, inner=inner, maxit=1000, **extra)),
                ("mixed", dgmg.default_opts(krylov=flex, inner=inner, smoother_prec=dgmg.FP32, maxit=1000,
                                            **extra))]
    if w["b"] is None and "vark" not in w:   # the double-float kernels cover diffusion
        variants.append(("df64", dgmg.default_opts(krylov=flex, inner=inner, smoother_prec=dgmg.DF64,
                                                   apply_prec=dgmg.DF64, maxit=1000, **extra)))
    if name == "reservoir":  # the piecewise-constant coarse space of the paper's SPE10 runs
        variants.append(("fp64_p0", dgmg.default_opts(krylov=kry, inner=inner, maxit=1000, coarse=dgmg.COARSE_P0,
                                                      coarse_cycles=3)))
        variants.append(("mixed_p0", dgmg.default_opts(krylov=flex, inner=inner, smoother_prec=dgmg.FP32,
                                                       maxit=1000, coarse=dgmg.COARSE_P0, coarse_cycles=3)))
    # stored block inverses (partially matrix-free smoother)
    t1 = time.perf_counter()
    ctx.block_inverse(dgmg.FP64)
    ctx.block_inverse(dgmg.FP32)
    out["block_inverse_setup_s"] = round(time.perf_counter() - t1, 3)
    variants.append(("fp64_direct", dgmg.default_opts(krylov=kry, inner=dgmg.INNER_DIRECT, maxit=1000, **extra)))
    variants.append(("mixed_direct", dgmg.default_opts(krylov=flex, inner=dgmg.INNER_DIRECT,
                                                       smoother_prec=dgmg.FP32, maxit=1000, **extra)))
    if w["b"] is None and "vark" not in w:
        variants.append(("df64_direct", dgmg.default_opts(krylov=flex, inner=dgmg.INNER_DIRECT,
                                                          smoother_prec=dgmg.DF64, apply_prec=dgmg.DF64,
                                                          maxit=1000, **extra)))
    for tag, opts in variants:
        u = torch.zeros_like(f)
        ms, st = [], None
        for _ in range(repeat):
            u.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            st = ctx.solve(f, u, opts, check=False)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        sols[tag] = u.clone()
        out[tag] = {"solve_s": round(statistics.median(ms) / 1e3, 4), "status": st["status"],
                    "iterations": st["iterations"], "rel_residual": st["rel_residual"],
                    "inner_mean": round(st["inner_mean"], 2), "inner_std": round(st["inner_std"], 2),
                    "inner_max": st["inner_max"],
                    "us_per_dof": round(statistics.median(ms) * 1e3 / s["ndof"], 5)}
    for tag in [t for t in sols if t != "fp64"]:
        d = (sols[tag] - sols["fp64"]).norm() / sols["fp64"].norm()
        out[f"{tag}_vs_fp64_rel_diff"] = float(d)
    if w["exact"] is not None:
        # exact solution at the GLL nodes (end points and roots of P_p')
        gll = np.polynomial.legendre.Legendre.basis(w["p"]).deriv().roots()
        z = np.sort(np.concatenate(([-1.0], np.real(gll), [1.0])))
        z = 0.5 * (z + 1.0)
        nx, ny, nz = w["nc"]
        h = np.array(w["L"]) / np.array(w["nc"])
        n = w["p"] + 1
        i3, i2, i1 = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        X = (cx.reshape(-1, 1) + z[i1.reshape(1, -1)]) * h[0]
        Y = (cy.reshape(-1, 1) + z[i2.reshape(1, -1)]) * h[1]
        Z = (cz.reshape(-1, 1) + z[i3.reshape(1, -1)]) * h[2]
        ue = w["exact"](X, Y, Z).reshape(-1)
        for tag in sols:
            out[tag]["max_nodal_error"] = float(np.abs(sols[tag].cpu().numpy() - ue).max())
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads",
                    default="poisson,lognormal,lognormal_p6,convection,reservoir,convection_pe2000,variable_k")
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args()
    for name in args.workloads.split(","):
        print(json.dumps(run(name, args.repeat)), flush=True)


if __name__ == "__main__":
    main()
