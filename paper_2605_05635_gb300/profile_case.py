"""Runs one fixed tracing case a few times, for profiling a kernel in
isolation (``ncu ... python -m paper_2605_05635_gb300.profile_case``).

Cases: ``kerr128`` (Kerr a = 0.5, i = 17 deg, 128^2 over [-10, 10]^2, no
refinement), ``sweep512`` (one 512^2 image of the six-image sweep, with
refinement) and ``sweep512l0`` (the same image without refinement, so that
the first trace launch carries all of the run's base rays).  The integrator
settings are those of the chosen precision's sweep.  ``shadow512`` brackets
the Fig. 5 cored-NFW shadow boundary along 512 directions to 1e-10 (FP64);
``scan64k`` classifies 65,536 spacetimes of the Figs. 3-4 grids with 16
angles.
"""
import argparse
import math
import sys

import torch

from . import bhrt, workloads


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="kerr128",
                    choices=["kerr128", "sweep512", "sweep512l0", "shadow512", "scan64k"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args(argv)
    if a.case == "shadow512":
        flats, psi, lo, hi, tol = workloads.shadow_fig5(512)
        st, cam, _, it = bhrt.from_flat(flats[2])
        for _ in range(a.repeat):
            b_in, b_out, fl = bhrt.shadow_boundary(st, cam, it, psi, lo, hi, tol)
        torch.cuda.synchronize()
        print(f"case shadow512: {int((fl != 0).sum())} flagged, mean b "
              f"{float((b_in + b_out).mean() / 2):.9f}")
        return 0
    if a.case == "scan64k":
        metric, chi, lam_E, eta, lam_c, theta = workloads.geometry_grid(256)
        sts = [bhrt.Spacetime(metric=int(metric[i]), chi=float(chi[i]),
                              lambda_E=float(lam_E[i]), eta=float(eta[i]),
                              lambda_c=float(lam_c[i])) for i in range(0, metric.shape[0], 2)]
        arr = bhrt.spacetime_array(sts)
        for _ in range(a.repeat):
            res = bhrt.geometry_scan(arr, theta)
        torch.cuda.synchronize()
        print(f"case scan64k: {len(sts)} spacetimes, {int((res['flags'] == 0).sum())} black holes")
        return 0
    prec = bhrt.FP64 if a.precision == "fp64" else bhrt.MIXED
    integ = workloads.FP64_INTEG if prec == bhrt.FP64 else workloads.MIXED_INTEG
    if a.case == "kerr128":
        flat = dict(workloads.kerr_64(), nx=128, ny=128, **integ)
    else:
        flat = dict(workloads.sweep_512()[0], **integ)
        if a.case == "sweep512l0":
            flat["levels"] = 0
    items = [bhrt.from_flat(flat)]
    plan = bhrt.Plan(items)
    for _ in range(a.repeat):
        plan.launch()
    torch.cuda.synchronize()
    plan.check()
    st = plan.stats()
    print(f"case {a.case} {a.precision} (last launch): rays {sum(st['rays'])} accepted fp32 "
          f"{st['accepted_fp32']} rejected fp32 {st['rejected_fp32']} fp64 "
          f"{st['accepted_fp64']} rejected fp64 {st['rejected_fp64']} promoted "
          f"{st['promoted_rays']} lane utilisation fp32 {st['lane_util_fp32']:.3f} "
          f"fp64 {st['lane_util_fp64']:.3f}")
    plan.close()


if __name__ == "__main__":
    sys.exit(main())
