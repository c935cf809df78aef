"""Small, self-contained launches of one kernel for profiling (ncu) runs.

  python -m paper_2004_04817_gb300.profile_case volume [--nv N] [--reps R]
  python -m paper_2004_04817_gb300.profile_case greedy [--m M] [--prec 32|64]
  python -m paper_2004_04817_gb300.profile_case solve
  python -m paper_2004_04817_gb300.profile_case cull [--nv N] [--vprec 32|48] [--radius R]
  python -m paper_2004_04817_gb300.profile_case modal [--nv N] [--modal-mode 1|2|3] [--n-out K]

Each case builds the GCB wing workload (N_b = 50,000), runs the calls once
untimed, then `--reps` more times, and exits 0.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["volume", "greedy", "solve", "cull", "modal"])
    ap.add_argument("--nv", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=241)
    ap.add_argument("--prec", type=int, default=48)
    ap.add_argument("--vprec", type=int, default=32)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--radius", type=float, default=0.25, help="cull: support radius")
    ap.add_argument("--modal-mode", type=int, default=3, choices=[1, 2, 3],
                    help="modal: 1 BF16, 2 FP16x2, 3 BF16x3")
    ap.add_argument("--n-out", type=int, default=96, help="modal: columns of W")
    a = ap.parse_args()
    c = synth.wing_gcb(n_vol=a.nv if a.case in ("volume", "cull", "modal") else 0)
    dev = lambda x, t=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=t,
                                                      device="cuda")
    xb, db = dev(c["xb"]), dev(c["db"])
    for _ in range(1 + a.reps):
        g = P.greedy_select(xb, db, radius=c["radius"], tol=c["tol_rel"], tol_mode=1,
                            m=a.m if a.case == "greedy" else 241, seed=1,
                            eval_prec=a.prec)
        if a.case == "greedy":
            continue
        if a.case == "cull":
            # the selected set's weights at the smaller radius; culled sum
            w, _ = P.solve_weights(xb, db, g["idx"], radius=a.radius)
            plan = P.VolumePlan(dev(c["xv"]), radius=a.radius, eval_prec=a.vprec,
                                nc_max=g["nc"])
            plan.run(xb, g["idx"], w)
            del plan
            continue
        if a.case == "modal":
            # random modal weights (N_c x n_out): the timing does not depend
            # on their values
            W = torch.randn((g["nc"], a.n_out), dtype=torch.float64, device="cuda",
                            generator=torch.Generator("cuda").manual_seed(1))
            P.deform_modal(dev(c["xv"]), xb, g["idx"], W, radius=c["radius"],
                           mode=a.modal_mode)
            continue
        w, _ = P.solve_weights(xb, db, g["idx"], radius=c["radius"])
        if a.case == "volume":
            P.deform_volume(dev(c["xv"]), xb, g["idx"], w, radius=c["radius"],
                            eval_prec=a.vprec)
    torch.cuda.synchronize()
    print("profile case done", a.case, g["nc"])


if __name__ == "__main__":
    main()
