"""Runs the RHS kernel a few times on one workload, for profiling under ncu.

  python -m paper_2210_06439_gb300.profile_rhs --precision 0 --nsub 8 --reps 3 [--autotune] [--recon 1]

precision 0 = FP64, 1 = mixed; recon 0 = conserved-field reconstruction,
1 = primitive; the workload is the periodic box of nsub^3 subgrids of 8^3
cells with 5 species (ghosts filled on the device)."""
import argparse

import torch

from . import binding, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--nsub", type=int, default=8)
    ap.add_argument("--edge", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--autotune", action="store_true", help="run the autotuner first (trial launches)")
    ap.add_argument("--recon", type=int, default=0, choices=(0, 1))
    a = ap.parse_args()
    p = inputs.periodic_box(nsub=a.nsub, E=a.edge)
    H = binding.Hydro.from_problem(p, precision=a.precision, recon=a.recon)
    U = torch.from_numpy(p.U).cuda()
    H.fill_ghosts(U)
    if a.autotune:
        H.autotune(U)
    d = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    for _ in range(a.reps):
        H.rhs(U, d)
    torch.cuda.synchronize()
    assert H.error_flags() == 0
    print("ok", float(d.abs().max()))


if __name__ == "__main__":
    main()
