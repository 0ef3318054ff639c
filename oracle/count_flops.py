"""Prints the algorithmic FP64 operation count per cell update of the method (one x sweep
plus one y sweep, second order with the MC limiter, eigenvalue guesses plus two Newton
steps), counted by the oracle's counting scalar on interior rows and columns of the
2048 x 2048 shelf workload (two layers; its three- and four-layer versions; and the unsplit step on
three 96 x 96 windows of it). Run:
python -m oracle.count_flops

TEST/MEASUREMENT INFRASTRUCTURE: the constant in bench.py comes from this script."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
from paper_1803_01450_gb300 import inputs as I  # noqa: E402


def main():
    w = I.scale(2048)
    dt = 0.9 * w["dx"] / 205.0
    for order, eigen in ((2, 0), (1, 0)):
        P = O.params(M=2, dry_tol=1e-3, order=order, eigen=eigen)
        f = O.flops_per_cell_update(P, w["q"], w["B"], w["dx"], w["dy"], dt, rows=[100, 1024, 1900],
                                    cols=[100, 1024, 1900])
        print(f"order={order} eigen={eigen}: {f:.2f} FP64 operations per cell update")
    w3 = I.scale3(2048)
    P3 = O.params(M=3, dry_tol=1e-3, order=2, rho=(1000.0, 1020.0, 1030.0))
    f3 = O.flops_per_cell_update(P3, w3["q"], w3["B"], w3["dx"], w3["dy"], dt, rows=[100, 1024, 1900],
                                 cols=[100, 1024, 1900])
    print(f"three layers (scale3 workload), order=2 eigen=0: {f3:.2f} FP64 operations per cell update")
    w4 = I.scale4(2048)
    P4 = O.params(M=4, dry_tol=1e-3, order=2, rho=(1000.0, 1020.0, 1030.0, 1040.0))
    f4 = O.flops_per_cell_update(P4, w4["q"], w4["B"], w4["dx"], w4["dy"], dt, rows=[100, 1024, 1900],
                                 cols=[100, 1024, 1900])
    print(f"four layers (scale4 workload), order=2 eigen=0: {f4:.2f} FP64 operations per cell update")
    Pu = O.params(M=2, dry_tol=1e-3, order=2, unsplit=1)
    fu = O.flops_per_cell_update_unsplit(Pu, w["q"], w["B"], w["dx"], w["dy"], dt,
                                         windows=[(100, 100, 96), (976, 976, 96), (1852, 1852, 96)])
    print(f"unsplit, order=2 eigen=0: {fu['total']:.2f} FP64 operations per cell update "
          f"(x edges {fu['x']:.2f}, y edges {fu['y']:.2f}, transverse fluxes and update {fu['update']:.2f})")
    P3u = O.params(M=3, dry_tol=1e-3, order=2, rho=(1000.0, 1020.0, 1030.0), unsplit=1)
    f3u = O.flops_per_cell_update_unsplit(P3u, w3["q"], w3["B"], w3["dx"], w3["dy"], dt,
                                          windows=[(100, 100, 96), (976, 976, 96), (1852, 1852, 96)])
    print(f"unsplit, three layers (scale3 workload): {f3u['total']:.2f} FP64 operations per cell update "
          f"(x edges {f3u['x']:.2f}, y edges {f3u['y']:.2f}, transverse fluxes and update {f3u['update']:.2f})")


if __name__ == "__main__":
    main()
