"""Set up one 2D plan and apply the sweeping preconditioner a few times.

A small driver for profilers (ncu launch lists and kernel captures of the
sweep stages): it builds the moving-PML plan of an n x n problem with the
smooth random velocity field (seed 0), omega = 2 pi (n+1)/16, b_p = b = 12,
then runs `napply` applications of M_alpha to `nrhs` random right-hand
sides and prints the device status and the kernel launch count.

    python -m paper_1007_4291_gb300.profile_apply N LAYERS NRHS CHUNK NAPPLY
"""
import sys

import numpy as np


def main(argv):
    import torch

    from . import build, hs
    from . import inputs as I

    n, dL, R, chunk, napply = (int(a) for a in argv[:5])
    build.build()
    c = I.random_velocity(n, 0)
    o = hs.hs_default_options(layers_per_step=dL, max_nrhs=R, chunk=chunk)
    plan = hs.hs_setup(c.ravel(), 2 * np.pi * (n + 1) / 16, n, 2, 12, 12, o)
    try:
        r = torch.from_numpy(I.random_rhs(n, R, 1)).to("cuda").to(torch.complex64)
        z = torch.empty_like(r)
        for _ in range(napply):
            hs.hs_apply(plan, r, z, R, hs.HS_C64)
        torch.cuda.synchronize()
        print("status", hs.hs_last_device_status(plan), "launches", hs.load().hs_kernel_launches())
    finally:
        hs.hs_destroy(plan)


if __name__ == "__main__":
    main(sys.argv[1:])
