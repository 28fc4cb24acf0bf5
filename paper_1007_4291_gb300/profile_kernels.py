"""Small drivers of single kernels for profilers (ncu captures).

    python -m paper_1007_4291_gb300.profile_kernels cnn N NRHS NAPPLY
        post-correction network on NRHS random n x n fields, tensor-core layer 2
    python -m paper_1007_4291_gb300.profile_kernels three_d N NRHS NAPPLY
        3D setup (n^3, b_p = 6, b = 5, d = 1, 3xTF32 frontal updates) and
        NAPPLY slab-sweep applications to NRHS random vectors
"""
import sys

import numpy as np


def cnn(n, R, napply):
    import torch

    from . import build, hs
    from . import inputs as I

    build.build()
    net = hs.hs_cnn_create(I.cnn_init_params(0, out_scale=1.0))
    try:
        hs.hs_cnn_set_mode(net, 1)
        x = torch.from_numpy(I.random_rhs(n, R, 1)).to("cuda").to(torch.complex64)
        z = torch.zeros_like(x)
        for _ in range(napply):
            hs.hs_cnn_apply(net, x, z, R, n, hs.HS_C64)
        print("status", hs.hs_cnn_sync(net), "launches", hs.hs_kernel_launches())
    finally:
        hs.hs_cnn_destroy(net)


def three_d(n, R, napply):
    import torch

    from . import build, hs
    from . import inputs as I

    build.build()
    c = I.random_velocity(n, 0, dim=3)
    o = hs.hs_default_options(alpha=1.0, pml_C=20.0, layers_per_step=1, max_nrhs=R, frontal_gemm=3)
    plan = hs.hs_setup(c.ravel(), 2 * np.pi * 4.0 * (n + 1) / 64, n, 3, 6, 5, o)
    try:
        r = torch.from_numpy(I.random_rhs(n, R, 1, dim=3)).to("cuda").to(torch.complex64)
        z = torch.empty_like(r)
        for _ in range(napply):
            hs.hs_apply(plan, r, z, R, hs.HS_C64)
        print("status", hs.hs_sync(plan), "launches", hs.hs_kernel_launches())
    finally:
        hs.hs_destroy(plan)


if __name__ == "__main__":
    what, args = sys.argv[1], [int(a) for a in sys.argv[2:]]
    {"cnn": cnn, "three_d": three_d}[what](*args)
