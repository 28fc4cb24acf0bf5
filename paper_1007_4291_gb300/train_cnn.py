"""Training of the sweep post-correction network on pairs the method makes.

Pairs (x, e) = (M_alpha r, A^{-1} r - M_alpha r), the sweep output and its
error, are generated on seeded smooth random velocity fields by the library
itself: r is either a batch of Gaussian point sources f (the right-hand
sides FGMRES starts from) or the residual f - A M_alpha f after one plain
sweep (the next Krylov direction); A^{-1} r comes from hs_solve to a tight
tolerance, M_alpha r from hs_apply.
Training runs the library's own forward, backward and Adam kernels
(hs_cnn_train_step); evaluation reports the relative error of the corrected
preconditioner on held-out pairs and FGMRES iteration counts with and
without the network.

    python -m paper_1007_4291_gb300.train_cnn --n 511 --pairs 2048 --steps 600 --out weights.npy
"""
import argparse
import json
import time

import numpy as np


def omega_of(n):
    return 2 * np.pi * (n + 1) / 16.0


def make_pairs(n, seeds, nrhs, bp=12, b=12, layers=12, tol=1e-9, src_seed0=1000):
    """Returns complex64 device tensors x = M r and e = A^{-1} r - M r of shape
    (len(seeds) * 2 * nrhs, n, n)."""
    import torch

    from . import hs
    from . import inputs as I

    rs, es = [], []
    for q, seed in enumerate(seeds):
        c = I.random_velocity(n, seed)
        o = hs.hs_default_options(layers_per_step=layers, max_nrhs=nrhs, factor_prec=hs.HS_C64, restart=30)
        plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, bp, b, o)
        try:
            f = torch.from_numpy(I.point_sources(n, nrhs, src_seed0 + seed, bp)).to("cuda")
            mf = torch.empty_like(f)
            hs.hs_apply(plan, f, mf, nrhs, hs.HS_C128)
            amf = torch.empty_like(f)
            hs.hs_matvec(plan, mf, amf, nrhs, hs.HS_C128)
            r1 = f - amf
            for r in (f, r1):
                u = torch.zeros_like(r)
                code, info = hs.hs_solve(plan, r, u, nrhs, tol, 400)
                if code != hs.HS_OK:
                    raise RuntimeError("training solve did not converge: %r" % (info,))
                mr = torch.empty_like(r)
                hs.hs_apply(plan, r, mr, nrhs, hs.HS_C128)
                rs.append(mr.to(torch.complex64))
                es.append((u - mr).to(torch.complex64))
        finally:
            hs.hs_destroy(plan)
    return torch.cat(rs), torch.cat(es)


def corrected_error(net, r, e, n, batch=16):
    """sum ||e - s N(x/s)||^2 / sum ||e||^2 over the pairs (x, e) (the plain sweep scores 1)."""
    import torch

    from . import hs

    num = den = 0.0
    for k in range(0, r.shape[0], batch):
        rr, ee = r[k:k + batch], e[k:k + batch]
        z = torch.zeros_like(rr)
        hs.hs_cnn_apply(net, rr, z, rr.shape[0], n, hs.HS_C64)
        num += float(((ee - z).abs() ** 2).sum())
        den += float((ee.abs() ** 2).sum())
    return num / den


def train(net, r, e, n, steps, batch=8, lr=1e-3, seed=0, log_every=0):
    import torch

    from . import hs

    g = torch.Generator().manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randperm(r.shape[0], generator=g)[:batch].to(r.device)
        rb, eb = r[idx].contiguous(), e[idx].contiguous()
        losses.append(hs.hs_cnn_train_step(net, rb, eb, rb.shape[0], n, hs.HS_C64, lr))
        if log_every and it % log_every == 0:
            print("step %d loss %.5g" % (it, losses[-1]), flush=True)
    return losses


def iterations(n, seed, net, nrhs=8, bp=12, b=12, layers=12, tol=1e-6):
    """FGMRES iterations to tol on a held-out field, without and with the network."""
    import torch

    from . import hs
    from . import inputs as I

    c = I.random_velocity(n, seed)
    out = {}
    for name, use in (("plain", None), ("cnn", net)):
        o = hs.hs_default_options(layers_per_step=layers, max_nrhs=nrhs, factor_prec=hs.HS_C64)
        plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, bp, b, o)
        try:
            if use is not None:
                hs.hs_attach_cnn(plan, use)
            f = torch.from_numpy(I.point_sources(n, nrhs, 7000 + seed, bp)).to("cuda")
            u = torch.zeros_like(f)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            code, info = hs.hs_solve(plan, f, u, nrhs, tol, 300)
            t1 = time.perf_counter()
            out[name] = {"status": code, "iterations": info["iterations"], "seconds": t1 - t0,
                         "max_relres": info["max_relres"], "cnn_applies": info["cnn_applies"]}
        finally:
            hs.hs_destroy(plan)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=511)
    ap.add_argument("--pairs", type=int, default=2048, help="training pairs (2 per source, 64 sources per field)")
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--out", default=None, help="save the trained parameters (.npy)")
    ap.add_argument("--eval-n", type=int, nargs="*", default=[511, 1023])
    args = ap.parse_args(argv)
    import torch

    from . import build, hs
    from . import inputs as I

    build.build()
    nfields = max(1, args.pairs // (2 * args.nrhs))
    t0 = time.perf_counter()
    r, e = make_pairs(args.n, list(range(1000, 1000 + nfields)), args.nrhs)
    rv, ev = make_pairs(args.n, [5000], min(args.nrhs, 16))
    t_data = time.perf_counter() - t0
    net = hs.hs_cnn_create(I.cnn_init_params(0))
    try:
        before = corrected_error(net, rv, ev, args.n)
        t0 = time.perf_counter()
        losses = train(net, r, e, args.n, args.steps, args.batch, args.lr, log_every=100)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        after = corrected_error(net, rv, ev, args.n)
        if args.out:
            np.save(args.out, hs.hs_cnn_get_params(net))
        report = {"n": args.n, "pairs": int(r.shape[0]), "steps": args.steps, "data_s": t_data, "train_s": t_train,
                  "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:])),
                  "heldout_rel_err_sq_before": before, "heldout_rel_err_sq_after": after,
                  "fgmres": {str(m): iterations(m, 5000 + m, net) for m in args.eval_n}}
        print(json.dumps(report))
    finally:
        hs.hs_cnn_destroy(net)


if __name__ == "__main__":
    main()
