"""Training of the sweep post-correction network on pairs the method makes.

Pairs (x, e) = (M_alpha v, A^{-1} v - M_alpha v), the sweep output and its
error, are generated on seeded smooth random velocity fields by the library
itself: v runs over the first Arnoldi vectors of right-preconditioned GMRES
started from Gaussian point sources (the vectors the preconditioner is
applied to inside FGMRES); A^{-1} v comes from hs_solve to a tight
tolerance, M_alpha v from hs_apply.
Training runs the library's own forward, backward and Adam kernels.  The
default loss is the residual one (hs_cnn_train_step_residual): for x = M v and
rho = v - A x it fits A c to rho, the quantity the solver's judge compares,
and needs no solves.  The error loss (hs_cnn_train_step) fits c to the sweep
error e.  Evaluation reports the held-out ratio |rho - A c| / |rho| (or the
error ratio) and FGMRES iteration counts with and without the network.

    python -m paper_1007_4291_gb300.train_cnn --n 511 --pairs 2048 --steps 600 --out weights.npy
"""
import argparse
import json
import time

import numpy as np


def omega_of(n):
    return 2 * np.pi * (n + 1) / 16.0


def make_pairs(n, seeds, nrhs, bp=12, b=12, layers=12, tol=1e-9, src_seed0=1000, krylov=6):
    """Returns complex64 device tensors x = M v and e = A^{-1} v - M v of shape
    (len(seeds) * krylov * nrhs, n, n) for the first ``krylov`` Arnoldi
    vectors v of plain right-preconditioned GMRES started from Gaussian point
    sources: the vectors the preconditioner meets inside FGMRES."""
    import torch

    from . import hs
    from . import inputs as I

    xs, es = [], []
    for q, seed in enumerate(seeds):
        c = I.random_velocity(n, seed)
        o = hs.hs_default_options(layers_per_step=layers, max_nrhs=nrhs, factor_prec=hs.HS_C64, restart=30)
        plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, bp, b, o)
        try:
            f = torch.from_numpy(I.point_sources(n, nrhs, src_seed0 + seed, bp)).to("cuda")
            V = [f / torch.linalg.vector_norm(f.reshape(nrhs, -1), dim=1).reshape(nrhs, 1, 1)]
            for j in range(krylov):
                v = V[-1].contiguous()
                mv = torch.empty_like(v)
                hs.hs_apply(plan, v, mv, nrhs, hs.HS_C128)
                u = torch.zeros_like(v)
                code, info = hs.hs_solve(plan, v, u, nrhs, tol, 400)
                if code != hs.HS_OK:
                    raise RuntimeError("training solve did not converge: %r" % (info,))
                xs.append(mv.to(torch.complex64))
                es.append((u - mv).to(torch.complex64))
                if j + 1 == krylov:
                    break
                w = torch.empty_like(v)
                hs.hs_matvec(plan, mv, w, nrhs, hs.HS_C128)          # next Arnoldi direction A M v_j
                for _ in range(2):                                     # Gram-Schmidt, twice
                    for vi in V:
                        h = (vi.conj() * w).reshape(nrhs, -1).sum(dim=1).reshape(nrhs, 1, 1)
                        w = w - h * vi
                V.append(w / torch.linalg.vector_norm(w.reshape(nrhs, -1), dim=1).reshape(nrhs, 1, 1))
        finally:
            hs.hs_destroy(plan)
    return torch.cat(xs), torch.cat(es)


class ResidualData:
    """Per field: the plan (kept for its operator A), sweep outputs x = M v
    and residuals rho = v - A x of the first Arnoldi vectors v of plain GMRES
    from point sources (complex64 device tensors).  No solves are needed:
    this is the quantity the solver's judge compares."""

    def __init__(self, n, seeds, nrhs, bp=12, b=12, layers=12, krylov=6, src_seed0=1000):
        import torch

        from . import hs
        from . import inputs as I

        self.n, self.fields = n, []
        for seed in seeds:
            c = I.random_velocity(n, seed)
            o = hs.hs_default_options(layers_per_step=layers, max_nrhs=nrhs, factor_prec=hs.HS_C64)
            plan = hs.hs_setup(c.ravel(), omega_of(n), n, 2, bp, b, o)
            f = torch.from_numpy(I.point_sources(n, nrhs, src_seed0 + seed, bp)).to("cuda")
            V = [f / torch.linalg.vector_norm(f.reshape(nrhs, -1), dim=1).reshape(nrhs, 1, 1)]
            xs, rhos = [], []
            for j in range(krylov):
                v = V[-1].contiguous()
                x = torch.empty_like(v)
                hs.hs_apply(plan, v, x, nrhs, hs.HS_C128)
                ax = torch.empty_like(v)
                hs.hs_matvec(plan, x, ax, nrhs, hs.HS_C128)
                xs.append(x.to(torch.complex64))
                rhos.append((v - ax).to(torch.complex64))
                w = ax
                for _ in range(2):
                    for vi in V:
                        h = (vi.conj() * w).reshape(nrhs, -1).sum(dim=1).reshape(nrhs, 1, 1)
                        w = w - h * vi
                V.append(w / torch.linalg.vector_norm(w.reshape(nrhs, -1), dim=1).reshape(nrhs, 1, 1))
            self.fields.append((plan, torch.cat(xs), torch.cat(rhos)))

    def close(self):
        from . import hs
        for plan, _, _ in self.fields:
            hs.hs_destroy(plan)
        self.fields = []


def train_residual(net, data, steps, batch=8, lr=1e-3, seed=0, log_every=0):
    import torch

    from . import hs

    g = torch.Generator().manual_seed(seed)
    losses = []
    for it in range(steps):
        k = int(torch.randint(len(data.fields), (1,), generator=g))
        plan, x, rho = data.fields[k]
        idx = torch.randperm(x.shape[0], generator=g)[:batch].to(x.device)
        losses.append(hs.hs_cnn_train_step_residual(net, plan, x[idx].contiguous(), rho[idx].contiguous(), batch, lr))
        if log_every and it % log_every == 0:
            print("step %d residual loss %.5g" % (it, losses[-1]), flush=True)
    return losses


def residual_ratio(net, data, batch=16):
    """Per direction |rho - A c| / |rho| (the judge keeps c where it is < 1):
    returns (mean ratio, fraction of directions kept)."""
    import torch

    from . import hs

    ratios = []
    for plan, x, rho in data.fields:
        for k in range(0, x.shape[0], batch):
            xb, rb = x[k:k + batch].contiguous(), rho[k:k + batch]
            c = torch.zeros_like(xb)
            hs.hs_cnn_apply(net, xb, c, xb.shape[0], data.n, hs.HS_C64)
            ac = torch.empty_like(c)
            hs.hs_matvec(plan, c, ac, c.shape[0], hs.HS_C64)
            num = torch.linalg.vector_norm((rb - ac).reshape(rb.shape[0], -1), dim=1)
            den = torch.linalg.vector_norm(rb.reshape(rb.shape[0], -1), dim=1)
            ratios.append((num / den).double().cpu())
    r = torch.cat(ratios)
    return float(r.mean()), float((r < 1).double().mean())


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
    ap.add_argument("--pairs", type=int, default=2048, help="training pairs (krylov per source, nrhs sources per field)")
    ap.add_argument("--krylov", type=int, default=6, help="Arnoldi vectors per source")
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--out", default=None, help="save the trained parameters (.npy)")
    ap.add_argument("--eval-n", type=int, nargs="*", default=[511, 1023])
    ap.add_argument("--report", default=None, help="write the JSON report to this file too")
    ap.add_argument("--loss", choices=["residual", "error"], default="residual",
                    help="residual: |A c - rho| (what the solver's judge compares); error: |c - e|")
    args = ap.parse_args(argv)
    import torch

    from . import build, hs
    from . import inputs as I

    build.build()
    nfields = max(1, args.pairs // (args.krylov * args.nrhs))
    if args.loss == "residual":
        t0 = time.perf_counter()
        data = ResidualData(args.n, list(range(1000, 1000 + nfields)), args.nrhs, krylov=args.krylov)
        held = ResidualData(args.n, [5000], min(args.nrhs, 16), krylov=args.krylov)
        t_data = time.perf_counter() - t0
        net = hs.hs_cnn_create(I.cnn_init_params(0))
        try:
            hs.hs_cnn_set_mode(net, 1)
            before = residual_ratio(net, held)
            t0 = time.perf_counter()
            losses = train_residual(net, data, args.steps, args.batch, args.lr, log_every=100)
            torch.cuda.synchronize()
            t_train = time.perf_counter() - t0
            after = residual_ratio(net, held)
            if args.out:
                np.save(args.out, hs.hs_cnn_get_params(net))
            report = {"loss": "residual", "n": args.n, "pairs": sum(int(x.shape[0]) for _, x, _ in data.fields),
                      "steps": args.steps, "data_s": t_data, "train_s": t_train, "loss_first": losses[0],
                      "loss_last": float(np.mean(losses[-20:])),
                      "heldout_residual_ratio_before": before[0], "heldout_kept_before": before[1],
                      "heldout_residual_ratio_after": after[0], "heldout_kept_after": after[1],
                      "fgmres": {str(m): iterations(m, 5000 + m, net) for m in args.eval_n}}
            print(json.dumps(report))
            if args.report:
                with open(args.report, "w") as fh:
                    json.dump(report, fh, indent=1)
        finally:
            hs.hs_cnn_destroy(net)
            data.close()
            held.close()
        return
    t0 = time.perf_counter()
    r, e = make_pairs(args.n, list(range(1000, 1000 + nfields)), args.nrhs, krylov=args.krylov)
    rv, ev = make_pairs(args.n, [5000], min(args.nrhs, 16), krylov=args.krylov)
    t_data = time.perf_counter() - t0
    net = hs.hs_cnn_create(I.cnn_init_params(0))
    try:
        hs.hs_cnn_set_mode(net, 1)            # tensor-core layer 2 for inference
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
        if args.report:
            with open(args.report, "w") as fh:
                json.dump(report, fh, indent=1)
    finally:
        hs.hs_cnn_destroy(net)


if __name__ == "__main__":
    main()
