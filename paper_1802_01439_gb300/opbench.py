"""Per-operator throughput of libdgns on one GPU (DoFs/s vs degree).

    python -m paper_1802_01439_gb300.opbench --op laplace --k 3 --n 64 --reps 20
    python -m paper_1802_01439_gb300.opbench --sweep      # k = 2..11 at ~16.8M DoFs

Each repetition is timed with CUDA events on the launching stream after an
L2 flush (256 MiB write).  Inputs: uniform[-1, 1] (seeded) for the linear
operators, the Taylor-Green field + 1e-3 noise for the convective term.
Prints one JSON line per (operator, k).  DoFs are those of the input vector.
"""
import argparse
import json
import os
import sys

import numpy as np
import torch

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1802_01439_gb300 import Context, inputs  # noqa: E402

# elements per direction giving ~16.8M scalar DoFs for k = 2..11
SWEEP_N = {2: 85, 3: 64, 4: 51, 5: 43, 6: 37, 7: 32, 8: 28, 9: 26, 10: 23, 11: 21}
OPS = ["laplace", "laplace_split", "laplace32", "cheb32", "convective", "viscous", "helmholtz", "invmass", "mass",
       "divergence", "gradient", "projection", "helmholtz_split", "projection_split"]


def run(op, k, n, reps, warmup, ku=None, fp64_mode=0, f32_kernel=0):
    dev = torch.device("cuda")
    # scalar operators act on space U of a context with degree k
    kk = ku if ku is not None else k
    kp = max(kk - 1, 1)
    mg = 32 if op in ("laplace32", "cheb32") else 0
    if op in ("laplace32", "cheb32"):   # FP32 level operator: pressure space of degree k
        ctx = Context(n, k, k, mg_precision=32, mg_coarse_n=n)
        if ctx.lib.dgns_debug_laplace_f32_kernel(f32_kernel) != 0:
            raise ValueError("unknown FP32 Laplace kernel %d" % f32_kernel)
    else:
        ctx = Context(n, kk, kp, mg_precision=mg, fp64_mode=fp64_mode)
    nu, np_ = ctx.n_u, ctx.n_p
    f64 = dict(dtype=torch.float64, device=dev)
    rng = lambda m, s: torch.from_numpy(inputs.uniform(s, m)).to(dev)
    if op in ("laplace", "laplace_split"):
        # laplace_split: cell term, face kernel and face-apply kernel apart
        x, y, dofs = rng(nu, 0), torch.empty(nu, **f64), nu
        if op == "laplace":
            fn = lambda: ctx.vmult_laplace(y, x, space=0)
        else:
            fn = lambda: ctx.vmult_laplace_split(y, x, space=0)
        nbytes = 16 * nu
    elif op == "laplace32":
        x = rng(np_, 0).float()
        y, dofs = torch.empty_like(x), np_
        fn = lambda: ctx.vmult_laplace_f32(y, x, 0)
        nbytes = 8 * np_
    elif op == "cheb32":
        # one Chebyshev smoothing step on the level: reads x, x_prev and b,
        # writes x_new (16 bytes per DoF; the diagonal is one cell's table)
        x, xp, b = rng(np_, 0).float(), rng(np_, 1).float(), rng(np_, 2).float()
        y, dofs = torch.empty_like(x), np_
        fn = lambda: ctx.mg_chebyshev_step_f32(y, x, xp, b, 0.37, 0.021, 0)
        nbytes = 16 * np_
    elif op == "convective":
        u = torch.from_numpy(inputs.taylor_green((n,) * 3, (-np.pi,) * 3, (np.pi,) * 3, ctx.nodes_1d(0),
                                                 noise=1e-3, seed=0).ravel()).to(dev)
        y, dofs = torch.empty(3 * nu, **f64), 3 * nu
        fn = lambda: ctx.vmult_convective(y, u)
        nbytes = 16 * 3 * nu
    elif op == "helmholtz_split":
        # the operator-by-operator Helmholtz operator: mass, viscous, then
        # y = 1500 M x + V x in a vector update (against the fused kernel)
        x, y, dofs = rng(3 * nu, 0), torch.empty(3 * nu, **f64), 3 * nu
        y1 = torch.empty(3 * nu, **f64)

        def fn():
            ctx.vmult_mass(y1, x, 3, 0)
            ctx.vmult_viscous(y, x)
            ctx.axpby(y, y1, 1500.0, 1.0)
        nbytes = 16 * 3 * nu
    elif op in ("viscous", "helmholtz"):
        x, y, dofs = rng(3 * nu, 0), torch.empty(3 * nu, **f64), 3 * nu
        fn = (lambda: ctx.vmult_viscous(y, x)) if op == "viscous" else (lambda: ctx.vmult_helmholtz(y, x, 1500.0))
        nbytes = 16 * 3 * nu
    elif op in ("invmass", "mass"):
        x, y, dofs = rng(3 * nu, 0), torch.empty(3 * nu, **f64), 3 * nu
        fn = (lambda: ctx.apply_inverse_mass(y, x, 3, 0)) if op == "invmass" else (lambda: ctx.vmult_mass(y, x, 3, 0))
        nbytes = 16 * 3 * nu
    elif op == "divergence":
        x, y, dofs = rng(3 * nu, 0), torch.empty(np_, **f64), 3 * nu
        fn = lambda: ctx.vmult_divergence(y, x)
        nbytes = 8 * (3 * nu + np_)
    elif op == "gradient":
        x, y, dofs = rng(np_, 0), torch.empty(3 * nu, **f64), np_
        fn = lambda: ctx.vmult_gradient(y, x)
        nbytes = 8 * (3 * nu + np_)
    elif op in ("projection", "projection_split"):
        # fused: M + A_D + A_C in one kernel; split (the operator-by-operator
        # evaluation): M, A_D and A_C each in its own pass, summed by two
        # vector updates
        from paper_1802_01439_gb300 import _lib
        u = torch.from_numpy(inputs.taylor_green((n,) * 3, (-np.pi,) * 3, (np.pi,) * 3, ctx.nodes_1d(0),
                                                 noise=1e-3, seed=0).ravel()).to(dev)
        td, tc = ctx.penalty_parameters(u, 1e-3)
        x, y, dofs = rng(3 * nu, 0), torch.empty(3 * nu, **f64), 3 * nu
        if op == "projection":
            fn = lambda: ctx.vmult_projection(y, x, td, tc)
        else:
            y1 = torch.empty(3 * nu, **f64)

            def fn():
                ctx.vmult_projection(y, x, None, None, terms=_lib.PROJ_MASS)
                ctx.vmult_projection(y1, x, td, None, terms=_lib.PROJ_DIV)
                ctx.axpby(y, y1, 1.0, 1.0)
                ctx.vmult_projection(y1, x, None, tc, terms=_lib.PROJ_CONT)
                ctx.axpby(y, y1, 1.0, 1.0)
        nbytes = 16 * 3 * nu
    else:
        raise ValueError(op)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    if op in ("laplace32", "cheb32"):
        ctx.lib.dgns_debug_laplace_f32_kernel(0)
    ctx.close()
    return {"op": op, "k": k, "n_elem": n, "fp64_mode": fp64_mode, "dofs": dofs, "ms_mean": round(ms, 5),
            "ms_min": round(float(np.min(ts)), 5), "dofs_per_s": round(dofs / (ms * 1e-3), 1),
            "algorithmic_GBps": round(nbytes / (ms * 1e-3) / 1e9, 1)}


def poisson(n, kp, reps, mg_precision=32, fp64_mode=1):
    """Wall time of the pressure Poisson solve to rel. res. 1e-10 (zero initial
    guess): b = D u_TG (k_u = k_p + 1) + 1e-3 noise, zero mean."""
    import time
    cu = Context(n, kp + 1, kp, mg_precision=0)
    u = torch.from_numpy(inputs.taylor_green((n,) * 3, (-np.pi,) * 3, (np.pi,) * 3, cu.nodes_1d(0)).ravel()).cuda()
    b = torch.empty(cu.n_p, dtype=torch.float64, device="cuda")
    cu.vmult_divergence(b, u)
    del u
    cu.close()
    b += 1e-3 * torch.from_numpy(inputs.uniform(1, b.numel())).cuda()
    b -= b.mean()
    ctx = Context(n, kp + 1, kp, mg_precision=mg_precision, fp64_mode=fp64_mode)
    x = torch.zeros_like(b)
    ctx.cg_mg_solve(x, b, rel_tol=1e-10)
    ts = []
    for _ in range(reps):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = ctx.cg_mg_solve(x, b, rel_tol=1e-10)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ctx.close()
    return {"op": "poisson", "n_elem": n, "k_p": kp, "mg_precision": mg_precision, "fp64_mode": fp64_mode,
            "dofs": int(b.numel()), "seconds_min": round(min(ts), 5), "iterations": info["iterations"],
            "rel_res": info["rel_res"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="laplace", choices=OPS + ["poisson"])
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--fp64-mode", type=int, default=0, help="0 native FP64, 1 double-float, 2 triple-float")
    ap.add_argument("--f32-kernel", type=int, default=0,
                    help="laplace32/cheb32: kernel of the FP32 level operator (dgns_debug_laplace_f32_kernel)")
    ap.add_argument("--ops", default="laplace,convective,laplace32,invmass,helmholtz")
    ap.add_argument("--mg-precision", type=int, default=0,
                    help="poisson: 32 or 64 (default: 32 with --fp64-mode 1, else 64)")
    a = ap.parse_args()
    if a.sweep:
        for op in a.ops.split(","):
            for k, n in SWEEP_N.items():
                print(json.dumps(run(op, k, n, a.reps, a.warmup, fp64_mode=a.fp64_mode)), flush=True)
        return
    if a.op == "poisson":
        mg = a.mg_precision or (32 if a.fp64_mode == 1 else 64)
        print(json.dumps(poisson(a.n or 64, a.k, a.reps, mg, a.fp64_mode)), flush=True)
        return
    n = a.n or SWEEP_N.get(a.k, 32)
    r = run(a.op, a.k, n, a.reps, a.warmup, fp64_mode=a.fp64_mode, f32_kernel=a.f32_kernel)
    if a.op in ("laplace32", "cheb32"):
        r["f32_kernel"] = a.f32_kernel
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
