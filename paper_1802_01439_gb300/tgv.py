"""Taylor-Green vortex simulation with the dual-splitting BDF2 solver (Sec. 4
of arXiv:1802.01439), with the diagnostics of the paper's evaluation.

Problem: periodic box [-pi, pi]^3, U0 = L = 1, u(t=0) = (sin x cos y cos z,
-cos x sin y cos z, 0), Re = 1600 (nu = 1/Re).  The time step follows the CFL
condition dt = Cr / k_u^1.5 * h / U0 with Cr = 0.125 (Sec. 2, Sec. 4.1);
the solvers use the paper's tolerances (absolute 1e-12, relative 1e-6 to the
initial residual) with initial guesses extrapolated from the previous steps
(Sec. 3.3), the projection step with the divergence and continuity penalty
terms.

Diagnostics per recorded step (Sec. 4): the kinetic energy
e_k = 1/|Omega| int 1/2 |u|^2, the kinetic energy dissipation rate -de_k/dt
(difference quotient between consecutive steps), the molecular dissipation
eps = nu/|Omega| int grad u : grad u (at the mid step, the mean of the two
steps), and the numerical dissipation eps_num = -de_k/dt - eps; plus the
iteration counts of the three solves.

Usage: python -m paper_1802_01439_gb300.tgv --n 8 --k 3 --t-end 1.0
"""
import argparse
import json
import math
import time

import torch

from . import inputs
from .context import Context
from .navier_stokes import DualSplitting


def cfl_time_step(k_u, h, u_max=1.0, courant=0.125, r=1.5):
    """dt = Cr / k_u^r * h_min / |u|_max (the paper's CFL condition)."""
    return courant / k_u ** r * h / u_max


def kinetic_energy(dg, u, work=None):
    """e_k = 1/|Omega| int 1/2 |u|^2 = u^T M u / (2 |Omega|)."""
    mu = work if work is not None else torch.empty_like(u)
    dg.vmult_mass(mu, u, ncomp=3, space=0)
    return 0.5 * dg.dot(u, mu) / (2.0 * math.pi) ** 3


def simulate(n, k, t_end, re=1600.0, courant=0.125, projection="penalty", rel_tol=1e-6, abs_tol=1e-12,
             guess="extrapolate", mg_precision=32, fp64_mode=1, every=1, max_steps=None):
    """Runs the TGV to t_end (or max_steps) and returns the list of records."""
    ctx = Context(n, k, k - 1, nu=1.0 / re, mg_precision=mg_precision, fp64_mode=fp64_mode)
    h = 2.0 * math.pi / n
    dt = cfl_time_step(k, h, 1.0, courant)
    nsteps = int(math.ceil(t_end / dt - 1e-12))
    if max_steps is not None:
        nsteps = min(nsteps, max_steps)
    u0 = torch.from_numpy(inputs.taylor_green((n,) * 3, (-math.pi,) * 3, (math.pi,) * 3, ctx.nodes_1d(0))
                          .ravel()).cuda()
    ds = DualSplitting(ctx, dt, solver_tol=rel_tol, abs_tol=abs_tol, projection=projection, guess=guess)
    ds.log = []
    work = torch.empty_like(u0)
    state = {"ek": kinetic_energy(ctx, u0, work), "eps": ctx.dissipation(u0)}
    records = [{"step": 0, "t": 0.0, "e_k": state["ek"], "eps": state["eps"]}]

    def record(step, u):
        its = {}
        for name, info in ds.log:
            its[name] = its.get(name, 0) + int(info["iterations"])
        ds.log.clear()
        ek, eps = kinetic_energy(ctx, u, work), ctx.dissipation(u)
        rate = -(ek - state["ek"]) / dt
        eps_mid = 0.5 * (eps + state["eps"])
        state["ek"], state["eps"] = ek, eps
        if step % every == 0 or step == nsteps:
            records.append({"step": step, "t": step * dt, "e_k": ek, "eps": eps, "minus_dek_dt": rate,
                            "eps_num": rate - eps_mid, "iterations": its})

    t0 = time.perf_counter()
    with torch.no_grad():
        ds.run(u0, nsteps, checkpoint_steps=False, callback=record)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    meta = {"n_elem": n, "k_u": k, "k_p": k - 1, "re": re, "dt": dt, "steps": nsteps, "courant": courant,
            "projection": projection, "guess": guess, "wall_s": wall,
            "dofs": 3 * ctx.n_u + ctx.n_p, "dofs_steps_per_s": (3 * ctx.n_u + ctx.n_p) * nsteps / wall}
    ctx.close()
    return meta, records


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=8, help="cells per direction")
    ap.add_argument("--k", type=int, default=3, help="velocity degree k_u (pressure k_u - 1)")
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--re", type=float, default=1600.0)
    ap.add_argument("--courant", type=float, default=0.125)
    ap.add_argument("--projection", default="penalty", choices=["penalty", "l2"])
    ap.add_argument("--guess", default="extrapolate", choices=["extrapolate", "zero"])
    ap.add_argument("--every", type=int, default=10, help="record every this many steps")
    ap.add_argument("--max-steps", type=int, default=None)
    a = ap.parse_args()
    meta, records = simulate(a.n, a.k, a.t_end, re=a.re, courant=a.courant, projection=a.projection,
                             guess=a.guess, every=a.every, max_steps=a.max_steps)
    print(json.dumps(meta))
    for r in records:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
