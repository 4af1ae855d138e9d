"""Benchmark of the matrix-free DG operator set on one GB300.

Workload (the paper's Taylor-Green setting, Sec. 4): periodic cube
[-pi, pi]^3 with 32^3 hexahedra, k_u = 3 (2,097,152 scalar DoFs per velocity
component), k_p = 2, 3/2-rule convective quadrature (6 points), nu = 1/1600;
velocity = Taylor-Green field at the LGL nodes + 1e-3 seeded uniform noise.
One step evaluates the full FP64 operator set once, chained as in the
dual-splitting substeps (Sec. 3.3):
    c = C(u);  uh = M^-1 c;  d = D uh;  l = L d;  g = G l;  v = (m M + V) uh
Throughput = operator DoFs per second, where each evaluation counts the DoFs
of the vector it acts on (the paper's N_dofs / t_wall per operator, Sec. 4.4):
12 n_u + 2 n_p = 26,935,296 per step.

L2 is flushed (a 256 MiB write) before every timed step; step times come from
CUDA events on the launching stream.  After the timed steps, bench.py also
times the pressure Poisson solve of the 64^3, k_p = 3 workload to relative
residual 1e-10 with the FP32 and the FP64 V-cycle (outside the timed region).

--impl reference times the CPU oracle (test infrastructure, plain FP64
numpy/LAPACK with explicit element and face matrices) on the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ELEM = 32
K_U = 3
K_P = 2
NU = 1.0 / 1600
MASS_FACTOR = 1.5 / 1e-3        # gamma_0 / dt of BDF2 with dt = 1e-3
WORKLOAD = ("full FP64 operator set (C, M^-1, D, L, G, mM+V) on 32^3 hex cells, k_u=3, k_p=2, "
            "q_conv=6, Taylor-Green + 1e-3 noise, periodic [-pi,pi]^3")
METRIC = "DG operator eval DoFs/s (FP64)"
FP64_PEAK_TFLOPS = 1.258  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25)
FP32_PEAK_TFLOPS = 80.6   # 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (probe: 73.3)
# FP32 flops the double-float emulation spends per FP64 flop of the algorithm:
# an emulated FMA (2 FP64 flops) is an exact product (FMUL + 3 FFMA) plus a
# two-sum and two adds (8 FADD) = 15 FP32 flops.
DF_FP32_PER_FP64 = 7.5
# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
# capture of the same workload (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by (kernel, fp64_mode); None where no capture of the current kernel
# exists.
KERNEL_TRAFFIC = {("conv_kernel", 1): 108.9e6, ("conv_kernel", 0): None,
                  ("conv_face_kernel", 1): 57.4e6, ("conv_face_kernel", 0): None}


# ----------------------------------------------------------- flop counts
def conv_cell_flops(N, Q):
    """FP64 flops (FMA = 2, add = 1) of the convective cell kernel per cell,
    counted from its loops: cell term by z-planes, then the six face
    integrals added to the face layers."""
    f = 2 * (3 * Q * N ** 3 + 3 * Q * Q * N * N)                      # interpolation x, y
    f += Q * (2 * 3 * Q * Q * N + Q * Q * (6 + 8 * 2 * N)           # plane values, 6 products u_c u_d, 8 x tests
              + 2 * 9 * N * N * Q + 2 * 6 * N ** 3)                   # y test, z accumulation
    return f + 6 * 3 * N * N


def conv_face_flops(N, Q):
    """FP64 flops of the convective face kernel per face: traces of both
    cells at the Q^2 points, LLF flux, tests with the face-layer basis."""
    return (2 * 6 * Q * N * N + 2 * 6 * Q * Q * N + 23 * Q * Q
            + 2 * 3 * Q * Q * N + 2 * 3 * Q * N * N + 3 * N * N)


def step_hbm(nu, npr, ms):
    """The whole step against the HBM roofline: algorithmic bytes (every
    operator reads its input vector once and writes its output once: C, M^-1
    and H on 3 velocity components, D velocity -> pressure, L on the pressure,
    G pressure -> velocity) per step time, over the measured copy bandwidth
    (MEASURED_PEAKS.json hbm_gbs, else the 6.8 TB/s fallback)."""
    peak, src = 6800.0, "fallback 6.8 TB/s"
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            peak, src = float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        pass
    nbytes = 8 * (2 * 3 * nu + 2 * 3 * nu + (3 * nu + npr) + 2 * npr + (npr + 3 * nu) + 2 * 3 * nu)
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"algorithmic_bytes": nbytes, "achieved_GBps": round(gbs, 1), "peak_GBps": peak,
            "frac": round(gbs / peak, 4), "peak_source": src}


# ------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            with open(self.path, "w") as log:     # the child keeps its own descriptor
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", dev, "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "50"],
                    stdout=log, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as log:
            lines = log.readlines()
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ GPU arm
def gpu_arm(args, rank, world):
    import torch

    from paper_1802_01439_gb300 import Context, inputs
    import __graft_entry__

    __graft_entry__.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ctx = Context(N_ELEM, K_U, K_P, nu=NU, mg_precision=0, fp64_mode=args.fp64_mode)
    nu_, np_ = ctx.n_u, ctx.n_p
    pi = np.pi
    u_host = inputs.taylor_green((N_ELEM,) * 3, (-pi,) * 3, (pi,) * 3, ctx.nodes_1d(0),
                                 noise=1e-3, seed=0).ravel()
    f64 = dict(dtype=torch.float64, device=dev)
    u = torch.from_numpy(u_host).to(dev)
    c, uh, g, v = (torch.empty(3 * nu_, **f64) for _ in range(4))
    d, lp = torch.empty(np_, **f64), torch.empty(np_, **f64)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    dofs_per_step = 12 * nu_ + 2 * np_
    rface = torch.empty(ctx.convective_face_size(), **f64)
    ev = {k: [torch.cuda.Event(enable_timing=True) for _ in range(2)] for k in
          ("Cf", "Cc", "Minv", "D", "L", "G", "H")}
    tsum = {k: 0.0 for k in ev}

    def step(timed):
        # the convective operator in its two phases (face kernel, cell kernel)
        ops = [("Cf", lambda: ctx.convective_faces(rface, u)),
               ("Cc", lambda: ctx.convective_cells(c, u, rface)),
               ("Minv", lambda: ctx.apply_inverse_mass(uh, c, ncomp=3, space=0)),
               ("D", lambda: ctx.vmult_divergence(d, uh)),
               ("L", lambda: ctx.vmult_laplace(lp, d, space=1)),
               ("G", lambda: ctx.vmult_gradient(g, lp)),
               ("H", lambda: ctx.vmult_helmholtz(v, uh, MASS_FACTOR))]
        for name, fn in ops:
            if timed:
                ev[name][0].record(stream)
            fn()
            if timed:
                ev[name][1].record(stream)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler()
    clocks.start()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        s0.record(stream)
        step(True)
        s1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        for name in ev:
            tsum[name] += ev[name][0].elapsed_time(ev[name][1])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, world)
    value = world * dofs_per_step / (ms * 1e-3)

    # end to end through the public API with host buffers: the input velocity
    # comes from pinned host memory through the C ABI's staging, the last
    # result goes back to pinned host memory; copies are inside the timing.
    u_pin = torch.from_numpy(u_host).pin_memory()
    v_pin = torch.empty(3 * nu_, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(args.warmup + max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.vmult_convective(c, u_pin)
        ctx.apply_inverse_mass(uh, c, ncomp=3, space=0)
        ctx.vmult_divergence(d, uh)
        ctx.vmult_laplace(lp, d, space=1)
        ctx.vmult_gradient(g, lp)
        ctx.vmult_helmholtz(v_pin, uh, MASS_FACTOR)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world)

    # roofline of the dominant kernel (the convective cell or face kernel):
    # ALU bound, on the FP64 pipe (native) or on the FP32 pipe (double-float)
    N, Q = K_U + 1, (3 * (K_U + 1)) // 2
    E = N_ELEM ** 3
    kern = {"Cc": ("conv_kernel", conv_cell_flops(N, Q) * E), "Cf": ("conv_face_kernel", conv_face_flops(N, Q) * 3 * E)}
    dom = max(("Cc", "Cf"), key=lambda k: tsum[k])
    kbase, conv_flops = kern[dom]
    kern_ms = tsum[dom] / args.steps
    if args.fp64_mode == 1:
        kname = "%s<DF64,%d,%d>" % (kbase, N, Q)
        achieved = DF_FP32_PER_FP64 * conv_flops / (kern_ms * 1e-3) / 1e12
        peak, psrc = FP32_PEAK_TFLOPS, ("FP32 ALU: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz; achieved counts "
                                        "7.5 FP32 flops of the double-float emulation per FP64 flop")
        fl = DF_FP32_PER_FP64 * conv_flops
    else:
        kname = "%s<F64,%d,%d>" % (kbase, N, Q)
        achieved = conv_flops / (kern_ms * 1e-3) / 1e12
        peak, psrc = FP64_PEAK_TFLOPS, "FP64 ALU: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"
        fl = conv_flops
    conv_split = {"face_kernel_ms": round(tsum["Cf"] / args.steps, 4),
                  "cell_kernel_ms": round(tsum["Cc"] / args.steps, 4)}
    tsum["C"] = tsum.pop("Cf") + tsum.pop("Cc")
    per_op = {k: round(dofs / (tsum[k] / args.steps * 1e-3), 1) for k, dofs in
              (("C", 3 * nu_), ("Minv", 3 * nu_), ("D", 3 * nu_), ("L", np_), ("G", np_), ("H", 3 * nu_))}
    share = {k: round(tsum[k] / sum(tsum.values()), 4) for k in tsum}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "DoFs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.fp64_mode == 0 else "f64 via double-float (2 x f32, 48-bit significand; "
                 "parity <= 1e-12 with the FP64 oracle) in every kernel of the step",
        "data": "synthetic (Taylor-Green + seeded noise)",
        "config": {"workload": WORKLOAD, "n_elem": N_ELEM, "degree_u": K_U, "degree_p": K_P,
                   "dofs_per_step": dofs_per_step, "l2": "flushed (256 MiB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_operator_dofs_per_s": per_op, "time_share": share, "convective_kernels": conv_split,
        "roofline": {"kernel": kname, "bound": "alu", "achieved": round(achieved, 4),
                     "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": KERNEL_TRAFFIC.get((kbase, args.fp64_mode)), "flops_per_launch": fl,
                     "peak_source": psrc},
        "step_hbm": step_hbm(nu_, np_, ms),
        "e2e": {"value": round(world * dofs_per_step / (e2e * 1e-3), 1), "unit": "DoFs/s",
                "h2d_bytes_per_step": 3 * nu_ * 8, "d2h_bytes_per_step": 3 * nu_ * 8},
        "gpu_launches": 7 * args.steps,  # face + cell convective, M^-1, D, L, G, H
        "timed_block_wall_s": round(wall, 4),
        "clocks": clk,
    }
    ctx.close()
    if args.fp64_mode == 1:
        line["native_fp64"] = native_fp64_step(u, min(args.steps, 20), flush)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sample_n=N_ELEM, repeats=5)
    if not args.no_solve and rank == 0:
        line["poisson_solve"] = poisson_solve()
        line["bdf2_tgv"] = bdf2_timing()
        line["tgv_time_loop"] = tgv_time_loop()
    return line


def native_fp64_step(u, steps, flush):
    """The same operator-set step with native FP64 kernels everywhere."""
    import torch

    from paper_1802_01439_gb300 import Context
    ctx = Context(N_ELEM, K_U, K_P, nu=NU, mg_precision=0, fp64_mode=0)
    nu_, np_ = ctx.n_u, ctx.n_p
    f64 = dict(dtype=torch.float64, device=u.device)
    c, uh, g, v = (torch.empty(3 * nu_, **f64) for _ in range(4))
    d, lp = torch.empty(np_, **f64), torch.empty(np_, **f64)

    def step():
        ctx.vmult_convective(c, u)
        ctx.apply_inverse_mass(uh, c, ncomp=3, space=0)
        ctx.vmult_divergence(d, uh)
        ctx.vmult_laplace(lp, d, space=1)
        ctx.vmult_gradient(g, lp)
        ctx.vmult_helmholtz(v, uh, MASS_FACTOR)

    for _ in range(3):
        step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    t = sum(ms) / len(ms)
    return {"value": round((12 * nu_ + 2 * np_) / (t * 1e-3), 1), "ms_per_step": round(t, 4), "steps": steps}


def bdf2_timing(steps=20):
    """The differentiated-solver workload: 32^3 cells, k_u = 4, k_p = 3,
    dt = 1e-3, Re = 1600, Taylor-Green + 1e-3 noise; wall time of `steps` BDF2
    steps (forward) and of the gradient of eps(u^steps) w.r.t. u^0 (forward
    with per-step checkpoints + backward)."""
    import torch

    from paper_1802_01439_gb300 import Context, inputs
    from paper_1802_01439_gb300.navier_stokes import DualSplitting
    n, ku = 32, 4
    ctx = Context(n, ku, ku - 1, nu=NU, mg_precision=32, fp64_mode=1)
    ds = DualSplitting(ctx, 1e-3, solver_tol=1e-12)
    pi = np.pi
    u0 = torch.from_numpy(inputs.taylor_green((n,) * 3, (-pi,) * 3, (pi,) * 3, ctx.nodes_1d(0),
                                              noise=1e-3, seed=0).ravel()).cuda()
    with torch.no_grad():
        ds.run(u0, 2, checkpoint_steps=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = ds.run(u0, steps, checkpoint_steps=False)
        eps = float(ds.dissipation(u))
        torch.cuda.synchronize()
        fwd = time.perf_counter() - t0
    # warm-up of the differentiated path (the first checkpointed step and the
    # first adjoint solves carry one-time costs of ~0.8 s)
    xw = u0.clone().requires_grad_()
    ds.dissipation(ds.run(xw, 2)).backward()
    x = u0.clone().requires_grad_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = ds.dissipation(ds.run(x, steps))
    J.backward()
    torch.cuda.synchronize()
    grad = time.perf_counter() - t0
    ctx.close()
    return {"workload": "32^3 cells, k_u=4, k_p=3, dt=1e-3, Re=1600, %d BDF2 steps" % steps,
            "forward_s": round(fwd, 4), "forward_ms_per_step": round(1e3 * fwd / steps, 3),
            "gradient_s": round(grad, 4), "eps_final": eps,
            "velocity_dofs": 3 * ctx.n_u, "pressure_dofs": ctx.n_p}


def tgv_time_loop(steps=100):
    """The paper's Taylor-Green time loop on 32^3 cells, k_u = 3 (effective
    resolution 128^3): CFL time step (Cr = 0.125), penalty projection,
    solver tolerances abs 1e-12 / rel 1e-6 with extrapolated initial guesses;
    wall time of `steps` steps and the solver iteration counts of the last."""
    from paper_1802_01439_gb300.tgv import simulate
    meta, rec = simulate(32, 3, 1e9, every=steps, max_steps=steps)
    return {"workload": "Taylor-Green, 32^3 cells, k_u=3, k_p=2, Re=1600, Cr=0.125, penalty projection, "
                        "abs/rel tol 1e-12/1e-6, extrapolated guesses, %d steps" % steps,
            "dt": meta["dt"], "wall_s": round(meta["wall_s"], 4),
            "ms_per_step": round(1e3 * meta["wall_s"] / steps, 3), "dofs": meta["dofs"],
            "dofs_steps_per_s": round(meta["dofs_steps_per_s"], 1),
            "iterations_last_step": rec[-1]["iterations"], "e_k": rec[-1]["e_k"], "eps": rec[-1]["eps"]}


def poisson_solve():
    """Pressure Poisson solve of the 64^3, k_p = 3 workload: b = D u_TG (k_u = 4)
    + 1e-3 noise, Euclidean zero mean; FP64 CG + FP32 V-cycle vs FP64 V-cycle."""
    import torch

    from paper_1802_01439_gb300 import Context, inputs
    n, kp = 64, 3
    pi = np.pi
    cu = Context(n, kp + 1, kp, mg_precision=0)
    uh = torch.from_numpy(inputs.taylor_green((n,) * 3, (-pi,) * 3, (pi,) * 3, cu.nodes_1d(0)).ravel()).cuda()
    b = torch.empty(cu.n_p, dtype=torch.float64, device="cuda")
    cu.vmult_divergence(b, uh)
    del uh
    cu.close()
    b += 1e-3 * torch.from_numpy(inputs.uniform(1, b.numel())).cuda()
    b -= b.mean()
    out = {"workload": "64^3 cells, k_p=3 (16,777,216 DoFs), rel. res. 1e-10, zero initial guess",
           "fp32_vcycle": "FP64-accurate CG (double-float matvec) + FP32 V-cycle",
           "fp64_vcycle": "all native FP64: CG matvec and V-cycle"}
    for prec in (32, 64):
        ctx = Context(n, kp + 1, kp, mg_precision=prec, fp64_mode=1 if prec == 32 else 0)
        x = torch.zeros(ctx.n_p, dtype=torch.float64, device="cuda")
        ctx.cg_mg_solve(x, b, rel_tol=1e-10)            # warm-up
        times = []
        for _ in range(3):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = ctx.cg_mg_solve(x, b, rel_tol=1e-10)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        out["fp%d_vcycle" % prec] = {"what": out["fp%d_vcycle" % prec], "seconds": round(min(times), 5),
                                     "iterations": info["iterations"], "rel_res": info["rel_res"],
                                     "levels": ctx.mg_info()["levels"]}
        ctx.close()
        del x
    out["speedup_mixed_vs_fp64"] = round(out["fp64_vcycle"]["seconds"] / out["fp32_vcycle"]["seconds"], 3)
    return out


# ------------------------------------------------------------ CPU oracle
def oracle_step_runner(n):
    """The oracle's operators on an n^3 sample of the workload; returns
    (run_one_step, dofs_per_step)."""
    from oracle import dg, rules
    from paper_1802_01439_gb300 import inputs
    m = dg.Mesh(n)
    su, sp = dg.Space(m, K_U), dg.Space(m, K_P)
    C, Mu = dg.Convective(su), dg.Mass(su)
    D, G = dg.Divergence(su, sp), dg.Gradient(su, sp)
    L, H = dg.Laplace(sp), dg.Helmholtz(su, NU, MASS_FACTOR)
    u = inputs.taylor_green(m.n, m.lo, m.hi, rules.lgl_nodes(K_U), noise=1e-3, seed=0)

    def run():
        c = C.apply(u)
        uh = Mu.apply_inverse(c)
        d = D.apply(uh)
        lp = L.apply(d)
        G.apply(lp)
        H.apply(uh)

    return run, 12 * su.size + 2 * sp.size


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(sample_n=None, repeats=5):
    sample_n = N_ELEM if sample_n is None else sample_n
    run, dofs = oracle_step_runner(sample_n)
    run()
    t = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        run()
        t.append(time.perf_counter() - t0)
    return {"value": round(dofs / min(t), 1), "unit": "DoFs/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": "oracle (numpy/LAPACK FP64, explicit element and face matrices) on %d^3 cells of the "
                      "same k_u=3/k_p=2 operator set, best of %d steps" % (sample_n, repeats)}


REF_BUDGET_S = 240.0   # wall time the reference arm's steps may take in total


def reference_sample_n(n_full, t_full, nsteps, budget=None):
    """Cells per direction of the reference arm's per-step sample: the full
    mesh if nsteps steps of t_full seconds fit the budget (REF_BUDGET_S by
    default), else the mesh halved per direction (cost ~ cells) until they
    do, 8^3 cells at least."""
    budget = REF_BUDGET_S if budget is None else budget
    n = n_full
    while n > 8 and nsteps * t_full * (n / n_full) ** 3 > budget:
        n //= 2
    return n


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    run, dofs = oracle_step_runner(N_ELEM)
    t0 = time.perf_counter()
    run()                                   # first warm-up step, on the full mesh
    n = reference_sample_n(N_ELEM, time.perf_counter() - t0, args.warmup - 1 + args.steps)
    if n != N_ELEM:
        run, dofs = oracle_step_runner(n)
    for _ in range(args.warmup - 1):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    sec = (time.perf_counter() - t0) / args.steps
    value = dofs / sec
    cores = oracle_threads()
    if n == N_ELEM:
        sample = ("oracle (numpy/LAPACK FP64) on the full %d^3, k_u=3/k_p=2 operator set, mean of the "
                  "timed steps" % N_ELEM)
    else:
        sample = ("oracle (numpy/LAPACK FP64), each step the k_u=3/k_p=2 operator set on a %d^3-cell sample "
                  "of the %d^3 workload (same operators and Taylor-Green input; the full mesh would take "
                  "more than %g s for these steps; the smaller arrays stay in cache, so the sample runs "
                  "faster per DoF than the full mesh), DoFs/s = sample DoFs / mean step time"
                  % (n, N_ELEM, REF_BUDGET_S))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "DoFs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Taylor-Green + seeded noise)",
            "config": {"workload": WORKLOAD, "n_elem": N_ELEM, "degree_u": K_U, "degree_p": K_P},
            "cpu_baseline": {"value": round(value, 1), "unit": "DoFs/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "DoFs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------ driver
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest of the ranks' x (the slowest replica's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dgns", choices=["dgns", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-mode", type=int, default=1,
                    help="1: double-float convective/SIPG kernels (default); 0: native FP64 everywhere")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = reference_arm(args, rank, world)
        if line:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    line = gpu_arm(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
