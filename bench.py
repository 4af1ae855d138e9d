"""Benchmark of the matrix-free DG operators on one GB300.

Workload (the paper's throughput experiment, Sec. 4.4, on its Taylor-Green
setting, Sec. 4): the degree sweep k = 2, 3, 4, 5, 7, 9, 11, each on the
periodic cube [-pi, pi]^3 with n^3 hexahedra chosen for ~16.8M scalar DoFs
(n = 85, 64, 51, 43, 32, 26, 21).  One step evaluates, for every k of the
sweep, the SIPG Laplace operator on a seeded uniform[-1, 1] vector and the
convective term (3/2-rule over-integration, local Lax-Friedrichs flux) on the
Taylor-Green field + 1e-3 seeded noise.  Throughput = operator DoFs per
second, each evaluation counting the DoFs of the vector it acts on (the
paper's N_dofs / t_wall, Sec. 4.4); the headline is the whole sweep's DoFs
over its time, in FP64 arithmetic.  The per-k table sits in the same line.

L2 is flushed (a 256 MiB write) before every operator evaluation, outside its
CUDA events; step time = the sum of the evaluations' event times on the
launching stream.  After the timed steps bench.py also times: the same sweep
in double-float arithmetic (a labelled extra, 48-bit significand); the full
operator set of the 32^3, k_u = 3 workload; the pressure Poisson solve of the
64^3, k_p = 3 workload to relative residual 1e-10 with FP64 CG and the FP32
V-cycle against the all-FP64 solve; the differentiated BDF2 workload and the
Taylor-Green time loop (all outside the timed region).

--impl reference times the CPU oracle (test infrastructure, plain FP64
numpy/LAPACK with explicit element and face matrices) on a bounded sample of
the same sweep.
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

# the degree sweep: (k, elements per direction), ~16.8M scalar DoFs each
SWEEP = [(2, 85), (3, 64), (4, 51), (5, 43), (7, 32), (9, 26), (11, 21)]
NU = 1.0 / 1600
MASS_FACTOR = 1.5 / 1e-3        # gamma_0 / dt of BDF2 with dt = 1e-3
METRIC = "DG operator eval DoFs/s vs degree k (FP64); Poisson solve s at rel. res 1e-10"
WORKLOAD = ("degree sweep k=2,3,4,5,7,9,11 at ~16.8M scalar DoFs each (85^3, 64^3, 51^3, 43^3, 32^3, "
            "26^3, 21^3 hex cells, periodic [-pi,pi]^3): SIPG Laplace vmult on uniform[-1,1] + convective "
            "vmult (floor(3(k+1)/2)-point rule, LLF flux) on Taylor-Green + 1e-3 noise")
MODES = {0: "f64", 1: "df64", 2: "f64_wide"}
MODE_DTYPE = {0: "f64",
              1: "f64 via double-float (2 x f32, 48-bit significand; parity <= 1e-12 with the FP64 oracle)",
              2: "f64-wide mix: triple-float (3 x f32, up to 72-bit significand) in the SIPG, mass and low-degree "
                 "convective face kernels, native-FP64 and triple-float blocks side by side in the k <= 3 "
                 "convective cell kernel, native FP64 elsewhere"}
FP64_PEAK_TFLOPS = 1.258  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25)
FP32_PEAK_TFLOPS = 80.6   # 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz
# FP32 flops the double-float emulation spends per FP64 operation: an
# emulated multiply-add is an exact product (FMUL + FFMA) with two cross
# terms (2 FFMA), a two-sum (6 FADD) and two additions: 15 flops; an
# emulated addition is a two-sum and two additions: 8 flops.
EMU_FP32_FLOPS = {1: (15, 8), 2: (51, 21)}
# (triple-float: an emulated multiply-add is three exact products (FMUL +
# FFMA each), four two-sums (24 FADD), six additions and three FFMA: 51
# flops; an addition is three two-sums and three additions: 21 flops)
# DRAM bytes (read + write) of one launch of a kernel, from one ncu capture
# of the same launch configuration (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (kernel, fp64 mode, k); absent where no
# capture of the current kernel exists.
# (kernel, fp64_mode, k) -> DRAM bytes (read + write) per launch from one ncu
# capture of the current kernel: k = 9 on 26^3 cells, k = 11 on 21^3 cells
KERNEL_TRAFFIC = {("conv_kernel", 0, 9): 551.5e6 + 384.6e6, ("conv_kernel", 0, 11): 483.0e6 + 345.9e6}


# ----------------------------------------------------------- flop counts
# Algorithmic work of the method as the kernels organise it (Kronecker
# factorisation of the SIPG operators on Cartesian cells, face kernel + cell
# kernel for the convective term), with every 1D contraction counted in its
# even-odd form (the 1D matrices are centrosymmetric or centro-antisymmetric
# on the symmetric LGL nodes and Gauss points).  Counts are (multiply-adds,
# additions); a multiply-add is 2 flops.
def eo_line(L, M):
    """One even-odd contraction of a line of L values to M outputs: fold the
    line into floor(L/2) sums and differences, two half-size products
    (ceil(M/2) x ceil(L/2) and floor(M/2) x floor(L/2) multiply-adds),
    recombine floor(M/2) output pairs."""
    fma = -(-M // 2) * -(-L // 2) + (M // 2) * (L // 2)
    return fma, 2 * (L // 2) + 2 * (M // 2)


def _add(acc, cnt, times=1):
    return acc[0] + times * cnt[0], acc[1] + times * cnt[1]


def laplace_ops(N):
    """SIPG Laplace per cell: L = T_x (x) M (x) M + M (x) T_y (x) M + M (x) M (x) T_z
    evaluated as M_z[M_y T_x x + M_x T_y x] + M_x M_y T_z x: 8 line sweeps of
    N^2 lines, the neighbour terms of the 1D SIPG operators T_d (per DoF and
    direction: the value and normal derivative of both neighbours' face
    layers, 4 multiply-adds, one more for the derivative sums amortised over
    the line), and 2 additions per DoF."""
    ops = (0, 0)
    ops = _add(ops, eo_line(N, N), 8 * N * N)
    ops = _add(ops, (12 * N ** 3, 2 * N ** 3))
    return ops


def conv_cell_ops(N, Q):
    """Convective cell term per cell: u_c interpolated to the Q^3 points
    (3 components, sweeps of N^2, QN and Q^2 lines N -> Q), the 6 distinct
    products u_c u_d (weights folded into the test tables), 8 distinct x
    tests (Q^2 lines Q -> N; F_12 = F_21 tested once), 9 y tests (NQ lines),
    6 z tests (N^2 lines, two per component) and their sums, and the six
    face integrals added to the face layers of 3 components."""
    ops = (0, 0)
    ops = _add(ops, eo_line(N, Q), 3 * (N * N + Q * N + Q * Q))
    ops = _add(ops, (0, 6 * Q ** 3))
    ops = _add(ops, eo_line(Q, N), 8 * Q * Q + 9 * N * Q + 6 * N * N)
    ops = _add(ops, (0, 3 * N ** 3 + 6 * 3 * N * N))
    return ops


def conv_face_ops(N, Q):
    """Convective face term per face: traces of 3 components of both cells
    at the Q^2 face points (the face layer's N^2 nodal values, sweeps of N and
    Q lines N -> Q), the LLF flux (per point and component a product, a
    multiply-add for the average of u_c u_n, the jump and a multiply-add with
    the penalty: 6 multiply-adds and 6 additions or products per point; the
    halving of the average belongs to the face-area factor and
    max(|a|, |b|) is a comparison), and the test of the 3 flux components
    back to the N^2 layer (Q and N lines Q -> N)."""
    ops = (0, 0)
    ops = _add(ops, eo_line(N, Q), 6 * (N + Q))
    ops = _add(ops, (6 * Q * Q, 6 * Q * Q))
    ops = _add(ops, eo_line(Q, N), 3 * (Q + N))
    return ops


def flops(ops):
    return 2 * ops[0] + ops[1]


def fp32_flops(ops, mode):
    """FP32-pipe flops of the emulated FP64 operations (double-float or
    triple-float)."""
    cf, ca = EMU_FP32_FLOPS[mode]
    return cf * ops[0] + ca * ops[1]


def read_peaks():
    """The measured copy bandwidth (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def alu_frac(ops, seconds, mode):
    """Achieved fraction of the ALU roof the arithmetic runs on: the FP64 pipe
    (native) or the FP32 pipe (emulation)."""
    if mode == 0:
        return flops(ops) / seconds / 1e12 / FP64_PEAK_TFLOPS
    return fp32_flops(ops, mode) / seconds / 1e12 / FP32_PEAK_TFLOPS


def step_hbm(nu, npr, ms):
    """The 32^3 operator-set step against the HBM roofline: algorithmic bytes
    (every operator reads its input vector once and writes its output once:
    C, M^-1 and H on 3 velocity components, D velocity -> pressure, L on the
    pressure, G pressure -> velocity) per step time, over the measured copy
    bandwidth (MEASURED_PEAKS.json hbm_gbs, else the 6.8 TB/s fallback)."""
    peak, src = read_peaks()
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
class Sweep:
    """Contexts, inputs and outputs of the degree sweep in one arithmetic
    mode, resident on the device."""

    def __init__(self, mode, dev):
        import torch

        from paper_1802_01439_gb300 import Context, inputs
        self.mode, self.items = mode, []
        f64 = dict(dtype=torch.float64, device=dev)
        for k, n in SWEEP:
            ctx = Context(n, k, k - 1, nu=NU, mg_precision=0, fp64_mode=mode)
            nu_ = ctx.n_u
            x = torch.from_numpy(inputs.uniform(0, nu_)).to(dev)
            u = torch.from_numpy(inputs.taylor_green((n,) * 3, (-np.pi,) * 3, (np.pi,) * 3, ctx.nodes_1d(0),
                                                     noise=1e-3, seed=0).ravel()).to(dev)
            self.items.append({"k": k, "n": n, "ctx": ctx, "x": x, "u": u, "y": torch.empty(nu_, **f64),
                               "c": torch.empty(3 * nu_, **f64),
                               "rface": torch.empty(ctx.convective_face_size(), **f64)})
        self.dofs = sum(4 * it["ctx"].n_u for it in self.items)

    def ops(self, it):
        """The timed pieces of one k: Laplace, convective faces, convective cells."""
        ctx = it["ctx"]
        return [("L", lambda: ctx.vmult_laplace(it["y"], it["x"], space=0)),
                ("Cf", lambda: ctx.convective_faces(it["rface"], it["u"])),
                ("Cc", lambda: ctx.convective_cells(it["c"], it["u"], it["rface"]))]

    def close(self):
        for it in self.items:
            it["ctx"].close()
        self.items = []


def run_sweep(sw, steps, warmup, flush, stream, world, sample_clocks=False):
    """Times `steps` passes over the sweep; returns (mean step ms, per-k mean
    ms of each piece, clocks, wall seconds of the timed block)."""
    import torch
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(3)] for _ in sw.items]
    tsum = [[0.0] * 3 for _ in sw.items]

    def step(timed):
        for i, it in enumerate(sw.items):
            for j, (name, fn) in enumerate(sw.ops(it)):
                if name != "Cc":             # the cell kernel reads the face kernel's output
                    flush.zero_()
                if timed:
                    ev[i][j][0].record(stream)
                fn()
                if timed:
                    ev[i][j][1].record(stream)

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler()
    if sample_clocks:
        clocks.start()
    step_ms = []
    wall0 = time.perf_counter()
    for _ in range(steps):
        step(True)
        torch.cuda.synchronize()
        t = 0.0
        for i in range(len(sw.items)):
            for j in range(3):
                dt = ev[i][j][0].elapsed_time(ev[i][j][1])
                tsum[i][j] += dt
                t += dt
        step_ms.append(t)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop() if sample_clocks else None
    per_k = [[v / steps for v in row] for row in tsum]
    return sum(step_ms) / len(step_ms), per_k, clk, wall


def sweep_table(sw, per_k, mode):
    """Per-k DoFs/s, HBM fraction (16 algorithmic bytes per DoF: the input
    read once, the output written once) and ALU fraction of each operator."""
    peak, _ = read_peaks()
    rows = []
    for it, (tl, tf, tc) in zip(sw.items, per_k):
        k, n = it["k"], it["n"]
        N, Q = k + 1, (3 * (k + 1)) // 2
        E, nu_ = n ** 3, it["ctx"].n_u
        lap, conv = nu_ / (tl * 1e-3), 3 * nu_ / ((tf + tc) * 1e-3)
        lap_ops = tuple(E * v for v in laplace_ops(N))
        cc, cf = conv_cell_ops(N, Q), conv_face_ops(N, Q)
        conv_ops = (E * (cc[0] + 3 * cf[0]), E * (cc[1] + 3 * cf[1]))
        rows.append({"k": k, "n_elem": n, "dofs": nu_,
                     "laplace_dofs_per_s": round(lap, 1), "convective_dofs_per_s": round(conv, 1),
                     "laplace_ms": round(tl, 4), "convective_ms": round(tf + tc, 4),
                     "conv_face_kernel_ms": round(tf, 4), "conv_cell_kernel_ms": round(tc, 4),
                     "laplace_hbm_frac": round(16 * lap / 1e9 / peak, 4),
                     "convective_hbm_frac": round(16 * conv / 1e9 / peak, 4),
                     "laplace_alu_frac": round(alu_frac(lap_ops, tl * 1e-3, mode), 4),
                     # the FP64-wide mix runs the convective kernels on both pipes
                     "convective_alu_frac": (None if mode == 2 else
                                             round(alu_frac(conv_ops, (tf + tc) * 1e-3, mode), 4))})
    return rows


def dominant_roofline(sw, per_k, mode):
    """Roofline of the kernel with the largest share of the sweep's time:
    algorithmic flops per launch (even-odd counts above) over its mean
    event-timed launch duration, against the peak of the pipe it runs on."""
    best = None
    for it, (tl, tf, tc) in zip(sw.items, per_k):
        k, n = it["k"], it["n"]
        N, Q = k + 1, (3 * (k + 1)) // 2
        E = n ** 3
        for name, ms, ops in (("sipg_kernel", tl, tuple(E * v for v in laplace_ops(N))),
                              ("conv_face_kernel", tf, tuple(3 * E * v for v in conv_face_ops(N, Q))),
                              ("conv_kernel", tc, tuple(E * v for v in conv_cell_ops(N, Q)))):
            if best is None or ms > best[1]:
                best = (name, ms, ops, k, N, Q)
    name, ms, ops, k, N, Q = best
    pol = {0: "F64", 1: "DF64", 2: "TF64"}[mode]
    kname = "%s<%s,%d>" % (name, pol, N) if name == "sipg_kernel" else "%s<%s,%d,%d>" % (name, pol, N, Q)
    if mode == 0:
        fl, peak = flops(ops), FP64_PEAK_TFLOPS
        psrc = "FP64 ALU: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (probe: 1.04 TFLOP/s)"
    else:
        fl, peak = fp32_flops(ops, mode), FP32_PEAK_TFLOPS
        psrc = ("FP32 ALU: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz; achieved counts the FP32 flops of the "
                "emulated FP64 operations (%d per multiply-add, %d per addition)" % EMU_FP32_FLOPS[mode])
    achieved = fl / (ms * 1e-3) / 1e12
    return {"kernel": kname, "k": k, "bound": "alu", "achieved": round(achieved, 4), "peak": peak,
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": KERNEL_TRAFFIC.get((name, mode, k)), "flops_per_launch": fl,
            "launch_ms": round(ms, 4), "peak_source": psrc,
            "flop_count": "even-odd algorithmic count (bench.laplace_ops / conv_cell_ops / conv_face_ops)"}


def e2e_sweep(sw, steps, warmup, world, stream):
    """The sweep end to end through the public API: every input starts in
    pinned host memory and every result ends there; the copies are inside
    the timing.  The host-to-device copies of all degrees are queued on one
    copy stream and the device-to-host copies on another, ordered against
    the context's stream by one event per vector, so the copy engines move
    the next operators' inputs in and the previous operators' results out
    while the kernels run: each operator waits only for its own input (the
    Laplace operator for x, the convective term for u) and each result leaves
    as soon as its operator is done (the library's calls with host pointers,
    which stage and wait per call, would serialise them)."""
    import torch
    host = []
    for it in sw.items:
        nu_ = it["ctx"].n_u
        host.append((it["x"].cpu().pin_memory(), torch.empty(nu_, dtype=torch.float64).pin_memory(),
                     it["u"].cpu().pin_memory(), torch.empty(3 * nu_, dtype=torch.float64).pin_memory()))
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    nk = len(sw.items)
    ts = []
    for rep in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev_x, ev_u, ev_y, ev_c = ([torch.cuda.Event() for _ in range(nk)] for _ in range(4))
        with torch.cuda.stream(h2d):
            for i, (it, (xh, _, uh, _)) in enumerate(zip(sw.items, host)):
                it["x"].copy_(xh, non_blocking=True)
                ev_x[i].record(h2d)
                it["u"].copy_(uh, non_blocking=True)
                ev_u[i].record(h2d)
        for i, it in enumerate(sw.items):
            stream.wait_event(ev_x[i])
            it["ctx"].vmult_laplace(it["y"], it["x"], space=0)
            ev_y[i].record(stream)
            stream.wait_event(ev_u[i])
            it["ctx"].vmult_convective(it["c"], it["u"])
            ev_c[i].record(stream)
        with torch.cuda.stream(d2h):
            for i, (it, (_, yh, _, ch)) in enumerate(zip(sw.items, host)):
                d2h.wait_event(ev_y[i])
                yh.copy_(it["y"], non_blocking=True)
                d2h.wait_event(ev_c[i])
                ch.copy_(it["c"], non_blocking=True)
        torch.cuda.synchronize()
        if rep >= warmup:
            ts.append(time.perf_counter() - t0)
    t = max_over_ranks(sum(ts) / len(ts), world)
    nbytes = sum(8 * 4 * it["ctx"].n_u for it in sw.items)
    return {"value": round(world * sw.dofs / t, 1), "unit": "DoFs/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": round(t * 1e3, 3), "steps": steps,
            "copies": "pinned host buffers, H2D and D2H on their own streams, overlapped with the kernels"}


def gpu_arm(args, rank, world):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    mode = args.fp64_mode

    sw = Sweep(mode, dev)
    ms, per_k, clk, wall = run_sweep(sw, args.steps, args.warmup, flush, stream, world, sample_clocks=True)
    ms = max_over_ranks(ms, world)
    table = sweep_table(sw, per_k, mode)
    roof = dominant_roofline(sw, per_k, mode)
    e2e = e2e_sweep(sw, max(4, args.steps // 2), 2, world, stream)
    sw.close()
    del sw
    line = {
        "metric": METRIC, "value": round(world * sum(4 * n ** 3 * (k + 1) ** 3 for k, n in SWEEP) / (ms * 1e-3), 1),
        "unit": "DoFs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": MODE_DTYPE[mode], "data": "synthetic (uniform[-1,1] and Taylor-Green + seeded noise)",
        "config": {"workload": WORKLOAD, "degrees": [k for k, _ in SWEEP], "n_elem": [n for _, n in SWEEP],
                   "dofs_per_step": sum(4 * n ** 3 * (k + 1) ** 3 for k, n in SWEEP),
                   "l2": "flushed (256 MiB write) before every operator evaluation, outside its events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_k": table, "roofline": roof, "e2e": e2e,
        "gpu_launches": 3 * len(SWEEP) * args.steps,   # SIPG, convective face and cell kernels per k
        "timed_block_wall_s": round(wall, 4), "clocks": clk,
    }
    if not args.no_extras:
        for other in sorted(MODES):
            if other == mode:
                continue
            sw = Sweep(other, dev)
            oms, oper_k, _, _ = run_sweep(sw, max(3, args.steps // 2), 2, flush, stream, world)
            line["sweep_" + MODES[other]] = {
                "dtype": MODE_DTYPE[other], "ms_per_step": round(oms, 4),
                "value": round(sum(4 * n ** 3 * (k + 1) ** 3 for k, n in SWEEP) / (oms * 1e-3), 1),
                "per_k": sweep_table(sw, oper_k, other),
                "roofline": dominant_roofline(sw, oper_k, other) if other != 2 else None}
            sw.close()
            del sw
        line["operator_set_32c_k3"] = {m: operator_set_step(dev, flush, m, 20) for m in (0, 1)}
        line["fused_vs_split"] = fused_vs_split()
        line["mg_smoother_64c_k3"] = mg_smoother_step()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if not args.no_solve and rank == 0:
        line["poisson_solve"] = poisson_solve()
        line["bdf2_tgv"] = bdf2_timing()
        line["tgv_time_loop"] = tgv_time_loop()
    return line


def operator_set_step(dev, flush, mode, steps):
    """The full FP64 operator set of the 32^3, k_u = 3, k_p = 2 workload chained
    as in the dual-splitting substeps (Sec. 3.3):
        c = C(u);  uh = M^-1 c;  d = D uh;  l = L d;  g = G l;  v = (m M + V) uh
    DoFs per step: 12 n_u + 2 n_p (each evaluation counts its input vector)."""
    import torch

    from paper_1802_01439_gb300 import Context, inputs
    n, ku, kp = 32, 3, 2
    ctx = Context(n, ku, kp, nu=NU, mg_precision=0, fp64_mode=mode)
    nu_, np_ = ctx.n_u, ctx.n_p
    f64 = dict(dtype=torch.float64, device=dev)
    u = torch.from_numpy(inputs.taylor_green((n,) * 3, (-np.pi,) * 3, (np.pi,) * 3, ctx.nodes_1d(0),
                                             noise=1e-3, seed=0).ravel()).to(dev)
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
    return {"dtype": MODE_DTYPE[mode], "value": round((12 * nu_ + 2 * np_) / (t * 1e-3), 1),
            "ms_per_step": round(t, 4), "steps": steps, "step_hbm": step_hbm(nu_, np_, t),
            "workload": "full operator set (C, M^-1, D, L, G, mM+V) on 32^3 cells, k_u=3, k_p=2, q_conv=6, "
                        "Taylor-Green + 1e-3 noise; L2 flushed before every step"}


def fused_vs_split(reps=5):
    """The paper's comparison of its optimised operators with the standard,
    operator-by-operator evaluation (Sec. 4.4), in native FP64 for every k of
    the sweep: the Helmholtz operator (one SIPG kernel with the mass term
    folded in, against the mass kernel, the viscous kernel and a vector
    update), the projection operator (one kernel for M + A_D + A_C, against
    M, A_D and A_C in three passes and two vector updates) and the SIPG
    Laplacian (the fused element-centric kernel against the cell term, a
    face kernel and a face-apply kernel; one scalar field).  Mean event
    times with L2 flushed; ratio = split / fused."""
    from paper_1802_01439_gb300.opbench import run
    out = {"workload": "~16.8M scalar DoFs per component (3 components, Laplace 1), native FP64, "
                       "L2 flushed, mean of %d" % reps}
    for k, n in SWEEP:
        row = {}
        for op in ("helmholtz", "helmholtz_split", "projection", "projection_split", "laplace", "laplace_split"):
            row[op + "_ms"] = run(op, k, n, reps, 2, fp64_mode=0)["ms_mean"]
        row["helmholtz_ratio"] = round(row["helmholtz_split_ms"] / row["helmholtz_ms"], 3)
        row["projection_ratio"] = round(row["projection_split_ms"] / row["projection_ms"], 3)
        row["laplace_ratio"] = round(row["laplace_split_ms"] / row["laplace_ms"], 3)
        out["k%d" % k] = row
    return out


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
    return {"workload": "32^3 cells, k_u=4, k_p=3, dt=1e-3, Re=1600, %d BDF2 steps (double-float operators, "
                        "FP32 multigrid)" % steps,
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


# the Poisson arms: (key, V-cycle precision, arithmetic of the CG matvec, what)
POISSON_ARMS = [("mixed", 32, 0, "native FP64 CG (matvec, residual, dots, updates) + FP32 V-cycle"),
                ("fp64", 64, 0, "native FP64 CG + FP64 V-cycle (all FP64)"),
                ("mixed_tf64_matvec", 32, 2, "FP64 CG with a triple-float (FP64-wide) matvec + FP32 V-cycle"),
                ("mixed_df64_matvec", 32, 1, "FP64 CG with a double-float matvec (48-bit) + FP32 V-cycle")]


# DRAM bytes (read + write) of one Chebyshev step of the staged FP32 kernel at
# 64^3 cells, k_p = 3, from one ncu capture (second launch on the finest
# level, with a previous iterate)
SMOOTHER_TRAFFIC = 203.45e6 + 40.50e6


def mg_smoother_step():
    """One Jacobi-Chebyshev smoothing step of the FP32 multigrid on the finest
    level of the 64^3, k_p = 3 Poisson workload (Sec. 3.3; the level operator
    with the update fused into its epilogue): x_new = x + c1 (x - x_prev) +
    c2 D^-1 (b - L x), 16 algorithmic bytes per DoF (read x, x_prev, b; write
    x_new).  The built-in kernel (staged by tensor copies) against the line
    kernel it replaced, CUDA events after an L2 flush, mean of 20."""
    from paper_1802_01439_gb300 import opbench
    peak, src = read_peaks()
    out = {"workload": "64^3 cells, k_p=3 (16,777,216 DoFs), FP32", "bytes_per_dof": 16}
    for key, kern in (("staged", 0), ("line", -1)):
        r = opbench.run("cheb32", 3, 64, 20, 3, f32_kernel=kern)
        gbs = 16 * r["dofs"] / (r["ms_mean"] * 1e-3) / 1e9
        out[key] = {"us": round(r["ms_mean"] * 1e3, 2), "GBps": round(gbs, 1), "frac": round(gbs / peak, 4)}
    out["staged"]["kernel"] = "sipg_tma_kernel<EPI_CHEB, 1, packed, 12 warps, 1 stage>"
    out["staged"]["traffic"] = SMOOTHER_TRAFFIC
    out["peak"] = {"GBps": peak, "source": src}
    return out


def poisson_solve():
    """Pressure Poisson solve of the 64^3, k_p = 3 workload: b = D u_TG (k_u = 4)
    + 1e-3 noise, Euclidean zero mean, to relative residual 1e-10 from a zero
    guess.  The controlled pair differs only in the V-cycle's precision (the
    CG matvec is native FP64 in both); a third arm uses the double-float CG
    matvec."""
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
    out = {"workload": "64^3 cells, k_p=3 (16,777,216 DoFs), rel. res. 1e-10, zero initial guess"}
    for key, prec, mode, what in POISSON_ARMS:
        ctx = Context(n, kp + 1, kp, mg_precision=prec, fp64_mode=mode)
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
        out[key] = {"what": what, "seconds": round(min(times), 5), "iterations": info["iterations"],
                    "rel_res": info["rel_res"], "levels": ctx.mg_info()["levels"]}
        ctx.close()
        del x
    out["speedup_mixed_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed"]["seconds"], 3)
    out["speedup_mixed_tf64_matvec_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_tf64_matvec"]["seconds"], 3)
    out["speedup_mixed_df64_matvec_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_df64_matvec"]["seconds"], 3)
    return out


# ------------------------------------------------------------ CPU oracle
CPU_SAMPLE_N = 8     # cells per direction of the oracle's sample, every k


def oracle_sweep_runner(n):
    """The oracle's Laplace and convective operators for every k of the sweep
    on an n^3 sample mesh with the same inputs; returns (run_one_step,
    dofs_per_step)."""
    from oracle import dg, rules
    from paper_1802_01439_gb300 import inputs
    m = dg.Mesh(n)
    work = []
    for k, _ in SWEEP:
        s = dg.Space(m, k)
        x = inputs.uniform(0, s.size).reshape(m.E, -1)
        u = inputs.taylor_green(m.n, m.lo, m.hi, rules.lgl_nodes(k), noise=1e-3, seed=0)
        work.append((dg.Laplace(s), dg.Convective(s), x, u, s.size))

    def run():
        for L, C, x, u, _ in work:
            L.apply(x)
            C.apply(u)

    return run, sum(4 * w[4] for w in work)


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(sample_n=None, repeats=3):
    sample_n = CPU_SAMPLE_N if sample_n is None else sample_n
    run, dofs = oracle_sweep_runner(sample_n)
    run()
    t = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        run()
        t.append(time.perf_counter() - t0)
    return {"value": round(dofs / min(t), 1), "unit": "DoFs/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": "oracle (numpy/LAPACK FP64, explicit element and face matrices): the Laplace and "
                      "convective operators of every k of the sweep on %d^3 cells (same inputs), best of %d "
                      "passes" % (sample_n, repeats)}


REF_BUDGET_S = 240.0   # wall time the reference arm's steps may take in total


def reference_sample_n(n_full, t_full, nsteps, budget=None):
    """Cells per direction of the reference arm's per-step sample: n_full if
    nsteps steps of t_full seconds fit the budget (REF_BUDGET_S by default),
    else halved (cost ~ cells) until they do, 2^3 cells at least."""
    budget = REF_BUDGET_S if budget is None else budget
    n = n_full
    while n > 2 and nsteps * t_full * (n / n_full) ** 3 > budget:
        n //= 2
    return n


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    run, dofs = oracle_sweep_runner(CPU_SAMPLE_N)
    t0 = time.perf_counter()
    run()                                   # first warm-up step
    n = reference_sample_n(CPU_SAMPLE_N, time.perf_counter() - t0, args.warmup - 1 + args.steps)
    if n != CPU_SAMPLE_N:
        run, dofs = oracle_sweep_runner(n)
    for _ in range(args.warmup - 1):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    sec = (time.perf_counter() - t0) / args.steps
    value = dofs / sec
    cores = oracle_threads()
    sample = ("oracle (numpy/LAPACK FP64, explicit element and face matrices), each step the Laplace and "
              "convective operators of every k of the sweep on a %d^3-cell sample of the ~16.8M-DoF meshes "
              "(same operators and inputs; the small arrays stay in cache, so the sample runs at least as fast "
              "per DoF as the full meshes would), DoFs/s = sample DoFs / mean step time" % n)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "DoFs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (uniform[-1,1] and Taylor-Green + seeded noise)",
            "config": {"workload": WORKLOAD, "degrees": [k for k, _ in SWEEP], "n_elem": [v for _, v in SWEEP],
                       "dofs_per_step": sum(4 * v ** 3 * (k + 1) ** 3 for k, v in SWEEP),
                       "l2": "flushed (256 MiB write) before every operator evaluation, outside its events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgns", choices=["dgns", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-mode", type=int, default=0, choices=sorted(MODES),
                    help="arithmetic of the headline sweep: 0 native FP64 (default), 1 double-float, "
                         "2 FP64-wide mix")
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
