"""Host-side logic of bench.py (no GPU): the algorithmic flop and byte
counts behind the roofline figures, the clock-log parsing, and the JSON line
of the reference arm (the CPU oracle) on a small mesh."""
import argparse
import json
import os

import numpy as np
import pytest

import bench


class _Counter:
    def __init__(self):
        self.fma = self.add = 0


def _even_odd_apply(A, x, cnt):
    """Applies the M x L matrix A (centrosymmetric: A[M-1-i, L-1-j] = A[i, j])
    to x in even-odd form, counting the operations: fold x into sums and
    differences of mirrored entries, contract the even and odd halves, and
    recombine mirrored outputs."""
    M, L = A.shape
    hl, hm = L // 2, M // 2
    e = [x[j] + x[L - 1 - j] for j in range(hl)] + ([x[hl]] if L % 2 else [])
    o = [x[j] - x[L - 1 - j] for j in range(hl)]
    cnt.add += 2 * hl
    # A = [[P, Q], [J Q J, J P J]] in blocks of mirrored rows/columns: the
    # even part uses (A[i, j] + A[i, L-1-j]) / 2-type half tables
    ye, yo = [], []
    for i in range(-(-M // 2)):
        acc = 0.0
        for j in range(hl):
            acc += 0.5 * (A[i, j] + A[i, L - 1 - j]) * e[j]
            cnt.fma += 1
        if L % 2:
            acc += A[i, hl] * e[hl]
            cnt.fma += 1
        ye.append(acc)
    for i in range(hm):
        acc = 0.0
        for j in range(hl):
            acc += 0.5 * (A[i, j] - A[i, L - 1 - j]) * o[j]
            cnt.fma += 1
        yo.append(acc)
    y = np.empty(M)
    for i in range(hm):
        y[i], y[M - 1 - i] = ye[i] + yo[i], ye[i] - yo[i]
    if M % 2:
        y[hm] = ye[hm]
    cnt.add += 2 * hm
    return y


@pytest.mark.parametrize("L,M", [(3, 3), (4, 4), (4, 6), (6, 4), (5, 7), (12, 18), (18, 12)])
def test_even_odd_line_count(L, M):
    """bench.eo_line counts exactly the operations of an even-odd contraction
    that reproduces the dense product of a centrosymmetric matrix."""
    rng = np.random.default_rng(L * 100 + M)
    B = rng.uniform(-1, 1, (M, L))
    A = 0.5 * (B + B[::-1, ::-1])                       # centrosymmetric
    x = rng.uniform(-1, 1, L)
    cnt = _Counter()
    y = _even_odd_apply(A, x, cnt)
    assert np.max(np.abs(y - A @ x)) < 1e-14
    assert (cnt.fma, cnt.add) == bench.eo_line(L, M)
    assert cnt.fma < L * M or L * M <= 2


def test_laplace_ops_k3_and_k11():
    # 8 sweeps of N^2 lines + 12 multiply-adds and 2 additions per DoF
    assert bench.laplace_ops(4) == (8 * 16 * 8 + 12 * 64, 8 * 16 * 8 + 2 * 64)
    assert bench.flops(bench.laplace_ops(4)) / 64 == 74.0           # 88 in direct form
    assert bench.flops(bench.laplace_ops(12)) / 12 ** 3 == pytest.approx(138.0)


def test_convective_ops_are_below_the_direct_form():
    for N in range(2, 13):
        Q = 3 * N // 2
        cc, cf = bench.conv_cell_ops(N, Q), bench.conv_face_ops(N, Q)
        direct_cell = (3 * (N * N * Q * N + Q * N * Q * N + Q * Q * Q * N)
                       + (8 * Q * Q + 9 * N * Q + 6 * N * N) * Q * N)
        assert cc[0] <= direct_cell
        assert cf[0] > 0 and cf[1] > 0
    # face: traces 6 (N + Q) lines N -> Q, flux 6 + 6 per point, tests 3 (Q + N) lines Q -> N
    assert bench.conv_face_ops(4, 6) == (6 * 10 * 12 + 6 * 36 + 3 * 10 * 12, 6 * 10 * 10 + 6 * 36 + 3 * 10 * 10)
    assert bench.conv_cell_ops(4, 6) == (3 * (16 + 24 + 36) * 12 + (8 * 36 + 9 * 24 + 6 * 16) * 12,
                                         3 * (16 + 24 + 36) * 10 + 6 * 216 + (8 * 36 + 9 * 24 + 6 * 16) * 10
                                         + 3 * 64 + 18 * 16)


def test_alu_fraction_by_mode():
    ops = (1000, 500)
    assert bench.alu_frac(ops, 1e-9, 0) == pytest.approx(2500e9 / 1e12 / bench.FP64_PEAK_TFLOPS)
    assert bench.alu_frac(ops, 1e-9, 1) == pytest.approx((15 * 1000 + 8 * 500) * 1e9 / 1e12 / bench.FP32_PEAK_TFLOPS)


def test_step_hbm_bytes_and_fraction():
    nu, npr = 2097152, 884736           # 32^3 cells, k_u = 3 (4^3 nodes), k_p = 2 (3^3)
    r = bench.step_hbm(nu, npr, 1.0)
    # each operator reads its input and writes its output once (doubles):
    # C, M^-1, H: 2 x 3 nu; D: 3 nu + np; L: 2 np; G: np + 3 nu
    assert r["algorithmic_bytes"] == 8 * (24 * nu + 4 * npr)
    assert r["achieved_GBps"] == pytest.approx(r["algorithmic_bytes"] / 1e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved_GBps"] / r["peak_GBps"], rel=1e-3)


def test_step_hbm_fallback_peak(monkeypatch):
    real_open = open

    def no_peaks(path, *a, **k):
        if str(path).endswith("MEASURED_PEAKS.json"):
            raise OSError("absent")
        return real_open(path, *a, **k)

    monkeypatch.setattr("builtins.open", no_peaks)
    r = bench.step_hbm(1000, 100, 1.0)
    assert r["peak_GBps"] == 6800.0 and "fallback" in r["peak_source"]


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_nvidia_smi_log(tmp_path):
    log = tmp_path / "clocks.csv"
    log.write_text("2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "1980, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                   "2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "garbage line\n")
    cs = bench.ClockSampler()
    cs.path, cs.proc = str(log), _DoneProc()
    r = cs.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert not os.path.exists(log)


def test_clock_sampler_without_process():
    assert bench.ClockSampler().stop() is None


SMALL_SWEEP = [(2, 4), (3, 4)]


def test_reference_arm_line(monkeypatch):
    monkeypatch.setattr(bench, "SWEEP", SMALL_SWEEP)
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 2)
    line = bench.reference_arm(argparse.Namespace(steps=1, warmup=1), 0, 1)
    json.dumps(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert bench.reference_arm(argparse.Namespace(steps=1, warmup=1), 1, 2) is None   # other ranks


def test_reference_sample_bounds_the_run():
    # fits: the full sample; 200 steps of 0.8 s: halved once (1/8 of the cost)
    assert bench.reference_sample_n(4, 0.5, 100, budget=150.0) == 4
    assert bench.reference_sample_n(4, 0.8, 200, budget=150.0) == 2
    assert bench.reference_sample_n(4, 0.8, 100000, budget=150.0) == 2      # floor
    assert bench.reference_sample_n(2, 10.0, 100, budget=1.0) == 2           # tiny meshes stay


def test_reference_arm_switches_to_a_sample(monkeypatch):
    """A budget the sample cannot meet halves it, and the line says so."""
    monkeypatch.setattr(bench, "SWEEP", SMALL_SWEEP)
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 4)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 1e-9)
    line = bench.reference_arm(argparse.Namespace(steps=1, warmup=3), 0, 1)
    assert "on a 2^3-cell sample" in line["cpu_baseline"]["sample"]
    assert line["value"] > 0 and line["config"]["degrees"] == [2, 3]


def test_cpu_baseline_line(monkeypatch):
    monkeypatch.setattr(bench, "SWEEP", SMALL_SWEEP)
    cb = bench.cpu_baseline(sample_n=2, repeats=1)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["sample"].startswith("oracle") and "2^3 cells" in cb["sample"]
