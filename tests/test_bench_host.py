"""Host-side logic of bench.py (no GPU): the algorithmic flop and byte
counts behind the roofline figures, the clock-log parsing, and the JSON line
of the reference arm (the CPU oracle) on a small mesh."""
import argparse
import json
import os

import pytest

import bench


def _conv_cell_flops_by_phase(N, Q):
    """The cell kernel's algorithmic FP64 flops per cell, phase by phase
    (multiply-add = 2 flops): x and y interpolation of 3 components, then per
    z-plane the z interpolation, the 6 distinct products u_c u_d, the 8
    distinct x tests, the 9 y tests (two per component for Y1, one for Y3)
    and the z accumulation (two per output), and the face integrals added to
    the 6 face layers of 3 components."""
    fma_x = 3 * (N * N) * Q * N            # lines (c, y, z): Q outputs of N terms
    fma_y = 3 * (Q * N) * Q * N            # lines (c, qx, z)
    per_plane = (2 * (3 * Q * Q * N)       # z interpolation: 3 Q^2 points of N terms
                 + 6 * Q * Q               # products (one flop each)
                 + 2 * (8 * Q * N * Q)     # x tests: 8 tests x Q rows x N outputs x Q terms
                 + 2 * (9 * N * N * Q)     # y tests
                 + 2 * (3 * 2 * N ** 3))   # z accumulation
    return 2 * (fma_x + fma_y) + Q * per_plane + 6 * 3 * N * N


@pytest.mark.parametrize("N", [2, 3, 4, 5, 8, 12])
def test_conv_cell_flops_match_phase_count(N):
    Q = 3 * N // 2
    assert bench.conv_cell_flops(N, Q) == _conv_cell_flops_by_phase(N, Q)


def test_conv_cell_flops_bench_value():
    # k = 3: the figure quoted for the dominant kernel
    assert bench.conv_cell_flops(4, 6) == 41328


def _conv_face_flops_by_phase(N, Q):
    """The face kernel's algorithmic FP64 flops per face (multiply-add = 2
    flops): the traces of 3 components of both cells (the face layer's N^2
    nodal values interpolated along one tangential direction to Q N points,
    then along the other to Q^2, multiply-adds of N terms), the LLF flux at
    the Q^2 points (per component: two products, their sum, the halving, the
    jump, its product with the penalty and the final sum, 7 flops; 2 more for
    max(|a|, |b|)), the test of the 3 flux components with the face-layer
    basis (Q^2 -> N Q -> N^2, multiply-adds of Q terms), and the scaling of
    the 3 N^2 results by the face area."""
    traces = 2 * (6 * (Q * N) * N + 6 * (Q * Q) * N)
    flux = Q * Q * (3 * 7 + 2)
    tests = 2 * (3 * (N * Q) * Q + 3 * (N * N) * Q)
    return traces + flux + tests + 3 * N * N


@pytest.mark.parametrize("N", [2, 3, 4, 5, 8, 12])
def test_conv_face_flops_match_phase_count(N):
    Q = 3 * N // 2
    assert bench.conv_face_flops(N, Q) == _conv_face_flops_by_phase(N, Q)


def test_conv_face_flops_bench_value():
    assert bench.conv_face_flops(4, 6) == 5196


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


def test_reference_arm_line(monkeypatch):
    monkeypatch.setattr(bench, "N_ELEM", 2)
    line = bench.reference_arm(argparse.Namespace(steps=1, warmup=1), 0, 1)
    json.dumps(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert bench.reference_arm(argparse.Namespace(steps=1, warmup=1), 1, 2) is None   # other ranks


def test_reference_sample_bounds_the_run():
    # fits: the full mesh; 200 steps of 0.8 s: halved once (1/8 of the cost)
    assert bench.reference_sample_n(32, 0.5, 100, budget=150.0) == 32
    assert bench.reference_sample_n(32, 0.8, 200, budget=150.0) == 16
    assert bench.reference_sample_n(32, 0.8, 100000, budget=150.0) == 8      # floor
    assert bench.reference_sample_n(2, 10.0, 100, budget=1.0) == 2           # tiny meshes stay


def test_reference_arm_switches_to_a_sample(monkeypatch):
    """A budget the full mesh cannot meet makes every step run on the 8^3
    sample, and the line says so."""
    monkeypatch.setattr(bench, "N_ELEM", 16)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 1e-9)
    line = bench.reference_arm(argparse.Namespace(steps=1, warmup=3), 0, 1)
    assert "8^3-cell sample of the 16^3 workload" in line["cpu_baseline"]["sample"]
    assert line["value"] > 0 and line["config"]["n_elem"] == 16


def test_cpu_baseline_line(monkeypatch):
    monkeypatch.setattr(bench, "N_ELEM", 2)
    cb = bench.cpu_baseline(repeats=1)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["sample"].startswith("oracle") and "2^3 cells" in cb["sample"]
