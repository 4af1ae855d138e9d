"""The Taylor-Green driver: energy diagnostics and the kinetic energy budget
of an early, resolved phase of the flow (the CFL time step is tested on the
CPU in tests/test_driver_host.py)."""
import pytest

from tests.gpu_common import build_lib

pytestmark = pytest.mark.gpu


def test_tgv_early_energy_budget():
    """Over t in [0, 0.5] the flow is smooth and resolved on 8^3 cells, k=3:
    e_k starts at 1/8, eps at 3 nu / 4, e_k decreases monotonically, and the
    energy budget closes: -de_k/dt matches eps to a few percent of eps (the
    numerical dissipation of the penalty terms and the LLF flux is small)."""
    build_lib()
    from paper_1802_01439_gb300.tgv import simulate
    meta, rec = simulate(8, 3, 0.5, every=1)
    nu = 1.0 / 1600
    assert rec[0]["e_k"] == pytest.approx(0.125, rel=1e-3)
    assert rec[0]["eps"] == pytest.approx(0.75 * nu, rel=1e-2)
    ek = [r["e_k"] for r in rec]
    assert all(b < a for a, b in zip(ek, ek[1:]))
    tail = rec[len(rec) // 2:]
    for r in tail:
        assert abs(r["eps_num"]) <= 0.05 * r["eps"], r
    assert meta["steps"] == len(rec) - 1
    assert all(sum(r["iterations"].values()) > 0 for r in rec[1:])
