"""Host logic of bench.py on the CPU: the bounded oracle sample behind `cpu_baseline` and the
reference arm (whole cycles for the 2D workloads, single SSP-RK3 steps of a lower-depth copy of the
3D configurations with one adaptation charged per adapt_every steps), the algorithmic work per
point the roofline uses, and the host description."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2306_06744_gb300 import workloads as W  # noqa: E402


def test_algorithmic_work_per_point():
    # element kernel, 3D p=3: primitives 13 + fluxes 18 + derivative 165 + RK 30 + traces 60
    assert bench.flops_per_point_stage(3, 3) == 286
    # read u_s, u^n, write the result (3 x 5 x 8 B) + read the common fluxes, write the traces
    # (2 x 6 x 5 / 4 values of 8 B)
    assert bench.bytes_per_point_stage(3, 3) == 240.0
    assert bench.bytes_per_point_stage(2, 3) == 160.0


def test_oracle_sample_keeps_the_configuration_but_the_depth():
    cfg = W.config("vortex3d_p3_multi")
    ocfg, whole, what = bench.oracle_sample(cfg, "vortex3d_p3_multi")
    assert not whole and ocfg["Dmax"] == bench.ORACLE_SAMPLE_DMAX["vortex3d_p3_multi"]
    for k in ("dim", "p", "L", "Dbase", "th_refine", "th_coarsen", "adapt_every"):
        assert ocfg[k] == cfg[k]
    assert (ocfg["vort"] == cfg["vort"]).all()
    c2 = W.config("vortex2d_p2_small")
    assert bench.oracle_sample(c2, "vortex2d_p2_small")[1]


@pytest.mark.parametrize("whole", [True, False])
def test_oracle_timer_rates(monkeypatch, whole):
    # a whole cycle of the small 2D workload, or single steps of a lower-depth 3D copy; the rate
    # is the DOF-updates over the charged time
    if whole:
        cfg, name = W.config("vortex2d_p2_small"), "vortex2d_p2_small"
    else:
        cfg = dict(W.config("vortex3d_p2_tube"), p=1, Dbase=2, Dmax=4)
        name = "vortex3d_p2_tube"
        monkeypatch.setitem(bench.ORACLE_SAMPLE_DMAX, name, 3)
    ot = bench.OracleTimer(cfg, name)
    ot.one(timed=False)
    M = ot.o.M
    ot.one()
    value, t = ot.finish()
    steps = cfg["adapt_every"] if whole else 1
    assert ot.steps == steps and t > 0
    assert abs(value * t - steps * M * ot.N * ot.nv) <= 1e-9 * value * t
    if not whole:
        assert ot.adapts == 1 and ot.t_adapt > 0  # one adaptation charged per adapt_every steps
    assert "SSP-RK3" in ot.sample_text()


def test_host_cpu():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["model"] and h["machine"]


def test_reference_arm_line(capsys, monkeypatch):
    # `bench.py --impl reference` on the small 2D workload (whole cycles of the oracle): one JSON
    # line with the reference arm's keys, the same config as the GPU arm's, and no host copies
    import json
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "vortex2d_p2_small",
                                      "--steps", "1", "--warmup", "3"])
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOAD)
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 3
    assert line["config"] == bench._config_line(W.config("vortex2d_p2_small"))
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
