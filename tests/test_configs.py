"""The workload configurations (configs.py) and the runner (run.py).

CPU: the configuration table expands to the runs the benchmark's
configurations describe, with the relaxation times of workloads.py. GPU: the
2-D Taylor-Green configuration run through the runner decays at the
viscosity c_s^2 (tau - 1/2) (closed form exp(-4 nu k^2 t) of the kinetic
energy, within 1% as the oracle's own decay pin), with its history lines.
"""
import json
import math

import pytest

from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import configs as C
from paper_1505_06900_gb300 import run as R
from paper_1505_06900_gb300 import workloads as W


def test_configuration_table_expands_to_the_workload_runs():
    rs = C.runs("tgv3d")
    assert [(r.n, r.mach) for r in rs] == [(256, 0.1), (256, 0.5), (512, 0.1), (512, 0.5)]
    assert all(r.lattice == B.D3Q27 and r.re == 1600.0 and r.steps == 5000 for r in rs)
    assert rs[2].tau() == W.taylor_green_3d_tau(512, 0.1, 1600.0)
    assert rs[2].shape == (512, 512, 512)
    sh = C.runs("shear2d_2048")
    assert [r.mach for r in sh] == [0.1, 0.3, 0.5] and sh[0].shape == (2048, 2048, 1)
    assert sh[0].tau() == pytest.approx(0.5 + 3.0 * 0.1 * math.sqrt(1 / 3) * 2048 / 1000)
    t2 = C.runs("tgv2d_128")[0]
    assert t2.tau() == W.taylor_green_2d_tau(128, 0.05, 100.0) and t2.u0 == 0.05
    assert C.runs("tgv3d_lowprec", storage="bf16")[0].storage == "bf16"
    assert C.runs("tgv3d_d3q19")[0].lattice == B.D3Q19
    over = C.runs("tgv3d", sizes=[64], machs=[0.3], steps=10, every=5)
    assert [(r.n, r.mach, r.steps, r.every) for r in over] == [(64, 0.3, 10, 5)]


def test_runner_lists_the_configurations(capsys):
    assert R.main(["--list"]) == 0
    out = capsys.readouterr().out
    for name in C.CONFIGS:
        assert name in out


@pytest.mark.gpu
def test_runner_tgv2d_decays_at_the_lattice_viscosity(tmp_path):
    out = tmp_path / "h.jsonl"
    assert R.main(["tgv2d_128", "--steps", "1000", "--every", "100", "--out", str(out)]) == 0
    lines = [json.loads(ln) for ln in out.read_text().splitlines()]
    hist = [ln for ln in lines if not ln.get("summary")]
    summary = [ln for ln in lines if ln.get("summary")][0]
    assert [h["step"] for h in hist] == list(range(0, 1001, 100))
    assert all(math.isfinite(h["kinetic_energy"]) and h["enstrophy"] > 0 for h in hist)
    assert abs(summary["nu_rel_error"]) < 1e-2
    assert summary["glups"] > 0
