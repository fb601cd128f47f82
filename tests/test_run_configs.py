"""The command-line runner (paper_2410_10503_gb300.run) and its configs: every
config parses and names a known workload; on the GPU a short run writes one
JSON line per epoch whose distance to x* falls."""
import glob
import json
import os
import subprocess
import sys

import pytest

import mc_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CONFIGS = sorted(glob.glob(os.path.join(ROOT, "paper_2410_10503_gb300", "configs", "*.json")))


def test_configs_parse_and_name_known_workloads():
    assert len(CONFIGS) == 5
    for path in CONFIGS:
        cfg = json.load(open(path))
        assert cfg["name"] and int(cfg["epochs"]) > 0
        if "batch" in cfg:
            assert int(cfg["batch"]["count"]) >= 1
        else:
            assert cfg["workload"] in S.WORKLOADS
            assert set(cfg["solvers"]) <= {"spdhg", "pdhg"}


@pytest.mark.gpu
def test_short_run_writes_a_falling_trace(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2410_10503_gb300 import build
    build.build()
    cfg = json.load(open(os.path.join(ROOT, "paper_2410_10503_gb300", "configs", "config1_rigid128.json")))
    cfg["epochs"] = 6
    cfg_path = tmp_path / "c.json"
    cfg_path.write_text(json.dumps(cfg))
    out = tmp_path / "t.jsonl"
    subprocess.run([sys.executable, "-m", "paper_2410_10503_gb300.run", str(cfg_path), "--out", str(out)],
                   check=True, cwd=ROOT)
    rows = [json.loads(l) for l in out.read_text().splitlines()]
    assert "x_star_cg_iterations" in rows[0]
    for solver in ("spdhg", "pdhg"):
        tr = [r for r in rows[1:] if r["solver"] == solver]
        assert [r["epoch"] for r in tr] == list(range(1, 7))
        assert tr[-1]["rel_err"] < tr[0]["rel_err"]
        assert all(r["seconds"] > 0 and "objective" in r for r in tr)
