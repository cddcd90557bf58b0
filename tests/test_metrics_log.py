"""The per-step metrics log of the Python binding: one JSON line per step with
the step number, wall time, dt, status and every field of gf_step_stats (host
logic, no GPU)."""
import json

from paper_2103_14870_gb300 import graphfem


def test_metrics_line_holds_every_stat():
    stats = graphfem.StepStats().as_dict()
    stats.update(cg_iters=7, rel_res=3.5e-7, n_broken=12)
    rec = json.loads(graphfem.metrics_line(4, 5e-4, 0, stats))
    assert rec["step"] == 4 and rec["dt"] == 5e-4 and rec["status"] == 0
    assert rec["cg_iters"] == 7 and rec["rel_res"] == 3.5e-7 and rec["n_broken"] == 12
    assert set(stats) <= set(rec) and rec["time"] > 0
