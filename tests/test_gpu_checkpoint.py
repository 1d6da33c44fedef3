"""Warm-state checkpoint (mcf_save_state / mcf_load_state) and the per-check diagnostics log
(mcf_options.check_log): a solve resumed from a saved state in a fresh problem equals the
uninterrupted warm solve bit for bit; the log has one line per stop test with the values the
result reports."""
import json

import numpy as np
import pytest

from paper_2501_17996_gb300 import instances as I

pytestmark = pytest.mark.gpu

CASES = {
    "mid_fp32": (lambda: I.mid(0), "fp32"),
    "tiny_fp64": (lambda: I.tiny(0), "fp64"),
    "insum_fp32": (lambda: I.ring_random_instance(2500, 10, 0, "lognormal", "pow", gamma=0.5), "fp32"),
    "insum_bf16": (lambda: I.ring_random_instance(2500, 10, 0, "lognormal", "pow", gamma=0.5), "bf16"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_resumed_solve_equals_uninterrupted(lib, tmp_path, case):
    make, precision = CASES[case]
    inst = make()
    opts = dict(stop_mode="none", k_check=50, precision=precision)
    path = str(tmp_path / "state.pdmcf")
    with lib.Problem(inst) as a:
        a.solve(max_iters=300, want_T=False, **opts)
        a.save_state(path)
        ra = a.solve(max_iters=200, warm_start=1, want_T=True, want_Y=True, **opts)
    with lib.Problem(inst) as b:
        b.load_state(path)
        rb = b.solve(max_iters=200, warm_start=1, want_T=True, want_Y=True, **opts)
    assert ra["iters"] == rb["iters"] == 200
    assert np.array_equal(ra["T"], rb["T"])
    assert np.array_equal(ra["Y"], rb["Y"])
    assert ra["omega"] == rb["omega"] and ra["rel_kkt"] == rb["rel_kkt"]


def test_state_of_another_network_is_refused(lib, tmp_path):
    path = str(tmp_path / "state.pdmcf")
    with lib.Problem(I.mid(0)) as a:
        a.solve(stop_mode="none", max_iters=20, k_check=10, want_T=False)
        a.save_state(path)
    with lib.Problem(I.mid(1)) as b:
        with pytest.raises(lib.MCFError) as ei:
            b.load_state(path)
        assert ei.value.code == lib.MCF_ERR_INVALID
        assert "different network" in lib.mcf_last_error()


def test_check_log_has_one_line_per_stop_test(lib, tmp_path):
    inst = I.mid(0)
    log = tmp_path / "checks.jsonl"
    with lib.Problem(inst) as p:
        r = p.solve(stop_mode="none", max_iters=200, k_check=50, check_log=str(log), want_T=False)
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["k"] for x in lines] == [50, 100, 150, 200]
    last = lines[-1]
    assert last["precision"] == "fp32" and last["omega"] == r["omega"]
    assert last["rel_kkt"] == r["rel_kkt"] or (last["rel_kkt"] is None and not np.isfinite(r["rel_kkt"]))
    assert 0.0 <= last["nonpos_frac"] <= 1.0 and isinstance(last["omega_adapting"], bool)
