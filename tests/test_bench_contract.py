"""bench.py on the CPU: the reference arm's JSON line (the oracle timed on host cores) and the
algorithmic-byte model used for the roofline."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "mid",
                          "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["n"] == 100 and line["config"]["m"] == 1000


def test_algorithmic_bytes_model():
    b = _bench_module()
    n, m = 10000, 100000
    a0 = b.algorithmic_bytes(n, m, 4, 4, kind=0)
    a2 = b.algorithmic_bytes(n, m, 4, 4, kind=2)
    assert a0["edge"] == 2 * 4 * n * m + 4 * n * n + 16 * m
    assert a0["node"] == 4 * n * m + 5 * 4 * n * n + 4 * (m + 2 * n)
    # the in-sum kinds' extra row of bytes is this design's, reported beside the method's
    assert a2["edge"] == a0["edge"] and a2["node"] == a0["node"]
    assert a2["design_extra"] == {"edge": 4 * n * n, "node": 4 * n * n}
    assert a0["design_extra"] == {"edge": 0.0, "node": 0.0}
    assert a0["iteration_floor"] == 2 * 4 * n * m + 3 * 4 * n * n


def test_knn_workload_is_strongly_connected():
    import numpy as np
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    b = _bench_module()
    inst = b.knn_connected(300, 10, 0)
    g = sp.coo_matrix((np.ones(inst.m), (inst.tail, inst.head)), shape=(inst.n, inst.n))
    assert connected_components(g, directed=True, connection="strong")[0] == 1
    assert set(zip(inst.tail.tolist(), inst.head.tolist())) == \
        set(zip(inst.head.tolist(), inst.tail.tolist()))   # edges both ways (Sec. 3.1)


def test_all_cores_oracle_matches_the_oracle():
    """oracle.parallel (the all-cores CPU baseline) performs the oracle's iterations: same
    F^{k+1/2}, Y^{k+1} and omega as oracle.pdmcf, to rounding, across an omega update."""
    import numpy as np

    from oracle import pdmcf as O
    from oracle.parallel import ParallelPDMCF
    from paper_2501_17996_gb300 import instances as I

    for inst in (I.mid(0), I.large(0, n=100)):
        K = 102   # omega adapts at k = 0 and k = 100
        ref = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                      stop_mode="none", max_iters=K, k_check=10**6)
        with ParallelPDMCF(inst, workers=3) as pp:
            F, Y, omega = pp.run(K)
        assert np.abs(F - ref.F).max() <= 1e-11 * np.abs(ref.F).max()
        assert np.abs(Y - ref.Y).max() <= 1e-11 * np.abs(ref.Y).max()
        assert abs(omega - ref.omega) <= 1e-11 * ref.omega


def test_oracle_with_the_parallel_step_matches_the_oracle():
    """oracle.pdmcf with oracle.parallel's step (the path make_golden.py uses for the large
    slice) reproduces the plain oracle: same stop, same iterations, T and U to rounding."""
    import numpy as np

    from oracle import pdmcf as O
    from oracle.parallel import ParallelPDMCF
    from paper_2501_17996_gb300 import instances as I

    inst = I.mid(0)
    kw = dict(eps=1e-3, stop_mode="kkt", max_iters=5000, k_check=50)
    ref = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma, **kw)
    with ParallelPDMCF(inst, workers=3) as pp:
        r = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                    step=pp.step, **kw)
        T, U, iters, om = r.T.copy(), r.utility, r.iters, r.omega
    assert iters == ref.iters and ref.status == "converged"
    assert np.abs(T - ref.T).max() <= 1e-9 * np.abs(ref.T).max()
    assert abs(U - ref.utility) <= 1e-11 * abs(ref.utility)
    assert abs(om - ref.omega) <= 1e-9 * ref.omega


def test_committed_traffic_captures_match_the_kernel_sources():
    """The DRAM bytes the bench reports as `roofline.traffic` come from the committed one-pass
    captures; each names the hash of the kernel sources it was taken on, and the bench uses it
    only while the hash matches. The committed captures are those of the current kernels."""
    bench = _bench_module()
    h = bench.kernel_source_hash()
    prof = os.path.join(ROOT, "profiles")
    caps = [f for f in os.listdir(prof) if f.startswith("edge_kernel_large_") and f.endswith(".json")]
    assert caps
    for f in caps:
        d = json.load(open(os.path.join(prof, f)))
        assert d["kernel_source_hash"] == h, f
        assert d["dram_bytes_per_launch"] == d["dram_bytes_read"] + d["dram_bytes_write"], f
        assert "--clock-control none" in d["command"], f
