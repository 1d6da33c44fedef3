"""Write the oracle's converged solutions used as expected values by the GPU parity tests.

Calls only the CPU oracle (oracle/) and the seeded input generators. Each case is solved
to a relative KKT measure of 1e-9 (or the stated tolerance) in float64; the file stores
T, Y^, the utility and the final metrics. The n = 1000 slice cases run oracle.pdmcf with
the update step of oracle.parallel (the same arithmetic on every host core).
Run: python tests/golden/make_golden.py [case...]
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pdmcf as O  # noqa: E402
from paper_2501_17996_gb300 import instances as I  # noqa: E402

PARALLEL = {"slice_s0_kkt1e-4", "slice_s0_kkt1e-6"}   # cases run with oracle.parallel's step

CASES = {
    # name: (instance factory, rel_kkt tolerance, iterations between stop tests)
    "tiny_s0": (lambda: I.tiny(0), 1e-10, 10),
    "mid_s0": (lambda: I.mid(0), 1e-9, 10),
    "midpow_s0": (lambda: I.large(0, n=100), 1e-9, 10),
    # stopped at the acceptance tolerance with the stop test every 50 iterations, as the
    # GPU solves they are compared with
    "mid_s0_kkt1e-4": (lambda: I.mid(0), 1e-4, 50),
    "midpow_s0_kkt1e-4": (lambda: I.large(0, n=100), 1e-4, 50),
    # the large recipe at n = 1000; its primal and dual values bracket the optimum U*
    "slice_s0_kkt1e-4": (lambda: I.large_slice(0), 1e-4, 50),
    # the same, close to the optimum: the reference T* for the slice
    "slice_s0_kkt1e-6": (lambda: I.large_slice(0), 1e-6, 50),
}


def make_adapt_history() -> str:
    """omega and rel_kkt at every stop test (k_check = 50) of the mid instance with the
    adaptation never stopped (adapt_guard = 0), 4000 iterations: the record the adaptation-stop
    pins read their trigger iterations from."""
    import json

    inst = I.mid(0)
    r = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                stop_mode="none", max_iters=4000, k_check=50, adapt_guard=0, history=True)
    rows = [[h["k"], h["omega"], h["rel_kkt"] if math.isfinite(h["rel_kkt"]) else None]
            for h in r.history]
    path = os.path.join(HERE, "adapt_history_mid_s0.json")
    with open(path, "w") as f:
        f.write('{"instance": "mid(0)", "k_check": 50, "adapt_guard": 0,\n'
                ' "columns": ["k", "omega", "rel_kkt"],\n "rows": [\n')
        f.write(",\n".join("  " + json.dumps(r) for r in rows))
        f.write("\n]}\n")
    print(f"adapt_history_mid_s0: {len(rows)} checks -> {path}", flush=True)
    return path


def make(name: str) -> str:
    if name == "adapt_history_mid_s0":
        return make_adapt_history()
    factory, tol, k_check = CASES[name]
    inst = factory()
    t0 = time.time()

    def progress(rec):
        if rec["k"] % 1000 == 0:
            print(f"  {name} k={rec['k']} omega={rec['omega']:.4g} rel_kkt={rec['rel_kkt']:.3g}",
                  flush=True)

    pool = None
    if name in PARALLEL:
        from oracle.parallel import ParallelPDMCF

        pool = ParallelPDMCF(inst, workers=int(os.environ.get("GOLDEN_WORKERS", "0")) or None)
    try:
        r = O.pdmcf(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w, inst.gamma,
                    eps=tol, stop_mode="kkt", max_iters=500000, k_check=k_check,
                    history=True, on_check=progress, step=pool.step if pool else None)
        T, Yhat = r.T.copy(), r.Yhat.copy()
    finally:
        if pool is not None:
            pool.close()
    path = os.path.join(HERE, f"oracle_{name}.npz")
    hk = np.array([h["k"] for h in r.history], dtype=np.int64)
    ho = np.array([h["omega"] for h in r.history])
    hr = np.array([h["rel_kkt"] for h in r.history])
    if name in PARALLEL:
        # the n = 1000 slice: T alone, rounded to float32 (relative 6e-8, far inside the 1e-3
        # it is compared at), keeps the file a few MB; Y^ is not compared at this size
        T, Yhat = T.astype(np.float32), np.zeros(0)
    np.savez_compressed(path, T=T, Yhat=Yhat, utility=r.utility, iters=r.iters,
                        rel_kkt=r.metrics.rel_kkt, rel_gap=r.metrics.rel_gap,
                        P=r.metrics.P, D=r.metrics.D,
                        status=r.status, omega=r.omega, omega_frozen_at=r.omega_frozen_at,
                        hist_k=hk, hist_omega=ho, hist_rel_kkt=hr)
    print(f"{name}: {r.status} iters={r.iters} rel_kkt={r.metrics.rel_kkt:.3g} "
          f"U={r.utility:.12g} {time.time() - t0:.1f}s -> {path}", flush=True)
    return path


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["tiny_s0", "mid_s0", "midpow_s0", "mid_s0_kkt1e-4",
                                  "midpow_s0_kkt1e-4"]):
        make(name)
