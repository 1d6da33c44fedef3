"""Device memory reuse: a problem's state comes from a per-device pool that hands freed
memory to the next problem, so a state may start in memory that held another network's
iterates. Every buffer the kernels read must be written before it is read (rows, pads,
in-sums, partial sums), so a solve gives bitwise the same result in fresh and in reused
memory, in every kernel kind and storage type."""
import numpy as np
import pytest

from paper_2501_17996_gb300 import instances as I

pytestmark = pytest.mark.gpu

CASES = {
    # (instance, precision, shape): the register kind, the in-sum kind (rows of 8 KB or
    # more), BF16 storage and FP64
    "register_fp32": (lambda s: I.mid(s), "fp32", -1),
    "insum_fp32": (lambda s: I.ring_random_instance(2500, 10, s, "lognormal", "pow", gamma=0.5), "fp32", -1),
    "insum_bf16": (lambda s: I.ring_random_instance(2500, 10, s, "lognormal", "pow", gamma=0.5), "bf16", -1),
    "register_fp64": (lambda s: I.tiny(s), "fp64", -1),
}


def _solve(lib, inst, precision, shape):
    with lib.Problem(inst) as p:
        return p.solve(stop_mode="none", max_iters=120, k_check=40, precision=precision,
                       shape=shape, want_T=True, want_Y=True)


@pytest.mark.parametrize("case", sorted(CASES))
def test_solve_in_reused_memory_equals_first_solve(lib, case):
    make, precision, shape = CASES[case]
    a, other = make(0), make(1)
    first = _solve(lib, a, precision, shape)
    # another network of the same size leaves its iterates in the memory the pool hands out
    # next
    _solve(lib, other, precision, shape)
    again = _solve(lib, a, precision, shape)
    assert np.array_equal(first["T"], again["T"])
    assert np.array_equal(first["Y"], again["Y"])
    assert first["omega"] == again["omega"]
    assert first["rel_kkt"] == again["rel_kkt"] or (
        np.isinf(first["rel_kkt"]) and np.isinf(again["rel_kkt"]))


def test_many_problems_alive_and_freed(lib):
    """Problems created and destroyed in an interleaved order (memory returned to the pool
    while other states are alive) all reproduce their own solo results."""
    insts = [I.mid(s) for s in range(4)]
    solo = [_solve(lib, x, "fp32", -1)["T"] for x in insts]
    probs = [lib.Problem(x) for x in insts]
    try:
        out = {}
        for k in (2, 0, 3, 1):
            out[k] = probs[k].solve(stop_mode="none", max_iters=120, k_check=40, want_T=True)["T"]
            if k in (2, 3):
                probs[k].close()
        for k in range(4):
            assert np.array_equal(out[k], solo[k]), k
    finally:
        for p in probs:
            p.close()
