"""Failure detection on the device without a fault: the bulk-copy edge phase bounds every
mbarrier wait. mcf_test_withhold_next_copy makes one stage wait for copies that are never
issued (nothing is in flight for it), so the wait must give up within its limit, the kernel
must return, the solve must report MCF_ERR_CUDA, and the next solve on the same problem
must run normally and match the register shape's trajectory."""
import time

import numpy as np
import pytest

from paper_2501_17996_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _kind1_shape(lib, n):
    ld = (n + 7) // 8 * 8
    for s, (group, vpt, block, kind) in enumerate(lib.mcf_shape_info()):
        if kind == 1 and group * vpt >= ld // 4:
            return s
    pytest.skip("no bulk-copy shape covers this size")


def test_bounded_wait_gives_up_and_the_context_survives(lib):
    inst = I.large(0, n=1000)
    s1 = _kind1_shape(lib, inst.n)
    off = ~np.eye(inst.n, dtype=bool)
    with lib.Problem(inst) as p:
        lib.mcf_test_withhold_next_copy()
        t0 = time.perf_counter()
        with pytest.raises(lib.MCFError) as ei:
            p.solve(shape=s1, stop_mode="none", max_iters=1, k_check=1, use_graphs=0)
        waited = time.perf_counter() - t0
        assert ei.value.code == lib.MCF_ERR_CUDA
        assert "bounded device-side wait" in lib.mcf_last_error()
        assert waited < 30.0, waited          # 2 s wait + 2 s drain, plus start-up
        # the same problem, the same shape: a normal solve (cold) runs and is correct
        r = p.solve(shape=s1, stop_mode="none", max_iters=30, k_check=10, want_T=True)
        ref = p.solve(stop_mode="none", max_iters=30, k_check=10, want_T=True, shape=-1)
        assert r["iters"] == 30 and ref["iters"] == 30
        scale = np.abs(ref["T"][off]).max()
        assert np.abs(r["T"][off] - ref["T"][off]).max() <= 1e-4 * scale
