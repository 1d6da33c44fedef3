"""One PDMCF iteration at the large configuration's full size (n = 10^4, m = 10^5, power
utility gamma = 1/2, FP32, the automatic launch configuration that bench.py times), checked on
sampled edges and nodes against the oracle's formulas (Eq. e-pdhg-step; Sec. 2.3 projection
and prox) applied in FP64 to the GPU's own state before that iteration. The state comes from
mcf_save_state (internal layout: F edge-major in mcf_problem_edge_order, Y as an FP32 head
plus a BF16 tail per row j = column j); the iteration's outputs F^ and Y^ come back through
the C ABI in the caller's layout. The oracle cannot run a whole iteration at this size; it
computes the sampled columns one by one."""
import os
import shutil

import numpy as np
import pytest

from oracle import pdmcf as O
from paper_2501_17996_gb300 import instances as I

pytestmark = pytest.mark.gpu

HEADER = 88   # magic[8], version, n, m, ld, precision, lo_live (int32), omega, hash, bytes[5]


def _read_state(path, n, m):
    with open(path, "rb") as f:
        head = f.read(HEADER)
    assert head[:8] == b"PDMCFWS1"
    ver, n_, m_, ld, prec, lo_live = np.frombuffer(head[8:32], dtype=np.int32)
    omega = float(np.frombuffer(head[32:40], dtype=np.float64)[0])
    sizes = np.frombuffer(head[48:88], dtype=np.uint64)
    assert (n_, m_, prec) == (n, m, 0) and ver == 1 and lo_live == 1
    off = HEADER
    F = np.memmap(path, dtype=np.float32, mode="r", offset=off, shape=(m, ld))
    off += int(sizes[0])
    Yhi = np.memmap(path, dtype=np.float32, mode="r", offset=off, shape=(n, ld))
    off += int(sizes[1])
    Ylo = np.memmap(path, dtype=np.uint16, mode="r", offset=off, shape=(n, ld))
    return F, Yhi, Ylo, omega, int(ld)


def _bf16(u16):
    return (u16.astype(np.uint32) << 16).view(np.float32)


def test_one_full_size_iteration_matches_the_oracle_on_samples(lib, tmp_path):
    inst = I.large(0)
    n, m = inst.n, inst.m
    if shutil.disk_usage(tmp_path).free < 12 * 2**30:
        pytest.skip("needs ~5 GB of scratch disk for the saved state")
    path = str(tmp_path / "large.pdmcf")
    with lib.Problem(inst) as p:
        p.solve(stop_mode="none", max_iters=60, k_check=50, want_T=False)
        p.save_state(path)
        g = p.solve(stop_mode="none", max_iters=1, k_check=1, warm_start=1,
                    want_T=False, want_F=True, want_Y=True)
        edge_of = p.edge_order()
        renumbered, _ = p.node_order()
    assert not renumbered                     # random chords keep the caller's numbering
    F, Yhi, Ylo, omega, ld = _read_state(path, n, m)
    eta = O.eta_bound(n, inst.tail, inst.head)
    alpha, beta = eta / omega, eta * omega
    row_of = np.empty(m, dtype=np.int64)      # caller edge -> internal row
    row_of[edge_of] = np.arange(m)

    def yfull(j):                             # column j of Y^k (FP32 head + BF16 tail)
        return Yhi[j, :n].astype(np.float64) + _bf16(Ylo[j, :n]).astype(np.float64)

    rng = np.random.default_rng(7)
    # edge phase: F^ column l = Pi(f_l + alpha (Y_{:,head} - Y_{:,tail}))
    e_err = 0.0
    for e in rng.choice(m, size=48, replace=False):
        ell = int(edge_of[e])
        q = F[e, :n].astype(np.float64) + alpha * (yfull(inst.head[ell]) - yfull(inst.tail[ell]))
        ref, _ = O.project_capped_simplex(q[:, None], inst.cap[ell:ell + 1])
        scale = max(np.abs(ref).max(), 1e-30)
        e_err = max(e_err, np.abs(g["F"][:, ell] - ref[:, 0]).max() / scale)
    # node phase: Y^ column j = prox(Y_{:,j} - beta (F+ A^T)_{:,j}), F+ = 2 F^ - F^{k-1/2}
    y_err = 0.0
    for j in rng.choice(n, size=24, replace=False):
        into = np.flatnonzero(inst.head == j)
        out = np.flatnonzero(inst.tail == j)
        fp = lambda ell: 2.0 * g["F"][:, ell] - F[row_of[ell], :n].astype(np.float64)
        s = sum(fp(ell) for ell in into) - sum(fp(ell) for ell in out)
        v = yfull(j) - beta * s
        keep = np.arange(n) != j
        ref = np.zeros(n)
        ref[keep] = O.prox_pow(v[keep], beta, inst.w[keep, j], inst.gamma)
        y_err = max(y_err, np.abs(g["Y"][:, j] - ref).max() / np.abs(ref).max())
    print(f"full size, iteration 61: edge phase F^ max error {e_err:.3g} of the column's scale "
          f"(48 edges), node phase Y^ {y_err:.3g} (24 nodes)")
    assert e_err <= 1e-6     # measured on GB300: 5.8e-8 (FP32 rounding of the inputs' use)
    assert y_err <= 1e-6     # measured: 5.8e-8
