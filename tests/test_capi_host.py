"""C ABI checks that need no GPU: the library loads, exports every declared symbol, and
rejects invalid input with the documented codes before touching a device."""
import json
import os
import re

import numpy as np
import pytest

from paper_2501_17996_gb300 import instances as I

from .conftest import HAS_GPU

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pdmcf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib.LIB, name), name
    assert set(names) == set(lib.SYMBOLS)


def test_options_defaults_are_the_paper_constants(lib):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    o = lib.mcf_options_default()
    assert o.rho == gold["rho"]["value"]
    assert o.theta == gold["theta"]["value"]
    assert o.k_adapt == gold["k_adapt"]["value"]
    assert o.tau == gold["tau"]["value"]
    assert o.omega0 == gold["omega0"]["value"]
    assert o.shape == -1 and o.precision == lib.MCF_FP32


def _create(lib, n, t, h, c, kind="log", w=None, gamma=None):
    if w is None:
        w = np.ones((n, n))
    return lib.mcf_create_problem(n, t, h, c, kind, w, gamma)


@pytest.mark.parametrize("case,code", [
    ("n1", -1), ("oob", -1), ("selfloop", -1), ("dup", -1), ("cap0", -1), ("capnan", -1),
    ("w0", -1), ("gamma_missing", -1), ("gamma_range", -1), ("disconnected", -2),
])
def test_invalid_problems_are_rejected(lib, case, code):
    n, t, h, c = 3, [0, 1, 2], [1, 2, 0], [1.0, 1.0, 1.0]
    kw = {}
    if case == "n1":
        n, t, h, c = 1, [0], [0], [1.0]
    elif case == "oob":
        h = [1, 2, 3]
    elif case == "selfloop":
        h = [0, 2, 0]
    elif case == "dup":
        t, h, c = [0, 1, 2, 0], [1, 2, 0, 1], [1.0] * 4
    elif case == "cap0":
        c = [1.0, 0.0, 1.0]
    elif case == "capnan":
        c = [1.0, float("nan"), 1.0]
    elif case == "w0":
        w = np.ones((3, 3))
        w[1, 2] = 0.0
        kw["w"] = w
    elif case == "gamma_missing":
        kw["kind"] = "pow"
    elif case == "gamma_range":
        kw["kind"] = "pow"
        kw["gamma"] = 1.5
    elif case == "disconnected":
        t, h, c = [0, 1], [1, 0], [1.0, 1.0]
    with pytest.raises(lib.MCFError) as ei:
        _create(lib, n, t, h, c, **kw)
    assert ei.value.code == code
    assert lib.mcf_last_error() != ""


def test_gamma_matrix_checked_off_the_diagonal_only(lib):
    n, t, h, c = 3, [0, 1, 2], [1, 2, 0], [1.0, 1.0, 1.0]
    g = np.full((n, n), 0.5)
    g[0, 0] = 7.0                                   # diagonal entries are not used
    lib.mcf_destroy_problem(_create(lib, n, t, h, c, kind="pow", gamma=g))
    g[2, 1] = 1.0
    with pytest.raises(lib.MCFError) as ei:
        _create(lib, n, t, h, c, kind="pow", gamma=g)
    assert ei.value.code == lib.MCF_ERR_INVALID and "gamma" in lib.mcf_last_error()


@pytest.mark.parametrize("row", [0, 1049, 2099])
def test_large_weight_matrix_checked_in_every_row(lib, row):
    """n = 2100 (35 MB of weights: the multi-threaded copy); one bad entry in any row is
    found, by creation and by an update, and a rejected update leaves the problem usable."""
    n = 2100
    t = np.arange(n, dtype=np.int32)
    h = ((t + 1) % n).astype(np.int32)
    c = np.ones(n)
    w = np.ones((n, n))
    bad = w.copy()
    bad[row, (row + 7) % n] = -1.0
    with pytest.raises(lib.MCFError) as ei:
        _create(lib, n, t, h, c, w=bad)
    assert ei.value.code == lib.MCF_ERR_INVALID
    with lib.Problem(I.Instance(n, t, h, c, "log", w, None, "ring2100")) as p:
        with pytest.raises(lib.MCFError) as ei:
            p.update_weights(bad)
        assert ei.value.code == lib.MCF_ERR_INVALID
        p.update_weights(w * 2.0)


def test_valid_problem_and_footprint(lib):
    inst = I.mid(0)
    with lib.Problem(inst) as p:
        b32 = p.device_bytes("fp32")
        b16 = p.device_bytes("bf16")
        b64 = p.device_bytes("fp64")
        ld = 104
        assert b32 >= 2 * inst.m * ld * 4 + 2 * inst.n * ld * 4
        assert b16 < b32 < b64


def test_invalid_options_are_rejected(lib):
    with lib.Problem(I.tiny(0)) as p:
        for bad in [dict(rho=2.0), dict(rho=0.0), dict(k_check=0), dict(max_iters=0),
                    dict(eps=0.0), dict(precision=7), dict(shape=99), dict(theta=1.5)]:
            with pytest.raises(lib.MCFError) as ei:
                p.solve(**bad)
            assert ei.value.code == lib.MCF_ERR_INVALID, bad


@pytest.mark.skipif(HAS_GPU, reason="checks the behaviour on a machine without a GPU")
def test_solve_without_gpu_fails_loudly(lib):
    with lib.Problem(I.tiny(0)) as p:
        with pytest.raises(lib.MCFError) as ei:
            p.solve()
        assert ei.value.code == lib.MCF_ERR_CUDA
    assert "no CUDA device" in lib.mcf_last_error() or "CUDA" in lib.mcf_last_error()


def test_shape_table(lib):
    shapes = lib.mcf_shape_info()
    assert len(shapes) >= 10
    for g, v, b, t in shapes:
        assert g in (32, 64, 128, 256, 512, 1024) and b % g == 0 and v >= 1 and t in (0, 1, 2)
    assert {t for *_, t in shapes} == {0, 1, 2}


def test_node_renumbering_rule(lib):
    """kNN networks (Sec. 3.1) get a bandwidth-reducing relabelling; random-chord networks,
    whose spans it cannot shorten 4x, keep the caller's numbering. The map is a permutation
    and the mean edge span drops at least 4x when it is used."""
    from paper_2501_17996_gb300 import instances as I
    knn = I.knn(400, 6, 0)
    for inst, expect in ((knn, True), (I.large(0, n=1000), False)):
        with lib.Problem(inst) as p:
            renumbered, node_of = p.node_order()
        assert renumbered == expect, inst.name
        assert sorted(node_of.tolist()) == list(range(inst.n))
        span0 = np.abs(inst.tail.astype(np.int64) - inst.head).mean()
        span1 = np.abs(node_of[inst.tail].astype(np.int64) - node_of[inst.head]).mean()
        if renumbered:
            assert 4 * span1 <= span0
        else:
            assert np.array_equal(node_of, np.arange(inst.n))


def test_readme_c_example_compiles_and_runs(lib, tmp_path):
    """The C example of README.md, built against include/pdmcf.h and libpdmcf.so: without a
    GPU the solve reports MCF_ERR_CUDA; with one it returns the two-node closed form
    (T_10 = c_a = 2, T_01 = c_b = 3, Sec. 1.1)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    readme = open(os.path.join(root, "README.md")).read()
    code = re.search(r"```c\n(.*?)```", readme, re.S).group(1)
    src = tmp_path / "example.c"
    src.write_text(code)
    from paper_2501_17996_gb300 import build as _build

    libdir = os.path.dirname(_build.LIB_PATH)
    exe = tmp_path / "example"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lpdmcf", f"-Wl,-rpath,{libdir}"],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    if "iters=" in out.stdout:
        t10 = float(re.search(r"T10=([\d.]+)", out.stdout).group(1))
        t01 = float(re.search(r"T01=([\d.]+)", out.stdout).group(1))
        assert abs(t10 - 2.0) < 1e-3 and abs(t01 - 3.0) < 1e-3
    else:
        assert not HAS_GPU and "solve: -4" in out.stdout


def test_renumbering_recovers_grid_locality(lib):
    """A 30 x 30 grid (edges both ways) with shuffled node labels: reverse Cuthill-McKee must
    bring the mean edge span back to the order of the grid side (30), from ~n/3 = 300."""
    rng = np.random.default_rng(0)
    side = 30
    n = side * side
    label = rng.permutation(n)
    tail, head = [], []
    for r in range(side):
        for c in range(side):
            v = r * side + c
            for dr, dc in ((0, 1), (1, 0)):
                if r + dr < side and c + dc < side:
                    u = (r + dr) * side + (c + dc)
                    tail += [label[v], label[u]]
                    head += [label[u], label[v]]
    tail = np.array(tail, np.int32)
    head = np.array(head, np.int32)
    w = np.ones((n, n))
    inst = I.Instance(n, tail, head, np.ones(len(tail)), "log", w, None, "grid")
    with lib.Problem(inst) as p:
        renumbered, node_of = p.node_order()
    assert renumbered
    span = np.abs(node_of[tail].astype(np.int64) - node_of[head]).mean()
    assert span <= 2 * side, span


def test_warm_state_file_errors_without_a_device(lib, tmp_path):
    """Saving needs a solved state; loading checks the file before touching the device."""
    from paper_2501_17996_gb300 import instances as I

    with lib.Problem(I.tiny(0)) as p:
        with pytest.raises(lib.MCFError) as ei:
            p.save_state(str(tmp_path / "none.pdmcf"))
        assert ei.value.code == lib.MCF_ERR_INVALID and "no solved state" in lib.mcf_last_error()
        with pytest.raises(lib.MCFError) as ei:
            p.load_state(str(tmp_path / "missing.pdmcf"))
        assert ei.value.code == lib.MCF_ERR_INVALID
        bad = tmp_path / "bad.pdmcf"
        bad.write_bytes(b"not a state file at all, not even close" * 4)
        with pytest.raises(lib.MCFError) as ei:
            p.load_state(str(bad))
        assert ei.value.code == lib.MCF_ERR_INVALID and "not a PDMCF" in lib.mcf_last_error()
