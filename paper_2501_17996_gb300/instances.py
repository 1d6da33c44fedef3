"""Seeded synthetic instance generators for the all-pairs multicommodity flow problem.

This module only draws inputs (topology, capacities, utility weights); it holds none of
the method's arithmetic. Both the CUDA path and the CPU oracle consume its output.

Conventions (Zhang & Boyd, Sec. 1.1):
  * edge l goes from ``tail[l]`` to ``head[l]``; the incidence matrix has
    A[head[l], l] = +1 and A[tail[l], l] = -1;
  * ``w[i, j]`` is the utility weight of traffic from source j to destination i
    (the diagonal is unused and stored as 0);
  * utilities are ``w log s`` (``kind == "log"``) or ``w s**gamma`` (``kind == "pow"``),
    with ``gamma`` a scalar or an n x n array.

Workload recipes:
  * ``tiny``     n=10, directed ring plus 30 random chords (m=40), c~U[1,2], log, w~U[0.5,1.5]
  * ``mid``      n=100, ring plus 9 random out-edges per node (m=1000), c~U[1,10], log
  * ``large``    n=10000, ring plus 9 (m=100000), c~lognormal(0,0.5), power gamma=0.5
  * ``slice``    the ``large`` recipe at n=1000 (m=10000)
  * ``batched``  64 instances, n~U[50,400], out-degree~U[4,16], c~U[1,10], half log and
                 half power with gamma~U[0.3,0.7]
  * ``served``   n in {100,300,1000,3000}, out-degree 8, c~U[1,10], log
  * ``knn``      the paper's Sec. 3.1 family: points in the unit square, bidirectional
                 q-nearest-neighbour edges, log c~U[log .5, log 5], log w~U[log .3, log 3]
All draws come from ``numpy.random.default_rng(seed)`` (PCG64), which gives the same
stream on x86 and Arm.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    n: int
    tail: np.ndarray          # int32 [m]
    head: np.ndarray          # int32 [m]
    cap: np.ndarray           # float64 [m]
    kind: str                 # "log" | "pow"
    w: np.ndarray             # float64 [n, n], w[i, j] for traffic j -> i
    gamma: object = None      # None (log), float, or float64 [n, n]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.tail.shape[0])

    @property
    def nm(self) -> int:
        return self.n * self.m

    def copy(self) -> "Instance":
        g = self.gamma.copy() if isinstance(self.gamma, np.ndarray) else self.gamma
        return Instance(self.n, self.tail.copy(), self.head.copy(), self.cap.copy(),
                        self.kind, self.w.copy(), g, self.name, dict(self.meta))


def _skip_map(v: np.ndarray, excluded: list[int]) -> np.ndarray:
    """Map v in [0, n-len(excluded)) to [0, n) skipping the excluded node ids."""
    out = v.copy()
    for x in sorted(excluded):
        out[out >= x] += 1
    return out


def ring_plus_random(n: int, out_deg: int, rng: np.random.Generator):
    """Directed ring i -> i+1 plus (out_deg - 1) distinct random out-edges per node.

    No self loops and no duplicate (tail, head) pairs; the ring makes the graph
    strongly connected. Edges are listed node by node, ring edge first.
    """
    if out_deg < 1 or out_deg > n - 1:
        raise ValueError("out_deg must be in [1, n-1]")
    tails = np.empty(n * out_deg, dtype=np.int64)
    heads = np.empty(n * out_deg, dtype=np.int64)
    k = out_deg - 1
    pos = 0
    for i in range(n):
        nxt = (i + 1) % n
        tails[pos] = i
        heads[pos] = nxt
        pos += 1
        if k:
            excl = [i] if nxt == i else [i, nxt]
            v = rng.choice(n - len(excl), size=k, replace=False)
            tails[pos:pos + k] = i
            heads[pos:pos + k] = _skip_map(np.asarray(v, dtype=np.int64), excl)
            pos += k
    return tails.astype(np.int32), heads.astype(np.int32)


def ring_plus_chords(n: int, m: int, rng: np.random.Generator):
    """Directed ring plus (m - n) distinct random chords (no self loops, no duplicates)."""
    ring = {(i, (i + 1) % n) for i in range(n)}
    cand = [(j, i) for j in range(n) for i in range(n) if i != j and (j, i) not in ring]
    if m - n > len(cand):
        raise ValueError("too many chords")
    pick = rng.choice(len(cand), size=m - n, replace=False)
    pairs = [(i, (i + 1) % n) for i in range(n)] + [cand[p] for p in pick]
    t = np.array([p[0] for p in pairs], dtype=np.int32)
    h = np.array([p[1] for p in pairs], dtype=np.int32)
    return t, h


def _weights(n: int, rng: np.random.Generator, lo: float, hi: float, log_uniform=False):
    if log_uniform:
        w = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n, n)))
    else:
        w = rng.uniform(lo, hi, size=(n, n))
    np.fill_diagonal(w, 0.0)
    return w


def tiny(seed: int = 0) -> Instance:
    rng = np.random.default_rng(seed)
    n, m = 10, 40
    t, h = ring_plus_chords(n, m, rng)
    cap = rng.uniform(1.0, 2.0, size=m)
    w = _weights(n, rng, 0.5, 1.5)
    return Instance(n, t, h, cap, "log", w, None, f"tiny-s{seed}")


def ring_random_instance(n: int, out_deg: int, seed: int, cap_dist: str, kind: str,
                         gamma=None, name: str = "") -> Instance:
    rng = np.random.default_rng(seed)
    t, h = ring_plus_random(n, out_deg, rng)
    m = t.shape[0]
    if cap_dist == "u1_10":
        cap = rng.uniform(1.0, 10.0, size=m)
    elif cap_dist == "u1_2":
        cap = rng.uniform(1.0, 2.0, size=m)
    elif cap_dist == "lognormal":
        cap = rng.lognormal(mean=0.0, sigma=0.5, size=m)
    else:
        raise ValueError(cap_dist)
    w = _weights(n, rng, 0.5, 1.5)
    return Instance(n, t, h, cap, kind, w, gamma if kind == "pow" else None,
                    name or f"ring{n}x{out_deg}-s{seed}")


def mid(seed: int = 0) -> Instance:
    return ring_random_instance(100, 10, seed, "u1_10", "log", name=f"mid-s{seed}")


def large(seed: int = 0, n: int = 10000) -> Instance:
    return ring_random_instance(n, 10, seed, "lognormal", "pow", gamma=0.5,
                                name=f"large-n{n}-s{seed}")


def large_slice(seed: int = 0) -> Instance:
    """The large recipe at n=1000 (m=10000): the size the oracle can still run."""
    return large(seed, n=1000)


def batched(seed: int = 0, count: int = 64) -> list[Instance]:
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(50, 401))
        deg = int(rng.integers(4, 17))
        sub = int(rng.integers(0, 2**31 - 1))
        if b % 2 == 0:
            inst = ring_random_instance(n, deg, sub, "u1_10", "log", name=f"batched{b}")
        else:
            g = float(rng.uniform(0.3, 0.7))
            inst = ring_random_instance(n, deg, sub, "u1_10", "pow", gamma=g, name=f"batched{b}")
        out.append(inst)
    return out


def served_network(n: int, seed: int) -> Instance:
    return ring_random_instance(n, 8, seed, "u1_10", "log", name=f"served-n{n}-s{seed}")


def perturb(inst: Instance, nu: float, what: str, rng: np.random.Generator) -> Instance:
    """Multiply each capacity (what='cap') or weight (what='w') by 1+nu or 1-nu, each with
    probability 1/2 (the warm-start perturbation of Sec. 3.1)."""
    out = inst.copy()
    if what == "cap":
        s = rng.choice([-1.0, 1.0], size=out.m)
        out.cap = out.cap * (1.0 + nu * s)
    elif what == "w":
        s = rng.choice([-1.0, 1.0], size=(out.n, out.n))
        out.w = out.w * (1.0 + nu * s)
        np.fill_diagonal(out.w, 0.0)
    else:
        raise ValueError(what)
    return out


def knn(n: int, q: int, seed: int) -> Instance:
    """Sec. 3.1 workload: bidirectional edges between q-nearest neighbours of uniform
    points in the unit square, log-uniform capacities and weights, log utility."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    xi = rng.uniform(0.0, 1.0, size=(n, 2))
    _, nbr = cKDTree(xi).query(xi, k=q + 1)
    pairs = set()
    for i in range(n):
        for j in nbr[i, 1:]:
            j = int(j)
            if j != i:
                pairs.add((i, j))
                pairs.add((j, i))
    pairs = sorted(pairs)
    t = np.array([p[0] for p in pairs], dtype=np.int32)
    h = np.array([p[1] for p in pairs], dtype=np.int32)
    cap = np.exp(rng.uniform(np.log(0.5), np.log(5.0), size=len(pairs)))
    w = _weights(n, rng, 0.3, 3.0, log_uniform=True)
    return Instance(n, t, h, cap, "log", w, None, f"knn-n{n}-q{q}-s{seed}")


def two_node(ca: float, cb: float, kind="log", w12=1.0, w21=1.0, gamma=None) -> Instance:
    """Two nodes, edge 0: 0 -> 1 (capacity ca), edge 1: 1 -> 0 (capacity cb)."""
    w = np.array([[0.0, w12], [w21, 0.0]])
    return Instance(2, np.array([0, 1], np.int32), np.array([1, 0], np.int32),
                    np.array([ca, cb], float), kind, w, gamma, "two-node")


def directed_ring(n: int, c: float, w: float, kind="log", gamma=None) -> Instance:
    """Directed ring i -> i+1 with uniform capacity and weight."""
    t = np.arange(n, dtype=np.int32)
    h = ((np.arange(n) + 1) % n).astype(np.int32)
    W = np.full((n, n), float(w))
    np.fill_diagonal(W, 0.0)
    return Instance(n, t, h, np.full(n, float(c)), kind, W, gamma, f"ring{n}")


def random_small(n: int, m: int, seed: int, kind="log") -> Instance:
    """Small strongly connected instance (ring plus chords), for brute-force checks."""
    rng = np.random.default_rng(seed)
    t, h = ring_plus_chords(n, m, rng)
    cap = rng.uniform(0.5, 3.0, size=m)
    w = _weights(n, rng, 0.5, 2.0)
    gamma = float(rng.uniform(0.3, 0.7)) if kind == "pow" else None
    return Instance(n, t, h, cap, kind, w, gamma, f"small-n{n}-m{m}-s{seed}")


CONFIGS = {
    "tiny": tiny,
    "mid": mid,
    "large": large,
    "slice": large_slice,
}
