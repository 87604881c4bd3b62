"""Seeded synthetic 3-SAT inputs shared by the oracle tests and the CUDA path.

This module only draws instances and checks that their solution is unique; it
holds none of the evolution arithmetic.  Both sides consume its output (lists of
signed 1-based literals), so no oracle input ever comes from the CUDA path.

Planted unique-solution instances (the workloads stand in for the clause/variable
ratio ~4.2 instances of Sec. 4.3, which were never published):

1. ``rng = numpy.random.default_rng(seed)``; the planted assignment is
   ``rng.integers(0, 2**n)`` (bit i-1 is the value of x_i).
2. Candidate clauses are drawn one at a time: three distinct variables
   ``rng.choice(n, 3, replace=False)`` then three signs ``rng.integers(0, 2, 3)``
   (1 = positive literal).  A candidate is dropped if the planted assignment
   falsifies it, or if it repeats an earlier clause (same literal set).
3. Accepted clauses are appended until exactly one assignment (the planted one)
   satisfies every clause.

Adding clauses can only remove solutions, so "unique" is monotone in the number
of accepted clauses; the two counters below (incremental survivor filtering for
small n, a chunked first-kill scan over a pre-drawn clause stream for large n)
therefore stop at the same clause count for the same seed.
"""

import json
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
INSTANCE_DIR = os.path.join(_HERE, "instances")


class _ClauseStream:
    """The deterministic candidate stream of steps 1-2."""

    def __init__(self, n, seed):
        if n < 3:
            raise ValueError("planted 3-SAT needs n >= 3")
        self.n = n
        self.rng = np.random.default_rng(seed)
        self.planted = int(self.rng.integers(0, 1 << n, dtype=np.int64))
        self.seen = set()

    def _sat_by_planted(self, lits):
        for lit in lits:
            bit = (self.planted >> (abs(lit) - 1)) & 1
            if (lit > 0) == (bit == 1):
                return True
        return False

    def next(self):
        while True:
            vs = self.rng.choice(self.n, size=3, replace=False)
            signs = self.rng.integers(0, 2, size=3)
            lits = [int(v) + 1 if s else -(int(v) + 1) for v, s in zip(vs, signs)]
            if not self._sat_by_planted(lits):
                continue
            key = tuple(sorted(lits))
            if key in self.seen:
                continue
            self.seen.add(key)
            return lits


def _satisfied(x, lits):
    """Vectorised truth of one clause over an array of assignments."""
    ok = np.zeros(x.shape, dtype=bool)
    for lit in lits:
        bit = (x >> (abs(lit) - 1)) & 1
        ok |= (bit == 1) if lit > 0 else (bit == 0)
    return ok


def _generate_incremental(n, seed):
    st = _ClauseStream(n, seed)
    alive = np.arange(1 << n, dtype=np.int64)
    clauses = []
    while alive.size > 1:
        lits = st.next()
        clauses.append(lits)
        alive = alive[_satisfied(alive, lits)]
    return st.planted, clauses


def _last_needed_clause(n, clauses, planted, chunk_bits):
    """Index of the clause that eliminates the last non-planted assignment, or None."""
    worst = -1
    chunk = 1 << min(chunk_bits, n)
    for base in range(0, 1 << n, chunk):
        alive = np.arange(base, base + chunk, dtype=np.int64)
        alive = alive[alive != planted]
        for ci, lits in enumerate(clauses):
            if alive.size == 0:
                break
            keep = _satisfied(alive, lits)
            if not keep.all():
                worst = max(worst, ci)
            alive = alive[keep]
        if alive.size:
            return None
    return worst


def _generate_chunked(n, seed, chunk_bits=22):
    st = _ClauseStream(n, seed)
    target = int(3.0 * (7.0 * n / 3.0) * math.log(n)) + 64
    clauses = [st.next() for _ in range(target)]
    while True:
        last = _last_needed_clause(n, clauses, st.planted, chunk_bits)
        if last is not None:
            return st.planted, clauses[: last + 1]
        clauses.extend(st.next() for _ in range(target))


def planted_instance(n, seed, method="auto"):
    """Draw the planted unique-solution instance for (n, seed).

    Returns a dict with keys n, seed, planted, m, clauses (list of 3 literals).
    """
    if method == "auto":
        method = "incremental" if n <= 24 else "chunked"
    if method == "incremental":
        planted, clauses = _generate_incremental(n, seed)
    elif method == "chunked":
        planted, clauses = _generate_chunked(n, seed)
    else:
        raise ValueError(method)
    return {"n": n, "seed": seed, "planted": planted, "m": len(clauses),
            "clauses": clauses, "generator": "satgen planted-unique v1"}


def random_instance(n, m, seed, width=3):
    """m uniformly random clauses (no planting, no uniqueness): for edge-case tests."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(m):
        w = min(width, n)
        vs = rng.choice(n, size=w, replace=False)
        signs = rng.integers(0, 2, size=w)
        out.append([int(v) + 1 if s else -(int(v) + 1) for v, s in zip(vs, signs)])
    return out


def count_solutions(n, clauses, chunk_bits=22):
    """Number of assignments satisfying every clause (brute force, n <= 26)."""
    if n > 26:
        raise ValueError("brute-force counting is for n <= 26")
    total = 0
    chunk = 1 << min(chunk_bits, n)
    for base in range(0, 1 << n, chunk):
        alive = np.arange(base, base + chunk, dtype=np.int64)
        for lits in clauses:
            alive = alive[_satisfied(alive, lits)]
            if alive.size == 0:
                break
        total += int(alive.size)
    return total


def ratio_instance(n, seed, ratio=4.2, min_solutions=1):
    """Uniform random 3-SAT at a clause/variable ratio (Sec. 4.3 uses ~4.2,
    near the satisfiability threshold; those instances were never published).

    ``rng = default_rng(seed)``; m = round(ratio * n) clauses, each three distinct
    variables ``rng.choice(n, 3, replace=False)`` and signs ``rng.integers(0, 2,
    3)``, repeats allowed; no planted solution, so the ground state may be
    degenerate.  Instances with fewer than ``min_solutions`` satisfying
    assignments are redrawn from the same generator (deterministic per seed).
    Returns a dict with keys n, seed, m, clauses, solutions, draws.
    """
    rng = np.random.default_rng(seed)
    m = int(round(ratio * n))
    for draw in range(1, 10001):
        clauses = []
        for _ in range(m):
            vs = rng.choice(n, size=3, replace=False)
            signs = rng.integers(0, 2, size=3)
            clauses.append([int(v) + 1 if sg else -(int(v) + 1) for v, sg in zip(vs, signs)])
        sols = count_solutions(n, clauses)
        if sols >= min_solutions:
            return {"n": n, "seed": seed, "m": m, "clauses": clauses, "solutions": sols, "draws": draw,
                    "generator": f"satgen random 3-SAT ratio {ratio:g} v1"}
    raise RuntimeError("no instance with enough solutions in 10000 draws")


def block_instance(n, nblocks, distinct, repeated, seed):
    """A 3-SAT instance whose clauses never mix variables of different blocks.

    Variable x_v (1-based) belongs to block (v - 1) mod nblocks, so every block
    spans the low, middle and high bits of the basis index.  Per block, with
    ``rng = default_rng(seed)`` drawn in block order: a planted assignment of
    the block's variables (``rng.integers(0, 2, size)``), then ``distinct``
    clauses drawn as in the planted generator (three distinct block variables,
    three signs; dropped if the planted assignment falsifies them or if they
    repeat an earlier clause), then ``repeated`` clauses whose three literals
    are all true under the planted assignment (three distinct block variables,
    repeats allowed), so that the complement of the planted assignment violates
    at least ``nblocks * repeated`` clauses (large violated-clause counts).

    Because E(x) is the sum of the blocks' energies and every factor of the
    Strang step factorises over qubits, the evolved state is the tensor product
    of the blocks' states: full-size results can be checked block by block.
    Returns a dict with keys n, seed, m, clauses (global literals), planted
    (global index) and blocks (list of {vars, clauses: local literals 1..len(vars)}).
    """
    if nblocks < 1 or n < 3 * nblocks:
        raise ValueError("each block needs at least 3 variables")
    rng = np.random.default_rng(seed)
    blocks, clauses, planted = [], [], 0
    for b in range(nblocks):
        vs = [v for v in range(1, n + 1) if (v - 1) % nblocks == b]
        k = len(vs)
        pl = [int(t) for t in rng.integers(0, 2, size=k)]
        for i, bit in enumerate(pl):
            planted |= bit << (vs[i] - 1)
        local, seen = [], set()
        while len(local) < distinct:
            idx = rng.choice(k, size=3, replace=False)
            signs = rng.integers(0, 2, size=3)
            lits = [int(i) + 1 if sg else -(int(i) + 1) for i, sg in zip(idx, signs)]
            if not any((lit > 0) == (pl[abs(lit) - 1] == 1) for lit in lits):
                continue
            key = tuple(sorted(lits))
            if key in seen:
                continue
            seen.add(key)
            local.append(lits)
        for _ in range(repeated):
            idx = rng.choice(k, size=3, replace=False)
            local.append([int(i) + 1 if pl[int(i)] else -(int(i) + 1) for i in idx])
        blocks.append({"vars": vs, "clauses": local})
        for lits in local:
            clauses.append([vs[abs(lit) - 1] * (1 if lit > 0 else -1) for lit in lits])
    return {"n": n, "seed": seed, "m": len(clauses), "clauses": clauses, "planted": planted, "blocks": blocks,
            "generator": "satgen block-product v1"}


def save_instance(inst, path):
    with open(path, "w") as f:
        json.dump(inst, f, separators=(",", ":"))
        f.write("\n")


def load_instance(path_or_name):
    path = path_or_name
    if not os.path.exists(path):
        path = os.path.join(INSTANCE_DIR, path_or_name)
        if not path.endswith(".json"):
            path += ".json"
    with open(path) as f:
        return json.load(f)


def serving_requests(count=1024, seed=0, n_lo=10, n_hi=22, t_lo=5.0, t_hi=80.0, rate=None):
    """Request mix of the batched-serving workload: (arrival, n, T, instance seed).

    n ~ U{n_lo..n_hi}, T ~ U[t_lo, t_hi]; arrivals are a Poisson process of the
    given rate (requests per second; None = all at t = 0).
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    Ts = rng.uniform(t_lo, t_hi, size=count)
    inst_seeds = rng.integers(0, 2 ** 31 - 1, size=count)
    if rate is None:
        arrivals = np.zeros(count)
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    return [(float(a), int(n), float(T), int(s)) for a, n, T, s in zip(arrivals, ns, Ts, inst_seeds)]
