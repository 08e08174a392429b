"""Pins for the oracle's Wing & Gong linearizability checker (CPU only).

Pinned against (a) hand-worked histories with known verdicts (tests/golden),
(b) an independent exhaustive search over all permutations written here, on
random tiny histories, and (c) planted mistakes in histories whose only valid
linearization is known, which the checker must reject.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ST = {"OK": 0, "FULL": 1, "EMPTY": 2}


def _load_cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "linearizability_cases.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        if f[0] == "case":
            kv = dict(x.split("=") for x in f[2:])
            cur = {"name": f[1], "cap": int(kv["cap"]), "expect": int(kv["expect"]), "ops": []}
            cases.append(cur)
        else:
            cur["ops"].append((f[0], 1 if f[1] == "enq" else 0, 0 if f[2] == "-" else int(f[2]),
                               ST[f[3]], int(f[4]), int(f[5])))
    return cases


def _arrays(ops):
    op = np.array([o[1] for o in ops], np.uint8)
    val = np.array([o[2] for o in ops], np.uint64)
    st = np.array([o[3] for o in ops], np.int8)
    call = np.array([o[4] for o in ops], np.uint64)
    end = np.array([o[5] for o in ops], np.uint64)
    return op, val, st, call, end


@pytest.mark.parametrize("case", _load_cases(), ids=lambda c: c["name"])
def test_hand_worked_verdicts(case):
    assert oracle.linearizable(*_arrays(case["ops"]), cap=case["cap"]) == case["expect"]


def brute_force(ops, cap):
    """Exhaustive search over all real-time-respecting permutations (independent of the oracle)."""
    n = len(ops)
    overlap = [sum(1 for j in range(n) if j != i and not (ops[j][5] < ops[i][4] or ops[i][5] < ops[j][4]))
               for i in range(n)]
    for perm in itertools.permutations(range(n)):
        pos = {o: k for k, o in enumerate(perm)}
        if any(ops[a][5] < ops[b][4] and pos[a] > pos[b] for a in range(n) for b in range(n)):
            continue
        q, good = [], True
        for o in perm:
            _, kind, v, st, _, _ = ops[o]
            if kind == 1 and st == 0:
                if cap and len(q) >= cap:
                    good = False; break
                q.append(v)
            elif kind == 1 and st == 1:
                if not (cap and len(q) + overlap[o] >= cap):
                    good = False; break
            elif kind == 0 and st == 2:
                if q:
                    good = False; break
            elif kind == 0 and st == 0:
                if not q or q[0] != v:
                    good = False; break
                q.pop(0)
            else:
                good = False; break
        if good:
            return 1
    return 0


def _random_history(rng, n, cap, linearizable_by_construction):
    """Random history: if by construction, results come from a sequential run at
    random linearization points inside random intervals."""
    points = sorted(rng.sample(range(1, 4 * n), n))
    q, ops = [], []
    nextv = 1
    for k, p in enumerate(points):
        lo = p - rng.randint(0, 3 * n)
        hi = p + rng.randint(0, 3 * n)
        lo = max(lo, 0)
        if rng.random() < 0.5:
            v = nextv; nextv += 1
            if cap and len(q) >= cap:
                ops.append(("P", 1, v, 1, lo, hi))
            else:
                q.append(v); ops.append(("P", 1, v, 0, lo, hi))
        else:
            if q:
                ops.append(("P", 0, q.pop(0), 0, lo, hi))
            else:
                ops.append(("P", 0, 0, 2, lo, hi))
    if not linearizable_by_construction:
        # random perturbation of one result
        i = rng.randrange(n)
        _, kind, v, st, lo, hi = ops[i]
        if kind == 0:
            ops[i] = ("P", 0, rng.randint(1, nextv), 0 if rng.random() < 0.7 else 2, lo, hi)
        else:
            ops[i] = ("P", 1, v, 1 - st if cap else st, lo, hi)
    return ops


@pytest.mark.parametrize("seed", range(6))
def test_agrees_with_exhaustive_search(seed):
    rng = random.Random(seed)
    seen = {0: 0, 1: 0}
    for trial in range(120):
        n = rng.randint(1, 7)
        cap = rng.choice([0, 0, 1, 2, 3])
        ops = _random_history(rng, n, cap, linearizable_by_construction=(trial % 2 == 0))
        want = brute_force(ops, cap)
        got = oracle.linearizable(*_arrays(ops), cap=cap)
        assert got == want, (ops, cap)
        if trial % 2 == 0:
            assert got == 1
        seen[want] += 1
    assert seen[0] > 5 and seen[1] > 5


def _sequential_history(rng, n):
    ops, q, v = [], [], 1
    for k in range(n):
        if rng.random() < 0.55 or not q:
            q.append(v); ops.append(("A", 1, v, 0, 10 * k, 10 * k + 5)); v += 1
        else:
            ops.append(("B", 0, q.pop(0), 0, 10 * k, 10 * k + 5))
    return ops


@pytest.mark.parametrize("mutation", ["swap", "duplicate", "lose", "early_empty", "foreign"])
def test_planted_mistakes_rejected(mutation):
    rng = random.Random(hash(mutation) & 0xFFFF)
    rejected = 0
    for _ in range(30):
        ops = _sequential_history(rng, 14)
        assert oracle.linearizable(*_arrays(ops)) == 1
        deqs = [i for i, o in enumerate(ops) if o[1] == 0]
        if len(deqs) < 2:
            continue
        bad = list(ops)
        a, b = sorted(rng.sample(deqs, 2))
        if mutation == "swap":
            bad[a], bad[b] = (bad[a][:2] + (ops[b][2],) + bad[a][3:], bad[b][:2] + (ops[a][2],) + bad[b][3:])
        elif mutation == "duplicate":
            bad[b] = bad[b][:2] + (ops[a][2],) + bad[b][3:]
        elif mutation == "lose":
            bad.append(("C", 0, 0, 2, 10 ** 6, 10 ** 6 + 1))  # final EMPTY although an item remains
            bad[b] = ("B", 0, 0, 2) + bad[b][4:]
        elif mutation == "early_empty":
            bad[a] = ("B", 0, 0, 2) + bad[a][4:]
        elif mutation == "foreign":
            bad[a] = bad[a][:2] + (10 ** 9,) + bad[a][3:]
        assert oracle.linearizable(*_arrays(bad)) == 0, (mutation, bad)
        rejected += 1
    assert rejected >= 20


def test_budget_and_bad_input():
    op = np.ones(64, np.uint8)
    z = np.zeros(64, np.uint64)
    assert oracle.linearizable(op, z, np.zeros(64, np.int8), z, z) == -2   # more than 63 ops
    assert oracle.linearizable([1], [1], [0], [5], [3]) == -2             # call after end
