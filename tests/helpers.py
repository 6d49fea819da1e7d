"""Shared test helpers: brute force, invariants, random BGPs (CPU only)."""

from __future__ import annotations

import itertools
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def brute_force(triples, patterns, n_vars):
    """Every assignment of the variables over the active domain that puts
    every pattern's triple in D; rows sorted.  Independent of the oracle."""
    D = set(map(tuple, np.asarray(triples).tolist()))
    dom = sorted({t[0] for t in D} | {t[2] for t in D})
    rows = []

    def val(x, is_var, a):
        return a[x] if is_var else x

    for a in itertools.product(dom, repeat=n_vars):
        ok = True
        for (s, p, o, sv, ov) in patterns:
            if (val(s, sv, a), p, val(o, ov, a)) not in D:
                ok = False
                break
        if ok:
            rows.append(a)
    if n_vars == 0:
        return np.zeros((len(rows), 0), dtype=np.int64)
    return np.asarray(sorted(rows), dtype=np.int64).reshape(-1, n_vars)


def satisfies_all(triples, patterns, rows) -> bool:
    D = set(map(tuple, np.asarray(triples).tolist()))
    for r in np.asarray(rows).tolist():
        for (s, p, o, sv, ov) in patterns:
            if ((r[s] if sv else s), p, (r[o] if ov else o)) not in D:
                return False
    return True


def is_sorted_unique(rows) -> bool:
    r = np.asarray(rows)
    if r.shape[0] <= 1:
        return True
    for i in range(1, r.shape[0]):
        if tuple(r[i - 1]) >= tuple(r[i]):
            return False
    return True


def random_bgp(rng, triples, n_vars_max=4, n_pats_max=4, p_const=0.25, p_absent=0.05,
               p_selfloop=0.1, pred_pool=None):
    """A random BGP over small graphs (may be disconnected, may repeat a
    variable inside a pattern, may name an absent predicate or constant)."""
    t = np.asarray(triples)
    preds = np.unique(t[:, 1]) if pred_pool is None else np.asarray(pred_pool)
    ents = np.unique(np.concatenate([t[:, 0], t[:, 2]]))
    n_vars = int(rng.integers(1, n_vars_max + 1))
    n_pats = int(rng.integers(1, n_pats_max + 1))
    pats = []
    for _ in range(n_pats):
        p = int(rng.choice(preds)) if rng.random() > p_absent else int(preds.max()) + 17
        ends = []
        for _e in range(2):
            if rng.random() < p_const:
                c = int(rng.choice(ents)) if rng.random() > p_absent else int(ents.max()) + 5
                ends.append((c, False))
            else:
                ends.append((int(rng.integers(n_vars)), True))
        if rng.random() < p_selfloop and ends[0][1]:
            ends[1] = ends[0]
        pats.append((ends[0][0], p, ends[1][0], ends[0][1], ends[1][1]))
    # renumber used variables to 0..V-1 by first appearance
    remap = {}
    out = []
    for (s, p, o, sv, ov) in pats:
        if sv:
            s = remap.setdefault(s, len(remap))
        if ov:
            o = remap.setdefault(o, len(remap))
        out.append((s, p, o, sv, ov))
    return out, len(remap)
