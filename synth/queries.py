"""Seeded BGP workloads drawn from concrete instances of a synthetic graph.

A BGP is a list of triple patterns (s, p, o) whose subject and object are
either variables or constants; the predicate is always a constant, because
the method assumes known predicates (Sec. 6.3).  Every query is read off a
concrete subgraph instance of the graph (a walk, a star, a snowflake or a
closed walk), so its result is never empty; a constant, when a query has
one, is that instance's value at the replaced position.

Size control: for each query the generator computes an upper bound on the
number of rows that any connected sub-pattern can produce (a walk-count
dynamic program over a spanning forest of the sub-pattern; dropped cycle
edges and dropped membership tests only loosen the bound) and redraws the
query when the bound exceeds the configuration's row limit.  This keeps
every intermediate table of every join order within the limit, independent
of the planner.
"""

from __future__ import annotations

import dataclasses
import itertools
import os

import numpy as np

from .graphs import CONFIGS, GraphConfig, make_graph


@dataclasses.dataclass
class BGP:
    """A basic graph pattern.

    ``patterns`` holds tuples (s, p, o, s_is_var, o_is_var); a variable end
    stores its variable number in 0..n_vars-1, a constant end stores an
    entity id.  ``p`` is a predicate id.
    """

    patterns: list
    n_vars: int
    shape: str = ""
    name: str = ""

    def as_array(self) -> np.ndarray:
        """(n_patterns, 6) int64 array: s, p, o, s_var, p_var(0), o_var."""
        rows = [(s, p, o, int(sv), 0, int(ov)) for (s, p, o, sv, ov) in self.patterns]
        return np.asarray(rows, dtype=np.int64).reshape(-1, 6)

    def permuted(self, order) -> "BGP":
        return BGP([self.patterns[i] for i in order], self.n_vars, self.shape, self.name)


# ----------------------------------------------------------------------------
# adjacency used for sampling instances


class _Adjacency:
    def __init__(self, triples: np.ndarray, n_entities: int):
        t = np.asarray(triples)
        self.s = t[:, 0].astype(np.int64)
        self.p = t[:, 1].astype(np.int64)
        self.o = t[:, 2].astype(np.int64)
        self.n = t.shape[0]
        self.E = int(max(n_entities, int(t[:, [0, 2]].max()) + 1))
        self.by_s = np.argsort(self.s, kind="stable")
        self.by_o = np.argsort(self.o, kind="stable")
        self.s_ptr = np.searchsorted(self.s[self.by_s], np.arange(self.E + 1))
        self.o_ptr = np.searchsorted(self.o[self.by_o], np.arange(self.E + 1))
        # pair keys for adjacency tests in any orientation
        pair = self.s * self.E + self.o
        self.pair_sorted = np.sort(pair)
        self.preds = np.unique(self.p)

    def out_deg(self, v):
        return self.s_ptr[np.asarray(v) + 1] - self.s_ptr[np.asarray(v)]

    def in_deg(self, v):
        return self.o_ptr[np.asarray(v) + 1] - self.o_ptr[np.asarray(v)]

    def random_incident(self, rng, v, direction=None):
        """A random triple index incident to entity v; direction 'out', 'in'
        or None (either, proportional to degree).  Returns (idx, dir) or
        (None, None) when v has no such edge."""
        od, idg = int(self.out_deg(v)), int(self.in_deg(v))
        if direction == "out":
            idg = 0
        elif direction == "in":
            od = 0
        tot = od + idg
        if tot == 0:
            return None, None
        r = int(rng.integers(tot))
        if r < od:
            return int(self.by_s[self.s_ptr[v] + r]), "out"
        return int(self.by_o[self.o_ptr[v] + r - od]), "in"

    def has_pair(self, a, b):
        """Vectorised: is there a triple a->b (any predicate)?"""
        key = np.asarray(a, dtype=np.int64) * self.E + np.asarray(b, dtype=np.int64)
        pos = np.searchsorted(self.pair_sorted, key)
        pos = np.minimum(pos, self.pair_sorted.size - 1)
        return self.pair_sorted[pos] == key

    def find_pair(self, rng, a, b):
        """A random triple index with s=a, o=b, or None."""
        lo, hi = self.s_ptr[a], self.s_ptr[a + 1]
        idx = self.by_s[lo:hi]
        hit = idx[self.o[idx] == b]
        if hit.size == 0:
            return None
        return int(hit[rng.integers(hit.size)])


# ----------------------------------------------------------------------------
# instance templates: each returns a list of (subject_slot, triple_idx,
# object_slot) "edges" over instance slots plus slot -> entity values


def _inst_chain(adj, rng, hops):
    for _ in range(1000):
        t = int(rng.integers(adj.n))
        vals = [int(adj.s[t]), int(adj.o[t])]
        edges = [(0, t, 1)]
        ok = True
        for h in range(1, hops):
            cur = vals[-1]
            idx, d = adj.random_incident(rng, cur)
            if idx is None:
                ok = False
                break
            nxt_slot = len(vals)
            if d == "out":
                vals.append(int(adj.o[idx]))
                edges.append((h, idx, nxt_slot))
            else:
                vals.append(int(adj.s[idx]))
                edges.append((nxt_slot, idx, h))
        if ok:
            return edges, vals
    raise RuntimeError("could not sample a chain")


def _inst_star(adj, rng, k):
    for _ in range(1000):
        t = int(rng.integers(adj.n))
        x = int(adj.s[t])
        vals = [x]
        edges = []
        for _i in range(k):
            idx, _ = adj.random_incident(rng, x, "out")
            vals.append(int(adj.o[idx]))
            edges.append((0, idx, len(vals) - 1))
        return edges, vals
    raise RuntimeError("could not sample a star")


def _inst_snowflake(adj, rng, n_pat):
    # centre with a arms; 1-2 arm ends carry their own out-stars
    for _ in range(1000):
        t = int(rng.integers(adj.n))
        x = int(adj.s[t])
        n_arms = int(rng.integers(2, max(3, n_pat - 1)))
        n_arms = min(n_arms, n_pat - 1)
        vals = [x]
        edges = []
        for _i in range(n_arms):
            idx, _ = adj.random_incident(rng, x, "out")
            vals.append(int(adj.o[idx]))
            edges.append((0, idx, len(vals) - 1))
        rest = n_pat - n_arms
        arm_slots = list(range(1, n_arms + 1))
        rng.shuffle(arm_slots)
        ok = True
        j = 0
        while rest > 0:
            slot = arm_slots[j % len(arm_slots)]
            idx, _ = adj.random_incident(rng, vals[slot], "out")
            if idx is None:
                j += 1
                if j > 4 * len(arm_slots):
                    ok = False
                    break
                continue
            vals.append(int(adj.o[idx]))
            edges.append((slot, idx, len(vals) - 1))
            rest -= 1
        if ok and len(edges) == n_pat:
            return edges, vals
    raise RuntimeError("could not sample a snowflake")


def _inst_cycle(adj, rng, length):
    """A closed walk a0 - a1 - ... - a_{L-1} - a0, edges in any orientation."""
    batch = 4096
    for _ in range(200):
        t = rng.integers(adj.n, size=batch)
        path = [adj.s[t], adj.o[t]]
        for _h in range(length - 2):
            cur = path[-1]
            od = adj.out_deg(cur)
            idg = adj.in_deg(cur)
            tot = od + idg
            good = tot > 0
            r = (rng.random(batch) * np.maximum(tot, 1)).astype(np.int64)
            out_pick = r < od
            nxt = np.where(
                out_pick,
                adj.o[adj.by_s[np.minimum(adj.s_ptr[cur] + r, adj.n - 1)]],
                adj.s[adj.by_o[np.minimum(adj.o_ptr[cur] + np.maximum(r - od, 0), adj.n - 1)]],
            )
            nxt = np.where(good, nxt, -1)
            path.append(nxt)
        last, first = path[-1], path[0]
        valid = last >= 0
        closes = valid & (adj.has_pair(np.maximum(last, 0), first) | adj.has_pair(first, np.maximum(last, 0)))
        # prefer closed walks over distinct vertices
        P = np.stack(path, axis=1)
        distinct = np.array([len(set(row.tolist())) == length for row in P]) if closes.any() else closes
        cand = np.flatnonzero(closes & distinct)
        if cand.size == 0:
            cand = np.flatnonzero(closes)
        if cand.size == 0:
            continue
        row = P[int(cand[rng.integers(cand.size)])]
        vals = [int(v) for v in row]
        edges = []
        for h in range(length):
            a, b = vals[h], vals[(h + 1) % length]
            idx = adj.find_pair(rng, a, b)
            if idx is not None and (h > 0 or True):
                edges.append((h, idx, (h + 1) % length))
                continue
            idx = adj.find_pair(rng, b, a)
            if idx is None:
                break
            edges.append(((h + 1) % length, idx, h))
        if len(edges) == length:
            return edges, vals
    raise RuntimeError("could not sample a cycle")


# ----------------------------------------------------------------------------
# size bound


class _BoundIndex:
    """Per-predicate sparse 0/1 matrices for the walk-count bound."""

    def __init__(self, triples, n_entities):
        import scipy.sparse as sp

        t = np.asarray(triples)
        self.E = int(max(n_entities, int(t[:, [0, 2]].max()) + 1))
        self.mats = {}
        self.outdeg = {}
        self.indeg = {}
        order = np.argsort(t[:, 1], kind="stable")
        ps = t[order, 1]
        cuts = np.flatnonzero(np.diff(ps)) + 1
        for seg in np.split(order, cuts):
            if seg.size == 0:
                continue
            p = int(t[seg[0], 1])
            s = t[seg, 0].astype(np.int64)
            o = t[seg, 2].astype(np.int64)
            m = sp.csr_matrix((np.ones(seg.size, dtype=np.float32), (s, o)), shape=(self.E, self.E))
            self.mats[p] = m
            self.outdeg[p] = np.bincount(s, minlength=self.E).astype(np.float32)
            self.indeg[p] = np.bincount(o, minlength=self.E).astype(np.float32)
        self._mt = {}

    def mat_t(self, p):
        if p not in self._mt:
            self._mt[p] = self.mats[p].T.tocsr()
        return self._mt[p]


def _component_bound(bi: _BoundIndex, pats, var_set, ids=None, memo=None):
    """Upper bound on the rows of the sub-BGP ``pats`` (all vars in var_set
    connected through pats).  ``ids`` (positions of pats in their query) and
    ``memo`` let messages of identical subtrees be reused across the
    sub-BGPs of one query."""
    E = bi.E
    if ids is None:
        ids = list(range(len(pats)))
    if memo is None:
        memo = {}
    unary = {}
    unary_ids = {v: [] for v in var_set}
    adj = {v: [] for v in var_set}
    parent = {v: v for v in var_set}

    def find(v):
        while parent[v] != v:
            parent[v] = parent[parent[v]]
            v = parent[v]
        return v

    def unary_vec(pid, kind, p, c):
        key = ("u", pid)
        if key not in memo:
            m = bi.mats[p]
            vec = np.zeros(E, dtype=np.float32)
            if kind == "diag":
                vec = m.diagonal().astype(np.float32)
            elif kind == "col":
                if 0 <= c < E:
                    mt = bi.mat_t(p)
                    vec[mt.indices[mt.indptr[c]:mt.indptr[c + 1]]] = 1.0
            else:
                if 0 <= c < E:
                    vec[m.indices[m.indptr[c]:m.indptr[c + 1]]] = 1.0
            memo[key] = vec
        return memo[key]

    def mul_unary(v, vec, pid):
        unary[v] = vec if v not in unary else unary[v] * vec
        unary_ids[v].append(pid)

    for pid, (s, p, o, sv, ov) in zip(ids, pats):
        if p not in bi.mats:
            return 0.0
        if sv and ov:
            if s == o:
                mul_unary(s, unary_vec(pid, "diag", p, 0), pid)
            else:
                rs, ro = find(s), find(o)
                if rs != ro:
                    parent[rs] = ro
                    adj[s].append((o, p, "out", pid))  # s -p-> o
                    adj[o].append((s, p, "in", pid))
                # else: a cycle edge; dropping it keeps an upper bound
        elif sv:
            mul_unary(s, unary_vec(pid, "col", p, o), pid)
        elif ov:
            mul_unary(o, unary_vec(pid, "row", p, s), pid)
    root = max(var_set, key=lambda v: len(adj[v]))

    def subtree_ids(v, par):
        out = list(unary_ids[v])
        for (c, p, d, pid) in adj[v]:
            if c != par:
                out.append(pid)
                out.extend(subtree_ids(c, v))
        return out

    def f(v, par):
        vec = unary.get(v)
        for (c, p, d, pid) in adj[v]:
            if c == par:
                continue
            key = ("m", pid, d, frozenset(subtree_ids(c, v)))
            if key in memo:
                msg = memo[key]
            else:
                fc = f(c, v)
                if fc is None:
                    msg = bi.outdeg[p] if d == "out" else bi.indeg[p]
                else:
                    msg = (bi.mats[p] @ fc) if d == "out" else (bi.mat_t(p) @ fc)
                memo[key] = msg
            vec = msg if vec is None else vec * msg
        return vec

    top = f(root, None)
    return float(E) if top is None else float(top.sum(dtype=np.float64))


def _single_bound(bi: _BoundIndex, pt) -> float:
    """Rows of one pattern alone: nnz, a constant's row size, or (?x p ?x)
    the diagonal count."""
    s, p, o, sv, ov = pt
    if p not in bi.mats:
        return 0.0
    m = bi.mats[p]
    if sv and ov:
        return float(m.diagonal().sum()) if s == o else float(m.nnz)
    if sv:
        return float(bi.indeg[p][o]) if 0 <= o < bi.E else 0.0
    if ov:
        return float(bi.outdeg[p][s]) if 0 <= s < bi.E else 0.0
    return 1.0


def _pattern_vars(pt):
    s, p, o, sv, ov = pt
    vs = set()
    if sv:
        vs.add(s)
    if ov:
        vs.add(o)
    return vs


def _connected(pats):
    if not pats:
        return True
    seen_vars = set(_pattern_vars(pats[0]))
    left = list(pats[1:])
    changed = True
    while left and changed:
        changed = False
        for pt in list(left):
            vs = _pattern_vars(pt)
            if vs & seen_vars:
                seen_vars |= vs
                left.remove(pt)
                changed = True
    return not left


def _components(pats):
    comps = []
    for i, pt in enumerate(pats):
        vs = _pattern_vars(pt)
        merged = [c for c in comps if c[1] & vs]
        new = ([i], set(vs))
        for c in merged:
            comps.remove(c)
            new = (new[0] + c[0], new[1] | c[1])
        comps.append(new)
    return comps


def bgp_row_bound(bi: _BoundIndex, bgp: BGP, limit: float = float("inf")) -> float:
    """Max over join prefixes any planner may build: for every connected
    subset S of one component, bound(S) times the full bounds of the other
    components.  Returns early with a value above ``limit`` as soon as one
    subset exceeds it."""
    comps = _components(bgp.patterns)
    full = []
    sub_max = []
    memo = {}
    for idx, vars_ in comps:
        pats = [bgp.patterns[i] for i in idx]
        best = 0.0
        full_b = None
        for r in range(1, len(pats) + 1):
            for sub in itertools.combinations(range(len(pats)), r):
                sp_ = [pats[i] for i in sub]
                if not _connected(sp_):
                    continue
                vs = set().union(*[_pattern_vars(x) for x in sp_])
                if not vs:
                    b = 1.0
                elif len(sp_) == 1:
                    b = _single_bound(bi, sp_[0])
                else:
                    b = _component_bound(bi, sp_, vs, [idx[i] for i in sub], memo)
                if b > limit:
                    return b
                best = max(best, b)
                if r == len(pats):
                    full_b = b
        full.append(full_b if full_b is not None else best)
        sub_max.append(best)
    worst = 0.0
    for i in range(len(comps)):
        prod = sub_max[i]
        for j in range(len(comps)):
            if j != i:
                prod *= max(full[j], 1.0)
        worst = max(worst, prod)
    return worst


# ----------------------------------------------------------------------------
# instance -> BGP


def _to_bgp(adj, edges, vals, const_slot, shape):
    """Convert instance edges over slots into patterns; slot const_slot (or
    None) becomes a constant, other slots become variables numbered by first
    appearance."""
    var_of = {}
    pats = []
    for (a, t, b) in edges:
        p = int(adj.p[t])
        ends = []
        for slot in (a, b):
            if slot == const_slot:
                ends.append((vals[slot], False))
            else:
                if slot not in var_of:
                    var_of[slot] = len(var_of)
                ends.append((var_of[slot], True))
        pats.append((ends[0][0], p, ends[1][0], ends[0][1], ends[1][1]))
    return BGP(pats, len(var_of), shape)


_SHAPES = {
    "chain": _inst_chain,
    "star": _inst_star,
    "snowflake": _inst_snowflake,
    "cycle": _inst_cycle,
}


def _draw(adj, bi, rng, shape, n_pat, p_const, limit, max_tries=400, force_after=None):
    last = None
    if force_after is None:
        force_after = max_tries // 4
    for attempt in range(max_tries):
        edges, vals = _SHAPES[shape](adj, rng, n_pat)
        n_slots = len(vals)
        # later attempts force a constant: unselective draws are the ones
        # rejected by the bound
        use_const = rng.random() < p_const or attempt >= force_after
        const_slot = int(rng.integers(n_slots)) if use_const else None
        bgp = _to_bgp(adj, edges, vals, const_slot, shape)
        if bgp.n_vars == 0:
            continue
        b = bgp_row_bound(bi, bgp, limit)
        last = (bgp, b)
        if b <= limit:
            bgp.bound = b
            return bgp
    raise RuntimeError(f"no {shape}/{n_pat} query within {limit} rows (last bound {last[1] if last else None})")


_PLANS = {
    # (shape, n_patterns) per query
    "tiny": [("chain", 2), ("chain", 3), ("star", 3), ("chain", 2), ("chain", 3),
             ("star", 3), ("chain", 2), ("chain", 3), ("star", 3), ("cycle", 3)],
}

_LIMITS = {"tiny": 2_000_000, "medium": 100_000_000, "large": 1_000_000_000}
_PCONST = {"tiny": 0.5, "medium": 0.5, "large": 0.3}

_INDEX_CACHE: dict = {}


def _indexes(cfg, triples):
    key = (cfg.name, id(triples))
    if key not in _INDEX_CACHE:
        _INDEX_CACHE.clear()
        _INDEX_CACHE[key] = (_Adjacency(triples, cfg.n_entities), _BoundIndex(triples, cfg.n_entities))
    return _INDEX_CACHE[key]


def _plan_for(cfg: GraphConfig, rng):
    if cfg.name in _PLANS:
        return _PLANS[cfg.name]
    if cfg.name == "medium":
        plan = []
        for i in range(39):
            shape = ("star", "chain", "snowflake")[i % 3]
            lo = 4 if shape == "snowflake" else 3
            plan.append((shape, int(rng.integers(lo, 7))))
        plan.insert(int(rng.integers(40)), ("cycle", 4))
        return plan
    if cfg.name == "large":
        plan = []
        for i in range(20):
            shape = ("star", "chain", "snowflake", "star", "chain")[i % 5]
            plan.append((shape, int(rng.integers(4, 9))))
        return plan
    raise ValueError(cfg.name)


def make_queries(cfg: GraphConfig | str, triples: np.ndarray | None = None, seed: int | None = None):
    """The configuration's BGP workload (list of BGP)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if triples is None:
        triples = make_graph(cfg)
    seed = cfg.query_seed if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    adj, bi = _indexes(cfg, triples)
    out = []
    for qi, (shape, n_pat) in enumerate(_plan_for(cfg, rng)):
        bgp = _draw(adj, bi, rng, shape, n_pat, _PCONST[cfg.name], _LIMITS[cfg.name])
        bgp.name = f"{cfg.name}-q{qi:02d}-{shape}{n_pat}"
        out.append(bgp)
    return out


_BATCH_SHAPES = ["star"] * 4 + ["chain"] * 3 + ["snowflake"] * 2 + ["cycle"]


def _batched_one(adj, bi, seed, qi, limit):
    """Query qi of the batched mix; its own generator (seed, qi) makes the
    mix independent of how the queries are split over processes."""
    rng = np.random.Generator(np.random.PCG64([seed, qi]))
    shape = _BATCH_SHAPES[int(rng.integers(len(_BATCH_SHAPES)))]
    if shape == "cycle":
        n_pat = int(rng.integers(3, 5))
    elif shape == "snowflake":
        n_pat = int(rng.integers(3, 9))
    else:
        n_pat = int(rng.integers(2, 9))
    while True:
        try:
            bgp = _draw(adj, bi, rng, shape, n_pat, 0.5, limit, max_tries=12, force_after=3)
            break
        except RuntimeError:
            # no instance of this size within the limit: one pattern fewer
            n_pat -= 1
            if n_pat < (3 if shape == "cycle" else 2):
                shape, n_pat = "star", 2
    bgp.name = f"batched-q{qi:04d}-{shape}{n_pat}"
    return bgp


_WORKER = {}


def _batched_worker_init(limit):
    cfg = CONFIGS["medium"]
    t = make_graph(cfg)
    _WORKER["idx"] = _indexes(cfg, t)
    _WORKER["limit"] = limit


def _batched_worker(args):
    seed, lo, hi = args
    adj, bi = _WORKER["idx"]
    return [_batched_one(adj, bi, seed, qi, _WORKER["limit"]) for qi in range(lo, hi)]


def make_batched_queries(n_queries: int = 4096, triples: np.ndarray | None = None, seed: int = 7691 + 3,
                         limit: int = 1_000_000, workers: int | None = None):
    """Mixed workload over the medium graph: 2-8 patterns, shapes
    star:chain:snowflake:cycle = 4:3:2:1, 0-1 constants (constant-free
    patterns over this graph's hubs almost never stay within the limit).
    Each query has its own seeded generator, so the mix does not depend on
    ``workers`` (spawned processes that rebuild the medium graph)."""
    cfg = CONFIGS["medium"]
    if workers is None:
        workers = min(8, os.cpu_count() or 1) if n_queries >= 512 else 1
    if workers <= 1:
        if triples is None:
            triples = make_graph(cfg)
        adj, bi = _indexes(cfg, triples)
        return [_batched_one(adj, bi, seed, qi, limit) for qi in range(n_queries)]
    import multiprocessing as mp

    chunk = (n_queries + workers * 4 - 1) // (workers * 4)
    jobs = [(seed, lo, min(n_queries, lo + chunk)) for lo in range(0, n_queries, chunk)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_batched_worker_init, initargs=(limit,)) as pool:
        parts = pool.map(_batched_worker, jobs)
    return [q for part in parts for q in part]


# ----------------------------------------------------------------------------
# large configuration: anchored queries with exact frontier counts
#
# Dense walk-count vectors over 4x10^7 entities per predicate do not fit, so
# every large query is anchored at a constant (a star's centre, a chain's
# first vertex, a snowflake's centre) whose row is far shorter than the
# smallest predicate; the planner then starts at the anchor, and every plan
# prefix is a sub-pattern containing it, whose size is bounded below from the
# sparse frontier of walks out of the anchor.


class _LargeAdjacency:
    def __init__(self, triples: np.ndarray, n_entities: int):
        t = np.asarray(triples)
        self.n = t.shape[0]
        self.E = int(max(n_entities, int(t[:, [0, 2]].max()) + 1))
        s = t[:, 0]
        if np.all(s[1:] >= s[:-1]):
            self.by_s = None  # already in subject order
        else:
            self.by_s = np.argsort(s, kind="stable")
        ss = s if self.by_s is None else s[self.by_s]
        self.s_ptr = np.searchsorted(ss, np.arange(self.E + 1, dtype=np.int64))
        self.out_p = t[:, 1] if self.by_s is None else t[self.by_s, 1]
        self.out_o = t[:, 2] if self.by_s is None else t[self.by_s, 2]
        self.by_o = np.argsort(t[:, 2], kind="stable")
        self.o_ptr = np.searchsorted(t[self.by_o, 2], np.arange(self.E + 1, dtype=np.int64))
        self.in_p = t[self.by_o, 1]
        self.in_s = t[self.by_o, 0]
        self.preds, self.pred_nnz = np.unique(t[:, 1], return_counts=True)

    def edges(self, v, direction):
        """(predicates, neighbours) of entity v's out- or in-edges."""
        if direction == "out":
            a, b = self.s_ptr[v], self.s_ptr[v + 1]
            return self.out_p[a:b], self.out_o[a:b]
        a, b = self.o_ptr[v], self.o_ptr[v + 1]
        return self.in_p[a:b], self.in_s[a:b]

    def frontier_step(self, verts, mult, pred, direction, cap):
        """Multiset of neighbours (by pred, in direction) of a weighted vertex
        set; None if it would exceed cap entries."""
        ptr = self.s_ptr if direction == "out" else self.o_ptr
        lo, hi = ptr[verts], ptr[verts + 1]
        lens = hi - lo
        if int(lens.sum()) > cap:
            return None
        idx = np.repeat(lo - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(int(lens.sum()))
        P = self.out_p if direction == "out" else self.in_p
        N = self.out_o if direction == "out" else self.in_s
        w = np.repeat(mult, lens)
        keep = P[idx] == pred
        nb, ww = N[idx][keep], w[keep]
        if nb.size == 0:
            return np.zeros(0, np.int64), np.zeros(0, np.float64)
        u, inv = np.unique(nb, return_inverse=True)
        return u.astype(np.int64), np.bincount(inv, weights=ww)


def _large_one(adj, rng, shape, n_pat, limit, max_anchor_deg, min_bound=0.0):
    for _ in range(20000):
        t = int(rng.integers(adj.n))
        if shape in ("star", "snowflake"):
            c = int(np.searchsorted(adj.s_ptr, t, side="right") - 1)  # subject of entry t
            ps, os_ = adj.edges(c, "out")
            if ps.size == 0 or ps.size > max_anchor_deg:
                continue
            n_arms = n_pat if shape == "star" else max(2, n_pat // 2)
            picks = rng.integers(ps.size, size=n_arms)
            arms = [(int(ps[i]), int(os_[i])) for i in picks]
            pats = [(c, p, v, False, True) for v, (p, _) in enumerate(arms)]
            # degree of c per arm predicate
            factors = [float(np.sum(ps == p)) for p, _ in arms]
            if shape == "snowflake":
                n_sub = n_pat - n_arms
                next_var = n_arms
                arm_prod = {}  # arm -> per candidate, product of max(1, sub-degree) over its sub-patterns
                for j in range(n_sub):
                    a = j % n_arms
                    y = arms[a][1]
                    yp, _ = adj.edges(y, "out")
                    if yp.size == 0:
                        break
                    pb = int(yp[rng.integers(yp.size)])
                    pats.append((a, pb, next_var, True, True))
                    next_var += 1
                    # bound for the arm: sum over its candidates y of the
                    # product, over the arm's sub-patterns, of max(1, deg(y))
                    # (an arm with two sub-patterns multiplies their degrees)
                    ys = os_[ps == arms[a][0]].astype(np.int64)
                    lo, hi = adj.s_ptr[ys], adj.s_ptr[ys + 1]
                    degs = np.array([np.sum(adj.out_p[l:h] == pb) for l, h in zip(lo, hi)], dtype=np.float64)
                    arm_prod[a] = arm_prod.get(a, np.ones(ys.size)) * np.maximum(degs, 1.0)
                    factors[a] = float(arm_prod[a].sum()) if factors[a] > 0 else 0.0
                if len(pats) != n_pat:
                    continue
            bound = float(np.prod(factors))
            if bound > limit or bound < max(1.0, min_bound):
                continue
            exact = bound if shape == "star" else None
            return pats, next_var if shape == "snowflake" else n_arms, bound, exact
        # chain from an anchor: exact frontier counts hop by hop
        c = int(np.searchsorted(adj.s_ptr, t, side="right") - 1)
        if adj.s_ptr[c + 1] - adj.s_ptr[c] > max_anchor_deg:
            continue
        verts, mult = np.array([c], np.int64), np.array([1.0])
        pats, cur_slot, best = [], None, 0.0
        ok = True
        for h in range(n_pat):
            d = "out" if (h == 0 or rng.random() < 0.6) else "in"
            v0 = int(verts[rng.integers(verts.size)])
            ps, nbs = adj.edges(v0, d)
            if ps.size == 0:
                ok = False
                break
            pred = int(ps[rng.integers(ps.size)])
            step = adj.frontier_step(verts, mult, pred, d, cap=50_000_000)
            if step is None or step[0].size == 0:
                ok = False
                break
            verts, mult = step
            total = float(mult.sum())
            best = max(best, total)
            if best > limit:
                ok = False
                break
            src = (c, False) if h == 0 else (h - 1, True)
            dst = (h, True)
            if d == "out":
                pats.append((src[0], pred, dst[0], src[1], dst[1]))
            else:
                pats.append((dst[0], pred, src[0], dst[1], src[1]))
        if ok and best >= min_bound:
            return pats, n_pat, best, float(mult.sum())
    raise RuntimeError(f"no large {shape}/{n_pat} query")


def _disk_cached(kind, triples, params, build):
    """build() once per (triples, params, generator source) and keep the
    result on disk (the large workloads take minutes to draw and several
    processes need the same one).  GSMAT_SYNTH_CACHE names the folder ("0":
    off); the key holds a fingerprint of the triples (shape and a strided
    sample) and a digest of this package's source."""
    import hashlib
    import pickle
    import tempfile

    where = os.environ.get("GSMAT_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "gsmat_synth"))
    if where == "0":
        return build()
    t = np.asarray(triples)
    h = hashlib.sha256()
    h.update(repr((t.shape, str(t.dtype), params)).encode())
    step = max(1, t.shape[0] // 65536)
    h.update(np.ascontiguousarray(t[::step]).tobytes())
    here = os.path.dirname(os.path.abspath(__file__))
    for name in ("graphs.py", "queries.py"):
        with open(os.path.join(here, name), "rb") as f:
            h.update(f.read())
    path = os.path.join(where, f"{kind}_{h.hexdigest()[:24]}.pkl")
    if os.path.exists(path):
        try:
            with open(path, "rb") as f:
                return pickle.load(f)
        except (OSError, pickle.UnpicklingError, EOFError):
            pass
    out = build()
    try:
        os.makedirs(where, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "wb") as f:
            pickle.dump(out, f)
        os.replace(tmp, path)
    except OSError:
        pass
    return out


def make_large_queries(triples: np.ndarray | None = None, seed: int | None = None, n_queries: int = 20,
                       limit: float = 1e9):
    """The large configuration's 20 anchored BGPs (see _make_large_queries),
    kept on disk between processes."""
    cfg = CONFIGS["large"]
    if triples is None:
        triples = make_graph(cfg)
    seed = cfg.query_seed if seed is None else seed
    return _disk_cached("large_queries", triples, (seed, n_queries, limit),
                        lambda: _make_large_queries(triples, seed, n_queries, limit))


def _make_large_queries(triples: np.ndarray, seed: int, n_queries: int, limit: float):
    """20 anchored BGPs of 4-8 patterns over the large graph: stars,
    chains and snowflakes, from selective ones to intermediates of 10^8-10^9
    rows.  ``bgp.bound`` is the exact row count (stars, chains' largest
    frontier) or an upper bound (snowflakes)."""
    cfg = CONFIGS["large"]
    rng = np.random.Generator(np.random.PCG64(seed))
    adj = _LargeAdjacency(triples, cfg.n_entities)
    min_pred = int(adj.pred_nnz.min())
    out = []
    for qi in range(n_queries):
        shape = ("star", "chain", "snowflake", "star", "chain")[qi % 5]
        n_pat = int(rng.integers(4, 9)) if shape != "chain" else int(rng.integers(4, 7))
        # every fourth query is unselective: some plan prefix reaches 10^8 rows
        pats, n_vars, bound, exact = _large_one(adj, rng, shape, n_pat, limit,
                                                max_anchor_deg=min(min_pred // 4, 20000),
                                                min_bound=1e8 if qi % 4 == 3 else 0.0)
        bgp = BGP(pats, n_vars, shape, f"large-q{qi:02d}-{shape}{len(pats)}")
        bgp.bound = bound
        bgp.count = exact  # exact result rows (stars, chains) or None
        out.append(bgp)
    return out


def make_large_served_queries(triples: np.ndarray | None = None, n_queries: int = 2048, seed: int | None = None,
                              limit: float = 1e6, n_entities: int | None = None):
    """The served mix over the large graph (see _make_large_served_queries),
    kept on disk between processes."""
    cfg = CONFIGS["large"]
    if triples is None:
        triples = make_graph(cfg)
    seed = cfg.query_seed + 1 if seed is None else seed
    return _disk_cached("large_served", triples, (n_queries, seed, limit, n_entities),
                        lambda: _make_large_served_queries(triples, n_queries, seed, limit, n_entities))


def _make_large_served_queries(triples: np.ndarray, n_queries: int, seed: int, limit: float,
                               n_entities: int | None):
    """Served mix over the large graph: 2-8 patterns, shapes
    star:chain:snowflake = 4:3:2, each anchored at one constant whose row is
    short, every plan prefix bounded by ``limit`` rows (uneven selectivity:
    bounds from a few rows up to the limit).  The batched mix's 4-cycles are
    left out: closing a cycle needs a walk-count search that the sparse
    frontier sampler does not do."""
    cfg = CONFIGS["large"]
    rng = np.random.Generator(np.random.PCG64(seed))
    adj = _LargeAdjacency(triples, cfg.n_entities if n_entities is None else n_entities)
    shapes = ("star",) * 4 + ("chain",) * 3 + ("snowflake",) * 2
    out = []
    for qi in range(n_queries):
        shape = shapes[qi % len(shapes)]
        if shape == "star":
            n_pat = int(rng.integers(2, 9))
        elif shape == "chain":
            n_pat = int(rng.integers(2, 7))
        else:
            n_pat = int(rng.integers(4, 9))
        pats, n_vars, bound, exact = _large_one(adj, rng, shape, n_pat, limit, max_anchor_deg=2000)
        bgp = BGP(pats, n_vars, shape, f"large-s{qi:04d}-{shape}{len(pats)}")
        bgp.bound = bound
        bgp.count = exact
        out.append(bgp)
    return out
