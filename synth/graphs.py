"""Seeded synthetic RDF graphs (int32 (s, p, o) triple sets).

An RDF dataset is a *set* of triples (Sec. 3.1), so every generator here
removes duplicates and returns exactly ``n_triples`` distinct rows in
generation order.  Entity ids and predicate ids live in separate id spaces,
as the two bijections h_so and h_p of Sec. 5.1 do; both are non-negative
int32.  Predicate ids are distinct random values, not 0..P-1, so that any
consumer has to look them up through an index rather than use them as
offsets.

Configurations (graph seed = 1807 + k):

* ``tiny``   (k=0): 10^4 entities, 8 predicates, 10^5 triples.  Subjects are
  taken in order 0, 1, 2, ...; each gets an out-degree drawn from a Zipf(1.5)
  law truncated to [1, 200]; predicates follow Zipf(1.1); objects are uniform.
* ``medium`` (k=1): 10^6 entities, 64 predicates, 10^7 triples, Chung-Lu
  style: subject and object ranks are drawn with weight (r + 1)^(-1/(alpha-1)),
  alpha = 2.1, through two independent random permutations of the entity ids;
  predicates follow Zipf(1.1).
* ``large``  (k=2): 4x10^7 entities, 256 predicates, 3x10^8 triples, the
  same laws with ranks drawn from the continuous power law's closed-form
  inverse CDF; returned in (s, p, o) key order (duplicates are removed by
  sorting and the surplus draws are dropped uniformly at random).
"""

from __future__ import annotations

import dataclasses
import os

import numpy as np


@dataclasses.dataclass(frozen=True)
class GraphConfig:
    name: str
    index: int  # k: graph seed is 1807 + k, query seed 7691 + k
    n_entities: int
    n_predicates: int
    n_triples: int
    model: str  # "zipf_subjects" | "chung_lu"
    alpha: float = 2.1  # power-law exponent of the Chung-Lu degree law
    out_zipf: float = 1.5  # tiny: out-degree law exponent
    out_cap: int = 200  # tiny: out-degree cap
    pred_zipf: float = 1.1

    @property
    def graph_seed(self) -> int:
        return 1807 + self.index

    @property
    def query_seed(self) -> int:
        return 7691 + self.index


CONFIGS = {
    "tiny": GraphConfig("tiny", 0, 10_000, 8, 100_000, "zipf_subjects"),
    "medium": GraphConfig("medium", 1, 1_000_000, 64, 10_000_000, "chung_lu"),
    "large": GraphConfig("large", 2, 40_000_000, 256, 300_000_000, "chung_lu"),
}


def _zipf_pmf(n: int, s: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


def _predicate_ids(rng: np.random.Generator, n: int) -> np.ndarray:
    """Distinct random predicate ids in [0, 2^24); rank r (0 = most frequent)
    maps to ids[r]."""
    ids = rng.choice(1 << 24, size=n, replace=False).astype(np.int64)
    return ids.astype(np.int32)


def _first_unique(keys: np.ndarray) -> np.ndarray:
    """Indices of the first occurrence of each distinct key, in input order."""
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return first


def _tiny(cfg: GraphConfig, rng: np.random.Generator) -> np.ndarray:
    pred_ids = _predicate_ids(rng, cfg.n_predicates)
    deg_pmf = _zipf_pmf(cfg.out_cap, cfg.out_zipf)
    pred_pmf = _zipf_pmf(cfg.n_predicates, cfg.pred_zipf)
    # Enough subjects for the target with margin; subjects are used in order.
    n_subj = min(cfg.n_entities, int(cfg.n_triples / 10.0 * 1.3))
    deg = rng.choice(np.arange(1, cfg.out_cap + 1), size=n_subj, p=deg_pmf)
    s = np.repeat(np.arange(n_subj, dtype=np.int64), deg)
    p = rng.choice(cfg.n_predicates, size=s.size, p=pred_pmf).astype(np.int64)
    o = rng.integers(0, cfg.n_entities, size=s.size, dtype=np.int64)
    keys = (s * cfg.n_predicates + p) * cfg.n_entities + o
    first = _first_unique(keys)
    if first.size < cfg.n_triples:
        raise RuntimeError("tiny generator ran out of subjects")
    first = first[: cfg.n_triples]
    out = np.empty((cfg.n_triples, 3), dtype=np.int32)
    out[:, 0] = s[first]
    out[:, 1] = pred_ids[p[first]]
    out[:, 2] = o[first]
    return out


def _power_law_ranks(u: np.ndarray, E: int, beta: float) -> np.ndarray:
    """Ranks r in [0, E) with density proportional to (r + 1)^(-beta): the
    closed-form inverse of the continuous law's CDF, floored (used for the
    large configuration, where a binary search per draw into an E-entry
    discrete CDF is too slow)."""
    g = 1.0 - beta
    hi = (E + 1.0) ** g
    x = (1.0 + u * (hi - 1.0)) ** (1.0 / g) - 1.0
    return np.minimum(x.astype(np.int64), E - 1)


def _chung_lu(cfg: GraphConfig, rng: np.random.Generator) -> np.ndarray:
    pred_ids = _predicate_ids(rng, cfg.n_predicates)
    E = cfg.n_entities
    expo = -1.0 / (cfg.alpha - 1.0)
    if cfg.n_triples >= 100_000_000:
        cdf = None
    else:
        w = (np.arange(E, dtype=np.float64) + 1.0) ** expo
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
    perm_out = rng.permutation(E).astype(np.int32)
    perm_in = rng.permutation(E).astype(np.int32)
    pred_cdf = np.cumsum(_zipf_pmf(cfg.n_predicates, cfg.pred_zipf))
    pred_cdf[-1] = 1.0
    # Draw with a surplus (hub pairs repeat) so that exactly n_triples
    # distinct remain; the surplus grows until it suffices.
    chunk = 1 << 24
    surplus = 1.10
    while True:
        n_draw = int(cfg.n_triples * surplus) + 1024
        s = np.empty(n_draw, dtype=np.int32)
        p = np.empty(n_draw, dtype=np.int16)
        o = np.empty(n_draw, dtype=np.int32)
        for a in range(0, n_draw, chunk):
            b = min(n_draw, a + chunk)
            if cfg.n_triples >= 100_000_000:
                s[a:b] = perm_out[_power_law_ranks(rng.random(b - a), E, -expo)]
                o[a:b] = perm_in[_power_law_ranks(rng.random(b - a), E, -expo)]
            else:
                s[a:b] = perm_out[np.searchsorted(cdf, rng.random(b - a), side="right").clip(0, E - 1)]
                o[a:b] = perm_in[np.searchsorted(cdf, rng.random(b - a), side="right").clip(0, E - 1)]
            p[a:b] = np.searchsorted(pred_cdf, rng.random(b - a), side="right").clip(0, cfg.n_predicates - 1)
        keys = (s.astype(np.int64) * cfg.n_predicates + p.astype(np.int64)) * E + o.astype(np.int64)
        if cfg.n_triples >= 100_000_000:
            # large sets: sort-based dedupe, then drop the surplus uniformly
            # at random (first-occurrence order would need an argsort)
            del s, p, o
            keys.sort()  # in place; numpy's hash-based unique is far slower here
            distinct = np.empty(keys.size, dtype=bool)
            distinct[0] = True
            np.not_equal(keys[1:], keys[:-1], out=distinct[1:])
            keys = keys[distinct]
            del distinct
            if keys.size >= cfg.n_triples:
                excess = keys.size - cfg.n_triples
                if excess:
                    drop = np.argpartition(rng.random(keys.size), excess)[:excess]
                    keep = np.ones(keys.size, dtype=bool)
                    keep[drop] = False
                    keys = keys[keep]
                out = np.empty((cfg.n_triples, 3), dtype=np.int32)
                out[:, 2] = (keys % E).astype(np.int32)
                keys //= E
                out[:, 1] = pred_ids[(keys % cfg.n_predicates).astype(np.int64)]
                out[:, 0] = (keys // cfg.n_predicates).astype(np.int32)
                return out
            del keys
            surplus *= 1.25
            continue
        first = _first_unique(keys)
        del keys
        if first.size >= cfg.n_triples:
            break
        surplus *= 1.25
    first = first[: cfg.n_triples]
    out = np.empty((cfg.n_triples, 3), dtype=np.int32)
    out[:, 0] = s[first]
    out[:, 1] = pred_ids[p[first].astype(np.int64)]
    out[:, 2] = o[first]
    return out


_CACHE: dict = {}

# Graphs of at least this many triples are also kept on disk (they take
# minutes to generate, and the tests and the benchmark need the same one in
# separate processes).  GSMAT_SYNTH_CACHE names the folder ("0" turns the
# disk cache off); the file name carries a digest of this module's source,
# so a changed generator never reads an old file.
_DISK_MIN_TRIPLES = 100_000_000


def _disk_path(cfg: GraphConfig, seed: int):
    import hashlib
    import tempfile

    where = os.environ.get("GSMAT_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "gsmat_synth"))
    if where == "0" or cfg.n_triples < _DISK_MIN_TRIPLES:
        return None
    with open(__file__, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()[:16]
    return os.path.join(where, f"{cfg.name}_{seed}_{cfg.n_triples}_{digest}.npy")


def make_graph(cfg: GraphConfig | str, seed: int | None = None, cache: bool = True) -> np.ndarray:
    """Return an (n_triples, 3) int32 array of distinct (s, p, o) triples."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    seed = cfg.graph_seed if seed is None else seed
    key = (cfg, seed)
    if cache and key in _CACHE:
        return _CACHE[key]
    path = _disk_path(cfg, seed) if cache else None
    g = None
    if path and os.path.exists(path):
        try:
            g = np.load(path)
            if g.shape != (cfg.n_triples, 3) or g.dtype != np.int32:
                g = None
        except (OSError, ValueError):
            g = None
    if g is None:
        rng = np.random.Generator(np.random.PCG64(seed))
        if cfg.model == "zipf_subjects":
            g = _tiny(cfg, rng)
        elif cfg.model == "chung_lu":
            g = _chung_lu(cfg, rng)
        else:
            raise ValueError(cfg.model)
        if path:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = f"{path}.{os.getpid()}.tmp"
                with open(tmp, "wb") as f:
                    np.save(f, g)
                os.replace(tmp, path)
            except OSError:
                pass  # no room or no permission: keep going without the disk copy
    g.setflags(write=False)
    if cache:
        _CACHE[key] = g
    return g


def small_random_graph(n_entities: int, n_predicates: int, n_triples: int, seed: int,
                       pred_ids: np.ndarray | None = None) -> np.ndarray:
    """A uniform random distinct triple set, for brute-force-sized tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if pred_ids is None:
        pred_ids = np.arange(n_predicates, dtype=np.int32)
    cap = n_entities * n_entities * n_predicates
    n_triples = min(n_triples, cap)
    flat = rng.choice(cap, size=n_triples, replace=False)
    s = flat // (n_entities * n_predicates)
    p = (flat // n_entities) % n_predicates
    o = flat % n_entities
    return np.stack([s, pred_ids[p], o], axis=1).astype(np.int32)


def graph_stats(triples: np.ndarray) -> dict:
    """Achieved shape statistics of a triple set (for reporting and checks)."""
    t = np.asarray(triples)
    ents = np.concatenate([t[:, 0], t[:, 2]])
    uniq, deg = np.unique(ents, return_counts=True)
    preds, pcount = np.unique(t[:, 1], return_counts=True)
    return {
        "n_triples": int(t.shape[0]),
        "n_entities_seen": int(uniq.size),
        "n_predicates": int(preds.size),
        "max_entity_id": int(ents.max()) if ents.size else -1,
        "frac_total_degree_le_43": float((deg <= 43).mean()) if deg.size else 1.0,
        "max_total_degree": int(deg.max()) if deg.size else 0,
        "top_predicate_share": float(pcount.max() / t.shape[0]) if t.shape[0] else 0.0,
        "min_predicate_share": float(pcount.min() / t.shape[0]) if t.shape[0] else 0.0,
    }
