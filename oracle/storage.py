"""SM-based storage, restated plainly -- TEST INFRASTRUCTURE ONLY.

Sec. 5.3 stores the RDF cube as one sparse matrix per predicate: M_h is the
m x 2 list of (s, o) pairs with (s, h, o) in the cube, m being the
predicate's statistic.  Sec. 6.3 adds auxiliary arrays per matrix and join
column: for every non-zero row, its id (Row), its number of entries (Num)
and the position of its first entry (Rpos, 1-based as printed).

Here the pairs of each M_h are listed sorted by (s, o); the paper's printed
matrices are in that order.
"""

from __future__ import annotations

import numpy as np


def unique_triples(triples) -> np.ndarray:
    """The triple set D (Sec. 3.1 defines a dataset as a set), sorted by
    (p, s, o)."""
    t = np.asarray(triples, dtype=np.int64).reshape(-1, 3)
    if t.shape[0] == 0:
        return t.astype(np.int32)
    order = np.lexsort((t[:, 2], t[:, 0], t[:, 1]))
    t = t[order]
    keep = np.ones(t.shape[0], dtype=bool)
    keep[1:] = np.any(t[1:] != t[:-1], axis=1)
    return t[keep].astype(np.int32)


def sparse_matrices(triples) -> dict:
    """{h: M_h} with M_h an (m, 2) int32 array of (s, o) rows (Sec. 5.3)."""
    t = unique_triples(triples)
    out = {}
    for h in np.unique(t[:, 1]):
        sel = t[t[:, 1] == h]
        out[int(h)] = sel[:, [0, 2]].copy()
    return out


def statistics(triples) -> dict:
    """Per predicate: m (= nnz of M_h, Sec. 5.3 'statistics'), and the
    numbers of distinct subjects and objects (non-zero rows by s and by o)."""
    out = {}
    for h, m in sparse_matrices(triples).items():
        out[h] = {
            "nnz": int(m.shape[0]),
            "nr_s": int(np.unique(m[:, 0]).size),
            "nr_o": int(np.unique(m[:, 1]).size),
        }
    return out


def aux_arrays(M: np.ndarray, col: int) -> np.ndarray:
    """Row/Num/Rpos of M on column ``col`` (0 = s side, 1 = o side), one
    (Row, Num, Rpos) triple per non-zero row, Rpos 1-based (Sec. 6.3).

    M is first ordered by (col, other column) so that each row's entries are
    contiguous; for col = 0 that is M_h's own order."""
    M = np.asarray(M)
    other = 1 - col
    order = np.lexsort((M[:, other], M[:, col]))
    key = M[order, col]
    rows, first, num = np.unique(key, return_index=True, return_counts=True)
    return np.stack([rows, num, first + 1], axis=1).astype(np.int64)


def csr_by(triples, side: str):
    """Per predicate, the doubly-compressed rows of M_h on one side.

    side 's' (CSR): rows are subjects, entries the objects; side 'o' (CSC):
    rows are objects, entries the subjects.  Returns {h: (row_ids, row_ptr,
    entries)} with entries sorted inside each row."""
    out = {}
    for h, m in sparse_matrices(triples).items():
        a, b = (0, 1) if side == "s" else (1, 0)
        order = np.lexsort((m[:, b], m[:, a]))
        keys = m[order, a]
        ent = m[order, b]
        rows, first = np.unique(keys, return_index=True)
        ptr = np.append(first, keys.size).astype(np.int64)
        out[h] = (rows.astype(np.int32), ptr, ent.astype(np.int32))
    return out
