"""Projection / DISTINCT on the device and SPARQL text end to end, against
the oracle (GPU)."""

import numpy as np
import pytest

import oracle
import synth
from oracle import frontend as fe
from tests.helpers import golden, random_bgp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch

    torch.cuda.init()
    import paper_1807_07691_b300 as g

    return g


@pytest.fixture(scope="module")
def tiny(gs):
    t = synth.make_graph("tiny")
    return t, oracle.OracleIndex(t), gs.Store(t), synth.make_queries("tiny", t)


def test_dg_text_end_to_end(gs):
    g, t = golden("dg_example.json"), golden("dg_text.json")
    d = gs.Dictionary(t["data"])
    S = gs.Store(d.triples())
    rows = S.sparql(t["query"], d).to_numpy()
    assert rows.tolist() == g["answer_xyzw"]
    x, y, z, w = rows[0]
    assert d.decode([x, w, z, y]) == t["answer_decoded_XWZY"]
    # Select|Project: (X, W) only, and DISTINCT over X
    P = S.sparql("SELECT ?x ?w WHERE { ?x :follows ?y . ?y :follows ?z . ?x :likes ?w . ?z :likes ?w }", d)
    assert d.decode_rows(P.to_numpy()) == [("A", "I2")]
    D = S.sparql("SELECT DISTINCT ?s { ?s :follows ?o }", d)
    assert d.decode_rows(D.to_numpy()) == [("A",), ("B",), ("C",)]
    B = S.sparql("SELECT ?s { ?s :follows ?o }", d)
    assert [r[0] for r in d.decode_rows(B.to_numpy())] == ["A", "B", "B", "C"]
    # a constant the dictionary does not hold matches nothing
    assert S.sparql("SELECT ?s { ?s :follows nobody }", d).shape == (0, 1)


def _subsets(rng, V):
    k = int(rng.integers(1, V + 1))
    return [int(v) for v in rng.permutation(V)[:k]]


def test_project_tiny_workload(gs, tiny):
    t, ix, S, qs = tiny
    rng = np.random.default_rng(2)
    n_sorted_path = 0
    for q in qs:
        want_rows = ix.query(q)
        T = S.query(q)
        V = q.n_vars
        cases = [list(range(V)), list(range(max(1, V - 1))), [V - 1]] + [_subsets(rng, V) for _ in range(3)]
        for vs in cases:
            for distinct in (False, True):
                got = T.project(vs, distinct).to_numpy()
                want = fe.project(want_rows, vs, distinct)
                assert got.shape == want.shape and np.array_equal(got, want), (q.name, vs, distinct)
                n_sorted_path += vs == list(range(len(vs)))
        # a table in plan column order projects the same way
        P = S.query(q, flags=gs.PLAN_ORDER)
        for vs in cases[:4]:
            got = P.project(vs, True).to_numpy()
            assert np.array_equal(got, fe.project(want_rows, vs, True))
    assert n_sorted_path > 0


@pytest.mark.parametrize("seed", range(12))
def test_project_random_bgps(gs, tiny, seed):
    t, ix, S, qs = tiny
    rng = np.random.default_rng(900 + seed)
    for _ in range(10):
        pats, V = random_bgp(rng, t, n_vars_max=5, n_pats_max=4, p_const=0.3)
        if V == 0:
            continue  # nothing to project
        try:
            want_rows = ix.query(pats, V, row_limit=3_000_000)
        except oracle.OracleError:
            continue
        T = S.query(pats, V)
        vs = _subsets(rng, V)
        d = bool(rng.random() < 0.6)
        got = T.project(vs, d).to_numpy()
        assert np.array_equal(got, fe.project(want_rows, vs, d)), (pats, vs, d)


def test_project_edge_cases(gs, tiny):
    t, ix, S, qs = tiny
    q = qs[0]
    T = S.query(q)
    with pytest.raises(gs.GsmatError):
        T.project([q.n_vars])  # not a column
    with pytest.raises(gs.GsmatError):
        T.project([0, 0])
    with pytest.raises(gs.GsmatError):
        T.project([])
    with pytest.raises(gs.GsmatError):
        S.query(q, flags=gs.COUNT_ONLY).project([0])
    E = S.query([(0, 987654, 1, 1, 1)], 2)  # absent predicate: empty
    assert E.project([1], True).shape == (0, 1)
    one = gs.Store(np.array([(5, 1, 6)], dtype=np.int32)).query([(0, 1, 1, 1, 1)], 2)
    assert one.project([1, 0], True).to_numpy().tolist() == [[6, 5]]


def test_sparql_text_random_queries(gs, tiny):
    """BGPs written as SPARQL text with decimal codes (no dictionary):
    the parsed query gives the oracle's projected relation."""
    t, ix, S, qs = tiny
    rng = np.random.default_rng(17)
    n = 0
    while n < 30:
        pats, V = random_bgp(rng, t, n_vars_max=4, n_pats_max=4, p_const=0.3)
        if V == 0:
            continue  # SELECT needs a variable
        try:
            want_rows = ix.query(pats, V, row_limit=3_000_000)
        except oracle.OracleError:
            continue
        body = " . ".join(f"{'?v%d' % s if sv else s} {p} {'?v%d' % o if ov else o}" for (s, p, o, sv, ov) in pats)
        vs = _subsets(rng, V)
        d = bool(rng.random() < 0.5)
        text = f"SELECT {'DISTINCT ' if d else ''}{' '.join('?v%d' % v for v in vs)} WHERE {{ {body} }}"
        q = gs.Sparql(text)
        # variables renumbered by first occurrence in the text
        first = []
        for (s, p, o, sv, ov) in pats:
            for x, isv in ((s, sv), (o, ov)):
                if isv and x not in first:
                    first.append(x)
        assert q.var_names == ["v%d" % x for x in first]
        got = S.sparql(q).to_numpy()
        assert np.array_equal(got, fe.project(want_rows, vs, d)), text
        n += 1


def test_dictionary_graph_end_to_end(gs):
    """A small graph written as text: encoded, loaded, queried by SPARQL
    text and decoded, against the oracle's front end and join."""
    rng = np.random.default_rng(4)
    lines = ["@prefix ex: <http://x.org/> ."]
    for _ in range(400):
        s, o = int(rng.integers(0, 60)), int(rng.integers(0, 60))
        p = int(rng.integers(0, 4))
        lines.append(f"ex:n{s} ex:r{p} ex:n{o} .")
    data = "\n".join(lines)
    d = gs.Dictionary(data)
    od = fe.Dictionary()
    codes = od.add_text(data)
    assert np.array_equal(d.triples(), codes)
    S = gs.Store(d.triples())
    text = ("PREFIX ex: <http://x.org/> SELECT DISTINCT ?a ?c WHERE "
            "{ ?a ex:r0 ?b . ?b ex:r1 ?c . ?c ex:r2 ?a }")
    q = fe.parse_sparql(text, od)
    rows = oracle.OracleIndex(codes).query(q["patterns"], q["n_vars"])
    want = fe.project(rows, q["projection"], q["distinct"])
    got = S.sparql(text, d).to_numpy()
    assert np.array_equal(got, want)
    assert d.decode_rows(got) == [tuple(od.decode_so(v) for v in r) for r in want.tolist()]
