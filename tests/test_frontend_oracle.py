"""Pins of the oracle's front end (encoding, data and SPARQL text,
projection) against the paper's worked example, hand-written expectations
and brute force (CPU only)."""

import itertools

import numpy as np
import pytest

import oracle
from oracle import frontend as fe
from tests.helpers import golden

RT = fe.RDF_TYPE


# --------------------------------------------------------------------------
# Sec. 5.2 encoding and the D_G example end to end


def test_dg_codes_are_the_papers():
    """h_p, h_so (Fig. 'The construction of h_p and h_so') and the cube
    (Table 'The RDF Cube C_{D_G}'): codes by order of first occurrence."""
    g, t = golden("dg_example.json"), golden("dg_text.json")
    d = fe.Dictionary()
    codes = d.add_text(t["data"])
    assert d.h_p == g["h_p"]
    assert d.h_so == g["h_so"]
    assert codes.tolist() == g["cube_spo"]


def test_dg_query_text_and_decoded_answer():
    """The example query (Sec. 3.2) parses to the BGP of dg_example.json and
    its answer decodes to (A, I2, C, B) over (X, W, Z, Y) (Sec. 6.3)."""
    g, t = golden("dg_example.json"), golden("dg_text.json")
    d = fe.Dictionary()
    d.add_text(t["data"])
    q = fe.parse_sparql(t["query"], d)
    assert [list(p) for p in q["patterns"]] == g["query"]
    assert q["var_names"] == g["query_vars"] and q["n_vars"] == 4
    assert q["projection"] == [0, 1, 2, 3] and not q["distinct"]
    rows = oracle.OracleIndex(np.array(d.triples)).query(q["patterns"], q["n_vars"])
    x, y, z, w = rows[0]
    assert [d.decode_so(v) for v in (x, w, z, y)] == t["answer_decoded_XWZY"]


def test_codes_start_at_one_and_subject_before_object():
    d = fe.Dictionary()
    got = d.add_text("<b> <p> <a> .\n<a> <q> <c> .\n<c> <p> <b> .")
    # b=1, a=2 (subject first), c=3; p=1, q=2
    assert got.tolist() == [[1, 1, 2], [2, 2, 3], [3, 1, 1]]
    # a second text continues both numberings
    assert d.add_text("<d> <r> <a> .").tolist() == [[4, 3, 2]]
    assert 0 not in d.h_so.values() and 0 not in d.h_p.values()


# --------------------------------------------------------------------------
# data text


def test_data_forms():
    text = """@prefix ex: <http://e/> .
    # a comment
    ex:a a ex:C ; ex:p "x y"@en-GB , "3"^^ex:int ; ex:q _:b1 .
    <http://e/a> ex:p "say \\"hi\\"" .
    _:b1 <http://e/q> ex:a.
    :likes :likes :likes .
    """
    got = fe.parse_data(text)
    assert got == [
        ("<http://e/a>", RT, "<http://e/C>"),
        ("<http://e/a>", "<http://e/p>", '"x y"@en-GB'),
        ("<http://e/a>", "<http://e/p>", '"3"^^<http://e/int>'),
        ("<http://e/a>", "<http://e/q>", "_:b1"),
        ("<http://e/a>", "<http://e/p>", '"say \\"hi\\""'),
        ("_:b1", "<http://e/q>", "<http://e/a>"),
        (":likes", ":likes", ":likes"),
    ]


@pytest.mark.parametrize("text", [
    "<a> <p> <b>",            # no final '.'
    "<a> <p> .",              # missing object
    "<a b> <p> <c> .",        # whitespace in an IRI
    '<a> <p> "open .',        # unterminated literal
    '"lit" <p> <b> .',        # literal subject
    "<a> <p> ?x .",           # variable in data
    "@prefix ex <http://e/> .",  # bad directive
    '<a> <p> "x"^^ .',        # empty datatype
    ". <a> <p> <b> .",        # lone '.'
])
def test_data_errors(text):
    with pytest.raises(fe.FrontEndError) as e:
        fe.parse_data(text)
    assert e.value.kind == "invalid"


# --------------------------------------------------------------------------
# SPARQL text


def _dict_with(*terms_so, preds=()):
    d = fe.Dictionary()
    for i, t in enumerate(terms_so):
        d.h_so[t] = i + 1
    for i, p in enumerate(preds):
        d.h_p[p] = i + 1
    return d


def test_sparql_forms():
    d = _dict_with("<http://e/a>", '"v"@en', preds=("<http://e/p>", "<http://e/q>", RT))
    q = fe.parse_sparql("""PREFIX ex: <http://e/>
        select distinct $y ?x where {
          ?x ex:p ex:a , "v"@en ; ex:q ?y ; a ?z .   # comment
          ?y <http://e/p> ?x }""", d)
    # x=0, y=1, z=2 by first occurrence; constants by the dictionary
    assert q["patterns"] == [(0, 1, 1, 1, 0), (0, 1, 2, 1, 0), (0, 2, 1, 1, 1), (0, 3, 2, 1, 1), (1, 1, 0, 1, 1)]
    assert q["n_vars"] == 3 and q["var_names"] == ["x", "y", "z"]
    assert q["projection"] == [1, 0] and q["distinct"]


def test_sparql_star_unknown_constants_and_plain_codes():
    d = _dict_with("<a>", preds=("<p>",))
    q = fe.parse_sparql("SELECT * { <a> <p> ?o . ?o <nope> <zzz> }", d)
    assert q["patterns"] == [(1, 1, 0, 0, 1), (0, 0, 0, 1, 0)]
    assert q["projection"] == [0]
    q = fe.parse_sparql("SELECT ?s WHERE { ?s 7 12 . ?s 3 ?t }")
    assert q["patterns"] == [(0, 7, 12, 1, 0), (0, 3, 1, 1, 1)]
    assert q["projection"] == [0] and q["n_vars"] == 2


@pytest.mark.parametrize("text,kind", [
    ("SELECT ?x { ?x ?p ?y }", "unsupported"),                  # variable predicate
    ("SELECT ?x { ?x 1 ?y FILTER (?y) }", "unsupported"),
    ("SELECT ?x { ?x 1 ?y . OPTIONAL { ?y 2 ?z } }", "unsupported"),
    ("SELECT ?x { { ?x 1 ?y } }", "unsupported"),
    ("SELECT ?x { ?x 1 ?y } LIMIT 5", "unsupported"),
    ("ASK { ?x 1 ?y }", "unsupported"),
    ("SELECT ?q { ?x 1 ?y }", "invalid"),                       # projected variable not bound
    ("SELECT ?x ?x { ?x 1 ?y }", "invalid"),
    ("SELECT { ?x 1 ?y }", "invalid"),
    ("SELECT ?x { }", "invalid"),
    ("SELECT ?x { ?x 1 ?y ?z 2 ?w }", "invalid"),               # no '.' between patterns
    ("SELECT ?x { ?x 1 ?y", "invalid"),
    ("SELECT ?x { ?x 1 ?y } junk", "invalid"),
    ("SELECT ?x { ?x 1 ex:y }", "invalid"),                     # not a code without a dictionary
    ("SELECT ?x { ?x 1 \"l\" . \"l\" \"l\" ?x }", "invalid"),   # literal predicate
    ("SELECT ?x- { ?x 1 ?y }", "invalid"),
])
def test_sparql_errors(text, kind):
    with pytest.raises(fe.FrontEndError) as e:
        fe.parse_sparql(text)
    assert e.value.kind == kind


def test_sparql_limits():
    pats = " . ".join("?a 1 ?b" for _ in range(65))
    q = fe.parse_sparql(f"SELECT * {{ {' . '.join(f'?a 1 ?b{i}' for i in range(31))} }}")
    assert q["n_vars"] == 32
    with pytest.raises(fe.FrontEndError):
        fe.parse_sparql(f"SELECT * {{ {' . '.join(f'?a 1 ?b{i}' for i in range(32))} }}")  # 33 variables
    with pytest.raises(fe.FrontEndError):
        fe.parse_sparql(f"SELECT * {{ {pats} }}")  # 65 patterns


# --------------------------------------------------------------------------
# projection and DISTINCT


def test_project_against_sets_and_bags():
    rng = np.random.default_rng(3)
    for _ in range(40):
        V = int(rng.integers(1, 5))
        rows = rng.integers(0, 4, size=(int(rng.integers(0, 60)), V))
        k = int(rng.integers(1, V + 1))
        vs = list(rng.permutation(V)[:k])
        want_set = sorted({tuple(int(r[v]) for v in vs) for r in rows})
        got = fe.project(rows, vs, True)
        assert [tuple(r) for r in got.tolist()] == want_set
        bag = fe.project(rows, vs, False)
        assert sorted(tuple(int(r[v]) for v in vs) for r in rows) == [tuple(r) for r in bag.tolist()]


def test_project_dg_example():
    g = golden("dg_example.json")
    rows = np.array(g["answer_xyzw"])
    assert fe.project(rows, [0, 3], True).tolist() == [[1, 3]]  # (X, W) = (A, I2)


def test_project_brute_force_small_graph():
    # SELECT DISTINCT ?x over {?x p ?y . ?y p ?z}: subjects with a 2-path
    t = np.array([(1, 5, 2), (2, 5, 3), (2, 5, 4), (3, 5, 1), (4, 6, 1)], dtype=np.int32)
    rows = oracle.OracleIndex(t).query([(0, 5, 1, 1, 1), (1, 5, 2, 1, 1)], 3)
    want = sorted({s for (s, p, o) in t.tolist() if p == 5
                   for (s2, p2, o2) in t.tolist() if p2 == 5 and s2 == o})
    assert fe.project(rows, [0], True).ravel().tolist() == want
    assert len(fe.project(rows, [0], False)) == len(rows)
    # rows (x, y, z): (1,2,3) (1,2,4) (2,3,1) (3,1,2); as (z, x): (3,1) (4,1) (1,2) (2,3)
    assert list(itertools.chain(*fe.project(rows, [2, 0], True).tolist())) == [1, 2, 2, 3, 3, 1, 4, 1]
