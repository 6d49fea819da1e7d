"""The library's dictionary and SPARQL reader (host code behind the C ABI)
against the oracle's front end: same codes, same BGPs, same error kinds
(CPU only)."""

import numpy as np
import pytest

from oracle import frontend as fe
from tests.helpers import golden

KIND = {1: "invalid", 2: "unsupported"}


@pytest.fixture(scope="module")
def gs():
    import paper_1807_07691_b300 as g

    return g


def _lib_parse_data(gs, text):
    d = gs.Dictionary()
    try:
        d.add_text(text)
    except gs.GsmatError as e:
        return KIND[e.code], d
    return d.triples(), d


def _oracle_parse_data(text):
    d = fe.Dictionary()
    try:
        return d.add_text(text), d
    except fe.FrontEndError as e:
        return e.kind, d


def test_dg_codes_and_decode(gs):
    g, t = golden("dg_example.json"), golden("dg_text.json")
    d = gs.Dictionary(t["data"])
    assert d.triples().tolist() == g["cube_spo"]
    assert d.size() == (3, 7)
    for term, code in g["h_so"].items():
        assert d.lookup(term, d.SO) == code
        assert d.decode([code], d.SO) == [term]
    for term, code in g["h_p"].items():
        assert d.lookup(term, d.P) == code
    assert d.lookup("nobody", d.SO) == 0
    with pytest.raises(gs.GsmatError):
        d.decode([0], d.SO)
    with pytest.raises(gs.GsmatError):
        d.decode([8], d.SO)


def test_dg_query_text(gs):
    g, t = golden("dg_example.json"), golden("dg_text.json")
    d = gs.Dictionary(t["data"])
    q = gs.Sparql(t["query"], d)
    assert [list(p) for p in q.patterns] == g["query"]
    assert q.var_names == g["query_vars"] and q.projection == [0, 1, 2, 3] and not q.distinct


# --------------------------------------------------------------------------
# random data texts


def _rand_term(rng, kind):
    r = rng.random()
    n = int(rng.integers(0, 12))
    if kind == "p":
        if r < 0.1:
            return "a"
        if r < 0.5:
            return f"<http://x.org/p{n}>"
        return f"ex:p{n}" if r < 0.8 else f":q{n}"
    if kind == "o" and r < 0.3:
        body = rng.choice(['"v{}"', '"a b {}"', '"q\\"{}"', '"{}"'])
        lit = body.format(n)
        r2 = rng.random()
        if r2 < 0.3:
            return lit + "@en"
        if r2 < 0.5:
            return lit + "^^ex:int"
        if r2 < 0.6:
            return lit + "^^<http://t/x>"
        return lit
    if r < 0.15:
        return f"_:b{n}"
    if r < 0.5:
        return f"<http://x.org/e{n}>"
    if r < 0.8:
        return f"ex:e{n}"
    return f"e{n}"


def _rand_data(rng):
    lines = []
    if rng.random() < 0.7:
        lines.append("@prefix ex: <http://x.org/> .")
    for _ in range(int(rng.integers(0, 25))):
        s = _rand_term(rng, "s")
        parts = []
        for _p in range(int(rng.integers(1, 3))):
            p = _rand_term(rng, "p")
            objs = [_rand_term(rng, "o") for _ in range(int(rng.integers(1, 3)))]
            parts.append(p + " " + " , ".join(objs))
        sep = rng.choice([" ; ", " ;\n  "])
        end = rng.choice([" .", ".", " ;.", " .  # note"])
        lines.append(s + " " + sep.join(parts) + end)
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed", range(30))
def test_random_data_matches_oracle(gs, seed):
    rng = np.random.default_rng(seed)
    d = gs.Dictionary()
    o = fe.Dictionary()
    for _ in range(3):  # several texts continue the numberings
        text = _rand_data(rng)
        n = d.add_text(text)
        want = o.add_text(text)
        assert n == len(want)
    got = d.triples()
    assert got.tolist() == np.array(o.triples, dtype=np.int32).reshape(-1, 3).tolist()
    assert d.size() == (len(o.h_p), len(o.h_so))
    so = sorted(o.h_so.items(), key=lambda kv: kv[1])
    assert d.decode([c for _, c in so], d.SO) == [t for t, _ in so]
    ps = sorted(o.h_p.items(), key=lambda kv: kv[1])
    assert d.decode([c for _, c in ps], d.P) == [t for t, _ in ps]


def _mutate(rng, text):
    chars = list(text)
    for _ in range(int(rng.integers(1, 4))):
        op = rng.random()
        i = int(rng.integers(0, max(1, len(chars))))
        if op < 0.4 and chars:
            del chars[i]
        elif op < 0.8:
            chars.insert(i, str(rng.choice(list('<>"{};,.?$#@^ \n:_ax1'))))
        elif chars:
            chars[i] = str(rng.choice(list('<>"{};,. ')))
    return "".join(chars)


@pytest.mark.parametrize("seed", range(20))
def test_mutated_data_same_outcome(gs, seed):
    """Damaged texts: the library and the oracle accept the same ones (with
    the same codes) and reject the others; a rejected text adds nothing."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        text = _mutate(rng, _rand_data(rng))
        got, d = _lib_parse_data(gs, text)
        want, _ = _oracle_parse_data(text)
        if isinstance(want, str):
            assert got == want, text
            assert d.size() == (0, 0) and d.triples().shape == (0, 3)
        else:
            assert not isinstance(got, str), (text, got)
            assert got.tolist() == want.tolist(), text


@pytest.mark.parametrize("text", [
    "<a> <p> <b>", "<a> <p> .", "<a b> <p> <c> .", '<a> <p> "open .', '"lit" <p> <b> .',
    "<a> <p> ?x .", "@prefix ex <http://e/> .", '<a> <p> "x"^^ .', ". <a> <p> <b> .",
])
def test_data_errors(gs, text):
    d = gs.Dictionary("<z> <q> <y> .")
    with pytest.raises(gs.GsmatError) as e:
        d.add_text(text)
    assert e.value.code == 1
    assert d.triples().tolist() == [[1, 1, 2]]  # unchanged


# --------------------------------------------------------------------------
# SPARQL text


def _both(gs, text, data=None):
    od = ld = None
    if data is not None:
        od = fe.Dictionary()
        od.add_text(data)
        ld = gs.Dictionary(data)
    try:
        want = fe.parse_sparql(text, od)
    except fe.FrontEndError as e:
        want = e.kind
    try:
        q = gs.Sparql(text, ld)
        got = {"patterns": [tuple(int(x) for x in p) for p in q.patterns], "n_vars": q.n_vars,
               "var_names": q.var_names, "projection": q.projection, "distinct": q.distinct}
    except gs.GsmatError as e:
        got = KIND.get(e.code, e.code)
    return got, want


SPARQL_CASES = [
    "SELECT ?x ?y ?z ?w WHERE { ?x :follows ?y . ?y :follows ?z . ?x :likes ?w . ?z :likes ?w .}",
    """PREFIX ex: <http://x.org/>
       select distinct $y ?x where { ?x ex:p0 ex:e1 , "v1"@en ; ex:p1 ?y ; a ?z .  # c
       ?y <http://x.org/p2> ?x }""",
    "SELECT * { ?s ex:p1 ?o }",
    "SELECT * { ?s <http://x.org/p1> ?o ; <http://x.org/p3> _:b2 . }",
    "SELECT ?x { ?x ?p ?y }",
    "SELECT ?x { ?x :q1 ?y FILTER (?y) }",
    "SELECT ?x { ?x :q1 ?y . OPTIONAL { ?y :q2 ?z } }",
    "SELECT ?x { { ?x :q1 ?y } }",
    "SELECT ?x { ?x :q1 ?y } LIMIT 5",
    "ASK { ?x :q1 ?y }",
    "SELECT ?q { ?x :q1 ?y }",
    "SELECT ?x ?x { ?x :q1 ?y }",
    "SELECT { ?x :q1 ?y }",
    "SELECT ?x { }",
    "SELECT ?x { ?x :q1 ?y ?z :q2 ?w }",
    "SELECT ?x { ?x :q1 ?y",
    "SELECT ?x { ?x :q1 ?y } junk",
    'SELECT ?x { ?x :q1 "l" . "l" "l" ?x }',
    "SELECT ?x- { ?x :q1 ?y }",
    'ASK { ?x :q1 "unterminated }',
    "SELECT ?s WHERE { ?s 7 12 . ?s 3 ?t }",
]


@pytest.mark.parametrize("i", range(len(SPARQL_CASES)))
def test_sparql_cases_match_oracle(gs, i):
    data = "@prefix ex: <http://x.org/> .\nex:e1 ex:p0 ex:e2 ; ex:p1 ex:e3 .\n:a :follows :b ; :likes :c .\n"
    got, want = _both(gs, SPARQL_CASES[i], data)
    assert got == want
    got, want = _both(gs, SPARQL_CASES[i], None)  # constants as decimal codes
    assert got == want


def _rand_query(rng):
    nv = int(rng.integers(1, 5))
    pats = []
    for _ in range(int(rng.integers(1, 6))):
        s = f"?v{int(rng.integers(nv))}" if rng.random() < 0.8 else _rand_term(rng, "s")
        p = _rand_term(rng, "p") if rng.random() < 0.97 else "?pv"
        o = f"${'v'}{int(rng.integers(nv))}" if rng.random() < 0.7 else _rand_term(rng, "o")
        pats.append(f"{s} {p} {o}")
    names = sorted({w[1:] for pt in pats for w in pt.split() if w[0] in "?$" and w != "?pv"})
    if rng.random() < 0.3 or not names:
        head = "*"
    else:
        k = int(rng.integers(1, len(names) + 1))
        head = " ".join("?" + n for n in rng.permutation(names)[:k])
    pre = "PREFIX ex: <http://x.org/>\n" if rng.random() < 0.7 else ""
    dist = "DISTINCT " if rng.random() < 0.4 else ""
    where = "WHERE " if rng.random() < 0.5 else ""
    return f"{pre}SELECT {dist}{head} {where}{{ " + " . ".join(pats) + (" ." if rng.random() < 0.5 else "") + " }"


@pytest.mark.parametrize("seed", range(20))
def test_random_and_mutated_queries_match_oracle(gs, seed):
    rng = np.random.default_rng(500 + seed)
    data = _rand_data(rng)
    n_ok = 0
    for _ in range(30):
        text = _rand_query(rng)
        got, want = _both(gs, text, data)
        assert got == want, text
        n_ok += isinstance(want, dict)
        bad = _mutate(rng, text)
        got, want = _both(gs, bad, data)
        assert got == want, bad
    assert n_ok > 5


def test_sparql_limits(gs):
    ok = "SELECT * { " + " . ".join(f"?a 1 ?b{i}" for i in range(31)) + " }"
    assert gs.Sparql(ok).n_vars == 32
    for bad in ("SELECT * { " + " . ".join(f"?a 1 ?b{i}" for i in range(32)) + " }",
                "SELECT * { " + " . ".join("?a 1 ?b" for _ in range(65)) + " }",
                "SELECT * { ?a 2147483648 ?b }"):
        with pytest.raises(gs.GsmatError) as e:
            gs.Sparql(bad)
        assert e.value.code == 1
    assert gs.Sparql("SELECT * { ?a 2147483647 ?b }").patterns[0][1] == 2147483647


@pytest.mark.parametrize("threads", [2, 3, 8, 64])
def test_parallel_numbering_matches_oracle(gs, threads):
    """Terms numbered by several host threads get the codes of a sequential
    reading (first occurrence), over several adds and with repeated terms."""
    rng = np.random.default_rng(threads)
    o = fe.Dictionary()
    d = gs.Dictionary(threads=threads)
    for _ in range(3):
        text = _rand_data(rng) + "\n".join(
            f"<http://x.org/n{int(a)}> <http://x.org/r{int(b)}> <http://x.org/n{int(c)}> ."
            for a, b, c in rng.integers(0, [3000, 7, 3000], size=(4000, 3)))
        assert d.add_text(text) == len(o.add_text(text))
    assert d.triples().tolist() == np.array(o.triples, dtype=np.int32).reshape(-1, 3).tolist()
    assert d.size() == (len(o.h_p), len(o.h_so))
    so = sorted(o.h_so.items(), key=lambda kv: kv[1])
    assert d.decode([c for _, c in so], d.SO) == [t for t, _ in so]
    for term, code in list(o.h_so.items())[::97]:
        assert d.lookup(term, d.SO) == code
    # a bad text after that leaves everything as it was
    with pytest.raises(gs.GsmatError):
        d.add_text("<a> <p> <b> . <c> <q> ")
    assert d.size() == (len(o.h_p), len(o.h_so))
    assert d.triples().shape[0] == len(o.triples)
    with pytest.raises(gs.GsmatError):
        d.set_threads(-1)


def test_host_entry_points_reject_bad_arguments(gs):
    import ctypes

    lib = gs.lib()
    h = ctypes.c_void_p()
    n = ctypes.c_int64()
    assert lib.gsmat_dict_create(None) == 1
    assert lib.gsmat_dict_create(ctypes.byref(h)) == 0
    assert lib.gsmat_dict_add_text(None, b"<a> <p> <b> .", 13, ctypes.byref(n)) == 1
    assert lib.gsmat_dict_add_text(h, None, 5, ctypes.byref(n)) == 1
    assert lib.gsmat_dict_add_text(h, b"x", -1, ctypes.byref(n)) == 1
    assert lib.gsmat_dict_add_text(h, None, 0, ctypes.byref(n)) == 0 and n.value == 0  # empty text
    assert lib.gsmat_dict_triples(h, None, ctypes.byref(n)) == 1
    code = ctypes.c_int32()
    assert lib.gsmat_dict_lookup(h, 2, b"<a>", 3, ctypes.byref(code)) == 1  # bad kind
    assert lib.gsmat_dict_lookup(h, 0, b"<a>", 3, None) == 1
    assert lib.gsmat_dict_decode(h, 0, None, 1, None, None) == 1
    assert lib.gsmat_dict_decode(h, 0, None, 0, None, None) == 0  # nothing to decode
    assert lib.gsmat_dict_set_threads(h, 257) == 1
    q = ctypes.c_void_p()
    assert lib.gsmat_sparql_parse(h, b"SELECT * { ?a 1 ?b }", 20, None) == 1
    assert lib.gsmat_sparql_parse(h, None, 4, ctypes.byref(q)) == 1
    assert lib.gsmat_sparql_info(None, None, None, None, None, None, None) == 1
    assert lib.gsmat_sparql_var_name(None, 0) is None
    assert lib.gsmat_sparql_parse(None, b"SELECT * { ?a 1 ?b }", 20, ctypes.byref(q)) == 0
    assert lib.gsmat_sparql_var_name(q, 2) is None and lib.gsmat_sparql_var_name(q, -1) is None
    assert lib.gsmat_sparql_var_name(q, 1) == b"b"
    lib.gsmat_sparql_free(q)
    lib.gsmat_sparql_free(None)
    lib.gsmat_dict_free(h)
    lib.gsmat_dict_free(None)
    assert lib.gsmat_last_error() is not None
