"""User-facing front end, restated plainly -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU baseline may use this
module; the library never does.

* Encoding (Sec. 5.2, "Generation of RDF Cubes"): the dataset's triples are
  read in order; predicates get codes 1, 2, ... (h_p) and subjects and
  objects share one numbering 1, 2, ... (h_so), each term its code at its
  first occurrence, the subject of a triple before its object.  Code 0 is
  never given out.
* Text of the data: statements of three terms ended by '.', in the
  N-Triples / Turtle subset below.
* SPARQL text (Sec. 3.2 shows the form: SELECT, variables, WHERE and a
  block of triple patterns): a prologue of PREFIX declarations, SELECT with
  optional DISTINCT, the projected variables or '*', optional WHERE, and a
  brace-enclosed basic graph pattern.
* Projection and DISTINCT: the solution rows restricted to the projected
  variables in the order given; DISTINCT keeps each row once; either way the
  rows come out ascending lexicographically.

Readings (the paper fixes none of the syntax; these are the build's):

* terms: <iri> (no whitespace inside); "literal" with backslash escapes and
  an optional @lang or ^^datatype suffix; _:blank; otherwise a bare token,
  a maximal run of characters other than whitespace and  < > " { } ; , .
  A term's identity is its text, except that a prefixed name whose prefix
  was declared (Turtle "@prefix p: <iri> ." in data, SPARQL "PREFIX p:
  <iri>" in queries) is rewritten as <iri + local part>, also inside a
  ^^datatype; an undeclared prefix leaves the token as written (so the
  paper's ":likes" is the term ":likes");
* the bare token 'a' in predicate position is rdf:type;
* ';' repeats the subject, ',' repeats subject and predicate (Turtle and
  SPARQL predicate-object lists); '#' at the start of a token opens a
  comment to the end of the line;
* query variables are ?name or $name (the same variable); they are numbered
  0, 1, ... in order of first occurrence in the WHERE block; a variable
  predicate, FILTER, OPTIONAL, UNION, GRAPH, MINUS, BIND, VALUES, nested
  groups and solution modifiers after the block are unsupported;
* a constant the dictionary does not hold becomes code 0, which matches
  nothing; without a dictionary, constants are decimal codes.
"""

from __future__ import annotations

import numpy as np

RDF_TYPE = "<http://www.w3.org/1999/02/22-rdf-syntax-ns#type>"

UNSUPPORTED_WORDS = {"FILTER", "OPTIONAL", "UNION", "GRAPH", "MINUS", "BIND", "VALUES", "SERVICE"}
TRAILING_UNSUPPORTED = {"ORDER", "LIMIT", "OFFSET", "GROUP", "HAVING"}
FORMS_UNSUPPORTED = {"ASK", "CONSTRUCT", "DESCRIBE", "BASE"}


class FrontEndError(Exception):
    """kind is 'invalid' (bad text or arguments) or 'unsupported'."""

    def __init__(self, kind: str, msg: str):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


# --------------------------------------------------------------------------
# tokens

SPECIAL = set('<>"{};,.')
WS = set(" \t\r\n")


def tokenize(text: str) -> list:
    """Split text into (kind, value) tokens: 'iri', 'lit', 'word', 'var',
    'punct' (one of { } ; , .)."""
    toks = []
    i, n = 0, len(text)
    while i < n:
        c = text[i]
        if c in WS:
            i += 1
            continue
        if c == "#":
            while i < n and text[i] != "\n":
                i += 1
            continue
        if c in "{};,.":
            toks.append(("punct", c))
            i += 1
            continue
        if c == "<":
            j = i + 1
            while j < n and text[j] != ">":
                if text[j] in WS:
                    raise FrontEndError("invalid", "whitespace inside an IRI")
                j += 1
            if j >= n:
                raise FrontEndError("invalid", "unterminated IRI")
            toks.append(("iri", text[i:j + 1]))
            i = j + 1
            continue
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            if j >= n:
                raise FrontEndError("invalid", "unterminated literal")
            j += 1  # past the closing quote
            body = text[i:j]
            dtype = None
            if j < n and text[j] == "@":
                k = j + 1
                while k < n and (text[k].isalnum() or text[k] == "-") and text[k].isascii():
                    k += 1
                body = text[i:k]
                j = k
            elif text.startswith("^^", j):
                k = j + 2
                if k < n and text[k] == "<":
                    while k < n and text[k] != ">":
                        k += 1
                    if k >= n:
                        raise FrontEndError("invalid", "unterminated datatype IRI")
                    dtype = ("iri", text[j + 2:k + 1])
                    k += 1
                else:
                    while k < n and text[k] not in WS and text[k] not in SPECIAL:
                        k += 1
                    if k == j + 2:
                        raise FrontEndError("invalid", "empty datatype")
                    dtype = ("word", text[j + 2:k])
                j = k
            toks.append(("lit", (body, dtype)))
            i = j
            continue
        if c == ">" or c == '"':
            raise FrontEndError("invalid", f"unexpected {c!r}")
        j = i
        while j < n and text[j] not in WS and text[j] not in SPECIAL:
            j += 1
        word = text[i:j]
        if word[0] in "?$":
            name = word[1:]
            if not name or not all((ch.isalnum() and ch.isascii()) or ch == "_" for ch in name):
                raise FrontEndError("invalid", f"bad variable {word!r}")
            toks.append(("var", name))
        else:
            toks.append(("word", word))
        i = j
    return toks


def expand(tok, prefixes: dict) -> str:
    """Identity text of a term token under the declared prefixes."""
    kind, val = tok
    if kind == "iri":
        return val
    if kind == "lit":
        body, dtype = val
        if dtype is None:
            return body
        return body + "^^" + expand(dtype, prefixes)
    if kind == "word":
        if ":" in val:
            pfx, local = val.split(":", 1)
            if pfx in prefixes:
                return "<" + prefixes[pfx][1:-1] + local + ">"
        return val
    raise FrontEndError("invalid", f"{kind} is not a term")


def _term(toks, k, what, query: bool):
    if k >= len(toks):
        raise FrontEndError("invalid", f"text ends where a {what} is expected")
    t = toks[k]
    if query and t[0] == "word" and t[1].upper() in UNSUPPORTED_WORDS:
        raise FrontEndError("unsupported", t[1])
    if t[0] == "var" and not query:
        raise FrontEndError("invalid", "a variable in data")
    if t[0] in ("iri", "lit", "word", "var"):
        return t
    raise FrontEndError("invalid", f"{t[1]!r} where a {what} is expected")


def _subject_triples(toks, pos, query: bool):
    """One subject with its predicate-object list ('; ' and ', ' forms):
    returns (list of (s, p, o) tokens, position after them)."""
    s = _term(toks, pos, "subject", query)
    pos += 1
    out = []
    while True:
        p = _term(toks, pos, "predicate", query)
        if p == ("word", "a"):
            p = ("iri", RDF_TYPE)
        pos += 1
        while True:
            o = _term(toks, pos, "object", query)
            pos += 1
            out.append((s, p, o))
            if pos < len(toks) and toks[pos] == ("punct", ","):
                pos += 1
                continue
            break
        if pos < len(toks) and toks[pos] == ("punct", ";"):
            while pos < len(toks) and toks[pos] == ("punct", ";"):
                pos += 1
            if pos < len(toks) and toks[pos][0] != "punct":
                continue  # another predicate of the same subject
        return out, pos


# --------------------------------------------------------------------------
# data


def parse_data(text: str) -> list:
    """(s, p, o) identity texts of the statements, in order."""
    toks = tokenize(text)
    prefixes = {}
    triples = []
    pos = 0
    while pos < len(toks):
        if toks[pos] == ("word", "@prefix"):
            if pos + 3 >= len(toks) or toks[pos + 1][0] != "word" or not toks[pos + 1][1].endswith(":") \
                    or toks[pos + 2][0] != "iri" or toks[pos + 3] != ("punct", "."):
                raise FrontEndError("invalid", "bad @prefix")
            prefixes[toks[pos + 1][1][:-1]] = toks[pos + 2][1]
            pos += 4
            continue
        got, pos = _subject_triples(toks, pos, query=False)
        if pos >= len(toks) or toks[pos] != ("punct", "."):
            raise FrontEndError("invalid", "statement not ended by '.'")
        pos += 1
        for s, p, o in got:
            if s[0] == "lit" or p[0] == "lit":
                raise FrontEndError("invalid", "a literal can only be an object")
            triples.append((expand(s, prefixes), expand(p, prefixes), expand(o, prefixes)))
    return triples


class Dictionary:
    """h_p and h_so by first occurrence (Sec. 5.2)."""

    def __init__(self):
        self.h_p: dict = {}
        self.h_so: dict = {}
        self.triples: list = []

    def add(self, text_triples) -> np.ndarray:
        codes = []
        for s, p, o in text_triples:
            if p not in self.h_p:
                self.h_p[p] = len(self.h_p) + 1
            for term in (s, o):
                if term not in self.h_so:
                    self.h_so[term] = len(self.h_so) + 1
            codes.append((self.h_so[s], self.h_p[p], self.h_so[o]))
        self.triples.extend(codes)
        return np.array(codes, dtype=np.int32).reshape(-1, 3)

    def add_text(self, text: str) -> np.ndarray:
        return self.add(parse_data(text))

    def decode_so(self, code: int) -> str:
        inv = {v: k for k, v in self.h_so.items()}
        return inv[int(code)]

    def decode_p(self, code: int) -> str:
        inv = {v: k for k, v in self.h_p.items()}
        return inv[int(code)]


# --------------------------------------------------------------------------
# SPARQL


def parse_sparql(text: str, dictionary: Dictionary | None = None) -> dict:
    """{'patterns': [(s, p, o, s_var, o_var)], 'n_vars', 'var_names',
    'projection': [var ids], 'distinct': bool}."""
    toks = tokenize(text)
    pos = 0
    prefixes = {}
    while pos < len(toks) and toks[pos][0] == "word" and toks[pos][1].upper() == "PREFIX":
        if pos + 2 >= len(toks) or toks[pos + 1][0] != "word" or not toks[pos + 1][1].endswith(":") \
                or toks[pos + 2][0] != "iri":
            raise FrontEndError("invalid", "bad PREFIX")
        prefixes[toks[pos + 1][1][:-1]] = toks[pos + 2][1]
        pos += 3
    if pos >= len(toks) or toks[pos][0] != "word":
        raise FrontEndError("invalid", "expected SELECT")
    head = toks[pos][1].upper()
    if head in FORMS_UNSUPPORTED:
        raise FrontEndError("unsupported", head)
    if head != "SELECT":
        raise FrontEndError("invalid", "expected SELECT")
    pos += 1
    distinct = False
    if pos < len(toks) and toks[pos][0] == "word" and toks[pos][1].upper() == "DISTINCT":
        distinct = True
        pos += 1
    proj_names = None
    if pos < len(toks) and toks[pos][0] == "word" and toks[pos][1] == "*":
        pos += 1
    else:
        proj_names = []
        while pos < len(toks) and toks[pos][0] == "var":
            proj_names.append(toks[pos][1])
            pos += 1
        if not proj_names:
            raise FrontEndError("invalid", "SELECT lists no variable")
    if pos < len(toks) and toks[pos][0] == "word" and toks[pos][1].upper() == "WHERE":
        pos += 1
    if pos >= len(toks) or toks[pos] != ("punct", "{"):
        raise FrontEndError("invalid", "expected '{'")
    pos += 1
    raw = []
    while True:
        if pos >= len(toks):
            raise FrontEndError("invalid", "pattern block not closed")
        if toks[pos] == ("punct", "}"):
            pos += 1
            break
        if toks[pos] == ("punct", "{"):
            raise FrontEndError("unsupported", "nested group")
        got, pos = _subject_triples(toks, pos, query=True)
        raw += got
        if pos < len(toks) and toks[pos] == ("punct", "."):
            pos += 1
        elif not (pos < len(toks) and toks[pos] == ("punct", "}")):
            if pos < len(toks) and toks[pos][0] == "word" and toks[pos][1].upper() in UNSUPPORTED_WORDS:
                raise FrontEndError("unsupported", toks[pos][1])
            raise FrontEndError("invalid", "expected '.' or '}' after a triple pattern")
    if pos < len(toks):
        t = toks[pos]
        if t[0] == "word" and t[1].upper() in TRAILING_UNSUPPORTED:
            raise FrontEndError("unsupported", t[1])
        raise FrontEndError("invalid", "text after the closing '}'")
    if not raw:
        raise FrontEndError("invalid", "empty pattern block")
    if len(raw) > 64:
        raise FrontEndError("invalid", "more than 64 patterns")
    var_id = {}
    pats = []

    def const_code(tok, pred: bool) -> int:
        if dictionary is None:
            if tok[0] != "word" or not tok[1].isdigit() or not tok[1].isascii():
                raise FrontEndError("invalid", f"constant {tok[1]!r} is not a decimal code")
            v = int(tok[1])
            if v > 2 ** 31 - 1:
                raise FrontEndError("invalid", "code out of range")
            return v
        term = expand(tok, prefixes)
        table = dictionary.h_p if pred else dictionary.h_so
        return table.get(term, 0)

    for s, p, o in raw:
        if p[0] == "var":
            raise FrontEndError("unsupported", "variable predicate")
        if p[0] == "lit":
            raise FrontEndError("invalid", "a literal cannot be a predicate")
        ends = []
        for t in (s, o):
            if t[0] == "var":
                if t[1] not in var_id:
                    var_id[t[1]] = len(var_id)
                ends.append((var_id[t[1]], 1))
            else:
                ends.append((const_code(t, False), 0))
        pats.append((ends[0][0], const_code(p, True), ends[1][0], ends[0][1], ends[1][1]))
    if len(var_id) > 32:
        raise FrontEndError("invalid", "more than 32 variables")
    names = sorted(var_id, key=var_id.get)
    if proj_names is None:
        proj = list(range(len(names)))
    else:
        proj = []
        for nm in proj_names:
            if nm not in var_id:
                raise FrontEndError("invalid", f"?{nm} is not in the pattern block")
            if var_id[nm] in proj:
                raise FrontEndError("invalid", f"?{nm} projected twice")
            proj.append(var_id[nm])
    return {"patterns": pats, "n_vars": len(names), "var_names": names, "projection": proj, "distinct": distinct}


# --------------------------------------------------------------------------
# projection


def project(rows, variables, distinct: bool) -> np.ndarray:
    """Rows (over variables 0..V-1) restricted to `variables` in that order,
    ascending lexicographically, each kept once when `distinct`."""
    rows = np.asarray(rows, dtype=np.int64)
    k = len(variables)
    if rows.shape[0] == 0:
        return np.zeros((0, k), dtype=np.int32)
    sel = rows[:, list(variables)]
    sel = sel[np.lexsort(sel.T[::-1])]
    if distinct:
        keep = np.ones(sel.shape[0], dtype=bool)
        keep[1:] = np.any(sel[1:] != sel[:-1], axis=1)
        sel = sel[keep]
    return sel.astype(np.int32)
