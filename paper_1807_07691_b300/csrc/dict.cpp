// String dictionary (Sec. 5.2, "Generation of RDF Cubes"): h_p numbers the
// predicates and h_so the subjects and objects (one numbering for both),
// each from 1 in order of first occurrence as the triples are read, the
// subject of a triple before its object.  Host code; the encoded triples
// feed gsmat_load.
#include <string.h>

#include <deque>
#include <string>
#include <string_view>
#include <unordered_map>
#include <vector>

#include "dict.h"
#include "text.h"

namespace gs {

namespace {

// One numbering: identity text -> code (1, 2, ...), code -> text.  Texts
// live in a deque, so the views that key the map stay valid.
struct Codebook {
    std::deque<std::string> texts;
    std::unordered_map<std::string_view, int32_t> code;

    int32_t find(std::string_view t) const {
        auto it = code.find(t);
        return it == code.end() ? 0 : it->second;
    }
    // The code of t, numbering it if new; -1 when the numbering is full.
    int32_t get(const std::string &t) {
        auto it = code.find(std::string_view(t));
        if (it != code.end()) return it->second;
        if (texts.size() >= (size_t)INT32_MAX) return -1;
        texts.push_back(t);
        const int32_t c = (int32_t)texts.size();
        code.emplace(std::string_view(texts.back()), c);
        return c;
    }
};

}  // namespace

}  // namespace gs

struct gsmat_dict {
    gs::Codebook p, so;
    std::vector<int32_t> triples;  // (s, p, o) codes, in text order
};

namespace gs {

int32_t dict_code(const gsmat_dict *d, int kind, std::string_view text) {
    return kind == GSMAT_DICT_P ? d->p.find(text) : d->so.find(text);
}

namespace {

// Read the statements of a data text; emit(s, p, o) with identity texts.
template <class Emit>
int read_data(std::string_view text, Emit &&emit) {
    txt::Lexer lx(text);
    txt::Prefixes pf;
    std::string es, ep, eo;
    for (;;) {
        const txt::Tok *nx;
        int rc = lx.peek(&nx);
        if (rc != GSMAT_OK) return rc;
        if (nx->kind == txt::kEnd) return GSMAT_OK;
        if (nx->kind == txt::kWord && nx->text == "@prefix") {
            txt::Tok kw, name, iri, dot;
            lx.take(kw);
            if ((rc = lx.take(name)) != GSMAT_OK || (rc = lx.take(iri)) != GSMAT_OK || (rc = lx.take(dot)) != GSMAT_OK) {
                return rc;
            }
            if (name.kind != txt::kWord || name.text.empty() || name.text.back() != ':' || iri.kind != txt::kIri ||
                !txt::is_punct(&dot, '.')) {
                return set_error(GSMAT_ERR_INVALID_ARG, "bad @prefix");
            }
            pf[std::string(name.text.substr(0, name.text.size() - 1))] = std::string(iri.text);
            continue;
        }
        rc = txt::read_subject(lx, false, [&](const txt::Tok &s, const txt::Tok &p, const txt::Tok &o) {
            if (s.kind == txt::kLit || p.kind == txt::kLit) {
                return set_error(GSMAT_ERR_INVALID_ARG, "a literal can only be an object");
            }
            txt::expand(s, pf, es);
            txt::expand(p, pf, ep);
            txt::expand(o, pf, eo);
            return emit(es, ep, eo);
        });
        if (rc != GSMAT_OK) return rc;
        txt::Tok dot;
        if ((rc = lx.take(dot)) != GSMAT_OK) return rc;
        if (!txt::is_punct(&dot, '.')) return set_error(GSMAT_ERR_INVALID_ARG, "statement not ended by '.'");
    }
}

}  // namespace

int dict_create(gsmat_dict **out) {
    if (!out) return set_error(GSMAT_ERR_INVALID_ARG, "out is NULL");
    *out = new gsmat_dict();
    return GSMAT_OK;
}

void dict_free(gsmat_dict *d) { delete d; }

int dict_add_text(gsmat_dict *d, const char *text, int64_t len, int64_t *n_added) {
    if (!d || (!text && len > 0) || len < 0) return set_error(GSMAT_ERR_INVALID_ARG, "dict, text or length");
    const std::string_view sv(text ? text : "", (size_t)len);
    // check the whole text first, so that a bad text changes nothing
    int64_t n = 0;
    int rc = read_data(sv, [&](const std::string &, const std::string &, const std::string &) {
        ++n;
        return GSMAT_OK;
    });
    if (rc != GSMAT_OK) return rc;
    const size_t old = d->triples.size();
    d->triples.reserve(old + 3 * (size_t)n);
    rc = read_data(sv, [&](const std::string &s, const std::string &p, const std::string &o) {
        const int32_t cp = d->p.get(p);
        const int32_t cs = d->so.get(s);
        const int32_t co = d->so.get(o);
        if (cp < 0 || cs < 0 || co < 0) return set_error(GSMAT_ERR_CAPACITY, "more than 2^31 - 1 terms");
        d->triples.push_back(cs);
        d->triples.push_back(cp);
        d->triples.push_back(co);
        return GSMAT_OK;
    });
    if (rc != GSMAT_OK) {
        d->triples.resize(old);  // the terms already numbered stay (unused)
        return rc;
    }
    if (n_added) *n_added = n;
    return GSMAT_OK;
}

int dict_triples(const gsmat_dict *d, const int32_t **triples, int64_t *n) {
    if (!d || !triples || !n) return set_error(GSMAT_ERR_INVALID_ARG, "NULL argument");
    *triples = d->triples.empty() ? nullptr : d->triples.data();
    *n = (int64_t)d->triples.size() / 3;
    return GSMAT_OK;
}

int dict_size(const gsmat_dict *d, int32_t *n_predicates, int32_t *n_terms) {
    if (!d) return set_error(GSMAT_ERR_INVALID_ARG, "dict is NULL");
    if (n_predicates) *n_predicates = (int32_t)d->p.texts.size();
    if (n_terms) *n_terms = (int32_t)d->so.texts.size();
    return GSMAT_OK;
}

int dict_lookup(const gsmat_dict *d, int kind, const char *term, int64_t len, int32_t *code) {
    if (!d || !code || (!term && len > 0) || len < 0 || (kind != GSMAT_DICT_SO && kind != GSMAT_DICT_P)) {
        return set_error(GSMAT_ERR_INVALID_ARG, "dict, kind, term or code");
    }
    *code = dict_code(d, kind, std::string_view(term ? term : "", (size_t)len));
    return GSMAT_OK;
}

int dict_decode(const gsmat_dict *d, int kind, const int32_t *codes, int64_t n, const char **terms, int32_t *lens) {
    if (!d || (n > 0 && (!codes || !terms)) || n < 0 || (kind != GSMAT_DICT_SO && kind != GSMAT_DICT_P)) {
        return set_error(GSMAT_ERR_INVALID_ARG, "dict, kind, codes or terms");
    }
    const Codebook &cb = kind == GSMAT_DICT_P ? d->p : d->so;
    const int64_t size = (int64_t)cb.texts.size();
    for (int64_t i = 0; i < n; ++i) {
        if (codes[i] < 1 || codes[i] > size) {
            return set_error(GSMAT_ERR_INVALID_ARG, "code %d at %lld is not in the dictionary", codes[i], (long long)i);
        }
        const std::string &t = cb.texts[(size_t)codes[i] - 1];
        terms[i] = t.c_str();
        if (lens) lens[i] = (int32_t)t.size();
    }
    return GSMAT_OK;
}

}  // namespace gs
