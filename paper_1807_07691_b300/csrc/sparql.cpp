// SPARQL reader: the Select|Project|Join core form of a query (Sec. 3.2)
// over one basic graph pattern, turned into the gsmat_pattern BGP that
// gsmat_query evaluates plus the projection that gsmat_table_project
// applies.  Host code.
#include <string.h>

#include <string>
#include <string_view>
#include <vector>

#include "dict.h"
#include "text.h"

struct gsmat_sparql {
    std::vector<gsmat_pattern> pats;
    int32_t n_vars = 0;
    std::vector<std::string> var_names;
    std::vector<int32_t> proj;
    int32_t distinct = 0;
};

namespace gs {

namespace {

struct RawPattern {
    txt::Tok s, p, o;
};

bool keyword_in(std::string_view w, std::initializer_list<const char *> kws) {
    for (const char *k : kws) {
        if (txt::keyword_is(w, k)) return true;
    }
    return false;
}

// Code of a constant: by the dictionary (0 when it does not hold the term),
// or, without one, the constant written as a decimal code.
int const_code(const gsmat_dict *d, const txt::Tok &t, const txt::Prefixes &pf, int kind, std::string &scratch,
               int32_t *code) {
    if (!d) {
        if (t.kind != txt::kWord || t.text.empty()) {
            return set_error(GSMAT_ERR_INVALID_ARG, "constant '%.*s' is not a decimal code", (int)t.text.size(),
                             t.text.data());
        }
        int64_t v = 0;
        for (char c : t.text) {
            if (c < '0' || c > '9') {
                return set_error(GSMAT_ERR_INVALID_ARG, "constant '%.*s' is not a decimal code", (int)t.text.size(),
                                 t.text.data());
            }
            v = v * 10 + (c - '0');
            if (v > INT32_MAX) return set_error(GSMAT_ERR_INVALID_ARG, "code out of range");
        }
        *code = (int32_t)v;
        return GSMAT_OK;
    }
    txt::expand(t, pf, scratch);
    *code = dict_code(d, kind, scratch);
    return GSMAT_OK;
}

int parse(const gsmat_dict *d, std::string_view text, gsmat_sparql &q) {
    {
        // a lexical error anywhere makes the text invalid, whatever comes first
        txt::Lexer all(text);
        txt::Tok t;
        do {
            const int rc = all.take(t);
            if (rc != GSMAT_OK) return rc;
        } while (t.kind != txt::kEnd);
    }
    txt::Lexer lx(text);
    txt::Prefixes pf;
    const txt::Tok *nx;
    txt::Tok t;
    int rc;
    // prologue
    for (;;) {
        if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
        if (!(nx->kind == txt::kWord && txt::keyword_is(nx->text, "PREFIX"))) break;
        txt::Tok name, iri;
        lx.take(t);
        if ((rc = lx.take(name)) != GSMAT_OK || (rc = lx.take(iri)) != GSMAT_OK) return rc;
        if (name.kind != txt::kWord || name.text.empty() || name.text.back() != ':' || iri.kind != txt::kIri) {
            return set_error(GSMAT_ERR_INVALID_ARG, "bad PREFIX");
        }
        pf[std::string(name.text.substr(0, name.text.size() - 1))] = std::string(iri.text);
    }
    // SELECT [DISTINCT] (vars | *) [WHERE]
    if ((rc = lx.take(t)) != GSMAT_OK) return rc;
    if (t.kind != txt::kWord) return set_error(GSMAT_ERR_INVALID_ARG, "expected SELECT");
    if (keyword_in(t.text, {"ASK", "CONSTRUCT", "DESCRIBE", "BASE"})) {
        return set_error(GSMAT_ERR_UNSUPPORTED, "'%.*s' queries are not supported", (int)t.text.size(), t.text.data());
    }
    if (!txt::keyword_is(t.text, "SELECT")) return set_error(GSMAT_ERR_INVALID_ARG, "expected SELECT");
    if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
    if (nx->kind == txt::kWord && txt::keyword_is(nx->text, "DISTINCT")) {
        q.distinct = 1;
        lx.take(t);
    }
    bool star = false;
    std::vector<std::string_view> proj_names;
    if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
    if (nx->kind == txt::kWord && nx->text == "*") {
        star = true;
        lx.take(t);
    } else {
        for (;;) {
            if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
            if (nx->kind != txt::kVar) break;
            proj_names.push_back(nx->text);
            lx.take(t);
        }
        if (proj_names.empty()) return set_error(GSMAT_ERR_INVALID_ARG, "SELECT lists no variable");
    }
    if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
    if (nx->kind == txt::kWord && txt::keyword_is(nx->text, "WHERE")) lx.take(t);
    if ((rc = lx.take(t)) != GSMAT_OK) return rc;
    if (!txt::is_punct(&t, '{')) return set_error(GSMAT_ERR_INVALID_ARG, "expected '{'");
    // the pattern block
    std::vector<RawPattern> raw;
    for (;;) {
        if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
        if (nx->kind == txt::kEnd) return set_error(GSMAT_ERR_INVALID_ARG, "pattern block not closed");
        if (txt::is_punct(nx, '}')) {
            lx.take(t);
            break;
        }
        if (txt::is_punct(nx, '{')) return set_error(GSMAT_ERR_UNSUPPORTED, "nested groups are not supported");
        rc = txt::read_subject(lx, true, [&](const txt::Tok &s, const txt::Tok &p, const txt::Tok &o) {
            raw.push_back({s, p, o});
            return GSMAT_OK;
        });
        if (rc != GSMAT_OK) return rc;
        if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
        if (txt::is_punct(nx, '.')) {
            lx.take(t);
        } else if (!txt::is_punct(nx, '}')) {
            if (nx->kind == txt::kWord && txt::unsupported_in_block(nx->text)) {
                return set_error(GSMAT_ERR_UNSUPPORTED, "'%.*s' is not supported", (int)nx->text.size(),
                                 nx->text.data());
            }
            return set_error(GSMAT_ERR_INVALID_ARG, "expected '.' or '}' after a triple pattern");
        }
    }
    if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
    if (nx->kind != txt::kEnd) {
        if (nx->kind == txt::kWord && keyword_in(nx->text, {"ORDER", "LIMIT", "OFFSET", "GROUP", "HAVING"})) {
            return set_error(GSMAT_ERR_UNSUPPORTED, "'%.*s' is not supported", (int)nx->text.size(), nx->text.data());
        }
        return set_error(GSMAT_ERR_INVALID_ARG, "text after the closing '}'");
    }
    if (raw.empty()) return set_error(GSMAT_ERR_INVALID_ARG, "empty pattern block");
    if (raw.size() > (size_t)GSMAT_MAX_PATTERNS) {
        return set_error(GSMAT_ERR_INVALID_ARG, "more than %d patterns", GSMAT_MAX_PATTERNS);
    }
    // patterns in order: variables numbered by first occurrence
    std::vector<std::string_view> names;
    auto var_id = [&](std::string_view n) {
        for (size_t i = 0; i < names.size(); ++i) {
            if (names[i] == n) return (int32_t)i;
        }
        names.push_back(n);
        return (int32_t)names.size() - 1;
    };
    std::string scratch;
    for (const RawPattern &r : raw) {
        if (r.p.kind == txt::kVar) return set_error(GSMAT_ERR_UNSUPPORTED, "variable predicate (Sec. 6.3)");
        if (r.p.kind == txt::kLit) return set_error(GSMAT_ERR_INVALID_ARG, "a literal cannot be a predicate");
        gsmat_pattern g;
        memset(&g, 0, sizeof(g));
        const txt::Tok *ends[2] = {&r.s, &r.o};
        int32_t val[2];
        uint8_t isv[2];
        for (int e = 0; e < 2; ++e) {
            if (ends[e]->kind == txt::kVar) {
                val[e] = var_id(ends[e]->text);
                isv[e] = 1;
            } else {
                if ((rc = const_code(d, *ends[e], pf, GSMAT_DICT_SO, scratch, &val[e])) != GSMAT_OK) return rc;
                isv[e] = 0;
            }
        }
        int32_t pc;
        if ((rc = const_code(d, r.p, pf, GSMAT_DICT_P, scratch, &pc)) != GSMAT_OK) return rc;
        g.s = val[0];
        g.s_var = isv[0];
        g.p = pc;
        g.o = val[1];
        g.o_var = isv[1];
        q.pats.push_back(g);
    }
    if (names.size() > 32) return set_error(GSMAT_ERR_INVALID_ARG, "more than 32 variables");
    q.n_vars = (int32_t)names.size();
    for (std::string_view n : names) q.var_names.emplace_back(n);
    if (star) {
        for (int32_t v = 0; v < q.n_vars; ++v) q.proj.push_back(v);
    } else {
        for (std::string_view n : proj_names) {
            int32_t v = -1;
            for (size_t i = 0; i < names.size(); ++i) {
                if (names[i] == n) v = (int32_t)i;
            }
            if (v < 0) {
                return set_error(GSMAT_ERR_INVALID_ARG, "?%.*s is not in the pattern block", (int)n.size(), n.data());
            }
            for (int32_t w : q.proj) {
                if (w == v) return set_error(GSMAT_ERR_INVALID_ARG, "?%.*s projected twice", (int)n.size(), n.data());
            }
            q.proj.push_back(v);
        }
    }
    return GSMAT_OK;
}

}  // namespace

int sparql_parse(const gsmat_dict *d, const char *text, int64_t len, gsmat_sparql **out) {
    if (!out || (!text && len > 0) || len < 0) return set_error(GSMAT_ERR_INVALID_ARG, "text, length or out");
    *out = nullptr;
    gsmat_sparql *q = new gsmat_sparql();
    const int rc = parse(d, std::string_view(text ? text : "", (size_t)len), *q);
    if (rc != GSMAT_OK) {
        delete q;
        return rc;
    }
    *out = q;
    return GSMAT_OK;
}

int sparql_info(const gsmat_sparql *q, const gsmat_pattern **pats, int32_t *n_pats, int32_t *n_vars,
                const int32_t **proj, int32_t *n_proj, int32_t *distinct) {
    if (!q) return set_error(GSMAT_ERR_INVALID_ARG, "query is NULL");
    if (pats) *pats = q->pats.data();
    if (n_pats) *n_pats = (int32_t)q->pats.size();
    if (n_vars) *n_vars = q->n_vars;
    if (proj) *proj = q->proj.data();
    if (n_proj) *n_proj = (int32_t)q->proj.size();
    if (distinct) *distinct = q->distinct;
    return GSMAT_OK;
}

const char *sparql_var_name(const gsmat_sparql *q, int32_t v) {
    if (!q || v < 0 || v >= q->n_vars) return nullptr;
    return q->var_names[(size_t)v].c_str();
}

void sparql_free(gsmat_sparql *q) { delete q; }

}  // namespace gs
