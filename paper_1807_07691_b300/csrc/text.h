// Lexer and statement reader shared by the dictionary loader (data text)
// and the SPARQL reader (query text).  Host code.
//
// Tokens: <iri> (no whitespace inside), "literal" (backslash escapes) with
// an optional @lang or ^^datatype (<iri> or a prefixed name), the
// punctuation { } ; , . and otherwise a word: a maximal run of bytes other
// than whitespace and < > " { } ; , .  A word that starts with ? or $ is a
// variable (ASCII letters, digits and _ after the sigil).  '#' where a token
// would start opens a comment to the end of the line.
#pragma once

#include <stdint.h>

#include <string>
#include <string_view>
#include <unordered_map>

#include "../../include/gsmat.h"

namespace gs {

int set_error(int status, const char *fmt, ...);

namespace txt {

enum Kind { kEnd, kIri, kLit, kWord, kVar, kPunct };

struct Tok {
    Kind kind = kEnd;
    // kIri: the IRI with its brackets; kLit: the quoted body with any
    // @lang; kWord: the word; kVar: the name without its sigil; kPunct: the
    // character
    std::string_view text;
    Kind dtype_kind = kEnd;  // kLit with ^^: kIri or kWord
    std::string_view dtype;
};

// Byte classes: whitespace, and the bytes that end a word.
struct ByteClass {
    uint8_t c[256];
    constexpr ByteClass() : c() {
        const char ws[] = " \t\r\n";
        const char sp[] = "<>\"{};,.";
        for (const char *q = ws; *q; ++q) c[(unsigned char)*q] = 3;  // whitespace ends a word too
        for (const char *q = sp; *q; ++q) c[(unsigned char)*q] = 2;
    }
};
inline constexpr ByteClass kByteClass{};
inline bool is_ws(char c) { return kByteClass.c[(unsigned char)c] == 3; }
inline bool is_special(char c) { return kByteClass.c[(unsigned char)c] == 2; }
inline bool ends_word(char c) { return kByteClass.c[(unsigned char)c] != 0; }
inline bool is_alnum_ascii(char c) {
    return (c >= '0' && c <= '9') || (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z');
}

// ASCII case-insensitive equality with an upper-case keyword.
inline bool keyword_is(std::string_view w, const char *kw) {
    size_t i = 0;
    for (; kw[i]; ++i) {
        if (i >= w.size()) return false;
        char c = w[i];
        if (c >= 'a' && c <= 'z') c = (char)(c - 32);
        if (c != kw[i]) return false;
    }
    return i == w.size();
}

class Lexer {
   public:
    explicit Lexer(std::string_view s) : s_(s) {}

    // The next token without consuming it.
    int peek(const Tok **t) {
        if (!have_) {
            rc_ = scan(la_);
            have_ = true;
        }
        *t = &la_;
        return rc_;
    }
    int take(Tok &t) {
        const Tok *p;
        const int rc = peek(&p);
        if (rc != GSMAT_OK) return rc;
        t = *p;
        have_ = false;
        return GSMAT_OK;
    }

   private:
    int scan(Tok &t);

    std::string_view s_;
    size_t i_ = 0;
    Tok la_;
    bool have_ = false;
    int rc_ = GSMAT_OK;
};

inline int Lexer::scan(Tok &t) {
    const size_t n = s_.size();
    for (;;) {
        while (i_ < n && is_ws(s_[i_])) ++i_;
        if (i_ < n && s_[i_] == '#') {
            while (i_ < n && s_[i_] != '\n') ++i_;
            continue;
        }
        break;
    }
    t = Tok();
    if (i_ >= n) return GSMAT_OK;
    const char c = s_[i_];
    if (c == '{' || c == '}' || c == ';' || c == ',' || c == '.') {
        t.kind = kPunct;
        t.text = s_.substr(i_, 1);
        ++i_;
        return GSMAT_OK;
    }
    if (c == '<') {
        size_t j = i_ + 1;
        for (; j < n && s_[j] != '>'; ++j) {
            if (is_ws(s_[j])) return set_error(GSMAT_ERR_INVALID_ARG, "whitespace inside an IRI at byte %zu", j);
        }
        if (j >= n) return set_error(GSMAT_ERR_INVALID_ARG, "unterminated IRI at byte %zu", i_);
        t.kind = kIri;
        t.text = s_.substr(i_, j + 1 - i_);
        i_ = j + 1;
        return GSMAT_OK;
    }
    if (c == '"') {
        size_t j = i_ + 1;
        while (j < n && s_[j] != '"') j += s_[j] == '\\' ? 2 : 1;
        if (j >= n) return set_error(GSMAT_ERR_INVALID_ARG, "unterminated literal at byte %zu", i_);
        ++j;  // the closing quote
        size_t body_end = j;
        if (j < n && s_[j] == '@') {
            size_t k = j + 1;
            while (k < n && (is_alnum_ascii(s_[k]) || s_[k] == '-')) ++k;
            body_end = j = k;
        } else if (j + 1 < n && s_[j] == '^' && s_[j + 1] == '^') {
            const size_t k = j + 2;
            if (k < n && s_[k] == '<') {
                size_t e = k;
                while (e < n && s_[e] != '>') ++e;
                if (e >= n) return set_error(GSMAT_ERR_INVALID_ARG, "unterminated datatype IRI at byte %zu", k);
                t.dtype_kind = kIri;
                t.dtype = s_.substr(k, e + 1 - k);
                j = e + 1;
            } else {
                size_t e = k;
                while (e < n && !ends_word(s_[e])) ++e;
                if (e == k) return set_error(GSMAT_ERR_INVALID_ARG, "empty datatype at byte %zu", k);
                t.dtype_kind = kWord;
                t.dtype = s_.substr(k, e - k);
                j = e;
            }
        }
        t.kind = kLit;
        t.text = s_.substr(i_, body_end - i_);
        i_ = j;
        return GSMAT_OK;
    }
    if (c == '>') return set_error(GSMAT_ERR_INVALID_ARG, "unexpected '>' at byte %zu", i_);
    size_t j = i_;
    while (j < n && !ends_word(s_[j])) ++j;
    const std::string_view w = s_.substr(i_, j - i_);
    i_ = j;
    if (w[0] == '?' || w[0] == '$') {
        const std::string_view name = w.substr(1);
        bool ok = !name.empty();
        for (char ch : name) ok = ok && (is_alnum_ascii(ch) || ch == '_');
        if (!ok) return set_error(GSMAT_ERR_INVALID_ARG, "bad variable '%.*s'", (int)w.size(), w.data());
        t.kind = kVar;
        t.text = name;
        return GSMAT_OK;
    }
    t.kind = kWord;
    t.text = w;
    return GSMAT_OK;
}

using Prefixes = std::unordered_map<std::string, std::string>;  // name (no ':') -> IRI with brackets

// Identity text of a term: a prefixed name whose prefix is declared becomes
// <IRI + local part> (also as a literal's datatype); anything else is kept
// as written.
inline void expand_word(std::string_view w, const Prefixes &pf, std::string &out) {
    const size_t colon = w.find(':');
    if (colon != std::string_view::npos) {
        auto it = pf.find(std::string(w.substr(0, colon)));
        if (it != pf.end()) {
            out.append(it->second, 0, it->second.size() - 1);  // without '>'
            out.append(w.substr(colon + 1));
            out.push_back('>');
            return;
        }
    }
    out.append(w);
}

// The identity text of t: a view of the token itself when nothing expands
// (no declared prefix involved), else of `scratch` holding the expansion.
inline std::string_view identity(const Tok &t, const Prefixes &pf, std::string &scratch);

inline void expand(const Tok &t, const Prefixes &pf, std::string &out) {
    out.clear();
    if (t.kind == kWord) {
        expand_word(t.text, pf, out);
        return;
    }
    out.append(t.text);
    if (t.kind == kLit && t.dtype_kind != kEnd) {
        out.append("^^");
        if (t.dtype_kind == kIri) out.append(t.dtype);
        else expand_word(t.dtype, pf, out);
    }
}

inline bool declared_prefix(std::string_view w, const Prefixes &pf) {
    if (pf.empty()) return false;
    const size_t colon = w.find(':');
    return colon != std::string_view::npos && pf.count(std::string(w.substr(0, colon))) != 0;
}

inline std::string_view identity(const Tok &t, const Prefixes &pf, std::string &scratch) {
    if (t.kind == kWord && declared_prefix(t.text, pf)) {
        expand(t, pf, scratch);
        return scratch;
    }
    if (t.kind == kLit && t.dtype_kind != kEnd) {
        if (t.dtype_kind == kWord && declared_prefix(t.dtype, pf)) {
            expand(t, pf, scratch);
            return scratch;
        }
        // body, "^^" and datatype lie back to back in the text
        return std::string_view(t.text.data(), (size_t)(t.dtype.data() + t.dtype.size() - t.text.data()));
    }
    return t.text;
}

constexpr const char *kRdfType = "<http://www.w3.org/1999/02/22-rdf-syntax-ns#type>";

// Keywords that the reader leaves unsupported inside a pattern block.
inline bool unsupported_in_block(std::string_view w) {
    static const char *kw[] = {"FILTER", "OPTIONAL", "UNION", "GRAPH", "MINUS", "BIND", "VALUES", "SERVICE"};
    for (const char *k : kw) {
        if (keyword_is(w, k)) return true;
    }
    return false;
}

// One term of a statement or pattern.  query: variables allowed and block
// keywords unsupported; otherwise (data) variables are invalid.
inline int read_term(Lexer &lx, bool query, const char *what, Tok &t) {
    int rc = lx.take(t);
    if (rc != GSMAT_OK) return rc;
    if (query && t.kind == kWord && unsupported_in_block(t.text)) {
        return set_error(GSMAT_ERR_UNSUPPORTED, "'%.*s' is not supported", (int)t.text.size(), t.text.data());
    }
    if (t.kind == kVar && !query) return set_error(GSMAT_ERR_INVALID_ARG, "a variable in data");
    if (t.kind == kIri || t.kind == kLit || t.kind == kWord || t.kind == kVar) return GSMAT_OK;
    if (t.kind == kEnd) return set_error(GSMAT_ERR_INVALID_ARG, "text ends where a %s is expected", what);
    return set_error(GSMAT_ERR_INVALID_ARG, "'%.*s' where a %s is expected", (int)t.text.size(), t.text.data(), what);
}

inline bool is_punct(const Tok *t, char c) { return t->kind == kPunct && t->text[0] == c; }

// One subject with its predicate-object list (';' repeats the subject, ','
// subject and predicate); emit(s, p, o) for every triple, in text order.
// The predicate word 'a' is rdf:type.
template <class Emit>
int read_subject(Lexer &lx, bool query, Emit &&emit) {
    Tok s, p, o;
    const Tok *nx;
    int rc = read_term(lx, query, "subject", s);
    if (rc != GSMAT_OK) return rc;
    for (;;) {
        if ((rc = read_term(lx, query, "predicate", p)) != GSMAT_OK) return rc;
        if (p.kind == kWord && p.text == "a") {
            p.kind = kIri;
            p.text = kRdfType;
        }
        for (;;) {
            if ((rc = read_term(lx, query, "object", o)) != GSMAT_OK) return rc;
            if ((rc = emit(s, p, o)) != GSMAT_OK) return rc;
            if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
            if (!is_punct(nx, ',')) break;
            Tok skip;
            lx.take(skip);
        }
        if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
        if (!is_punct(nx, ';')) return GSMAT_OK;
        while (is_punct(nx, ';')) {
            Tok skip;
            lx.take(skip);
            if ((rc = lx.peek(&nx)) != GSMAT_OK) return rc;
        }
        if (nx->kind == kPunct || nx->kind == kEnd) return GSMAT_OK;  // a ';' may close the list
    }
}

}  // namespace txt
}  // namespace gs
