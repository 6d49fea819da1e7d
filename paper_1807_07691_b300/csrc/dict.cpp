// String dictionary (Sec. 5.2, "Generation of RDF Cubes"): h_p numbers the
// predicates and h_so the subjects and objects (one numbering for both),
// each from 1 in order of first occurrence as the triples are read, the
// subject of a triple before its object.  Host code; the encoded triples
// feed gsmat_load.
#include <string.h>

#include <algorithm>
#include <memory>
#include <string>
#include <string_view>
#include <unordered_map>
#include <vector>

#include "dict.h"
#include "text.h"

namespace gs {

namespace {

// One numbering: identity text -> code (1, 2, ...), code -> text.  Texts
// are stored NUL-terminated, back to back, in blocks that never move; the
// index is an open-addressing table, at most half full and probed
// linearly, whose slots carry the hash and the text's place so that a
// lookup touches one slot and one text.
struct Codebook {
    static constexpr size_t kBlock = (size_t)1 << 20;
    struct Slot {
        uint64_t h;
        const char *p;
        uint32_t len;
        int32_t code;  // 0: empty
    };
    std::vector<std::unique_ptr<char[]>> blocks;
    size_t block_used = kBlock, block_cap = kBlock;
    std::vector<std::string_view> texts;  // code - 1 -> text
    std::vector<Slot> slots;
    size_t mask = 0;

    // FNV-1a over the bytes, then the 64-bit finaliser of MurmurHash3 (the
    // low bits pick the slot)
    static uint64_t hash(std::string_view t) {
        uint64_t h = 1469598103934665603ull;
        for (unsigned char c : t) h = (h ^ c) * 1099511628211ull;
        h ^= h >> 33;
        h *= 0xff51afd7ed558ccdull;
        h ^= h >> 33;
        return h;
    }

    size_t probe(std::string_view t, uint64_t h) const {
        size_t i = h & mask;
        for (;;) {
            const Slot &s = slots[i];
            if (s.code == 0 || (s.h == h && s.len == t.size() && memcmp(s.p, t.data(), t.size()) == 0)) return i;
            i = (i + 1) & mask;
        }
    }

    int32_t find(std::string_view t) const {
        if (texts.empty()) return 0;
        return slots[probe(t, hash(t))].code;
    }

    void rehash(size_t n_slots) {
        slots.assign(n_slots, Slot{0, nullptr, 0, 0});
        mask = n_slots - 1;
        for (size_t c = 1; c <= texts.size(); ++c) {
            const std::string_view t = texts[c - 1];
            const uint64_t h = hash(t);
            size_t i = h & mask;
            while (slots[i].code != 0) i = (i + 1) & mask;
            slots[i] = Slot{h, t.data(), (uint32_t)t.size(), (int32_t)c};
        }
    }

    std::string_view store(std::string_view t) {
        if (block_used + t.size() + 1 > block_cap) {
            block_cap = std::max(kBlock, t.size() + 1);
            blocks.emplace_back(new char[block_cap]);
            block_used = 0;
        }
        char *p = blocks.back().get() + block_used;
        memcpy(p, t.data(), t.size());
        p[t.size()] = 0;
        block_used += t.size() + 1;
        return std::string_view(p, t.size());
    }

    // The code of t, numbering it if new; -1 when the numbering is full.
    int32_t get(std::string_view t) {
        if (2 * (texts.size() + 1) > slots.size()) rehash(std::max<size_t>(1024, 2 * slots.size()));
        const uint64_t h = hash(t);
        const size_t i = probe(t, h);
        if (slots[i].code != 0) return slots[i].code;
        if (texts.size() >= (size_t)INT32_MAX || t.size() > UINT32_MAX) return -1;
        const std::string_view kept = store(t);
        texts.push_back(kept);
        slots[i] = Slot{h, kept.data(), (uint32_t)kept.size(), (int32_t)texts.size()};
        return slots[i].code;
    }

    // Forget every term numbered after the first `size` (their bytes stay
    // in the blocks, unused).
    void truncate(size_t size) {
        if (texts.size() <= size) return;
        texts.resize(size);
        rehash(std::max<size_t>(1024, slots.size()));
    }

    const char *c_str(int32_t code) const { return texts[(size_t)code - 1].data(); }
    size_t size() const { return texts.size(); }
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

// Read the statements of a data text; emit(s, p, o) with identity texts
// (views valid during the call).
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
            return emit(txt::identity(s, pf, es), txt::identity(p, pf, ep), txt::identity(o, pf, eo));
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
    // one pass; a text that turns out bad is rolled back, so that it changes
    // nothing (the terms it numbered are forgotten again)
    const size_t old = d->triples.size(), old_p = d->p.size(), old_so = d->so.size();
    const int rc = read_data(sv, [&](std::string_view s, std::string_view p, std::string_view o) {
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
        d->triples.resize(old);
        d->p.truncate(old_p);
        d->so.truncate(old_so);
        return rc;
    }
    if (n_added) *n_added = (int64_t)(d->triples.size() - old) / 3;
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
    if (n_predicates) *n_predicates = (int32_t)d->p.size();
    if (n_terms) *n_terms = (int32_t)d->so.size();
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
    const int64_t size = (int64_t)cb.size();
    for (int64_t i = 0; i < n; ++i) {
        if (codes[i] < 1 || codes[i] > size) {
            return set_error(GSMAT_ERR_INVALID_ARG, "code %d at %lld is not in the dictionary", codes[i], (long long)i);
        }
        terms[i] = cb.c_str(codes[i]);
        if (lens) lens[i] = (int32_t)cb.texts[(size_t)codes[i] - 1].size();
    }
    return GSMAT_OK;
}

}  // namespace gs
