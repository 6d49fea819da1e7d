// String dictionary (Sec. 5.2, "Generation of RDF Cubes"): h_p numbers the
// predicates and h_so the subjects and objects (one numbering for both),
// each from 1 in order of first occurrence as the triples are read, the
// subject of a triple before its object.  Host code; the encoded triples
// feed gsmat_load.
//
// A text is read in chunks of statements.  For each chunk the terms of one
// numbering are hashed, then numbered in parallel: the numbering's table is
// split into hash partitions, each thread owns some partitions and walks the
// chunk's terms in order, looking up (or adding, with a provisional mark
// that records the term's first position) those that fall in its
// partitions.  An exclusive scan over the first positions of the new terms
// then gives their codes in order of first occurrence, exactly as a
// sequential reading would.
#include <string.h>

#include <algorithm>
#include <deque>
#include <memory>
#include <string>
#include <string_view>
#include <system_error>
#include <thread>
#include <vector>

#include "dict.h"
#include "text.h"

namespace gs {

namespace {

// FNV-1a over the bytes, then the 64-bit finaliser of MurmurHash3: the top
// bits pick the partition, the low bits the slot.
uint64_t term_hash(std::string_view t) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : t) h = (h ^ c) * 1099511628211ull;
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    return h;
}

// Run f(i) for i in [0, n) on up to `threads` threads (inline for one).
template <class F>
void parallel_for(int threads, int n, F &&f) {
    if (threads <= 1 || n <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    const int t = std::min(threads, n);
    for (int k = 0; k < t; ++k) {
        try {
            pool.emplace_back([&, k] {
                for (int i = k; i < n; i += t) f(i);
            });
        } catch (const std::system_error &) {
            for (int i = k; i < n; i += t) f(i);  // no thread to be had: this share inline
        }
    }
    for (auto &th : pool) th.join();
}

// One hash partition of a numbering: an open-addressing table, at most
// half full, probed linearly; texts stored NUL-terminated, back to back,
// in blocks that never move.  A slot's code is the term's code, or -(first
// position + 1) while the term is new in the chunk being read.
struct Partition {
    static constexpr size_t kBlock = (size_t)1 << 18;
    struct Slot {
        uint64_t h;
        const char *p;
        uint32_t len;
        int32_t code;  // 0: empty
    };
    std::vector<std::unique_ptr<char[]>> blocks;
    size_t block_used = kBlock, block_cap = kBlock;
    std::vector<Slot> slots;
    size_t mask = 0, used = 0;

    size_t probe(std::string_view t, uint64_t h) const {
        size_t i = h & mask;
        for (;;) {
            const Slot &s = slots[i];
            if (s.code == 0 || (s.h == h && s.len == t.size() && memcmp(s.p, t.data(), t.size()) == 0)) return i;
            i = (i + 1) & mask;
        }
    }
    int32_t find(std::string_view t, uint64_t h) const { return slots.empty() ? 0 : slots[probe(t, h)].code; }

    void grow() {
        std::vector<Slot> old = std::move(slots);
        const size_t n = std::max<size_t>(64, 2 * old.size());
        slots.assign(n, Slot{0, nullptr, 0, 0});
        mask = n - 1;
        for (const Slot &s : old) {
            if (s.code == 0) continue;
            size_t i = s.h & mask;
            while (slots[i].code != 0) i = (i + 1) & mask;
            slots[i] = s;
        }
    }
    const char *store(std::string_view t) {
        if (block_used + t.size() + 1 > block_cap) {
            block_cap = std::max(kBlock, t.size() + 1);
            blocks.emplace_back(new char[block_cap]);
            block_used = 0;
        }
        char *p = blocks.back().get() + block_used;
        memcpy(p, t.data(), t.size());
        p[t.size()] = 0;
        block_used += t.size() + 1;
        return p;
    }
    // The slot's code for t, adding it with `code_if_new` when absent.
    int32_t find_or_add(std::string_view t, uint64_t h, int32_t code_if_new) {
        if (2 * (used + 1) > slots.size()) grow();
        const size_t i = probe(t, h);
        if (slots[i].code != 0) return slots[i].code;
        slots[i] = Slot{h, store(t), (uint32_t)t.size(), code_if_new};
        ++used;
        return code_if_new;
    }
    // Drop every term whose code is above `keep` (or still provisional).
    void drop_above(int32_t keep) {
        std::vector<Slot> old = std::move(slots);
        slots.assign(old.size(), Slot{0, nullptr, 0, 0});
        used = 0;
        for (const Slot &s : old) {
            if (s.code <= 0 || s.code > keep) continue;
            size_t i = s.h & mask;
            while (slots[i].code != 0) i = (i + 1) & mask;
            slots[i] = s;
            ++used;
        }
    }
};

// One numbering (h_p or h_so): code -> text, text -> code.
struct Codebook {
    static constexpr int kParts = 64;
    Partition part[kParts];
    std::vector<std::string_view> texts;  // code - 1 -> text

    static int part_of(uint64_t h) { return (int)(h >> 58); }

    int32_t find(std::string_view t) const {
        const uint64_t h = term_hash(t);
        const int32_t c = part[part_of(h)].find(t, h);
        return c > 0 ? c : 0;
    }
    size_t size() const { return texts.size(); }

    // Codes of terms[0..m) by first occurrence, numbering the new ones after
    // the existing codes.  CAPACITY (and nothing numbered) above 2^31 - 1.
    int number(const std::vector<std::string_view> &terms, int32_t *codes, int threads) {
        const size_t m = terms.size();
        if (m == 0) return GSMAT_OK;
        std::vector<uint64_t> h(m);
        const int chunks = threads > 1 ? threads * 4 : 1;
        parallel_for(threads, chunks, [&](int c) {
            const size_t lo = m * c / chunks, hi = m * (c + 1) / chunks;
            for (size_t i = lo; i < hi; ++i) h[i] = term_hash(terms[i]);
        });
        // each thread owns the partitions q = k (mod T) and walks the terms
        // in order, so a new term's provisional mark holds its first position
        const int T = std::max(1, std::min(threads, kParts));
        std::vector<uint8_t> first(m, 0);
        parallel_for(T, T, [&](int k) {
            for (size_t i = 0; i < m; ++i) {
                const int q = part_of(h[i]);
                if (q % T != k) continue;
                const int32_t c = part[q].find_or_add(terms[i], h[i], -(int32_t)(i + 1));
                codes[i] = c;
                if (c == -(int32_t)(i + 1)) first[i] = 1;
            }
        });
        // codes of the new terms: the base plus the rank of the first position
        std::vector<int32_t> rank(m);
        int64_t n_new = 0;
        for (size_t i = 0; i < m; ++i) {
            rank[i] = (int32_t)n_new;
            n_new += first[i];
        }
        const int64_t base = (int64_t)texts.size();
        if (base + n_new > INT32_MAX) {
            parallel_for(T, kParts, [&](int q) { part[q].drop_above((int32_t)base); });
            return set_error(GSMAT_ERR_CAPACITY, "more than 2^31 - 1 terms");
        }
        texts.resize((size_t)(base + n_new));
        parallel_for(T, kParts, [&](int q) {
            for (Partition::Slot &s : part[q].slots) {
                if (s.code >= 0) continue;
                const size_t fp = (size_t)(-s.code - 1);
                s.code = (int32_t)(base + rank[fp] + 1);
                texts[(size_t)s.code - 1] = std::string_view(s.p, s.len);
            }
        });
        parallel_for(threads, chunks, [&](int c) {
            const size_t lo = m * c / chunks, hi = m * (c + 1) / chunks;
            for (size_t i = lo; i < hi; ++i) {
                if (codes[i] < 0) codes[i] = (int32_t)(base + rank[(size_t)(-codes[i] - 1)] + 1);
            }
        });
        return GSMAT_OK;
    }

    // Forget every term numbered after the first `keep`.
    void truncate(size_t keep) {
        if (texts.size() <= keep) return;
        texts.resize(keep);
        for (int q = 0; q < kParts; ++q) part[q].drop_above((int32_t)keep);
    }
};

}  // namespace

}  // namespace gs

struct gsmat_dict {
    gs::Codebook p, so;
    std::vector<int32_t> triples;  // (s, p, o) codes, in text order
    int threads = 0;               // 0: automatic
};

namespace gs {

int32_t dict_code(const gsmat_dict *d, int kind, std::string_view text) {
    return kind == GSMAT_DICT_P ? d->p.find(text) : d->so.find(text);
}

namespace {

// Statements of a data text, a chunk at a time: identity texts of the
// subjects and objects (interleaved, subject first) and of the predicates.
// Views point into the text or, for expanded names, into `held_`.
class DataReader {
   public:
    explicit DataReader(std::string_view text) : lx_(text) {}

    // Read up to max_triples statements' triples; *done at the end of text.
    int next(size_t max_triples, std::vector<std::string_view> &so, std::vector<std::string_view> &p, bool *done) {
        so.clear();
        p.clear();
        held_.clear();
        *done = false;
        while (p.size() < max_triples) {
            const txt::Tok *nx;
            int rc = lx_.peek(&nx);
            if (rc != GSMAT_OK) return rc;
            if (nx->kind == txt::kEnd) {
                *done = true;
                return GSMAT_OK;
            }
            if (nx->kind == txt::kWord && nx->text == "@prefix") {
                txt::Tok kw, name, iri, dot;
                lx_.take(kw);
                if ((rc = lx_.take(name)) != GSMAT_OK || (rc = lx_.take(iri)) != GSMAT_OK ||
                    (rc = lx_.take(dot)) != GSMAT_OK) {
                    return rc;
                }
                if (name.kind != txt::kWord || name.text.empty() || name.text.back() != ':' || iri.kind != txt::kIri ||
                    !txt::is_punct(&dot, '.')) {
                    return set_error(GSMAT_ERR_INVALID_ARG, "bad @prefix");
                }
                pf_[std::string(name.text.substr(0, name.text.size() - 1))] = std::string(iri.text);
                continue;
            }
            rc = txt::read_subject(lx_, false, [&](const txt::Tok &s, const txt::Tok &pr, const txt::Tok &o) {
                if (s.kind == txt::kLit || pr.kind == txt::kLit) {
                    return set_error(GSMAT_ERR_INVALID_ARG, "a literal can only be an object");
                }
                so.push_back(keep(txt::identity(s, pf_, scratch_)));
                p.push_back(keep(txt::identity(pr, pf_, scratch_)));
                so.push_back(keep(txt::identity(o, pf_, scratch_)));
                return GSMAT_OK;
            });
            if (rc != GSMAT_OK) return rc;
            txt::Tok dot;
            if ((rc = lx_.take(dot)) != GSMAT_OK) return rc;
            if (!txt::is_punct(&dot, '.')) return set_error(GSMAT_ERR_INVALID_ARG, "statement not ended by '.'");
        }
        return GSMAT_OK;
    }

   private:
    // A view that outlives the scratch buffer it may point into.
    std::string_view keep(std::string_view v) {
        if (v.data() != scratch_.data()) return v;
        held_.emplace_back(v);
        return held_.back();
    }

    txt::Lexer lx_;
    txt::Prefixes pf_;
    std::string scratch_;
    std::deque<std::string> held_;
};

int auto_threads(const gsmat_dict *d, size_t n_triples) {
    if (d->threads > 0) return d->threads;
    if (n_triples < ((size_t)1 << 16)) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw, 16u));
}

}  // namespace

int dict_create(gsmat_dict **out) {
    if (!out) return set_error(GSMAT_ERR_INVALID_ARG, "out is NULL");
    *out = new gsmat_dict();
    return GSMAT_OK;
}

void dict_free(gsmat_dict *d) { delete d; }

int dict_set_threads(gsmat_dict *d, int32_t n_threads) {
    if (!d || n_threads < 0 || n_threads > 256) return set_error(GSMAT_ERR_INVALID_ARG, "dict or thread count");
    d->threads = n_threads;
    return GSMAT_OK;
}

int dict_add_text(gsmat_dict *d, const char *text, int64_t len, int64_t *n_added) {
    if (!d || (!text && len > 0) || len < 0) return set_error(GSMAT_ERR_INVALID_ARG, "dict, text or length");
    // a text that turns out bad (or too big) is rolled back: the dictionary
    // is left as it was
    const size_t old = d->triples.size(), old_p = d->p.size(), old_so = d->so.size();
    auto rollback = [&](int rc) {
        d->triples.resize(old);
        d->p.truncate(old_p);
        d->so.truncate(old_so);
        return rc;
    };
    DataReader rd(std::string_view(text ? text : "", (size_t)len));
    std::vector<std::string_view> so, p;
    std::vector<int32_t> cso, cp;
    constexpr size_t kChunk = (size_t)1 << 22;  // triples per chunk
    for (bool done = false; !done;) {
        int rc = rd.next(kChunk, so, p, &done);
        if (rc != GSMAT_OK) return rollback(rc);
        const size_t n = p.size();
        if (n == 0) continue;
        const int threads = auto_threads(d, n);
        cso.resize(so.size());
        cp.resize(n);
        if ((rc = d->so.number(so, cso.data(), threads)) != GSMAT_OK) return rollback(rc);
        if ((rc = d->p.number(p, cp.data(), threads)) != GSMAT_OK) return rollback(rc);
        const size_t at = d->triples.size();
        d->triples.resize(at + 3 * n);
        int32_t *t = d->triples.data() + at;
        for (size_t i = 0; i < n; ++i) {
            t[3 * i] = cso[2 * i];
            t[3 * i + 1] = cp[i];
            t[3 * i + 2] = cso[2 * i + 1];
        }
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
        const std::string_view t = cb.texts[(size_t)codes[i] - 1];
        terms[i] = t.data();  // NUL-terminated in its block
        if (lens) lens[i] = (int32_t)t.size();
    }
    return GSMAT_OK;
}

}  // namespace gs
