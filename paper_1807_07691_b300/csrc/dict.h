// String dictionary and SPARQL reader (host code; see dict.cpp, sparql.cpp).
#pragma once

#include <stdint.h>

#include <string_view>

#include "../../include/gsmat.h"

namespace gs {

int dict_create(gsmat_dict **out);
void dict_free(gsmat_dict *d);
int dict_set_threads(gsmat_dict *d, int32_t n_threads);
int dict_add_text(gsmat_dict *d, const char *text, int64_t len, int64_t *n_added);
int dict_triples(const gsmat_dict *d, const int32_t **triples, int64_t *n);
int dict_size(const gsmat_dict *d, int32_t *n_predicates, int32_t *n_terms);
int dict_lookup(const gsmat_dict *d, int kind, const char *term, int64_t len, int32_t *code);
int dict_decode(const gsmat_dict *d, int kind, const int32_t *codes, int64_t n, const char **terms, int32_t *lens);
// Code of an identity text (0 if absent).
int32_t dict_code(const gsmat_dict *d, int kind, std::string_view text);

int sparql_parse(const gsmat_dict *d, const char *text, int64_t len, gsmat_sparql **out);
int sparql_info(const gsmat_sparql *q, const gsmat_pattern **pats, int32_t *n_pats, int32_t *n_vars,
                const int32_t **proj, int32_t *n_proj, int32_t *distinct);
const char *sparql_var_name(const gsmat_sparql *q, int32_t v);
void sparql_free(gsmat_sparql *q);

}  // namespace gs
