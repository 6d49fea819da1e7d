/* A plain C client of libgsmat's host entry points (no GPU needed): the
 * dictionary, the SPARQL reader and both planners on the paper's D_G
 * example.  Prints one line per check; tests/test_c_client.py compiles,
 * runs and reads it. */
#include <stdio.h>
#include <string.h>

#include "gsmat.h"

static const char *kData =
    "A :likes I1 .\nA :likes I2 .\nA :follows B .\nB :related h .\nB :follows C .\n"
    "B :follows D .\nC :likes I2 .\nC :follows D .\nD :related h .\n";
static const char *kQuery =
    "SELECT ?x ?y ?z ?w WHERE { ?x :follows ?y . ?y :follows ?z . ?x :likes ?w . ?z :likes ?w .}";

int main(void) {
    gsmat_dict *d = NULL;
    int64_t n = 0;
    if (gsmat_dict_create(&d) != GSMAT_OK) return 1;
    if (gsmat_dict_add_text(d, kData, (int64_t)strlen(kData), &n) != GSMAT_OK) return 2;
    const int32_t *t = NULL;
    gsmat_dict_triples(d, &t, &n);
    printf("triples %lld:", (long long)n);
    for (int64_t i = 0; i < 3 * n; ++i) printf(" %d", t[i]);
    printf("\n");
    int32_t np = 0, nt = 0;
    gsmat_dict_size(d, &np, &nt);
    printf("sizes %d %d\n", np, nt);
    int32_t codes[4] = {1, 3, 6, 4};
    const char *terms[4];
    int32_t lens[4];
    if (gsmat_dict_decode(d, GSMAT_DICT_SO, codes, 4, terms, lens) != GSMAT_OK) return 3;
    printf("decode %s %s %s %s\n", terms[0], terms[1], terms[2], terms[3]);
    int32_t bad = 99;
    printf("decode_bad %d\n", gsmat_dict_decode(d, GSMAT_DICT_SO, &bad, 1, terms, lens));

    gsmat_sparql *q = NULL;
    if (gsmat_sparql_parse(d, kQuery, (int64_t)strlen(kQuery), &q) != GSMAT_OK) return 4;
    const gsmat_pattern *pats = NULL;
    const int32_t *proj = NULL;
    int32_t n_pats = 0, n_vars = 0, n_proj = 0, distinct = 0;
    gsmat_sparql_info(q, &pats, &n_pats, &n_vars, &proj, &n_proj, &distinct);
    printf("bgp %d %d:", n_pats, n_vars);
    for (int i = 0; i < n_pats; ++i) printf(" (%d %d %d %d %d)", pats[i].s, pats[i].p, pats[i].o, pats[i].s_var, pats[i].o_var);
    printf("\n");
    printf("vars");
    for (int v = 0; v < n_vars; ++v) printf(" %s", gsmat_sparql_var_name(q, v));
    printf(" proj %d distinct %d\n", n_proj, distinct);

    /* plan with m = nnz per predicate: likes 3, follows 4 */
    int64_t keys[4];
    gsmat_pred_stats st[4];
    memset(st, 0, sizeof(st));
    for (int i = 0; i < n_pats; ++i) {
        const int likes = pats[i].p == 1;
        keys[i] = likes ? 3 : 4;
        st[i].pred_id = pats[i].p;
        st[i].nnz = likes ? 3 : 4;
        st[i].nr_s = likes ? 2 : 3;
        st[i].nr_o = likes ? 2 : 3;
    }
    int32_t order[4], kinds[4];
    double est[4];
    if (gsmat_plan(pats, n_pats, n_vars, keys, st, order, kinds, est) != GSMAT_OK) return 5;
    printf("plan %d %d %d %d\n", order[0], order[1], order[2], order[3]);
    if (gsmat_plan_cost(pats, n_pats, n_vars, keys, st, order, kinds, est) != GSMAT_OK) return 6;
    printf("plan_cost %d %d %d %d\n", order[0], order[1], order[2], order[3]);

    const char *bad_q = "SELECT ?x { ?x ?p ?y }";
    gsmat_sparql *q2 = NULL;
    printf("unsupported %d\n", gsmat_sparql_parse(d, bad_q, (int64_t)strlen(bad_q), &q2));
    printf("strerror %s\n", gsmat_strerror(GSMAT_ERR_UNSUPPORTED));
    gsmat_sparql_free(q);
    gsmat_dict_free(d);
    printf("ok\n");
    return 0;
}
