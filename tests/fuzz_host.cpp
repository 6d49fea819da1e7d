/* Damaged data and query texts through the library's host readers (the
 * dictionary and the SPARQL reader) and random BGPs through both planners,
 * built with AddressSanitizer and UndefinedBehaviorSanitizer by
 * tests/test_host_fuzz.py: any read past a buffer, overflow or leak fails
 * the run.  Every text is copied into an exact-size heap buffer. */
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>
#include "dict.h"
#include "plan.h"
// The library's error recorder is not linked in: a stand-in that only
// returns the status.
namespace gs {
int set_error(int s, const char *, ...) { return s; }
}
static const char *kSeeds[] = {
  "@prefix ex: <http://x.org/> .\nex:a a ex:C ; ex:p \"x y\"@en-GB , \"3\"^^ex:int ; ex:q _:b1 .\n<http://x.org/a> ex:p \"say \\\"hi\\\"\" .\n_:b1 <http://e/q> ex:a.\n",
  "A :likes I1 .\nA :likes I2 .\nA :follows B .\n",
  "PREFIX ex: <http://x.org/>\nselect distinct $y ?x where { ?x ex:p ex:a , \"v\"@en ; ex:q ?y ; a ?z . ?y <http://x.org/p> ?x }",
  "SELECT * { ?s 7 12 . ?s 3 ?t } LIMIT 5",
  "SELECT ?x { ?x :q1 \"l\"^^<http://t/x> . OPTIONAL { ?y :q2 ?z } }",
};
int main(int argc, char **argv) {
  std::mt19937_64 rng(12345);
  const char alphabet[] = "<>\"{};,.?$#@^ \n:_ax1\\";
  long ok = 0, err = 0;
  const int iters = argc > 1 ? atoi(argv[1]) : 30000;
  for (int it = 0; it < iters; ++it) {
    std::string s = kSeeds[rng() % (sizeof(kSeeds) / sizeof(kSeeds[0]))];
    int muts = 1 + rng() % 6;
    for (int m = 0; m < muts; ++m) {
      size_t i = s.empty() ? 0 : rng() % (s.size() + 1);
      int op = rng() % 3;
      if (op == 0 && !s.empty() && i < s.size()) s.erase(i, 1 + rng() % 3);
      else if (op == 1) s.insert(i, 1, alphabet[rng() % (sizeof(alphabet) - 1)]);
      else if (!s.empty() && i < s.size()) s[i] = alphabet[rng() % (sizeof(alphabet) - 1)];
    }
    // exact-size heap copy so that any read past the end is caught
    char *buf = new char[s.size() ? s.size() : 1];
    memcpy(buf, s.data(), s.size());
    gsmat_dict *d; gs::dict_create(&d);
    if (it % 7 == 0) gs::dict_set_threads(d, 1 + it % 5);
    int64_t n;
    int rc = gs::dict_add_text(d, buf, (int64_t)s.size(), &n);
    (rc == 0 ? ok : err)++;
    gsmat_sparql *q = nullptr;
    rc = gs::sparql_parse(it % 2 ? d : nullptr, buf, (int64_t)s.size(), &q);
    (rc == 0 ? ok : err)++;
    if (q) {
      const gsmat_pattern *p; const int32_t *pr; int32_t np, nv, npr, di;
      gs::sparql_info(q, &p, &np, &nv, &pr, &npr, &di);
      for (int v = 0; v < nv; ++v) if (!gs::sparql_var_name(q, v)) return 3;
      gs::sparql_free(q);
    }
    const int32_t *t; gs::dict_triples(d, &t, &n);
    int32_t npred, nterm; gs::dict_size(d, &npred, &nterm);
    std::vector<int32_t> codes; for (int c = 1; c <= nterm; ++c) codes.push_back(c);
    std::vector<const char*> terms(codes.size() + 1); std::vector<int32_t> lens(codes.size() + 1);
    if (!codes.empty() && gs::dict_decode(d, GSMAT_DICT_SO, codes.data(), (int64_t)codes.size(), terms.data(), lens.data()) != 0) return 4;
    gs::dict_free(d);
    delete[] buf;
  }
  std::mt19937_64 prng(7);
  for (int it = 0; it < iters / 10; ++it) {
    int n = 1 + prng() % 10, nv = 1 + prng() % 6;
    std::vector<gsmat_pattern> p(n);
    std::vector<int64_t> keys(n);
    std::vector<gsmat_pred_stats> st(n);
    for (int i = 0; i < n; ++i) {
      p[i] = gsmat_pattern{(int32_t)(prng() % nv), (int32_t)(prng() % 5), (int32_t)(prng() % nv),
                           (uint8_t)(prng() % 5 != 0), 0, (uint8_t)(prng() % 5 != 0), 0};
      keys[i] = (int64_t)(prng() % 100000);
      st[i] = gsmat_pred_stats{p[i].p, (int32_t)(prng() % 100000), (int32_t)(prng() % 1000), (int32_t)(prng() % 1000)};
    }
    std::vector<int32_t> order(n), kinds(n);
    std::vector<double> est(n);
    if (gs::plan_bgp_cost(p.data(), n, keys.data(), st.data(), order.data(), kinds.data(), est.data()) != 0) return 5;
    std::vector<int> seen(n, 0);
    for (int i = 0; i < n; ++i) {
      if (order[i] < 0 || order[i] >= n || seen[order[i]]++) return 6;
    }
  }
  printf("fuzz ok: %ld accepted, %ld rejected\n", ok, err);
  return 0;
}
