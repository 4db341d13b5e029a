// Reduction stage: weighted CNF -> tensor network (Thm 3.2).
//
// Each clause C becomes the clause tensor B_C over its distinct variables,
// equal to 1 except at the unique falsifying assignment.  Each variable x
// becomes the weight vector [W(x,0), W(x,1)]: the COPY tensor A_x of
// Thm 3.2 with all of its indices (x, C) identified into one hyperedge
// index x, which leaves the contraction unchanged.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

namespace wmc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

}  // namespace wmc

using namespace wmc;

struct wmc_network : public Network {};

extern "C" const char *wmc_last_error(void) { return g_err; }

extern "C" int wmc_network_create(int32_t n_vars, int64_t n_clauses, const int32_t *lits,
                                  const int64_t *clause_off, const double *w_pos,
                                  const double *w_neg, wmc_network_t **out) {
  if (!out) { set_error("out is NULL"); return WMC_EINVAL; }
  *out = nullptr;
  if (n_vars < 0 || n_clauses < 0) { set_error("negative size"); return WMC_EINVAL; }
  if (n_clauses > 0 && (!clause_off)) { set_error("clause_off is NULL"); return WMC_EINVAL; }
  if (n_clauses > 0 && clause_off[0] != 0) { set_error("clause_off[0] must be 0"); return WMC_EINVAL; }
  for (int64_t c = 0; c < n_clauses; ++c)
    if (clause_off[c + 1] < clause_off[c]) { set_error("clause_off not monotone at %lld", (long long)c); return WMC_EINVAL; }
  if (n_clauses > 0 && clause_off[n_clauses] > 0 && !lits) { set_error("lits is NULL"); return WMC_EINVAL; }
  wmc_network *net = new (std::nothrow) wmc_network();
  if (!net) { set_error("out of host memory"); return WMC_ENOMEM; }
  net->n_vars = n_vars;
  net->n_clauses_in = n_clauses;
  try {
    net->w_pos.assign((size_t)n_vars, 1.0);
    net->w_neg.assign((size_t)n_vars, 1.0);
    if (w_pos) std::memcpy(net->w_pos.data(), w_pos, sizeof(double) * (size_t)n_vars);
    if (w_neg) std::memcpy(net->w_neg.data(), w_neg, sizeof(double) * (size_t)n_vars);
    std::vector<int8_t> sign((size_t)n_vars + 1, 0);
    for (int64_t c = 0; c < n_clauses; ++c) {
      Clause cl;
      bool taut = false;
      std::vector<int32_t> touched;
      for (int64_t i = clause_off[c]; i < clause_off[c + 1]; ++i) {
        int32_t l = lits[i];
        int32_t v = l > 0 ? l : -l;
        if (l == 0 || v > n_vars) {
          for (int32_t t : touched) sign[t] = 0;
          delete net;
          set_error("clause %lld: literal %d out of range [1, %d]", (long long)c, l, n_vars);
          return WMC_EINVAL;
        }
        int8_t s = l > 0 ? 1 : -1;
        if (sign[v] == 0) { sign[v] = s; touched.push_back(v); }
        else if (sign[v] != s) taut = true;  // x | ~x: B_C == 1
      }
      for (int32_t t : touched) sign[t] = 0;
      if (taut) continue;
      // distinct variables ascending; a literal +v is falsified by v = 0
      std::vector<std::pair<int32_t, int8_t>> vs;
      for (int64_t i = clause_off[c]; i < clause_off[c + 1]; ++i) {
        int32_t l = lits[i];
        int32_t v = (l > 0 ? l : -l) - 1;
        bool seen = false;
        for (auto &p : vs) seen |= (p.first == v);
        if (!seen) vs.push_back({v, (int8_t)(l > 0 ? 0 : 1)});
      }
      std::sort(vs.begin(), vs.end());
      const bool wide = vs.size() > 62;  // kept as per-literal values (factoring only)
      for (size_t j = 0; j < vs.size(); ++j) {
        cl.vars.push_back(vs[j].first);
        if (wide) cl.fvals.push_back((uint8_t)vs[j].second);
        else if (vs[j].second) cl.fals |= (1ull << j);
      }
      if (cl.vars.empty()) net->has_empty = true;
      net->n_indices_strict += (int64_t)cl.vars.size();
      if ((int64_t)cl.vars.size() > net->max_clause_rank) net->max_clause_rank = (int64_t)cl.vars.size();
      net->clauses.push_back(std::move(cl));
    }
  } catch (const std::bad_alloc &) {
    delete net;
    set_error("out of host memory");
    return WMC_ENOMEM;
  }
  *out = net;
  return WMC_OK;
}

extern "C" void wmc_network_destroy(wmc_network_t *net) { delete net; }

extern "C" int wmc_network_info(const wmc_network_t *net, wmc_network_info_t *out) {
  if (!net || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  std::memset(out, 0, sizeof(*out));
  out->n_vars = net->n_vars;
  out->n_clauses_kept = (int64_t)net->clauses.size();
  out->n_tensors_strict = net->n_vars + (int64_t)net->clauses.size();
  out->n_indices_strict = net->n_indices_strict;
  out->max_clause_rank = net->max_clause_rank;
  out->has_empty_clause = net->has_empty ? 1 : 0;
  return WMC_OK;
}

namespace wmc {
const Network &network_of(const wmc_network_t *n) { return *n; }
}
