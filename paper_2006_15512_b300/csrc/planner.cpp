// Planning stage (Sec. 3.3): contraction tree by bucket elimination.
//
// An elimination order of the primal graph is turned into a rooted binary
// contraction tree (Def. 3.2): for each variable x in order, the live
// tensors that mention x are contracted pairwise, smallest first; an index
// is summed at the first contraction after which no other live tensor
// mentions it.  The structure-based objective of Sec. 3.3 (minimise the
// max-rank) chooses among several orders.  Each intermediate tensor's index
// order (its memory layout) is then chosen from its larger operand so that
// the streaming contraction keeps most bit positions in place.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <set>
#include <tuple>

#include "internal.h"

namespace wmc {

static std::vector<std::vector<int32_t>> primal_graph(const Network &net) {
  std::vector<std::vector<int32_t>> adj((size_t)net.n_all());
  for (const Clause &c : net.clauses)
    for (int32_t a : c.vars)
      for (int32_t b : c.vars)
        if (a != b) adj[(size_t)a].push_back(b);
  for (auto &v : adj) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  return adj;
}

// ------------------------------------------------------------ orders

namespace {
struct DynGraph {
  int32_t n;
  size_t words;
  std::vector<uint64_t> bits;                 // n x words adjacency bitsets
  std::vector<std::vector<int32_t>> nb;       // neighbour lists (live only)
  std::vector<uint8_t> dead;
  explicit DynGraph(int32_t n_, const std::vector<std::vector<int32_t>> &adj)
      : n(n_), words(((size_t)n_ + 63) / 64), bits((size_t)n_ * (((size_t)n_ + 63) / 64), 0),
        nb(adj), dead((size_t)n_, 0) {
    for (int32_t v = 0; v < n; ++v)
      for (int32_t u : nb[(size_t)v]) set(v, u);
  }
  bool has(int32_t a, int32_t b) const { return (bits[(size_t)a * words + (size_t)b / 64] >> (b % 64)) & 1; }
  void set(int32_t a, int32_t b) { bits[(size_t)a * words + (size_t)b / 64] |= 1ull << (b % 64); }
  void clr(int32_t a, int32_t b) { bits[(size_t)a * words + (size_t)b / 64] &= ~(1ull << (b % 64)); }
  int64_t fill(int32_t v) const {
    const auto &N = nb[(size_t)v];
    int64_t f = 0;
    for (size_t i = 0; i < N.size(); ++i)
      for (size_t j = i + 1; j < N.size(); ++j) f += has(N[i], N[j]) ? 0 : 1;
    return f;
  }
  // eliminate v: make its neighbourhood a clique, remove v
  void eliminate(int32_t v) {
    const std::vector<int32_t> N = nb[(size_t)v];
    for (size_t i = 0; i < N.size(); ++i)
      for (size_t j = 0; j < N.size(); ++j) {
        if (i == j) continue;
        int32_t a = N[i], b = N[j];
        if (!has(a, b)) { set(a, b); nb[(size_t)a].push_back(b); }
      }
    for (int32_t a : N) {
      clr(a, v);
      auto &L = nb[(size_t)a];
      L.erase(std::find(L.begin(), L.end(), v));
    }
    nb[(size_t)v].clear();
    dead[(size_t)v] = 1;
  }
};
}  // namespace

std::vector<int32_t> order_min_fill(int32_t n, const std::vector<std::vector<int32_t>> &adj) {
  DynGraph g(n, adj);
  std::set<std::tuple<int64_t, int64_t, int32_t>> pq;
  std::vector<std::tuple<int64_t, int64_t, int32_t>> key((size_t)n);
  for (int32_t v = 0; v < n; ++v) {
    key[(size_t)v] = {g.fill(v), (int64_t)g.nb[(size_t)v].size(), v};
    pq.insert(key[(size_t)v]);
  }
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  std::vector<int32_t> stamp((size_t)n, -1);
  for (int32_t step = 0; step < n; ++step) {
    int32_t v = std::get<2>(*pq.begin());
    pq.erase(pq.begin());
    order.push_back(v);
    std::vector<int32_t> N = g.nb[(size_t)v];
    g.eliminate(v);
    // the fill of N(v) and of their neighbours may change
    std::vector<int32_t> touch;
    for (int32_t a : N) {
      if (stamp[(size_t)a] != step) { stamp[(size_t)a] = step; touch.push_back(a); }
      for (int32_t b : g.nb[(size_t)a])
        if (stamp[(size_t)b] != step) { stamp[(size_t)b] = step; touch.push_back(b); }
    }
    for (int32_t a : touch) {
      pq.erase(key[(size_t)a]);
      key[(size_t)a] = {g.fill(a), (int64_t)g.nb[(size_t)a].size(), a};
      pq.insert(key[(size_t)a]);
    }
  }
  return order;
}

std::vector<int32_t> order_min_degree(int32_t n, const std::vector<std::vector<int32_t>> &adj) {
  DynGraph g(n, adj);
  std::set<std::pair<int64_t, int32_t>> pq;
  std::vector<int64_t> deg((size_t)n);
  for (int32_t v = 0; v < n; ++v) {
    deg[(size_t)v] = (int64_t)g.nb[(size_t)v].size();
    pq.insert({deg[(size_t)v], v});
  }
  std::vector<int32_t> order;
  for (int32_t step = 0; step < n; ++step) {
    int32_t v = pq.begin()->second;
    pq.erase(pq.begin());
    order.push_back(v);
    std::vector<int32_t> N = g.nb[(size_t)v];
    g.eliminate(v);
    for (int32_t a : N) {
      pq.erase({deg[(size_t)a], a});
      deg[(size_t)a] = (int64_t)g.nb[(size_t)a].size();
      pq.insert({deg[(size_t)a], a});
    }
  }
  return order;
}

static std::vector<int32_t> bfs_dist(const std::vector<std::vector<int32_t>> &adj,
                                     const std::vector<int32_t> &src) {
  std::vector<int32_t> d(adj.size(), -1);
  std::deque<int32_t> q;
  for (int32_t s : src) { d[(size_t)s] = 0; q.push_back(s); }
  while (!q.empty()) {
    int32_t u = q.front(); q.pop_front();
    for (int32_t w : adj[(size_t)u])
      if (d[(size_t)w] < 0) { d[(size_t)w] = d[(size_t)u] + 1; q.push_back(w); }
  }
  return d;
}

// Level sweep: inside each connected component, find a far vertex u by
// repeated BFS, take the set S of vertices farthest from u, and order the
// component by the BFS level from the whole set S (a layered sweep that
// follows the long axis of grid-like graphs), ties by id.
std::vector<int32_t> order_sweep(int32_t n, const std::vector<std::vector<int32_t>> &adj,
                                 bool descending) {
  std::vector<int32_t> comp((size_t)n, -1);
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  for (int32_t s0 = 0; s0 < n; ++s0) {
    if (comp[(size_t)s0] >= 0) continue;
    std::vector<int32_t> d0 = bfs_dist(adj, {s0});
    std::vector<int32_t> members;
    for (int32_t v = 0; v < n; ++v)
      if (d0[(size_t)v] >= 0) { comp[(size_t)v] = s0; members.push_back(v); }
    int32_t u = s0;
    for (int it = 0; it < 4; ++it) {
      std::vector<int32_t> d = bfs_dist(adj, {u});
      int32_t best = u;
      for (int32_t v : members)
        if (d[(size_t)v] > d[(size_t)best]) best = v;
      if (best == u) break;
      u = best;
    }
    std::vector<int32_t> du = bfs_dist(adj, {u});
    int32_t mx = 0;
    for (int32_t v : members) mx = std::max(mx, du[(size_t)v]);
    std::vector<int32_t> far;
    for (int32_t v : members)
      if (du[(size_t)v] == mx) far.push_back(v);
    std::vector<int32_t> dl = bfs_dist(adj, far);
    std::sort(members.begin(), members.end(), [&](int32_t a, int32_t b) {
      int32_t la = dl[(size_t)a], lb = dl[(size_t)b];
      if (la != lb) return descending ? la > lb : la < lb;
      return a < b;
    });
    order.insert(order.end(), members.begin(), members.end());
  }
  return order;
}

// ------------------------------------------------------------ tree build

namespace {
struct Candidate {
  std::vector<TensorInfo> tensors;
  std::vector<Node> nodes;
  int32_t max_rank = 0, max_node_rank = 0;
  double cost = 0;
  int32_t ordering = 0;
};

std::vector<int32_t> union_sorted(const std::vector<int32_t> &a, const std::vector<int32_t> &b) {
  std::vector<int32_t> u;
  std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(u));
  return u;
}

// Builds the tree on sorted label sets (layouts are assigned later).
bool build_tree(const Network &net, const std::vector<int32_t> &order, int32_t rank_cap,
                Candidate &out) {
  std::vector<TensorInfo> &T = out.tensors;
  T.clear();
  out.nodes.clear();
  for (size_t c = 0; c < net.clauses.size(); ++c) {
    TensorInfo t;
    t.labels = net.clauses[c].vars;
    t.kind = LEAF_CLAUSE;
    t.fals = net.clauses[c].fals;
    t.clause = (int64_t)c;
    // under index slicing a clause with a sliced literal depends on the
    // slice assignment: it carries the lanes, so that slices can run along
    // them as queries do
    t.has_q = net.clauses[c].smask != 0;
    T.push_back(t);
  }
  for (int32_t x = 0; x < net.n_vars; ++x) {
    if (!net.sliced.empty() && net.sliced[(size_t)x]) continue;  // a factor of the slice, not a leaf
    TensorInfo t;
    t.labels = {x};
    t.kind = LEAF_WEIGHT;
    t.has_q = true;
    T.push_back(t);
  }
  if (T.empty()) {  // no variables and no clauses: W = 1
    TensorInfo t; t.kind = LEAF_ONE; T.push_back(t);
  }
  int32_t max_rank = 0;
  for (auto &t : T) max_rank = std::max(max_rank, (int32_t)t.labels.size());
  const size_t n_leaves = T.size();
  std::vector<int32_t> cnt((size_t)net.n_all(), 0);         // live tensors per var
  std::vector<std::vector<int64_t>> holders((size_t)net.n_all());
  std::vector<uint8_t> live(n_leaves, 1);
  for (size_t i = 0; i < n_leaves; ++i)
    for (int32_t v : T[i].labels) { cnt[(size_t)v]++; holders[(size_t)v].push_back((int64_t)i); }
  int32_t max_node_rank = 0;
  double cost = 0;

  auto contract = [&](int64_t a, int64_t b) -> int64_t {
    TensorInfo c;
    std::vector<int32_t> u = union_sorted(T[(size_t)a].labels, T[(size_t)b].labels);
    int32_t summed = 0;
    for (int32_t v : u) {
      bool ina = std::binary_search(T[(size_t)a].labels.begin(), T[(size_t)a].labels.end(), v);
      bool inb = std::binary_search(T[(size_t)b].labels.begin(), T[(size_t)b].labels.end(), v);
      cnt[(size_t)v] -= (int32_t)ina + (int32_t)inb;
      if (cnt[(size_t)v] == 0) { ++summed; continue; }
      c.labels.push_back(v);
    }
    int64_t id = (int64_t)T.size();
    for (int32_t v : c.labels) { cnt[(size_t)v]++; holders[(size_t)v].push_back(id); }
    c.has_q = T[(size_t)a].has_q || T[(size_t)b].has_q;
    c.node = (int64_t)out.nodes.size();
    Node nd;
    nd.a = a; nd.b = b; nd.c = id;
    nd.iter_rank = (int32_t)u.size();
    nd.n_summed = summed;
    max_node_rank = std::max(max_node_rank, nd.iter_rank);
    max_rank = std::max(max_rank, (int32_t)c.labels.size());
    cost += std::ldexp(1.0, (int)T[(size_t)a].labels.size()) + std::ldexp(1.0, (int)T[(size_t)b].labels.size()) +
            std::ldexp(1.0, (int)c.labels.size()) + std::ldexp(1.0, nd.iter_rank);
    out.nodes.push_back(nd);
    T.push_back(std::move(c));
    live.push_back(1);
    live[(size_t)a] = live[(size_t)b] = 0;
    return id;
  };
  auto by_size = [&](int64_t x, int64_t y) {
    size_t rx = T[(size_t)x].labels.size(), ry = T[(size_t)y].labels.size();
    if (rx != ry) return rx < ry;
    return x < y;
  };

  for (int32_t x : order) {
    std::vector<int64_t> bucket;
    for (int64_t id : holders[(size_t)x])
      if (live[(size_t)id]) bucket.push_back(id);
    holders[(size_t)x].clear();
    while (bucket.size() > 1) {
      std::sort(bucket.begin(), bucket.end(), by_size);
      int64_t a = bucket[0], b = bucket[1];
      size_t ur = union_sorted(T[(size_t)a].labels, T[(size_t)b].labels).size();
      if ((int32_t)ur > rank_cap + 2) return false;
      int64_t c = contract(a, b);
      bucket.erase(bucket.begin(), bucket.begin() + 2);
      if (std::binary_search(T[(size_t)c].labels.begin(), T[(size_t)c].labels.end(), x))
        bucket.push_back(c);
      if (max_rank > rank_cap) return false;
    }
    for (int64_t id : bucket) holders[(size_t)x].push_back(id);
  }
  // remaining live tensors (scalars and tensors with dangling indices)
  std::vector<int64_t> rest;
  for (size_t i = 0; i < T.size(); ++i)
    if (live[i]) rest.push_back((int64_t)i);
  if (rest.size() == 1 && (!T[(size_t)rest[0]].labels.empty() || out.nodes.empty())) {
    TensorInfo one; one.kind = LEAF_ONE;
    // leaves must precede node outputs: a late leaf is inserted by id remap
    T.push_back(one);
    live.push_back(1);
    rest.push_back((int64_t)T.size() - 1);
  }
  while (rest.size() > 1) {
    std::sort(rest.begin(), rest.end(), by_size);
    int64_t c = contract(rest[0], rest[1]);
    rest.erase(rest.begin(), rest.begin() + 2);
    rest.push_back(c);
    if (max_rank > rank_cap) return false;
  }
  out.max_rank = max_rank;
  out.max_node_rank = max_node_rank;
  out.cost = cost;
  return true;
}

// Leaves first: move any LEAF_ONE added after node outputs to the leaf block.
void normalise_ids(Candidate &c) {
  std::vector<int64_t> leaves, others;
  for (size_t i = 0; i < c.tensors.size(); ++i)
    (c.tensors[i].kind != NOT_LEAF ? leaves : others).push_back((int64_t)i);
  std::vector<int64_t> remap(c.tensors.size());
  std::vector<TensorInfo> T;
  for (int64_t i : leaves) { remap[(size_t)i] = (int64_t)T.size(); T.push_back(c.tensors[(size_t)i]); }
  for (int64_t i : others) { remap[(size_t)i] = (int64_t)T.size(); T.push_back(c.tensors[(size_t)i]); }
  for (Node &nd : c.nodes) { nd.a = remap[(size_t)nd.a]; nd.b = remap[(size_t)nd.b]; nd.c = remap[(size_t)nd.c]; }
  c.tensors.swap(T);
}

// Index order of each intermediate: start from the larger operand P's
// order; the indices of the other operand that survive take the places of
// P's summed indices (in order), extra ones go on top, and unused summed
// places are closed up.  Bit positions of P's kept indices therefore stay
// monotone, and mostly unchanged.
void assign_layouts(Candidate &c) {
  for (Node &nd : c.nodes) {
    const TensorInfo &A = c.tensors[(size_t)nd.a];
    const TensorInfo &B = c.tensors[(size_t)nd.b];
    TensorInfo &C = c.tensors[(size_t)nd.c];
    bool a_primary = A.labels.size() >= B.labels.size();
    const TensorInfo &P = a_primary ? A : B;
    const TensorInfo &S = a_primary ? B : A;
    std::vector<int32_t> keep = C.labels;  // sorted set of C's labels
    auto inC = [&](int32_t v) { return std::binary_search(keep.begin(), keep.end(), v); };
    auto inP = [&](int32_t v) { return std::find(P.labels.begin(), P.labels.end(), v) != P.labels.end(); };
    std::vector<int32_t> extra;  // S-only survivors in S's order
    for (int32_t v : S.labels)
      if (inC(v) && !inP(v)) extra.push_back(v);
    std::vector<int32_t> out;
    size_t ei = 0;
    for (int32_t v : P.labels) {
      if (inC(v)) out.push_back(v);
      else if (ei < extra.size()) out.push_back(extra[ei++]);
    }
    while (ei < extra.size()) out.push_back(extra[ei++]);
    C.labels = out;
  }
}

void assign_roundings(Candidate &c, int32_t precision) {
  for (size_t i = 0; i < c.tensors.size(); ++i) {
    TensorInfo &t = c.tensors[i];
    if (t.kind == LEAF_WEIGHT) t.roundings = precision == WMC_SCALED_FP32 ? 1 : 0;
    else if (t.kind != NOT_LEAF) t.roundings = 0;
  }
  for (Node &nd : c.nodes) {
    // a serial fused multiply-add chain over 2^k terms rounds the first
    // term 2^k times
    int32_t r = std::max(c.tensors[(size_t)nd.a].roundings, c.tensors[(size_t)nd.b].roundings);
    c.tensors[(size_t)nd.c].roundings = r + (1 << std::min(nd.n_summed, 24));
  }
}
}  // namespace

// Index slicing (Alg. 3): fixes variables one at a time until the best
// plan's largest tensor has at most `target` indices.  Each round picks the
// variable whose tensors in the current best tree weigh most (the sum of
// 2^rank over the tensors holding it: what fixing it halves), removes it
// from every clause (recording the literal in the clause's slice bits) and
// plans again.  At most kMaxSliceVars variables.
static constexpr int kMaxSliceVars = 24;

static int best_candidate(const Network &net, const wmc_plan_opts &opts, int32_t cap, Candidate &best);
static int plan_unsliced(const Network &net, const wmc_plan_opts &opts, int32_t cap, Plan &plan);

static int choose_slices(const Network &net, const wmc_plan_opts &opts, int32_t target, Network &work,
                         std::vector<int32_t> &slice_vars) {
  work = net;
  work.sliced.assign((size_t)net.n_vars, 0);
  slice_vars.clear();
  for (;;) {
    Candidate probe;
    int rc = best_candidate(work, opts, 62, probe);
    if (rc) return rc;
    if (probe.max_rank <= target) return WMC_OK;
    if ((int)slice_vars.size() >= kMaxSliceVars) {
      set_error("slicing %d variables leaves a tensor of rank %d (target %d)", kMaxSliceVars, probe.max_rank, target);
      return WMC_EPLAN_TOO_BIG;
    }
    std::vector<double> score((size_t)net.n_all(), 0.0);
    for (const TensorInfo &t : probe.tensors)
      for (int32_t v : t.labels) score[(size_t)v] += std::ldexp(1.0, (int)t.labels.size());
    int32_t best = -1;
    for (int32_t v = 0; v < net.n_vars; ++v)
      if (!work.sliced[(size_t)v] && score[(size_t)v] > 0 && (best < 0 || score[(size_t)v] > score[(size_t)best]))
        best = v;
    if (best < 0) {
      set_error("no variable left to slice (largest tensor rank %d, target %d)", probe.max_rank, target);
      return WMC_EPLAN_TOO_BIG;
    }
    const uint32_t kbit = 1u << slice_vars.size();
    for (Clause &c : work.clauses) {
      auto it = std::find(c.vars.begin(), c.vars.end(), best);
      if (it == c.vars.end()) continue;
      const size_t j = (size_t)(it - c.vars.begin());
      const uint64_t fv = (c.fals >> j) & 1ull;
      const uint64_t low = c.fals & ((1ull << j) - 1ull);
      c.fals = low | ((c.fals >> (j + 1)) << j);
      c.vars.erase(it);
      c.smask |= kbit;
      if (fv) c.sfals |= kbit;
    }
    work.sliced[(size_t)best] = 1;
    slice_vars.push_back(best);
  }
}

// Clause factoring (FactorTree of Sec. 3.3 for clause tensors: Def. 3.4,
// Thm 3.3).  A clause tensor is tree-factorable: a clause with r > `above`
// literals l_1 .. l_r (ascending variable order) becomes a chain of OR
// gates over new indices y_1 .. y_{r-2}, y_1 = l_1 | l_2 and
// y_k = y_{k-1} | l_{k+1}, closed by the clause (y_{r-2} | l_r).  A gate
// y = a | b is the product of the clause tensors (~a | y), (~b | y) and
// (a | b | ~y), so every tensor has rank <= 3.  For each assignment of the
// formula's variables exactly one assignment of the y's satisfies every
// gate, so with weight 1 for both values of each y the count is unchanged.
namespace {
struct Lit {
  int32_t v;
  uint32_t f;  // the value of v that falsifies the literal
};
Clause clause_of(std::vector<Lit> lits) {
  std::sort(lits.begin(), lits.end(), [](const Lit &a, const Lit &b) { return a.v < b.v; });
  Clause c;
  for (size_t j = 0; j < lits.size(); ++j) {
    c.vars.push_back(lits[j].v);
    if (lits[j].f) c.fals |= 1ull << j;
  }
  return c;
}
void factor_clauses(const Network &net, int32_t above, Network &out) {
  out = net;
  out.clauses.clear();
  out.n_aux = 0;
  out.n_indices_strict = 0;
  out.max_clause_rank = 0;
  auto push = [&](Clause c) {
    out.n_indices_strict += (int64_t)c.vars.size();
    out.max_clause_rank = std::max(out.max_clause_rank, (int64_t)c.vars.size());
    out.clauses.push_back(std::move(c));
  };
  for (const Clause &c : net.clauses) {
    const size_t r = c.vars.size();
    if ((int32_t)r <= above) { push(c); continue; }
    std::vector<Lit> l(r);
    for (size_t j = 0; j < r; ++j)
      l[j] = {c.vars[j], c.fvals.empty() ? (uint32_t)((c.fals >> j) & 1ull) : (uint32_t)c.fvals[j]};
    Lit prev = l[0];
    for (size_t k = 1; k + 1 < r; ++k) {
      const Lit y{net.n_vars + out.n_aux++, 0u};  // y = prev | l[k]
      const Lit a = prev, b = l[k];
      push(clause_of({{a.v, 1u - a.f}, y}));
      push(clause_of({{b.v, 1u - b.f}, y}));
      push(clause_of({a, b, {y.v, 1u}}));
      prev = y;
    }
    push(clause_of({prev, l[r - 1]}));
  }
}
}  // namespace

static int build_plan_on(const Network &net, const wmc_plan_opts &opts, Plan &plan);

int build_plan(const Network &net, const wmc_plan_opts &opts, Plan &plan) {
  if (opts.factor_clauses_above == 0) return build_plan_on(net, opts, plan);
  if (opts.factor_clauses_above < 3) {
    set_error("factor_clauses_above must be 0 (off) or at least 3 (got %d)", opts.factor_clauses_above);
    return WMC_EINVAL;
  }
  Network factored;
  try {
    factor_clauses(net, opts.factor_clauses_above, factored);
  } catch (const std::bad_alloc &) {
    set_error("out of host memory while factoring clauses");
    return WMC_ENOMEM;
  }
  if ((int64_t)net.n_vars + factored.n_aux > INT32_MAX / 2) { set_error("too many auxiliary indices"); return WMC_EINVAL; }
  const int rc = build_plan_on(factored, opts, plan);
  if (rc == WMC_OK) plan.n_aux = factored.n_aux;
  return rc;
}

static int build_plan_on(const Network &net, const wmc_plan_opts &opts, Plan &plan) {
  const int32_t cap = opts.max_rank_cap > 0 ? opts.max_rank_cap : 30;
  for (size_t c = 0; c < net.clauses.size(); ++c)
    if (!net.clauses[c].fvals.empty()) {
      set_error("clause %zu has %zu literals (a rank-%zu tensor): plan with factor_clauses_above", c,
                net.clauses[c].vars.size(), net.clauses[c].vars.size());
      return WMC_EPLAN_TOO_BIG;
    }
  if (opts.slice_to_rank > 0) {
    Network work;
    std::vector<int32_t> slice_vars;
    int rc;
    try {
      rc = choose_slices(net, opts, std::min(opts.slice_to_rank, cap), work, slice_vars);
    } catch (const std::bad_alloc &) {
      set_error("out of host memory while slicing");
      return WMC_ENOMEM;
    }
    if (rc) return rc;
    rc = plan_unsliced(work, opts, cap, plan);
    if (rc) return rc;
    plan.slice_vars = slice_vars;
    plan.w_pos = net.w_pos;  // the sliced variables' weights enter as factors
    plan.w_neg = net.w_neg;
    return WMC_OK;
  }
  return plan_unsliced(net, opts, cap, plan);
}

// The best tree over the portfolio of elimination orders (lowest max rank,
// then lowest cost) whose tensors stay within `cap` indices.
static int best_candidate(const Network &net, const wmc_plan_opts &opts, int32_t cap, Candidate &best) {
  std::vector<std::pair<int32_t, std::vector<int32_t>>> orders;
  try {
    if (opts.ordering == WMC_ORDER_GIVEN) {
      if (!opts.order) { set_error("WMC_ORDER_GIVEN without an order"); return WMC_EINVAL; }
      if (net.n_aux) { set_error("a given order cannot be combined with clause factoring"); return WMC_EINVAL; }
      std::vector<int32_t> o((size_t)net.n_vars);
      std::vector<uint8_t> seen((size_t)net.n_vars, 0);
      for (int32_t i = 0; i < net.n_vars; ++i) {
        int32_t v = opts.order[i] - 1;
        if (v < 0 || v >= net.n_vars || seen[(size_t)v]) { set_error("order is not a permutation of 1..n"); return WMC_EINVAL; }
        seen[(size_t)v] = 1;
        o[(size_t)i] = v;
      }
      orders.push_back({WMC_ORDER_GIVEN, o});
    } else {
      auto adj = primal_graph(net);
      const int32_t n = net.n_all();
      bool all = opts.ordering == WMC_ORDER_BEST;
      if (all || opts.ordering == WMC_ORDER_SWEEP) {
        orders.push_back({WMC_ORDER_SWEEP, order_sweep(n, adj, false)});
        if (all) orders.push_back({WMC_ORDER_SWEEP, order_sweep(n, adj, true)});
      }
      if ((all && n <= 8192) || opts.ordering == WMC_ORDER_MINFILL)
        orders.push_back({WMC_ORDER_MINFILL, order_min_fill(n, adj)});
      if (all || opts.ordering == WMC_ORDER_MINDEGREE)
        orders.push_back({WMC_ORDER_MINDEGREE, order_min_degree(n, adj)});
      if (orders.empty()) { set_error("unknown ordering %d", opts.ordering); return WMC_EINVAL; }
    }
    bool have = false;
    for (auto &o : orders) {
      Candidate c;
      if (!build_tree(net, o.second, cap, c)) continue;
      c.ordering = o.first;
      if (!have || std::make_pair(c.max_rank, c.cost) < std::make_pair(best.max_rank, best.cost)) {
        best = std::move(c);
        have = true;
      }
    }
    if (!have) {
      set_error("no elimination order keeps every tensor within rank %d", cap);
      return WMC_EPLAN_TOO_BIG;
    }
  } catch (const std::bad_alloc &) {
    set_error("out of host memory while planning");
    return WMC_ENOMEM;
  }
  return WMC_OK;
}

static int plan_unsliced(const Network &net, const wmc_plan_opts &opts, int32_t cap, Plan &plan) {
  try {
    Candidate best;
    int rc = best_candidate(net, opts, cap, best);
    if (rc) return rc;
    normalise_ids(best);
    assign_layouts(best);
    assign_roundings(best, opts.precision);
    plan.n_vars = net.n_vars;
    plan.w_pos = net.w_pos;
    plan.w_neg = net.w_neg;
    plan.unit_weights = true;
    plan.any_negative = false;
    for (int32_t v = 0; v < net.n_vars; ++v) {
      if (net.w_pos[(size_t)v] != 1.0 || net.w_neg[(size_t)v] != 1.0) plan.unit_weights = false;
      if (net.w_pos[(size_t)v] < 0 || net.w_neg[(size_t)v] < 0) plan.any_negative = true;
    }
    plan.tensors = std::move(best.tensors);
    plan.nodes = std::move(best.nodes);
    plan.n_leaves = 0;
    for (auto &t : plan.tensors) plan.n_leaves += (t.kind != NOT_LEAF);
    plan.precision = opts.precision;
    plan.ordering_used = best.ordering;
    plan.max_rank = best.max_rank;
    plan.max_node_rank = best.max_node_rank;
    plan.clauses = net.clauses;
  } catch (const std::bad_alloc &) {
    set_error("out of host memory while planning");
    return WMC_ENOMEM;
  }
  return WMC_OK;
}

}  // namespace wmc
