// Internal host-side structures of the WMC execution library.
// Not part of the ABI (see include/wmc.h).
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "wmc.h"

namespace wmc {

// Workspace regions start on 256-byte boundaries.
constexpr int64_t kAlign = 256;
inline int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit arena of a walk's intermediate tensors: offsets relative to
// the arena's start, each block rounded up to kAlign; released blocks merge
// with their free neighbours.
struct FirstFit {
  std::map<int64_t, int64_t> free_;  // offset -> size
  int64_t top = 0;
  int64_t alloc(int64_t bytes) {
    bytes = align_up(std::max<int64_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        int64_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        return off;
      }
    }
    // extend the top (merging a free block that ends at the top)
    if (!free_.empty()) {
      auto last = std::prev(free_.end());
      if (last->first + last->second == top) {
        int64_t off = last->first;
        free_.erase(last);
        top = off + bytes;
        return off;
      }
    }
    int64_t off = top;
    top += bytes;
    return off;
  }
  void release(int64_t off, int64_t bytes) {
    bytes = align_up(std::max<int64_t>(bytes, 1));
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Thread-local error message behind wmc_last_error().
void set_error(const char *fmt, ...);

// One clause after reduction: its distinct variables (0-based, ascending)
// and the unique falsifying assignment (bit j = falsifying value of
// vars[j]).  The clause tensor B_C of Thm 3.2 is 1 everywhere except at
// `fals`, where it is 0.
struct Clause {
  std::vector<int32_t> vars;
  uint64_t fals = 0;
  // index slicing (Alg. 3): literals on sliced variables, as bits over the
  // slice index (variable slice_vars[k] is bit k): smask = the clause's
  // sliced variables, sfals = their falsifying values.  Under the slice
  // assignment eta the clause is satisfied outright iff some sliced literal
  // is true, i.e. ((eta ^ sfals) & smask) != 0; otherwise it is the clause
  // over its remaining variables.
  uint32_t smask = 0, sfals = 0;
  // clauses over more than 62 variables (plannable only when factored):
  // the falsifying value of vars[j] is fvals[j], and `fals` is unused
  std::vector<uint8_t> fvals;
};

struct Network {
  int32_t n_vars = 0;
  int64_t n_clauses_in = 0;
  std::vector<Clause> clauses;  // tautologies dropped; empty clause kept
  std::vector<double> w_pos, w_neg;
  bool has_empty = false;
  int64_t n_indices_strict = 0;
  int64_t max_clause_rank = 0;
  std::vector<uint8_t> sliced;  // per variable: fixed by the slice (no weight leaf, in no clause)
  // clause factoring (Def. 3.4, Thm 3.3): auxiliary indices n_vars ..
  // n_vars + n_aux - 1, the OR-gate outputs of factored clauses; weight 1
  // for both values (no weight leaf)
  int32_t n_aux = 0;
  int32_t n_all() const { return n_vars + n_aux; }
};

enum LeafKind : int32_t { LEAF_CLAUSE = 0, LEAF_WEIGHT = 1, LEAF_ONE = 2, NOT_LEAF = -1 };

struct TensorInfo {
  std::vector<int32_t> labels;  // variable labels, bit j of the offset = labels[j]
  bool has_q = false;           // depends on the weights: carries the query index
  int32_t kind = NOT_LEAF;
  uint64_t fals = 0;            // LEAF_CLAUSE
  int64_t clause = -1;          // LEAF_CLAUSE: clause id
  int64_t node = -1;            // producing node (or -1 for a leaf)
  int32_t roundings = 0;        // most roundings on a path from a leaf (FP32 counts)
};

struct Node {
  int64_t a = -1, b = -1, c = -1;  // tensor ids (c = output)
  int32_t iter_rank = 0;           // |I(A) u I(B)|
  int32_t n_summed = 0;
};

struct ExecState;  // executor.cu

struct Plan {
  int32_t n_vars = 0;
  std::vector<double> w_pos, w_neg;  // default weights
  bool unit_weights = false;
  bool any_negative = false;
  std::vector<TensorInfo> tensors;   // leaves [0, n_leaves), then node outputs
  int64_t n_leaves = 0;
  std::vector<Node> nodes;           // post-order; nodes.back() is the root
  int32_t precision = WMC_SCALED_FP32;
  int32_t ordering_used = 0;
  int32_t max_rank = 0;
  int32_t max_node_rank = 0;
  std::vector<Clause> clauses;       // for leaf materialisation
  // index slicing: the sliced variables (slice bit k = slice_vars[k]); the
  // walk runs once per slice assignment and the results are summed
  std::vector<int32_t> slice_vars;
  int32_t n_aux = 0;  // auxiliary indices of factored clauses (labels n_vars ..)
  int32_t bfp_b = -1;  // block floating point: block bits b (-1: off)

  std::mutex exec_mu;
  std::map<int32_t, std::unique_ptr<ExecState>> exec;  // keyed by Q
  // one pass per node in post-order, every tensor its own offset (no chains,
  // no small-node phase): the layout other executors reuse
  std::map<int32_t, std::unique_ptr<ExecState>> exec_plain;
  // the same tree in float64 for queries whose scaled-FP32 walk may have
  // flushed (WMC_FLAG_FELL_BACK_FP64)
  std::map<int32_t, std::unique_ptr<ExecState>> exec_f64;
  // states replaced by wmc_autotune_plan (kept until the plan is destroyed:
  // a server or graph may still hold them)
  std::vector<std::unique_ptr<ExecState>> retired;
  ~Plan();
};

// Planner entry (planner.cpp).
int build_plan(const Network &net, const wmc_plan_opts &opts, Plan &plan);

// Elimination orders (planner.cpp), 0-based variable ids.
std::vector<int32_t> order_min_fill(int32_t n, const std::vector<std::vector<int32_t>> &adj);
std::vector<int32_t> order_min_degree(int32_t n, const std::vector<std::vector<int32_t>> &adj);
std::vector<int32_t> order_sweep(int32_t n, const std::vector<std::vector<int32_t>> &adj,
                                 bool descending);

// Executor (executor.cu).
int64_t plan_workspace_bytes(Plan &plan, int32_t Q, int64_t *arena_bytes);
void destroy_exec_state(ExecState *st);
// Lays out (once) and returns the execution state of batch size Q.
int exec_state(Plan &plan, int32_t Q, ExecState **out);
// Lays out the device tables and captures the walk's graph for workspace
// `ws` without running it (the first wave of that size then starts at once).
int exec_prepare(Plan &plan, ExecState *st, void *ws);
int64_t exec_ws_bytes(const ExecState *st);
// Enqueues one walk on `stream` (device pointers; weights [Q][n_vars]).
int exec_run_device(Plan &plan, ExecState *st, const double *d_w_pos, const double *d_w_neg,
                    void *ws, double *d_mant, int64_t *d_exp2, uint32_t *d_flags, void *stream);
void exec_fill_result(const ExecState *st, double mant, int64_t exp2, uint32_t flags,
                      bool unit, bool negative, wmc_result *out);
Plan &plan_of(wmc_plan_t *p);

// Host-side layout of a plan's walk at batch size Q (executor.cu): one pass
// per node in post-order, every node's output at its own offset.
struct LayoutView {
  int64_t ws_bytes = 0, off_io = 0, off_flags = 0, off_err = 0, off_exp = 0, off_max = 0,
          off_min = 0, n_slots = 0;
  int64_t arena0 = 0;  // start of the intermediates' arena (leaves and metadata below it)
  const std::vector<int64_t> *t_off = nullptr;   // byte offset of each tensor
  const std::vector<int64_t> *t_meta = nullptr;  // first metadata slot
  const std::vector<int64_t> *t_bytes = nullptr;
  const std::vector<uint8_t> *t_dbl = nullptr;   // stored as float64
};
int exec_layout(Plan &plan, int32_t Q, LayoutView *out);
// Bit maps of the generic kernel for C = A . B given full label lists.
void k1_bitmaps(const std::vector<int32_t> &LA, const std::vector<int32_t> &LB,
                const std::vector<int32_t> &LC, int32_t *rC, int32_t *k, int8_t *posA,
                int8_t *posB, int8_t *sposA, int8_t *sposB);
// Kernel launches issued by this library (accounting).
void count_launches(int64_t n);
// Test hook state: allocation failures to inject (consumed by device_alloc).
int device_alloc(void **p, size_t bytes);

}  // namespace wmc
