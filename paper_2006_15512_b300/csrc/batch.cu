// Uneven batches: many formulas, one persistent launch.
//
// Every admitted formula keeps its own single-query walk layout (its plan at
// Q = 1: leaves, metadata, first-fit arena), placed side by side in one
// batch workspace.  The contractions of all formulas become one task list:
// a task is a chunk of one node's outputs.  A persistent kernel pulls tasks
// from an atomic counter; within a formula, nodes run in post-order (a
// node's tasks wait until the previous node of the same formula has
// completed, which also keeps the arena's first-fit reuse safe), while the
// tasks of one node and the nodes of different formulas run concurrently.
// Tasks are listed round-robin across formulas in post-order, so a task's
// dependency was always handed out earlier; only running blocks take tasks,
// so every wait ends.  Each wait is also bounded by %globaltimer (one
// second); on timeout the block records an error word and stops.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"

using namespace wmc;

namespace wmc {
namespace bdev {

using dev::kThreads;
using dev::kNoMin;

struct BNode {
  int64_t a, b, c;          // byte offsets of the operands and the output
  int64_t ea, eb, ec;       // byte offsets of the exponent slots (int64)
  int64_t xa, xb, xc;       // ... max bit patterns (uint64)
  int64_t na, nb, nc;       // ... min-nonzero bit patterns (uint64)
  int64_t flags;            // byte offset of the formula's flag word
  int32_t prev;             // node that must complete first (-1: none)
  int32_t n_tasks;
  int32_t chunk_log2;       // outputs per task = 2^chunk_log2
  int32_t rC, k;
  int8_t ti, ta, to;        // element types: 0 float, 1 double
  int8_t vec4;              // float32, C's two lowest bits are A's, B has neither: 4 outputs per thread
  int8_t posA[32], posB[32], sposA[24], sposB[24];
};

struct BTask {
  int32_t node;
  int32_t chunk;
};

struct BLeaf {
  int64_t data, e, x, n;    // byte offsets: data, exponent, max, min slots
  uint64_t fals;
  double w0, w1;
  int32_t kind, rank;
  int8_t dbl, pad[7];
};

struct BRoot {
  int64_t data, e, flags;
};

struct BatchArgs {
  char *ws;
  const BNode *nodes;
  const BTask *tasks;
  int32_t n_tasks;
  uint32_t *next;           // task counter
  uint32_t *done;           // completed tasks per node
  uint32_t *err;
};

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ bool wait_count(const uint32_t *ctr, uint32_t target) {
  if (*(volatile const uint32_t *)ctr >= target) return true;
  const unsigned long long t0 = dev::globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i) {
      __nanosleep(64);
      if (*(volatile const uint32_t *)ctr >= target) return true;
    }
    if (dev::globaltimer_ns() - t0 > 1000000000ull) return false;
  }
}

// The node's per-byte lookup tables (they depend on the node alone, so they
// are built before the previous node is waited for).
__device__ __forceinline__ void batch_lut(const BNode &nd, uint32_t (*lut)[256]) {
  // per-byte offset tables: rows 0-3 A, 4-7 B (output bits); 8-10 A, 11-13 B (summed bits).
  // Entry v of a row is the OR over v's set bits of that bit's offset: the
  // single-bit offsets first, then entries [2^b, 2^(b+1)) = entries [0, 2^b)
  // OR bit b's offset, for b = 0..7
  if (threadIdx.x < 14 * 8) {
    const int row = threadIdx.x >> 3, bit = threadIdx.x & 7;
    uint32_t o = 0;
    if (row < 8) {
      const int j = (row & 3) * 8 + bit;
      const int8_t pos = row < 4 ? nd.posA[j] : nd.posB[j];
      if (j < nd.rC && pos >= 0) o = 1u << pos;
    } else {
      const int j = ((row - 8) % 3) * 8 + bit;
      const int8_t pos = row < 11 ? nd.sposA[j] : nd.sposB[j];
      if (j < nd.k && pos >= 0) o = 1u << pos;
    }
    lut[row][1 << bit] = o;  // the single-bit entries
    if (bit == 0) lut[row][0] = 0u;
  }
  __syncthreads();
  for (int b = 1; b < 8; ++b) {
    const int half = 1 << b;  // entries [half + 1, 2 half) from [1, half)
    for (int i = threadIdx.x; i < 14 * (half - 1); i += blockDim.x) {
      const int row = i / (half - 1), v = 1 + i % (half - 1);
      lut[row][half + v] = lut[row][half] | lut[row][v];
    }
    __syncthreads();
  }
}

template <typename TI, typename TA, typename TO>
__device__ void run_task(const BatchArgs &ba, const BNode &nd, int chunk, uint32_t (*lut)[256],
                         unsigned long long *red) {
  char *ws = ba.ws;
  const TI *A = (const TI *)(ws + nd.a);
  const TI *B = (const TI *)(ws + nd.b);
  TO *C = (TO *)(ws + nd.c);
  const unsigned long long ma = ldcg((const unsigned long long *)(ws + nd.xa));
  const unsigned long long mb = ldcg((const unsigned long long *)(ws + nd.xb));
  const TA sa = (TA)dev::pow2_scale(dev::pow2_exp_of(ma, TI()), TI());
  const TA sb = (TA)dev::pow2_scale(dev::pow2_exp_of(mb, TI()), TI());
  if (chunk == 0 && threadIdx.x == 32) {
    // C's exponent and the float32 flush test (as in the single-plan
    // kernels), from the operands' metadata alone, beside the outputs
    *(int64_t *)(ws + nd.ec) = ldcg((const int64_t *)(ws + nd.ea)) + dev::pow2_exp_of(ma, TI()) +
                               ldcg((const int64_t *)(ws + nd.eb)) + dev::pow2_exp_of(mb, TI());
    const unsigned long long na = ldcg((const unsigned long long *)(ws + nd.na));
    const unsigned long long nb = ldcg((const unsigned long long *)(ws + nd.nb));
    if (na != kNoMin && nb != kNoMin) {
      const TI lo = (dev::from_bits<TI>(na) * dev::pow2_scale(dev::pow2_exp_of(ma, TI()), TI())) *
                    (dev::from_bits<TI>(nb) * dev::pow2_scale(dev::pow2_exp_of(mb, TI()), TI()));
      if (dev::below_normal(lo)) atomicOr((uint32_t *)(ws + nd.flags), 2u);
    }
  }
  const uint64_t o0 = (uint64_t)chunk << nd.chunk_log2;
  const uint64_t o1 = o0 + (1ull << nd.chunk_log2);
  const uint32_t ns = 1u << nd.k;
  TO tmax = (TO)0;
  unsigned long long tmin = kNoMin;
  if constexpr (sizeof(TI) == 4 && sizeof(TA) == 4 && sizeof(TO) == 4) {
    if (nd.vec4 && nd.k <= 8) {
      // four consecutive outputs per thread: A's four values per summed
      // term in one 16-byte load, one B value, the same sums in the same
      // order as below
      for (uint64_t o = o0 + 4 * threadIdx.x; o < o1; o += 4 * blockDim.x) {
        const uint32_t oo = (uint32_t)o;
        const uint32_t bA = lut[0][oo & 255] | lut[1][(oo >> 8) & 255] | lut[2][(oo >> 16) & 255] | lut[3][oo >> 24];
        const uint32_t bB = lut[4][oo & 255] | lut[5][(oo >> 8) & 255] | lut[6][(oo >> 16) & 255] | lut[7][oo >> 24];
        TA acc[4] = {(TA)0, (TA)0, (TA)0, (TA)0};
        for (uint32_t s = 0; s < ns; ++s) {
          const float4 a4 = __ldcg(reinterpret_cast<const float4 *>(A + (bA | lut[8][s])));
          const TA b = (TA)ldcg(B + (bB | lut[11][s])) * sb;
          acc[0] = dev::fma_t((TA)a4.x * sa, b, acc[0]);
          acc[1] = dev::fma_t((TA)a4.y * sa, b, acc[1]);
          acc[2] = dev::fma_t((TA)a4.z * sa, b, acc[2]);
          acc[3] = dev::fma_t((TA)a4.w * sa, b, acc[3]);
        }
        *reinterpret_cast<float4 *>(C + o) = make_float4(acc[0], acc[1], acc[2], acc[3]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const TO m = acc[e] < (TO)0 ? -acc[e] : acc[e];
          tmax = m > tmax ? m : tmax;
          if (m != (TO)0) {
            const unsigned long long bits = dev::abs_bits(m);
            tmin = bits < tmin ? bits : tmin;
          }
        }
      }
      goto reduce;
    }
  }
  for (uint64_t o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const uint32_t oo = (uint32_t)o;
    const uint32_t bA = lut[0][oo & 255] | lut[1][(oo >> 8) & 255] | lut[2][(oo >> 16) & 255] | lut[3][oo >> 24];
    const uint32_t bB = lut[4][oo & 255] | lut[5][(oo >> 8) & 255] | lut[6][(oo >> 16) & 255] | lut[7][oo >> 24];
    TA acc = (TA)0;
    if (nd.k <= 8) {
      for (uint32_t s = 0; s < ns; ++s) {
        const TA a = (TA)ldcg(A + (bA | lut[8][s])) * sa;
        const TA b = (TA)ldcg(B + (bB | lut[11][s])) * sb;
        acc = dev::fma_t(a, b, acc);
      }
    } else {
      for (uint32_t hi = 0; hi < (ns >> 8); ++hi) {
        const uint32_t hA = bA | lut[9][hi & 255] | lut[10][hi >> 8];
        const uint32_t hB = bB | lut[12][hi & 255] | lut[13][hi >> 8];
        TA part = (TA)0;
        for (uint32_t lo = 0; lo < 256; ++lo) {
          const TA a = (TA)ldcg(A + (hA | lut[8][lo])) * sa;
          const TA b = (TA)ldcg(B + (hB | lut[11][lo])) * sb;
          part = dev::fma_t(a, b, part);
        }
        acc += part;
      }
    }
    const TO c = (TO)acc;
    C[o] = c;
    const TO m = c < (TO)0 ? -c : c;
    tmax = m > tmax ? m : tmax;
    if (m != (TO)0) {
      const unsigned long long bits = dev::abs_bits(m);
      tmin = bits < tmin ? bits : tmin;
    }
  }
reduce:
  // block reduction into red[0] (max) and red[1] (min): folded across each
  // warp first (max and min are exact), one shared atomic per warp, then
  // one global atomic each
  if (threadIdx.x == 0) { red[0] = 0; red[1] = kNoMin; }
  __syncthreads();
  unsigned long long bmax = tmax != (TO)0 ? dev::abs_bits(tmax) : 0ull, bmin = tmin;
  for (int o = 16; o; o >>= 1) {
    const unsigned long long xm = __shfl_xor_sync(0xffffffffu, bmax, o);
    const unsigned long long xn = __shfl_xor_sync(0xffffffffu, bmin, o);
    bmax = xm > bmax ? xm : bmax;
    bmin = xn < bmin ? xn : bmin;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bmax) atomicMax(&red[0], bmax);
    if (bmin != kNoMin) atomicMin(&red[1], bmin);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (red[0]) atomicMax((unsigned long long *)(ws + nd.xc), red[0]);
    if (red[1] != kNoMin) atomicMin((unsigned long long *)(ws + nd.nc), red[1]);
  }
}

__global__ void __launch_bounds__(kThreads) k6_persistent(BatchArgs ba) {
  __shared__ uint32_t lut[14][256];
  __shared__ unsigned long long red[2];
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_task = (int)atomicAdd(ba.next, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= ba.n_tasks) break;
    const BTask task = ba.tasks[t];
    const BNode &nd = ba.nodes[task.node];
    batch_lut(nd, lut);  // overlaps the wait for the previous node
    if (threadIdx.x == 0) {
      bool ok = *(volatile uint32_t *)ba.err == 0;
      if (ok && nd.prev >= 0) ok = wait_count(ba.done + nd.prev, (uint32_t)ba.nodes[nd.prev].n_tasks);
      if (!ok) atomicOr(ba.err, 1u);
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (nd.ti == 1) run_task<double, double, double>(ba, nd, task.chunk, lut, red);
    else if (nd.to == 1) run_task<float, double, double>(ba, nd, task.chunk, lut, red);
    else if (nd.ta == 1) run_task<float, double, float>(ba, nd, task.chunk, lut, red);
    else run_task<float, float, float>(ba, nd, task.chunk, lut, red);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this task's outputs and metadata before its completion count
      atomicAdd(ba.done + task.node, 1u);
    }
  }
}

// Leaves of every formula: clause tensors, weight vectors, the scalar 1.
__global__ void k6_leaves(char *ws, const BLeaf *leaves, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const BLeaf L = leaves[i];
    int64_t e = 0;
    unsigned long long mx = 0, mn = kNoMin;
    if (L.kind == LEAF_CLAUSE) {
      for (uint64_t a = 0; a < (1ull << L.rank); ++a) {
        const double v = (a == L.fals) ? 0.0 : 1.0;
        if (L.dbl) ((double *)(ws + L.data))[a] = v;
        else ((float *)(ws + L.data))[a] = (float)v;
      }
      if (L.rank > 0) { mx = L.dbl ? dev::abs_bits(1.0) : dev::abs_bits(1.0f); mn = mx; }
    } else if (L.kind == LEAF_WEIGHT) {
      const double m = fmax(fabs(L.w0), fabs(L.w1));
      int ex = 0;
      if (m > 0) {
        ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023;
        ex = ex < -1022 ? -1022 : (ex > 1022 ? 1022 : ex);
      }
      const double s = __longlong_as_double((long long)(1023 - ex) << 52);
      unsigned long long b0, b1;
      if (L.dbl) {
        ((double *)(ws + L.data))[0] = L.w0 * s;
        ((double *)(ws + L.data))[1] = L.w1 * s;
        b0 = dev::abs_bits(L.w0 * s); b1 = dev::abs_bits(L.w1 * s);
      } else {
        const float v0 = (float)(L.w0 * s), v1 = (float)(L.w1 * s);
        ((float *)(ws + L.data))[0] = v0;
        ((float *)(ws + L.data))[1] = v1;
        b0 = dev::abs_bits(v0); b1 = dev::abs_bits(v1);
      }
      e = ex;
      mx = b0 > b1 ? b0 : b1;
      const unsigned long long n0 = b0 ? b0 : kNoMin, n1 = b1 ? b1 : kNoMin;
      mn = n0 < n1 ? n0 : n1;
    } else {
      if (L.dbl) ((double *)(ws + L.data))[0] = 1.0;
      else ((float *)(ws + L.data))[0] = 1.0f;
      mx = mn = L.dbl ? dev::abs_bits(1.0) : dev::abs_bits(1.0f);
    }
    *(int64_t *)(ws + L.e) = e;
    *(unsigned long long *)(ws + L.x) = mx;
    *(unsigned long long *)(ws + L.n) = mn;
  }
}

__global__ void k6_finalize(const char *ws, const BRoot *roots, int32_t n, const uint32_t *err,
                            double *mant, int64_t *exp2, uint32_t *flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    mant[i] = *(const double *)(ws + roots[i].data);
    exp2[i] = *(const int64_t *)(ws + roots[i].e);
    flags[i] = *(const uint32_t *)(ws + roots[i].flags) | (*err ? 0x8u : 0u);
  }
}

// Sets `bytes` bytes at each listed offset to 0 (maxima, exponents, flags)
// or 0xff (minima).
struct BClear {
  int64_t off, bytes;
  int32_t value, pad;
};
__global__ void k6_clear(char *ws, const BClear *ranges, int32_t n) {
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const BClear c = ranges[r];
    for (int64_t i = threadIdx.x; i < c.bytes; i += blockDim.x) ws[c.off + i] = (char)c.value;
  }
}

}  // namespace bdev
}  // namespace wmc

using namespace wmc::bdev;

struct wmc_batch {
  std::vector<Plan *> plans;
  std::vector<int64_t> base;       // byte offset of each formula's workspace
  std::vector<BNode> nodes;
  std::vector<BTask> tasks;
  std::vector<BLeaf> leaves;
  std::vector<BRoot> roots;
  std::vector<BClear> clears;
  std::vector<int32_t> root_order; // batch index of each root
  int64_t ws_bytes = 0;            // formulas
  int64_t total_bytes = 0;         // + tables and counters
  double alg_bytes = 0;
  int32_t precision = WMC_SCALED_FP32;
  int32_t max_rank = 0;
  int32_t max_roundings = 0;
  // device state
  char *d_ws = nullptr;            // formulas' workspaces
  char *d_tab = nullptr;           // tables + counters
  BNode *d_nodes = nullptr;
  BTask *d_tasks = nullptr;
  BLeaf *d_leaves = nullptr;
  BRoot *d_roots = nullptr;
  BClear *d_clears = nullptr;
  uint32_t *d_next = nullptr, *d_done = nullptr, *d_err = nullptr;
  double *d_mant = nullptr;
  int64_t *d_exp = nullptr;
  uint32_t *d_flags = nullptr;
  double *h_mant = nullptr;
  int64_t *h_exp = nullptr;
  uint32_t *h_flags = nullptr;
  int32_t grid = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap = nullptr;
  std::mutex mu;
  ~wmc_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_ws);
    cudaFree(d_tab);
    cudaFreeHost(h_mant);
    cudaFreeHost(h_exp);
    cudaFreeHost(h_flags);
  }
};

static std::vector<int32_t> qlabels(const TensorInfo &t) { return t.labels; }  // Q = 1

extern "C" int wmc_batch_create(wmc_plan_t *const *plans, int32_t n_plans, int64_t mem_budget_bytes,
                                wmc_batch_t **out, int32_t *n_admitted) {
  if (!plans || !out || n_plans < 1) { set_error("bad argument"); return WMC_EINVAL; }
  *out = nullptr;
  wmc_batch *b = new (std::nothrow) wmc_batch();
  if (!b) { set_error("out of host memory"); return WMC_ENOMEM; }
  const int32_t prec = plan_of(plans[0]).precision;
  b->precision = prec;
  constexpr int kChunkLog2 = 15;
  int64_t off = 0;
  std::vector<std::vector<int32_t>> node_ids;  // per formula: global node ids in post-order
  for (int32_t f = 0; f < n_plans; ++f) {
    Plan &plan = plan_of(plans[f]);
    if (plan.precision != prec) { delete b; set_error("plans of one batch must share a precision"); return WMC_EINVAL; }
    if (!plan.slice_vars.empty()) { delete b; set_error("sliced plans run through wmc_execute, not a batch"); return WMC_EINVAL; }
    LayoutView lv;
    int rc = exec_layout(plan, 1, &lv);
    if (rc) { delete b; return rc; }
    const int64_t need = (lv.ws_bytes + 255) / 256 * 256;
    if (mem_budget_bytes > 0 && off + need > mem_budget_bytes) break;  // admission by workspace bytes
    b->plans.push_back(&plan);
    b->base.push_back(off);
    const int64_t base = off;
    off += need;
    b->max_rank = std::max(b->max_rank, plan.max_rank);
    auto slot = [&](int64_t region, int64_t t) { return base + region + 8 * (*lv.t_meta)[(size_t)t]; };
    // leaves
    for (int64_t i = 0; i < plan.n_leaves; ++i) {
      const TensorInfo &t = plan.tensors[(size_t)i];
      BLeaf L;
      std::memset(&L, 0, sizeof(L));
      L.data = base + (*lv.t_off)[(size_t)i];
      L.e = slot(lv.off_exp, i);
      L.x = slot(lv.off_max, i);
      L.n = slot(lv.off_min, i);
      L.fals = t.fals;
      L.kind = t.kind;
      L.rank = (int32_t)t.labels.size();
      L.dbl = (*lv.t_dbl)[(size_t)i];
      if (t.kind == LEAF_WEIGHT) {
        L.w0 = plan.w_neg[(size_t)t.labels[0]];
        L.w1 = plan.w_pos[(size_t)t.labels[0]];
      }
      b->leaves.push_back(L);
    }
    // metadata regions to clear each run: flags + error + exponents + maxima, then minima
    b->clears.push_back({base + lv.off_flags, lv.off_max + 8 * lv.n_slots - lv.off_flags, 0, 0});
    b->clears.push_back({base + lv.off_min, 8 * lv.n_slots, 0xff, 0});
    // nodes
    std::vector<int32_t> ids;
    int32_t prev = -1;
    for (const Node &nd : plan.nodes) {
      BNode n;
      std::memset(&n, 0, sizeof(n));
      n.a = base + (*lv.t_off)[(size_t)nd.a];
      n.b = base + (*lv.t_off)[(size_t)nd.b];
      n.c = base + (*lv.t_off)[(size_t)nd.c];
      n.ea = slot(lv.off_exp, nd.a); n.eb = slot(lv.off_exp, nd.b); n.ec = slot(lv.off_exp, nd.c);
      n.xa = slot(lv.off_max, nd.a); n.xb = slot(lv.off_max, nd.b); n.xc = slot(lv.off_max, nd.c);
      n.na = slot(lv.off_min, nd.a); n.nb = slot(lv.off_min, nd.b); n.nc = slot(lv.off_min, nd.c);
      n.flags = base + lv.off_flags;
      k1_bitmaps(qlabels(plan.tensors[(size_t)nd.a]), qlabels(plan.tensors[(size_t)nd.b]),
                 qlabels(plan.tensors[(size_t)nd.c]), &n.rC, &n.k, n.posA, n.posB, n.sposA, n.sposB);
      if (n.k > 24 || n.rC > 31) { delete b; set_error("node too large for the batch executor"); return WMC_EPLAN_TOO_BIG; }
      n.chunk_log2 = std::min<int32_t>(n.rC, kChunkLog2);
      n.n_tasks = 1 << (n.rC - n.chunk_log2);
      n.ti = prec == WMC_FP64 ? 1 : 0;
      n.to = (*lv.t_dbl)[(size_t)nd.c];
      n.ta = (prec == WMC_FP64 || n.to || n.k > 16) ? 1 : 0;
      {
        bool low = n.rC >= n.chunk_log2 && n.chunk_log2 >= 2 && n.posA[0] == 0 && n.posA[1] == 1 &&
                   n.posB[0] < 0 && n.posB[1] < 0;
        for (int j = 0; j < n.k && low; ++j) low = n.sposA[j] >= 2;
        n.vec4 = (low && !n.ti && !n.ta && !n.to) ? 1 : 0;
      }
      n.prev = prev;
      prev = (int32_t)b->nodes.size();
      ids.push_back(prev);
      b->nodes.push_back(n);
      b->alg_bytes += (double)(*lv.t_bytes)[(size_t)nd.a] + (double)(*lv.t_bytes)[(size_t)nd.b] +
                      (double)(*lv.t_bytes)[(size_t)nd.c];
    }
    node_ids.push_back(ids);
    const int64_t root = plan.nodes.back().c;
    b->roots.push_back({base + (*lv.t_off)[(size_t)root], slot(lv.off_exp, root), base + lv.off_flags});
    b->max_roundings = std::max(b->max_roundings, plan.tensors[(size_t)root].roundings);
  }
  if (b->plans.empty()) { delete b; set_error("no formula fits the memory budget"); return WMC_EPLAN_TOO_BIG; }
  b->ws_bytes = off;
  // tasks: round-robin over formulas, each formula in post-order
  size_t longest = 0;
  for (auto &v : node_ids) longest = std::max(longest, v.size());
  for (size_t r = 0; r < longest; ++r)
    for (auto &v : node_ids)
      if (r < v.size()) {
        const BNode &n = b->nodes[(size_t)v[r]];
        for (int32_t c = 0; c < n.n_tasks; ++c) b->tasks.push_back({v[r], c});
      }
  if (n_admitted) *n_admitted = (int32_t)b->plans.size();
  *out = b;
  return WMC_OK;
}

static int batch_ensure_device(wmc_batch *b) {
  if (b->d_ws) return WMC_OK;
  auto al = [](int64_t x) { return (x + 255) / 256 * 256; };
  const int64_t n_nodes = (int64_t)b->nodes.size(), n_roots = (int64_t)b->roots.size();
  int64_t o = 0;
  const int64_t o_nodes = o; o += al(sizeof(BNode) * n_nodes);
  const int64_t o_tasks = o; o += al(sizeof(BTask) * (int64_t)b->tasks.size());
  const int64_t o_leaves = o; o += al(sizeof(BLeaf) * (int64_t)b->leaves.size());
  const int64_t o_roots = o; o += al(sizeof(BRoot) * n_roots);
  const int64_t o_clears = o; o += al(sizeof(BClear) * (int64_t)b->clears.size());
  const int64_t o_ctr = o; o += al(4 * (2 + n_nodes));  // next, err, done[]
  const int64_t o_mant = o; o += al(8 * n_roots);
  const int64_t o_exp = o; o += al(8 * n_roots);
  const int64_t o_flags = o; o += al(4 * n_roots);
  int rc;
  if ((rc = device_alloc((void **)&b->d_ws, (size_t)b->ws_bytes))) return rc;
  if ((rc = device_alloc((void **)&b->d_tab, (size_t)o))) { cudaFree(b->d_ws); b->d_ws = nullptr; return rc; }
  b->total_bytes = b->ws_bytes + o;
  char *t = b->d_tab;
  b->d_nodes = (BNode *)(t + o_nodes);
  b->d_tasks = (BTask *)(t + o_tasks);
  b->d_leaves = (BLeaf *)(t + o_leaves);
  b->d_roots = (BRoot *)(t + o_roots);
  b->d_clears = (BClear *)(t + o_clears);
  b->d_next = (uint32_t *)(t + o_ctr);
  b->d_err = b->d_next + 1;
  b->d_done = b->d_next + 2;
  b->d_mant = (double *)(t + o_mant);
  b->d_exp = (int64_t *)(t + o_exp);
  b->d_flags = (uint32_t *)(t + o_flags);
  auto up = [](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  if (up(b->d_nodes, b->nodes.data(), sizeof(BNode) * b->nodes.size()) ||
      up(b->d_tasks, b->tasks.data(), sizeof(BTask) * b->tasks.size()) ||
      up(b->d_leaves, b->leaves.data(), sizeof(BLeaf) * b->leaves.size()) ||
      up(b->d_roots, b->roots.data(), sizeof(BRoot) * b->roots.size()) ||
      up(b->d_clears, b->clears.data(), sizeof(BClear) * b->clears.size())) {
    set_error("uploading the batch tables failed");
    return WMC_ECUDA;
  }
  if (cudaMallocHost((void **)&b->h_mant, 8 * (size_t)n_roots) ||
      cudaMallocHost((void **)&b->h_exp, 8 * (size_t)n_roots) ||
      cudaMallocHost((void **)&b->h_flags, 4 * (size_t)n_roots)) {
    set_error("pinned allocation failed");
    return WMC_ENOMEM;
  }
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k6_persistent, kThreads, 0);
  b->grid = std::max(1, per_sm) * std::max(1, sms);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) { set_error("stream creation failed"); return WMC_ECUDA; }
  return WMC_OK;
}

// leaves, clears, counters, the persistent contraction, the results
static void batch_enqueue(wmc_batch *b, cudaStream_t s) {
  const int32_t n_nodes = (int32_t)b->nodes.size();
  k6_clear<<<std::min<int64_t>((int64_t)b->clears.size(), 4096), 256, 0, s>>>(b->d_ws, b->d_clears,
                                                                              (int32_t)b->clears.size());
  cudaMemsetAsync(b->d_next, 0, 4 * (size_t)(2 + n_nodes), s);
  const int64_t nl = (int64_t)b->leaves.size();
  k6_leaves<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nl + 255) / 256, 4096)), 256, 0, s>>>(
      b->d_ws, b->d_leaves, nl);
  BatchArgs a;
  a.ws = b->d_ws;
  a.nodes = b->d_nodes;
  a.tasks = b->d_tasks;
  a.n_tasks = (int32_t)b->tasks.size();
  a.next = b->d_next;
  a.done = b->d_done;
  a.err = b->d_err;
  k6_persistent<<<(unsigned)b->grid, kThreads, 0, s>>>(a);
  const int32_t nr = (int32_t)b->roots.size();
  k6_finalize<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(b->d_ws, b->d_roots, nr, b->d_err, b->d_mant,
                                                          b->d_exp, b->d_flags);
}

extern "C" int wmc_batch_execute(wmc_batch_t *b, void *stream, wmc_result *out) {
  if (!b || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  std::lock_guard<std::mutex> lk(b->mu);
  int rc = batch_ensure_device(b);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) { set_error("capture failed"); return WMC_ECUDA; }
    batch_enqueue(b, b->cap);
    if (cudaStreamEndCapture(b->cap, &g) || cudaGraphInstantiate(&b->graph, g, 0)) {
      if (g) cudaGraphDestroy(g);
      set_error("batch graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
      return WMC_ECUDA;
    }
    cudaGraphDestroy(g);
  }
  if (cudaGraphLaunch(b->graph, s)) { set_error("graph launch failed"); return WMC_ECUDA; }
  count_launches(4);
  const size_t n = b->roots.size();
  if (cudaMemcpyAsync(b->h_mant, b->d_mant, 8 * n, cudaMemcpyDeviceToHost, s) ||
      cudaMemcpyAsync(b->h_exp, b->d_exp, 8 * n, cudaMemcpyDeviceToHost, s) ||
      cudaMemcpyAsync(b->h_flags, b->d_flags, 4 * n, cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s)) {
    set_error("batch execution failed: %s", cudaGetErrorString(cudaGetLastError()));
    return WMC_ECUDA;
  }
  const double u = b->precision == WMC_FP64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  for (size_t i = 0; i < n; ++i) {
    if (b->h_flags[i] & WMC_FLAG_DEVICE_TIMEOUT) { set_error("a bounded wait timed out"); return WMC_ETIMEOUT; }
    wmc_result &r = out[i];
    int fe = 0;
    const double fr = std::frexp(b->h_mant[i], &fe);
    r.mant = fr;
    r.exp2 = b->h_mant[i] == 0.0 ? 0 : b->h_exp[i] + fe;
    r.log10 = b->h_mant[i] == 0.0 ? -INFINITY : std::log10(std::fabs(fr)) + (double)r.exp2 * std::log10(2.0);
    r.flags = b->h_flags[i] & WMC_FLAG_FP32_FLUSH;
    const double d = (double)b->plans[i]->tensors[(size_t)b->plans[i]->nodes.back().c].roundings;
    r.rel_err_bound = d * u / (1.0 - d * u);
    if (b->plans[i]->any_negative) r.flags |= WMC_FLAG_NO_BOUND;
    r.reserved = 0;
  }
  return WMC_OK;
}

extern "C" int wmc_batch_info(const wmc_batch_t *b, wmc_batch_info_t *out) {
  if (!b || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  std::memset(out, 0, sizeof(*out));
  out->n_formulas = (int64_t)b->plans.size();
  out->n_nodes = (int64_t)b->nodes.size();
  out->n_tasks = (int64_t)b->tasks.size();
  out->workspace_bytes = b->ws_bytes;
  out->algorithmic_bytes = b->alg_bytes;
  out->max_rank = b->max_rank;
  out->grid = b->grid;
  return WMC_OK;
}

extern "C" int wmc_batch_formula_info(const wmc_batch_t *b, int32_t i, int64_t *ws_offset,
                                      int32_t *max_rank, int64_t *n_nodes) {
  if (!b || i < 0 || (size_t)i >= b->plans.size()) { set_error("bad batch or formula index"); return WMC_EINVAL; }
  if (ws_offset) *ws_offset = b->base[(size_t)i];
  if (max_rank) *max_rank = b->plans[(size_t)i]->max_rank;
  if (n_nodes) *n_nodes = (int64_t)b->plans[(size_t)i]->nodes.size();
  return WMC_OK;
}

extern "C" void wmc_batch_destroy(wmc_batch_t *b) { delete b; }
