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
//
// Task order.  Each formula is a chain of nodes, so the batch's length is at
// least its longest formula's chain.  The list is built on the host by list
// scheduling (Algorithm 2's post-order within each formula): a simulation
// of the resident blocks, with a cost model of each task, repeatedly gives
// the next free block a task of the ready node whose formula has the most
// estimated work left on its chain (its bottom level), so the long chains
// start at once and never queue behind the short formulas' large nodes.  A
// node enters the simulation only after its predecessor's tasks have
// finished there, so a task's dependency always comes earlier in the list;
// only running blocks take tasks, so every wait ends.  Each wait is also
// bounded by %globaltimer (one second); on timeout the block records an
// error word and stops.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <queue>
#include <cstring>
#include <map>
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
  int32_t chunk_log2;       // outputs per task = 2^chunk_log2 (<= 16)
  int32_t rC, k;
  int8_t ti, ta, to;        // element types: 0 float, 1 double
  int8_t vec4;              // float32, C's two lowest bits are A's, B has neither: 4 outputs per thread
  int8_t stream;            // stream mode (below); chunk_log2 then counts u, not outputs
  int8_t f;                 // stream mode: output bits absent from A ("S-free", <= 4)
  int8_t rB;                // rank of B
  int8_t bglob;             // stream mode: B read from global memory (L2), not staged (rank > 8)
  int32_t chain;            // chain mode (stream == 2): index of its BChain; subtrees
                            // (stream == 3): index of the formula's first BGroup
  float est_us;             // subtrees: estimated microseconds per task (list scheduling)
  int8_t posA[32], posB[32], sposA[24], sposB[24];
};

// Chain mode: D <= 4 consecutive frontier steps of one formula in one pass.
// Step i contracts the running tensor with S_i, summing x_i (an index of
// the chain's first operand A_1) and adding y_i (no index when the last
// step `shrink`s), so C_i = sum over x_i of C_{i-1} S_i with C_0 = A_1.  A
// work unit is one assignment u of A_1's passive indices (those no step
// sums); the thread holds the 2^D values over the chain state in
// registers: bit i is x_i before step i and y_i after it.  S_i may hold
// passive indices, x_i, y_i and the two indices added last (y_{i-1},
// y_{i-2}).
struct BChain {
  int64_t s[4], es[4], xs[4], ns[4];  // S_i: data, exponent, max, min slots (byte offsets)
  int8_t D, shrink, nu, grow;         // steps, last step adds nothing, passive indices, first adds two
  int8_t rs[4];                       // rank of S_i
  int8_t xa[4];                       // A_1 bit of x_i
  int8_t yc[4];                       // C_D bit of y_i (-1: the shrink step)
  int8_t zc, pad2[3];                 // C_D bit of z, the second index a growth step adds
  // S_i bit of x_i, y_i and of the two indices added last before step i
  // (in the order y_0, z, y_1, ...), or of z at a growth step (-1: none)
  int8_t sx[4], sy[4], s1[4], s2[4];
  int8_t ua[32], uc[32];              // u bit -> A_1 bit, C_D bit (u: passive indices in C_D order)
  int8_t us[4][32];                   // u bit -> S_i bit (-1: none)
};

// One small subtree of a formula, run by one block as one task: its nodes
// (members[first .. first + n), in post-order) one after another, each in
// a single pass over its outputs, with no waits (every operand is a leaf
// or an earlier member's output).
struct BGroup {
  int32_t first, n;
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
  const BChain *chains;
  const BGroup *groups;
  const BNode *members;
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
// are built before the previous node is waited for, and kept while a block
// takes consecutive tasks of one node).  A task covers 2^chunk_log2
// consecutive outputs, at most 2^16: rows 0-1 map the task-local output
// bits to A's offset, rows 2-3 to B's, rows 4/6/8 the summed bits 0-7,
// 8-15, 16-23 to A's, rows 5/7/9 to B's.  Entry v of a row is the OR of
// the single-bit offsets of v's set bits.
constexpr int kLutRows = 12;        // (12 for chain mode: 2 per operand)
#ifndef WMC_BATCH_THREADS
#define WMC_BATCH_THREADS 256
#endif
constexpr int kBThreads = WMC_BATCH_THREADS;  // threads of a persistent block
constexpr int kBlocksPerSM = 1024 / kBThreads;  // resident blocks per SM (the launch bounds)

// Scratch of the table builders: each row's eight single-bit offsets and
// its two 16-entry nibble tables.
struct RowScratch {
  uint32_t bit[kLutRows][8];
  uint32_t nib[kLutRows][2][16];
};

// Rows 0..n_rows-1 of 256 entries from rs.bit (filled by the caller before
// a barrier): entry v = OR of bit[r][b] over the set bits b of v, as the
// OR of two nibble-table entries, so every thread builds whole entries
// with two shared loads.  Ends with a barrier.
__device__ __forceinline__ void rows_from_bits(uint32_t (*rows)[256], RowScratch &rs, int n_rows) {
  for (int i = threadIdx.x; i < n_rows * 32; i += blockDim.x) {
    const int r = i >> 5, h = (i >> 4) & 1, v = i & 15;
    uint32_t o = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if ((v >> b) & 1) o |= rs.bit[r][4 * h + b];
    rs.nib[r][h][v] = o;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_rows * 256; i += blockDim.x) {
    const int r = i >> 8, v = i & 255;
    rows[r][v] = rs.nib[r][0][v & 15] | rs.nib[r][1][v >> 4];
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t bit_of(int8_t pos) { return pos >= 0 ? 1u << pos : 0u; }

__device__ __forceinline__ void batch_lut(const BNode &nd, uint32_t (*lut)[256], RowScratch &rs) {
  const int lbits = nd.chunk_log2;  // task-local output bits
  // every row (entry 0 of the unused ones is read where an index's high
  // byte is zero, and must be 0)
  const int n_rows = 10;
  for (int i = threadIdx.x; i < n_rows * 8; i += blockDim.x) {
    const int row = i >> 3, b = i & 7;
    uint32_t o = 0;
    if (row < 4) {
      const int j = (row & 1) * 8 + b;
      if (j < lbits) o = bit_of(row < 2 ? nd.posA[j] : nd.posB[j]);
    } else {
      const int j = ((row - 4) >> 1) * 8 + b;
      if (j < nd.k) o = bit_of((row & 1) == 0 ? nd.sposA[j] : nd.sposB[j]);
    }
    rs.bit[row][b] = o;
  }
  __syncthreads();
  rows_from_bits(lut, rs, n_rows);
}

// A's and B's offsets of a task's first output (its bits above the task's
// local bits).
__device__ __forceinline__ void batch_base(const BNode &nd, uint64_t o0, uint32_t &bA, uint32_t &bB) {
  bA = 0; bB = 0;
  for (int j = nd.chunk_log2; j < nd.rC; ++j)
    if ((o0 >> j) & 1) {
      if (nd.posA[j] >= 0) bA |= 1u << nd.posA[j];
      if (nd.posB[j] >= 0) bB |= 1u << nd.posB[j];
    }
}

// C's exponent and the float32 flush test (as in the single-plan
// kernels), from the operands' metadata alone, by one thread of a node's
// first task, beside the outputs.
template <typename TI>
__device__ __forceinline__ void node_exponent(char *ws, const BNode &nd, unsigned long long ma,
                                              unsigned long long mb) {
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

// Block reduction of the task's max |C| and min nonzero |C| into red[0]
// (max) and red[1] (min): folded across each warp first (max and min are
// exact), one shared atomic per warp, then one global atomic each.
template <typename TO>
__device__ __forceinline__ void task_maxmin(char *ws, const BNode &nd, TO tmax, unsigned long long tmin,
                                            unsigned long long *red) {
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

template <typename T>
__device__ __forceinline__ void track_out(T c, T &tmax, unsigned long long &tmin) {
  const T m = c < (T)0 ? -c : c;
  tmax = m > tmax ? m : tmax;
  if (m != (T)0) {
    const unsigned long long bits = dev::abs_bits(m);
    tmin = bits < tmin ? bits : tmin;
  }
}

// ---- stream mode
//
// The frontier-times-bucket shape that carries almost all of a batch's
// bytes: A = P holds every output index except f <= 4 "S-free" ones, B = S
// has at most 8 indices, k <= 2 indices are summed.  A task owns 2^cl
// consecutive assignments u of C's indices that A holds; a thread loads
// A's 2^k entries of its u once and writes the 2^f outputs that differ
// only in the S-free indices (so A and C cross memory once each, as in the
// single-plan streaming kernels), with S staged in shared memory,
// pre-scaled.  The summed terms are added as in the generic path (operands
// scaled first, one fused multiply-add per term in ascending summed
// assignment, from zero), so the results are the same bits.
struct StreamGeom {
  uint32_t lut[6][256];          // u-local bits 0-7 / 8-15 -> C, A, S offsets
  uint32_t cv[16], sv[16];       // S-free assignment v -> C offset, S offset
  uint32_t as[4], ss[4];         // summed assignment s -> A offset, S offset
  uint32_t sl[4];                // u's two lowest bits -> S offset (vector path)
  int8_t uc[32], ua[32], us[32]; // u bit -> C bit, A bit, S bit (-1: none)
  int8_t vc[4], vs[4], nv;       // S-free bit -> C bit, S bit; their number
};
constexpr int kSMaxS = 256;      // S entries staged (B rank <= 8)

__device__ __forceinline__ void stream_geom(const BNode &nd, StreamGeom &g, RowScratch &rs) {
  // u bits (C's bits that A holds) and S-free bits, in C's order: one
  // warp compacts them with ballots
  if (threadIdx.x < 32) {
    const int j = threadIdx.x;
    const int8_t pa = j < nd.rC ? nd.posA[j] : (int8_t)-1, pb = j < nd.rC ? nd.posB[j] : (int8_t)-1;
    const unsigned mu = __ballot_sync(0xffffffffu, j < nd.rC && pa >= 0);
    const unsigned mv = __ballot_sync(0xffffffffu, j < nd.rC && pa < 0);
    const unsigned below = (1u << j) - 1u;
    if (j < nd.rC && pa >= 0) {
      const int r = __popc(mu & below);
      g.uc[r] = (int8_t)j; g.ua[r] = pa; g.us[r] = pb;
    } else if (j < nd.rC) {
      const int r = __popc(mv & below);
      if (r < 4) { g.vc[r] = (int8_t)j; g.vs[r] = pb; }
    }
    if (j == 0) g.nv = (int8_t)min(4, __popc(mv));
  }
  __syncthreads();
  const int cl = nd.chunk_log2, lo = nd.vec4 ? 2 : 0;
  const int t = threadIdx.x;
  if (t < 16) {  // S-free assignment v -> C and S offsets
    uint32_t c = 0, sv = 0;
    for (int i = 0; i < g.nv; ++i)
      if ((t >> i) & 1) { c |= 1u << g.vc[i]; sv |= bit_of(g.vs[i]); }
    g.cv[t] = c; g.sv[t] = sv;
  } else if (t < 20) {  // summed assignment -> A and S offsets
    const int sidx = t - 16;
    uint32_t a = 0, sb = 0;
    for (int i = 0; i < nd.k; ++i)
      if ((sidx >> i) & 1) { a |= bit_of(nd.sposA[i]); sb |= bit_of(nd.sposB[i]); }
    g.as[sidx] = a; g.ss[sidx] = sb;
  } else if (t < 24) {  // u's two lowest bits -> S offset (vector path)
    const int e = t - 20;
    uint32_t o = 0;
    for (int i = 0; i < 2 && i < cl; ++i)
      if ((e >> i) & 1) o |= bit_of(g.us[i]);
    g.sl[e] = o;
  } else if (t >= 32 && t < 32 + 48) {
    // rows over u-local bits 0-7 and 8-15 (vector path, groups of four
    // u: bits 2-9 and 10-17, so that consecutive threads, which take
    // consecutive groups, read consecutive entries, no bank conflicts)
    const int row = (t - 32) >> 3, b = (t - 32) & 7, jb = lo + (row & 1) * 8 + b;
    const int8_t *pos = row < 2 ? g.uc : (row < 4 ? g.ua : g.us);
    rs.bit[row][b] = jb < cl ? bit_of(pos[jb]) : 0u;
  }
  __syncthreads();
  rows_from_bits(g.lut, rs, 6);
}

template <typename T, int NS, bool BG>
__device__ void run_stream(const BatchArgs &ba, const BNode &nd, int chunk, const StreamGeom &g, T *sS,
                           unsigned long long *red) {
  char *ws = ba.ws;
  const T *A = (const T *)(ws + nd.a);
  const T *B = (const T *)(ws + nd.b);
  T *C = (T *)(ws + nd.c);
  const unsigned long long ma = ldcg((const unsigned long long *)(ws + nd.xa));
  const unsigned long long mb = ldcg((const unsigned long long *)(ws + nd.xb));
  const T sa = dev::pow2_scale(dev::pow2_exp_of(ma, T()), T());
  const T sb = dev::pow2_scale(dev::pow2_exp_of(mb, T()), T());
  if (chunk == 0 && threadIdx.x == 32) node_exponent<T>(ws, nd, ma, mb);
  if (!BG)
    for (int i = threadIdx.x; i < (1 << nd.rB); i += blockDim.x) sS[i] = ldcg(B + i) * sb;
  // S's entry at `off`: staged and pre-scaled, or (BG: a large B) from L2
  auto sval = [&](uint32_t off) { return BG ? ldcg(B + off) * sb : sS[off]; };
  // offsets of the task's first u (its bits above the task's local bits)
  const uint32_t u0 = (uint32_t)chunk << nd.chunk_log2;
  uint32_t bC = 0, bA = 0, bS = 0;
  for (int i = nd.chunk_log2; i < nd.rC - nd.f; ++i)
    if ((u0 >> i) & 1) {
      bC |= 1u << g.uc[i];
      bA |= 1u << g.ua[i];
      if (g.us[i] >= 0) bS |= 1u << g.us[i];
    }
  __syncthreads();  // sS
  const uint32_t n_loc = 1u << nd.chunk_log2;
  const int nv = 1 << nd.f;  // NS = 2^k summed assignments
  T tmax = (T)0;
  unsigned long long tmin = kNoMin;
  if constexpr (sizeof(T) == 4) {
    if (nd.vec4) {
      // four consecutive u per group (C's and A's two lowest bits), two
      // groups per step with their loads issued first
      // groups g of four u (l = 4 g): a thread takes groups g0 and
      // g0 + blockDim, so a warp's table reads are consecutive entries
      const uint32_t n_grp = n_loc >> 2;
      for (uint32_t g0 = threadIdx.x; g0 < n_grp; g0 += 2 * blockDim.x) {
        float4 a4[2][NS];
        uint32_t cb[2], sbx[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          // the second group is past the task when it has fewer than
          // 2 blockDim groups (n_grp is a power of two)
          const uint32_t gi = g0 + q * blockDim.x;
          const uint32_t gv = gi < n_grp ? gi : g0;
          const uint32_t ab = bA | g.lut[2][gv & 255] | g.lut[3][gv >> 8];
          cb[q] = bC | g.lut[0][gv & 255] | g.lut[1][gv >> 8];
          sbx[q] = bS | g.lut[4][gv & 255] | g.lut[5][gv >> 8];
#pragma unroll
          for (int sidx = 0; sidx < NS; ++sidx)
            a4[q][sidx] = __ldcg(reinterpret_cast<const float4 *>(A + (ab | g.as[sidx])));
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q == 1 && g0 + blockDim.x >= n_grp) break;
          float a[NS][4];
#pragma unroll
          for (int sidx = 0; sidx < NS; ++sidx) {
              a[sidx][0] = a4[q][sidx].x * sa; a[sidx][1] = a4[q][sidx].y * sa;
              a[sidx][2] = a4[q][sidx].z * sa; a[sidx][3] = a4[q][sidx].w * sa;
            }
          for (int v = 0; v < nv; ++v) {
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const uint32_t so = sbx[q] | g.sl[e] | g.sv[v];
              float acc = 0.0f;
#pragma unroll
              for (int sidx = 0; sidx < NS; ++sidx)
                acc = dev::fma_t(a[sidx][e], sval(so | g.ss[sidx]), acc);
              out[e] = acc;
              track_out(acc, tmax, tmin);
            }
            *reinterpret_cast<float4 *>(C + (cb[q] | g.cv[v])) = make_float4(out[0], out[1], out[2], out[3]);
          }
        }
      }
      task_maxmin<T>(ws, nd, tmax, tmin, red);
      return;
    }
  }
  for (uint32_t l = threadIdx.x; l < n_loc; l += blockDim.x) {
    const uint32_t ab = bA | g.lut[2][l & 255] | g.lut[3][l >> 8];
    const uint32_t cb = bC | g.lut[0][l & 255] | g.lut[1][l >> 8];
    const uint32_t sbx = bS | g.lut[4][l & 255] | g.lut[5][l >> 8];
    T a[NS];
#pragma unroll
    for (int sidx = 0; sidx < NS; ++sidx) a[sidx] = ldcg(A + (ab | g.as[sidx])) * sa;
    for (int v = 0; v < nv; ++v) {
      T acc = (T)0;
#pragma unroll
      for (int sidx = 0; sidx < NS; ++sidx) acc = dev::fma_t(a[sidx], sval(sbx | g.sv[v] | g.ss[sidx]), acc);
      C[cb | g.cv[v]] = acc;
      track_out(acc, tmax, tmin);
    }
  }
  task_maxmin<T>(ws, nd, tmax, tmin, red);
}

// ---- chain mode
struct ChainGeom {
  uint32_t lut[12][256];  // rows 2t, 2t+1: u-local bits 0-7, 8-15 -> offset in A_1, C_D, S_1..S_4
  uint32_t dS[4][16];     // S_i offset of (x_i, y_i, y_{i-1}, y_{i-2}) = bits 0-3 of the entry
  uint32_t pA[16];        // A_1 offset of the x-state s (bit i = x_i)
  uint32_t dC[16];        // C_D offset of the final state s (bit i = y_i, bit D = z)
};

__device__ __forceinline__ void chain_geom(const BNode &nd, const BChain &ch, ChainGeom &g, RowScratch &rs) {
  const int D = ch.D, cl = nd.chunk_log2;
  for (int t = threadIdx.x; t < 16 + 64 + 96; t += blockDim.x) {
    if (t < 16) {  // x-state -> A_1 offset, final state -> C_D offset
      uint32_t pa = 0, dc = 0;
      for (int i = 0; i < D; ++i)
        if ((t >> i) & 1) { pa |= 1u << ch.xa[i]; dc |= bit_of(ch.yc[i]); }
      if (ch.grow && ((t >> D) & 1)) dc |= bit_of(ch.zc);
      g.pA[t] = pa; g.dC[t] = dc;
    } else if (t < 16 + 64) {  // S_i offset of (x_i, y_i, y_{i-1}, y_{i-2})
      const int i = (t - 16) >> 4, j = (t - 16) & 15;
      uint32_t o = 0;
      if (i < D) {
        if (j & 1) o |= bit_of(ch.sx[i]);
        if (j & 2) o |= bit_of(ch.sy[i]);
        if (j & 4) o |= bit_of(ch.s1[i]);
        if (j & 8) o |= bit_of(ch.s2[i]);
      }
      g.dS[i][j] = o;
    } else {  // rows 2t'+h: u-local bits 8h..8h+7 -> A_1, C_D, S_1..S_4
      const int row = (t - 80) >> 3, b = (t - 80) & 7, jb = (row & 1) * 8 + b, tg = row >> 1;
      uint32_t o = 0;
      if (jb < cl && tg < 2 + D) o = bit_of(tg == 0 ? ch.ua[jb] : (tg == 1 ? ch.uc[jb] : ch.us[tg - 2][jb]));
      rs.bit[row][b] = o;
    }
  }
  __syncthreads();
  rows_from_bits(g.lut, rs, 2 * (2 + D));
}

// C_D's exponent: A_1's and every S_i's (the intermediates are never
// rescaled: their scales are powers of two, so only this bookkeeping
// moves); the flush test over the smallest nonzero scaled entries of all
// D + 1 operands, a lower bound on every product the chain forms.
template <typename T>
__device__ __forceinline__ void chain_exponent(char *ws, const BNode &nd, const BChain &ch,
                                               unsigned long long ma) {
  int64_t e = ldcg((const int64_t *)(ws + nd.ea)) + dev::pow2_exp_of(ma, T());
  const unsigned long long na = ldcg((const unsigned long long *)(ws + nd.na));
  bool zero = na == kNoMin;
  T lo = zero ? (T)0 : dev::from_bits<T>(na) * dev::pow2_scale(dev::pow2_exp_of(ma, T()), T());
  for (int i = 0; i < ch.D; ++i) {
    const unsigned long long mb = ldcg((const unsigned long long *)(ws + ch.xs[i]));
    const unsigned long long nb = ldcg((const unsigned long long *)(ws + ch.ns[i]));
    e += ldcg((const int64_t *)(ws + ch.es[i])) + dev::pow2_exp_of(mb, T());
    if (nb == kNoMin) zero = true;
    else lo *= dev::from_bits<T>(nb) * dev::pow2_scale(dev::pow2_exp_of(mb, T()), T());
  }
  *(int64_t *)(ws + nd.ec) = e;
  if (!zero && dev::below_normal(lo)) atomicOr((uint32_t *)(ws + nd.flags), 2u);
}

// State bit of the index added `back` additions before step I (0: the last
// one, 1: the one before), in the order y_0, z (growth), y_1, y_2, ...; -1
// when there is none.  y_j sits at bit j, z at bit D.
__host__ __device__ constexpr int added_bit(int D, bool GROW, int I, int back) {
  int seq[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int n = 0;
  for (int j = 0; j < I; ++j) {
    seq[n++] = j;
    if (j == 0 && GROW) seq[n++] = D;
  }
  return n - 1 - back >= 0 ? seq[n - 1 - back] : -1;
}

// Step I on the register block.  In place (the usual step): for each state
// of the other bits, the two values over x_I become the values over y_I (one
// value when the last step shrinks).  Growth (step 0 of a growth chain): the
// two values over x_0 become four over (y_0, z).  Every output is a
// two-term fused multiply-add chain over x_I = 0, 1 from zero: the order of
// every other kernel for one summed index.  S_I's value for a state is
// sv[x | y << 1 | d1 << 2 | d2 << 3] with d1, d2 the two indices added last
// (at a growth step: sv[x | y_0 << 1 | z << 2]).
template <typename T, int D, bool SHRINK, bool GROW, int I>
__device__ __forceinline__ void chain_step(T (&a)[1 << (D + GROW)], const T *S, uint32_t sb, const uint32_t *dS) {
  constexpr int NB = D + GROW;
  constexpr bool last = SHRINK && I == D - 1;
  constexpr bool growth = GROW && I == 0;
  constexpr int b1 = added_bit(D, GROW, I, 0), b2 = added_bit(D, GROW, I, 1);
  T sv[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if ((last && (j & 2)) || ((growth ? 0 : b1) < 0 && (j & 4)) || (b2 < 0 && (j & 8)) || (growth && (j & 8)))
      continue;
    sv[j] = S[sb | dS[j]];
  }
#pragma unroll
  for (int o = 0; o < (1 << NB); ++o) {
    if (o & (1 << I)) continue;
    if (growth && (o & (1 << D))) continue;  // z is not there yet
    const T a0 = a[o], a1 = a[o | (1 << I)];
    if (growth) {
#pragma unroll
      for (int yz = 0; yz < 4; ++yz) {
        const int j = (yz & 1) << 1 | (yz >> 1) << 2;
        T c = dev::fma_t(a0, sv[j], (T)0);
        c = dev::fma_t(a1, sv[j | 1], c);
        a[o | ((yz & 1) << I) | ((yz >> 1) << D)] = c;
      }
      continue;
    }
    const int dd = (b1 >= 0 ? ((o >> b1) & 1) << 2 : 0) | (b2 >= 0 ? ((o >> b2) & 1) << 3 : 0);
    T c0 = dev::fma_t(a0, sv[dd], (T)0);
    c0 = dev::fma_t(a1, sv[dd | 1], c0);
    a[o] = c0;
    if (!last) {
      T c1 = dev::fma_t(a0, sv[dd | 2], (T)0);
      c1 = dev::fma_t(a1, sv[dd | 3], c1);
      a[o | (1 << I)] = c1;
    }
  }
}

template <typename T, int D, bool SHRINK, bool GROW, int I>
struct ChainSteps {
  __device__ static __forceinline__ void run(T (&a)[1 << (D + GROW)], const T *sS, const uint32_t (&sb)[D],
                                             const ChainGeom &g) {
    chain_step<T, D, SHRINK, GROW, I>(a, sS + I * kSMaxS, sb[I], g.dS[I]);
    ChainSteps<T, D, SHRINK, GROW, I + 1>::run(a, sS, sb, g);
  }
};
template <typename T, int D, bool SHRINK, bool GROW>
struct ChainSteps<T, D, SHRINK, GROW, D> {
  __device__ static __forceinline__ void run(T (&)[1 << (D + GROW)], const T *, const uint32_t (&)[D],
                                             const ChainGeom &) {}
};

template <typename T, int D, bool SHRINK, bool GROW>
__device__ void run_chain(const BatchArgs &ba, const BNode &nd, const BChain &ch, int chunk, const ChainGeom &g,
                          T *sS, unsigned long long *red) {
  constexpr int NB = D + GROW;
  char *ws = ba.ws;
  const T *A = (const T *)(ws + nd.a);
  T *C = (T *)(ws + nd.c);
  const unsigned long long ma = ldcg((const unsigned long long *)(ws + nd.xa));
  const T sa = dev::pow2_scale(dev::pow2_exp_of(ma, T()), T());
  if (chunk == 0 && threadIdx.x == 32) chain_exponent<T>(ws, nd, ch, ma);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const unsigned long long mb = ldcg((const unsigned long long *)(ws + ch.xs[i]));
    const T sb = dev::pow2_scale(dev::pow2_exp_of(mb, T()), T());
    const T *S = (const T *)(ws + ch.s[i]);
    for (int j = threadIdx.x; j < (1 << ch.rs[i]); j += blockDim.x) sS[i * kSMaxS + j] = ldcg(S + j) * sb;
  }
  // offsets of the task's first u (its bits above the task's local bits)
  const int cl = nd.chunk_log2;
  const uint32_t u0 = (uint32_t)chunk << cl;
  uint32_t bA = 0, bC = 0, bS[D];
#pragma unroll
  for (int i = 0; i < D; ++i) bS[i] = 0;
  for (int j = cl; j < ch.nu; ++j)
    if ((u0 >> j) & 1) {
      bA |= 1u << ch.ua[j];
      bC |= 1u << ch.uc[j];
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (ch.us[i][j] >= 0) bS[i] |= 1u << ch.us[i][j];
    }
  __syncthreads();  // sS
  const uint32_t n_loc = 1u << cl;
  T tmax = (T)0;
  unsigned long long tmin = kNoMin;
  for (uint32_t l = threadIdx.x; l < n_loc; l += blockDim.x) {
    const uint32_t lo = l & 255, hi = l >> 8;
    const uint32_t cb = bC | g.lut[2][lo] | g.lut[3][hi];
    uint32_t sb[D];
#pragma unroll
    for (int i = 0; i < D; ++i) sb[i] = bS[i] | g.lut[4 + 2 * i][lo] | g.lut[5 + 2 * i][hi];
    const uint32_t ab = bA | g.lut[0][lo] | g.lut[1][hi];
    T a[1 << NB];
#pragma unroll
    for (int st = 0; st < (1 << D); ++st) a[st] = ldcg(A + (ab | g.pA[st]));
#pragma unroll
    for (int st = 0; st < (1 << D); ++st) a[st] *= sa;
    ChainSteps<T, D, SHRINK, GROW, 0>::run(a, sS, sb, g);
#pragma unroll
    for (int st = 0; st < (1 << NB); ++st) {
      if (SHRINK && ((st >> (D - 1)) & 1)) continue;  // summed away
      C[cb | g.dC[st]] = a[st];
      track_out(a[st], tmax, tmin);
    }
  }
  task_maxmin<T>(ws, nd, tmax, tmin, red);
}

template <typename T>
__device__ __forceinline__ void chain_dispatch(const BatchArgs &ba, const BNode &nd, const BChain &ch, int chunk,
                                               const ChainGeom &g, T *sS, unsigned long long *red) {
  if (ch.grow) {  // growth chains: two or three steps, no shrink
    if (ch.D == 2) run_chain<T, 2, false, true>(ba, nd, ch, chunk, g, sS, red);
    else run_chain<T, 3, false, true>(ba, nd, ch, chunk, g, sS, red);
    return;
  }
  const int sel = ch.D * 2 + (ch.shrink ? 1 : 0);
  switch (sel) {
    case 4: run_chain<T, 2, false, false>(ba, nd, ch, chunk, g, sS, red); break;
    case 5: run_chain<T, 2, true, false>(ba, nd, ch, chunk, g, sS, red); break;
    case 6: run_chain<T, 3, false, false>(ba, nd, ch, chunk, g, sS, red); break;
    case 7: run_chain<T, 3, true, false>(ba, nd, ch, chunk, g, sS, red); break;
    case 8: run_chain<T, 4, false, false>(ba, nd, ch, chunk, g, sS, red); break;
    default: run_chain<T, 4, true, false>(ba, nd, ch, chunk, g, sS, red); break;
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
  if (chunk == 0 && threadIdx.x == 32) node_exponent<TI>(ws, nd, ma, mb);
  const uint64_t o0 = (uint64_t)chunk << nd.chunk_log2;
  const uint32_t n_loc = 1u << nd.chunk_log2;  // outputs of this task
  uint32_t baseA, baseB;
  batch_base(nd, o0, baseA, baseB);
  const uint32_t ns = 1u << nd.k;
  TO tmax = (TO)0;
  unsigned long long tmin = kNoMin;
  if constexpr (sizeof(TI) == 4 && sizeof(TA) == 4 && sizeof(TO) == 4) {
    if (nd.vec4 && nd.k <= 8) {
      // four consecutive outputs per thread: A's four values per summed
      // term in one 16-byte load, one B value, the same sums in the same
      // order as below
      for (uint32_t l = 4 * threadIdx.x; l < n_loc; l += 4 * blockDim.x) {
        const uint64_t o = o0 + l;
        const uint32_t bA = baseA | lut[0][l & 255] | lut[1][l >> 8];
        const uint32_t bB = baseB | lut[2][l & 255] | lut[3][l >> 8];
        TA acc[4] = {(TA)0, (TA)0, (TA)0, (TA)0};
        for (uint32_t s = 0; s < ns; ++s) {
          const float4 a4 = __ldcg(reinterpret_cast<const float4 *>(A + (bA | lut[4][s])));
          const TA b = (TA)ldcg(B + (bB | lut[5][s])) * sb;
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
      task_maxmin<TO>(ws, nd, tmax, tmin, red);
      return;
    }
  }
  for (uint32_t l = threadIdx.x; l < n_loc; l += blockDim.x) {
    const uint64_t o = o0 + l;
    const uint32_t bA = baseA | lut[0][l & 255] | lut[1][l >> 8];
    const uint32_t bB = baseB | lut[2][l & 255] | lut[3][l >> 8];
    TA acc = (TA)0;
    if (nd.k <= 8) {
      for (uint32_t s = 0; s < ns; ++s) {
        const TA a = (TA)ldcg(A + (bA | lut[4][s])) * sa;
        const TA b = (TA)ldcg(B + (bB | lut[5][s])) * sb;
        acc = dev::fma_t(a, b, acc);
      }
    } else {
      for (uint32_t hi = 0; hi < (ns >> 8); ++hi) {
        const uint32_t hA = bA | lut[6][hi & 255] | lut[8][hi >> 8];
        const uint32_t hB = bB | lut[7][hi & 255] | lut[9][hi >> 8];
        TA part = (TA)0;
        for (uint32_t lo = 0; lo < 256; ++lo) {
          const TA a = (TA)ldcg(A + (hA | lut[4][lo])) * sa;
          const TA b = (TA)ldcg(B + (hB | lut[5][lo])) * sb;
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
  task_maxmin<TO>(ws, nd, tmax, tmin, red);
}

// One task of a node in the generic or the stream mode.
__device__ __forceinline__ void run_one(const BatchArgs &ba, const BNode &nd, int chunk, uint32_t (*lut)[256],
                                        const StreamGeom &geom, double *s_S, unsigned long long *red) {
  float *s_Sf = reinterpret_cast<float *>(s_S);
  if (nd.stream && nd.ti == 1) {
    if (nd.bglob) {
      if (nd.k == 0) run_stream<double, 1, true>(ba, nd, chunk, geom, s_S, red);
      else if (nd.k == 1) run_stream<double, 2, true>(ba, nd, chunk, geom, s_S, red);
      else run_stream<double, 4, true>(ba, nd, chunk, geom, s_S, red);
    }
    else if (nd.k == 0) run_stream<double, 1, false>(ba, nd, chunk, geom, s_S, red);
    else if (nd.k == 1) run_stream<double, 2, false>(ba, nd, chunk, geom, s_S, red);
    else run_stream<double, 4, false>(ba, nd, chunk, geom, s_S, red);
  } else if (nd.stream) {
    if (nd.bglob) {
      if (nd.k == 0) run_stream<float, 1, true>(ba, nd, chunk, geom, s_Sf, red);
      else if (nd.k == 1) run_stream<float, 2, true>(ba, nd, chunk, geom, s_Sf, red);
      else run_stream<float, 4, true>(ba, nd, chunk, geom, s_Sf, red);
    }
    else if (nd.k == 0) run_stream<float, 1, false>(ba, nd, chunk, geom, s_Sf, red);
    else if (nd.k == 1) run_stream<float, 2, false>(ba, nd, chunk, geom, s_Sf, red);
    else run_stream<float, 4, false>(ba, nd, chunk, geom, s_Sf, red);
  }
  else if (nd.ti == 1) run_task<double, double, double>(ba, nd, chunk, lut, red);
  else if (nd.to == 1) run_task<float, double, double>(ba, nd, chunk, lut, red);
  else if (nd.ta == 1) run_task<float, double, float>(ba, nd, chunk, lut, red);
  else run_task<float, float, float>(ba, nd, chunk, lut, red);
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kTabBytes = cmax(cmax(sizeof(StreamGeom), kLutRows * 256 * 4), sizeof(ChainGeom));

__global__ void __launch_bounds__(kBThreads, kBlocksPerSM) k6_persistent(BatchArgs ba) {
  // a node's tables: the generic path's lookup rows or the stream mode's
  // geometry, and the stream mode's staged S
  __shared__ __align__(16) unsigned char s_tab[kTabBytes];
  __shared__ __align__(16) double s_S[4 * kSMaxS];  // S (stream mode), S_1..S_4 (chain mode)
  uint32_t (*lut)[256] = reinterpret_cast<uint32_t (*)[256]>(s_tab);
  StreamGeom &geom = *reinterpret_cast<StreamGeom *>(s_tab);
  ChainGeom &cgeom = *reinterpret_cast<ChainGeom *>(s_tab);
  __shared__ RowScratch s_rows;
  __shared__ unsigned long long red[2];
  __shared__ int s_task, s_ok;
  int lut_node = -1;  // node whose tables the block holds
  for (;;) {
    if (threadIdx.x == 0) s_task = (int)atomicAdd(ba.next, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= ba.n_tasks) break;
    const BTask task = ba.tasks[t];
    const BNode &nd = ba.nodes[task.node];
    if (task.node != lut_node && nd.stream != 3) {  // overlaps the wait for the previous node
      if (nd.stream == 2) chain_geom(nd, ba.chains[nd.chain], cgeom, s_rows);
      else if (nd.stream) stream_geom(nd, geom, s_rows);
      else batch_lut(nd, lut, s_rows);
      lut_node = task.node;
    }
    if (threadIdx.x == 0) {
      bool ok = *(volatile uint32_t *)ba.err == 0;
      if (ok && nd.prev >= 0) ok = wait_count(ba.done + nd.prev, (uint32_t)ba.nodes[nd.prev].n_tasks);
      if (!ok) atomicOr(ba.err, 1u);
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (nd.stream == 2) {
      if (nd.ti == 1) chain_dispatch<double>(ba, nd, ba.chains[nd.chain], task.chunk, cgeom, s_S, red);
      else chain_dispatch<float>(ba, nd, ba.chains[nd.chain], task.chunk, cgeom, reinterpret_cast<float *>(s_S), red);
    } else if (nd.stream == 3) {
      // one small subtree: its nodes in turn, each over all its outputs
      const BGroup grp = ba.groups[nd.chain + task.chunk];
      for (int m = 0; m < grp.n; ++m) {
        const BNode &mn = ba.members[grp.first + m];
        if (mn.stream) stream_geom(mn, geom, s_rows);
        else batch_lut(mn, lut, s_rows);
        run_one(ba, mn, 0, lut, geom, s_S, red);
        __syncthreads();  // outputs and metadata before the next member; tables free
      }
      lut_node = -1;
    } else {
      run_one(ba, nd, task.chunk, lut, geom, s_S, red);
    }
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
  std::vector<BChain> chains;
  std::vector<BGroup> groups;
  std::vector<BNode> members;      // the groups' nodes
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
  BChain *d_chains = nullptr;
  BGroup *d_groups = nullptr;
  BNode *d_members = nullptr;
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

// Task size and order of batches created after wmc_set_batch_schedule.
static std::atomic<int32_t> g_batch_chunk{14};  // log2 outputs (stream mode: u) per task
static std::atomic<int32_t> g_batch_order{0};   // 0 list scheduling, 1 round-robin

// Longest chain of frontier steps run as one pass (0: none).
static std::atomic<int32_t> g_batch_fuse{4};

// Largest output rank of a node that runs inside a small-subtree task (0: none).
static std::atomic<int32_t> g_batch_sub{12};

extern "C" void wmc_set_batch_subtrees(int32_t max_rank) {
  g_batch_sub.store(max_rank <= 0 ? 0 : std::min(14, max_rank));
}

extern "C" void wmc_set_batch_fusion(int32_t max_steps) {
  g_batch_fuse.store(max_steps < 2 ? 0 : std::min(4, max_steps));
}

extern "C" void wmc_set_batch_schedule(int32_t chunk_log2, int32_t order) {
  g_batch_chunk.store(chunk_log2 <= 0 ? 14 : std::min(16, std::max(8, chunk_log2)));
  g_batch_order.store(order == 1 ? 1 : 0);
}

namespace {

// Estimated microseconds of one task (cost model of the list scheduling):
// a fixed part (counter, tables, epilogue) and a rate per element moved,
// as measured per block with every block of the persistent kernel busy
// (4 per SM; float32, 512-formula batch): chains 0.53 ns per element
// (2^D loads and up to 2^(D+1) stores per unit), stream mode 0.62 ns (2^k
// loads and 2^f stores per unit), the generic path 1.1 ns per output and
// summed term, small subtrees 5.5 us per node.
double task_us(const BNode &n) {
  const double el = n.ti ? 2.0 : 1.0;  // element size in float32 units
  if (n.stream == 3) return n.est_us;
  const double units = std::ldexp(1.0, n.chunk_log2);
  if (n.stream == 2) return 2.0 + 0.00053 * el * units * (std::ldexp(1.0, n.k) + std::ldexp(1.0, n.f));
  if (n.stream) return 2.0 + 0.00062 * el * units * (std::ldexp(1.0, n.k) + std::ldexp(1.0, n.f));
  return 2.0 + 0.0011 * el * units * (1.0 + std::ldexp(1.0, n.k));
}

int pos_in(const std::vector<int32_t> &L, int32_t v) {
  for (size_t i = 0; i < L.size(); ++i)
    if (L[i] == v) return (int)i;
  return -1;
}

// A frontier step R . S -> C: one summed index x, an index of R (the
// running tensor), at most two added indices y, z (-1: none), S of rank
// <= 8.
bool frontier_step(const std::vector<int32_t> &LR, const std::vector<int32_t> &LS, const std::vector<int32_t> &LC,
                   int32_t &x, int32_t &y, int32_t &z) {
  if (LS.size() > 8) return false;
  int n_sum = 0, n_add = 0;
  x = y = z = -1;
  for (int32_t l : LR)
    if (pos_in(LC, l) < 0) { ++n_sum; x = l; }
  for (int32_t l : LS)
    if (pos_in(LC, l) < 0 && pos_in(LR, l) < 0) ++n_sum;
  for (int32_t l : LC)
    if (pos_in(LR, l) < 0) { (n_add == 0 ? y : z) = l; ++n_add; }
  return n_sum == 1 && x >= 0 && n_add <= 2;
}

// A chain of one formula (chain mode): its nodes n_1..n_D in order, the
// first operand A_1, S_i, and the summed and added index of each step.
struct ChainSpec {
  std::vector<int64_t> nodes, s;
  std::vector<int32_t> x, y;  // y = -1: the step adds none (shrink; last only)
  int32_t z = -1;             // second index the first step adds (growth chains)
  int64_t a1 = -1;
};

// Chains of consecutive frontier steps (Algorithm 2's post-order, the
// output of each step the running operand of the next), at most max_d
// steps each: the first step adds one index, or two (a growth chain, then
// at most 3 steps and no shrink), the others one or none (a step adding
// none ends the chain), every x_i is an index of A_1 that no earlier S
// holds, and the indices added so far (in the order y_0, z, y_1, ...) that
// S_i holds are among the two added last.
// Nodes of small subtrees (they run in subtree tasks) take no part.
// chain_at[n] = the chain node n starts (-1: none); absorbed[n] = 1 for the
// other members, 2 for the other nodes that run before their chain (of the
// subtrees of S_2..S_D, between n_1 and n_D in post-order).
void find_chains(const Plan &plan, const std::vector<uint8_t> &t_dbl, bool f64, int max_d,
                 const std::vector<uint8_t> &small, std::vector<ChainSpec> &chains, std::vector<int32_t> &chain_at,
                 std::vector<uint8_t> &absorbed) {
  const size_t nn = plan.nodes.size();
  chain_at.assign(nn, -1);
  absorbed.assign(nn, 0);
  if (max_d < 2) return;
  auto L = [&](int64_t t) -> const std::vector<int32_t> & { return plan.tensors[(size_t)t].labels; };
  std::vector<int64_t> consumer(plan.tensors.size(), -1);
  for (size_t ni = 0; ni < nn; ++ni) {
    consumer[(size_t)plan.nodes[ni].a] = (int64_t)ni;
    consumer[(size_t)plan.nodes[ni].b] = (int64_t)ni;
  }
  // float32 plans keep the float64 root out of chains
  auto typed = [&](int64_t c) { return f64 || !t_dbl[(size_t)c]; };
  for (size_t ni = 0; ni < nn; ++ni) {
    if (absorbed[ni] || small[ni]) continue;
    const Node &n0 = plan.nodes[ni];
    int64_t r = n0.a, sid = n0.b;
    if (L(sid).size() > L(r).size()) std::swap(r, sid);
    int32_t x, y, z;
    if (!typed(n0.c) || !frontier_step(L(r), L(sid), L(n0.c), x, y, z) || y < 0) continue;
    ChainSpec cs;
    cs.a1 = r;
    cs.z = z;
    cs.nodes.push_back((int64_t)ni);
    cs.s.push_back(sid);
    cs.x.push_back(x);
    cs.y.push_back(y);
    std::vector<int32_t> added{y};
    if (z >= 0) added.push_back(z);
    const int cap = z >= 0 ? std::min(max_d, 3) : max_d;
    while ((int)cs.nodes.size() < cap && cs.y.back() >= 0) {
      const int64_t last = cs.nodes.back();
      const int64_t cprev = plan.nodes[(size_t)last].c;
      const int64_t nj = consumer[(size_t)cprev];
      if (nj < 0 || absorbed[(size_t)nj] || small[(size_t)nj]) break;
      const Node &nd = plan.nodes[(size_t)nj];
      const int64_t sj = nd.a == cprev ? nd.b : nd.a;
      int32_t xj, yj, zj;
      if (!typed(nd.c) || !frontier_step(L(cprev), L(sj), L(nd.c), xj, yj, zj) || zj >= 0) break;
      if (pos_in(L(r), xj) < 0 || (cs.z >= 0 && yj < 0)) break;
      const size_t j = cs.nodes.size();
      bool ok = true;
      for (size_t i = 0; i < j && ok; ++i) ok = pos_in(L(cs.s[i]), xj) < 0;
      for (size_t i = 0; i + 2 < added.size() && ok; ++i) ok = pos_in(L(sj), added[i]) < 0;
      for (int64_t q = last + 1; q < nj && ok; ++q) ok = !absorbed[(size_t)q] && chain_at[(size_t)q] < 0;
      if (!ok) break;
      cs.nodes.push_back(nj);
      cs.s.push_back(sj);
      cs.x.push_back(xj);
      cs.y.push_back(yj);
      if (yj >= 0) added.push_back(yj);
    }
    if (cs.nodes.size() < 2) continue;
    const int64_t last = cs.nodes.back();
    for (size_t i = 1; i < cs.nodes.size(); ++i) absorbed[(size_t)cs.nodes[i]] = 1;
    for (int64_t q = (int64_t)ni + 1; q < last; ++q)
      if (!absorbed[(size_t)q] && !small[(size_t)q]) absorbed[(size_t)q] = 2;
    chain_at[ni] = (int32_t)chains.size();
    chains.push_back(std::move(cs));
  }
}

// List scheduling of the formulas' node chains onto `slots` resident
// blocks: whenever a simulated block frees, it takes the next task of the
// ready node whose formula has the largest bottom level (the estimated time
// of its remaining chain); a node becomes ready `dep_us` after the last of
// its predecessor's tasks finishes.  Tasks are listed in the order they are
// taken.
void list_schedule(const std::vector<BNode> &nodes, const std::vector<std::vector<int32_t>> &chains,
                   int32_t slots, double dep_us, std::vector<BTask> &tasks) {
  const size_t F = chains.size();
  std::vector<std::vector<double>> bottom(F);
  for (size_t f = 0; f < F; ++f) {
    const auto &c = chains[f];
    bottom[f].assign(c.size(), 0.0);
    double acc = 0.0;
    for (size_t j = c.size(); j-- > 0;) {
      acc += task_us(nodes[(size_t)c[j]]) + dep_us;
      bottom[f][j] = acc;
    }
  }
  std::vector<size_t> cur(F, 0);
  std::vector<int32_t> left(F, 0);
  std::vector<double> fin(F, 0.0);
  typedef std::pair<double, int64_t> Item;  // (key, formula)
  std::priority_queue<Item> ready;           // largest bottom level first
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> waiting;  // earliest ready time
  std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
  for (int32_t i = 0; i < slots; ++i) free_at.push(0.0);
  for (size_t f = 0; f < F; ++f)
    if (!chains[f].empty()) {
      left[f] = nodes[(size_t)chains[f][0]].n_tasks;
      ready.push({bottom[f][0], (int64_t)f});
    }
  while (!ready.empty() || !waiting.empty()) {
    double t = free_at.top();
    free_at.pop();
    while (!waiting.empty() && waiting.top().first <= t) {
      const int64_t f = waiting.top().second;
      waiting.pop();
      ready.push({bottom[(size_t)f][cur[(size_t)f]], f});
    }
    if (ready.empty()) {  // the block idles until the earliest node is ready
      t = std::max(t, waiting.top().first);
      const int64_t f = waiting.top().second;
      waiting.pop();
      ready.push({bottom[(size_t)f][cur[(size_t)f]], f});
    }
    const size_t f = (size_t)ready.top().second;
    const int32_t node = chains[f][cur[f]];
    const BNode &n = nodes[(size_t)node];
    const double end = t + task_us(n);
    tasks.push_back({node, n.n_tasks - left[f]});
    free_at.push(end);
    fin[f] = std::max(fin[f], end);
    if (--left[f] == 0) {
      ready.pop();
      if (++cur[f] < chains[f].size()) {
        left[f] = nodes[(size_t)chains[f][cur[f]]].n_tasks;
        waiting.push({fin[f] + dep_us, (int64_t)f});
        fin[f] = 0.0;
      }
    }
  }
}

}  // namespace

extern "C" int wmc_batch_create(wmc_plan_t *const *plans, int32_t n_plans, int64_t mem_budget_bytes,
                                wmc_batch_t **out, int32_t *n_admitted) {
  if (!plans || !out || n_plans < 1) { set_error("bad argument"); return WMC_EINVAL; }
  *out = nullptr;
  wmc_batch *b = new (std::nothrow) wmc_batch();
  if (!b) { set_error("out of host memory"); return WMC_ENOMEM; }
  const int32_t prec = plan_of(plans[0]).precision;
  b->precision = prec;
  const int32_t chunk_log2 = g_batch_chunk.load();
  int64_t off = 0;
  std::vector<std::vector<int32_t>> node_ids;  // per formula: global node ids in post-order
  for (int32_t f = 0; f < n_plans; ++f) {
    Plan &plan = plan_of(plans[f]);
    if (plan.precision != prec) { delete b; set_error("plans of one batch must share a precision"); return WMC_EINVAL; }
    if (!plan.slice_vars.empty()) { delete b; set_error("sliced plans run through wmc_execute, not a batch"); return WMC_EINVAL; }
    if (plan.bfp_b >= 0) { delete b; set_error("block-floating-point plans run through wmc_execute, not a batch"); return WMC_EINVAL; }
    LayoutView lv;
    int rc = exec_layout(plan, 1, &lv);
    if (rc) { delete b; return rc; }
    const std::vector<int64_t> &tb = *lv.t_bytes;
    auto lab = [&](int64_t t) -> const std::vector<int32_t> & { return plan.tensors[(size_t)t].labels; };
    const size_t nn = plan.nodes.size();
    auto node_of = [&](int64_t t) { return (size_t)plan.tensors[(size_t)t].node; };
    // small subtrees: nodes of output rank <= g_batch_sub with at most 2^8
    // summed terms whose children are leaves or such nodes (never the
    // root); each maximal one runs as one task, all of a formula's such
    // tasks before its other nodes
    std::vector<uint8_t> small(nn, 0);
    const int32_t sub_rank = g_batch_sub.load();
    if (sub_rank > 0)
      for (size_t ni = 0; ni + 1 < nn; ++ni) {
        const Node &nd = plan.nodes[ni];
        bool ok = (int32_t)lab(nd.c).size() <= sub_rank && nd.n_summed <= 8;
        for (int64_t ch : {nd.a, nd.b})
          if (ch >= plan.n_leaves && !small[node_of(ch)]) ok = false;
        small[ni] = ok ? 1 : 0;
      }
    // each maximal small subtree's nodes, in the plan's order (children
    // first); the node list is topologically ordered, so a subtree need not
    // be contiguous in it
    std::vector<std::vector<int64_t>> groups;
    {
      std::vector<int64_t> consumer(plan.tensors.size(), -1), stack;
      for (size_t ni = 0; ni < nn; ++ni) {
        consumer[(size_t)plan.nodes[ni].a] = (int64_t)ni;
        consumer[(size_t)plan.nodes[ni].b] = (int64_t)ni;
      }
      for (size_t ni = 0; ni < nn; ++ni) {
        if (!small[ni]) continue;
        const int64_t cons = consumer[(size_t)plan.nodes[ni].c];
        if (cons >= 0 && small[(size_t)cons]) continue;  // not a subtree's root
        std::vector<int64_t> g;
        stack.assign(1, (int64_t)ni);
        while (!stack.empty()) {
          const int64_t q = stack.back();
          stack.pop_back();
          g.push_back(q);
          for (int64_t ch : {plan.nodes[(size_t)q].a, plan.nodes[(size_t)q].b})
            if (ch >= plan.n_leaves) stack.push_back((int64_t)node_of(ch));
        }
        std::sort(g.begin(), g.end());
        groups.push_back(std::move(g));
      }
    }
    // chains, and the execution order of the other nodes: a chain's
    // S_2..S_D subtrees run before its first step
    std::vector<ChainSpec> specs;
    std::vector<int32_t> chain_at;
    std::vector<uint8_t> absorbed;
    find_chains(plan, *lv.t_dbl, prec == WMC_FP64, g_batch_fuse.load(), small, specs, chain_at, absorbed);
    std::vector<int64_t> order;
    for (size_t ni = 0; ni < nn; ++ni) {
      if (absorbed[ni] || small[ni]) continue;
      if (chain_at[ni] >= 0)
        for (int64_t q = (int64_t)ni + 1; q < specs[(size_t)chain_at[ni]].nodes.back(); ++q)
          if (absorbed[(size_t)q] == 2) order.push_back(q);
      order.push_back((int64_t)ni);
    }
    // layout: the small subtrees' outputs side by side after the leaves
    // (64-byte aligned, never reused), then the other intermediates' arena,
    // first fit in execution order (a chain's inner outputs are never
    // stored); leaves and metadata as in the plan's layout
    std::vector<int64_t> t_off(*lv.t_off);
    int64_t gtop = lv.arena0;
    for (const auto &g : groups)
      for (int64_t m : g) {
        const int64_t c = plan.nodes[(size_t)m].c;
        t_off[(size_t)c] = gtop;
        gtop += (tb[(size_t)c] + 63) / 64 * 64;
      }
    const int64_t arena1 = align_up(gtop);
    FirstFit ff;
    auto in_arena = [&](int64_t t) { return t >= plan.n_leaves && !small[node_of(t)]; };
    auto release = [&](int64_t t) {
      if (in_arena(t)) ff.release(t_off[(size_t)t] - arena1, tb[(size_t)t]);
    };
    for (int64_t ni : order) {
      const Node &nd = plan.nodes[(size_t)ni];
      if (chain_at[(size_t)ni] >= 0) {
        const ChainSpec &cs = specs[(size_t)chain_at[(size_t)ni]];
        const int64_t cD = plan.nodes[(size_t)cs.nodes.back()].c;
        t_off[(size_t)cD] = arena1 + ff.alloc(tb[(size_t)cD]);
        release(cs.a1);
        for (int64_t sid : cs.s) release(sid);
      } else {
        t_off[(size_t)nd.c] = arena1 + ff.alloc(tb[(size_t)nd.c]);
        release(nd.a);
        release(nd.b);
      }
    }
    // replay of the order: every arena operand is live when read (an
    // output not yet consumed; leaves and subtree outputs stay) and no
    // output overlaps a live tensor or leaves the arena
    {
      std::map<int64_t, int64_t> live;  // tensor -> its arena block's end
      bool ok = true;
      auto use = [&](int64_t t) {
        if (in_arena(t)) ok = ok && live.erase(t) == 1;
      };
      for (int64_t ni : order) {
        const Node &nd = plan.nodes[(size_t)ni];
        int64_t c = nd.c;
        std::vector<int64_t> in{nd.a, nd.b};
        if (chain_at[(size_t)ni] >= 0) {
          const ChainSpec &cs = specs[(size_t)chain_at[(size_t)ni]];
          c = plan.nodes[(size_t)cs.nodes.back()].c;
          in.assign(cs.s.begin(), cs.s.end());
          in.push_back(cs.a1);
        }
        const int64_t c0 = t_off[(size_t)c], c1 = c0 + align_up(tb[(size_t)c]);
        ok = ok && c0 >= arena1;
        for (const auto &kv : live) ok = ok && (c1 <= t_off[(size_t)kv.first] || kv.second <= c0);
        for (int64_t t : in) use(t);
        live[c] = c1;
      }
      if (!ok || live.size() != 1 || live.begin()->first != plan.nodes.back().c) {
        delete b;
        set_error("internal: the batch layout of formula %d failed its replay", f);
        return WMC_EPLAN_TOO_BIG;
      }
    }
    const int64_t need = align_up(arena1 + align_up(ff.top));
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
      L.data = base + t_off[(size_t)i];
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
    // one node in the generic or the stream mode; `whole`: one task over
    // all its outputs (a subtree member)
    auto fill_node = [&](const Node &nd, BNode &n, bool whole) -> bool {
      std::memset(&n, 0, sizeof(n));
      n.chain = -1;
      n.a = base + t_off[(size_t)nd.a];
      n.b = base + t_off[(size_t)nd.b];
      n.c = base + t_off[(size_t)nd.c];
      n.ea = slot(lv.off_exp, nd.a); n.eb = slot(lv.off_exp, nd.b); n.ec = slot(lv.off_exp, nd.c);
      n.xa = slot(lv.off_max, nd.a); n.xb = slot(lv.off_max, nd.b); n.xc = slot(lv.off_max, nd.c);
      n.na = slot(lv.off_min, nd.a); n.nb = slot(lv.off_min, nd.b); n.nc = slot(lv.off_min, nd.c);
      n.flags = base + lv.off_flags;
      k1_bitmaps(qlabels(plan.tensors[(size_t)nd.a]), qlabels(plan.tensors[(size_t)nd.b]),
                 qlabels(plan.tensors[(size_t)nd.c]), &n.rC, &n.k, n.posA, n.posB, n.sposA, n.sposB);
      if (n.k > 24 || n.rC > 31) return false;
      int32_t ra = (int32_t)plan.tensors[(size_t)nd.a].labels.size();
      int32_t rb = (int32_t)plan.tensors[(size_t)nd.b].labels.size();
      if (rb > ra) {  // A = the operand with more indices (the product commutes, term by term)
        std::swap(n.a, n.b); std::swap(n.ea, n.eb); std::swap(n.xa, n.xb); std::swap(n.na, n.nb);
        for (int j = 0; j < 32; ++j) std::swap(n.posA[j], n.posB[j]);
        for (int j = 0; j < 24; ++j) std::swap(n.sposA[j], n.sposB[j]);
        std::swap(ra, rb);
      }
      n.rB = (int8_t)rb;
      n.ti = prec == WMC_FP64 ? 1 : 0;
      n.to = (*lv.t_dbl)[(size_t)nd.c];
      n.ta = (prec == WMC_FP64 || n.to || n.k > 16) ? 1 : 0;
      int32_t fr = 0;
      for (int j = 0; j < n.rC; ++j) fr += n.posA[j] < 0;
      // (a B of rank 9..22 -- at most 16 MB in float32 -- is read from L2
      // instead of staged: joins whose B-only indices are few)
      const bool b_l2 = rb > 8 && (int64_t(1) << rb) * (n.ti ? 8 : 4) <= (int64_t(16) << 20);
      n.stream = (n.ti == n.ta && n.ta == n.to && n.k <= 2 && (rb <= 8 || b_l2) && fr <= 4) ? 1 : 0;
      n.bglob = (n.stream && rb > 8) ? 1 : 0;
      if (n.stream) {
        // tasks over u, the assignments of C's indices that A holds
        n.f = (int8_t)fr;
        n.chunk_log2 = whole ? n.rC - fr : std::min<int32_t>(n.rC - fr, chunk_log2);
        n.n_tasks = 1 << (n.rC - fr - n.chunk_log2);
        n.vec4 = (!n.ti && n.chunk_log2 >= 3 && n.rC >= 2 && n.posA[0] == 0 && n.posA[1] == 1) ? 1 : 0;
      } else {
        n.chunk_log2 = whole ? n.rC : std::min<int32_t>(n.rC, chunk_log2);
        n.n_tasks = 1 << (n.rC - n.chunk_log2);
        bool low = n.rC >= n.chunk_log2 && n.chunk_log2 >= 2 && n.posA[0] == 0 && n.posA[1] == 1 &&
                   n.posB[0] < 0 && n.posB[1] < 0;
        for (int j = 0; j < n.k && low; ++j) low = n.sposA[j] >= 2;
        n.vec4 = (low && !n.ti && !n.ta && !n.to) ? 1 : 0;
      }
      b->alg_bytes += (double)tb[(size_t)nd.a] + (double)tb[(size_t)nd.b] + (double)tb[(size_t)nd.c];
      return true;
    };
    std::vector<int32_t> ids;
    int32_t prev = -1;
    if (!groups.empty()) {
      // every small subtree of the formula: one task each, no waits
      BNode g;
      std::memset(&g, 0, sizeof(g));
      g.stream = 3;
      g.prev = -1;
      g.chain = (int32_t)b->groups.size();
      g.n_tasks = (int32_t)groups.size();
      int64_t n_members = 0;
      for (const auto &gr : groups) {
        b->groups.push_back({(int32_t)b->members.size(), (int32_t)gr.size()});
        for (int64_t m : gr) {
          BNode mn;
          if (!fill_node(plan.nodes[(size_t)m], mn, true)) {
            delete b;
            set_error("node too large for the batch executor");
            return WMC_EPLAN_TOO_BIG;
          }
          b->members.push_back(mn);
        }
        n_members += (int64_t)gr.size();
      }
      if (b->members.size() > (size_t)INT32_MAX) { delete b; set_error("batch has more than 2^31 subtree nodes"); return WMC_EPLAN_TOO_BIG; }
      g.est_us = (float)(2.0 + 5.5 * (double)n_members / (double)groups.size());
      prev = (int32_t)b->nodes.size();
      ids.push_back(prev);
      b->nodes.push_back(g);
    }
    // the other nodes, in execution order (the first waits for the subtrees)
    for (int64_t ni : order) {
      const Node &nd = plan.nodes[(size_t)ni];
      BNode n;
      if (chain_at[(size_t)ni] >= 0) {
        std::memset(&n, 0, sizeof(n));
        const ChainSpec &cs = specs[(size_t)chain_at[(size_t)ni]];
        const int D = (int)cs.nodes.size();
        const int64_t cD = plan.nodes[(size_t)cs.nodes.back()].c;
        const std::vector<int32_t> &LA = lab(cs.a1), &LC = lab(cD);
        BChain ch;
        std::memset(&ch, 0xff, sizeof(ch));  // positions: -1 = none
        ch.D = (int8_t)D;
        ch.shrink = cs.y.back() < 0 ? 1 : 0;
        ch.grow = cs.z >= 0 ? 1 : 0;
        ch.zc = ch.grow ? (int8_t)pos_in(LC, cs.z) : (int8_t)-1;
        int nu = 0;
        for (size_t j = 0; j < LC.size(); ++j) {
          const int pa = pos_in(LA, LC[j]);
          if (pa < 0) continue;  // an added index
          ch.ua[nu] = (int8_t)pa;
          ch.uc[nu] = (int8_t)j;
          for (int i = 0; i < D; ++i) ch.us[i][nu] = (int8_t)pos_in(lab(cs.s[(size_t)i]), LC[j]);
          ++nu;
        }
        ch.nu = (int8_t)nu;
        if (nu + D != (int)LA.size() || (int)LC.size() != nu + D - ch.shrink + ch.grow) {
          delete b;
          set_error("internal: chain geometry does not add up");
          return WMC_EPLAN_TOO_BIG;
        }
        for (int i = 0; i < D; ++i) {
          const int64_t sid = cs.s[(size_t)i];
          const std::vector<int32_t> &LS = lab(sid);
          ch.s[i] = base + t_off[(size_t)sid];
          ch.es[i] = slot(lv.off_exp, sid);
          ch.xs[i] = slot(lv.off_max, sid);
          ch.ns[i] = slot(lv.off_min, sid);
          ch.rs[i] = (int8_t)LS.size();
          ch.xa[i] = (int8_t)pos_in(LA, cs.x[(size_t)i]);
          ch.yc[i] = cs.y[(size_t)i] >= 0 ? (int8_t)pos_in(LC, cs.y[(size_t)i]) : (int8_t)-1;
          ch.sx[i] = (int8_t)pos_in(LS, cs.x[(size_t)i]);
          ch.sy[i] = cs.y[(size_t)i] >= 0 ? (int8_t)pos_in(LS, cs.y[(size_t)i]) : (int8_t)-1;
          // the indices behind the state bits the step's S may depend on
          // (at a growth step: z)
          auto label_of_bit = [&](int bit) { return bit < 0 ? -1 : (bit == D ? cs.z : cs.y[(size_t)bit]); };
          const int b1 = added_bit(D, ch.grow != 0, i, 0), b2 = added_bit(D, ch.grow != 0, i, 1);
          const int32_t l1 = (ch.grow && i == 0) ? cs.z : label_of_bit(b1), l2 = label_of_bit(b2);
          ch.s1[i] = l1 >= 0 ? (int8_t)pos_in(LS, l1) : (int8_t)-1;
          ch.s2[i] = l2 >= 0 ? (int8_t)pos_in(LS, l2) : (int8_t)-1;
          b->alg_bytes += (double)tb[(size_t)sid];
        }
        n.a = base + t_off[(size_t)cs.a1];
        n.ea = slot(lv.off_exp, cs.a1); n.xa = slot(lv.off_max, cs.a1); n.na = slot(lv.off_min, cs.a1);
        n.b = ch.s[0]; n.eb = ch.es[0]; n.xb = ch.xs[0]; n.nb = ch.ns[0];
        n.c = base + t_off[(size_t)cD];
        n.ec = slot(lv.off_exp, cD); n.xc = slot(lv.off_max, cD); n.nc = slot(lv.off_min, cD);
        n.flags = base + lv.off_flags;
        n.rC = (int32_t)LC.size();
        n.k = D;                        // 2^D loads per unit
        n.f = (int8_t)(D + ch.grow - ch.shrink);  // 2^f stores per unit
        n.stream = 2;
        n.ti = n.ta = n.to = prec == WMC_FP64 ? 1 : 0;
        // a unit moves 2^D values in and up to 2^D out (four times a
        // stream-mode unit at D = 2): tasks of a quarter as many units
        n.chunk_log2 = std::min<int32_t>(nu, std::max<int32_t>(8, chunk_log2 - 2));
        n.n_tasks = 1 << (nu - n.chunk_log2);
        n.chain = (int32_t)b->chains.size();
        b->chains.push_back(ch);
        b->alg_bytes += (double)tb[(size_t)cs.a1] + (double)tb[(size_t)cD];
      } else if (!fill_node(nd, n, false)) {
        delete b;
        set_error("node too large for the batch executor");
        return WMC_EPLAN_TOO_BIG;
      }
      n.prev = prev;
      prev = (int32_t)b->nodes.size();
      ids.push_back(prev);
      b->nodes.push_back(n);
    }
    node_ids.push_back(ids);
    const int64_t root = plan.nodes.back().c;
    b->roots.push_back({base + t_off[(size_t)root], slot(lv.off_exp, root), base + lv.off_flags});
    b->max_roundings = std::max(b->max_roundings, plan.tensors[(size_t)root].roundings);
  }
  if (b->plans.empty()) { delete b; set_error("no formula fits the memory budget"); return WMC_EPLAN_TOO_BIG; }
  b->ws_bytes = off;
  // tasks: list scheduling onto the resident blocks (4 per SM on 148 SMs;
  // the order stays valid for any block count), or round-robin over the
  // formulas, each formula in post-order
  int64_t n_tasks = 0;
  for (const BNode &n : b->nodes) n_tasks += n.n_tasks;
  if (n_tasks > INT32_MAX) { delete b; set_error("batch has more than 2^31 tasks"); return WMC_EPLAN_TOO_BIG; }
  b->tasks.reserve((size_t)n_tasks);
  if (g_batch_order.load() == 0) {
    list_schedule(b->nodes, node_ids, 148 * kBlocksPerSM, 2.0, b->tasks);
  } else {
    size_t longest = 0;
    for (auto &v : node_ids) longest = std::max(longest, v.size());
    for (size_t r = 0; r < longest; ++r)
      for (auto &v : node_ids)
        if (r < v.size()) {
          const BNode &n = b->nodes[(size_t)v[r]];
          for (int32_t c = 0; c < n.n_tasks; ++c) b->tasks.push_back({v[r], c});
        }
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
  const int64_t o_chains = o; o += al(sizeof(BChain) * (int64_t)b->chains.size());
  const int64_t o_groups = o; o += al(sizeof(BGroup) * (int64_t)b->groups.size());
  const int64_t o_members = o; o += al(sizeof(BNode) * (int64_t)b->members.size());
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
  b->d_chains = (BChain *)(t + o_chains);
  b->d_groups = (BGroup *)(t + o_groups);
  b->d_members = (BNode *)(t + o_members);
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
      up(b->d_chains, b->chains.data(), sizeof(BChain) * b->chains.size()) ||
      up(b->d_groups, b->groups.data(), sizeof(BGroup) * b->groups.size()) ||
      up(b->d_members, b->members.data(), sizeof(BNode) * b->members.size()) ||
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
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k6_persistent, kBThreads, 0);
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
  a.chains = b->d_chains;
  a.groups = b->d_groups;
  a.members = b->d_members;
  a.tasks = b->d_tasks;
  a.n_tasks = (int32_t)b->tasks.size();
  a.next = b->d_next;
  a.done = b->d_done;
  a.err = b->d_err;
  k6_persistent<<<(unsigned)b->grid, kBThreads, 0, s>>>(a);
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
