// Device kernels of the WMC execution stage (sm_103a).
//
// Every contraction node computes, for the two-tensor network {A, B}
// (Eq. (1), Sec. 2.3),
//
//     C[o] = sum_{s in {0,1}^k} A[offA(o, s)] * B[offB(o, s)]
//
// where o enumerates the indices of C and s the summed indices; offA/offB
// scatter the index bits into each operand's own bit order, so the permute
// of the "permute + batched GEMM" view (Sec. 4.2) is folded into the
// addressing and never materialised.  Tensors are stored as mantissas with
// a power-of-two exponent per (tensor, query): true = mant * 2^exp.  A
// consumer rescales each operand on load by 2^-E, E = floor(log2 max|mant|)
// (exact: a power of two), and the producer records max|C| with an atomic
// max on the IEEE bit pattern (valid for nonnegative values, which is what
// |x| is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dev_common.cuh"

namespace wmc {
namespace dev {

// Per-operand metadata, one entry per query if the tensor carries the
// query index (qmask = Qp-1), else one: the exponent, and the IEEE bit
// patterns of max|x| and of the smallest nonzero |x| (all-ones: none).
struct Meta {
  const int64_t *exp;
  const unsigned long long *maxb;
  const unsigned long long *minb;
  int32_t qmask;
};

struct OutMeta {
  int64_t *exp;
  unsigned long long *maxb;
  unsigned long long *minb;
  uint32_t *flags;       // per query lane
  int32_t Qc;            // entries of C's metadata (Qp or 1)
  int32_t Q;             // query lanes (flags entries)
  int32_t scale_inputs;  // 0: inputs are used as stored (contract_pair)
};


template <typename T>
__device__ __forceinline__ T operand_scale(const Meta &m, int q, int scale_inputs) {
  return scale_inputs ? pow2_scale(pow2_exp_of(m.maxb[q & m.qmask], T()), T()) : (T)1;
}

// Block epilogue: C's exponents (block 0), the per-query max and min of
// |C| (atomics on the bit patterns), and the float32 flush test.  A flush
// is possible only when the smallest nonzero scaled operands' product is
// below the smallest normal number; with nonnegative terms no sum can then
// be below it either, so the test is conservative and complete.
template <typename T>
__device__ __forceinline__ void finish_meta(const Meta &ma, const Meta &mb, const OutMeta &mc,
                                            unsigned long long *smax, unsigned long long *smin) {
  if (blockIdx.x == 0) {
    for (int q = threadIdx.x; q < mc.Qc; q += blockDim.x) {
      const int qa = q & ma.qmask, qb = q & mb.qmask;
      if (mc.exp) {
        int64_t e = 0;
        if (ma.exp) e += ma.exp[qa] + (mc.scale_inputs ? pow2_exp_of(ma.maxb[qa], T()) : 0);
        if (mb.exp) e += mb.exp[qb] + (mc.scale_inputs ? pow2_exp_of(mb.maxb[qb], T()) : 0);
        mc.exp[q] = e;
      }
      if (mc.flags && ma.minb && mb.minb && ma.minb[qa] != kNoMin && mb.minb[qb] != kNoMin) {
        const T lo = (from_bits<T>(ma.minb[qa]) * operand_scale<T>(ma, qa, 1)) *
                     (from_bits<T>(mb.minb[qb]) * operand_scale<T>(mb, qb, 1));
        if (below_normal(lo)) {
          if (mc.Qc > 1) atomicOr(mc.flags + q, 2u);
          else
            for (int qq = 0; qq < mc.Q; ++qq) atomicOr(mc.flags + qq, 2u);
        }
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < mc.Qc; q += blockDim.x) {
    if (mc.maxb && smax[q]) atomicMax(mc.maxb + q, smax[q]);
    if (mc.minb && smin[q] != kNoMin) atomicMin(mc.minb + q, smin[q]);
  }
}

template <typename T>
__device__ __forceinline__ void track(T c, T &tmax, T &tmin) {
  const T a = c < (T)0 ? -c : c;
  tmax = a > tmax ? a : tmax;
  tmin = (a != (T)0 && a < tmin) ? a : tmin;
}
// float64: the same max and min from the bit patterns on the integer units
// (nonnegative IEEE values order as their bits; NaNs are skipped), leaving
// B300's few FP64 units to the products
// (compared as 32-bit halves: high words first, low words on a tie)
template <>
__device__ __forceinline__ void track<double>(double c, double &tmax, double &tmin) {
  const uint32_t ah = (uint32_t)__double2hiint(c) & 0x7fffffffu, al = (uint32_t)__double2loint(c);
  const uint32_t xh = (uint32_t)__double2hiint(tmax), xl = (uint32_t)__double2loint(tmax);
  const uint32_t nh = (uint32_t)__double2hiint(tmin), nl = (uint32_t)__double2loint(tmin);
  const bool finite_or_inf = ah < 0x7ff00000u || (ah == 0x7ff00000u && al == 0u);
  const bool gt = ah > xh || (ah == xh && al > xl);
  const bool lt = ah < nh || (ah == nh && al < nl);
  const bool nz = (ah | al) != 0u;
  if (gt && finite_or_inf) tmax = __hiloint2double((int)ah, (int)al);
  if (lt && nz) tmin = __hiloint2double((int)ah, (int)al);
}

template <typename T>
__device__ __forceinline__ void publish(unsigned long long *smax, unsigned long long *smin, int q,
                                        T tmax, T tmin) {
  if (tmax != (T)0) atomicMax(smax + q, abs_bits(tmax));
  if (tmin != (T)INFINITY) atomicMin(smin + q, abs_bits(tmin));
}

// publish() after folding the max/min of the warp's lanes that share a
// query lane: lanes l and l ^ o hold the same q for every o that is a
// multiple of `period` (1: the whole warp shares one q; Qc <= 32 when
// q = lane mod Qc; >= 32: every lane its own).  Max and min are exact, so
// the result does not depend on the grouping.  All 32 lanes must call it.
template <typename T>
__device__ __forceinline__ void publish_warp(unsigned long long *smax, unsigned long long *smin, int q,
                                             T tmax, T tmin, int period) {
  for (int o = 16; o >= period; o >>= 1) {
    tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
  }
  if ((int)(threadIdx.x & 31u) < period) publish(smax, smin, q, tmax, tmin);
}

// ------------------------------------------------------------ K1 generic

struct K1Params {
  const void *A;
  const void *B;
  void *C;
  Meta ma, mb;
  OutMeta mc;
  int32_t rC;        // bits of C (incl. query bits)
  int32_t k;         // summed bits (<= 24)
  int8_t posA[32];   // C bit j -> bit of A (-1: absent)
  int8_t posB[32];
  int8_t sposA[24];  // summed bit i -> bit of A (-1: absent)
  int8_t sposB[24];
};

// Any bit mapping.  Offsets come from per-byte lookup tables built in
// shared memory.  TI: stored type of A and B; TA: accumulation; TO: stored
// type of C.  The grid-stride step is a multiple of Qc, so each thread
// sees one query for all of its outputs.
template <typename TI, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) k1_generic(K1Params p) {
  __shared__ uint32_t lutA[4][256], lutB[4][256];
  __shared__ uint32_t slutA[3][256], slutB[3][256];
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    int byte = i >> 8, v = i & 255;
    uint32_t oa = 0, ob = 0;
    for (int b = 0; b < 8; ++b) {
      int j = byte * 8 + b;
      if (((v >> b) & 1) && j < p.rC) {
        if (p.posA[j] >= 0) oa |= 1u << p.posA[j];
        if (p.posB[j] >= 0) ob |= 1u << p.posB[j];
      }
    }
    lutA[byte][v] = oa;
    lutB[byte][v] = ob;
  }
  for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) {
    int byte = i >> 8, v = i & 255;
    uint32_t oa = 0, ob = 0;
    for (int b = 0; b < 8; ++b) {
      int j = byte * 8 + b;
      if (((v >> b) & 1) && j < p.k) {
        if (p.sposA[j] >= 0) oa |= 1u << p.sposA[j];
        if (p.sposB[j] >= 0) ob |= 1u << p.sposB[j];
      }
    }
    slutA[byte][v] = oa;
    slutB[byte][v] = ob;
  }
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  __syncthreads();

  const uint64_t n_out = 1ull << p.rC;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int qc = (int)(gtid & (uint64_t)(p.mc.Qc - 1));
  const TA sa = (TA)operand_scale<TI>(p.ma, qc, p.mc.scale_inputs);
  const TA sb = (TA)operand_scale<TI>(p.mb, qc, p.mc.scale_inputs);
  const TI *A = (const TI *)p.A;
  const TI *B = (const TI *)p.B;
  TO *C = (TO *)p.C;
  const uint32_t ns = 1u << p.k;
  TO tmax = (TO)0, tmin = (TO)INFINITY;
  for (uint64_t o = gtid; o < n_out; o += stride) {
    const uint32_t oo = (uint32_t)o;
    const uint32_t ba = lutA[0][oo & 255] | lutA[1][(oo >> 8) & 255] | lutA[2][(oo >> 16) & 255] |
                        lutA[3][oo >> 24];
    const uint32_t bb = lutB[0][oo & 255] | lutB[1][(oo >> 8) & 255] | lutB[2][(oo >> 16) & 255] |
                        lutB[3][oo >> 24];
    TA acc = (TA)0;
    if (p.k <= 8) {
      for (uint32_t s = 0; s < ns; ++s) {
        const TA a = (TA)__ldg(A + (ba | slutA[0][s])) * sa;
        const TA b = (TA)__ldg(B + (bb | slutB[0][s])) * sb;
        acc = fma_t(a, b, acc);
      }
    } else {
      // blocked: 256-term serial partial sums, then a serial sum of blocks
      for (uint32_t hi = 0; hi < (ns >> 8); ++hi) {
        const uint32_t ha = ba | slutA[1][hi & 255] | slutA[2][hi >> 8];
        const uint32_t hb = bb | slutB[1][hi & 255] | slutB[2][hi >> 8];
        TA part = (TA)0;
        for (uint32_t lo = 0; lo < 256; ++lo) {
          const TA a = (TA)__ldg(A + (ha | slutA[0][lo])) * sa;
          const TA b = (TA)__ldg(B + (hb | slutB[0][lo])) * sb;
          part = fma_t(a, b, part);
        }
        acc += part;
      }
    }
    const TO c = (TO)acc;
    C[o] = c;
    track(c, tmax, tmin);
  }
  publish_warp(smax, smin, qc, tmax, tmin, p.mc.Qc);
  __syncthreads();
  finish_meta<TI>(p.ma, p.mb, p.mc, smax, smin);
}

// ------------------------------------------------------------ K2 stream
//
// C = P . S with P the large operand whose kept indices keep their
// relative order in C.  A thread owns one assignment w of P's kept indices
// (V consecutive ones when the V lowest bits of P and C coincide): it loads
// P once for every summed assignment, and writes every output that differs
// only in S's free indices.  P and C are read and written exactly once,
// contiguously and vectorised; S is small and served from L1.

struct K2Params {
  const void *A;  // P
  const void *B;  // S
  void *C;
  Meta ma, mb;
  OutMeta mc;
  int32_t log2_nu;  // work units
  int32_t vbits;    // log2 V
  int32_t k, f;     // summed bits, free bits of S
  int32_t n_insA, n_insC, n_seg;
  int32_t b_vec;      // S lanes: 0 per-lane loads, 1 contiguous, 2 broadcast
  int8_t insA[4];     // ascending positions of summed bits in P
  int8_t insC[4];     // ascending positions of S's free bits in C
  int8_t seg_c[16];   // S batch bits as runs: C position of the run's low bit,
  int8_t seg_b[16];   //   S position of the run's low bit,
  int8_t seg_len[16]; //   run length (C vector lanes excluded)
  uint32_t dA[16];   // offset of summed assignment s in P
  uint32_t dBs[16];  // ... in S
  uint32_t dBf[16];  // offset of S-free assignment f in S
  uint32_t dC[16];   // ... in C
  uint32_t dBv[4];  // offset in S of vector lane e
  int32_t s_staged;  // S (2^s_log2 entries) staged in shared memory, pre-scaled (k2_stream, K = 4)
  int32_t s_contig;  // staged, 4 summed bits at S's lowest 4 positions: 16-byte loads of S
  int32_t s_log2;
  int32_t quad;      // staged float32, one query lane: four consecutive units per thread (k2_stream_s16q)
};

template <typename T, int V> struct VecT;
template <> struct VecT<float, 1> { typedef float t; };
template <> struct VecT<float, 2> { typedef float2 t; };
template <> struct VecT<float, 4> { typedef float4 t; };
template <> struct VecT<double, 1> { typedef double t; };
template <> struct VecT<double, 2> { typedef double2 t; };

template <typename T, int V>
__device__ __forceinline__ void vload(const T *p, T (&r)[V]) {
  typedef typename VecT<T, V>::t VT;
  VT v = __ldg(reinterpret_cast<const VT *>(p));
  const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) r[i] = e[i];
}
template <typename T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&r)[V]) {
  typedef typename VecT<T, V>::t VT;
  VT v;
  T *e = reinterpret_cast<T *>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) e[i] = r[i];
  *reinterpret_cast<VT *>(p) = v;
}

// four consecutive entries from a 16-byte aligned shared-memory address
template <typename T>
__device__ __forceinline__ void lds4(const T *ptr, T (&r)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(ptr);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  } else {
    const double2 v0 = reinterpret_cast<const double2 *>(ptr)[0];
    const double2 v1 = reinterpret_cast<const double2 *>(ptr)[1];
    r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
  }
}

// K (summed bits) and F (S-free bits) are compile-time upper bounds; the
// runtime p.k / p.f select the active terms.  K = F = 4 runs with one lane
// per thread (V = 1): 16 P values, 16 scales and 16 max/min pairs.
template <typename T, int V, int K, int F>
__global__ void __launch_bounds__(kThreads, (K <= 1 ? 4 : (K == 2 || (K == 4 && sizeof(T) == 4) ? 2 : 1)))
    k2_stream(K2Params p) {
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  __syncthreads();
  constexpr int NS = 1 << K, NF = 1 << F;
  const int ns = 1 << p.k, nf = 1 << p.f;
  const T *A = (const T *)p.A;
  const T *B = (const T *)p.B;
  T *C = (T *)p.C;
  const uint64_t nu = 1ull << p.log2_nu;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t qmask_c = (uint32_t)(p.mc.Qc - 1);
  T sa[V], sb[NF][V], tmax[NF][V], tmin[NF][V];
  uint32_t qbase = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int e = 0; e < V; ++e) { tmax[f][e] = (T)0; tmin[f][e] = (T)INFINITY; sb[f][e] = (T)1; }
#pragma unroll
  for (int e = 0; e < V; ++e) sa[e] = (T)1;
  bool first = true;
  for (uint64_t u = gtid; u < nu; u += stride) {
    const uint32_t w = (uint32_t)u << p.vbits;
    uint32_t oa = w, oc = w, gb = 0;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < p.n_insA) oa = insert0(oa, p.insA[i]);
#pragma unroll
    for (int i = 0; i < F; ++i)
      if (i < p.n_insC) oc = insert0(oc, p.insC[i]);
    for (int i = 0; i < p.n_seg; ++i)
      gb |= ((oc >> p.seg_c[i]) & ((1u << p.seg_len[i]) - 1u)) << p.seg_b[i];
    if (first) {
      // each lane's query is fixed across the grid-stride loop (the stride
      // is a multiple of the query lanes)
      first = false;
      qbase = oc;
      if (p.mc.scale_inputs) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          sa[e] = operand_scale<T>(p.ma, (int)(oa + e), 1);
#pragma unroll
          for (int f = 0; f < NF; ++f)
            if (f < nf) sb[f][e] = operand_scale<T>(p.mb, (int)(gb + p.dBf[f] + p.dBv[e]), 1);
        }
      }
    }
    T a[NS][V];
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s < ns) {
        vload<T, V>(A + oa + p.dA[s], a[s]);
#pragma unroll
        for (int e = 0; e < V; ++e) a[s][e] *= sa[e];
      }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (f < nf) {
        T c[V];
#pragma unroll
        for (int e = 0; e < V; ++e) c[e] = (T)0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (s < ns) {
            T b[V];
            const uint32_t ob = gb + p.dBs[s] + p.dBf[f];
            if constexpr (V == 1) {
              b[0] = __ldg(B + ob);  // one lane: every S mode is this load
            } else if (p.b_vec == 1) {
              vload<T, V>(B + ob, b);
            } else if (p.b_vec == 2) {
              const T v = __ldg(B + ob);
#pragma unroll
              for (int e = 0; e < V; ++e) b[e] = v;
            } else {
#pragma unroll
              for (int e = 0; e < V; ++e) b[e] = __ldg(B + ob + p.dBv[e]);
            }
#pragma unroll
            for (int e = 0; e < V; ++e) c[e] = fma_t(a[s][e], b[e] * sb[f][e], c[e]);
          }
        }
        vstore<T, V>(C + oc + p.dC[f], c);
#pragma unroll
        for (int e = 0; e < V; ++e) track(c[e], tmax[f][e], tmin[f][e]);
      }
    }
  }
  if (!first) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (f < nf) publish(smax, smin, (int)((qbase + p.dC[f] + e) & qmask_c), tmax[f][e], tmin[f][e]);
  }
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// k2_stream for four summed or S-free bits at one lane per thread with S
// staged in shared memory (K2Params.s_staged), in a kernel of its own so
// that it holds only what this path needs (64 registers: four blocks per SM).  S is
// staged once per block, already times its lane scale (the products b * sb
// of k2_stream); the summed offsets sit in registers.  Every output of a
// unit is in one query lane (the S-free bits sit above the query bits), so
// one max/min pair tracks them all.  CONTIG: S's 4 summed indices are its
// lowest bits (K2Params.s_contig), read with 16-byte loads.
template <typename T, bool CONTIG>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k2_stream_s16(K2Params p) {
  extern __shared__ __align__(16) unsigned char k2s_smem[];
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  T *sS = reinterpret_cast<T *>(k2s_smem);
  {
    const T *Bg = (const T *)p.B;
    for (uint32_t j = threadIdx.x; j < (1u << p.s_log2); j += blockDim.x)
      sS[j] = p.mc.scale_inputs ? __ldg(Bg + j) * operand_scale<T>(p.mb, (int)j, 1) : __ldg(Bg + j);
  }
  __syncthreads();
  constexpr int K = 4, NS = 16;
  const int ns = 1 << p.k, nf = 1 << p.f;
  const T *A = (const T *)p.A;
  T *C = (T *)p.C;
  const uint64_t nu = 1ull << p.log2_nu;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t qmask_c = (uint32_t)(p.mc.Qc - 1);
  T sa = (T)1, tmax = (T)0, tmin = (T)INFINITY;
  uint32_t qbase = 0;
  uint32_t bsv[NS];  // summed offsets of S (unused when CONTIG)
#pragma unroll
  for (int s = 0; s < NS; ++s) bsv[s] = (!CONTIG && s < ns) ? p.dBs[s] : 0u;
  bool first = true;
  auto p_offset = [&](uint64_t uu) {
    uint32_t o = (uint32_t)uu;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < p.n_insA) o = insert0(o, p.insA[i]);
    return o;
  };
  // P entries of the next unit, requested before this unit's products
  T an[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) an[s] = (T)0;
  if (gtid < nu) {
    const uint32_t o = p_offset(gtid);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s < ns) an[s] = __ldg(A + o + p.dA[s]);
  }
  for (uint64_t u = gtid; u < nu; u += stride) {
    const uint32_t oa = p_offset(u);
    uint32_t oc = (uint32_t)u, gb = 0;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < p.n_insC) oc = insert0(oc, p.insC[i]);
    for (int i = 0; i < p.n_seg; ++i)
      gb |= ((oc >> p.seg_c[i]) & ((1u << p.seg_len[i]) - 1u)) << p.seg_b[i];
    if (first) {
      first = false;
      qbase = oc;
      if (p.mc.scale_inputs) sa = operand_scale<T>(p.ma, (int)oa, 1);
    }
    T a[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) a[s] = an[s] * sa;
    if (u + stride < nu) {
      const uint32_t o = p_offset(u + stride);
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (s < ns) an[s] = __ldg(A + o + p.dA[s]);
    }
    // Four outputs at a time (nf is a power of two): four independent
    // FMA chains hide the shared-memory and FMA latencies; each output
    // still adds its terms in order.
    const T *sS = reinterpret_cast<const T *>(k2s_smem);
    if (nf >= 4) {
#pragma unroll 1
      for (int f = 0; f < nf; f += 4) {
        const T *s0 = sS + gb + p.dBf[f], *s1 = sS + gb + p.dBf[f + 1];
        const T *s2 = sS + gb + p.dBf[f + 2], *s3 = sS + gb + p.dBf[f + 3];
        T c0 = (T)0, c1 = (T)0, c2 = (T)0, c3 = (T)0;
        if constexpr (CONTIG) {
          // the 16 summed entries of each output are consecutive in S
#pragma unroll
          for (int g4 = 0; g4 < NS; g4 += 4) {
            T v0[4], v1[4], v2[4], v3[4];
            lds4(s0 + g4, v0); lds4(s1 + g4, v1); lds4(s2 + g4, v2); lds4(s3 + g4, v3);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              c0 = fma_t(a[g4 + r], v0[r], c0);
              c1 = fma_t(a[g4 + r], v1[r], c1);
              c2 = fma_t(a[g4 + r], v2[r], c2);
              c3 = fma_t(a[g4 + r], v3[r], c3);
            }
          }
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s)
            if (s < ns) {
              c0 = fma_t(a[s], s0[bsv[s]], c0);
              c1 = fma_t(a[s], s1[bsv[s]], c1);
              c2 = fma_t(a[s], s2[bsv[s]], c2);
              c3 = fma_t(a[s], s3[bsv[s]], c3);
            }
        }
        C[oc + p.dC[f]] = c0;
        C[oc + p.dC[f + 1]] = c1;
        C[oc + p.dC[f + 2]] = c2;
        C[oc + p.dC[f + 3]] = c3;
        track(c0, tmax, tmin);
        track(c1, tmax, tmin);
        track(c2, tmax, tmin);
        track(c3, tmax, tmin);
      }
    } else {
#pragma unroll 1
      for (int f = 0; f < nf; ++f) {
        const T *sf = sS + gb + p.dBf[f];
        T c = (T)0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if (s < ns) c = fma_t(a[s], sf[CONTIG ? (uint32_t)s : bsv[s]], c);
        C[oc + p.dC[f]] = c;
        track(c, tmax, tmin);
      }
    }
  }
  if (!first) publish(smax, smin, (int)(qbase & qmask_c), tmax, tmin);
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// k2_stream_s16 with four consecutive work units per thread (float32, C
// without query bits): when the two lowest bits of a unit are P's and C's
// two lowest bits and S does not depend on them, the four units share
// every S value, so each thread loads P's 16 summed entries of its four
// units as 16-byte vectors, uses each staged S value for four outputs and
// stores four outputs with one 16-byte store.  Each output adds its terms
// in the same order as k2_stream_s16 (one FMA per summed assignment in
// ascending order, operands scaled first), so the bits are the same.
template <bool CONTIG>
__global__ void __launch_bounds__(kThreads, 2) k2_stream_s16q(K2Params p) {
  extern __shared__ __align__(16) unsigned char k2s_smem[];
  __shared__ unsigned long long smax[1], smin[1];
  if (threadIdx.x == 0) { smax[0] = 0; smin[0] = kNoMin; }
  float *sS = reinterpret_cast<float *>(k2s_smem);
  {
    const float *Bg = (const float *)p.B;
    for (uint32_t j = threadIdx.x; j < (1u << p.s_log2); j += blockDim.x)
      sS[j] = p.mc.scale_inputs ? __ldg(Bg + j) * operand_scale<float>(p.mb, 0, 1) : __ldg(Bg + j);
  }
  __syncthreads();
  constexpr int K = 4, NS = 16;
  const int ns = 1 << p.k, nf = 1 << p.f;
  const float *A = (const float *)p.A;
  float *C = (float *)p.C;
  const uint64_t nq = 1ull << (p.log2_nu - 2);  // quads of units
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const float sa = p.mc.scale_inputs ? operand_scale<float>(p.ma, 0, 1) : 1.0f;
  float tmax = 0.0f, tmin = INFINITY;
  uint32_t bsv[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) bsv[s] = (!CONTIG && s < ns) ? p.dBs[s] : 0u;
  for (uint64_t qd = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; qd < nq; qd += stride) {
    const uint32_t u = (uint32_t)(qd << 2);
    uint32_t oa = u, oc = u, gb = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (i < p.n_insA) oa = insert0(oa, p.insA[i]);
      if (i < p.n_insC) oc = insert0(oc, p.insC[i]);
    }
    for (int i = 0; i < p.n_seg; ++i)
      gb |= ((oc >> p.seg_c[i]) & ((1u << p.seg_len[i]) - 1u)) << p.seg_b[i];
    float a[NS][4];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s < ns) v = __ldg(reinterpret_cast<const float4 *>(A + oa + p.dA[s]));
      a[s][0] = v.x * sa; a[s][1] = v.y * sa; a[s][2] = v.z * sa; a[s][3] = v.w * sa;
    }
#pragma unroll 1
    for (int f = 0; f < nf; f += 2) {
      // two outputs of S-free assignments f, f + 1 for the four units
      const float *s0 = sS + gb + p.dBf[f], *s1 = sS + gb + p.dBf[f + 1];
      float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
      if constexpr (CONTIG) {
#pragma unroll
        for (int g4 = 0; g4 < NS; g4 += 4) {
          float v0[4], v1[4];
          lds4(s0 + g4, v0);
          lds4(s1 + g4, v1);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              c0[e] = fma_t(a[g4 + r][e], v0[r], c0[e]);
              c1[e] = fma_t(a[g4 + r][e], v1[r], c1[e]);
            }
        }
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if (s < ns) {
            const float v0 = s0[bsv[s]], v1 = s1[bsv[s]];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              c0[e] = fma_t(a[s][e], v0, c0[e]);
              c1[e] = fma_t(a[s][e], v1, c1[e]);
            }
          }
      }
      __stcs(reinterpret_cast<float4 *>(C + oc + p.dC[f]), make_float4(c0[0], c0[1], c0[2], c0[3]));
      if (f + 1 < nf)
        __stcs(reinterpret_cast<float4 *>(C + oc + p.dC[f + 1]), make_float4(c1[0], c1[1], c1[2], c1[3]));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        track(c0[e], tmax, tmin);
        if (f + 1 < nf) track(c1[e], tmax, tmin);
      }
    }
  }
  publish_warp(smax, smin, 0, tmax, tmin, 1);
  __syncthreads();
  finish_meta<float>(p.ma, p.mb, p.mc, smax, smin);
}

// ------------------------------------------------- K2 with TMA staging
//
// Same contraction as k2_stream, but P is brought on chip by bulk async
// copies (cp.async.bulk, the TMA engine) into a ring of shared-memory
// stages guarded by mbarriers: one elected thread keeps kStages tiles in
// flight while every thread computes the current tile, so HBM latency is
// hidden by the copy engine rather than by warps.  A tile is 2^tb
// consecutive assignments w of P's kept indices; its P data are nruns
// contiguous runs of 2^run_log2 elements (one per assignment of the summed
// indices that lie above the tile's bit range).
//
// Bit deposits are linear over disjoint bits, so every offset splits into
// a per-tile part (computed once per tile by the issuing thread) and a
// per-thread part (computed once per launch): the inner loop only ORs.  S
// is small: each block stages it in shared memory already multiplied by
// its per-query scale.
//
// Every mbarrier wait is bounded by %globaltimer (about one second): on
// timeout the block records an error word, drains its own copies (again
// bounded) and returns.

struct K2TParams {
  K2Params k;           // mapping shared with k2_stream
  int32_t tb;           // log2 tile size (in w)
  int32_t run_log2;     // log2 elements per run
  int32_t nruns;
  int32_t n_lowA;       // summed positions of P inside the tile's span
  int8_t lowA[4];
  int32_t s_log2;       // log2 elements of S (staged in shared memory)
  int32_t fold_sa;      // S carries P's query lanes: P's scale is folded into S
  uint32_t run_off[8];  // P offset of run r (high summed bits)
  uint32_t sA_off[8];   // shared-memory offset of summed assignment s
  uint32_t *err;        // error word (bit 0: an mbarrier wait timed out)
  int32_t debug_stall;  // test hook: never issue the first tile's copy
};

constexpr int kStages = 3;
constexpr int kMaxJ = 4;                        // work units per thread per tile
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of one wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Programmatic dependent launch: wait until the grids this launch depends
// on have completed and their memory is visible (no-op without the launch
// attribute), and allow the next launch to start its independent part.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// wait bounded in time; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitNs) return false;
  }
}

// max(m, |x|); float64 on the integer units as in track<double>
template <typename T>
__device__ __forceinline__ T max_abs(T m, T x) { return fmax(m, fabs(x)); }
template <>
__device__ __forceinline__ double max_abs<double>(double m, double x) {
  const uint32_t ah = (uint32_t)__double2hiint(x) & 0x7fffffffu, al = (uint32_t)__double2loint(x);
  const uint32_t mh = (uint32_t)__double2hiint(m), ml = (uint32_t)__double2loint(m);
  const bool finite_or_inf = ah < 0x7ff00000u || (ah == 0x7ff00000u && al == 0u);
  const bool gt = ah > mh || (ah == mh && al > ml);
  return (gt && finite_or_inf) ? __hiloint2double((int)ah, (int)al) : m;
}

// min(bits - 1, cur) on IEEE bit patterns: zero maps to the largest value,
// so the running minimum is the smallest nonzero magnitude minus one
__device__ __forceinline__ uint32_t min_m1(uint32_t bits, uint32_t cur) {
  return __viaddmin_u32(bits, 0xffffffffu, cur);
}
// float64: the same in 32-bit halves (subtract with borrow, compare high
// words first), off the slower 64-bit integer path
__device__ __forceinline__ unsigned long long min_m1(unsigned long long bits, unsigned long long cur) {
  const uint32_t lo = (uint32_t)bits, hi = (uint32_t)(bits >> 32);
  const uint32_t mlo = lo - 1u, mhi = hi - (lo == 0u ? 1u : 0u);
  const uint32_t clo = (uint32_t)cur, chi = (uint32_t)(cur >> 32);
  const bool lt = mhi < chi || (mhi == chi && mlo < clo);
  return lt ? (((unsigned long long)mhi << 32) | mlo) : cur;
}

template <typename T>
__device__ __forceinline__ void track_fast(T c, T &tmax, T &tmin) {
  if constexpr (sizeof(T) == 8) {
    track<double>(c, tmax, tmin);
  } else {
    const T a = fabs(c);
    tmax = fmax(tmax, a);
    tmin = fmin(tmin, a != (T)0 ? a : (T)INFINITY);
  }
}

constexpr int kConsumerWarps = kThreads / 32;

template <typename T> struct Bits;
template <> struct Bits<float> { typedef uint32_t t; };
template <> struct Bits<double> { typedef unsigned long long t; };

// 32-bit shared-memory vector loads at a byte address
template <typename T, int V> struct LdsV;
template <> struct LdsV<float, 4> {
  static __device__ __forceinline__ void ld(uint32_t a, float (&r)[4]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]) : "r"(a));
  }
};
template <> struct LdsV<float, 2> {
  static __device__ __forceinline__ void ld(uint32_t a, float (&r)[2]) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r[0]), "=f"(r[1]) : "r"(a));
  }
};
template <> struct LdsV<float, 1> {
  static __device__ __forceinline__ void ld(uint32_t a, float (&r)[1]) {
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r[0]) : "r"(a));
  }
};
template <> struct LdsV<double, 2> {
  static __device__ __forceinline__ void ld(uint32_t a, double (&r)[2]) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(r[0]), "=d"(r[1]) : "r"(a));
  }
};
template <> struct LdsV<double, 1> {
  static __device__ __forceinline__ void ld(uint32_t a, double (&r)[1]) {
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(r[0]) : "r"(a));
  }
};
__device__ __forceinline__ float lds1(uint32_t a, float) {
  float r;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a));
  return r;
}
__device__ __forceinline__ double lds1(uint32_t a, double) {
  double r;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(r) : "r"(a));
  return r;
}
__device__ __forceinline__ uint32_t to_bits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long to_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// Warp-specialised: warps 0..kConsumerWarps-1 compute, the last warp's
// lane 0 produces.  full[st] completes when a tile's bytes have landed
// (arrive.expect_tx + complete_tx); empty[st] completes when every consumer
// warp has finished reading the stage.  No block-wide barrier in the loop.
// With EXACT the runtime k, f equal K, F and every guard folds away.
// Tracking: max|c| as a float max, min nonzero as an unsigned min of the
// bit pattern minus one (zero wraps to the largest value; nonnegative
// entries, which is what the flush test covers).
template <typename T, int V, int K, int F, bool EXACT>
__global__ void __launch_bounds__(kThreads + 32, (K + F <= 2 ? 3 : (K + F <= 4 ? 2 : 1))) k2_tma(K2TParams tp) {
  typedef typename Bits<T>::t BT;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
  __shared__ uint32_t tile_oc[kStages], tile_gb[kStages];
  __shared__ int s_skip;
  const K2Params &p = tp.k;
  if (threadIdx.x == 0) s_skip = (tp.err && *(volatile uint32_t *)tp.err) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // an earlier launch of this walk gave up: skip the work
  const uint32_t run_len = 1u << tp.run_log2;
  const uint32_t tile_elems = (uint32_t)tp.nruns * run_len;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
  const uint32_t n_tiles = 1u << (p.log2_nu + p.vbits - tp.tb);
  T *stage_buf = reinterpret_cast<T *>(dyn_smem);
  T *sS = stage_buf + (size_t)kStages * tile_elems;  // S, pre-scaled
  const size_t s_bytes = (((size_t)sizeof(T) << tp.s_log2) + 15) & ~(size_t)15;
  unsigned long long *smax =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(sS) + s_bytes);
  unsigned long long *smin = smax + p.mc.Qc;
  const T *A = (const T *)p.A;
  const T *B = (const T *)p.B;
  T *C = (T *)p.C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nthr = kConsumerWarps * 32;
  // The producer sets up the barriers and puts the first tiles in flight
  // before the block stages S, so the copies overlap the prologue.
  auto produce = [&](uint32_t i) -> bool {
    const int st = (int)(i % kStages);
    if (i >= (uint32_t)kStages && !mbar_wait(&empty[st], ((i / kStages) - 1) & 1)) return false;
    const uint32_t bw = (blockIdx.x + i * gridDim.x) << tp.tb;
    uint32_t base = bw, oc = bw, gb = 0;
    for (int j = 0; j < p.n_insA; ++j) base = insert0(base, p.insA[j]);
    for (int j = 0; j < p.n_insC; ++j) oc = insert0(oc, p.insC[j]);
    for (int j = 0; j < p.n_seg; ++j)
      gb |= ((oc >> p.seg_c[j]) & ((1u << p.seg_len[j]) - 1u)) << p.seg_b[j];
    tile_oc[st] = oc;
    tile_gb[st] = gb;
    fence_proxy_async_smem();
    mbar_expect_tx(&full[st], tile_bytes);  // release: tile_oc/gb visible
    if (tp.debug_stall && i == 0) return true;  // test hook: the wait must run out
    for (int r = 0; r < tp.nruns; ++r)
      bulk_g2s(stage_buf + (size_t)st * tile_elems + (size_t)r * run_len, A + base + tp.run_off[r],
               run_len * (uint32_t)sizeof(T), &full[st]);
    return true;
  };
  const bool producer = (warp == kConsumerWarps) && lane == 0;
  uint32_t n_pre = 0;
  if (producer) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumerWarps);
    }
    mbar_fence_init();
    for (; n_pre < (uint32_t)kStages && blockIdx.x + n_pre * gridDim.x < n_tiles; ++n_pre) produce(n_pre);
  }
  // per-query scale of the staged S (S's own scale, times P's when folded)
  T *sscale = reinterpret_cast<T *>(smin + p.mc.Qc);
  const int qs = p.mb.qmask + 1;
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  for (int q = threadIdx.x; q < qs; q += blockDim.x) {
    T v = operand_scale<T>(p.mb, q, p.mc.scale_inputs);
    if (tp.fold_sa) v *= operand_scale<T>(p.ma, q, p.mc.scale_inputs);
    sscale[q] = v;
  }
  __syncthreads();
  // stage S (independent coalesced loads)
  const uint32_t n_s = 1u << tp.s_log2;
#pragma unroll 4
  for (uint32_t j = threadIdx.x; j < n_s; j += blockDim.x) sS[j] = __ldg(B + j) * sscale[j & p.mb.qmask];
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t i = n_pre;
      bool ok = true;
      for (; blockIdx.x + i * gridDim.x < n_tiles; ++i) {
        if (!produce(i)) {
          ok = false;
          break;
        }
      }
      if (!ok && tp.err) atomicOr(tp.err, 1u);
      // drain: copies of the last kStages issued tiles may still be in flight
      const uint32_t n_issued = i;
      for (uint32_t j = n_issued > (uint32_t)kStages ? n_issued - kStages : 0; j < n_issued; ++j)
        if (!mbar_wait(&full[j % kStages], (j / kStages) & 1) && tp.err) atomicOr(tp.err, 1u);
    }
    __syncwarp();  // the producer warp reconverges before the block barrier
  } else {
    // ----------------------------------------------------------- consumers
    constexpr int NS = 1 << K, NF = 1 << F;
    const int ns = EXACT ? NS : (1 << p.k);
    const int nf = EXACT ? NF : (1 << p.f);
    constexpr int J = (V == 1) ? 4 : 2;  // work units per thread per tile (host: T_w = 256*V*J)
    constexpr uint32_t es = (uint32_t)sizeof(T);
    const uint32_t stage0 = smem_addr(stage_buf), sS0 = smem_addr(sS);
    // per-thread parts of the offsets (constant across tiles), in bytes
    uint32_t la4[J], ocl[J], gbl4[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const uint32_t wl = (threadIdx.x + (uint32_t)j * nthr) * V;
      uint32_t a = wl, c = wl, g = 0;
      for (int i = 0; i < tp.n_lowA; ++i) a = insert0(a, tp.lowA[i]);
      for (int i = 0; i < p.n_insC; ++i) c = insert0(c, p.insC[i]);
      for (int i = 0; i < p.n_seg; ++i)
        g |= ((c >> p.seg_c[i]) & ((1u << p.seg_len[i]) - 1u)) << p.seg_b[i];
      la4[j] = a * es; ocl[j] = c; gbl4[j] = g * es + sS0;
    }
    uint32_t aoff[NS], boff[NS][NF];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      aoff[s] = (s < ns) ? tp.sA_off[s] * es : 0u;
#pragma unroll
      for (int f = 0; f < NF; ++f) boff[s][f] = (s < ns && f < nf) ? (p.dBs[s] + p.dBf[f]) * es : 0u;
    }
    uint32_t dCf[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) dCf[f] = (f < nf) ? p.dC[f] : 0u;
    // each lane's query is the same in every tile
    T sa[V];
#pragma unroll
    for (int e = 0; e < V; ++e)
      sa[e] = tp.fold_sa ? (T)1 : operand_scale<T>(p.ma, (int)(threadIdx.x * V + e), p.mc.scale_inputs);
    T tmax[NF][V];
    BT tminm1[NF][V];  // (bits of the smallest nonzero) - 1
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int e = 0; e < V; ++e) { tmax[f][e] = (T)0; tminm1[f][e] = (BT)~(BT)0; }
    for (uint32_t i = 0; blockIdx.x + i * gridDim.x < n_tiles; ++i) {
      const int st = (int)(i % kStages);
      // every lane waits (acquire), the warp agrees on the outcome
      const bool landed = __all_sync(0xffffffffu, mbar_wait(&full[st], (i / kStages) & 1));
      if (!landed) {
        if (lane == 0 && tp.err) atomicOr(tp.err, 1u);
        break;
      }
      const uint32_t tile0 = stage0 + (uint32_t)st * tile_bytes;
      const uint32_t ocb = tile_oc[st], gbb4 = tile_gb[st] * es;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const uint32_t oc = ocb | ocl[j];
        const uint32_t gaddr = gbb4 + gbl4[j];
        T a[NS][V];
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if (s < ns) {
            LdsV<T, V>::ld(tile0 + la4[j] + aoff[s], a[s]);
            if (!tp.fold_sa) {
#pragma unroll
              for (int e = 0; e < V; ++e) a[s][e] *= sa[e];
            }
          }
        T *cptr = C + oc;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f < nf) {
            T c[V];
#pragma unroll
            for (int e = 0; e < V; ++e) c[e] = (T)0;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              if (s < ns) {
                T b[V];
                const uint32_t ba = gaddr + boff[s][f];
                if (V > 1 && p.b_vec == 1) {
                  LdsV<T, V>::ld(ba, b);
                } else if (p.b_vec == 2) {
                  const T v = lds1(ba, T());
#pragma unroll
                  for (int e = 0; e < V; ++e) b[e] = v;
                } else {
#pragma unroll
                  for (int e = 0; e < V; ++e) b[e] = lds1(ba + p.dBv[e] * es, T());
                }
#pragma unroll
                for (int e = 0; e < V; ++e) c[e] = fma_t(a[s][e], b[e], c[e]);
              }
            }
            vstore<T, V>(cptr + dCf[f], c);
#pragma unroll
            for (int e = 0; e < V; ++e) {
              tmax[f][e] = max_abs(tmax[f][e], c[e]);
              tminm1[f][e] = min_m1(to_bits(c[e]), tminm1[f][e]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    const uint32_t qmask_c = (uint32_t)(p.mc.Qc - 1);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (f < nf) {
          const int q = (int)((ocl[0] + dCf[f] + e) & qmask_c);
          if (tmax[f][e] != (T)0) atomicMax(smax + q, abs_bits(tmax[f][e]));
          if (tminm1[f][e] != (BT)~(BT)0) atomicMin(smin + q, (unsigned long long)(tminm1[f][e] + (BT)1));
        }
  }
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// ------------------------------------------- batched small contractions
//
// Joins of two large operands whose free and summed sets are small: C[u,
// fa, fb] = sum over s of A[u, fa, s] B[u, s, fb], u the batch indices
// (shared and kept, the query lanes among them), fa / fb the free indices
// of A / B (at most 4 / 3 bits), s the summed ones (at most 2 bits; every
// summed index in both operands).  A thread takes one u at a time
// (grid-stride): it loads A's 2^(fA+k) and B's 2^(k+fB) values, forms the
// 2^(fA+fB) outputs in registers (each a fused multiply-add chain over s
// ascending from zero: the order of every other kernel) and stores them.
// For a fixed (fa, s) a warp reads 32 consecutive u when the operands'
// lowest indices are batch ones (the lanes), so every access is coalesced,
// and each operand crosses memory once.  u enumerates the batch indices in
// C's order: its bits are deposited around C's other positions (insC,
// ascending) and mapped to A's and B's positions (any order) through
// per-block tables over u's four bytes.
constexpr int kBatchedNA = 16, kBatchedNB = 8, kBatchedNC = 32;

struct K2BParams {
  const void *A, *B;
  void *C;
  Meta ma, mb;
  OutMeta mc;
  int32_t log2_nu;               // batch bits
  int32_t n_insC;
  int8_t insC[8];                // C's positions of the free indices, ascending
  int8_t posA[32], posB[32];     // u bit j -> A's, B's position (-1: a lane the operand lacks)
  int32_t fA, fB, k;
  uint32_t offA[kBatchedNA];     // A offset of (fa, s): index fa | s << fA
  uint32_t offB[kBatchedNB];     // B offset of (s, fb): index s | fb << k
  uint32_t offC[kBatchedNC];     // C offset of (fa, fb): index fa | fb << fA
};

// KS, FA, FB >= 0: the shape at compile time (register arrays with static
// indices); -1: the runtime shape (arrays indexed at run time, in local
// memory)
template <typename T, int KS, int FA, int FB>
__global__ void __launch_bounds__(kThreads, KS >= 0 ? 3 : 2) k2_batched(K2BParams p) {
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  __shared__ uint32_t lutA[4][256], lutB[4][256];  // u's byte r -> A's, B's offset
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const int r = i >> 8, v = i & 255;
    uint32_t oa = 0, ob = 0;
    for (int bb = 0; bb < 8 && 8 * r + bb < p.log2_nu; ++bb)
      if ((v >> bb) & 1) {
        if (p.posA[8 * r + bb] >= 0) oa |= 1u << p.posA[8 * r + bb];  // (-1: broadcast over it)
        if (p.posB[8 * r + bb] >= 0) ob |= 1u << p.posB[8 * r + bb];
      }
    lutA[r][v] = oa;
    lutB[r][v] = ob;
  }
  __syncthreads();
  const T *A = static_cast<const T *>(p.A);
  const T *B = static_cast<const T *>(p.B);
  T *C = static_cast<T *>(p.C);
  uint32_t mc = 0;
  for (int j = 0; j < p.n_insC; ++j) mc |= 1u << p.insC[j];
  const uint32_t n_units = 1u << p.log2_nu;
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t oc = u, dc = stride;
  for (int j = 0; j < p.n_insC; ++j) { oc = insert0(oc, p.insC[j]); dc = insert0(dc, p.insC[j]); }
  auto offA = [&](uint32_t x) { return lutA[0][x & 255] | lutA[1][(x >> 8) & 255] | lutA[2][(x >> 16) & 255] | lutA[3][x >> 24]; };
  auto offB = [&](uint32_t x) { return lutB[0][x & 255] | lutB[1][(x >> 8) & 255] | lutB[2][(x >> 16) & 255] | lutB[3][x >> 24]; };
  const uint32_t oa0 = offA(u), ob0 = offB(u);
  // a thread's units share their lanes (the stride is a multiple of the
  // lane count and the lanes are the lowest batch bits)
  const int qa = (int)(oa0 & (uint32_t)p.ma.qmask), qb = (int)(ob0 & (uint32_t)p.mb.qmask);
  const T sa = operand_scale<T>(p.ma, qa, p.mc.scale_inputs), sb = operand_scale<T>(p.mb, qb, p.mc.scale_inputs);
  constexpr bool CT = KS >= 0;
  const int fA = CT ? FA : p.fA, fB = CT ? FB : p.fB, kk = CT ? KS : p.k;
  const int na = 1 << (fA + kk), nb = 1 << (kk + fB), nfa = 1 << fA, nfb = 1 << fB, ns = 1 << kk;
  T tmax = (T)0, tmin = (T)INFINITY;
  for (; u < n_units; u += stride) {
    const uint32_t oa = offA(u), ob = offB(u);
    T a[kBatchedNA], b[kBatchedNB];
#pragma unroll
    for (int i = 0; i < kBatchedNA; ++i)
      if (i < na) a[i] = __ldcs(A + (oa | p.offA[i])) * sa;
#pragma unroll
    for (int i = 0; i < kBatchedNB; ++i)
      if (i < nb) b[i] = __ldcs(B + (ob | p.offB[i])) * sb;
#pragma unroll
    for (int fb = 0; fb < kBatchedNB; ++fb) {
      if (fb >= nfb) break;
#pragma unroll
      for (int fa = 0; fa < kBatchedNA; ++fa) {
        if (fa >= nfa) break;
        T acc = (T)0;
#pragma unroll
        for (int sidx = 0; sidx < 4; ++sidx)
          if (sidx < ns) acc = fma_t(a[fa | (sidx << fA)], b[sidx | (fb << kk)], acc);
        C[oc | p.offC[fa | (fb << fA)]] = acc;
        track(acc, tmax, tmin);
      }
    }
    oc = ((oc | mc) + dc) & ~mc;
  }
  {
    const int qc = (int)((blockIdx.x * blockDim.x + threadIdx.x) & (uint32_t)(p.mc.Qc - 1));
    if (tmax != (T)0) atomicMax(smax + qc, abs_bits(tmax));
    if (tmin != (T)INFINITY) atomicMin(smin + qc, abs_bits(tmin));
  }
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// ---------------------------------------------- chain of frontier eliminations
//
// D consecutive frontier contractions C_i = C_{i-1} . S_i (C_0 = P) in one
// pass over P, each summing one index x_i of P.  Step i adds y_i at x_i's
// position (in place); with GROW the first step adds a second index z at
// the top of the frontier, with SHRINK the last step adds none (the
// frontier's higher indices move down one position).  A work unit is one
// assignment of P's other (kept) indices: the thread loads the 2^D values
// of P over (x_1..x_D) into registers and applies the steps in place:
// bit i of the register index means x_i before step i and y_i after it,
// bit D (GROW) means z.  Only P and C_D touch memory: |P| + |C_D| bytes for
// D eliminations instead of the sum over the D separate passes.
//
// Each output of a step is a two-term FMA chain over x_i = 0, 1 starting
// from zero, the order every other kernel uses for one summed index, and
// the intermediates are not rescaled (their scales are powers of two, so
// only the exponent bookkeeping moves): results are bit-identical to D
// separate launches.  S_i may depend on other chain indices; the host
// passes S_i's offset for every state of the chain bits.  The FAST
// variants are compiled for the common layout: S_i depends on no chain
// index but the two added last before y_i (so each block of S_i is loaded
// once per dependency combination, not once per pair), every S_i holds
// its lanes contiguously or one value for all of them, and P's scale
// folds into S_1.  The S_i
// arrive in shared memory by bulk async copies and are scaled there; P is
// staged tile by tile by bulk async copies that the whole producer warp
// issues, with NW consumer warps.

// Up to 4 eliminations with vector lanes or a growth step (2^(D + GROW)
// values per lane), up to 6 on one lane (64 values per thread).
constexpr int kMaxChain = 6;
constexpr int kChainDRow = 128;  // entries of one step's S offset table (2^NB x added values)
constexpr int kMaxStagesC = 4;
constexpr int kChainNW = 8;  // consumer warps

struct K2CParams {
  const void *P;
  void *C;
  Meta mp;
  OutMeta mc;
  const void *S[kMaxChain];
  Meta ms[kMaxChain];
  int32_t vbits;
  int32_t log2_nu;                // kept bits of P above the lane bits
  int32_t n_ins;                  // chain positions in P (x_i), ascending
  int8_t ins[kMaxChain];
  int32_t n_insc;                 // positions in C of the added indices, ascending
  int8_t insc[kMaxChain + 1];
  int32_t tb;                     // log2 work units per tile
  int32_t run_log2, nruns;        // P runs per tile
  int32_t n_low;                  // chain positions inside a run
  int8_t low[kMaxChain];
  uint32_t run_off[1 << kMaxChain];
  int32_t n_stages;
  int32_t fold_sp;                // P's scale is folded into the staged S_1
  uint32_t s_bytes_off[kMaxChain + 1];  // byte offset of staged S_i after the stages
  uint32_t s_copy_bytes;          // sum of the S_i sizes
  int32_t s_log2[kMaxChain];
  int32_t n_seg[kMaxChain];       // gathers of S_i's other indices from C's offset
  int8_t seg_c[kMaxChain][8], seg_b[kMaxChain][8], seg_len[kMaxChain][8];
  int32_t b_vec[kMaxChain];       // S_i lanes: 0 per lane, 1 contiguous, 2 broadcast
  uint32_t dv[kMaxChain][4];      // S_i element offset of lane e (mode 0)
  // S_i byte offset of (state s, added value(s) a): d[i][s | a << NB], NB =
  // D + GROW state bits; a = y_i, or y_0 + 2 z for a growth step, or 0
  uint32_t d[kMaxChain][kChainDRow];
  uint32_t pA[1 << kMaxChain];    // stage byte offset of P for x-state s
  uint32_t dC[1 << kMaxChain];    // C element offset of final state s (2^NB <= 64)
  uint32_t *err;
  int32_t debug_stall;
  int32_t units;                  // work units per consumer thread per tile (1, 2)
  int32_t variant;                // 0 plain, 1 growth (first step adds two indices), 2 shrink
};

__host__ __device__ constexpr uint32_t pdep_c(uint32_t t, uint32_t mask) {
  uint32_t r = 0;
  int k = 0;
  for (int j = 0; j < 32; ++j)
    if ((mask >> j) & 1u) {
      if ((t >> k) & 1u) r |= 1u << j;
      ++k;
    }
  return r;
}
__host__ __device__ constexpr int popc_c(uint32_t m) { return m ? (int)(m & 1u) + popc_c(m >> 1) : 0; }
// state bits other than x_i present at step i: the added ones of the
// earlier steps (y_j, and z once the growth step is done) and the x_j of
// the later steps
__host__ __device__ constexpr uint32_t chain_others(int D, int grow, int i) {
  return (((1u << D) - 1u) & ~(1u << i)) | ((grow && i > 0) ? 1u << D : 0u);
}
// chain bits that S_i may depend on: the FAST layout allows the two
// indices added last before step i (in the order y_0, z, y_1, y_2, ...),
// the generic one any
__host__ __device__ constexpr uint32_t chain_deps(int D, bool fast, int grow, int i) {
  uint32_t m = 0;
  int n = 0;
  for (int j = i - 1; j >= 0 && n < 2; --j) {
    if (j == 0 && grow) {
      m |= 1u << D;
      if (++n == 2) break;
    }
    m |= 1u << j;
    ++n;
  }
  return fast ? (m & chain_others(D, grow, i)) : chain_others(D, grow, i);
}

// V lanes of a staged S_i at shared-memory byte address `a`; LM is the lane
// mode when known at compile time (1 contiguous, 2 one value for all
// lanes, 3 one load per lane at its own offset), 0 to follow the runtime mode
template <typename T, int V, int LM>
__device__ __forceinline__ void ld_lanes(uint32_t a, int mode, const uint32_t *dv, T (&r)[V]) {
  if (LM == 1 || (LM == 0 && (V == 1 || mode == 1))) {
    LdsV<T, V>::ld(a, r);
  } else if (LM == 2 || (LM == 0 && mode == 2)) {
    const T v = lds1(a, T());
#pragma unroll
    for (int i = 0; i < V; ++i) r[i] = v;
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) r[i] = lds1(a + dv[i] * (uint32_t)sizeof(T), T());
  }
}

// out = fma(in1, b1, fma(in0, b0, 0)) on V lanes; float lanes go two at a
// time through the packed FP32 FMA (each half is an ordinary
// round-to-nearest fma, so the results are those of the scalar chain)
template <typename T, int V>
__device__ __forceinline__ void fma2terms(const T (&x0)[V], const T (&x1)[V], const T (&b0)[V],
                                          const T (&b1)[V], T (&out)[V]) {
#pragma unroll
  for (int e = 0; e < V; ++e) out[e] = fma_t(x1[e], b1[e], fma_t(x0[e], b0[e], (T)0));
}
template <int V>
__device__ __forceinline__ void fma2terms_f2(const float (&x0)[V], const float (&x1)[V], const float (&b0)[V],
                                             const float (&b1)[V], float (&out)[V]) {
  const float2 z = make_float2(0.f, 0.f);
#pragma unroll
  for (int h = 0; h < V; h += 2) {
    float2 c = __ffma2_rn(make_float2(x0[h], x0[h + 1]), make_float2(b0[h], b0[h + 1]), z);
    c = __ffma2_rn(make_float2(x1[h], x1[h + 1]), make_float2(b1[h], b1[h + 1]), c);
    out[h] = c.x;
    out[h + 1] = c.y;
  }
}
template <>
__device__ __forceinline__ void fma2terms<float, 2>(const float (&x0)[2], const float (&x1)[2], const float (&b0)[2],
                                                    const float (&b1)[2], float (&out)[2]) {
  fma2terms_f2<2>(x0, x1, b0, b1, out);
}
template <>
__device__ __forceinline__ void fma2terms<float, 4>(const float (&x0)[4], const float (&x1)[4], const float (&b0)[4],
                                                    const float (&b1)[4], float (&out)[4]) {
  fma2terms_f2<4>(x0, x1, b0, b1, out);
}

// step I of the chain on the register block a (compile-time indices);
// KIND 1 in place, 2 growth (adds z at bit D), 0 shrink (adds nothing);
// LM: S_I's lane mode (see ld_lanes)
template <typename T, int V, int D, bool FAST, int GROW, int KIND, int I, int LM>
__device__ __forceinline__ void chain_step_m(const K2CParams &cp, uint32_t g, T (&a)[1 << (D + GROW)][V]) {
  constexpr int NB = D + GROW;
  constexpr uint32_t G = chain_deps(D, FAST, GROW, I);
  constexpr uint32_t O = chain_others(D, GROW, I) & ~G;
  constexpr int nG = popc_c(G), nO = popc_c(O);
  constexpr uint32_t XB = 1u << I;
  const int mode = cp.b_vec[I];
#pragma unroll
  for (uint32_t tg = 0; tg < (1u << nG); ++tg) {
    const uint32_t sg = pdep_c(tg, G);
    constexpr int NA = KIND == 2 ? 4 : (KIND == 1 ? 2 : 1);  // added-value combinations
    T b[2][NA][V];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int av = 0; av < NA; ++av)
        ld_lanes<T, V, LM>(g + cp.d[I][(sg | (x ? XB : 0u)) | ((uint32_t)av << NB)], mode, cp.dv[I], b[x][av]);
#pragma unroll
    for (uint32_t to = 0; to < (1u << nO); ++to) {
      const uint32_t s0 = sg | pdep_c(to, O), s1 = s0 | XB;
      if (KIND == 1) {
        T c0[V], c1[V];
        fma2terms<T, V>(a[s0], a[s1], b[0][0], b[1][0], c0);
        fma2terms<T, V>(a[s0], a[s1], b[0][NA - 1], b[1][NA - 1], c1);
#pragma unroll
        for (int e = 0; e < V; ++e) { a[s0][e] = c0[e]; a[s1][e] = c1[e]; }
      } else if (KIND == 2) {
        constexpr uint32_t ZB = 1u << D;
        T c[4][V];
#pragma unroll
        for (int av = 0; av < 4; ++av) fma2terms<T, V>(a[s0], a[s1], b[0][av & (NA - 1)], b[1][av & (NA - 1)], c[av]);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          a[s0][e] = c[0][e];
          a[s1][e] = c[1][e];
          a[(s0 | ZB) & ((1u << NB) - 1u)][e] = c[2][e];
          a[(s1 | ZB) & ((1u << NB) - 1u)][e] = c[3][e];
        }
      } else {
        T c0[V];
        fma2terms<T, V>(a[s0], a[s1], b[0][0], b[1][0], c0);
#pragma unroll
        for (int e = 0; e < V; ++e) a[s0][e] = c0[e];
      }
    }
  }
}

// FAST chains: every step's lanes contiguous (BC 0), or each step
// contiguous, broadcast or per lane (BC 1: one branch per step picks the
// variant); the generic chains follow the runtime mode per load
template <typename T, int V, int D, bool FAST, int BC, int GROW, int KIND, int I>
__device__ __forceinline__ void chain_step(const K2CParams &cp, uint32_t g, T (&a)[1 << (D + GROW)][V]) {
  if (!FAST) chain_step_m<T, V, D, FAST, GROW, KIND, I, 0>(cp, g, a);
  else if (BC && V > 1 && cp.b_vec[I] == 2) chain_step_m<T, V, D, FAST, GROW, KIND, I, 2>(cp, g, a);
  else if (BC && V > 1 && cp.b_vec[I] == 0) chain_step_m<T, V, D, FAST, GROW, KIND, I, 3>(cp, g, a);
  else chain_step_m<T, V, D, FAST, GROW, KIND, I, 1>(cp, g, a);
}

template <typename T, int V, int D, bool FAST, int BC, int GROW, int SHRINK, int I>
struct ChainSteps {
  static __device__ __forceinline__ void run(const K2CParams &cp, const uint32_t (&g)[D],
                                             T (&a)[1 << (D + GROW)][V]) {
    constexpr int KIND = (I == 0 && GROW) ? 2 : ((I == D - 1 && SHRINK) ? 0 : 1);
    chain_step<T, V, D, FAST, BC, GROW, KIND, I>(cp, g[I], a);
    ChainSteps<T, V, D, FAST, BC, GROW, SHRINK, I + 1>::run(cp, g, a);
  }
};
template <typename T, int V, int D, bool FAST, int BC, int GROW, int SHRINK>
struct ChainSteps<T, V, D, FAST, BC, GROW, SHRINK, D> {
  static __device__ __forceinline__ void run(const K2CParams &, const uint32_t (&)[D],
                                             T (&)[1 << (D + GROW)][V]) {}
};

// min over nonzero bit patterns, tracked as (bits - 1) with zero wrapping

// End of a chain launch, after the block's tiles: block 0 writes C_D's
// exponent -- P's and every S_i's (the intermediates are never rescaled) --
// and runs the flush test over the smallest nonzero scaled entries of all
// D + 1 operands (a lower bound on every product the chain forms); every
// block merges its per-lane max and min of |C_D| (smax, smin) into C_D's.
template <typename T, int D>
__device__ __forceinline__ void chain_epilogue(const K2CParams &cp, const unsigned long long *smax,
                                               const unsigned long long *smin) {
  if (blockIdx.x == 0) {
    for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
      const int qp = q & cp.mp.qmask;
      int64_t e = cp.mp.exp[qp] + pow2_exp_of(cp.mp.maxb[qp], T());
      bool any_zero = cp.mp.minb[qp] == kNoMin;
      T lo = any_zero ? (T)0 : from_bits<T>(cp.mp.minb[qp]) * operand_scale<T>(cp.mp, qp, 1);
#pragma unroll
      for (int s = 0; s < D; ++s) {
        const int qs = q & cp.ms[s].qmask;
        e += cp.ms[s].exp[qs] + pow2_exp_of(cp.ms[s].maxb[qs], T());
        if (cp.ms[s].minb[qs] == kNoMin) any_zero = true;
        else lo *= from_bits<T>(cp.ms[s].minb[qs]) * operand_scale<T>(cp.ms[s], qs, 1);
      }
      cp.mc.exp[q] = e;
      if (cp.mc.flags && !any_zero && below_normal(lo)) {
        if (cp.mc.Qc > 1) atomicOr(cp.mc.flags + q, 2u);
        else
          for (int qq = 0; qq < cp.mc.Q; ++qq) atomicOr(cp.mc.flags + qq, 2u);
      }
    }
  }
  for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
    if (smax[q]) atomicMax(cp.mc.maxb + q, smax[q]);
    if (smin[q] != kNoMin) atomicMin(cp.mc.minb + q, smin[q]);
  }
}

template <typename T, int V, int D, bool FAST, int BC, int GROW, int SHRINK>
__global__ void __launch_bounds__(kChainNW * 32 + 32, 1) k2_chain(K2CParams cp) {
  typedef typename Bits<T>::t BT;
  constexpr int NW = kChainNW;
  constexpr int NB = D + GROW;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  __shared__ __align__(8) unsigned long long full[kMaxStagesC], empty[kMaxStagesC], sbar;
  __shared__ uint32_t tile_oc[kMaxStagesC], tile_gb[kMaxChain][kMaxStagesC];
  __shared__ int s_skip;
  const int n_stages = cp.n_stages;
  const uint32_t run_len = 1u << cp.run_log2;
  const uint32_t tile_elems = (uint32_t)cp.nruns * run_len;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
  const uint32_t n_tiles = 1u << (cp.log2_nu + cp.vbits - cp.tb);
  T *stage_buf = reinterpret_cast<T *>(dyn_smem);
  unsigned char *s_area = dyn_smem + (size_t)n_stages * tile_bytes;
  unsigned long long *smax = reinterpret_cast<unsigned long long *>(s_area + cp.s_bytes_off[D]);
  unsigned long long *smin = smax + cp.mc.Qc;
  T *sscale = reinterpret_cast<T *>(smin + cp.mc.Qc);  // [D][Qc]
  const T *P = (const T *)cp.P;
  T *C = (T *)cp.C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Producer state, per lane, set up once: tile offsets advance by a masked
  // add (the tile index's bits are deposited around the chain positions:
  // adding the deposited grid stride with the chain bits held at 1 carries
  // across them); lane r < nruns keeps run r's offsets, lane s < D the
  // segments that gather S_s's per-tile base (no indexed parameter loads
  // and no loops over them inside the tile loop).
  uint32_t p_base = 0, p_oc = 0, p_dstride = 0, p_cstride = 0, p_pmask = 0, p_cmask = 0;
  uint32_t p_run_src = 0, p_run_dst = 0;
  uint32_t g_c[8], g_b[8], g_m[8];
  int g_n = 0;
  if (warp == NW) {
    for (int j = 0; j < cp.n_ins; ++j) p_pmask |= 1u << cp.ins[j];
    for (int j = 0; j < cp.n_insc; ++j) p_cmask |= 1u << cp.insc[j];
    uint32_t b0 = blockIdx.x << cp.tb, c0 = b0, sd = gridDim.x << cp.tb, sc = sd;
    for (int j = 0; j < cp.n_ins; ++j) { b0 = insert0(b0, cp.ins[j]); sd = insert0(sd, cp.ins[j]); }
    for (int j = 0; j < cp.n_insc; ++j) { c0 = insert0(c0, cp.insc[j]); sc = insert0(sc, cp.insc[j]); }
    p_base = b0; p_oc = c0; p_dstride = sd; p_cstride = sc;
    if (lane < cp.nruns) {
      p_run_src = cp.run_off[lane];
      p_run_dst = (uint32_t)lane * run_len;
    }
    if (lane < D) {
      g_n = cp.n_seg[lane];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        g_c[j] = j < g_n ? (uint32_t)cp.seg_c[lane][j] : 0u;
        g_b[j] = j < g_n ? (uint32_t)cp.seg_b[lane][j] : 0u;
        g_m[j] = j < g_n ? (1u << cp.seg_len[lane][j]) - 1u : 0u;
      }
    }
  }
  // tile i into its stage (tiles are produced in order, each call advances
  // the offsets by one grid stride)
  auto produce = [&](uint32_t i) -> bool {
    const int st = (int)(i % (uint32_t)n_stages);
    if (i >= (uint32_t)n_stages &&
        !__all_sync(0xffffffffu, mbar_wait(&empty[st], ((i / n_stages) - 1) & 1)))
      return false;
    const uint32_t base = p_base, oc = p_oc;
    p_base = ((p_base | p_pmask) + p_dstride) & ~p_pmask;
    p_oc = ((p_oc | p_cmask) + p_cstride) & ~p_cmask;
    if (lane < D) {
      uint32_t gb = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) gb |= ((oc >> g_c[j]) & g_m[j]) << g_b[j];
      tile_gb[lane][st] = gb;
    }
    if (lane == 0) {
      tile_oc[st] = oc;
      mbar_expect_tx(&full[st], tile_bytes);
    }
    __syncwarp();
    if (cp.debug_stall && i == 0) return true;
    if (lane < cp.nruns)
      bulk_g2s(stage_buf + (size_t)st * tile_elems + p_run_dst, P + base + p_run_src,
               run_len * (uint32_t)sizeof(T), &full[st]);
    return true;
  };
  // Part 1, independent of the previous launch of the walk (with
  // programmatic dependent launch it overlaps that launch's tail): the
  // barriers and the S_i copies (the S_i and their metadata come from
  // launches that completed before the previous one began).
  if (warp == NW && lane == 0) {
    for (int i = 0; i < n_stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NW);
    }
    mbar_init(&sbar, 1);
    mbar_fence_init();
    mbar_expect_tx(&sbar, cp.s_copy_bytes);
#pragma unroll
    for (int s = 0; s < D; ++s)
      bulk_g2s(s_area + cp.s_bytes_off[s], cp.S[s], (uint32_t)sizeof(T) << cp.s_log2[s], &sbar);
  }
  // Part 2: P, P's metadata and the error word are the previous launch's
  grid_dependency_wait();
  if (threadIdx.x == 0) s_skip = (cp.err && *(volatile uint32_t *)cp.err) ? 1 : 0;
  __syncthreads();
  if (s_skip) {  // an earlier launch of this walk gave up: skip the work
    if (threadIdx.x == 0) mbar_wait(&sbar, 0);  // (the S_i copies land first)
    __syncthreads();
    return;
  }
  uint32_t n_pre = 0;
  if (warp == NW)
    for (; n_pre < (uint32_t)n_stages && blockIdx.x + n_pre * gridDim.x < n_tiles; ++n_pre) produce(n_pre);
  // per-lane scales of each S_i (S_1's times P's when folded)
  for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
    smax[q] = 0;
    smin[q] = kNoMin;
#pragma unroll
    for (int s = 0; s < D; ++s) {
      T v = operand_scale<T>(cp.ms[s], q, 1);
      if (s == 0 && cp.fold_sp) v *= operand_scale<T>(cp.mp, q, 1);
      sscale[s * cp.mc.Qc + q] = v;
    }
  }
  __syncthreads();  // barriers initialised, scales written
  const bool s_landed = __syncthreads_and(mbar_wait(&sbar, 0) ? 1 : 0) != 0;
  if (s_landed) {
#pragma unroll
    for (int s = 0; s < D; ++s) {
      T *dst = reinterpret_cast<T *>(s_area + cp.s_bytes_off[s]);
      const uint32_t n = 1u << cp.s_log2[s];
      const T *sc = sscale + s * cp.mc.Qc;
      const uint32_t qm = (uint32_t)cp.ms[s].qmask;
#pragma unroll 4
      for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) dst[j] *= sc[j & qm];
    }
  } else if (threadIdx.x == 0 && cp.err) {
    atomicOr(cp.err, 1u);
  }
  __syncthreads();

  if (warp == NW) {
    uint32_t i = n_pre;
    bool ok = s_landed;
    for (; ok && blockIdx.x + i * gridDim.x < n_tiles; ++i)
      if (!produce(i)) { ok = false; break; }
    if (lane == 0) {
      if (!ok && cp.err) atomicOr(cp.err, 1u);
      // drain: copies of the last issued tiles may still be in flight
      const uint32_t n_issued = i;
      for (uint32_t j = n_issued > (uint32_t)n_stages ? n_issued - n_stages : 0; j < n_issued; ++j)
        if (!mbar_wait(&full[j % n_stages], (j / n_stages) & 1) && cp.err) atomicOr(cp.err, 1u);
    }
    __syncwarp();
  } else if (s_landed) {
    constexpr uint32_t es = (uint32_t)sizeof(T);
    // J work units per thread per tile (J = 2 doubles the tile, and so the
    // length of its contiguous runs, without more registers)
    const int J = cp.units;
    // per-unit offsets of unit 0 and unit 1, kept in named registers and
    // selected per unit (an array indexed by the runtime unit would live
    // in local memory)
    uint32_t la_0 = 0, la_1 = 0, ocl_0 = 0, ocl_1 = 0, gl_0[D], gl_1[D];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t wl = (threadIdx.x + (uint32_t)j * NW * 32) * V;
      uint32_t la = wl, ocl = wl;
      for (int i = 0; i < cp.n_low; ++i) la = insert0(la, cp.low[i]);
      for (int i = 0; i < cp.n_insc; ++i) ocl = insert0(ocl, cp.insc[i]);
      (j ? la_1 : la_0) = la * es;
      (j ? ocl_1 : ocl_0) = ocl;
#pragma unroll
      for (int s = 0; s < D; ++s) {
        uint32_t g = 0;
        for (int jj = 0; jj < cp.n_seg[s]; ++jj)
          g |= ((ocl >> cp.seg_c[s][jj]) & ((1u << cp.seg_len[s][jj]) - 1u)) << cp.seg_b[s][jj];
        (j ? gl_1[s] : gl_0[s]) = g * es + cp.s_bytes_off[s];
      }
    }
    const uint32_t wl0 = threadIdx.x * V, ocl = ocl_0;
    const uint32_t stage0 = smem_addr(dyn_smem), s_area0 = smem_addr(s_area);
    T sp[V];
#pragma unroll
    for (int e = 0; e < V; ++e)
      sp[e] = (FAST || cp.fold_sp) ? (T)1 : operand_scale<T>(cp.mp, (int)(wl0 + e), 1);
    T tmax[V];
    BT tminm1[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { tmax[e] = (T)0; tminm1[e] = (BT)~(BT)0; }
    for (uint32_t i = 0; blockIdx.x + i * gridDim.x < n_tiles; ++i) {
      const int st = (int)(i % (uint32_t)n_stages);
      const bool landed = __all_sync(0xffffffffu, mbar_wait(&full[st], (i / n_stages) & 1));
      if (!landed) {
        if (lane == 0 && cp.err) atomicOr(cp.err, 1u);
        break;
      }
      for (int j = 0; j < J; ++j) {
        const uint32_t tile = stage0 + (uint32_t)st * tile_bytes + (j ? la_1 : la_0);
        T *cbase = C + (tile_oc[st] | (j ? ocl_1 : ocl_0));
        uint32_t g[D];
#pragma unroll
        for (int s = 0; s < D; ++s) g[s] = s_area0 + (j ? gl_1[s] : gl_0[s]) + tile_gb[s][st] * es;
        T a[1 << NB][V];
#pragma unroll
        for (int s = 0; s < (1 << D); ++s) {
          LdsV<T, V>::ld(tile + cp.pA[s], a[s]);
          if (!FAST) {
#pragma unroll
            for (int e = 0; e < V; ++e) a[s][e] *= sp[e];
          }
        }
        if (j == J - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[st]);  // the stage is in registers
        }
        ChainSteps<T, V, D, FAST, BC, GROW, SHRINK, 0>::run(cp, g, a);
#pragma unroll
        for (int s = 0; s < (1 << NB); ++s) {
          if (SHRINK && ((s >> (D - 1)) & 1)) continue;  // summed away
          vstore<T, V>(cbase + cp.dC[s], a[s]);
#pragma unroll
          for (int e = 0; e < V; ++e) {
            tmax[e] = max_abs(tmax[e], a[s][e]);
            tminm1[e] = min_m1(to_bits(a[s][e]), tminm1[e]);
          }
        }
      }
    }
    const uint32_t qmask_c = (uint32_t)(cp.mc.Qc - 1);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int q = (int)((ocl + e) & qmask_c);
      if (tmax[e] != (T)0) atomicMax(smax + q, abs_bits(tmax[e]));
      if (tminm1[e] != (BT)~(BT)0) atomicMin(smin + q, (unsigned long long)(tminm1[e] + (BT)1));
    }
  }
  __syncthreads();
  grid_dependents_launch();  // this block's tiles are done: the next launch may start
  chain_epilogue<T, D>(cp, smax, smin);
}

// ----------------------------------------- long chains, direct loads
//
// Runs of D = 5..6 frontier eliminations (no growth step): 2^D values per
// work unit and lane, one unit of V lanes (V = 1 in the walks: two lanes of
// 64 states took 254 registers and ran slower) per thread at a time.  The thread loads its unit's
// 2^D values of P straight from global memory (for a fixed chain state a
// warp's lanes read consecutive units when P's lowest indices are kept
// ones), applies the D steps in registers with the step code of k2_chain
// (FAST layout, contiguous lanes, P's scale folded into the staged S_1) and
// stores C_D.  There is no staging ring: 2^D independent loads per thread
// keep enough bytes in flight, and tiles of 64-state units would leave
// bulk copies of only 1 KB.  pA and dC hold element offsets of the chain
// states in P and C_D; units are the assignments of P's other indices.
constexpr int kDirectThreads = 256;

template <typename T, int V>
__device__ __forceinline__ void vload_cs(const T *p, T (&r)[V]) {
  typedef typename VecT<T, V>::t VT;
  VT v = __ldcs(reinterpret_cast<const VT *>(p));
  const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) r[i] = e[i];
}

template <typename T, int V, int D, bool SHRINK>
__global__ void __launch_bounds__(kDirectThreads, V == 1 ? 2 : 1) k2_chain_direct(K2CParams cp) {
  typedef typename Bits<T>::t BT;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  unsigned char *s_area = dyn_smem;
  unsigned long long *smax = reinterpret_cast<unsigned long long *>(s_area + cp.s_bytes_off[D]);
  unsigned long long *smin = smax + cp.mc.Qc;
  __shared__ int s_skip;
  // Part 1, independent of the previous launch of the walk: the raw S_i
  // (they come from launches that completed before the previous one began)
#pragma unroll
  for (int sidx = 0; sidx < D; ++sidx) {
    const T *S = static_cast<const T *>(cp.S[sidx]);
    T *dst = reinterpret_cast<T *>(s_area + cp.s_bytes_off[sidx]);
    for (uint32_t j = threadIdx.x; j < (1u << cp.s_log2[sidx]); j += blockDim.x) dst[j] = __ldg(S + j);
  }
  for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
    smax[q] = 0;
    smin[q] = kNoMin;
  }
  // Part 2: P, its metadata and the error word are the previous launch's
  grid_dependency_wait();
  if (threadIdx.x == 0) s_skip = (cp.err && *(volatile uint32_t *)cp.err) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // an earlier launch of this walk gave up
#pragma unroll
  for (int sidx = 0; sidx < D; ++sidx) {
    T *dst = reinterpret_cast<T *>(s_area + cp.s_bytes_off[sidx]);
    const uint32_t qm = (uint32_t)cp.ms[sidx].qmask;
    for (uint32_t j = threadIdx.x; j < (1u << cp.s_log2[sidx]); j += blockDim.x) {
      T v = operand_scale<T>(cp.ms[sidx], (int)(j & qm), 1);
      if (sidx == 0) v *= operand_scale<T>(cp.mp, (int)(j & qm), 1);
      dst[j] *= v;
    }
  }
  __syncthreads();
  const T *P = static_cast<const T *>(cp.P);
  T *C = static_cast<T *>(cp.C);
  constexpr uint32_t es = (uint32_t)sizeof(T);
  uint32_t pmask = 0, cmask = 0;
  for (int j = 0; j < cp.n_ins; ++j) pmask |= 1u << cp.ins[j];
  for (int j = 0; j < cp.n_insc; ++j) cmask |= 1u << cp.insc[j];
  const uint32_t n_units = 1u << cp.log2_nu;
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t op = u << cp.vbits, oc = u << cp.vbits, dp = stride << cp.vbits, dc = stride << cp.vbits;
  for (int j = 0; j < cp.n_ins; ++j) { op = insert0(op, cp.ins[j]); dp = insert0(dp, cp.ins[j]); }
  for (int j = 0; j < cp.n_insc; ++j) { oc = insert0(oc, cp.insc[j]); dc = insert0(dc, cp.insc[j]); }
  const uint32_t s_area0 = smem_addr(s_area);
  T tmax[V];
  BT tminm1[V];
#pragma unroll
  for (int e = 0; e < V; ++e) { tmax[e] = (T)0; tminm1[e] = (BT)~(BT)0; }
  for (; u < n_units; u += stride) {
    T a[1 << D][V];
#pragma unroll
    for (int st = 0; st < (1 << D); ++st) vload_cs<T, V>(P + (op | cp.pA[st]), a[st]);
    uint32_t g[D];
#pragma unroll
    for (int sidx = 0; sidx < D; ++sidx) {
      uint32_t gg = 0;
      for (int jj = 0; jj < cp.n_seg[sidx]; ++jj)
        gg |= ((oc >> cp.seg_c[sidx][jj]) & ((1u << cp.seg_len[sidx][jj]) - 1u)) << cp.seg_b[sidx][jj];
      g[sidx] = s_area0 + cp.s_bytes_off[sidx] + gg * es;
    }
    ChainSteps<T, V, D, true, 0, 0, SHRINK, 0>::run(cp, g, a);
#pragma unroll
    for (int st = 0; st < (1 << D); ++st) {
      if (SHRINK && ((st >> (D - 1)) & 1)) continue;  // summed away
      vstore<T, V>(C + (oc | cp.dC[st]), a[st]);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        tmax[e] = max_abs(tmax[e], a[st][e]);
        tminm1[e] = min_m1(to_bits(a[st][e]), tminm1[e]);
      }
    }
    op = ((op | pmask) + dp) & ~pmask;
    oc = ((oc | cmask) + dc) & ~cmask;
  }
  // the lane of every unit this thread took (the stride is a multiple of
  // the lane count and the lane bits are C's lowest)
#pragma unroll
  for (int e = 0; e < V; ++e) {
    const int q = (int)((((blockIdx.x * blockDim.x + threadIdx.x) << cp.vbits) + e) & (uint32_t)(cp.mc.Qc - 1));
    if (tmax[e] != (T)0) atomicMax(smax + q, abs_bits(tmax[e]));
    if (tminm1[e] != (BT)~(BT)0) atomicMin(smin + q, (unsigned long long)(tminm1[e] + (BT)1));
  }
  __syncthreads();
  grid_dependents_launch();  // this block's units are done: the next launch may start
  chain_epilogue<T, D>(cp, smax, smin);
}

// ------------------------------------------ runs of chains in one launch
//
// At small batches a chain launch is bound by latency (the launch, the
// previous grid's completion, one tile's copy-in and write-out), not by
// HBM.  k2_chain_seq executes a run of consecutive chains of the walk (one
// T, V, D, FAST, BC; each chain plain, growth or shrink) in one launch.
// Work is handed out in chain order from per-chain atomic tile counters
// (next[c]); a block that took tiles of chain c adds their number to
// done[c] after its stores and its max/min are published (release), and
// block 0 adds one more after writing C's exponents.  Before chain c's
// tiles, a block waits (acquire, bounded by %globaltimer) until done[c-1]
// is complete.  Every tile of chain c-1 was taken by a running block
// before any tile of chain c is handed out, so the waits end without any
// assumption about which blocks are resident.  The chain parameters live
// in global memory with workspace offsets in place of pointers, and are
// copied to shared memory per chain.

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// waits until *cnt >= target or the walk's error word is set (bounded)
__device__ __forceinline__ bool seq_wait_count(const uint32_t *cnt, uint32_t target, const uint32_t *err) {
  if (ld_acquire_u32(cnt) >= target) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (ld_acquire_u32(cnt) >= target) return true;
    if (err && *(volatile const uint32_t *)err) return false;
    if (globaltimer_ns() - t0 > kWaitNs) return false;
  }
}

// a pointer stored as an offset into the workspace, made absolute
template <typename P>
__device__ __forceinline__ void rebase(P *&p, char *ws) {
  p = reinterpret_cast<P *>(ws + reinterpret_cast<uintptr_t>(p));
}

struct ChainSeqShared {
  unsigned long long full[kMaxStagesC], empty[kMaxStagesC], sbar;
  uint32_t tile_oc[kMaxStagesC], tile_gb[kMaxChain][kMaxStagesC];
  int32_t tile_id[kMaxStagesC];
  int skip;
  int owns_first;     // this block took tile 0: C's exponent and the extra count are its
  uint32_t pre_tile;  // the next chain's first tile, taken at the end of this one
};
constexpr uint32_t kNoTile = 0xffffffffu;

__device__ __forceinline__ void chain_seq_rebase(K2CParams &cp, char *ws) {
  rebase(cp.P, ws); rebase(cp.C, ws);
  rebase(cp.mp.exp, ws); rebase(cp.mp.maxb, ws); rebase(cp.mp.minb, ws);
  rebase(cp.mc.exp, ws); rebase(cp.mc.maxb, ws); rebase(cp.mc.minb, ws); rebase(cp.mc.flags, ws);
  rebase(cp.err, ws);
  for (int s = 0; s < kMaxChain; ++s) {
    rebase(cp.S[s], ws);
    rebase(cp.ms[s].exp, ws); rebase(cp.ms[s].maxb, ws); rebase(cp.ms[s].minb, ws);
  }
}

// One chain of a run, by this block: tiles taken from next[c] until none
// are left.
template <typename T, int V, int D, bool FAST, int BC, int GROW, int SHRINK>
__device__ __forceinline__ void chain_seq_pass(const K2CParams &cp, ChainSeqShared &sh, unsigned char *dyn_smem,
                                               uint32_t *next, uint32_t *done, const uint32_t *prev_done,
                                               uint32_t prev_total, bool reinit, bool stall,
                                               const K2CParams *next_src, K2CParams *next_dst, char *ws,
                                               uint32_t *next_ctr) {
  typedef typename Bits<T>::t BT;
  constexpr int NW = kChainNW;
  constexpr int NB = D + GROW;
  const int n_stages = cp.n_stages;
  const uint32_t run_len = 1u << cp.run_log2;
  const uint32_t tile_elems = (uint32_t)cp.nruns * run_len;
  const uint32_t tile_bytes = tile_elems * (uint32_t)sizeof(T);
  const uint32_t n_tiles = 1u << (cp.log2_nu + cp.vbits - cp.tb);
  T *stage_buf = reinterpret_cast<T *>(dyn_smem);
  unsigned char *s_area = dyn_smem + (size_t)n_stages * tile_bytes;
  unsigned long long *smax = reinterpret_cast<unsigned long long *>(s_area + cp.s_bytes_off[D]);
  unsigned long long *smin = smax + cp.mc.Qc;
  T *sscale = reinterpret_cast<T *>(smin + cp.mc.Qc);  // [D][Qc]
  const T *P = (const T *)cp.P;
  T *C = (T *)cp.C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // barriers (re-initialised per chain: every phase of the previous chain
  // has completed) and the S_i copies (the S_i come from earlier launches)
  if (warp == NW && lane == 0) {
    if (reinit) {
      for (int i = 0; i < kMaxStagesC; ++i) {
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&sh.full[i])) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&sh.empty[i])) : "memory");
      }
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&sh.sbar)) : "memory");
    }
    for (int i = 0; i < kMaxStagesC; ++i) {
      mbar_init(&sh.full[i], 1);
      mbar_init(&sh.empty[i], NW);
    }
    mbar_init(&sh.sbar, 1);
    mbar_fence_init();
    mbar_expect_tx(&sh.sbar, cp.s_copy_bytes);
#pragma unroll
    for (int s = 0; s < D; ++s)
      bulk_g2s(s_area + cp.s_bytes_off[s], cp.S[s], (uint32_t)sizeof(T) << cp.s_log2[s], &sh.sbar);
  }
  // the previous chain's outputs and metadata, complete
  if (threadIdx.x == 0) {
    bool ok = true;
    if (prev_done) ok = seq_wait_count(prev_done, prev_total, cp.err);
    if (!ok && cp.err) atomicOr(cp.err, 1u);
    sh.skip = (cp.err && *(volatile uint32_t *)cp.err) ? 1 : 0;
  }
  __syncthreads();
  const bool skip = sh.skip != 0;
  for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
    smax[q] = 0;
    smin[q] = kNoMin;
    if (!skip) {
#pragma unroll
      for (int s = 0; s < D; ++s) {
        T v = operand_scale<T>(cp.ms[s], q, 1);
        if (s == 0 && cp.fold_sp) v *= operand_scale<T>(cp.mp, q, 1);
        sscale[s * cp.mc.Qc + q] = v;
      }
    }
  }
  __syncthreads();
  const bool s_landed = __syncthreads_and(mbar_wait(&sh.sbar, 0) ? 1 : 0) != 0;
  if (!skip && s_landed) {
#pragma unroll
    for (int s = 0; s < D; ++s) {
      T *dst = reinterpret_cast<T *>(s_area + cp.s_bytes_off[s]);
      const uint32_t n = 1u << cp.s_log2[s];
      const T *sc = sscale + s * cp.mc.Qc;
      const uint32_t qm = (uint32_t)cp.ms[s].qmask;
#pragma unroll 4
      for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) dst[j] *= sc[j & qm];
    }
  } else if (!s_landed && threadIdx.x == 0 && cp.err) {
    atomicOr(cp.err, 1u);
  }
  __syncthreads();
  const bool run = !skip && s_landed;
  uint32_t my_tiles = 0;
  if (warp == NW) {
    // ---- producer: tiles from the chain's counter, a sentinel at the end
    if (run) {
      const uint32_t run_src = lane < cp.nruns ? cp.run_off[lane] : 0u;
      const uint32_t run_dst = (uint32_t)lane * run_len;
      fence_proxy_async_global();  // generic-proxy writes of the previous chain, seen by the bulk copies
      bool ok = true;
      uint32_t n_issued = 0;  // tiles whose copies were issued
      for (uint32_t i = 0;; ++i) {
        const int st = (int)(i % (uint32_t)n_stages);
        if (i >= (uint32_t)n_stages &&
            !__all_sync(0xffffffffu, mbar_wait(&sh.empty[st], ((i / n_stages) - 1) & 1))) {
          ok = false;
          break;
        }
        uint32_t t = 0;
        if (lane == 0) t = (i == 0 && sh.pre_tile != kNoTile) ? sh.pre_tile : atomicAdd(next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_tiles) {
          if (lane == 0) {
            sh.tile_id[st] = -1;
            mbar_arrive(&sh.full[st]);  // the sentinel: no copies
          }
          __syncwarp();
          break;
        }
        if (t == 0 && lane == 0) sh.owns_first = 1;
        uint32_t base = t << cp.tb, oc = base;
        for (int j = 0; j < cp.n_ins; ++j) base = insert0(base, cp.ins[j]);
        for (int j = 0; j < cp.n_insc; ++j) oc = insert0(oc, cp.insc[j]);

        if (lane < D) {
          uint32_t gb = 0;
          for (int j = 0; j < cp.n_seg[lane]; ++j)
            gb |= ((oc >> cp.seg_c[lane][j]) & ((1u << cp.seg_len[lane][j]) - 1u)) << cp.seg_b[lane][j];
          sh.tile_gb[lane][st] = gb;
        }
        if (lane == 0) {
          sh.tile_oc[st] = oc;
          sh.tile_id[st] = (int32_t)t;
          mbar_expect_tx(&sh.full[st], tile_bytes);
        }
        __syncwarp();
        if (!(stall && t == 0) && lane < cp.nruns)  // test hook: tile 0's copies never issued
          bulk_g2s(stage_buf + (size_t)st * tile_elems + run_dst, P + base + run_src,
                   run_len * (uint32_t)sizeof(T), &sh.full[st]);
        n_issued = i + 1;
      }
      if (!ok && lane == 0) {
        if (cp.err) atomicOr(cp.err, 1u);
        // a wait gave up: copies of the last issued tiles may be in flight
        for (uint32_t j = n_issued > (uint32_t)n_stages ? n_issued - n_stages : 0; j < n_issued; ++j)
          mbar_wait(&sh.full[j % n_stages], (j / n_stages) & 1);
      }
    }
    __syncwarp();
    // while the consumers finish: the next chain's parameters, and its first
    // tile (every tile of this chain has been taken, so holding one of the
    // next chain cannot keep this chain from completing)
    if (next_src) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(next_src);
      uint32_t *dst = reinterpret_cast<uint32_t *>(next_dst);
      for (uint32_t k = lane; k < sizeof(K2CParams) / 4; k += 32) dst[k] = __ldg(src + k);
      __syncwarp();
      if (lane == 0) {
        chain_seq_rebase(*next_dst, ws);
        sh.pre_tile = atomicAdd(next_ctr, 1u);
      }
      __syncwarp();
    }
  } else if (run) {
    // ---- consumers, as in k2_chain (tiles in the order the producer took them)
    constexpr uint32_t es = (uint32_t)sizeof(T);
    const int J = cp.units;
    uint32_t la_0 = 0, la_1 = 0, ocl_0 = 0, ocl_1 = 0, gl_0[D], gl_1[D];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t wl = (threadIdx.x + (uint32_t)j * NW * 32) * V;
      uint32_t la = wl, ocl = wl;
      for (int i = 0; i < cp.n_low; ++i) la = insert0(la, cp.low[i]);
      for (int i = 0; i < cp.n_insc; ++i) ocl = insert0(ocl, cp.insc[i]);
      (j ? la_1 : la_0) = la * es;
      (j ? ocl_1 : ocl_0) = ocl;
#pragma unroll
      for (int s = 0; s < D; ++s) {
        uint32_t g = 0;
        for (int jj = 0; jj < cp.n_seg[s]; ++jj)
          g |= ((ocl >> cp.seg_c[s][jj]) & ((1u << cp.seg_len[s][jj]) - 1u)) << cp.seg_b[s][jj];
        (j ? gl_1[s] : gl_0[s]) = g * es + cp.s_bytes_off[s];
      }
    }
    const uint32_t wl0 = threadIdx.x * V, ocl = ocl_0;
    const uint32_t stage0 = smem_addr(dyn_smem), s_area0 = smem_addr(s_area);
    T sp[V];
#pragma unroll
    for (int e = 0; e < V; ++e)
      sp[e] = (FAST || cp.fold_sp) ? (T)1 : operand_scale<T>(cp.mp, (int)(wl0 + e), 1);
    T tmax[V];
    BT tminm1[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { tmax[e] = (T)0; tminm1[e] = (BT)~(BT)0; }
    for (uint32_t i = 0;; ++i) {
      const int st = (int)(i % (uint32_t)n_stages);
      const bool landed = __all_sync(0xffffffffu, mbar_wait(&sh.full[st], (i / n_stages) & 1));
      if (!landed) {
        if (lane == 0 && cp.err) atomicOr(cp.err, 1u);
        break;
      }
      if (sh.tile_id[st] < 0) break;  // no more tiles of this chain
      ++my_tiles;
      for (int j = 0; j < J; ++j) {
        const uint32_t tile = stage0 + (uint32_t)st * tile_bytes + (j ? la_1 : la_0);
        T *cbase = C + (sh.tile_oc[st] | (j ? ocl_1 : ocl_0));
        uint32_t g[D];
#pragma unroll
        for (int s = 0; s < D; ++s) g[s] = s_area0 + (j ? gl_1[s] : gl_0[s]) + sh.tile_gb[s][st] * es;
        T a[1 << NB][V];
#pragma unroll
        for (int s = 0; s < (1 << D); ++s) {
          LdsV<T, V>::ld(tile + cp.pA[s], a[s]);
          if (!FAST) {
#pragma unroll
            for (int e = 0; e < V; ++e) a[s][e] *= sp[e];
          }
        }
        if (j == J - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.empty[st]);
        }
        ChainSteps<T, V, D, FAST, BC, GROW, SHRINK, 0>::run(cp, g, a);
#pragma unroll
        for (int s = 0; s < (1 << NB); ++s) {
          if (SHRINK && ((s >> (D - 1)) & 1)) continue;
          vstore<T, V>(cbase + cp.dC[s], a[s]);
#pragma unroll
          for (int e = 0; e < V; ++e) {
            tmax[e] = max_abs(tmax[e], a[s][e]);
            tminm1[e] = min_m1(to_bits(a[s][e]), tminm1[e]);
          }
        }
      }
    }
    const uint32_t qmask_c = (uint32_t)(cp.mc.Qc - 1);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int q = (int)((ocl + e) & qmask_c);
      if (tmax[e] != (T)0) atomicMax(smax + q, abs_bits(tmax[e]));
      if (tminm1[e] != (BT)~(BT)0) atomicMin(smin + q, (unsigned long long)(tminm1[e] + (BT)1));
    }
  }
  __syncthreads();
  // C's exponent and flush test (the block that took tile 0), then this
  // block's max/min
  const bool first = sh.owns_first != 0;
  if (first && run) {
    for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
      const int qp = q & cp.mp.qmask;
      int64_t e = cp.mp.exp[qp] + pow2_exp_of(cp.mp.maxb[qp], T());
      bool any_zero = cp.mp.minb[qp] == kNoMin;
      T lo = any_zero ? (T)0 : from_bits<T>(cp.mp.minb[qp]) * operand_scale<T>(cp.mp, qp, 1);
#pragma unroll
      for (int s = 0; s < D; ++s) {
        const int qs = q & cp.ms[s].qmask;
        e += cp.ms[s].exp[qs] + pow2_exp_of(cp.ms[s].maxb[qs], T());
        if (cp.ms[s].minb[qs] == kNoMin) any_zero = true;
        else lo *= from_bits<T>(cp.ms[s].minb[qs]) * operand_scale<T>(cp.ms[s], qs, 1);
      }
      cp.mc.exp[q] = e;
      if (cp.mc.flags && !any_zero && below_normal(lo)) {
        if (cp.mc.Qc > 1) atomicOr(cp.mc.flags + q, 2u);
        else
          for (int qq = 0; qq < cp.mc.Q; ++qq) atomicOr(cp.mc.flags + qq, 2u);
      }
    }
  }
  if (run)
    for (int q = threadIdx.x; q < cp.mc.Qc; q += blockDim.x) {
      if (smax[q]) atomicMax(cp.mc.maxb + q, smax[q]);
      if (smin[q] != kNoMin) atomicMin(cp.mc.minb + q, smin[q]);
    }
  // every consumer thread counted the same tiles; one count per block
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_proxy_async_global();
    __threadfence();
    red_release_add_u32(done, my_tiles + (first ? 1u : 0u));
    sh.owns_first = (next_src && sh.pre_tile == 0) ? 1 : 0;  // the next chain's tile 0, taken early
    if (!next_src) sh.pre_tile = kNoTile;
  }
  __syncthreads();
}

// seq: the run's chain parameters with workspace offsets for pointers;
// ctr: 2 counters per chain (next, done), zero at the start of the walk
template <typename T, int V, int D, bool FAST, int BC>
__global__ void __launch_bounds__(kChainNW * 32 + 32, 1)
    k2_chain_seq(const K2CParams *__restrict__ seq, int32_t n_chains, uint32_t *ctr, char *ws, int32_t debug_stall) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  __shared__ K2CParams cpb[2];  // this chain's parameters and the next one's
  __shared__ ChainSeqShared sh;
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(seq);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&cpb[0]);
    for (uint32_t i = threadIdx.x; i < sizeof(K2CParams) / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    chain_seq_rebase(cpb[0], ws);
    sh.pre_tile = kNoTile;
    sh.owns_first = 0;
  }
  __syncthreads();
  for (int32_t c = 0; c < n_chains; ++c) {
    const K2CParams &cp = cpb[c & 1];
    uint32_t *next = ctr + 2 * c, *done = next + 1;
    const uint32_t *prev_done = c ? ctr + 2 * (c - 1) + 1 : nullptr;
    const K2CParams &pp = cpb[(c + 1) & 1];  // the previous chain's (until the prefetch overwrites it)
    const uint32_t prev_total = c ? (1u << (pp.log2_nu + pp.vbits - pp.tb)) + 1u : 0u;
    const bool more = c + 1 < n_chains;
    const K2CParams *nsrc = more ? seq + c + 1 : nullptr;
    K2CParams *ndst = &cpb[(c + 1) & 1];
    uint32_t *nctr = more ? ctr + 2 * (c + 1) : nullptr;
    const bool stall = debug_stall && c == 0;
    if (cp.variant == 1)
      chain_seq_pass<T, V, D, FAST, BC, 1, 0>(cp, sh, dyn_smem, next, done, prev_done, prev_total, c > 0, stall,
                                               nsrc, ndst, ws, nctr);
    else if (cp.variant == 2)
      chain_seq_pass<T, V, D, FAST, BC, 0, 1>(cp, sh, dyn_smem, next, done, prev_done, prev_total, c > 0, stall,
                                               nsrc, ndst, ws, nctr);
    else
      chain_seq_pass<T, V, D, FAST, BC, 0, 0>(cp, sh, dyn_smem, next, done, prev_done, prev_total, c > 0, stall,
                                               nsrc, ndst, ws, nctr);
  }
}


// ------------------------------------------------------------ K4 dense
//
// C[b, i, j] = sum_s A[b, i, s] * B[b, s, j] when the node is a real
// batched matrix product: i = A-only kept indices, j = S... B-only kept
// indices, s = summed indices present in both operands, b = batch indices.
// A 64 x 64 output tile per block (256 threads, 4 x 4 outputs each), the
// summed range in chunks of 32 staged in shared memory.  Offsets are bit
// scatters: per index group a table for the tile-local bits plus a base
// for the high bits.  Summation order equals k1_generic's (ascending s,
// serial within 256-term blocks, then a serial sum of the blocks), so the
// two kernels give identical results.

struct K4Params {
  const void *A;
  const void *B;
  void *C;
  Meta ma, mb;
  OutMeta mc;
  int32_t ni, nj, ns, nb;     // bits of i, j, s, b
  int8_t iA[32], iC[32];      // i bit -> position in A, in C
  int8_t jB[32], jC[32];      // j bit -> position in B, in C
  int8_t sA[32], sB[32];      // s bit -> position in A, in B
  int8_t bA[32], bB[32], bC[32];
  int32_t groups_log2;  // split of the summed range (0: none)
  void *partial;        // [2^groups_log2][tiles * 4096] partial sums when split
  int32_t a_i_fast;   // A's lowest (i, s) bit is an i bit: load A along i
  int32_t b_j_fast;   // B's lowest (s, j) bit is a j bit: load B along j
  int32_t c_i_fast;   // C's lowest (i, j) bit is an i bit: threads along i
  int32_t outer_u;    // k4_outer: 1 when C's low 10 bits are i's first 10, 2 when j's
};

__device__ __forceinline__ uint32_t scatter_bits(uint32_t v, const int8_t *pos, int n) {
  uint32_t o = 0;
  for (int t = 0; t < n; ++t)
    if ((v >> t) & 1u) o |= 1u << pos[t];
  return o;
}

template <typename T>
__global__ void __launch_bounds__(256) k4_dense(K4Params p) {
  constexpr int TI = 64, TJ = 64, TK = 32, RI = 4, RJ = 4;
  // the operand chunks, and at the end the 64 x 64 output tile
  // (2 x 32 x 65 = 64 x 65 elements)
  __shared__ T AB[2][TK][TI + 1];
  T (*As)[TI + 1] = AB[0];
  T (*Bs)[TJ + 1] = AB[1];
  T (*Cs)[TJ + 1] = reinterpret_cast<T (*)[TJ + 1]>(&AB[0][0][0]);
  __shared__ uint32_t offA_i[TI], offB_j[TJ], offC_i[TI], offC_j[TJ];
  __shared__ uint32_t offA_s[TK], offB_s[TK];
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  const T *A = (const T *)p.A;
  const T *B = (const T *)p.B;
  T *C = (T *)p.C;
  const uint32_t i_tiles = 1u << (p.ni - 6), j_tiles = 1u << (p.nj - 6);
  const uint32_t n_tiles = i_tiles * j_tiles << p.nb;
  const uint32_t tile = blockIdx.x % n_tiles;
  const uint32_t group = blockIdx.x / n_tiles;
  const uint32_t it = tile % i_tiles, jt = (tile / i_tiles) % j_tiles, bb = tile / (i_tiles * j_tiles);
  // tile-local tables (low 6 bits of i and j, low 5 bits of s)
  for (int x = threadIdx.x; x < TI; x += blockDim.x) {
    offA_i[x] = scatter_bits(x, p.iA, 6);
    offC_i[x] = scatter_bits(x, p.iC, 6);
  }
  for (int x = threadIdx.x; x < TJ; x += blockDim.x) {
    offB_j[x] = scatter_bits(x, p.jB, 6);
    offC_j[x] = scatter_bits(x, p.jC, 6);
  }
  const int tk = p.ns < 5 ? p.ns : 5;  // summed bits per chunk
  const int TKr = 1 << tk;
  for (int x = threadIdx.x; x < TK; x += blockDim.x) {
    offA_s[x] = scatter_bits(x, p.sA, tk);
    offB_s[x] = scatter_bits(x, p.sB, tk);
  }
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  // high parts
  const uint32_t baseA = scatter_bits(it, p.iA + 6, p.ni - 6) | scatter_bits(bb, p.bA, p.nb);
  const uint32_t baseB = scatter_bits(jt, p.jB + 6, p.nj - 6) | scatter_bits(bb, p.bB, p.nb);
  const uint32_t baseC = scatter_bits(it, p.iC + 6, p.ni - 6) | scatter_bits(jt, p.jC + 6, p.nj - 6) |
                         scatter_bits(bb, p.bC, p.nb);
  __syncthreads();
  // every output of the block has the same query lane? the query bits are
  // batch bits (bb), so yes: one scale per operand per block
  const int q = (int)(baseC & (uint32_t)(p.mc.Qc - 1));
  const T sa = operand_scale<T>(p.ma, q, p.mc.scale_inputs);
  const T sb = operand_scale<T>(p.mb, q, p.mc.scale_inputs);
  // output mapping: consecutive threads along whichever of i, j is C's fast index
  const int ty = p.c_i_fast ? (int)(threadIdx.x % 16) : (int)(threadIdx.x / 16);
  const int tx = p.c_i_fast ? (int)(threadIdx.x / 16) : (int)(threadIdx.x % 16);
  T acc[RI][RJ], part[RI][RJ];
#pragma unroll
  for (int r = 0; r < RI; ++r)
#pragma unroll
    for (int c = 0; c < RJ; ++c) acc[r][c] = part[r][c] = (T)0;
  const uint32_t n_s = 1u << p.ns;
  const bool blocked = p.ns > 8;
  const uint32_t s_len = n_s >> p.groups_log2;  // a multiple of 256 when split
  for (uint32_t s0 = group * s_len; s0 < (group + 1) * s_len; s0 += TKr) {
    const uint32_t hiA = scatter_bits(s0 >> tk, p.sA + tk, p.ns - tk);
    const uint32_t hiB = scatter_bits(s0 >> tk, p.sB + tk, p.ns - tk);
    for (int x = threadIdx.x; x < TKr * TI; x += blockDim.x) {
      const int kk = p.a_i_fast ? x / TI : x % TKr, ii = p.a_i_fast ? x % TI : x / TKr;
      As[kk][ii] = __ldg(A + (baseA | hiA | offA_i[ii] | offA_s[kk])) * sa;
    }
    for (int x = threadIdx.x; x < TKr * TJ; x += blockDim.x) {
      const int jj = p.b_j_fast ? x % TJ : x / TKr, kk = p.b_j_fast ? x / TJ : x % TKr;
      Bs[kk][jj] = __ldg(B + (baseB | hiB | offB_j[jj] | offB_s[kk])) * sb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TKr; ++kk) {
      T a[RI], b[RJ];
#pragma unroll
      for (int r = 0; r < RI; ++r) a[r] = As[kk][ty * RI + r];
#pragma unroll
      for (int c = 0; c < RJ; ++c) b[c] = Bs[kk][tx * RJ + c];
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < RJ; ++c) part[r][c] = fma_t(a[r], b[c], part[r][c]);
    }
    __syncthreads();
    if (blocked && ((s0 + TKr) & 255u) == 0) {
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < RJ; ++c) { acc[r][c] += part[r][c]; part[r][c] = (T)0; }
    }
  }
  if (p.groups_log2) {
    // this group's partial sums; k4_reduce adds the groups in order
    T *P = (T *)p.partial + ((size_t)group * n_tiles + tile) * (TI * TJ);
#pragma unroll
    for (int r = 0; r < RI; ++r)
#pragma unroll
      for (int c = 0; c < RJ; ++c) P[(ty * RI + r) * TJ + tx * RJ + c] = acc[r][c];
    return;
  }
  // the tile through shared memory, then stored with C's fast index along
  // consecutive threads (the chunk loop ended with a barrier)
#pragma unroll
  for (int r = 0; r < RI; ++r)
#pragma unroll
    for (int c = 0; c < RJ; ++c) Cs[ty * RI + r][tx * RJ + c] = blocked ? acc[r][c] : part[r][c];
  __syncthreads();
  T tmax = (T)0, tmin = (T)INFINITY;
  for (int x = threadIdx.x; x < TI * TJ; x += blockDim.x) {
    const int ii = p.c_i_fast ? x % TI : x / TJ, jj = p.c_i_fast ? x / TI : x % TJ;
    const T v = Cs[ii][jj];
    C[baseC | offC_i[ii] | offC_j[jj]] = v;
    track(v, tmax, tmin);
  }
  publish_warp(smax, smin, q, tmax, tmin, 1);
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// Outer products with a short summed range (at most 2 summed bits, one
// query lane): C's lowest 10 bits are the first 10 free bits u of one
// operand U, in order; v are the other operand's free bits.  A block owns
// 1024 consecutive u (4 per thread, one vector store each) and 64 values of
// v, for one value of u's and v's high bits and of the batch bits.  Each
// thread keeps its U entries in registers and loops over the 64 v, whose
// entries are staged in shared memory; every output is written once.  The
// summed terms are added as k4_dense adds them (fma chain over s in order
// from 0, operands scaled first), so the values are the same bits.
template <typename T, int NS>
__global__ void __launch_bounds__(256) k4_outer(K4Params p) {
  // NS = 2^ns summed terms, a template parameter: with a runtime count the
  // unrolled term loop issued predicated-off products on the (scarce)
  // float64 pipe
  constexpr int LU = 10, LV = 6, NV = 1 << LV;
  __shared__ T Vs[NV][4];
  __shared__ uint32_t offC_v[NV];
  __shared__ unsigned long long smax[1], smin[1];
  const bool ui = p.outer_u == 1;
  const int nu = ui ? p.ni : p.nj, nv = ui ? p.nj : p.ni, ns = p.ns;
  const int8_t *uU = ui ? p.iA : p.jB, *uC = ui ? p.iC : p.jC;
  const int8_t *vV = ui ? p.jB : p.iA, *vC = ui ? p.jC : p.iC;
  const int8_t *sU = ui ? p.sA : p.sB, *sV = ui ? p.sB : p.sA;
  const int8_t *bU = ui ? p.bA : p.bB, *bV = ui ? p.bB : p.bA;
  const T *U = (const T *)(ui ? p.A : p.B);
  const T *Vop = (const T *)(ui ? p.B : p.A);
  const T su = operand_scale<T>(ui ? p.ma : p.mb, 0, p.mc.scale_inputs);
  const T sv = operand_scale<T>(ui ? p.mb : p.ma, 0, p.mc.scale_inputs);
  const uint32_t u_tiles = 1u << (nu - LU), v_tiles = 1u << (nv - LV);
  const uint32_t ut = blockIdx.x % u_tiles, vt = (blockIdx.x / u_tiles) % v_tiles;
  const uint32_t bb = blockIdx.x / (u_tiles * v_tiles);
  if (threadIdx.x == 0) { smax[0] = 0; smin[0] = kNoMin; }
  const uint32_t baseV = scatter_bits(vt, vV + LV, nv - LV) | scatter_bits(bb, bV, p.nb);
  for (int x = threadIdx.x; x < NV * NS; x += blockDim.x) {
    const int vv = x >> ns, k = x & (NS - 1);
    Vs[vv][k] = __ldg(Vop + (baseV | scatter_bits(vv, vV, LV) | scatter_bits(k, sV, ns))) * sv;
  }
  for (int x = threadIdx.x; x < NV; x += blockDim.x) offC_v[x] = scatter_bits(x, vC, LV);
  // this thread's 4 values of u and their entries of U, scaled
  const uint32_t baseU = scatter_bits(ut, uU + LU, nu - LU) | scatter_bits(bb, bU, p.nb);
  T a[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint32_t o = baseU | scatter_bits(threadIdx.x * 4u + e, uU, LU);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[e][k] = k < NS ? __ldg(U + (o | scatter_bits(k, sU, ns))) * su : (T)0;
  }
  const uint32_t baseC = scatter_bits(ut, uC + LU, nu - LU) | scatter_bits(vt, vC + LV, nv - LV) |
                         scatter_bits(bb, p.bC, p.nb);
  T *C = (T *)p.C + baseC + threadIdx.x * 4u;
  __syncthreads();
  T tmax = (T)0, tmin = (T)INFINITY;
#pragma unroll 4
  for (int vv = 0; vv < NV; ++vv) {
    T c[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      T acc = (T)0;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < NS) acc = fma_t(a[e][k], Vs[vv][k], acc);
      c[e] = acc;
      track_fast(acc, tmax, tmin);
    }
    T *dst = C + offC_v[vv];
    if constexpr (sizeof(T) == 4) {
      __stcs(reinterpret_cast<float4 *>(dst), make_float4(c[0], c[1], c[2], c[3]));
    } else {
      __stcs(reinterpret_cast<double2 *>(dst), make_double2(c[0], c[1]));
      __stcs(reinterpret_cast<double2 *>(dst) + 1, make_double2(c[2], c[3]));
    }
  }
  publish_warp(smax, smin, 0, tmax, tmin, 1);
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// Split summed range: C = sum over groups (in group order) of the partials.
// 16 blocks per 64 x 64 tile, one output per thread; each thread requests
// eight groups' partials at a time and adds them in group order.
template <typename T>
__global__ void __launch_bounds__(256) k4_reduce(K4Params p) {
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  const uint32_t i_tiles = 1u << (p.ni - 6), j_tiles = 1u << (p.nj - 6);
  const uint32_t n_tiles = i_tiles * j_tiles << p.nb;
  const uint32_t tile = blockIdx.x >> 4;
  const uint32_t it = tile % i_tiles, jt = (tile / i_tiles) % j_tiles, bb = tile / (i_tiles * j_tiles);
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  const uint32_t baseC = scatter_bits(it, p.iC + 6, p.ni - 6) | scatter_bits(jt, p.jC + 6, p.nj - 6) |
                         scatter_bits(bb, p.bC, p.nb);
  __syncthreads();
  const int q = (int)(baseC & (uint32_t)(p.mc.Qc - 1));
  const uint32_t x = ((blockIdx.x & 15u) << 8) | threadIdx.x;  // output within the tile
  const uint32_t ii = x / 64, jj = x % 64;
  const uint32_t G = 1u << p.groups_log2;
  const T *P = (const T *)p.partial + (size_t)tile * 4096 + x;
  const size_t gstride = (size_t)n_tiles * 4096;
  T v = (T)0;
  for (uint32_t g = 0; g < G; g += 8) {
    T t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = g + u < G ? P[(size_t)(g + u) * gstride] : (T)0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (g + u < G) v += t[u];
  }
  ((T *)p.C)[baseC | scatter_bits(ii, p.iC, 6) | scatter_bits(jj, p.jC, 6)] = v;
  T tmax = (T)0, tmin = (T)INFINITY;
  track(v, tmax, tmin);
  publish_warp(smax, smin, q, tmax, tmin, 1);
  __syncthreads();
  finish_meta<T>(p.ma, p.mb, p.mc, smax, smin);
}

// ------------------------------------------------ K4 on the tensor cores
//
// The dense batched product of K4 in float32 on the 5th-generation tensor
// cores (tcgen05, kind::tf32) with the 3xTF32 split: every operand value x
// is stored as hi = x with the low 13 mantissa bits cleared (exactly a
// TF32 value) and lo = x - hi (exact in float32, TF32 to within a few
// bits), and C += A_hi.B_hi + A_hi.B_lo + A_lo.B_hi accumulates in float32
// in tensor memory: about float32 accuracy at a tensor-core rate.
//
// Two launches.  k4_tc_pack rewrites each operand once, scaled and split,
// into blocks of (batch assignment, 128 or N rows, 16 summed terms) in the
// canonical K-major layout without swizzle (8-row x 16-byte core
// matrices: 128 bytes between neighbours along K, 512 between 8-row
// groups), hi block then lo block.  k4_tc is persistent (one block per
// SM) and warp-specialised: warp 0 moves each chunk's A and B blocks into
// a ring of shared-memory stages with two bulk async copies (full/empty
// mbarriers), warp 1 owns 2 x N columns of tensor memory and issues the
// six MMAs of a chunk (two steps of K = 8, three products each), warps
// 2..5 read a finished 128 x N accumulator back with tcgen05.ld and write
// C while the MMAs of the next tile go to the other accumulator.  Waits are
// bounded by %globaltimer; on timeout the block records the error, lets
// its copies and MMAs in flight finish (bounded) and frees its tensor
// memory.  The summation order differs from the scalar kernels: results
// agree within float32 rounding, not bit for bit.

constexpr int kTcM = 128, kTcKC = 16, kTcStages = 4, kTcThreads = 192;
constexpr uint32_t kTcRowGroup = 8u * kTcKC * 4u;  // bytes between 8-row groups (512)

struct TcPackParams {
  const float *X;           // operand (bit-scattered layout)
  float *Xp;                // packed: [batch][row tile][chunk][hi, lo][rows x 16]
  Meta m;                   // the operand's metadata (scale on load)
  int32_t scale_inputs;
  int32_t rows_log2;        // log2 rows per block (7 or 8)
  int32_t nr, ns, nb;       // row, summed and batch bits of the operand
  int8_t r_pos[32], s_pos[32], b_pos[32];  // bit -> position in X
  int8_t bC[32];            // batch bit -> position in C (query lane of the block)
  int32_t Qc;
  int32_t row_fast;         // X's lowest (row, summed) bit is a row bit
};

// byte offset of element (row m, summed k) inside a packed rows x 16 block
__device__ __forceinline__ uint32_t tc_off(uint32_t m, uint32_t k) {
  return (m >> 3) * kTcRowGroup + (k >> 2) * 128u + (m & 7u) * 16u + (k & 3u) * 4u;
}

// One block per packed (batch, row tile, chunk): each thread loads four
// consecutive summed terms of one row and stores them as one 16-byte hi
// and one 16-byte lo vector.
__global__ void __launch_bounds__(256) k4_tc_pack(TcPackParams p) {
  __shared__ uint32_t off_r[256], off_s[kTcKC];
  const uint32_t R = 1u << p.rows_log2;
  const uint32_t n_chunks = 1u << (p.ns - 4), n_rt = 1u << (p.nr - p.rows_log2);
  const uint32_t c = blockIdx.x % n_chunks, rt = (blockIdx.x / n_chunks) % n_rt;
  const uint32_t bb = blockIdx.x / (n_chunks * n_rt);
  for (uint32_t x = threadIdx.x; x < R; x += blockDim.x) off_r[x] = scatter_bits(x, p.r_pos, p.rows_log2);
  if (threadIdx.x < kTcKC) off_s[threadIdx.x] = scatter_bits(threadIdx.x, p.s_pos, 4);
  __syncthreads();
  const uint32_t base = scatter_bits(rt, p.r_pos + p.rows_log2, p.nr - p.rows_log2) |
                        scatter_bits(c, p.s_pos + 4, p.ns - 4) | scatter_bits(bb, p.b_pos, p.nb);
  const int q = (int)(scatter_bits(bb, p.bC, p.nb) & (uint32_t)(p.Qc - 1));
  const float sc = operand_scale<float>(p.m, q, p.scale_inputs);
  unsigned char *dst = reinterpret_cast<unsigned char *>(p.Xp) + (size_t)blockIdx.x * 2u * R * kTcKC * 4u;
  for (uint32_t x = threadIdx.x; x < R * (kTcKC / 4); x += blockDim.x) {
    const uint32_t m = p.row_fast ? x % R : x / (kTcKC / 4), kq = p.row_fast ? x / R : x % (kTcKC / 4);
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float v = __ldg(p.X + (base | off_r[m] | off_s[kq * 4 + t])) * sc;
      h[t] = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      l[t] = v - h[t];
    }
    const uint32_t o = tc_off(m, kq * 4);
    *reinterpret_cast<float4 *>(dst + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(dst + R * kTcKC * 4u + o) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
  // start address, leading byte offset (neighbour core matrix along K),
  // stride byte offset (next 8-row group), descriptor version 1, no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((128u >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kTcRowGroup >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::tf32 instruction descriptor: float32 accumulator, TF32 A and B,
// both K-major, N columns, M = 128 rows
template <int N>
struct TcIdesc {
  static constexpr uint32_t value = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                                    ((uint32_t)(kTcM >> 4) << 24);
};

template <int N>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(TcIdesc<N>::value), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// bounded wait that also gives up once another role of the block failed
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, uint32_t parity, volatile int *fail) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (*fail) return false;
    if (globaltimer_ns() - t0 > kWaitNs) return false;
  }
}

template <int N>
struct TcShape {
  static constexpr uint32_t a_bytes = 2u * kTcM * kTcKC * 4u;  // hi + lo block of A (16 KB)
  static constexpr uint32_t b_bytes = 2u * N * kTcKC * 4u;     // hi + lo block of B
  static constexpr uint32_t stage = a_bytes + b_bytes;
  static constexpr uint32_t smem = kTcStages * stage + 4u * 32u * 33u * 4u;  // ring + epilogue transposes
  static constexpr uint32_t tmem_cols = 2u * N;                              // two accumulators
};

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
    k4_tc(K4Params p, const float *__restrict__ Ap, const float *__restrict__ Bp, uint32_t *err) {
  using S = TcShape<N>;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long full[kTcStages], empty[kTcStages], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t offC_i[kTcM], offC_j[N];
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  __shared__ int s_fail;
  volatile int *fail = &s_fail;
  float *C = (float *)p.C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nlog = N == 256 ? 8 : 7;
  const uint32_t i_tiles = 1u << (p.ni - 7), j_tiles = 1u << (p.nj - nlog);
  const uint32_t n_tiles = (i_tiles * j_tiles) << p.nb;
  const uint32_t n_chunks = 1u << (p.ns - 4);
  for (int x = threadIdx.x; x < kTcM; x += blockDim.x) offC_i[x] = scatter_bits((uint32_t)x, p.iC, 7);
  for (int x = threadIdx.x; x < N; x += blockDim.x) offC_j[x] = scatter_bits((uint32_t)x, p.jC, nlog);
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) { smax[q] = 0; smin[q] = kNoMin; }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull[a], 1); mbar_init(&tempty[a], 4); }
    mbar_init(&drain, 1);
    mbar_fence_init();
    s_fail = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(S::tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t ring = smem_addr(tc_smem);

  if (warp == 0) {
    // ---- producer: one elected lane moves each chunk's two packed blocks
    if (lane == 0) {
      uint32_t fill = 0;
      for (uint32_t t = blockIdx.x; t < n_tiles && !*fail; t += gridDim.x) {
        const uint32_t jt = t % j_tiles, it = (t / j_tiles) % i_tiles, bb = t / (i_tiles * j_tiles);
        const unsigned char *a = reinterpret_cast<const unsigned char *>(Ap) +
                                 (size_t)((bb * i_tiles + it) * n_chunks) * S::a_bytes;
        const unsigned char *b = reinterpret_cast<const unsigned char *>(Bp) +
                                 (size_t)((bb * j_tiles + jt) * n_chunks) * S::b_bytes;
        for (uint32_t c = 0; c < n_chunks; ++c, ++fill) {
          const uint32_t s = fill % kTcStages;
          if (fill >= (uint32_t)kTcStages && !tc_wait(&empty[s], ((fill / kTcStages) - 1) & 1, fail)) {
            *fail = 1;
            break;
          }
          mbar_expect_tx(&full[s], S::stage);
          bulk_g2s(tc_smem + s * S::stage, a + (size_t)c * S::a_bytes, S::a_bytes, &full[s]);
          bulk_g2s(tc_smem + s * S::stage + S::a_bytes, b + (size_t)c * S::b_bytes, S::b_bytes, &full[s]);
        }
        if (*fail) break;
      }
      // every copy issued has landed before the block may exit
      const uint32_t first = fill > (uint32_t)kTcStages ? fill - kTcStages : 0;
      for (uint32_t f = first; f < fill; ++f)
        if (!mbar_wait(&full[f % kTcStages], (f / kTcStages) & 1)) *fail = 1;
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t fill = 0, lt = 0;
      bool issued = false;
      for (uint32_t t = blockIdx.x; t < n_tiles && !*fail; t += gridDim.x, ++lt) {
        const uint32_t acc = lt & 1u;
        if (lt >= 2 && !tc_wait(&tempty[acc], ((lt >> 1) - 1) & 1, fail)) { *fail = 1; break; }
        tc_fence_after();
        const uint32_t d = tmem + acc * (uint32_t)N;
        for (uint32_t c = 0; c < n_chunks; ++c, ++fill) {
          const uint32_t s = fill % kTcStages;
          if (!tc_wait(&full[s], (fill / kTcStages) & 1, fail)) { *fail = 1; break; }
          tc_fence_after();
          const uint32_t a0 = ring + s * S::stage, b0 = a0 + S::a_bytes;
#pragma unroll
          for (uint32_t kk = 0; kk < (uint32_t)(kTcKC / 8); ++kk) {
            const uint64_t ahi = tc_smem_desc(a0 + kk * 256u), alo = tc_smem_desc(a0 + S::a_bytes / 2 + kk * 256u);
            const uint64_t bhi = tc_smem_desc(b0 + kk * 256u), blo = tc_smem_desc(b0 + S::b_bytes / 2 + kk * 256u);
            tc_mma<N>(d, alo, bhi, (c | kk) != 0u);
            tc_mma<N>(d, ahi, blo, 1u);
            tc_mma<N>(d, ahi, bhi, 1u);
          }
          issued = true;
          tc_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (*fail) break;
        tc_commit(&tfull[acc]);  // the accumulator is complete
      }
      // every MMA issued has finished before tensor memory is freed
      if (issued) {
        tc_commit(&drain);
        if (!mbar_wait(&drain, 0)) *fail = 1;
      }
    }
  } else {
    // ---- epilogue: warp w reads lanes 32 (w mod 4) .. + 31 of the accumulator
    const uint32_t quarter = (uint32_t)warp & 3u;
    const uint32_t row = quarter * 32u + (uint32_t)lane;
    float *tr = reinterpret_cast<float *>(tc_smem + kTcStages * S::stage) + (warp - 2) * 32 * 33;
    uint32_t lt = 0;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      const uint32_t acc = lt & 1u;
      const bool ok = tc_wait(&tfull[acc], (lt >> 1) & 1, fail);
      if (__any_sync(0xffffffffu, !ok)) { if (lane == 0) *fail = 1; break; }
      tc_fence_after();
      const uint32_t jt = t % j_tiles, it = (t / j_tiles) % i_tiles, bb = t / (i_tiles * j_tiles);
      const uint32_t baseC = scatter_bits(it, p.iC + 7, p.ni - 7) | scatter_bits(jt, p.jC + nlog, p.nj - nlog) |
                             scatter_bits(bb, p.bC, p.nb);
      const int q = (int)(baseC & (uint32_t)(p.mc.Qc - 1));
      float tmax = 0.f, tmin = INFINITY;
#pragma unroll 1
      for (uint32_t col = 0; col < (uint32_t)N; col += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((quarter * 32u) << 16) + acc * (uint32_t)N + col;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (p.c_i_fast) {
          // lanes are consecutive rows: each column is one coalesced store
          const uint32_t ci = baseC | offC_i[row];
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float v = __uint_as_float(r[k]);
            C[ci | offC_j[col + (uint32_t)k]] = v;
            track(v, tmax, tmin);
          }
        } else {
          // transpose 32 x 32 through shared memory: lanes along the columns
#pragma unroll
          for (int k = 0; k < 32; ++k) tr[lane * 33 + k] = __uint_as_float(r[k]);
          __syncwarp();
          const uint32_t cj = baseC | offC_j[col + (uint32_t)lane];
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const float v = tr[rr * 33 + lane];
            C[cj | offC_i[quarter * 32u + (uint32_t)rr]] = v;
            track(v, tmax, tmin);
          }
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);  // the accumulator may be overwritten
      publish_warp(smax, smin, q, tmax, tmin, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_fail && threadIdx.x == 0 && err) atomicOr(err, 1u);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::tmem_cols)
                 : "memory");
  if (!s_fail) finish_meta<float>(p.ma, p.mb, p.mc, smax, smin);
}

// ------------------------------------------------------ small-node phase
//
// Every node whose whole subtree is small (bucket products of clause
// tensors and weight vectors, the small formulas of a batch of queries)
// runs inside one persistent launch at the start of the walk: a task is a
// chunk of one node's outputs; a block takes tasks from an atomic counter
// in post-order and waits (bounded by %globaltimer, one second) until the
// node's children are complete.  Tensors produced inside the launch are
// read through L2 (ld.global.cg).

struct SNode {
  int64_t a, b, c;            // byte offsets in the workspace
  int64_t ma, mb, mc;         // first metadata slot of A, B, C
  int32_t qmask_a, qmask_b, Qc;
  int32_t dep_a, dep_b;       // small-phase node of each child (-1: a leaf)
  int32_t n_chunks, chunk_log2;
  int32_t rC, k;
  int8_t ti, ta, to, pad;
  int8_t posA[16], posB[16], sposA[8], sposB[8];
  // one-block walk (nodes ordered by level): the node's lookup tables at
  // word lut_base of its level's tables, its outputs at out_base of the
  // level's outputs, and one past the level's last node
  int32_t lut_base, out_base, level_end, pad2;
};

struct STask {
  int32_t node, chunk;
};

struct SmallArgs {
  char *ws;
  const SNode *nodes;
  const STask *tasks;
  int32_t n_tasks;
  int32_t Q;                  // query lanes of the flags array
  uint32_t *next, *done, *err, *flags;
  int64_t *mexp;
  unsigned long long *mmax, *mmin;
};

__device__ __forceinline__ bool wait_ctr(const uint32_t *ctr, uint32_t target) {
  if (*(volatile const uint32_t *)ctr >= target) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i) {
      __nanosleep(64);
      if (*(volatile const uint32_t *)ctr >= target) return true;
    }
    if (globaltimer_ns() - t0 > 1000000000ull) return false;
  }
}

// The node's per-byte lookup tables (they depend on the node alone, so they
// are built before its children are waited for, and kept while a block
// takes consecutive chunks of one node): rows 0-1 A, 2-3 B (output bits),
// 4 A, 5 B (summed bits).  Entry v is the OR over v's set bits of that
// bit's offset, built as the OR of two 16-entry nibble tables.
__device__ __forceinline__ void small_lut(const SNode &nd, uint32_t (*lut)[256], uint32_t (*bits)[8],
                                          uint32_t (*nib)[2][16]) {
  if (threadIdx.x < 6 * 8) {
    const int row = threadIdx.x >> 3, bit = threadIdx.x & 7;
    uint32_t o = 0;
    if (row < 4) {
      const int j = (row & 1) * 8 + bit;
      const int8_t pos = row < 2 ? nd.posA[j] : nd.posB[j];
      if (j < nd.rC && pos >= 0) o = 1u << pos;
    } else if (bit < nd.k) {
      const int8_t pos = row == 4 ? nd.sposA[bit] : nd.sposB[bit];
      if (pos >= 0) o = 1u << pos;
    }
    bits[row][bit] = o;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * 32; i += blockDim.x) {
    const int row = i >> 5, h = (i >> 4) & 1, v = i & 15;
    uint32_t o = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if ((v >> t) & 1) o |= bits[row][4 * h + t];
    nib[row][h][v] = o;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * 256; i += blockDim.x) {
    const int row = i >> 8, v = i & 255;
    lut[row][v] = nib[row][0][v & 15] | nib[row][1][v >> 4];
  }
}

template <typename TI, typename TA, typename TO>
__device__ void small_task(const SmallArgs &sa_, const SNode &nd, int chunk, uint32_t (*lut)[256],
                           TA *scl, unsigned long long *smax, unsigned long long *smin) {
  char *ws = sa_.ws;
  const TI *A = (const TI *)(ws + nd.a);
  const TI *B = (const TI *)(ws + nd.b);
  TO *C = (TO *)(ws + nd.c);
  // per-lane operand scales (their max patterns are final: children done);
  // chunk 0 also writes C's exponents and runs the flush test now, from the
  // children's metadata alone (off the path that waits for the outputs)
  for (int q = threadIdx.x; q < nd.Qc; q += blockDim.x) {
    const int qa = q & nd.qmask_a, qb = q & nd.qmask_b;
    const unsigned long long xa = __ldcg(sa_.mmax + nd.ma + qa), xb = __ldcg(sa_.mmax + nd.mb + qb);
    scl[q] = (TA)pow2_scale(pow2_exp_of(xa, TI()), TI());
    scl[nd.Qc + q] = (TA)pow2_scale(pow2_exp_of(xb, TI()), TI());
    smax[q] = 0;
    smin[q] = kNoMin;
    if (chunk == 0) {
      sa_.mexp[nd.mc + q] = __ldcg(sa_.mexp + nd.ma + qa) + pow2_exp_of(xa, TI()) +
                            __ldcg(sa_.mexp + nd.mb + qb) + pow2_exp_of(xb, TI());
      const unsigned long long na = __ldcg(sa_.mmin + nd.ma + qa), nb = __ldcg(sa_.mmin + nd.mb + qb);
      if (na != kNoMin && nb != kNoMin) {
        const TI lo = (from_bits<TI>(na) * pow2_scale(pow2_exp_of(xa, TI()), TI())) *
                      (from_bits<TI>(nb) * pow2_scale(pow2_exp_of(xb, TI()), TI()));
        if (below_normal(lo)) {
          if (nd.Qc > 1) atomicOr(sa_.flags + q, 2u);
          else
            for (int qq = 0; qq < sa_.Q; ++qq) atomicOr(sa_.flags + qq, 2u);
        }
      }
    }
  }
  __syncthreads();
  const uint32_t o0 = (uint32_t)chunk << nd.chunk_log2, o1 = o0 + (1u << nd.chunk_log2);
  const uint32_t ns = 1u << nd.k;
  // a thread's outputs share one query lane when the lanes divide the block
  // size (o advances by blockDim): its max/min are then folded across the
  // warp's lanes of that query before the shared atomics; otherwise every
  // output publishes
  const bool lane_fixed = nd.Qc <= (int)blockDim.x;
  TO tmax = (TO)0, tmin = (TO)INFINITY;
  for (uint32_t o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const uint32_t bA = lut[0][o & 255] | lut[1][(o >> 8) & 255];
    const uint32_t bB = lut[2][o & 255] | lut[3][(o >> 8) & 255];
    const int q = (int)(o & (uint32_t)(nd.Qc - 1));
    const TA sa = scl[q], sb = scl[nd.Qc + q];
    TA acc = (TA)0;
    for (uint32_t s = 0; s < ns; ++s) {
      const TA a = (TA)__ldcg(A + (bA | lut[4][s])) * sa;
      const TA b = (TA)__ldcg(B + (bB | lut[5][s])) * sb;
      acc = fma_t(a, b, acc);
    }
    const TO c = (TO)acc;
    C[o] = c;
    if (lane_fixed) {
      track(c, tmax, tmin);
    } else {
      const unsigned long long bits = abs_bits(c);
      if (bits) {
        atomicMax(smax + q, bits);
        atomicMin(smin + q, bits);
      }
    }
  }
  if (lane_fixed)
    publish_warp(smax, smin, (int)((o0 + threadIdx.x) & (uint32_t)(nd.Qc - 1)), tmax, tmin,
                 nd.Qc < 32 ? nd.Qc : 32);
  __syncthreads();
  for (int q = threadIdx.x; q < nd.Qc; q += blockDim.x) {
    if (smax[q]) atomicMax(sa_.mmax + nd.mc + q, smax[q]);
    if (smin[q] != kNoMin) atomicMin(sa_.mmin + nd.mc + q, smin[q]);
  }
}

__global__ void __launch_bounds__(kThreads) k_small_phase(SmallArgs a) {
  __shared__ uint32_t lut[6][256];
  __shared__ uint32_t lut_bits[6][8], lut_nib[6][2][16];
  __shared__ double scl_d[2 * kMaxQ];
  __shared__ unsigned long long smax[kMaxQ], smin[kMaxQ];
  __shared__ int s_task, s_ok;
  int lut_node = -1;  // node whose tables the block holds
  for (;;) {
    if (threadIdx.x == 0) s_task = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int t = s_task;
    if (t >= a.n_tasks) break;
    const STask task = a.tasks[t];
    const SNode &nd = a.nodes[task.node];
    if (task.node != lut_node) {  // overlaps the wait for the children
      small_lut(nd, lut, lut_bits, lut_nib);
      lut_node = task.node;
    }
    if (threadIdx.x == 0) {
      bool ok = *(volatile uint32_t *)a.err == 0;
      if (ok && nd.dep_a >= 0) ok = wait_ctr(a.done + nd.dep_a, (uint32_t)a.nodes[nd.dep_a].n_chunks);
      if (ok && nd.dep_b >= 0) ok = wait_ctr(a.done + nd.dep_b, (uint32_t)a.nodes[nd.dep_b].n_chunks);
      if (!ok) atomicOr(a.err, 1u);
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (nd.ti == 1) small_task<double, double, double>(a, nd, task.chunk, lut, scl_d, smax, smin);
    else if (nd.to == 1) small_task<float, double, double>(a, nd, task.chunk, lut, scl_d, smax, smin);
    else small_task<float, float, float>(a, nd, task.chunk, lut, reinterpret_cast<float *>(scl_d), smax, smin);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // outputs and metadata before the completion count
      atomicAdd(a.done + task.node, 1u);
    }
  }
}

// --------------------------------------------------------------- leaves

// Pointers that change from call to call; read from device memory so a
// captured graph can be replayed with new inputs and outputs.
struct IoDesc {
  const double *w_pos;
  const double *w_neg;
  double *mant;
  int64_t *exp2;
  uint32_t *flags;
  // index slicing (Alg. 3): this walk's slice assignment (bit k fixes
  // slice_var[k]); accumulate != 0 adds the result to what the outputs hold
  uint64_t slice;
  int32_t accumulate;
  int32_t n_slice;
  int32_t slice_var[24];
  // slice assignments along the lanes (0: every lane has `slice`): lane l
  // (l < n_lanes; padding lanes repeat lane n_lanes - 1) has slice
  // slice + l / lanes_per_slice
  int32_t lanes_per_slice;
  int32_t n_lanes;
};

struct ClauseLeaf {
  int64_t off;      // element offset in the tensor arena
  int64_t meta;     // metadata slot
  uint64_t fals;    // falsifying assignment
  int32_t rank;
  uint32_t smask;   // index slicing: the clause's sliced variables (slice bits)
  uint32_t sfals;   // ... and their falsifying values
  int32_t lbits;    // lane bits (the clause depends on the slice: log2 Qp, else 0)
};

// Clause tensors B_C (Thm 3.2): 1 everywhere except 0 at the falsifying
// assignment.  One thread per entry of a flat list; `first` holds the
// first flat entry of each leaf (sorted), n_leaves entries.  Under index
// slicing a clause that a sliced literal satisfies is 1 everywhere; such a
// clause carries the lanes, each lane its own slice assignment when the
// slices run along the lanes.
template <typename T>
__global__ void k_clause_leaves(const ClauseLeaf *leaves, const int64_t *first, int64_t n_leaves,
                                int64_t n_entries, T *arena, int64_t *meta_exp,
                                unsigned long long *meta_max, unsigned long long *meta_min,
                                const IoDesc *io) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_entries;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n_leaves - 1;
    while (lo < hi) {  // last leaf with first <= i
      int64_t mid = (lo + hi + 1) >> 1;
      if (first[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const ClauseLeaf L = leaves[lo];
    // element (a, lane): the lane bits are the lowest
    const uint64_t e = (uint64_t)(i - first[lo]);
    const uint32_t lane = (uint32_t)(e & ((1ull << L.lbits) - 1ull));
    const uint64_t a = e >> L.lbits;
    uint32_t eta = (uint32_t)io->slice;
    if (io->lanes_per_slice > 0)
      eta += (uint32_t)(min((int32_t)lane, io->n_lanes - 1) / io->lanes_per_slice);
    const bool sat = ((eta ^ L.sfals) & L.smask) != 0u;
    arena[L.off + (int64_t)e] = (a == L.fals && !sat) ? (T)0 : (T)1;
    if (a == 0) {
      meta_exp[L.meta + lane] = 0;
      // max is 1 unless the tensor is a rank-0 clause with value 0
      const bool zero = L.rank == 0 && !sat;
      meta_max[L.meta + lane] = zero ? 0ull : abs_bits((T)1);
      meta_min[L.meta + lane] = zero ? kNoMin : abs_bits((T)1);
    }
  }
}

// Weight vectors [W(x,0), W(x,1)] per query, normalised so the larger
// magnitude lies in [1, 2); the scale is an exact power of two.
// Element [b * Q + q] of variable x's tensor.
// Q queries fill the Qp = 2^m query lanes; padding lanes repeat the last
// query (their results are never read).
template <typename T>
__global__ void k_weight_leaves(const IoDesc *io, int32_t n_vars, int32_t Q, int32_t Qp,
                                const int64_t *off, const int64_t *meta, T *arena,
                                int64_t *meta_exp, unsigned long long *meta_max,
                                unsigned long long *meta_min, uint32_t *flags) {
  const double *w_pos = io->w_pos;
  const double *w_neg = io->w_neg;
  const int64_t total = (int64_t)n_vars * Qp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)(i / Qp), q = (int32_t)(i % Qp);
    if (off[x] < 0) continue;  // no weight leaf: a variable fixed by index slicing
    const int32_t qs = q < Q ? q : Q - 1;
    const double w1 = w_pos[(int64_t)qs * n_vars + x];
    const double w0 = w_neg[(int64_t)qs * n_vars + x];
    const double m = fmax(fabs(w0), fabs(w1));
    int e = 0;
    if (m > 0) {
      e = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023;
      if (e < -1022) e = -1022;  // subnormal weights: keep an exact scale
      if (e > 1022) e = 1022;
    }
    const double s = __longlong_as_double((long long)(1023 - e) << 52);
    const T v0 = (T)(w0 * s), v1 = (T)(w1 * s);
    arena[off[x] + q] = v0;
    arena[off[x] + Qp + q] = v1;
    if (((w0 * s != 0.0) && below_normal(v0)) || ((w1 * s != 0.0) && below_normal(v1)))
      atomicOr(flags + q, 2u);
    meta_exp[meta[x] + q] = e;
    const unsigned long long b0 = abs_bits(v0), b1 = abs_bits(v1);
    meta_max[meta[x] + q] = b0 > b1 ? b0 : b1;
    const unsigned long long n0 = b0 ? b0 : kNoMin, n1 = b1 ? b1 : kNoMin;
    meta_min[meta[x] + q] = n0 < n1 ? n0 : n1;
  }
}

// ------------------------------------------------------ one-CTA walk
//
// A formula whose whole tree is small (every node at most 2^16 outputs
// with the query bits and 2^8 summed terms) and whose live tensors fit in
// one block's shared memory runs as ONE block: the leaves are materialised
// in shared memory, then the nodes run level by level with block barriers
// between the levels -- no launches, no dependency waits through global
// memory, no L2 round trips on the walk's critical path.
// Every node computes exactly what the small-node phase computes (the same
// operand scales, terms in ascending summed order, the same max/min and
// exponents), so the results are the same bits.  The root is written to
// the workspace for the finaliser.

struct CtaLeaf {
  uint64_t fals;      // clause: the falsifying assignment
  uint32_t off;       // byte offset in the block's tensor arena
  int32_t slot;       // metadata slot (per lane: slot + q)
  int32_t kind;       // LEAF_CLAUSE 0, LEAF_WEIGHT 1, LEAF_ONE 2
  int32_t rank;       // clause: its indices
  int32_t var;        // weight vector: its variable
  uint32_t smask, sfals;  // clause: sliced literals (index slicing)
  int32_t pad;
};

struct CtaArgs {
  char *ws;                   // workspace: the root's data and exponent slots
  const SNode *nodes;         // post-order; a, b, c are arena byte offsets (the root's c: workspace)
  const CtaLeaf *leaves;
  const IoDesc *io;
  uint32_t *flags;            // per-lane flags (workspace)
  int64_t *gexp;              // workspace exponent slots (the root's are read by the finaliser)
  int32_t n_nodes, n_leaves, n_slots;
  int32_t n_vars, Q, Qp;
  int32_t f64;
  uint32_t nodes_off, leaves_off;  // shared-memory offsets of the node program and the leaf descriptors
  uint32_t meta_bytes;        // shared memory before the arena: metadata, program, leaves
  uint32_t lut_off;           // shared memory of one level's lookup tables (after the arena)
};

// The one-block walk runs the tree level by level: a node's level is one
// more than its children's (leaves 0), so the nodes of a level are
// independent.  Per level: every node's lookup tables and C's exponents
// and flush test (from the children's metadata), a barrier, all the
// level's outputs spread over the block's threads (max and min straight
// into C's metadata slots by shared atomics), a barrier.  The barriers
// follow the tree's height instead of its node count.
//
// A node's tables (2 (n0 + n1 + ns) words at lut_base): A's offsets of
// output bits 0-7 (n0 = 2^min(8, rC)), of bits 8-15 (n1 = 2^max(0, rC - 8))
// and of the summed bits (ns = 2^k), then the same for B.
__device__ __forceinline__ void cta_table_entry(const SNode &nd, uint32_t *T, int i) {
  const int rc = nd.rC, n0 = 1 << (rc < 8 ? rc : 8), n1 = 1 << (rc > 8 ? rc - 8 : 0), ns = 1 << nd.k;
  const int half = n0 + n1 + ns;
  const int op = i >= half ? 1 : 0, k = i - op * half;
  int v, base, nb;
  const int8_t *pos;
  if (k < n0) { v = k; base = 0; nb = rc < 8 ? rc : 8; pos = op ? nd.posB : nd.posA; }
  else if (k < n0 + n1) { v = k - n0; base = 8; nb = rc - 8; pos = op ? nd.posB : nd.posA; }
  else { v = k - n0 - n1; base = 0; nb = nd.k; pos = op ? nd.sposB : nd.sposA; }
  uint32_t o = 0;
  for (int b = 0; b < nb; ++b)
    if (((v >> b) & 1) && pos[base + b] >= 0) o |= 1u << pos[base + b];
  T[i] = o;
}

// C's exponent per lane and the float32 flush test, from the operands'
// metadata (their max and min are final: earlier levels)
template <typename TI>
__device__ __forceinline__ void cta_node_meta(const CtaArgs &a, const SNode &nd, int q, int64_t *mexp,
                                              const unsigned long long *mmax, const unsigned long long *mmin,
                                              bool root) {
  const int qa = q & nd.qmask_a, qb = q & nd.qmask_b;
  const unsigned long long xa = mmax[nd.ma + qa], xb = mmax[nd.mb + qb];
  const int64_t e = mexp[nd.ma + qa] + pow2_exp_of(xa, TI()) + mexp[nd.mb + qb] + pow2_exp_of(xb, TI());
  mexp[nd.mc + q] = e;
  if (root) a.gexp[nd.mc + q] = e;
  const unsigned long long na = mmin[nd.ma + qa], nb = mmin[nd.mb + qb];
  if (na != kNoMin && nb != kNoMin) {
    const TI lo = (from_bits<TI>(na) * pow2_scale(pow2_exp_of(xa, TI()), TI())) *
                  (from_bits<TI>(nb) * pow2_scale(pow2_exp_of(xb, TI()), TI()));
    if (below_normal(lo)) {
      if (nd.Qc > 1) atomicOr(a.flags + q, 2u);
      else
        for (int qq = 0; qq < a.Qp; ++qq) atomicOr(a.flags + qq, 2u);
    }
  }
}

// Output o of a node: its terms in ascending summed order (the canonical
// chain of every other kernel), operands scaled per lane by their pow2
// scales
template <typename TI, typename TA, typename TO>
__device__ __forceinline__ void cta_output(const CtaArgs &a, const SNode &nd, uint32_t o, unsigned char *arena,
                                           unsigned long long *mmax, unsigned long long *mmin, const uint32_t *T,
                                           bool root) {
  const TI *A = (const TI *)(arena + nd.a);
  const TI *B = (const TI *)(arena + nd.b);
  TO *C = root ? (TO *)(a.ws + nd.c) : (TO *)(arena + nd.c);
  const int q = (int)(o & (uint32_t)(nd.Qc - 1));
  const TA sa = (TA)pow2_scale(pow2_exp_of(mmax[nd.ma + (q & nd.qmask_a)], TI()), TI());
  const TA sb = (TA)pow2_scale(pow2_exp_of(mmax[nd.mb + (q & nd.qmask_b)], TI()), TI());
  const uint32_t n0 = 1u << (nd.rC < 8 ? nd.rC : 8), n1 = 1u << (nd.rC > 8 ? nd.rC - 8 : 0), ns = 1u << nd.k;
  const uint32_t *TA0 = T, *TA1 = TA0 + n0, *TSA = TA1 + n1, *TB0 = TSA + ns, *TB1 = TB0 + n0, *TSB = TB1 + n1;
  const uint32_t bA = TA0[o & 255] | TA1[o >> 8];
  const uint32_t bB = TB0[o & 255] | TB1[o >> 8];
  TA acc = (TA)0;
  for (uint32_t s = 0; s < ns; ++s) acc = fma_t((TA)A[bA | TSA[s]] * sa, (TA)B[bB | TSB[s]] * sb, acc);
  const TO c = (TO)acc;
  C[o] = c;
  const unsigned long long bits = abs_bits(c);
  if (bits) {
    atomicMax(mmax + nd.mc + q, bits);
    atomicMin(mmin + nd.mc + q, bits);
  }
}

__global__ void __launch_bounds__(1024, 1) k_cta_walk(CtaArgs a) {
  // dynamic shared memory: metadata (exp, max, min per slot), the node
  // program, the leaf descriptors, then the tensor arena
  extern __shared__ __align__(16) unsigned char cta_smem[];
  int64_t *mexp = (int64_t *)cta_smem;
  unsigned long long *mmax = (unsigned long long *)(cta_smem + 8 * (size_t)a.n_slots);
  unsigned long long *mmin = (unsigned long long *)(cta_smem + 16 * (size_t)a.n_slots);
  SNode *nodes = (SNode *)(cta_smem + a.nodes_off);
  CtaLeaf *leaves = (CtaLeaf *)(cta_smem + a.leaves_off);
  unsigned char *arena = cta_smem + a.meta_bytes;
  static_assert(sizeof(SNode) % 4 == 0 && sizeof(CtaLeaf) % 4 == 0, "copied as 32-bit words");
  // the program into shared memory at once (one latency, not one per node)
  {
    const int nw = a.n_nodes * (int)(sizeof(SNode) / 4), lw = a.n_leaves * (int)(sizeof(CtaLeaf) / 4);
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
      reinterpret_cast<uint32_t *>(nodes)[i] = reinterpret_cast<const uint32_t *>(a.nodes)[i];
    for (int i = threadIdx.x; i < lw; i += blockDim.x)
      reinterpret_cast<uint32_t *>(leaves)[i] = reinterpret_cast<const uint32_t *>(a.leaves)[i];
  }
  for (int i = threadIdx.x; i < a.n_slots; i += blockDim.x) { mexp[i] = 0; mmax[i] = 0; mmin[i] = kNoMin; }
  __syncthreads();
  // ---- leaves, one thread per leaf (as k_clause_leaves, k_weight_leaves
  // and k_one_leaf)
  const uint32_t eta = (uint32_t)a.io->slice;
  for (int li = threadIdx.x; li < a.n_leaves; li += blockDim.x) {
    const CtaLeaf &L = leaves[li];
    if (L.kind == 0) {
      const bool sat = ((eta ^ L.sfals) & L.smask) != 0u;
      for (uint32_t e = 0; e < (1u << L.rank); ++e) {
        const bool z = (e == (uint32_t)L.fals && !sat);
        if (a.f64) ((double *)(arena + L.off))[e] = z ? 0.0 : 1.0;
        else ((float *)(arena + L.off))[e] = z ? 0.0f : 1.0f;
      }
      const bool zero = L.rank == 0 && !sat;
      mmax[L.slot] = zero ? 0ull : (a.f64 ? abs_bits(1.0) : abs_bits(1.0f));
      mmin[L.slot] = zero ? kNoMin : (a.f64 ? abs_bits(1.0) : abs_bits(1.0f));
    } else if (L.kind == 1) {
      for (int q = 0; q < a.Qp; ++q) {
        const int qs = q < a.Q ? q : a.Q - 1;
        const double w1 = a.io->w_pos[(int64_t)qs * a.n_vars + L.var];
        const double w0 = a.io->w_neg[(int64_t)qs * a.n_vars + L.var];
        const double m = fmax(fabs(w0), fabs(w1));
        int e = 0;
        if (m > 0) {
          e = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023;
          if (e < -1022) e = -1022;
          if (e > 1022) e = 1022;
        }
        const double sc = __longlong_as_double((long long)(1023 - e) << 52);
        unsigned long long b0, b1;
        bool flush;
        if (a.f64) {
          const double v0 = w0 * sc, v1 = w1 * sc;
          ((double *)(arena + L.off))[q] = v0;
          ((double *)(arena + L.off))[a.Qp + q] = v1;
          b0 = abs_bits(v0); b1 = abs_bits(v1);
          flush = ((w0 * sc != 0.0) && below_normal(v0)) || ((w1 * sc != 0.0) && below_normal(v1));
        } else {
          const float v0 = (float)(w0 * sc), v1 = (float)(w1 * sc);
          ((float *)(arena + L.off))[q] = v0;
          ((float *)(arena + L.off))[a.Qp + q] = v1;
          b0 = abs_bits(v0); b1 = abs_bits(v1);
          flush = ((w0 * sc != 0.0) && below_normal(v0)) || ((w1 * sc != 0.0) && below_normal(v1));
        }
        if (flush) atomicOr(a.flags + q, 2u);
        mexp[L.slot + q] = e;
        mmax[L.slot + q] = b0 > b1 ? b0 : b1;
        const unsigned long long n0 = b0 ? b0 : kNoMin, n1 = b1 ? b1 : kNoMin;
        mmin[L.slot + q] = n0 < n1 ? n0 : n1;
      }
    } else {
      if (a.f64) *(double *)(arena + L.off) = 1.0;
      else *(float *)(arena + L.off) = 1.0f;
      mmax[L.slot] = mmin[L.slot] = a.f64 ? abs_bits(1.0) : abs_bits(1.0f);
    }
  }
  // ---- the nodes, level by level
  uint32_t *luts = (uint32_t *)(cta_smem + a.lut_off);
  for (int f0 = 0; f0 < a.n_nodes;) {
    const int f1 = nodes[f0].level_end;
    const SNode &last = nodes[f1 - 1];
    const int n_words = last.lut_base + 2 * ((1 << (last.rC < 8 ? last.rC : 8)) +
                                             (1 << (last.rC > 8 ? last.rC - 8 : 0)) + (1 << last.k));
    const uint32_t n_out = (uint32_t)last.out_base + (1u << last.rC);
    // __syncthreads() before: the previous level's outputs, max and min (and the leaves)
    __syncthreads();
    for (int i = threadIdx.x; i < n_words; i += blockDim.x) {
      int lo = f0, hi = f1 - 1;  // the node whose tables hold word i
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nodes[mid].lut_base <= i) lo = mid; else hi = mid - 1;
      }
      cta_table_entry(nodes[lo], luts + nodes[lo].lut_base, i - nodes[lo].lut_base);
    }
    for (int i = threadIdx.x; i < 4 * (f1 - f0); i += blockDim.x) {
      const SNode &nd = nodes[f0 + (i >> 2)];
      const int q = i & 3;
      if (q >= nd.Qc) continue;
      const bool root = f0 + (i >> 2) == a.n_nodes - 1;
      if (nd.ti == 1) cta_node_meta<double>(a, nd, q, mexp, mmax, mmin, root);
      else cta_node_meta<float>(a, nd, q, mexp, mmax, mmin, root);
    }
    __syncthreads();  // tables
    for (uint32_t g = threadIdx.x; g < n_out; g += blockDim.x) {
      int lo = f0, hi = f1 - 1;  // the node of output g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)nodes[mid].out_base <= g) lo = mid; else hi = mid - 1;
      }
      const SNode &nd = nodes[lo];
      const uint32_t o = g - (uint32_t)nd.out_base;
      const bool root = lo == a.n_nodes - 1;
      const uint32_t *T = luts + nd.lut_base;
      if (nd.ti == 1) cta_output<double, double, double>(a, nd, o, arena, mmax, mmin, T, root);
      else if (nd.to == 1) cta_output<float, double, double>(a, nd, o, arena, mmax, mmin, T, root);
      else cta_output<float, float, float>(a, nd, o, arena, mmax, mmin, T, root);
    }
    f0 = f1;
  }
}

// ------------------------------------------------ block floating point
//
// Block-floating-point float32 (a plan option): every tensor's entries are
// float32 mantissas, and each block of 2^b consecutive assignments of its
// non-query indices has its own int32 exponent per query lane (weight
// vectors: one exponent per entry), so one tensor may span any range: only
// entries of one block share float32's 2^126 range.  A node adds its
// products in float64 (a product of two float32 mantissas is exact there),
// each term brought to the largest exponent met so far, then each output
// block is normalised so its largest |entry| lies in [1, 2) and its
// exponent stored.  Value of entry o of a tensor with m query bits and b
// block bits: mant[o] * 2^exp[(o >> (m + b)) * 2^m + (o & (2^m - 1))].

struct BfpParams {
  K1Params k1;                   // addressing (C bits -> A, B bits; summed bits)
  const int32_t *eA, *eB;        // block exponents of the operands
  int32_t *eC;
  int8_t mA, mB, mC;             // query bits of each tensor (0 or m)
  int8_t bA, bB, bC;             // block bits of each tensor
  int8_t c_double;               // the root: float64 mantissas, exponent also to root_exp
  int8_t pad;
  int64_t *root_exp;             // per-lane exponent slots of the root (k_finalize)
  uint32_t *flags;               // per-lane flags (WMC_FLAG_FP32_FLUSH)
  int64_t n_blocks;              // output blocks: 2^(non-query bits of C - bC)
};

constexpr int kBfpMaxOut = 2048;  // outputs of one block (all lanes) held in shared memory
constexpr int kNoExp = -2147483647 - 1;  // no nonzero term yet

__device__ __forceinline__ double pow2_d(int e) {  // 2^e for e in [-1022, 1023], else 0 / inf-free clamp
  if (e < -1022) return 0.0;
  if (e > 1023) e = 1023;
  return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ int ilogb_d(double x) {  // floor(log2 |x|) of a normal nonzero double
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

template <typename TO>
__global__ void __launch_bounds__(kThreads) k_bfp_node(BfpParams p) {
  __shared__ uint32_t lutA[4][256], lutB[4][256];
  __shared__ uint32_t slutA[3][256], slutB[3][256];
  __shared__ double s_acc[kBfpMaxOut];
  __shared__ int s_t[kBfpMaxOut];
  __shared__ int s_emax[kMaxQ];
  const K1Params &k = p.k1;
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const int byte = i >> 8, v = i & 255;
    uint32_t oa = 0, ob = 0;
    for (int b = 0; b < 8; ++b) {
      const int j = byte * 8 + b;
      if (((v >> b) & 1) && j < k.rC) {
        if (k.posA[j] >= 0) oa |= 1u << k.posA[j];
        if (k.posB[j] >= 0) ob |= 1u << k.posB[j];
      }
    }
    lutA[byte][v] = oa;
    lutB[byte][v] = ob;
  }
  for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) {
    const int byte = i >> 8, v = i & 255;
    uint32_t oa = 0, ob = 0;
    for (int b = 0; b < 8; ++b) {
      const int j = byte * 8 + b;
      if (((v >> b) & 1) && j < k.k) {
        if (k.sposA[j] >= 0) oa |= 1u << k.sposA[j];
        if (k.sposB[j] >= 0) ob |= 1u << k.sposB[j];
      }
    }
    slutA[byte][v] = oa;
    slutB[byte][v] = ob;
  }
  __syncthreads();
  const float *A = (const float *)k.A;
  const float *B = (const float *)k.B;
  const int qa = (1 << p.mA) - 1, qb = (1 << p.mB) - 1, qc = (1 << p.mC) - 1;
  const int shA = p.mA + p.bA, shB = p.mB + p.bB;
  const uint32_t n_out = 1u << (p.mC + p.bC);  // outputs of one block, all lanes
  const uint32_t ns = 1u << k.k;
  for (int64_t blk = blockIdx.x; blk < p.n_blocks; blk += gridDim.x) {
    for (int q = threadIdx.x; q <= qc; q += blockDim.x) s_emax[q] = kNoExp;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_out; i += blockDim.x) {
      const uint32_t o = ((uint32_t)blk << (p.mC + p.bC)) | i;
      const uint32_t ba = lutA[0][o & 255] | lutA[1][(o >> 8) & 255] | lutA[2][(o >> 16) & 255] | lutA[3][o >> 24];
      const uint32_t bb = lutB[0][o & 255] | lutB[1][(o >> 8) & 255] | lutB[2][(o >> 16) & 255] | lutB[3][o >> 24];
      // terms in ascending summed assignment; the running sum is kept at
      // the largest exponent met so far (a power-of-two rescale is exact)
      double acc = 0.0;
      int t = kNoExp;
      for (uint32_t sidx = 0; sidx < ns; ++sidx) {
        const uint32_t oa = ba | slutA[0][sidx & 255] | slutA[1][(sidx >> 8) & 255] | slutA[2][sidx >> 16];
        const uint32_t ob = bb | slutB[0][sidx & 255] | slutB[1][(sidx >> 8) & 255] | slutB[2][sidx >> 16];
        const float ma = A[oa], mb = B[ob];
        if (ma == 0.0f || mb == 0.0f) continue;
        const int e = p.eA[((oa >> shA) << p.mA) | (oa & qa)] + p.eB[((ob >> shB) << p.mB) | (ob & qb)];
        const double prod = (double)ma * (double)mb;  // exact
        if (t == kNoExp) { acc = prod; t = e; }
        else if (e > t) { acc = acc * pow2_d(t - e) + prod; t = e; }
        else acc += prod * pow2_d(e - t);
      }
      if (acc == 0.0 || fabs(acc) < 2.2250738585072014e-308) { acc = 0.0; t = kNoExp; }
      s_acc[i] = acc;
      s_t[i] = t;
      if (t != kNoExp) atomicMax(&s_emax[i & qc], t + ilogb_d(acc));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_out; i += blockDim.x) {
      const uint32_t o = ((uint32_t)blk << (p.mC + p.bC)) | i;
      const int q = (int)(i & qc);
      const double acc = s_acc[i];
      TO v = (TO)0;
      if (acc != 0.0) {
        const int d = s_t[i] - s_emax[q];  // <= -ilogb(acc): |v| < 2
        v = (TO)(acc * pow2_d(d));
        if (below_normal(v)) atomicOr(p.flags + q, 2u);  // an entry more than float's range below its block's top
      }
      ((TO *)k.C)[o] = v;
    }
    for (int q = threadIdx.x; q <= qc; q += blockDim.x) {
      const int em = s_emax[q] == kNoExp ? 0 : s_emax[q];
      p.eC[(blk << p.mC) | q] = em;
      if (p.c_double) p.root_exp[q] = em;
    }
    __syncthreads();
  }
}

// Weight vectors in block-floating-point form: each entry its own exponent
// per lane (W = mant * 2^e, mant in [1, 2)), so a weight ratio of any size
// is kept exactly.  Layout of a leaf: mantissas [value][lane] at off, then
// (exp_delta bytes later) exponents [value][lane].
__global__ void k_bfp_weights(const IoDesc *io, int32_t n_vars, int32_t Q, int32_t Qp, const int64_t *off,
                              float *arena, int64_t exp_delta, uint32_t *flags) {
  const double *w_pos = io->w_pos;
  const double *w_neg = io->w_neg;
  const int64_t total = (int64_t)n_vars * Qp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)(i / Qp), q = (int32_t)(i % Qp);
    if (off[x] < 0) continue;
    const int32_t qs = q < Q ? q : Q - 1;
    int32_t *ex = (int32_t *)((char *)(arena + off[x]) + exp_delta);
    for (int val = 0; val < 2; ++val) {
      const double w = val ? w_pos[(int64_t)qs * n_vars + x] : w_neg[(int64_t)qs * n_vars + x];
      float m = 0.0f;
      int e = 0;
      if (w != 0.0) {
        double aw = fabs(w);
        int adj = 0;
        if (aw < 2.2250738585072014e-308) { aw *= 18014398509481984.0; adj = -54; }  // subnormal: scale by 2^54
        e = ilogb_d(aw) + adj;
        m = (float)(w * pow2_d(-(e - adj)) * (adj ? 18014398509481984.0 : 1.0));
        if (!isfinite(w)) atomicOr(flags + q, 2u);
      }
      arena[off[x] + (int64_t)val * Qp + q] = m;
      ex[val * Qp + q] = e;
    }
  }
}

template <typename T>
__global__ void k_one_leaf(T *dst, int64_t meta, int64_t *meta_exp, unsigned long long *meta_max,
                           unsigned long long *meta_min) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dst[0] = (T)1;
    meta_exp[meta] = 0;
    meta_max[meta] = abs_bits((T)1);
    meta_min[meta] = abs_bits((T)1);
  }
}

// Root: value[q] = mant[q] * 2^exp[q] with the root tensor stored in
// float64 (its exponents already account for its inputs' scales).
// The root (float64 mantissa and int64 exponent per query) into the
// outputs.  Under index slicing the value is multiplied by the sliced
// variables' weights at the lane's slice assignment (Thm 4.2: the slice's
// share of W) and, after the first slice, added to the outputs with the
// exponents aligned (all terms nonnegative for nonnegative weights).
__global__ void k_finalize(const IoDesc *io, const double *root, const int64_t *root_exp,
                           int32_t root_qc, const uint32_t *flags, const uint32_t *err,
                           int32_t Q, int32_t n_vars) {
  double *mant = io->mant;
  int64_t *exp2 = io->exp2;
  uint32_t *out_flags = io->flags;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    const int qr = root_qc > 1 ? q : 0;
    double m = root[qr];
    int64_t e = root_exp[qr];
    // this lane's slice assignment (slices along the lanes: see IoDesc)
    uint64_t eta = io->slice;
    if (io->lanes_per_slice > 0) eta += (uint64_t)(min(q, io->n_lanes - 1) / io->lanes_per_slice);
    for (int k = 0; k < io->n_slice; ++k) {
      const int64_t at = (int64_t)q * n_vars + io->slice_var[k];
      m *= ((eta >> k) & 1ull) ? io->w_pos[at] : io->w_neg[at];
      int fe = 0;
      m = frexp(m, &fe);
      e += fe;
    }
    const uint32_t f = flags[q] | (*err ? 0x8u : 0u);
    if (io->accumulate) {
      double om = mant[q];
      int64_t oe = exp2[q];
      if (om == 0.0) {
        mant[q] = m;
        exp2[q] = e;
      } else if (m != 0.0) {
        int fo = 0, fn = 0;
        om = frexp(om, &fo);
        m = frexp(m, &fn);
        oe += fo;
        e += fn;
        if (oe >= e) {
          const int64_t d = oe - e;
          mant[q] = om + (d > 1100 ? 0.0 : ldexp(m, -(int)d));
          exp2[q] = oe;
        } else {
          const int64_t d = e - oe;
          mant[q] = m + (d > 1100 ? 0.0 : ldexp(om, -(int)d));
          exp2[q] = e;
        }
      }
      out_flags[q] |= f;
    } else {
      mant[q] = m;
      exp2[q] = e;
      out_flags[q] = f;
    }
  }
}

// float64 -> scaled float32 (two passes: max, then scale).
__global__ void k_absmax_f64(const double *x, int64_t n, unsigned long long *maxb) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long b = abs_bits(x[i]);
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(maxb, m);
}

__global__ void k_scale_to_f32(const double *x, int64_t n, const unsigned long long *maxb,
                               float *out) {
  const int e = pow2_exp_of(*maxb, double());
  const double s = pow2_scale(e, double());
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(x[i] * s);
}

// In place: the max bit pattern becomes the exponent it implies.
__global__ void k_max_to_exp(unsigned long long *slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int e = pow2_exp_of(*slot, double());
    *reinterpret_cast<int64_t *>(slot) = e;
  }
}

}  // namespace dev
}  // namespace wmc
