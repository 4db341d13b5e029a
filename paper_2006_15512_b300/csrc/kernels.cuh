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

namespace wmc {
namespace dev {

constexpr int kThreads = 256;
constexpr int kMaxQ = 1024;

// --------------------------------------------------------------- helpers

__device__ __forceinline__ int pow2_exp_of(unsigned long long bits, float) {
  if (bits == 0) return 0;
  int e = (int)((bits >> 23) & 0xff) - 127;
  e = e < -126 ? -126 : e;
  return e > 126 ? 126 : e;
}
__device__ __forceinline__ int pow2_exp_of(unsigned long long bits, double) {
  if (bits == 0) return 0;
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  e = e < -1022 ? -1022 : e;
  return e > 1022 ? 1022 : e;
}
__device__ __forceinline__ float pow2_scale(int e, float) { return __int_as_float((127 - e) << 23); }
__device__ __forceinline__ double pow2_scale(int e, double) {
  return __longlong_as_double((long long)(1023 - e) << 52);
}
__device__ __forceinline__ unsigned long long abs_bits(float x) {
  return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool below_normal(float x) { return fabsf(x) < 1.17549435e-38f; }
__device__ __forceinline__ bool below_normal(double x) { return fabs(x) < 2.2250738585072014e-308; }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// insert a zero bit at position p
__device__ __forceinline__ uint32_t insert0(uint32_t x, int p) {
  uint32_t lo = x & ((1u << p) - 1u);
  return ((x >> p) << (p + 1)) | lo;
}

// Per-operand metadata: exponents and max bit patterns, one entry per
// query if the tensor carries the query index (qmask = Q-1), else one.
struct Meta {
  const int64_t *exp;
  const unsigned long long *maxb;
  int32_t qmask;
};

struct OutMeta {
  int64_t *exp;
  unsigned long long *maxb;
  uint32_t *flags;  // per query
  int32_t Qc;       // entries of C's metadata (Q or 1)
  int32_t Q;        // queries in the batch (flags entries)
  int32_t scale_inputs;  // 0: inputs are used as stored (contract_pair)
};

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

template <typename T>
__device__ __forceinline__ void finish_meta(const Meta &ma, const Meta &mb, const OutMeta &mc,
                                            unsigned long long *smax, bool flush_any,
                                            int qc_thread) {
  // exponent of C: sum of both operands' effective exponents
  if (blockIdx.x == 0 && mc.exp) {
    for (int q = threadIdx.x; q < mc.Qc; q += blockDim.x) {
      int64_t e = 0;
      if (ma.exp) {
        int qa = q & ma.qmask;
        e += ma.exp[qa] + (mc.scale_inputs ? pow2_exp_of(ma.maxb[qa], T()) : 0);
      }
      if (mb.exp) {
        int qb = q & mb.qmask;
        e += mb.exp[qb] + (mc.scale_inputs ? pow2_exp_of(mb.maxb[qb], T()) : 0);
      }
      mc.exp[q] = e;
    }
  }
  __syncthreads();
  if (mc.maxb)
    for (int q = threadIdx.x; q < mc.Qc; q += blockDim.x)
      if (smax[q]) atomicMax(mc.maxb + q, smax[q]);
  if (flush_any && mc.flags) {
    if (mc.Qc > 1) atomicOr(mc.flags + qc_thread, 2u);
    else
      for (int q = 0; q < mc.Q; ++q) atomicOr(mc.flags + q, 2u);
  }
}

// TI: stored type of A and B; TA: accumulation; TO: stored type of C.
// The grid is sized so that the grid-stride step is a multiple of Qc, so
// every thread sees one query for all its outputs.
template <typename TI, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) k1_generic(K1Params p) {
  __shared__ uint32_t lutA[4][256], lutB[4][256];
  __shared__ uint32_t slutA[3][256], slutB[3][256];
  __shared__ unsigned long long smax[kMaxQ];
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
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) smax[q] = 0;
  __syncthreads();

  const uint64_t n_out = 1ull << p.rC;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int qc = (int)(gtid & (uint64_t)(p.mc.Qc - 1));
  TA sa = (TA)1, sb = (TA)1;
  if (p.mc.scale_inputs) {
    sa = (TA)pow2_scale(pow2_exp_of(p.ma.maxb[qc & p.ma.qmask], TI()), TI());
    sb = (TA)pow2_scale(pow2_exp_of(p.mb.maxb[qc & p.mb.qmask], TI()), TI());
  }
  const TI *A = (const TI *)p.A;
  const TI *B = (const TI *)p.B;
  TO *C = (TO *)p.C;
  const uint32_t ns = 1u << p.k;
  unsigned long long tmax = 0;
  bool flush = false;
  for (uint64_t o = gtid; o < n_out; o += stride) {
    const uint32_t oo = (uint32_t)o;
    const uint32_t ba = lutA[0][oo & 255] | lutA[1][(oo >> 8) & 255] | lutA[2][(oo >> 16) & 255] |
                        lutA[3][oo >> 24];
    const uint32_t bb = lutB[0][oo & 255] | lutB[1][(oo >> 8) & 255] | lutB[2][(oo >> 16) & 255] |
                        lutB[3][oo >> 24];
    TA acc = (TA)0;
    bool nz = false;
    if (p.k <= 8) {
      for (uint32_t s = 0; s < ns; ++s) {
        const TA a = (TA)__ldg(A + (ba | slutA[0][s])) * sa;
        const TA b = (TA)__ldg(B + (bb | slutB[0][s])) * sb;
        nz |= (a != (TA)0) & (b != (TA)0);
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
          nz |= (a != (TA)0) & (b != (TA)0);
          part = fma_t(a, b, part);
        }
        acc += part;
      }
    }
    const TO c = (TO)acc;
    C[o] = c;
    const unsigned long long bits = abs_bits(c);
    tmax = bits > tmax ? bits : tmax;
    flush |= nz && below_normal(c);
  }
  if (tmax) atomicMax(smax + qc, tmax);
  finish_meta<TI>(p.ma, p.mb, p.mc, smax, __syncthreads_or(flush), qc);
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
  int32_t n_insA, n_insC, nbb;
  int8_t insA[8];   // ascending positions of summed bits in P
  int8_t insC[8];   // ascending positions of S's free bits in C
  int8_t bbC[32];   // S batch bit i: position in C
  int8_t bbB[32];   //               position in S
  uint32_t dA[8];   // offset of summed assignment s in P
  uint32_t dBs[8];  // ... in S
  uint32_t dBf[8];  // offset of S-free assignment f in S
  uint32_t dC[8];   // ... in C
  uint32_t dBv[4];  // offset in S of vector lane e
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

// K (summed bits) and F (S-free bits) are compile-time upper bounds; the
// runtime p.k / p.f select the active terms.
template <typename T, int V, int K, int F>
__global__ void __launch_bounds__(kThreads) k2_stream(K2Params p) {
  __shared__ unsigned long long smax[kMaxQ];
  for (int q = threadIdx.x; q < p.mc.Qc; q += blockDim.x) smax[q] = 0;
  __syncthreads();
  constexpr int NS = 1 << K, NF = 1 << F;
  const int ns = 1 << p.k, nf = 1 << p.f;
  const T *A = (const T *)p.A;
  const T *B = (const T *)p.B;
  T *C = (T *)p.C;
  const uint64_t nu = 1ull << p.log2_nu;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T sa[V], sb[NF][V];
  unsigned long long tmax[NF][V];
  int qcs[NF][V];
  bool flush = false;
  bool first = true;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int e = 0; e < V; ++e) tmax[f][e] = 0, qcs[f][e] = 0;
  for (uint64_t u = gtid; u < nu; u += stride) {
    const uint32_t w = (uint32_t)(u << p.vbits);
    uint32_t oa = w, oc = w, gb = 0;
    for (int i = 0; i < p.n_insA; ++i) oa = insert0(oa, p.insA[i]);
    for (int i = 0; i < p.n_insC; ++i) oc = insert0(oc, p.insC[i]);
    for (int i = 0; i < p.nbb; ++i) gb |= ((oc >> p.bbC[i]) & 1u) << p.bbB[i];
    if (first) {
      // the query of every lane is fixed across the grid-stride loop
      first = false;
#pragma unroll
      for (int e = 0; e < V; ++e) {
        sa[e] = (T)1;
        if (p.mc.scale_inputs)
          sa[e] = pow2_scale(pow2_exp_of(p.ma.maxb[(oa + e) & p.ma.qmask], T()), T());
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          sb[f][e] = (T)1;
          if (f < nf) {
            if (p.mc.scale_inputs)
              sb[f][e] = pow2_scale(
                  pow2_exp_of(p.mb.maxb[(gb + p.dBf[f] + p.dBv[e]) & p.mb.qmask], T()), T());
            qcs[f][e] = (int)((oc + p.dC[f] + e) & (uint32_t)(p.mc.Qc - 1));
          }
        }
      }
    }
    T a[NS][V];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (s < ns) {
        vload<T, V>(A + oa + p.dA[s], a[s]);
#pragma unroll
        for (int e = 0; e < V; ++e) a[s][e] *= sa[e];
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (f < nf) {
        T c[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          T acc = (T)0;
          bool nz = false;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if (s < ns) {
              const T b = __ldg(B + (gb + p.dBs[s] + p.dBf[f] + p.dBv[e])) * sb[f][e];
              nz |= (a[s][e] != (T)0) & (b != (T)0);
              acc = fma_t(a[s][e], b, acc);
            }
          }
          c[e] = acc;
          const unsigned long long bits = abs_bits(acc);
          tmax[f][e] = bits > tmax[f][e] ? bits : tmax[f][e];
          flush |= nz && below_normal(acc);
        }
        vstore<T, V>(C + oc + p.dC[f], c);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (tmax[f][e]) atomicMax(smax + qcs[f][e], tmax[f][e]);
  finish_meta<T>(p.ma, p.mb, p.mc, smax, __syncthreads_or(flush), qcs[0][0]);
}

// --------------------------------------------------------------- leaves

struct ClauseLeaf {
  int64_t off;      // element offset in the tensor arena
  int64_t meta;     // metadata slot
  uint64_t fals;    // falsifying assignment
  int32_t rank;
  int32_t pad;
};

// Clause tensors B_C (Thm 3.2): 1 everywhere except 0 at the falsifying
// assignment.  One thread per entry of a flat list; `first` holds the
// first flat entry of each leaf (sorted), n_leaves entries.
template <typename T>
__global__ void k_clause_leaves(const ClauseLeaf *leaves, const int64_t *first, int64_t n_leaves,
                                int64_t n_entries, T *arena, int64_t *meta_exp,
                                unsigned long long *meta_max) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_entries;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n_leaves - 1;
    while (lo < hi) {  // last leaf with first <= i
      int64_t mid = (lo + hi + 1) >> 1;
      if (first[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const ClauseLeaf L = leaves[lo];
    const uint64_t a = (uint64_t)(i - first[lo]);
    arena[L.off + (int64_t)a] = (a == L.fals) ? (T)0 : (T)1;
    if (a == 0) {
      meta_exp[L.meta] = 0;
      // max is 1 unless the tensor is the rank-0 empty clause (value 0)
      meta_max[L.meta] = (L.rank == 0) ? 0ull : abs_bits((T)1);
    }
  }
}

// Weight vectors [W(x,0), W(x,1)] per query, normalised so the larger
// magnitude lies in [1, 2); the scale is an exact power of two.
// Element [b * Q + q] of variable x's tensor.
// Pointers that change from call to call; read from device memory so a
// captured graph can be replayed with new inputs and outputs.
struct IoDesc {
  const double *w_pos;
  const double *w_neg;
  double *mant;
  int64_t *exp2;
  uint32_t *flags;
  int64_t pad[3];
};

// Q queries fill the Qp = 2^m query lanes; padding lanes repeat the last
// query (their results are never read).
template <typename T>
__global__ void k_weight_leaves(const IoDesc *io, int32_t n_vars, int32_t Q, int32_t Qp,
                                const int64_t *off, const int64_t *meta, T *arena,
                                int64_t *meta_exp, unsigned long long *meta_max,
                                uint32_t *flags) {
  const double *w_pos = io->w_pos;
  const double *w_neg = io->w_neg;
  const int64_t total = (int64_t)n_vars * Qp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)(i / Qp), q = (int32_t)(i % Qp);
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
  }
}

template <typename T>
__global__ void k_one_leaf(T *dst, int64_t meta, int64_t *meta_exp, unsigned long long *meta_max) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    dst[0] = (T)1;
    meta_exp[meta] = 0;
    meta_max[meta] = abs_bits((T)1);
  }
}

// Root: value[q] = mant[q] * 2^exp[q] with the root tensor stored in
// float64 (its exponents already account for its inputs' scales).
__global__ void k_finalize(const IoDesc *io, const double *root, const int64_t *root_exp,
                           int32_t root_qc, const uint32_t *flags, int32_t Q) {
  double *mant = io->mant;
  int64_t *exp2 = io->exp2;
  uint32_t *out_flags = io->flags;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    const int qr = root_qc > 1 ? q : 0;
    mant[q] = root[qr];
    exp2[q] = root_exp[qr];
    out_flags[q] = flags[q];
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
