// Execution stage (Algorithm 2) on one GPU.
//
// The recursive Execute(N, T) of Algorithm 2 becomes an iterative
// post-order walk over the plan's node array.  For a query batch size Q the
// walk is laid out once (tensor arena offsets with first-fit reuse of
// freed children, per-node kernel choice and parameters) and captured into
// a CUDA graph per workspace, so one wmc_execute is one H2D copy of the
// inputs, one graph launch and one D2H copy of the results.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <cstdio>
#include <cstdlib>

#include "internal.h"
#include "kernels.cuh"

using namespace wmc;
using wmc::dev::ClauseLeaf;
using wmc::dev::IoDesc;
using wmc::dev::K1Params;
using wmc::dev::K2Params;

struct wmc_plan : public Plan {};
struct wmc_network;
namespace wmc { const Network &network_of(const wmc_network_t *n); }

static std::atomic<int64_t> g_launches{0};
static std::atomic<int32_t> g_fail_allocs{0};
static std::atomic<int32_t> g_debug_stall{0};
// fusion of consecutive frontier eliminations into one k2_chain launch:
// chains of up to this many (0 or 1: off)
static std::atomic<int32_t> g_fuse{-1};  // -1: by the walk's lane count
static std::atomic<int32_t> g_small_phase{1};  // small nodes in one persistent launch
static std::atomic<int32_t> g_pdl{1};  // programmatic dependent launch of chain kernels
static thread_local bool t_chain_pdl = true;  // the chain being launched may overlap the launch in front
static std::atomic<int32_t> g_tensor_cores{1};  // dense float32 pair contractions on tcgen05
static std::atomic<int32_t> g_fp64_fallback{1};  // flushed float32 queries run again in float64
// runs of consecutive chains whose every chain has at most this many tiles
// execute as one k2_chain_seq launch (0, the default: every chain its own
// launch, which measured faster at every batch size on the grid walks)
static std::atomic<int32_t> g_chain_runs{0};
// dynamic shared memory a run of chains may use: 227 KB per block less the
// run kernel's static part (two chains' parameters and its barriers)
constexpr size_t kSeqDynSmem = 227 * 1024 - 2 * sizeof(wmc::dev::K2CParams) - 2048;
static std::atomic<int32_t> g_autotune{0};  // wmc_contract_pair: time same-order variants per shape
static std::atomic<int32_t> g_cta_walk{0};  // small formulas: the whole walk in one block (opt-in)
static std::atomic<int32_t> g_force_kind{-1};  // test hook: force one variant (-1: off)
static std::atomic<int64_t> g_force_blocks{0};

extern "C" int64_t wmc_kernel_launch_count(void) { return g_launches.load(); }
extern "C" void wmc_debug_fail_next_allocs(int32_t n) { g_fail_allocs.store(n); }
extern "C" void wmc_debug_stall_copies(int32_t on) { g_debug_stall.store(on); }
extern "C" void wmc_set_fusion(int32_t on) { g_fuse.store(on); }
extern "C" void wmc_set_small_phase(int32_t on) { g_small_phase.store(on); }
extern "C" void wmc_set_dependent_launch(int32_t on) { g_pdl.store(on); }
extern "C" void wmc_set_tensor_cores(int32_t on) { g_tensor_cores.store(on); }
static std::atomic<int32_t> g_outer{1};  // short summed ranges: k4_outer in place of k4_dense
static std::atomic<int32_t> g_batched{1};  // walk nodes: k2_batched in place of the generic kernel
extern "C" void wmc_set_batched_pairs(int32_t on) { g_batched.store(on); }
extern "C" void wmc_set_outer_products(int32_t on) { g_outer.store(on); }
extern "C" void wmc_set_fp64_fallback(int32_t on) { g_fp64_fallback.store(on); }
extern "C" void wmc_set_chain_runs(int32_t max_tiles) { g_chain_runs.store(max_tiles < 0 ? 0 : max_tiles); }
extern "C" void wmc_set_cta_walk(int32_t on) { g_cta_walk.store(on ? 1 : 0); }

#define CUDA_TRY(x)                                                              \
  do {                                                                           \
    cudaError_t _e = (x);                                                        \
    if (_e != cudaSuccess) {                                                     \
      set_error("%s failed: %s (%s:%d)", #x, cudaGetErrorString(_e), __FILE__,   \
                __LINE__);                                                       \
      return WMC_ECUDA;                                                          \
    }                                                                            \
  } while (0)

static int dev_alloc(void **p, size_t bytes) {
  if (g_fail_allocs.load() > 0) {
    g_fail_allocs.fetch_sub(1);
    set_error("injected allocation failure (%zu bytes)", bytes);
    return WMC_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 256);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return WMC_ENOMEM;
  }
  return WMC_OK;
}

namespace {


enum Kind { L_K1, L_K2, L_K2T, L_K4, L_K2C, L_SMALL, L_CLAUSES, L_WEIGHTS, L_ONE, L_FINAL, L_MEMSET, L_K2CSEQ,
            L_BFP, L_BFPW, L_CTA, L_K2B };
enum Ty { TF = 0, TD = 1 };

struct Launch {
  Kind kind;
  int ti = TF, ta = TF, to = TF;  // K1 types; K2 uses ti
  int v = 1, kmax = 1, fmax = 1;  // K2 template choice
  int64_t blocks = 1;
  K1Params k1;
  K2Params k2;
  wmc::dev::K2TParams k2t;
  wmc::dev::K4Params k4;
  wmc::dev::K2BParams k2b;
  wmc::dev::K2CParams k2c;
  int chain_d = 0, chain_fast = 0, chain_grow = 0, chain_shrink = 0;
  int threads = 0;  // block size of a direct-load chain (0: kDirectThreads)
  int no_pdl = 0;   // chain launched in plain stream order (its launch before writes an S_i)
  int64_t id_sc[wmc::dev::kMaxChain] = {-1, -1, -1, -1, -1, -1};  // chain: S_1..S_D
  int64_t off_sc[wmc::dev::kMaxChain] = {-1, -1, -1, -1, -1, -1};
  int64_t meta_sc[wmc::dev::kMaxChain] = {-1, -1, -1, -1, -1, -1};
  size_t smem = 0;
  // relative byte offsets (patched with the workspace base at capture)
  int64_t off_a = -1, off_b = -1, off_c = -1;
  int64_t meta_a = -1, meta_b = -1, meta_c = -1;  // slot indices
  int64_t id_a = -1, id_b = -1, id_c = -1;        // tensor ids (A/P, B/S, C)
  int64_t one_off = -1, one_meta = -1;
  int64_t memset_off = 0, memset_bytes = 0;
  int memset_value = 0;
  double alg_bytes = 0;  // contraction: |A| + |B| + |C| bytes
  // run of chains in one launch (L_K2CSEQ): the chain launches it replaces,
  // its first entry in the state's parameter table, its counters' offset
  std::vector<Launch> chains;
  int64_t seq_first = 0, seq_ctr_off = 0;
};

}  // namespace

namespace wmc {

static std::atomic<uint64_t> g_state_serial{0};

// Walk options of one execution state (the process-wide defaults come from
// the wmc_set_* calls; the plan tuner builds states with others).
struct WalkOpts {
  int32_t fuse = -1;        // longest chain of frontier eliminations per pass (0 or 1: none; -1 by lanes)
  int32_t small_phase = 1;  // small-node phase
  int32_t chain_runs = 0;   // runs of chains in one launch: max tiles (0: off)
  int32_t cta_walk = 0;     // a small formula's whole walk in one block (when it fits)
};

struct ExecState {
  WalkOpts wo;
  // block floating point: block bits (-1: off), per tensor the exponent
  // array's byte offset (right after its mantissas) and block bits
  int32_t bfp_b = -1;
  std::vector<int64_t> t_eoff;
  std::vector<int8_t> t_bb;
  // one-block walk: leaf descriptors (its node program is h_snodes), the
  // shared memory it needs (metadata + tensor arena)
  std::vector<wmc::dev::CtaLeaf> h_cta;
  wmc::dev::CtaLeaf *d_cta = nullptr;
  int64_t cta_smem = 0, cta_meta = 0;  // total; before the arena
  // one-block walk: the nodes by level (a level's nodes are independent),
  // and the shared-memory offset and size (words) of the per-level tables
  std::vector<int64_t> cta_order;
  std::vector<int32_t> cta_level_end;  // per position: one past its level's last
  int64_t cta_lut_off = 0, cta_lut_words = 0;
  std::vector<int64_t> cta_off;  // shared-memory arena offset per tensor (-1: none; the root: none)
  uint64_t serial = ++g_state_serial;  // unique per state for the life of the process
  int32_t Q = 1, m = 0;
  int32_t Qp = 1;  // Q padded to 2^m: the query index is m bits
  bool f64 = false;
  std::vector<int64_t> t_off;   // byte offset of tensor data in the workspace
  std::vector<int64_t> t_meta;  // first metadata slot
  std::vector<int32_t> t_qc;
  std::vector<uint8_t> t_dbl;
  std::vector<int64_t> t_bytes;
  int64_t off_io = 0, off_flags = 0, off_err = 0, off_exp = 0, off_max = 0, off_min = 0, n_slots = 0;
  int64_t arena_bytes = 0, ws_bytes = 0;
  double alg_bytes = 0, flops = 0;
  int32_t max_roundings = 0;
  int32_t n_slice_vars = 0;   // index slicing: walks per execution = 2^n_slice_vars
  std::vector<Launch> launches;
  int64_t kernels_per_run = 0;
  // constant tables (device, owned)
  std::vector<ClauseLeaf> h_clause;
  std::vector<int64_t> h_first, h_woff, h_wmeta;
  std::vector<wmc::dev::SNode> h_snodes;   // small-node phase
  std::vector<wmc::dev::STask> h_stasks;
  wmc::dev::SNode *d_snodes = nullptr;
  wmc::dev::STask *d_stasks = nullptr;
  int64_t off_sp = 0;                      // task counter + per-node completion counters
  // runs of chains (k2_chain_seq): parameters with workspace offsets for
  // pointers, and two counters per chain (zeroed with the flags)
  std::vector<wmc::dev::K2CParams> h_seq;
  wmc::dev::K2CParams *d_seq = nullptr;
  int64_t off_seqctr = 0;
  int64_t n_clause_entries = 0;
  ClauseLeaf *d_clause = nullptr;
  int64_t *d_first = nullptr, *d_woff = nullptr, *d_wmeta = nullptr;
  bool dev_ready = false;
  std::map<uintptr_t, cudaGraphExec_t> graphs;
  cudaStream_t capture_stream = nullptr;
  // resources of the host-pointer path
  void *own_ws = nullptr;
  double *d_w = nullptr;          // [2][Q][n_vars]
  // results: [Q] mantissas, [Q] exponents, [Q] flags in one allocation
  // (one device-to-host copy), mirrored in pinned host memory
  double *d_res_mant = nullptr;
  int64_t *d_res_exp = nullptr;
  uint32_t *d_res_flags = nullptr;
  double *h_res_mant = nullptr;
  int64_t *h_res_exp = nullptr;
  uint32_t *h_res_flags = nullptr;
  // pinned staging of small calls' inputs: the call descriptor, then the
  // weights (w_pos, w_neg), so that each crosses in one copy from pinned
  // memory instead of through the driver's pageable path
  unsigned char *h_stage = nullptr;
  std::mutex run_mu;    // the owned workspace of the host-pointer path
  std::mutex graph_mu;  // graphs map

  ~ExecState() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    cudaFree(d_clause); cudaFree(d_first); cudaFree(d_woff); cudaFree(d_wmeta);
    cudaFree(d_snodes); cudaFree(d_stasks); cudaFree(d_seq); cudaFree(d_cta);
    cudaFree(own_ws); cudaFree(d_w); cudaFree(d_res_mant);
    cudaFreeHost(h_res_mant); cudaFreeHost(h_stage);
  }
};

Plan::~Plan() {}
void destroy_exec_state(ExecState *st) { delete st; }

}  // namespace wmc

// ------------------------------------------------------------ layout

namespace {

// Full label list of a tensor at batch size 2^m: the m query bits occupy
// the lowest positions (labels -1 .. -m) of every weight-dependent tensor.
std::vector<int32_t> full_labels(const TensorInfo &t, int32_t m) {
  std::vector<int32_t> L;
  if (t.has_q)
    for (int32_t i = 0; i < m; ++i) L.push_back(-1 - i);
  L.insert(L.end(), t.labels.begin(), t.labels.end());
  return L;
}

int pos_of(const std::vector<int32_t> &L, int32_t v) {
  for (size_t i = 0; i < L.size(); ++i)
    if (L[i] == v) return (int)i;
  return -1;
}

// Chooses K2 (streaming, P the operand whose kept indices stay in order)
// when its structural conditions hold, else K1.
bool try_k2(const std::vector<int32_t> &LP, const std::vector<int32_t> &LS,
            const std::vector<int32_t> &LC, bool f64, K2Params &p, int &vmax, int &kmax,
            int &fmax) {
  std::vector<int32_t> keptP, cP, freeS, summed;
  for (int32_t l : LP) if (pos_of(LC, l) >= 0) keptP.push_back(l);
  for (int32_t l : LC) if (pos_of(LP, l) >= 0) cP.push_back(l);
  if (keptP != cP) return false;
  for (int32_t l : LS) if (pos_of(LC, l) >= 0 && pos_of(LP, l) < 0) freeS.push_back(l);
  for (int32_t l : LP) if (pos_of(LC, l) < 0) summed.push_back(l);
  for (int32_t l : LS) if (pos_of(LC, l) < 0 && pos_of(LP, l) < 0) summed.push_back(l);
  // one summation order for every kernel and batch size: ascending label
  std::sort(summed.begin(), summed.end());
  const int k = (int)summed.size(), f = (int)freeS.size();
  if (k > 4 || f > 4 || LS.size() > 16) return false;
  std::memset(&p, 0, sizeof(p));
  p.k = k;
  p.f = f;
  std::vector<int> insA, insC;
  for (int32_t l : summed) { int q = pos_of(LP, l); if (q >= 0) insA.push_back(q); }
  for (int32_t l : freeS) insC.push_back(pos_of(LC, l));
  std::sort(insA.begin(), insA.end());
  std::sort(insC.begin(), insC.end());
  // four summed or four S-free bits: one lane per thread (registers)
  const int want_v = std::max(k, f) == 4 ? 0 : (f64 ? 1 : 2);
  int vbits = want_v;
  const int rC = (int)LC.size();
  if (rC - f < vbits) vbits = 0;
  for (int q : insA) if (q < vbits) vbits = 0;
  for (int q : insC) if (q < vbits) vbits = 0;
  p.vbits = vbits;
  p.log2_nu = rC - f - vbits;
  p.n_insA = (int)insA.size();
  p.n_insC = (int)insC.size();
  for (size_t i = 0; i < insA.size(); ++i) p.insA[i] = (int8_t)insA[i];
  for (size_t i = 0; i < insC.size(); ++i) p.insC[i] = (int8_t)insC[i];
  // S batch bits (in P, S and C): lanes below vbits go to dBv, the rest
  // are grouped into runs that are consecutive in both C and S
  std::vector<std::pair<int, int>> bb;  // (C position, S position)
  for (size_t j = 0; j < LS.size(); ++j) {
    int32_t l = LS[j];
    int pc = pos_of(LC, l), pp = pos_of(LP, l);
    if (pc < 0 || pp < 0) continue;  // not a batch index
    if (pc < vbits) {
      for (int e = 0; e < (1 << vbits); ++e)
        if ((e >> pc) & 1) p.dBv[e] |= 1u << j;
    } else {
      bb.push_back({pc, (int)j});
    }
  }
  std::sort(bb.begin(), bb.end());
  int nseg = 0;
  for (size_t i = 0; i < bb.size();) {
    size_t j = i + 1;
    while (j < bb.size() && bb[j].first == bb[j - 1].first + 1 && bb[j].second == bb[j - 1].second + 1) ++j;
    if (nseg >= 16) return false;
    p.seg_c[nseg] = (int8_t)bb[i].first;
    p.seg_b[nseg] = (int8_t)bb[i].second;
    p.seg_len[nseg] = (int8_t)(j - i);
    ++nseg;
    i = j;
  }
  p.n_seg = nseg;
  // S lanes: 1 = contiguous (vector load), 2 = one value for all lanes
  bool contiguous = true, broadcast = true;
  for (int e = 0; e < (1 << vbits); ++e) {
    contiguous &= (p.dBv[e] == (uint32_t)e);
    broadcast &= (p.dBv[e] == 0u);
  }
  p.b_vec = contiguous ? 1 : (broadcast ? 2 : 0);
  for (int s = 0; s < (1 << k); ++s) {
    uint32_t da = 0, db = 0;
    for (int i = 0; i < k; ++i) {
      if (!((s >> i) & 1)) continue;
      int qa = pos_of(LP, summed[i]), qb = pos_of(LS, summed[i]);
      if (qa >= 0) da |= 1u << qa;
      if (qb >= 0) db |= 1u << qb;
    }
    p.dA[s] = da;
    p.dBs[s] = db;
  }
  for (int ff = 0; ff < (1 << f); ++ff) {
    uint32_t db = 0, dc = 0;
    for (int i = 0; i < f; ++i) {
      if (!((ff >> i) & 1)) continue;
      db |= 1u << pos_of(LS, freeS[i]);
      dc |= 1u << pos_of(LC, freeS[i]);
    }
    p.dBf[ff] = db;
    p.dC[ff] = dc;
  }
  vmax = 1 << vbits;
  kmax = std::max(k, f) <= 1 ? 1 : (std::max(k, f) <= 2 ? 2 : (std::max(k, f) == 3 ? 3 : 4));
  // four summed or S-free bits: 16 x 16 S terms per unit, read from shared
  // memory (S staged once per block, at most 2^12 entries)
  p.s_log2 = (int32_t)LS.size();
  p.s_staged = (kmax == 4 && vbits == 0 && LS.size() <= 12) ? 1 : 0;
  p.s_contig = 0;
  if (p.s_staged && k == 4) {
    p.s_contig = 1;
    for (int s = 0; s < 16; ++s) p.s_contig &= p.dBs[s] == (uint32_t)s;
  }
  fmax = kmax;
  return true;
}

// Tiles for the TMA-staged variant of K2; false when the node is too
// small or its lanes would not keep one query per thread.
bool try_k2_tma(const K2Params &p2, const std::vector<int32_t> &LP, const std::vector<int32_t> &LS,
                bool f64, bool p_has_q, bool s_has_q, int32_t Qp, wmc::dev::K2TParams &tp,
                size_t &smem) {
  if (p2.k > 3 || p2.f > 3) return false;  // the staged variant's tables hold 8 summed assignments
  const int V = 1 << p2.vbits;
  const int J = V == 1 ? 4 : 2;  // work units per thread per tile (<= kMaxJ)
  int tb = 0;
  while ((1 << tb) < dev::kThreads * V * J) ++tb;
  const int total_w_log2 = p2.log2_nu + p2.vbits;
  if (total_w_log2 < tb + 3) return false;
  if (p_has_q && (dev::kThreads * V) % Qp != 0) return false;
  if (LS.size() > 13) return false;  // S is staged in shared memory
  std::vector<int> ins(p2.insA, p2.insA + p2.n_insA);
  std::vector<int> kept;
  for (int q = 0; q < (int)LP.size(); ++q)
    if (std::find(ins.begin(), ins.end(), q) == ins.end()) kept.push_back(q);
  if ((int)kept.size() < tb) return false;
  const int top = kept[(size_t)tb - 1] + 1;
  std::vector<int> low, high;
  for (int q : ins) (q < top ? low : high).push_back(q);
  std::memset(&tp, 0, sizeof(tp));
  tp.k = p2;
  tp.tb = tb;
  tp.run_log2 = top;
  tp.nruns = 1 << (int)high.size();
  tp.n_lowA = (int)low.size();
  tp.s_log2 = (int)LS.size();
  // P's scale can be folded into the staged S when S's query bits are
  // exactly P's (both carry the query index at their lowest positions)
  tp.fold_sa = (p_has_q && s_has_q) ? 1 : 0;
  for (size_t j = 0; j < low.size(); ++j) tp.lowA[j] = (int8_t)low[j];
  for (int r = 0; r < tp.nruns; ++r) {
    uint32_t o = 0;
    for (size_t j = 0; j < high.size(); ++j)
      if ((r >> j) & 1) o |= 1u << high[j];
    tp.run_off[r] = o;
  }
  for (int s = 0; s < (1 << p2.k); ++s) {
    const uint32_t da = p2.dA[s];
    uint32_t r = 0;
    for (size_t j = 0; j < high.size(); ++j)
      if ((da >> high[j]) & 1) r |= 1u << j;
    tp.sA_off[s] = (r << top) | (da & ((1u << top) - 1u));
  }
  const size_t es = f64 ? 8 : 4;
  smem = (size_t)dev::kStages * ((size_t)tp.nruns << top) * es + (((es << tp.s_log2) + 15) & ~(size_t)15) +
         (16 + es) * (size_t)Qp;  // stages, staged S (16-byte padded), per-query max/min/scale
  return smem <= 160 * 1024;
}

// Chain of D frontier eliminations (k2_chain): node i = C_{i-1} . S_i -> C_i
// (C_0 = P) for i = 1..D, each summing one index x_i of P; step i adds y_i
// at x_i's position, except that the first step may also add a second
// index z at the top (growth) and the last may add none (shrink; the
// indices above x_D move down one position).  Labels are full
// (with query bits).  `allow_gs` admits growth and shrink steps.  `fast`
// is set when the chain has the FAST layout (S_i depends on no chain index
// but the two added last; contiguous or broadcast lanes; P's scale folds
// into S_1).
bool try_chain(const std::vector<int32_t> &LP, const std::vector<std::vector<int32_t>> &LS,
               const std::vector<std::vector<int32_t>> &LC, bool f64, bool p_has_q, bool s1_has_q,
               int32_t Qp, bool allow_gs, wmc::dev::K2CParams &cp, int &v_out, bool &fast, int &grow,
               int &shrink, size_t &smem, bool one_lane = false) {
  const int D = (int)LS.size();
  if (D < 2 || D > wmc::dev::kMaxChain || (int)LC.size() != D) return false;
  const int rP = (int)LP.size();
  const int nthr = wmc::dev::kChainNW * 32;
  std::vector<int32_t> x(D), y(D, INT32_MIN);
  std::vector<int> p(D);
  int32_t z = INT32_MIN;
  grow = shrink = 0;
  std::vector<int32_t> cur = LP;
  for (int i = 0; i < D; ++i) {
    const std::vector<int32_t> &S = LS[(size_t)i], &C = LC[(size_t)i];
    std::vector<int32_t> summed, added;
    for (int32_t l : cur) if (pos_of(C, l) < 0) summed.push_back(l);
    for (int32_t l : S) if (pos_of(C, l) < 0 && pos_of(cur, l) < 0) summed.push_back(l);
    for (int32_t l : S) if (pos_of(C, l) >= 0 && pos_of(cur, l) < 0) added.push_back(l);
    if (summed.size() != 1 || S.size() > 13) return false;
    x[(size_t)i] = summed[0];
    p[(size_t)i] = pos_of(LP, x[(size_t)i]);
    if (p[(size_t)i] < 0 || pos_of(cur, x[(size_t)i]) != p[(size_t)i] || pos_of(S, x[(size_t)i]) < 0) return false;
    for (int j = 0; j < i; ++j) if (p[(size_t)j] == p[(size_t)i]) return false;
    std::vector<int32_t> want = cur;
    if (added.size() == 1) {
      y[(size_t)i] = added[0];
      want[(size_t)p[(size_t)i]] = y[(size_t)i];
    } else if (added.size() == 2 && i == 0 && allow_gs) {
      // one added index takes x_0's position, the other the new top one
      const int32_t a0 = added[0], a1 = added[1];
      const bool first_in_place = pos_of(C, a0) == p[0];
      y[0] = first_in_place ? a0 : a1;
      z = first_in_place ? a1 : a0;
      want[(size_t)p[0]] = y[0];
      want.push_back(z);
      grow = 1;
    } else if (added.empty() && i == D - 1 && allow_gs && !grow) {
      want.erase(want.begin() + p[(size_t)i]);  // the indices above x_D move down
      shrink = 1;
    } else {
      return false;
    }
    if (want != C) return false;
    cur = want;
  }
  if (grow && shrink) return false;  // P and C of one size: not needed by any layout seen
  // five or six steps: float32, no growth step, one lane (direct loads,
  // k2_chain_direct)
  const bool direct = D > 4;
  if (direct && (f64 || grow)) return false;
  const std::vector<int32_t> &LCD = LC.back();
  const int NB = D + grow;
  std::memset(&cp, 0, sizeof(cp));
  std::vector<int> ins(p.begin(), p.end());
  std::sort(ins.begin(), ins.end());
  // C positions of the added indices (kept indices keep their order)
  std::vector<int> insc;
  for (int i = 0; i < D; ++i) if (y[(size_t)i] != INT32_MIN) insc.push_back(pos_of(LCD, y[(size_t)i]));
  if (grow) insc.push_back(pos_of(LCD, z));
  std::sort(insc.begin(), insc.end());
  // lanes: at most 64 registers of chain values per thread, 32 KB tiles
  int vbits = f64 ? (NB <= 3 ? 1 : 0) : (NB <= 3 ? 2 : 1);
  if ((direct && one_lane) || vbits < 0 || rP - D < vbits || ins[0] < vbits || (!insc.empty() && insc[0] < vbits))
    vbits = 0;
  const int V = 1 << vbits;
  if ((grow || shrink) && (f64 || (V == 1 && !direct))) return false;  // instantiated for float lanes only
  if (p_has_q && (nthr * V) % Qp != 0) return false;
  cp.vbits = vbits;
  cp.log2_nu = rP - D - vbits;
  cp.n_ins = D;
  for (int i = 0; i < D; ++i) cp.ins[i] = (int8_t)ins[(size_t)i];
  cp.n_insc = (int)insc.size();
  for (size_t i = 0; i < insc.size(); ++i) cp.insc[i] = (int8_t)insc[i];
  cp.fold_sp = (p_has_q && !s1_has_q) ? 0 : 1;
  fast = cp.fold_sp != 0;
  // the chain index behind state bit j at step i: y_j (j < i), x_j (j > i), z (bit D)
  auto chain_bit_of = [&](int i, int32_t l) {
    for (int j = 0; j < D; ++j) {
      if (j == i) continue;
      if (l == (j < i ? y[(size_t)j] : x[(size_t)j])) return j;
    }
    if (grow && i > 0 && l == z) return D;
    return -1;
  };
  auto label_of_bit = [&](int i, int j) { return j == D ? z : (j < i ? y[(size_t)j] : x[(size_t)j]); };
  const size_t es = f64 ? 8 : 4;
  bool any_broadcast = false;
  for (int i = 0; i < D; ++i) {
    const std::vector<int32_t> &S = LS[(size_t)i];
    std::vector<std::pair<int, int>> bb;
    uint32_t deps = 0;
    for (size_t j = 0; j < S.size(); ++j) {
      const int32_t l = S[j];
      if (l == x[(size_t)i] || l == y[(size_t)i] || (i == 0 && grow && l == z)) continue;
      const int cb = chain_bit_of(i, l);
      if (cb >= 0) { deps |= 1u << cb; continue; }
      const int pc = pos_of(LCD, l);
      if (pc < 0 || std::find(insc.begin(), insc.end(), pc) != insc.end()) return false;
      if (pc < vbits) {
        for (int e = 0; e < V; ++e)
          if ((e >> pc) & 1) cp.dv[i][e] |= 1u << j;
      } else {
        bb.push_back({pc, (int)j});
      }
    }
    if (deps & ~wmc::dev::chain_deps(D, true, grow, i)) fast = false;
    std::sort(bb.begin(), bb.end());
    int nseg = 0;
    for (size_t a = 0; a < bb.size();) {
      size_t b = a + 1;
      while (b < bb.size() && bb[b].first == bb[b - 1].first + 1 && bb[b].second == bb[b - 1].second + 1) ++b;
      if (nseg >= 8) return false;
      cp.seg_c[i][nseg] = (int8_t)bb[a].first;
      cp.seg_b[i][nseg] = (int8_t)bb[a].second;
      cp.seg_len[i][nseg] = (int8_t)(b - a);
      ++nseg;
      a = b;
    }
    cp.n_seg[i] = nseg;
    bool contiguous = true, broadcast = true;
    for (int e = 0; e < V; ++e) {
      contiguous &= (cp.dv[i][e] == (uint32_t)e);
      broadcast &= (cp.dv[i][e] == 0u);
    }
    cp.b_vec[i] = contiguous ? 1 : (broadcast ? 2 : 0);
    if (!contiguous && V > 1) any_broadcast = true;
    const int sx = pos_of(S, x[(size_t)i]);
    const int sy = y[(size_t)i] != INT32_MIN ? pos_of(S, y[(size_t)i]) : -1;
    const int sz = (i == 0 && grow) ? pos_of(S, z) : -1;
    const uint32_t n_av = (grow && i == 0) ? 4u : 2u;  // added-value combinations the step reads
    if ((n_av << NB) > (uint32_t)wmc::dev::kChainDRow) return false;
    for (uint32_t st = 0; st < (1u << NB); ++st)
      for (uint32_t av = 0; av < n_av; ++av) {
        uint32_t o = 0;
        if ((st >> i) & 1u) o |= 1u << sx;
        if ((av & 1u) && sy >= 0) o |= 1u << sy;
        if ((av & 2u) && sz >= 0) o |= 1u << sz;
        for (int j = 0; j < NB; ++j) {
          if (j == i || !((st >> j) & 1u)) continue;
          if (j == D && i == 0) continue;  // z is added by step 0 itself
          const int32_t l = label_of_bit(i, j);
          const int sj = l == INT32_MIN ? -1 : pos_of(S, l);
          if (sj >= 0) o |= 1u << sj;
        }
        cp.d[i][st | (av << NB)] = o * (uint32_t)es;
      }
    cp.s_log2[i] = (int)S.size();
  }
  // growth and shrink steps: FAST variants with contiguous lanes only
  if ((grow || shrink) && (!fast || any_broadcast)) return false;
  if (direct) {
    // units are the assignments of P's other indices (with V lanes); a
    // thread's units share its lanes (the stride is a multiple of the lane
    // count), so no added index may sit below the query bits
    if (!fast || (V > 1 && any_broadcast)) return false;
    int m = 0;
    while ((1 << m) < Qp) ++m;
    if ((p_has_q && ins[0] < m) || (!insc.empty() && insc[0] < m)) return false;
    cp.units = 1;
    cp.tb = 0;
    for (uint32_t st = 0; st < (1u << D); ++st) {
      uint32_t da = 0;
      for (int j = 0; j < D; ++j)
        if ((st >> j) & 1u) da |= 1u << p[(size_t)j];
      cp.pA[st] = da;  // element offset in P
    }
    for (uint32_t st = 0; st < (1u << NB); ++st) {
      uint32_t dc = 0;
      for (int j = 0; j < NB; ++j)
        if (((st >> j) & 1u) && y[(size_t)j] != INT32_MIN) dc |= 1u << pos_of(LCD, y[(size_t)j]);
      cp.dC[st] = dc;
    }
    size_t s_off = 0, s_copy = 0;
    for (int i = 0; i < D; ++i) {
      cp.s_bytes_off[i] = (uint32_t)s_off;
      s_off += ((es << cp.s_log2[i]) + 15) & ~(size_t)15;
      s_copy += es << cp.s_log2[i];
    }
    cp.s_bytes_off[D] = (uint32_t)s_off;
    cp.s_copy_bytes = (uint32_t)s_copy;
    smem = s_off + 16 * (size_t)Qp;
    if (smem > 220 * 1024) return false;
    v_out = V;
    return true;
  }
  // tiling of P over its kept indices: 2 work units per thread when 16
  // chain states would leave runs of only 2 KB (bulk copies that short
  // lower the read rate); a growth chain's 32 states per unit already
  // fill the registers (one unit measured ~1% faster)
  cp.units = (D == 4 && !f64 && !grow) ? 2 : 1;  // growth chains hold 32 states: one unit
  int tb = 0;
  while ((1 << tb) < nthr * V * cp.units) ++tb;
  if (cp.units == 2 && cp.log2_nu + vbits < tb + 3) { cp.units = 1; --tb; }
  {
    // two stages of two-unit tiles must fit beside the staged S_i (large
    // batches carry the query bits in every S_i: 2^13 entries at Q = 512)
    size_t s_need = (16 + (size_t)D * es) * (size_t)Qp;
    for (int i = 0; i < D; ++i) s_need += ((es << cp.s_log2[i]) + 15) & ~(size_t)15;
    if (cp.units == 2 && 2 * ((size_t)es << (tb + D)) + s_need > 220 * 1024) { cp.units = 1; --tb; }
  }
  if (cp.log2_nu + vbits < tb + 3) return false;
  std::vector<int> kept;
  for (int q = 0; q < rP; ++q)
    if (std::find(p.begin(), p.end(), q) == p.end()) kept.push_back(q);
  if ((int)kept.size() < tb) return false;
  const int top = kept[(size_t)tb - 1] + 1;
  std::vector<int> lowv, highv;
  for (int q : ins) (q < top ? lowv : highv).push_back(q);
  cp.tb = tb;
  cp.run_log2 = top;
  cp.nruns = 1 << (int)highv.size();
  cp.n_low = (int)lowv.size();
  for (size_t j = 0; j < lowv.size(); ++j) cp.low[j] = (int8_t)lowv[j];
  for (int r = 0; r < cp.nruns; ++r) {
    uint32_t o = 0;
    for (size_t j = 0; j < highv.size(); ++j)
      if ((r >> j) & 1) o |= 1u << highv[j];
    cp.run_off[r] = o;
  }
  for (uint32_t st = 0; st < (1u << D); ++st) {
    uint32_t da = 0;
    for (int j = 0; j < D; ++j)
      if ((st >> j) & 1u) da |= 1u << p[(size_t)j];
    uint32_t r = 0;
    for (size_t j = 0; j < highv.size(); ++j)
      if ((da >> highv[j]) & 1) r |= 1u << j;
    cp.pA[st] = (uint32_t)((((size_t)r << top) | (da & ((1u << top) - 1u))) * es);
  }
  // C offsets of the final states (bit D-1 of a shrink chain stays 0)
  for (uint32_t st = 0; st < (1u << NB); ++st) {
    uint32_t dc = 0;
    for (int j = 0; j < NB; ++j) {
      if (!((st >> j) & 1u)) continue;
      const int32_t l = j == D ? z : y[(size_t)j];
      if (l == INT32_MIN) continue;
      dc |= 1u << pos_of(LCD, l);
    }
    cp.dC[st] = dc;
  }
  // shared memory: stages, the staged S_i (16-byte aligned bulk copies),
  // per-lane max, min and D scales
  size_t s_off = 0, s_copy = 0;
  for (int i = 0; i < D; ++i) {
    cp.s_bytes_off[i] = (uint32_t)s_off;
    s_off += ((es << cp.s_log2[i]) + 15) & ~(size_t)15;
    s_copy += es << cp.s_log2[i];
    if ((es << cp.s_log2[i]) % 16) return false;
  }
  cp.s_bytes_off[D] = (uint32_t)s_off;
  cp.s_copy_bytes = (uint32_t)s_copy;
  const size_t tile_bytes = ((size_t)cp.nruns << top) * es;
  const size_t fixed = s_off + (16 + (size_t)D * es) * (size_t)Qp;
  const size_t limit = 220 * 1024;
  int stages = 0;
  for (int n = wmc::dev::kMaxStagesC; n >= 2; --n)
    if ((size_t)n * tile_bytes + fixed <= limit) { stages = n; break; }
  if (!stages) return false;
  cp.n_stages = stages;
  smem = (size_t)stages * tile_bytes + fixed;
  v_out = V;
  return true;
}

// Dense batched-matrix-product form (K4): every summed index in both
// operands, at least 2^6 values of i and of j, 2^5 of s; query bits only
// as batch indices.
// Batched small contraction (K2B): every index of A and of B either kept
// (in C) or summed in both (at most 2 bits).  Of the kept indices that
// only one operand holds, up to fA + k <= 4 of A's and k + fB <= 3 of B's
// (fA + fB <= 5) are free indices held in registers; the rest, and the
// query lanes, are batch indices, enumerated in C's order (at least 2^8
// assignments), over which an operand that lacks one is broadcast.
bool try_k2b(const std::vector<int32_t> &LA, const std::vector<int32_t> &LB, const std::vector<int32_t> &LC,
             wmc::dev::K2BParams &p, int64_t bytes_a = 0, int64_t bytes_b = 0) {
  std::vector<int32_t> fa, fb, sm;
  for (int32_t l : LA) {
    const bool inB = pos_of(LB, l) >= 0, inC = pos_of(LC, l) >= 0;
    if (!inC && inB) sm.push_back(l);
    else if (!inC) return false;  // summed in A only
    else if (!inB && l >= 0) fa.push_back(l);
  }
  for (int32_t l : LB) {
    const bool inA = pos_of(LA, l) >= 0, inC = pos_of(LC, l) >= 0;
    if (!inC && !inA) return false;  // summed in B only
    if (inC && !inA && l >= 0) fb.push_back(l);
  }
  const int k = (int)sm.size();
  if (k > 2) return false;
  // free indices beyond the registers' budget become batch indices the
  // other operand is broadcast over (re-read from L2: only when it is at
  // most 32 MB)
  const size_t keep_a = std::min<size_t>(fa.size(), (size_t)(4 - k));
  const size_t keep_b = std::min<size_t>({fb.size(), (size_t)(3 - k), (size_t)5 - keep_a});
  const int64_t kL2 = int64_t(32) << 20;
  if ((fa.size() > keep_a && bytes_b > kL2) || (fb.size() > keep_b && bytes_a > kL2)) return false;
  fa.resize(keep_a);
  fb.resize(keep_b);
  const int nfa = (int)fa.size(), nfb = (int)fb.size();
  std::vector<int32_t> bC;  // every other index of C, in C's order
  for (int32_t l : LC)
    if (std::find(fa.begin(), fa.end(), l) == fa.end() && std::find(fb.begin(), fb.end(), l) == fb.end())
      bC.push_back(l);
  if (bC.size() < 8 || bC.size() > 31) return false;
  std::memset(&p, 0, sizeof(p));
  p.log2_nu = (int32_t)bC.size();
  p.fA = nfa; p.fB = nfb; p.k = k;
  for (size_t j = 0; j < LC.size(); ++j)
    if (std::find(bC.begin(), bC.end(), LC[j]) == bC.end()) p.insC[p.n_insC++] = (int8_t)j;
  for (size_t j = 0; j < bC.size(); ++j) {
    p.posA[j] = (int8_t)pos_of(LA, bC[j]);
    p.posB[j] = (int8_t)pos_of(LB, bC[j]);
  }
  auto bit = [&](const std::vector<int32_t> &L, int32_t l) { return 1u << pos_of(L, l); };
  for (int i = 0; i < (1 << (nfa + k)); ++i) {
    uint32_t o = 0;
    for (int j = 0; j < nfa; ++j) if ((i >> j) & 1) o |= bit(LA, fa[(size_t)j]);
    for (int j = 0; j < k; ++j) if ((i >> (nfa + j)) & 1) o |= bit(LA, sm[(size_t)j]);
    p.offA[i] = o;
  }
  for (int i = 0; i < (1 << (k + nfb)); ++i) {
    uint32_t o = 0;
    for (int j = 0; j < k; ++j) if ((i >> j) & 1) o |= bit(LB, sm[(size_t)j]);
    for (int j = 0; j < nfb; ++j) if ((i >> (k + j)) & 1) o |= bit(LB, fb[(size_t)j]);
    p.offB[i] = o;
  }
  for (int i = 0; i < (1 << (nfa + nfb)); ++i) {
    uint32_t o = 0;
    for (int j = 0; j < nfa; ++j) if ((i >> j) & 1) o |= bit(LC, fa[(size_t)j]);
    for (int j = 0; j < nfb; ++j) if ((i >> (nfa + j)) & 1) o |= bit(LC, fb[(size_t)j]);
    p.offC[i] = o;
  }
  return true;
}

bool try_k4(const std::vector<int32_t> &LA, const std::vector<int32_t> &LB,
            const std::vector<int32_t> &LC, bool f64, wmc::dev::K4Params &p) {
  std::vector<int32_t> iv, jv, sv, bv;
  for (int32_t l : LA) {
    const bool inB = pos_of(LB, l) >= 0, inC = pos_of(LC, l) >= 0;
    if (inC && inB) bv.push_back(l);
    else if (inC) iv.push_back(l);
    else if (inB) sv.push_back(l);
    else return false;  // summed in A only
  }
  for (int32_t l : LB) {
    const bool inA = pos_of(LA, l) >= 0, inC = pos_of(LC, l) >= 0;
    if (!inA && inC) jv.push_back(l);
    else if (!inA && !inC) return false;  // summed in B only
  }
  for (int32_t l : iv) if (l < 0) return false;
  for (int32_t l : jv) if (l < 0) return false;
  if (iv.size() < 6 || jv.size() < 6 || sv.size() < 1) return false;
  if (!f64 && sv.size() > 16) return false;  // float64 accumulation beyond 2^16 terms (k1)
  if (iv.size() + jv.size() + sv.size() + bv.size() > 62) return false;
  std::sort(sv.begin(), sv.end());  // the canonical summation order
  auto by_pos = [](const std::vector<int32_t> &L) {
    return [&L](int32_t x, int32_t y) { return pos_of(L, x) < pos_of(L, y); };
  };
  std::sort(iv.begin(), iv.end(), by_pos(LA));
  std::sort(jv.begin(), jv.end(), by_pos(LB));
  std::memset(&p, 0, sizeof(p));
  p.ni = (int32_t)iv.size(); p.nj = (int32_t)jv.size(); p.ns = (int32_t)sv.size(); p.nb = (int32_t)bv.size();
  for (size_t t = 0; t < iv.size(); ++t) { p.iA[t] = (int8_t)pos_of(LA, iv[t]); p.iC[t] = (int8_t)pos_of(LC, iv[t]); }
  for (size_t t = 0; t < jv.size(); ++t) { p.jB[t] = (int8_t)pos_of(LB, jv[t]); p.jC[t] = (int8_t)pos_of(LC, jv[t]); }
  for (size_t t = 0; t < sv.size(); ++t) { p.sA[t] = (int8_t)pos_of(LA, sv[t]); p.sB[t] = (int8_t)pos_of(LB, sv[t]); }
  for (size_t t = 0; t < bv.size(); ++t) {
    p.bA[t] = (int8_t)pos_of(LA, bv[t]); p.bB[t] = (int8_t)pos_of(LB, bv[t]); p.bC[t] = (int8_t)pos_of(LC, bv[t]);
  }
  int minAi = 99, minAs = 99, minBj = 99, minBs = 99, minCi = 99, minCj = 99;
  for (int t = 0; t < p.ni; ++t) { minAi = std::min(minAi, (int)p.iA[t]); minCi = std::min(minCi, (int)p.iC[t]); }
  for (int t = 0; t < p.nj; ++t) { minBj = std::min(minBj, (int)p.jB[t]); minCj = std::min(minCj, (int)p.jC[t]); }
  for (int t = 0; t < p.ns; ++t) { minAs = std::min(minAs, (int)p.sA[t]); minBs = std::min(minBs, (int)p.sB[t]); }
  p.a_i_fast = minAi < minAs;
  p.b_j_fast = minBj < minBs;
  p.c_i_fast = minCi < minCj;
  return true;
}

// k4_outer in place of k4_dense (wmc_contract_pair): at most 2 summed bits,
// one query lane, C's low 10 bits the first 10 free bits of A (u = i) or of
// B (u = j), and at least 2^8 blocks of 1024 x 64 outputs.  Sets p.outer_u;
// returns the block count, or 0 to keep k4_dense.
int64_t k4_outer_pick(wmc::dev::K4Params &p) {
  p.outer_u = 0;
  if (p.ns > 2 || p.mc.Qc != 1) return 0;
  auto low10 = [](const int8_t *pos, int n) {
    if (n < 10) return false;
    for (int t = 0; t < 10; ++t)
      if (pos[t] != t) return false;
    return true;
  };
  int nu = 0, nv = 0;
  if (low10(p.iC, p.ni)) { p.outer_u = 1; nu = p.ni; nv = p.nj; }
  else if (low10(p.jC, p.nj)) { p.outer_u = 2; nu = p.nj; nv = p.ni; }
  else return 0;
  const int blog2 = nu - 10 + nv - 6 + p.nb;
  if (nv < 6 || blog2 < 8 || blog2 > 30) { p.outer_u = 0; return 0; }
  return (int64_t)1 << blog2;
}

void fill_k1(const std::vector<int32_t> &LA, const std::vector<int32_t> &LB,
             const std::vector<int32_t> &LC, K1Params &p) {
  std::memset(&p, 0, sizeof(p));
  std::vector<int32_t> summed;
  for (int32_t l : LA) if (pos_of(LC, l) < 0) summed.push_back(l);
  for (int32_t l : LB) if (pos_of(LC, l) < 0 && pos_of(LA, l) < 0) summed.push_back(l);
  std::sort(summed.begin(), summed.end());
  p.rC = (int32_t)LC.size();
  p.k = (int32_t)summed.size();
  for (int j = 0; j < 32; ++j) { p.posA[j] = -1; p.posB[j] = -1; }
  for (int j = 0; j < 24; ++j) { p.sposA[j] = -1; p.sposB[j] = -1; }
  for (size_t j = 0; j < LC.size(); ++j) {
    p.posA[j] = (int8_t)pos_of(LA, LC[j]);
    p.posB[j] = (int8_t)pos_of(LB, LC[j]);
  }
  for (size_t i = 0; i < summed.size(); ++i) {
    p.sposA[i] = (int8_t)pos_of(LA, summed[i]);
    p.sposB[i] = (int8_t)pos_of(LB, summed[i]);
  }
}

int64_t grid_for(uint64_t work) {
  const int64_t max_blocks = 148 * 8;
  uint64_t b = (work + dev::kThreads - 1) / dev::kThreads;
  if (b < 1) b = 1;
  return (int64_t)std::min<uint64_t>(b, (uint64_t)max_blocks);
}

}  // namespace

static WalkOpts walk_opts_now() {
  WalkOpts wo;
  wo.fuse = g_fuse.load();
  wo.small_phase = g_small_phase.load();
  wo.chain_runs = g_chain_runs.load();
  wo.cta_walk = g_cta_walk.load();
  return wo;
}

// Builds the host-side layout for batch size Q (no device work).
static int build_exec(Plan &plan, int32_t Q, ExecState &st, bool plain = false, bool force_f64 = false,
                      const WalkOpts *wo = nullptr) {
  st.wo = wo ? *wo : walk_opts_now();
  st.bfp_b = (plan.bfp_b >= 0 && !plain && !force_f64) ? plan.bfp_b : -1;
  if (st.bfp_b >= 0) { st.wo.fuse = 0; st.wo.small_phase = 0; st.wo.chain_runs = 0; }
  st.Q = Q;
  int32_t m = 0;
  while ((1 << m) < Q) ++m;
  // a lone float32 query on a small network runs as two lanes (the second
  // repeats it, as padding lanes do): such walks are bound by launch
  // latency, and vector lanes let the growth and shrink steps join chains
  // (about 413 launches instead of 605 on the 16x100 grid); results are
  // the same bits at every batch size
  // (not in the one-pass layout other executors reuse: the uneven batch
  // runs every formula on one lane)
  if (Q == 1 && plan.precision != WMC_FP64 && !force_f64 && !plain && plan.max_rank <= 20) m = 1;
  st.m = m;
  const int32_t Qp = 1 << m;
  st.Qp = Qp;
  st.f64 = plan.precision == WMC_FP64 || force_f64;
  const size_t nt = plan.tensors.size();
  const int64_t root = plan.nodes.back().c;
  st.t_off.assign(nt, 0);
  st.t_meta.assign(nt, 0);
  st.t_qc.assign(nt, 1);
  st.t_dbl.assign(nt, st.f64 ? 1 : 0);
  st.t_dbl[(size_t)root] = 1;
  std::vector<int64_t> &bytes = st.t_bytes;
  bytes.assign(nt, 0);
  int64_t slots = 0;
  for (size_t i = 0; i < nt; ++i) {
    const TensorInfo &t = plan.tensors[i];
    int64_t r = (int64_t)t.labels.size() + (t.has_q ? m : 0);
    if (r > 31) {
      set_error("tensor %zu has %lld index bits (max 31)", i, (long long)r);
      return WMC_EPLAN_TOO_BIG;
    }
    bytes[i] = (int64_t(1) << r) * (st.t_dbl[i] ? 8 : 4);
    st.t_qc[i] = t.has_q ? Qp : 1;
    if (st.bfp_b >= 0) {
      // the mantissas, then one int32 exponent per (block, lane)
      const int32_t n = (int32_t)t.labels.size();
      const int32_t bb = t.kind == LEAF_WEIGHT ? 0 : std::min(st.bfp_b, n);
      if ((t.has_q ? m : 0) + bb > 11) {
        set_error("block floating point: blocks of 2^%d outputs with the query bits (max 2^11)",
                  (t.has_q ? m : 0) + bb);
        return WMC_EINVAL;
      }
      st.t_bb.push_back((int8_t)bb);
      bytes[i] = align_up(bytes[i]) + 4 * (int64_t)st.t_qc[i] * (int64_t(1) << (n - bb));
    }
    st.t_meta[i] = slots;
    slots += st.t_qc[i];
  }
  st.n_slots = slots;
  int64_t off = 0;
  st.off_io = off; off += align_up(sizeof(IoDesc));
  st.off_flags = off; off += align_up(4 * (int64_t)Qp);
  st.off_err = off; off += align_up(4);
  st.off_seqctr = off; off += align_up(8 * (int64_t)plan.nodes.size());  // at most one chain per node
  // small-node phase: which nodes run inside the persistent launch (every
  // node whose subtree is small: at most 2^16 outputs with the query bits,
  // at most 2^8 summed terms)
  std::vector<int32_t> sp_index(plan.nodes.size(), -1);
  std::vector<int64_t> sp_nodes;
  // one-block walk: every node small, the live tensors within shared memory
  bool cta = st.wo.cta_walk && !plain && st.bfp_b < 0 && Qp <= 4 && slots <= 1536 && !plan.nodes.empty() &&
             plan.slice_vars.empty();
  std::vector<int64_t> cta_off(cta ? nt : 0, -1);
  // shared memory: metadata, the node program, the leaf descriptors, the arena
  int64_t cta_meta = align_up(24 * slots) + align_up((int64_t)sizeof(wmc::dev::SNode) * (int64_t)plan.nodes.size()) +
                     align_up((int64_t)sizeof(wmc::dev::CtaLeaf) * plan.n_leaves);
  if (cta) {
    for (const Node &nd : plan.nodes) {
      const TensorInfo &C = plan.tensors[(size_t)nd.c];
      if ((int)C.labels.size() + (C.has_q ? m : 0) > 16 || nd.n_summed > 8) { cta = false; break; }
    }
  }
  std::vector<int64_t> cta_order;
  std::vector<int32_t> cta_level_end;
  int64_t cta_lut_words = 0;
  if (cta) {
    // levels, as late as possible: the root's is the tree's height, every
    // other node's one below its parent's, so a node runs just before its
    // parent and its output lives for one level (children always sit at
    // lower levels).  The block runs one level at a time, so outputs are
    // placed level by level and a level's children freed after it.
    std::vector<int32_t> depth(plan.nodes.size(), 0);
    int32_t top = 0;
    for (size_t r = plan.nodes.size(); r-- > 0;) {  // parents before children
      const Node &nd = plan.nodes[r];
      for (int64_t t : {nd.a, nd.b}) {
        const int64_t ch = plan.tensors[(size_t)t].node;
        if (ch >= 0) depth[(size_t)ch] = depth[r] + 1;
      }
      top = std::max(top, depth[r] + 1);
    }
    std::vector<int32_t> lev(plan.nodes.size(), 0);
    for (size_t ni = 0; ni < plan.nodes.size(); ++ni) lev[ni] = top - depth[ni];
    for (int32_t L = 1; L <= top; ++L)
      for (size_t ni = 0; ni < plan.nodes.size(); ++ni)
        if (lev[ni] == L) cta_order.push_back((int64_t)ni);
    if (plan.nodes[(size_t)cta_order.back()].c != root) cta = false;  // (the root is the one top node)
    FirstFit sf;
    for (int64_t i = 0; i < plan.n_leaves; ++i) cta_off[(size_t)i] = sf.alloc(bytes[(size_t)i]);
    for (size_t f0 = 0; cta && f0 < cta_order.size();) {
      size_t f1 = f0;
      int64_t words = 0;
      while (f1 < cta_order.size() && lev[(size_t)cta_order[f1]] == lev[(size_t)cta_order[f0]]) {
        const Node &nd = plan.nodes[(size_t)cta_order[f1]];
        const TensorInfo &C = plan.tensors[(size_t)nd.c];
        const int rC = (int)C.labels.size() + (C.has_q ? m : 0);
        words += 2 * ((1 << std::min(rC, 8)) + (1 << std::max(rC - 8, 0)) + (1 << nd.n_summed));
        if (nd.c != root) cta_off[(size_t)nd.c] = sf.alloc(bytes[(size_t)nd.c]);
        ++f1;
      }
      for (size_t f = f0; f < f1; ++f) {
        const Node &nd = plan.nodes[(size_t)cta_order[f]];
        sf.release(cta_off[(size_t)nd.a], bytes[(size_t)nd.a]);
        sf.release(cta_off[(size_t)nd.b], bytes[(size_t)nd.b]);
        cta_level_end.push_back((int32_t)f1);
      }
      cta_lut_words = std::max(cta_lut_words, words);
      f0 = f1;
    }
    const int64_t need = cta_meta + align_up(sf.top) + align_up(4 * cta_lut_words);
    if (need > 200 * 1024) cta = false;
    else {
      st.cta_smem = need;
      st.cta_lut_off = cta_meta + align_up(sf.top);
      st.cta_lut_words = cta_lut_words;
    }
  }
  if (cta) { st.wo.small_phase = 0; st.cta_off = cta_off; st.cta_meta = cta_meta; st.cta_order = cta_order;
    st.cta_level_end = cta_level_end; }
  if (st.wo.small_phase && !plain) {
    for (size_t ni = 0; ni < plan.nodes.size(); ++ni) {
      const Node &nd = plan.nodes[ni];
      const TensorInfo &C = plan.tensors[(size_t)nd.c];
      const int rc = (int)C.labels.size() + (C.has_q ? m : 0);
      if (rc > 16 || nd.n_summed > 8) continue;
      bool ok = true;
      for (int64_t ch : {nd.a, nd.b}) {
        if (ch < plan.n_leaves) continue;
        ok &= sp_index[(size_t)plan.tensors[(size_t)ch].node] >= 0;
      }
      if (!ok) continue;
      sp_index[ni] = (int32_t)sp_nodes.size();
      sp_nodes.push_back((int64_t)ni);
    }
  }
  st.off_sp = off; off += align_up(4 * (1 + (int64_t)sp_nodes.size()));
  st.off_exp = off; off += align_up(8 * slots);
  st.off_max = off; off += align_up(8 * slots);
  st.off_min = off; off += align_up(8 * slots);
  // leaves: resident for the whole walk
  for (int64_t i = 0; i < plan.n_leaves; ++i) { st.t_off[(size_t)i] = off; off += align_up(bytes[(size_t)i]); }
  const int64_t arena0 = off;
  st.max_roundings = plan.tensors[(size_t)root].roundings;
  st.n_slice_vars = (int32_t)plan.slice_vars.size();

  // ---- per-node kernel choice (offsets are filled in once laid out)
  std::vector<Launch> node_l(plan.nodes.size());
  for (size_t ni = 0; ni < plan.nodes.size(); ++ni) {
    const Node &nd = plan.nodes[ni];
    const TensorInfo &A = plan.tensors[(size_t)nd.a];
    const TensorInfo &B = plan.tensors[(size_t)nd.b];
    const TensorInfo &C = plan.tensors[(size_t)nd.c];
    std::vector<int32_t> LA = full_labels(A, m), LB = full_labels(B, m), LC = full_labels(C, m);
    Launch &l = node_l[ni];
    const bool is_root = nd.c == root;
    bool used_k2 = false;
    if (st.bfp_b >= 0) {  // block floating point: one kernel for every node
      l.kind = L_BFP;
      fill_k1(LA, LB, LC, l.k1);
      if (l.k1.k > 24) { set_error("node sums %d indices (max 24)", l.k1.k); return WMC_EPLAN_TOO_BIG; }
      l.ti = TF;
      l.to = st.t_dbl[(size_t)nd.c] ? TD : TF;
      l.id_a = nd.a;
      l.id_b = nd.b;
      const int64_t nb = int64_t(1) << ((int64_t)C.labels.size() - st.t_bb[(size_t)nd.c]);
      l.blocks = std::min<int64_t>(nb, 148 * 8);
      used_k2 = true;  // (no other kernel)
    }
    if (!is_root && !used_k2) {
      const bool a_first = LA.size() >= LB.size();
      int vmax = 1, kmax = 1, fmax = 1;
      K2Params p2;
      for (int attempt = 0; attempt < 2 && !used_k2; ++attempt) {
        bool use_a = (attempt == 0) == a_first;
        const std::vector<int32_t> &LP = use_a ? LA : LB;
        const std::vector<int32_t> &LS = use_a ? LB : LA;
        if (try_k2(LP, LS, LC, st.f64, p2, vmax, kmax, fmax)) {
          used_k2 = true;
          l.kind = L_K2;
          l.ti = st.f64 ? TD : TF;
          l.v = vmax; l.kmax = kmax; l.fmax = fmax;
          l.k2 = p2;
          l.id_a = use_a ? nd.a : nd.b;
          l.id_b = use_a ? nd.b : nd.a;
          l.k2.ma.qmask = (use_a ? A : B).has_q ? Qp - 1 : 0;
          l.k2.mb.qmask = (use_a ? B : A).has_q ? Qp - 1 : 0;
          l.blocks = grid_for(1ull << p2.log2_nu);
          if (try_k2_tma(l.k2, use_a ? LA : LB, use_a ? LB : LA, st.f64, (use_a ? A : B).has_q,
                         (use_a ? B : A).has_q, Qp, l.k2t, l.smem)) {
            l.kind = L_K2T;
            const uint64_t n_tiles = 1ull << (p2.log2_nu + p2.vbits - l.k2t.tb);
            const int kf = l.k2.k + l.k2.f;  // register-limited CTAs per SM (launch bounds)
            const int per_sm_regs = kf <= 2 ? 3 : (kf <= 4 ? 2 : 1);
            const int per_sm = std::min(per_sm_regs, l.smem <= 72 * 1024 ? 3 : (l.smem <= 108 * 1024 ? 2 : 1));
            l.blocks = (int64_t)std::min<uint64_t>(n_tiles, (uint64_t)(148 * per_sm));
          }
        }
      }
    }
    wmc::dev::K4Params p4;
    if (!used_k2 && !is_root && try_k4(LA, LB, LC, st.f64, p4)) {
      // dense batched product; unsplit, so its summation order is k1's
      used_k2 = true;
      l.kind = L_K4;
      l.k4 = p4;
      l.ti = st.f64 ? TD : TF;
      l.id_a = nd.a;
      l.id_b = nd.b;
      l.k4.ma.qmask = A.has_q ? Qp - 1 : 0;
      l.k4.mb.qmask = B.has_q ? Qp - 1 : 0;
      l.blocks = (int64_t)1 << (p4.ni - 6 + p4.nj - 6 + p4.nb);
    }
    // batched small contraction: both operands large, few free and summed
    // indices; the query lanes (if any) batch indices of all three
    // (either operand as A: A takes up to 4 free bits, B up to 3)
    bool k2b_swap = false;
    if (!used_k2 && !is_root && g_batched.load() &&
        (try_k2b(LA, LB, LC, l.k2b, bytes[(size_t)nd.a], bytes[(size_t)nd.b]) ||
                                 (k2b_swap = try_k2b(LB, LA, LC, l.k2b, bytes[(size_t)nd.b], bytes[(size_t)nd.a])))) {
      used_k2 = true;
      l.kind = L_K2B;
      l.ti = st.f64 ? TD : TF;
      l.id_a = k2b_swap ? nd.b : nd.a;
      l.id_b = k2b_swap ? nd.a : nd.b;
      l.k2b.ma.qmask = A.has_q ? Qp - 1 : 0;
      l.k2b.mb.qmask = B.has_q ? Qp - 1 : 0;
      // (grid-stride: the stride must be a multiple of the lane count)
      const uint64_t units = 1ull << l.k2b.log2_nu;
      const int64_t g = (C.has_q && Qp > 256) ? Qp / 256 : 1;
      const bool ct = l.k2b.k == 1 && l.k2b.fA <= 3 && l.k2b.fB <= 2;  // (compile-time shape: 3 blocks per SM)
      l.blocks = (int64_t)std::min<uint64_t>((units + 255) / 256, 148ull * (ct ? 3 : 2));
      l.blocks = std::max<int64_t>(g, l.blocks / g * g);
    }
    if (!used_k2) {
      l.kind = L_K1;
      fill_k1(LA, LB, LC, l.k1);
      if (l.k1.k > 24) { set_error("node sums %d indices (max 24)", l.k1.k); return WMC_EPLAN_TOO_BIG; }
      l.ti = st.f64 ? TD : TF;
      l.ta = (st.f64 || is_root || l.k1.k > 16) ? TD : TF;
      l.to = st.t_dbl[(size_t)nd.c] ? TD : TF;
      l.id_a = nd.a;
      l.id_b = nd.b;
      l.k1.ma.qmask = A.has_q ? Qp - 1 : 0;
      l.k1.mb.qmask = B.has_q ? Qp - 1 : 0;
      l.blocks = grid_for(1ull << l.k1.rC);
    }
    l.id_c = nd.c;
    l.alg_bytes = (double)bytes[(size_t)nd.a] + (double)bytes[(size_t)nd.b] + (double)bytes[(size_t)nd.c];
    dev::OutMeta &mc = l.kind == L_K1 ? l.k1.mc : (l.kind == L_K4 ? l.k4.mc : (l.kind == L_K2B ? l.k2b.mc : l.k2.mc));
    mc.Qc = C.has_q ? Qp : 1;
    mc.Q = Qp;
    mc.scale_inputs = 1;
  }

  // ---- fuse consecutive frontier eliminations (i, j): node j's large
  // operand is node i's output; the nodes between them (j's small subtree)
  // move in front of i.  Steps are listed in execution order.
  struct Step { int64_t node; int64_t fused_with; };  // fused_with = j or -1
  std::vector<Step> steps;
  {
    std::vector<int64_t> consumer(plan.tensors.size(), -1);
    for (size_t ni = 0; ni < plan.nodes.size(); ++ni) {
      consumer[(size_t)plan.nodes[ni].a] = (int64_t)ni;
      consumer[(size_t)plan.nodes[ni].b] = (int64_t)ni;
    }
    std::vector<int64_t> fuse_next(plan.nodes.size(), -1);
    std::vector<uint8_t> absorbed(plan.nodes.size(), 0);
    // by default, runs of up to six on walks of at most 16 lanes (launch
    // bound: fewer, longer passes win), up to four on wider ones (bound by
    // HBM, where the staged four-step kernel moves the bytes faster)
    const int fuse_level = plain ? 0 : (st.wo.fuse < 0 ? (Qp <= 16 ? 6 : 4) : st.wo.fuse);
    // frontier steps: one summed index; f added ones (1 in place, 2 growth,
    // 0 shrink); a chain starts with f >= 1 and ends at its first f = 0
    auto frontier_f = [&](const Launch &l) { return (l.kind == L_K2T && l.k2.k == 1) ? l.k2.f : -1; };
    for (size_t ni = 0; ni < plan.nodes.size() && fuse_level >= 2; ++ni) {
      if (absorbed[ni] || frontier_f(node_l[ni]) < 1) continue;
      // the longest run of frontier steps, each consuming the previous output
      std::vector<int64_t> chain{(int64_t)ni};
      while ((int)chain.size() < std::min(fuse_level, wmc::dev::kMaxChain)) {
        const int64_t last = chain.back();
        const int64_t nj = consumer[(size_t)plan.nodes[(size_t)last].c];
        if (nj < 0 || absorbed[(size_t)nj]) break;
        const int fj = frontier_f(node_l[(size_t)nj]);
        if (fj != 0 && fj != 1) break;
        if (node_l[(size_t)nj].id_a != plan.nodes[(size_t)last].c) break;
        bool clean = true;  // nodes between must not be fused already
        for (int64_t q = last + 1; q < nj; ++q) clean &= !absorbed[(size_t)q] && fuse_next[(size_t)q] < 0;
        if (!clean) break;
        chain.push_back(nj);
        if (fj == 0) break;
      }
      const TensorInfo &P = plan.tensors[(size_t)node_l[ni].id_a];
      Launch f;
      int d_ok = 0;
      for (int D = (int)chain.size(); D >= 2 && !d_ok; --D) {
        std::vector<std::vector<int32_t>> LS, LC;
        for (int i = 0; i < D; ++i) {
          const Launch &l = node_l[(size_t)chain[(size_t)i]];
          LS.push_back(full_labels(plan.tensors[(size_t)l.id_b], m));
          LC.push_back(full_labels(plan.tensors[(size_t)plan.nodes[(size_t)chain[(size_t)i]].c], m));
        }
        const bool s1q = plan.tensors[(size_t)node_l[ni].id_b].has_q;
        bool fast = false;
        int grow = 0, shrink = 0;
        // (five or six steps on one lane: two lanes of 64 states each were
        // slower, 254 registers and one block per SM)
        if (try_chain(full_labels(P, m), LS, LC, st.f64, P.has_q, s1q, Qp, true, f.k2c, f.v, fast, grow, shrink,
                      f.smem, D > 4)) {
          d_ok = D;
          f.chain_fast = fast ? 1 : 0;
          f.chain_grow = grow;
          f.chain_shrink = shrink;
        }
      }
      if (!d_ok) continue;
      const int64_t nlast = chain[(size_t)d_ok - 1];
      const TensorInfo &CD = plan.tensors[(size_t)plan.nodes[(size_t)nlast].c];
      f.kind = L_K2C;
      f.ti = st.f64 ? TD : TF;
      f.chain_d = d_ok;
      f.id_a = node_l[ni].id_a;
      f.id_b = node_l[ni].id_b;
      f.id_c = plan.nodes[(size_t)nlast].c;
      f.k2c.mp.qmask = P.has_q ? Qp - 1 : 0;
      f.alg_bytes = (double)bytes[(size_t)f.id_a] + (double)bytes[(size_t)f.id_c];
      for (int i = 0; i < d_ok; ++i) {
        const Launch &l = node_l[(size_t)chain[(size_t)i]];
        f.id_sc[i] = l.id_b;
        f.k2c.ms[i].qmask = plan.tensors[(size_t)l.id_b].has_q ? Qp - 1 : 0;
        f.alg_bytes += (double)bytes[(size_t)l.id_b];
      }
      f.k2c.mc.Qc = CD.has_q ? Qp : 1;
      f.k2c.mc.Q = Qp;
      f.k2c.mc.scale_inputs = 1;
      const int per_sm = std::max<int>(1, std::min<int>(2, (int)((227u * 1024u) / (f.smem + 2048))));
      if (d_ok > 4) {  // direct loads: one unit per thread at a time, grid-stride
        const uint64_t units = 1ull << f.k2c.log2_nu;
        // fewer units than one full block per SM (small walks, launch
        // bound): smaller blocks spread them over more SMs, so that each
        // warp has a scheduler to itself (at least 32 lanes per block, a
        // multiple of the lane count), while every block's copy of the
        // staged S_i stays at most 8 entries per thread
        int threads = wmc::dev::kDirectThreads;
        const uint64_t s_words = f.k2c.s_copy_bytes / 4;
        while (threads > 32 && (uint64_t)threads * 148ull > units && s_words <= (uint64_t)(threads / 2) * 8 &&
               ((threads / 2) * f.v) % std::max<int>(1, f.k2c.mc.Qc) == 0)
          threads /= 2;
        f.threads = threads;
        const uint64_t need = (units + (uint64_t)threads - 1) / (uint64_t)threads;
        const uint64_t resident = 148ull * (uint64_t)(f.v == 1 ? per_sm : 1) * (uint64_t)(wmc::dev::kDirectThreads / threads);
        f.blocks = (int64_t)std::max<uint64_t>(1, std::min<uint64_t>(need, resident));
      } else {
        const uint64_t n_tiles = 1ull << (f.k2c.log2_nu + f.k2c.vbits - f.k2c.tb);
        // (registers: NW*32+32 threads of at most 96 registers leave room for two blocks)
        f.blocks = (int64_t)std::min<uint64_t>(n_tiles, 148ull * (uint64_t)per_sm);
      }
      fuse_next[ni] = nlast;
      for (int i = 1; i < d_ok; ++i) absorbed[(size_t)chain[(size_t)i]] = 1;
      for (int64_t q = (int64_t)ni + 1; q < nlast; ++q)
        if (!absorbed[(size_t)q]) absorbed[(size_t)q] = 2;  // moved before the chain
      node_l[ni] = f;
    }
    for (size_t ni = 0; ni < plan.nodes.size(); ++ni) {
      if (absorbed[ni]) continue;
      if (fuse_next[ni] >= 0)
        for (int64_t q = (int64_t)ni + 1; q < fuse_next[ni]; ++q)
          if (absorbed[(size_t)q] == 2 && sp_index[(size_t)q] < 0) steps.push_back({q, -1});
      if (sp_index[ni] >= 0) continue;  // runs in the small-node phase
      steps.push_back({(int64_t)ni, fuse_next[ni]});
    }
  }

  // ---- arena: first fit in execution order; children freed after use
  FirstFit ff;
  st.alg_bytes = 0;
  st.flops = 0;
  auto release = [&](int64_t t) {
    if (t < plan.n_leaves) return;
    if (sp_index[(size_t)plan.tensors[(size_t)t].node] >= 0) return;  // small-phase output: kept
    ff.release(st.t_off[(size_t)t] - arena0, bytes[(size_t)t]);
  };
  for (int64_t ni : sp_nodes) {
    const Node &nd = plan.nodes[(size_t)ni];
    st.t_off[(size_t)nd.c] = arena0 + ff.alloc(bytes[(size_t)nd.c]);
    st.alg_bytes += node_l[(size_t)ni].alg_bytes;
  }
  for (const Step &stp : steps) {
    const Launch &l = node_l[(size_t)stp.node];
    st.t_off[(size_t)l.id_c] = arena0 + ff.alloc(bytes[(size_t)l.id_c]);
    release(l.id_a);
    release(l.id_b);
    if (l.kind == L_K2C)
      for (int i = 1; i < l.chain_d; ++i) release(l.id_sc[i]);
    st.alg_bytes += l.alg_bytes;
  }
  for (const Node &nd : plan.nodes) {
    const TensorInfo &C = plan.tensors[(size_t)nd.c];
    st.flops += 2.0 * std::ldexp(1.0, nd.iter_rank + (C.has_q ? m : 0));
  }
  st.arena_bytes = ff.top;
  st.ws_bytes = arena0 + align_up(ff.top);
  if (st.bfp_b >= 0) {
    st.t_eoff.assign(nt, 0);
    for (size_t i = 0; i < nt; ++i) {
      const TensorInfo &t = plan.tensors[i];
      const int64_t r = (int64_t)t.labels.size() + (t.has_q ? m : 0);
      st.t_eoff[i] = st.t_off[i] + align_up((int64_t(1) << r) * (st.t_dbl[i] ? 8 : 4));
    }
  }

  // ---- launches
  st.launches.clear();
  Launch ms;
  ms.kind = L_MEMSET;
  ms.memset_off = st.off_flags;
  ms.memset_bytes = st.off_max + align_up(8 * slots) - st.off_flags;  // flags, exps, maxima
  ms.memset_value = 0;
  st.launches.push_back(ms);
  Launch ms1 = ms;
  ms1.memset_off = st.off_min;  // minima start at "none" (all ones)
  ms1.memset_bytes = align_up(8 * slots);
  ms1.memset_value = 0xff;
  st.launches.push_back(ms1);
  if (st.bfp_b >= 0 && plan.n_leaves > 0) {
    // block floating point: the leaves' exponents start at 0 (clause
    // tensors and the scalar 1 keep them; weight vectors write their own)
    Launch z = ms;
    z.memset_off = st.t_off[0];
    z.memset_bytes = arena0 - st.t_off[0];
    st.launches.push_back(z);
  }
  // clause leaves
  st.h_clause.clear(); st.h_first.clear();
  int64_t entries = 0;
  for (int64_t i = 0; i < plan.n_leaves; ++i) {
    const TensorInfo &t = plan.tensors[(size_t)i];
    if (t.kind != LEAF_CLAUSE) continue;
    ClauseLeaf L;
    L.off = st.t_off[(size_t)i] / (st.f64 ? 8 : 4);
    L.meta = st.t_meta[(size_t)i];
    L.fals = t.fals;
    L.rank = (int32_t)t.labels.size();
    L.smask = t.clause >= 0 ? plan.clauses[(size_t)t.clause].smask : 0u;
    L.sfals = t.clause >= 0 ? plan.clauses[(size_t)t.clause].sfals : 0u;
    L.lbits = t.has_q ? m : 0;  // (a clause with a sliced literal carries the lanes)
    st.h_clause.push_back(L);
    st.h_first.push_back(entries);
    entries += int64_t(1) << (L.rank + L.lbits);
  }
  st.n_clause_entries = entries;
  if (!st.h_clause.empty()) {
    Launch l; l.kind = L_CLAUSES; l.blocks = grid_for((uint64_t)entries);
    st.launches.push_back(l);
  }
  // -1: a variable without a weight leaf (a sliced one), skipped by the kernel
  st.h_woff.assign((size_t)plan.n_vars, -1);
  st.h_wmeta.assign((size_t)plan.n_vars, -1);
  bool have_w = false;
  for (int64_t i = 0; i < plan.n_leaves; ++i) {
    const TensorInfo &t = plan.tensors[(size_t)i];
    if (t.kind == LEAF_WEIGHT) {
      st.h_woff[(size_t)t.labels[0]] = st.t_off[(size_t)i] / (st.f64 ? 8 : 4);
      st.h_wmeta[(size_t)t.labels[0]] = st.t_meta[(size_t)i];
      have_w = true;
    } else if (t.kind == LEAF_ONE) {
      Launch l; l.kind = L_ONE; l.one_off = st.t_off[(size_t)i]; l.one_meta = st.t_meta[(size_t)i];
      st.launches.push_back(l);
    }
  }
  if (have_w) {
    Launch l; l.kind = st.bfp_b >= 0 ? L_BFPW : L_WEIGHTS;
    l.blocks = grid_for((uint64_t)plan.n_vars * (uint64_t)Qp);
    st.launches.push_back(l);
  }
  st.h_snodes.clear();
  st.h_stasks.clear();
  if (!sp_nodes.empty()) {
    double sp_bytes = 0;
    for (int64_t ni : sp_nodes) {
      const Node &nd = plan.nodes[(size_t)ni];
      const TensorInfo &A = plan.tensors[(size_t)nd.a], &B = plan.tensors[(size_t)nd.b];
      const TensorInfo &C = plan.tensors[(size_t)nd.c];
      wmc::dev::SNode sn;
      std::memset(&sn, 0, sizeof(sn));
      sn.a = st.t_off[(size_t)nd.a]; sn.b = st.t_off[(size_t)nd.b]; sn.c = st.t_off[(size_t)nd.c];
      sn.ma = st.t_meta[(size_t)nd.a]; sn.mb = st.t_meta[(size_t)nd.b]; sn.mc = st.t_meta[(size_t)nd.c];
      sn.qmask_a = A.has_q ? Qp - 1 : 0;
      sn.qmask_b = B.has_q ? Qp - 1 : 0;
      sn.Qc = C.has_q ? Qp : 1;
      sn.dep_a = nd.a < plan.n_leaves ? -1 : sp_index[(size_t)A.node];
      sn.dep_b = nd.b < plan.n_leaves ? -1 : sp_index[(size_t)B.node];
      int8_t pa[32], pb[32], spa[24], spb[24];
      k1_bitmaps(full_labels(A, m), full_labels(B, m), full_labels(C, m), &sn.rC, &sn.k, pa, pb, spa, spb);
      std::memcpy(sn.posA, pa, 16); std::memcpy(sn.posB, pb, 16);
      std::memcpy(sn.sposA, spa, 8); std::memcpy(sn.sposB, spb, 8);
      // up to 16 chunks of at least 256 outputs (one per thread): a node on
      // the tree's critical path spreads over blocks instead of one block
      // walking its outputs one L2 round trip after another
      sn.chunk_log2 = std::min<int32_t>(sn.rC, std::max<int32_t>(8, std::min<int32_t>(12, sn.rC - 4)));
      sn.n_chunks = 1 << (sn.rC - sn.chunk_log2);
      sn.ti = st.f64 ? 1 : 0;
      sn.to = st.t_dbl[(size_t)nd.c];
      sn.ta = (st.f64 || sn.to) ? 1 : 0;
      const int32_t idx = (int32_t)st.h_snodes.size();
      st.h_snodes.push_back(sn);
      for (int32_t c = 0; c < sn.n_chunks; ++c) st.h_stasks.push_back({idx, c});
      sp_bytes += node_l[(size_t)ni].alg_bytes;
    }
    Launch l;
    l.kind = L_SMALL;
    l.blocks = (int64_t)std::min<size_t>(st.h_stasks.size(), 148 * 4);
    l.alg_bytes = sp_bytes;
    st.launches.push_back(l);
  }
  for (const Step &stp : steps) {
    Launch l = node_l[(size_t)stp.node];
    l.off_a = st.t_off[(size_t)l.id_a];
    l.off_b = st.t_off[(size_t)l.id_b];
    l.off_c = st.t_off[(size_t)l.id_c];
    l.meta_a = st.t_meta[(size_t)l.id_a];
    l.meta_b = st.t_meta[(size_t)l.id_b];
    l.meta_c = st.t_meta[(size_t)l.id_c];
    if (l.kind == L_K2C)
      for (int i = 0; i < l.chain_d; ++i) {
        l.off_sc[i] = st.t_off[(size_t)l.id_sc[i]];
        l.meta_sc[i] = st.t_meta[(size_t)l.id_sc[i]];
      }
    st.launches.push_back(l);
  }
  // runs of consecutive chains with small tile counts: one k2_chain_seq
  // launch each (float32, four eliminations, contiguous lanes)
  if (st.wo.chain_runs > 0 && !st.f64) {
    auto eligible = [&](const Launch &l) {
      if (l.kind != L_K2C || l.ti != TF || l.chain_d != 4 || !l.chain_fast || (l.v != 1 && l.v != 2)) return false;
      for (int i = 0; i < l.chain_d; ++i)
        if (l.v > 1 && l.k2c.b_vec[i] != 1) return false;
      // (the run kernel keeps two chains' parameters in static shared memory)
      if (l.smem > kSeqDynSmem) return false;
      const int64_t tiles = int64_t(1) << (l.k2c.log2_nu + l.k2c.vbits - l.k2c.tb);
      return tiles <= (int64_t)st.wo.chain_runs;
    };
    std::vector<Launch> out;
    int64_t n_seq_chains = 0;
    for (size_t i = 0; i < st.launches.size();) {
      size_t j = i;
      while (j < st.launches.size() && eligible(st.launches[j]) && st.launches[j].v == st.launches[i].v) ++j;
      if (j - i < 2) {
        out.push_back(st.launches[i]);
        ++i;
        continue;
      }
      Launch r;
      r.kind = L_K2CSEQ;
      r.ti = TF;
      r.v = st.launches[i].v;
      r.chain_d = 4;
      r.chain_fast = 1;
      r.seq_first = (int64_t)st.h_seq.size();
      r.seq_ctr_off = st.off_seqctr + 8 * n_seq_chains;
      for (size_t k = i; k < j; ++k) {
        const Launch &l = st.launches[k];
        wmc::dev::K2CParams cp = l.k2c;
        // pointers as workspace offsets (the kernel adds the workspace base)
        auto at = [](int64_t off) { return reinterpret_cast<void *>((uintptr_t)off); };
        auto meta = [&](int64_t base, int64_t slot) { return at(base + 8 * slot); };
        cp.P = at(l.off_a);
        cp.C = at(l.off_c);
        cp.mp.exp = (const int64_t *)meta(st.off_exp, l.meta_a);
        cp.mp.maxb = (const unsigned long long *)meta(st.off_max, l.meta_a);
        cp.mp.minb = (const unsigned long long *)meta(st.off_min, l.meta_a);
        for (int d = 0; d < l.chain_d; ++d) {
          cp.S[d] = at(l.off_sc[d]);
          cp.ms[d].exp = (const int64_t *)meta(st.off_exp, l.meta_sc[d]);
          cp.ms[d].maxb = (const unsigned long long *)meta(st.off_max, l.meta_sc[d]);
          cp.ms[d].minb = (const unsigned long long *)meta(st.off_min, l.meta_sc[d]);
        }
        cp.mc.exp = (int64_t *)meta(st.off_exp, l.meta_c);
        cp.mc.maxb = (unsigned long long *)meta(st.off_max, l.meta_c);
        cp.mc.minb = (unsigned long long *)meta(st.off_min, l.meta_c);
        cp.mc.flags = (uint32_t *)at(st.off_flags);
        cp.err = (uint32_t *)at(st.off_err);
        cp.debug_stall = 0;
        cp.variant = l.chain_grow ? 1 : (l.chain_shrink ? 2 : 0);
        st.h_seq.push_back(cp);
        r.smem = std::max(r.smem, l.smem);
        r.blocks = std::max(r.blocks, l.blocks);
        r.alg_bytes += l.alg_bytes;
        r.chains.push_back(l);
      }
      n_seq_chains += (int64_t)(j - i);
      r.blocks = std::min<int64_t>(r.blocks, 148);
      out.push_back(std::move(r));
      i = j;
    }
    st.launches.swap(out);
  }
  Launch fin;
  fin.kind = L_FINAL;
  fin.off_c = st.t_off[(size_t)root];
  fin.meta_c = st.t_meta[(size_t)root];
  fin.blocks = grid_for((uint64_t)Q);
  // A chain copies its S_i before it waits for the launch in front of it
  // (programmatic dependent launch): that is safe when the launch in front
  // is another chain (it writes only its C, this chain's P, read after the
  // wait) or a single node whose output is no S_i; otherwise the chain
  // starts in plain stream order.
  for (size_t i = 0; i < st.launches.size(); ++i) {
    Launch &l = st.launches[i];
    if (l.kind != L_K2C) continue;
    bool safe = false;
    if (i > 0) {
      const Launch &pv = st.launches[i - 1];
      if (pv.kind == L_K2C) {
        safe = true;
      } else if (pv.kind == L_K1 || pv.kind == L_K2 || pv.kind == L_K2T || pv.kind == L_K4 || pv.kind == L_K2B) {
        safe = true;
        for (int j = 0; j < l.chain_d; ++j) safe &= pv.id_c != l.id_sc[j];
      }
    }
    l.no_pdl = safe ? 0 : 1;
  }
  st.launches.push_back(fin);
  if (cta) {
    // the whole walk in one block: the metadata clears, the walk, the root
    st.h_snodes.clear();
    st.h_stasks.clear();
    st.h_cta.clear();
    for (int64_t i = 0; i < plan.n_leaves; ++i) {
      const TensorInfo &t = plan.tensors[(size_t)i];
      wmc::dev::CtaLeaf L;
      std::memset(&L, 0, sizeof(L));
      L.off = (uint32_t)cta_off[(size_t)i];
      L.slot = (int32_t)st.t_meta[(size_t)i];
      L.kind = t.kind;
      L.rank = (int32_t)t.labels.size();
      if (t.kind == LEAF_CLAUSE) {
        L.fals = t.fals;
        L.smask = t.clause >= 0 ? plan.clauses[(size_t)t.clause].smask : 0u;
        L.sfals = t.clause >= 0 ? plan.clauses[(size_t)t.clause].sfals : 0u;
      } else if (t.kind == LEAF_WEIGHT) {
        L.var = t.labels[0];
      }
      st.h_cta.push_back(L);
    }
    int32_t lut_base = 0, out_base = 0;
    for (size_t oi = 0; oi < st.cta_order.size(); ++oi) {
      const int64_t ni = st.cta_order[oi];
      const Node &nd = plan.nodes[(size_t)ni];
      const TensorInfo &A = plan.tensors[(size_t)nd.a], &B = plan.tensors[(size_t)nd.b];
      const TensorInfo &C = plan.tensors[(size_t)nd.c];
      const bool is_root = nd.c == root;
      wmc::dev::SNode sn;
      std::memset(&sn, 0, sizeof(sn));
      sn.a = cta_off[(size_t)nd.a];
      sn.b = cta_off[(size_t)nd.b];
      sn.c = is_root ? st.t_off[(size_t)nd.c] : cta_off[(size_t)nd.c];
      sn.ma = st.t_meta[(size_t)nd.a]; sn.mb = st.t_meta[(size_t)nd.b]; sn.mc = st.t_meta[(size_t)nd.c];
      sn.qmask_a = A.has_q ? Qp - 1 : 0;
      sn.qmask_b = B.has_q ? Qp - 1 : 0;
      sn.Qc = C.has_q ? Qp : 1;
      sn.dep_a = sn.dep_b = -1;
      int8_t pa[32], pb[32], spa[24], spb[24];
      k1_bitmaps(full_labels(A, m), full_labels(B, m), full_labels(C, m), &sn.rC, &sn.k, pa, pb, spa, spb);
      std::memcpy(sn.posA, pa, 16); std::memcpy(sn.posB, pb, 16);
      std::memcpy(sn.sposA, spa, 8); std::memcpy(sn.sposB, spb, 8);
      sn.n_chunks = 1;
      sn.chunk_log2 = sn.rC;
      sn.ti = st.f64 ? 1 : 0;
      sn.to = st.t_dbl[(size_t)nd.c];
      sn.ta = (st.f64 || is_root) ? 1 : 0;
      // (the order lists the levels one after another)
      if (oi == 0 || st.cta_level_end[oi - 1] == (int32_t)oi) { lut_base = 0; out_base = 0; }
      sn.level_end = st.cta_level_end[oi];
      sn.lut_base = lut_base;
      sn.out_base = out_base;
      lut_base += 2 * ((1 << std::min<int32_t>(sn.rC, 8)) + (1 << std::max<int32_t>(sn.rC - 8, 0)) + (1 << sn.k));
      out_base += 1 << sn.rC;
      st.h_snodes.push_back(sn);
    }
    std::vector<Launch> keep;
    for (const Launch &l : st.launches)
      if (l.kind == L_MEMSET && (l.memset_off == st.off_flags || l.memset_off == st.off_min)) keep.push_back(l);
    Launch w;
    w.kind = L_CTA;
    w.blocks = 1;
    w.smem = (size_t)st.cta_smem;
    double alg = 0;
    for (const Launch &l : st.launches) alg += l.alg_bytes;
    w.alg_bytes = alg;
    keep.push_back(w);
    keep.push_back(fin);
    st.launches.swap(keep);
  }
  st.kernels_per_run = 0;
  for (auto &l : st.launches) st.kernels_per_run += (l.kind != L_MEMSET);
  return WMC_OK;
}

// ------------------------------------------------------------ launching

template <typename T, int V, int K>
static void launch_k2_t(const K2Params &p, int64_t blocks, cudaStream_t s) {
  if constexpr (K == 4 && V == 1) {
    if (p.s_staged) {  // S staged in shared memory (at most 32 KB)
      // grid-stride over the units: one wave of three (float64: two) blocks per SM
      const size_t smem = sizeof(T) << p.s_log2;
      const unsigned b4 = (unsigned)std::min<int64_t>(blocks, 148 * (sizeof(T) == 4 ? 3 : 2));
      if (p.s_contig) dev::k2_stream_s16<T, true><<<b4, dev::kThreads, smem, s>>>(p);
      else dev::k2_stream_s16<T, false><<<b4, dev::kThreads, smem, s>>>(p);
      return;
    }
  }
  dev::k2_stream<T, V, K, K><<<(unsigned)blocks, dev::kThreads, 0, s>>>(p);
}

template <typename T, int V>
static void launch_k2_v(const K2Params &p, int kmax, int64_t blocks, cudaStream_t s) {
  if (kmax <= 1) launch_k2_t<T, V, 1>(p, blocks, s);
  else if (kmax == 2) launch_k2_t<T, V, 2>(p, blocks, s);
  else if (kmax == 3) launch_k2_t<T, V, 3>(p, blocks, s);
  else if constexpr (V == 1) launch_k2_t<T, 1, 4>(p, blocks, s);  // try_k2 gives V = 1 here
}

static void launch_k2(const Launch &l, const K2Params &p, cudaStream_t s) {
  if (l.ti == TF) {
    if (l.v == 4) launch_k2_v<float, 4>(p, l.kmax, l.blocks, s);
    else launch_k2_v<float, 1>(p, l.kmax, l.blocks, s);
  } else {
    if (l.v == 2) launch_k2_v<double, 2>(p, l.kmax, l.blocks, s);
    else launch_k2_v<double, 1>(p, l.kmax, l.blocks, s);
  }
}

template <typename T, int V, int K, int F, bool EXACT>
static void launch_k2t_t(const wmc::dev::K2TParams &p, int64_t blocks, size_t smem, cudaStream_t s) {
  static bool attr_set = false;  // opt in to large dynamic shared memory once
  if (!attr_set) {
    cudaFuncSetAttribute(dev::k2_tma<T, V, K, F, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         160 * 1024);
    attr_set = true;
  }
  dev::k2_tma<T, V, K, F, EXACT><<<(unsigned)blocks, dev::kThreads + 32, smem, s>>>(p);
}

// Exact specialisations for the common (summed, S-free) splits, a bounded
// generic one for the rest.
template <typename T, int V>
static void launch_k2t_v(const wmc::dev::K2TParams &p, int64_t blocks, size_t smem, cudaStream_t s) {
  const int k = p.k.k, f = p.k.f;
  if (k == 1 && f == 1) launch_k2t_t<T, V, 1, 1, true>(p, blocks, smem, s);
  else if (k == 1 && f == 0) launch_k2t_t<T, V, 1, 0, true>(p, blocks, smem, s);
  else if (k == 0 && f == 1) launch_k2t_t<T, V, 0, 1, true>(p, blocks, smem, s);
  else if (k == 1 && f == 2) launch_k2t_t<T, V, 1, 2, true>(p, blocks, smem, s);
  else if (k == 2 && f == 1) launch_k2t_t<T, V, 2, 1, true>(p, blocks, smem, s);
  else if (k == 2 && f == 2) launch_k2t_t<T, V, 2, 2, true>(p, blocks, smem, s);
  else if (k <= 1 && f <= 1) launch_k2t_t<T, V, 1, 1, false>(p, blocks, smem, s);
  else launch_k2t_t<T, V, 3, 3, false>(p, blocks, smem, s);
}

static void launch_k2t(const Launch &l, const wmc::dev::K2TParams &p, cudaStream_t s) {
  if (l.ti == TF) {
    if (l.v == 4) launch_k2t_v<float, 4>(p, l.blocks, l.smem, s);
    else launch_k2t_v<float, 1>(p, l.blocks, l.smem, s);
  } else {
    if (l.v == 2) launch_k2t_v<double, 2>(p, l.blocks, l.smem, s);
    else launch_k2t_v<double, 1>(p, l.blocks, l.smem, s);
  }
}

// batched small contractions: one summed index with up to 3 free bits of A
// and 2 of B at compile time, the other shapes at run time
template <typename T>
static void launch_k2b_t(const Launch &l, const wmc::dev::K2BParams &p, cudaStream_t s) {
  const unsigned g = (unsigned)l.blocks, b = dev::kThreads;
  const int code = p.k == 1 && p.fA <= 3 && p.fB <= 2 ? p.fA * 3 + p.fB : -1;
  switch (code) {
    case 0: dev::k2_batched<T, 1, 0, 0><<<g, b, 0, s>>>(p); break;
    case 1: dev::k2_batched<T, 1, 0, 1><<<g, b, 0, s>>>(p); break;
    case 2: dev::k2_batched<T, 1, 0, 2><<<g, b, 0, s>>>(p); break;
    case 3: dev::k2_batched<T, 1, 1, 0><<<g, b, 0, s>>>(p); break;
    case 4: dev::k2_batched<T, 1, 1, 1><<<g, b, 0, s>>>(p); break;
    case 5: dev::k2_batched<T, 1, 1, 2><<<g, b, 0, s>>>(p); break;
    case 6: dev::k2_batched<T, 1, 2, 0><<<g, b, 0, s>>>(p); break;
    case 7: dev::k2_batched<T, 1, 2, 1><<<g, b, 0, s>>>(p); break;
    case 8: dev::k2_batched<T, 1, 2, 2><<<g, b, 0, s>>>(p); break;
    case 9: dev::k2_batched<T, 1, 3, 0><<<g, b, 0, s>>>(p); break;
    case 10: dev::k2_batched<T, 1, 3, 1><<<g, b, 0, s>>>(p); break;
    case 11: dev::k2_batched<T, 1, 3, 2><<<g, b, 0, s>>>(p); break;
    default: dev::k2_batched<T, -1, 0, 0><<<g, b, 0, s>>>(p); break;
  }
}
static void launch_k2b(const Launch &l, const wmc::dev::K2BParams &p, cudaStream_t s) {
  if (l.ti == TD) launch_k2b_t<double>(l, p, s);
  else launch_k2b_t<float>(l, p, s);
}

template <typename T, int V, int D, bool FAST, int BC, int GROW, int SHRINK>
static void launch_k2c_t(const wmc::dev::K2CParams &p, int64_t blocks, size_t smem, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(dev::k2_chain<T, V, D, FAST, BC, GROW, SHRINK>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  // programmatic dependent launch: the kernel's barrier set-up and S_i
  // copies overlap the previous launch's tail (it waits for that launch
  // before touching anything it wrote)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(dev::kChainNW * 32 + 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = (g_pdl.load() && t_chain_pdl) ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, dev::k2_chain<T, V, D, FAST, BC, GROW, SHRINK>, p);
}

static bool chain_broadcast(const Launch &l) {
  for (int i = 0; i < l.chain_d; ++i)
    if (l.k2c.b_vec[i] != 1) return true;
  return false;
}

// vector lanes: FAST plain chains (contiguous lanes, or some steps with
// one value for all lanes or one load per lane), growth-first and
// shrink-last variants
template <int V, int D>
static void launch_k2c_vec(const Launch &l, const wmc::dev::K2CParams &p, cudaStream_t s) {
  if (!l.chain_fast) launch_k2c_t<float, V, D, false, 0, 0, 0>(p, l.blocks, l.smem, s);
  else if (l.chain_grow) launch_k2c_t<float, V, D, true, 0, 1, 0>(p, l.blocks, l.smem, s);
  else if (l.chain_shrink) launch_k2c_t<float, V, D, true, 0, 0, 1>(p, l.blocks, l.smem, s);
  else if (chain_broadcast(l)) launch_k2c_t<float, V, D, true, 1, 0, 0>(p, l.blocks, l.smem, s);
  else launch_k2c_t<float, V, D, true, 0, 0, 0>(p, l.blocks, l.smem, s);
}
template <typename T, int V, int D>
static void launch_k2c_plain(const Launch &l, const wmc::dev::K2CParams &p, cudaStream_t s) {
  if (!l.chain_fast) launch_k2c_t<T, V, D, false, 0, 0, 0>(p, l.blocks, l.smem, s);
  else if (V > 1 && chain_broadcast(l)) launch_k2c_t<T, V, D, true, 1, 0, 0>(p, l.blocks, l.smem, s);
  else launch_k2c_t<T, V, D, true, 0, 0, 0>(p, l.blocks, l.smem, s);
}

// instantiated (T, V, D) as try_chain chooses them: V at its largest for
// the state size, or 1 when the chain positions leave no vector lanes
template <int V, int D, bool SHRINK>
static void launch_k2c_direct(const Launch &l, const wmc::dev::K2CParams &p, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(dev::k2_chain_direct<float, V, D, SHRINK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         220 * 1024);
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)l.blocks);
  cfg.blockDim = dim3(l.threads > 0 ? (unsigned)l.threads : (unsigned)dev::kDirectThreads);
  cfg.dynamicSmemBytes = l.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = (g_pdl.load() && t_chain_pdl) ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, dev::k2_chain_direct<float, V, D, SHRINK>, p);
}

static void launch_k2c(const Launch &l, const wmc::dev::K2CParams &p, cudaStream_t s) {
  const int D = l.chain_d, V = l.v, NB = D + l.chain_grow;
  if (D > 4) {  // five or six steps, float32, one lane
    if (D == 5) {
      if (l.chain_shrink) launch_k2c_direct<1, 5, true>(l, p, s); else launch_k2c_direct<1, 5, false>(l, p, s);
    } else if (l.chain_shrink) {
      launch_k2c_direct<1, 6, true>(l, p, s);
    } else {
      launch_k2c_direct<1, 6, false>(l, p, s);
    }
    return;
  }
  if (l.ti == TF) {
    if (V == 1) {
      if (D == 2) launch_k2c_plain<float, 1, 2>(l, p, s);
      else if (D == 3) launch_k2c_plain<float, 1, 3>(l, p, s);
      else launch_k2c_plain<float, 1, 4>(l, p, s);
    } else if (D == 2) {
      launch_k2c_vec<4, 2>(l, p, s);
    } else if (D == 3 && NB == 3) {
      launch_k2c_vec<4, 3>(l, p, s);
    } else if (D == 3) {
      launch_k2c_vec<2, 3>(l, p, s);
    } else {
      launch_k2c_vec<2, 4>(l, p, s);
    }
  } else {
    if (D == 2) { if (V == 2) launch_k2c_plain<double, 2, 2>(l, p, s); else launch_k2c_plain<double, 1, 2>(l, p, s); }
    else if (D == 3) { if (V == 2) launch_k2c_plain<double, 2, 3>(l, p, s); else launch_k2c_plain<double, 1, 3>(l, p, s); }
    else launch_k2c_plain<double, 1, 4>(l, p, s);
  }
}

template <int V>
static void launch_k2cseq_t(const Launch &l, const wmc::dev::K2CParams *seq, char *ws, int stall, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(dev::k2_chain_seq<float, V, 4, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSeqDynSmem);
    attr_set = true;
  }
  dev::k2_chain_seq<float, V, 4, true, 0><<<(unsigned)l.blocks, dev::kChainNW * 32 + 32, l.smem, s>>>(
      seq + l.seq_first, (int32_t)l.chains.size(), (uint32_t *)(ws + l.seq_ctr_off), ws, stall);
}
static void launch_k2cseq(const Launch &l, const wmc::dev::K2CParams *seq, char *ws, int stall, cudaStream_t s) {
  if (l.v == 2) launch_k2cseq_t<2>(l, seq, ws, stall, s);
  else launch_k2cseq_t<1>(l, seq, ws, stall, s);
}

static void launch_k1(const Launch &l, const K1Params &p, cudaStream_t s) {
  const unsigned g = (unsigned)l.blocks;
  if (l.ti == TD) dev::k1_generic<double, double, double><<<g, dev::kThreads, 0, s>>>(p);
  else if (l.ta == TF) dev::k1_generic<float, float, float><<<g, dev::kThreads, 0, s>>>(p);
  else if (l.to == TD) dev::k1_generic<float, double, double><<<g, dev::kThreads, 0, s>>>(p);
  else dev::k1_generic<float, double, float><<<g, dev::kThreads, 0, s>>>(p);
}

static int ensure_dev(ExecState &st) {
  if (st.dev_ready) return WMC_OK;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    int rc = dev_alloc(dst, bytes);
    if (rc) return rc;
    if (bytes) CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return WMC_OK;
  };
  int rc;
  if ((rc = up((void **)&st.d_clause, st.h_clause.data(), sizeof(ClauseLeaf) * st.h_clause.size()))) return rc;
  if ((rc = up((void **)&st.d_first, st.h_first.data(), sizeof(int64_t) * st.h_first.size()))) return rc;
  if ((rc = up((void **)&st.d_woff, st.h_woff.data(), sizeof(int64_t) * st.h_woff.size()))) return rc;
  if ((rc = up((void **)&st.d_wmeta, st.h_wmeta.data(), sizeof(int64_t) * st.h_wmeta.size()))) return rc;
  if ((rc = up((void **)&st.d_snodes, st.h_snodes.data(), sizeof(wmc::dev::SNode) * st.h_snodes.size()))) return rc;
  if ((rc = up((void **)&st.d_stasks, st.h_stasks.data(), sizeof(wmc::dev::STask) * st.h_stasks.size()))) return rc;
  if ((rc = up((void **)&st.d_seq, st.h_seq.data(), sizeof(wmc::dev::K2CParams) * st.h_seq.size()))) return rc;
  if ((rc = up((void **)&st.d_cta, st.h_cta.data(), sizeof(wmc::dev::CtaLeaf) * st.h_cta.size()))) return rc;
  CUDA_TRY(cudaStreamCreateWithFlags(&st.capture_stream, cudaStreamNonBlocking));
  st.dev_ready = true;
  return WMC_OK;
}

// Enqueues the whole walk on `s` for workspace `ws`.  With `events`, an
// event is recorded after every launch (measurement only).
struct LeafTables {
  const ClauseLeaf *clause;
  const int64_t *first, *woff, *wmeta;
  const wmc::dev::SNode *snodes;
  const wmc::dev::STask *stasks;
  const wmc::dev::K2CParams *seq;
  const wmc::dev::CtaLeaf *cta;
};

static void enqueue_walk(Plan &plan, ExecState &st, char *ws, cudaStream_t s,
                         cudaEvent_t *events = nullptr, const LeafTables *tables = nullptr) {
  const LeafTables own{st.d_clause, st.d_first, st.d_woff, st.d_wmeta, st.d_snodes, st.d_stasks, st.d_seq, st.d_cta};
  const LeafTables &tb = tables ? *tables : own;
  int64_t *mexp = (int64_t *)(ws + st.off_exp);
  unsigned long long *mmax = (unsigned long long *)(ws + st.off_max);
  unsigned long long *mmin = (unsigned long long *)(ws + st.off_min);
  uint32_t *flags = (uint32_t *)(ws + st.off_flags);
  const IoDesc *io = (const IoDesc *)(ws + st.off_io);
  // test hook: 1 = the first staged launch (bulk copies), 2 = the first run of chains
  const int stall_mode = g_debug_stall.load();
  bool stall_armed = stall_mode == 1;
  bool stall_run_armed = stall_mode == 2;
  for (size_t li = 0; li < st.launches.size(); ++li) {
    const Launch &l = st.launches[li];
    switch (l.kind) {
      case L_MEMSET:
        cudaMemsetAsync(ws + l.memset_off, l.memset_value, (size_t)l.memset_bytes, s);
        break;
      case L_CLAUSES:
        if (st.f64)
          dev::k_clause_leaves<double><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
              tb.clause, tb.first, (int64_t)st.h_clause.size(), st.n_clause_entries,
              (double *)ws, mexp, mmax, mmin, io);
        else
          dev::k_clause_leaves<float><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
              tb.clause, tb.first, (int64_t)st.h_clause.size(), st.n_clause_entries,
              (float *)ws, mexp, mmax, mmin, io);
        break;
      case L_WEIGHTS:
        if (st.f64)
          dev::k_weight_leaves<double><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
              io, plan.n_vars, st.Q, st.Qp, tb.woff, tb.wmeta, (double *)ws, mexp, mmax, mmin, flags);
        else
          dev::k_weight_leaves<float><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
              io, plan.n_vars, st.Q, st.Qp, tb.woff, tb.wmeta, (float *)ws, mexp, mmax, mmin, flags);
        break;
      case L_ONE:
        if (st.f64) dev::k_one_leaf<double><<<1, 32, 0, s>>>((double *)(ws + l.one_off), l.one_meta, mexp, mmax, mmin);
        else dev::k_one_leaf<float><<<1, 32, 0, s>>>((float *)(ws + l.one_off), l.one_meta, mexp, mmax, mmin);
        break;
      case L_K1: {
        K1Params p = l.k1;
        p.A = ws + l.off_a; p.B = ws + l.off_b; p.C = ws + l.off_c;
        p.ma.exp = mexp + l.meta_a; p.ma.maxb = mmax + l.meta_a; p.ma.minb = mmin + l.meta_a;
        p.mb.exp = mexp + l.meta_b; p.mb.maxb = mmax + l.meta_b; p.mb.minb = mmin + l.meta_b;
        p.mc.exp = mexp + l.meta_c; p.mc.maxb = mmax + l.meta_c; p.mc.minb = mmin + l.meta_c;
        p.mc.flags = flags;
        launch_k1(l, p, s);
        break;
      }
      case L_K2T: {
        dev::K2TParams tp = l.k2t;
        K2Params &p = tp.k;
        p = l.k2;
        p.A = ws + l.off_a; p.B = ws + l.off_b; p.C = ws + l.off_c;
        p.ma.exp = mexp + l.meta_a; p.ma.maxb = mmax + l.meta_a; p.ma.minb = mmin + l.meta_a;
        p.mb.exp = mexp + l.meta_b; p.mb.maxb = mmax + l.meta_b; p.mb.minb = mmin + l.meta_b;
        p.mc.exp = mexp + l.meta_c; p.mc.maxb = mmax + l.meta_c; p.mc.minb = mmin + l.meta_c;
        p.mc.flags = flags;
        tp.err = (uint32_t *)(ws + st.off_err);
        tp.debug_stall = stall_armed ? 1 : 0;
        stall_armed = false;
        launch_k2t(l, tp, s);
        break;
      }
      case L_SMALL: {
        wmc::dev::SmallArgs a;
        a.ws = ws;
        a.nodes = tb.snodes;
        a.tasks = tb.stasks;
        a.n_tasks = (int32_t)st.h_stasks.size();
        a.Q = st.Qp;
        a.next = (uint32_t *)(ws + st.off_sp);
        a.done = a.next + 1;
        a.err = (uint32_t *)(ws + st.off_err);
        a.flags = flags;
        a.mexp = mexp;
        a.mmax = mmax;
        a.mmin = mmin;
        dev::k_small_phase<<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(a);
        break;
      }
      case L_K2C: {
        wmc::dev::K2CParams cp = l.k2c;
        cp.P = ws + l.off_a;
        cp.C = ws + l.off_c;
        cp.mp.exp = mexp + l.meta_a; cp.mp.maxb = mmax + l.meta_a; cp.mp.minb = mmin + l.meta_a;
        for (int i = 0; i < l.chain_d; ++i) {
          cp.S[i] = ws + l.off_sc[i];
          cp.ms[i].exp = mexp + l.meta_sc[i]; cp.ms[i].maxb = mmax + l.meta_sc[i]; cp.ms[i].minb = mmin + l.meta_sc[i];
        }
        cp.mc.exp = mexp + l.meta_c; cp.mc.maxb = mmax + l.meta_c; cp.mc.minb = mmin + l.meta_c;
        cp.mc.flags = flags;
        cp.err = (uint32_t *)(ws + st.off_err);
        t_chain_pdl = l.no_pdl == 0;
        // (the test hook stalls a staged copy: direct-load chains have none)
        cp.debug_stall = (stall_armed && l.chain_d <= 4) ? 1 : 0;
        if (l.chain_d <= 4) stall_armed = false;
        launch_k2c(l, cp, s);
        break;
      }
      case L_K2CSEQ:
        launch_k2cseq(l, tb.seq, ws, (stall_armed || stall_run_armed) ? 1 : 0, s);
        stall_armed = stall_run_armed = false;
        break;
      case L_K4: {
        wmc::dev::K4Params p = l.k4;
        p.A = ws + l.off_a; p.B = ws + l.off_b; p.C = ws + l.off_c;
        p.ma.exp = mexp + l.meta_a; p.ma.maxb = mmax + l.meta_a; p.ma.minb = mmin + l.meta_a;
        p.mb.exp = mexp + l.meta_b; p.mb.maxb = mmax + l.meta_b; p.mb.minb = mmin + l.meta_b;
        p.mc.exp = mexp + l.meta_c; p.mc.maxb = mmax + l.meta_c; p.mc.minb = mmin + l.meta_c;
        p.mc.flags = flags;
        if (l.ti == TD) dev::k4_dense<double><<<(unsigned)l.blocks, 256, 0, s>>>(p);
        else dev::k4_dense<float><<<(unsigned)l.blocks, 256, 0, s>>>(p);
        break;
      }
      case L_K2B: {
        wmc::dev::K2BParams p = l.k2b;
        p.A = ws + l.off_a; p.B = ws + l.off_b; p.C = ws + l.off_c;
        p.ma.exp = mexp + l.meta_a; p.ma.maxb = mmax + l.meta_a; p.ma.minb = mmin + l.meta_a;
        p.mb.exp = mexp + l.meta_b; p.mb.maxb = mmax + l.meta_b; p.mb.minb = mmin + l.meta_b;
        p.mc.exp = mexp + l.meta_c; p.mc.maxb = mmax + l.meta_c; p.mc.minb = mmin + l.meta_c;
        p.mc.flags = flags;
        launch_k2b(l, p, s);
        break;
      }
      case L_K2: {
        K2Params p = l.k2;
        p.A = ws + l.off_a; p.B = ws + l.off_b; p.C = ws + l.off_c;
        p.ma.exp = mexp + l.meta_a; p.ma.maxb = mmax + l.meta_a; p.ma.minb = mmin + l.meta_a;
        p.mb.exp = mexp + l.meta_b; p.mb.maxb = mmax + l.meta_b; p.mb.minb = mmin + l.meta_b;
        p.mc.exp = mexp + l.meta_c; p.mc.maxb = mmax + l.meta_c; p.mc.minb = mmin + l.meta_c;
        p.mc.flags = flags;
        launch_k2(l, p, s);
        break;
      }
      case L_CTA: {
        wmc::dev::CtaArgs a;
        a.ws = ws;
        a.nodes = tb.snodes;
        a.leaves = tb.cta;
        a.io = io;
        a.flags = flags;
        a.gexp = mexp;
        a.n_nodes = (int32_t)st.h_snodes.size();
        a.n_leaves = (int32_t)st.h_cta.size();
        a.n_slots = (int32_t)st.n_slots;
        a.n_vars = plan.n_vars;
        a.Q = st.Q;
        a.Qp = st.Qp;
        a.f64 = st.f64 ? 1 : 0;
        a.nodes_off = (uint32_t)align_up(24 * st.n_slots);
        a.leaves_off = a.nodes_off + (uint32_t)align_up((int64_t)sizeof(wmc::dev::SNode) * (int64_t)st.h_snodes.size());
        a.meta_bytes = (uint32_t)st.cta_meta;
        a.lut_off = (uint32_t)st.cta_lut_off;
        static bool attr_set = false;  // opt in to large dynamic shared memory once
        if (!attr_set) {
          cudaFuncSetAttribute(dev::k_cta_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
          attr_set = true;
        }
        dev::k_cta_walk<<<1, 1024, l.smem, s>>>(a);
        break;
      }
      case L_BFPW:
        dev::k_bfp_weights<<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
            io, plan.n_vars, st.Q, st.Qp, tb.woff, (float *)ws, align_up(8 * (int64_t)st.Qp), flags);
        break;
      case L_BFP: {
        dev::BfpParams p;
        std::memset(&p, 0, sizeof(p));
        p.k1 = l.k1;
        p.k1.A = ws + l.off_a; p.k1.B = ws + l.off_b; p.k1.C = ws + l.off_c;
        const TensorInfo &TA = plan.tensors[(size_t)l.id_a], &TB = plan.tensors[(size_t)l.id_b];
        const TensorInfo &TC = plan.tensors[(size_t)l.id_c];
        p.eA = (const int32_t *)(ws + st.t_eoff[(size_t)l.id_a]);
        p.eB = (const int32_t *)(ws + st.t_eoff[(size_t)l.id_b]);
        p.eC = (int32_t *)(ws + st.t_eoff[(size_t)l.id_c]);
        p.mA = (int8_t)(TA.has_q ? st.m : 0); p.mB = (int8_t)(TB.has_q ? st.m : 0); p.mC = (int8_t)(TC.has_q ? st.m : 0);
        p.bA = st.t_bb[(size_t)l.id_a]; p.bB = st.t_bb[(size_t)l.id_b]; p.bC = st.t_bb[(size_t)l.id_c];
        p.c_double = l.to == TD ? 1 : 0;
        p.root_exp = mexp + l.meta_c;
        p.flags = flags;
        p.n_blocks = int64_t(1) << ((int64_t)TC.labels.size() - p.bC);
        if (l.to == TD) dev::k_bfp_node<double><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(p);
        else dev::k_bfp_node<float><<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(p);
        break;
      }
      case L_FINAL: {
        const int32_t root_qc = plan.tensors[(size_t)plan.nodes.back().c].has_q ? st.Qp : 1;
        dev::k_finalize<<<(unsigned)l.blocks, dev::kThreads, 0, s>>>(
            io, (const double *)(ws + l.off_c), mexp + l.meta_c, root_qc, flags,
            (const uint32_t *)(ws + st.off_err), st.Q, plan.n_vars);
        break;
      }
    }
    if (events) cudaEventRecord(events[li + 1], s);
  }
}

static int get_graph(Plan &plan, ExecState &st, char *ws, cudaGraphExec_t *out) {
  auto it = st.graphs.find((uintptr_t)ws);
  if (it != st.graphs.end()) { *out = it->second; return WMC_OK; }
  if (st.graphs.size() >= 8) {  // bound the cache
    cudaGraphExecDestroy(st.graphs.begin()->second);
    st.graphs.erase(st.graphs.begin());
  }
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(st.capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_walk(plan, st, ws, st.capture_stream);
  cudaError_t e = cudaStreamEndCapture(st.capture_stream, &g);
  if (e != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    if (g) cudaGraphDestroy(g);
    return WMC_ECUDA;
  }
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error("graph instantiate failed: %s", cudaGetErrorString(e));
    return WMC_ECUDA;
  }
  st.graphs[(uintptr_t)ws] = ge;
  *out = ge;
  return WMC_OK;
}

static int get_state(Plan &plan, int32_t Q, ExecState **out, bool plain = false, bool f64 = false) {
  std::lock_guard<std::mutex> lk(plan.exec_mu);
  auto &cache = f64 ? plan.exec_f64 : (plain ? plan.exec_plain : plan.exec);
  auto it = cache.find(Q);
  if (it != cache.end()) { *out = it->second.get(); return WMC_OK; }
  std::unique_ptr<ExecState> st(new (std::nothrow) ExecState());
  if (!st) { set_error("out of host memory"); return WMC_ENOMEM; }
  int rc = build_exec(plan, Q, *st, plain, f64);
  if (rc) return rc;
  *out = st.get();
  cache[Q] = std::move(st);
  return WMC_OK;
}

namespace wmc {
int64_t plan_workspace_bytes(Plan &plan, int32_t Q, int64_t *arena_bytes) {
  ExecState *st = nullptr;
  if (get_state(plan, Q, &st)) return -1;
  if (arena_bytes) *arena_bytes = st->arena_bytes;
  return st->ws_bytes;
}
}  // namespace wmc

static int check_q(int32_t Q) {
  if (Q < 1 || Q > dev::kMaxQ) { set_error("Q = %d out of [1, %d]", Q, dev::kMaxQ); return WMC_EINVAL; }
  return WMC_OK;
}

static IoDesc io_desc(const Plan &plan, const double *d_wp, const double *d_wn, double *d_mant,
                      int64_t *d_exp, uint32_t *d_flags) {
  IoDesc io;
  std::memset(&io, 0, sizeof(io));
  io.w_pos = d_wp; io.w_neg = d_wn; io.mant = d_mant; io.exp2 = d_exp; io.flags = d_flags;
  io.n_slice = (int32_t)plan.slice_vars.size();
  for (size_t k = 0; k < plan.slice_vars.size(); ++k) io.slice_var[k] = plan.slice_vars[k];
  return io;
}

static int64_t n_slices(const Plan &plan) { return int64_t(1) << plan.slice_vars.size(); }

// Runs the walk for a power-of-two batch Qp >= Q on device pointers, once
// per slice assignment in [slice_lo, slice_hi) (index slicing: the results
// accumulate in the outputs; an unsliced plan has the single slice 0).
// With lanes_per_slice > 0 it runs one walk whose lane l (l < n_lanes)
// takes slice slice_lo + l / lanes_per_slice.
static int run_device(Plan &plan, ExecState &st, const double *d_wp, const double *d_wn,
                      char *ws, double *d_mant, int64_t *d_exp, uint32_t *d_flags,
                      cudaStream_t s, int64_t slice_lo = 0, int64_t slice_hi = -1, int32_t lanes_per_slice = 0,
                      int32_t n_lanes = 0, IoDesc *h_io = nullptr) {
  if (slice_hi < 0) slice_hi = n_slices(plan);
  if (slice_lo < 0 || slice_lo >= slice_hi || slice_hi > n_slices(plan)) {
    set_error("slice range [%lld, %lld) outside [0, %lld)", (long long)slice_lo, (long long)slice_hi,
              (long long)n_slices(plan));
    return WMC_EINVAL;
  }
  int rc = ensure_dev(st);
  if (rc) return rc;
  cudaGraphExec_t ge = nullptr;
  {
    std::lock_guard<std::mutex> lk(st.graph_mu);
    rc = get_graph(plan, st, ws, &ge);
  }
  if (rc) return rc;
  IoDesc io = io_desc(plan, d_wp, d_wn, d_mant, d_exp, d_flags);
  if (lanes_per_slice > 0) {
    io.slice = (uint64_t)slice_lo;
    io.lanes_per_slice = lanes_per_slice;
    io.n_lanes = n_lanes;
    if (h_io) *h_io = io;
    CUDA_TRY(cudaMemcpyAsync(ws + st.off_io, h_io ? h_io : &io, sizeof(io), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(ge, s));
    g_launches.fetch_add(st.kernels_per_run);
    return WMC_OK;
  }
  // (the pinned descriptor serves one launch: a later one would overwrite
  // it before the earlier copy has run)
  if (slice_hi - slice_lo != 1) h_io = nullptr;
  for (int64_t eta = slice_lo; eta < slice_hi; ++eta) {
    io.slice = (uint64_t)eta;
    io.accumulate = eta != slice_lo;
    if (h_io) *h_io = io;
    CUDA_TRY(cudaMemcpyAsync(ws + st.off_io, h_io ? h_io : &io, sizeof(io), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(ge, s));
    g_launches.fetch_add(st.kernels_per_run);
  }
  return WMC_OK;
}

// ------------------------------------------------------ walk autotuning
//
// For one plan and batch size, times the walk under several layouts --
// chains of up to 4, 3 or 2 frontier eliminations per pass or none, the
// small-node phase on or off, runs of chains in one launch -- and installs
// the fastest as the plan's state for that Q.  Every layout adds each
// node's terms in the canonical order and differs from the others only by
// power-of-two scales, so all give the same bits; a layout whose results
// differ from the first one's is rejected.
extern "C" int wmc_autotune_plan(wmc_plan_t *cplan, int32_t Q, void *stream, wmc_tune_report *rep) {
  if (!cplan || !rep) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  Plan &plan = *cplan;
  std::memset(rep, 0, sizeof(*rep));
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = plan.precision == WMC_FP64;
  std::vector<WalkOpts> cands;
  auto add = [&](int fuse, int sp, int runs) {
    WalkOpts w; w.fuse = fuse; w.small_phase = sp; w.chain_runs = runs;
    cands.push_back(w);
  };
  add(6, 1, 0); add(4, 1, 0); add(3, 1, 0); add(2, 1, 0); add(0, 1, 0); add(6, 0, 0);
  if (!f64) add(4, 1, 512);
  // inputs: the network's default weights for every query
  const size_t nv = (size_t)plan.n_vars;
  std::vector<double> hw(2 * (size_t)Q * std::max<size_t>(nv, 1), 1.0);
  for (int32_t q = 0; q < Q; ++q)
    for (size_t v = 0; v < nv; ++v) {
      hw[(size_t)q * nv + v] = plan.w_pos[v];
      hw[(size_t)Q * nv + (size_t)q * nv + v] = plan.w_neg[v];
    }
  char *dbuf = nullptr;
  const size_t w_bytes = sizeof(double) * hw.size();
  const size_t o_out = (w_bytes + 255) / 256 * 256;
  int rc = device_alloc((void **)&dbuf, o_out + (size_t)Q * (8 + 8 + 4) + 64);
  if (rc) return rc;
  const double *d_wp = (const double *)dbuf, *d_wn = d_wp + (size_t)Q * nv;
  double *d_mant = (double *)(dbuf + o_out);
  int64_t *d_exp = (int64_t *)(d_mant + Q);
  uint32_t *d_flags = (uint32_t *)(d_exp + Q);
  std::vector<std::unique_ptr<ExecState>> states;
  std::vector<double> ref_m;
  std::vector<int64_t> ref_e;
  std::vector<uint32_t> ref_f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto fail = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(dbuf);
    return code;
  };
  if (cudaMemcpyAsync(dbuf, hw.data(), w_bytes, cudaMemcpyHostToDevice, s) || cudaEventCreate(&e0) ||
      cudaEventCreate(&e1)) {
    set_error("autotune set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(WMC_ECUDA);
  }
  int best = -1;
  for (size_t i = 0; i < cands.size() && i < 8; ++i) {
    std::unique_ptr<ExecState> st(new (std::nothrow) ExecState());
    if (!st) { set_error("out of host memory"); return fail(WMC_ENOMEM); }
    if ((rc = build_exec(plan, Q, *st, false, false, &cands[i]))) return fail(rc);
    if ((rc = ensure_dev(*st))) return fail(rc);
    char *ws = nullptr;
    if ((rc = device_alloc((void **)&ws, (size_t)st->ws_bytes))) return fail(rc);
    std::vector<float> times;
    for (int r = 0; r < 7 && rc == WMC_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = run_device(plan, *st, d_wp, d_wn, ws, d_mant, d_exp, d_flags, s);
      cudaEventRecord(e1, s);
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("autotune walk failed: %s", cudaGetErrorString(cudaGetLastError()));
        rc = WMC_ECUDA;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r >= 2) times.push_back(ms);  // two warm-up walks (graph capture)
    }
    std::vector<double> m((size_t)Q);
    std::vector<int64_t> ex((size_t)Q);
    std::vector<uint32_t> fl((size_t)Q);
    if (!rc && (cudaMemcpy(m.data(), d_mant, 8 * (size_t)Q, cudaMemcpyDeviceToHost) ||
                cudaMemcpy(ex.data(), d_exp, 8 * (size_t)Q, cudaMemcpyDeviceToHost) ||
                cudaMemcpy(fl.data(), d_flags, 4 * (size_t)Q, cudaMemcpyDeviceToHost))) {
      set_error("autotune read-back failed");
      rc = WMC_ECUDA;
    }
    cudaFree(ws);
    if (rc) return fail(rc);
    std::sort(times.begin(), times.end());
    float med = times[times.size() / 2];
    if (i == 0) { ref_m = m; ref_e = ex; ref_f = fl; }
    else {
      // compare values as mant * 2^exp (the unnormalised mantissas of two
      // layouts may differ by powers of two)
      for (int32_t q = 0; q < Q && med >= 0; ++q) {
        int fa = 0, fb = 0;
        const double ma = std::frexp(m[(size_t)q], &fa), mb = std::frexp(ref_m[(size_t)q], &fb);
        const bool same = ma == mb && (ma == 0.0 || ex[(size_t)q] + fa == ref_e[(size_t)q] + fb) &&
                          fl[(size_t)q] == ref_f[(size_t)q];
        if (!same) med = -1.0f;
      }
    }
    rep->fuse[i] = cands[i].fuse;
    rep->small_phase[i] = cands[i].small_phase;
    rep->chain_runs[i] = cands[i].chain_runs;
    rep->launches[i] = (int32_t)st->kernels_per_run;
    rep->ms[i] = med;
    rep->n_candidates = (int32_t)i + 1;
    if (med >= 0 && (best < 0 || med < rep->ms[best])) best = (int)i;
    states.push_back(std::move(st));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dbuf);
  if (best < 0) { set_error("no layout could be timed"); return WMC_ECUDA; }
  rep->chosen = best;
  std::lock_guard<std::mutex> lk(plan.exec_mu);
  auto it = plan.exec.find(Q);
  if (it != plan.exec.end()) plan.retired.push_back(std::move(it->second));  // may still be in use
  plan.exec[Q] = std::move(states[(size_t)best]);
  return WMC_OK;
}

static void fill_result(const ExecState &st, double mant, int64_t e,
                        uint32_t flags, bool unit, bool negative, wmc_result *r) {
  int fe = 0;
  double fr = std::frexp(mant, &fe);
  r->mant = fr;
  r->exp2 = (mant == 0.0) ? 0 : e + fe;
  r->log10 = (mant == 0.0) ? -INFINITY : std::log10(std::fabs(fr)) + (double)r->exp2 * std::log10(2.0);
  r->flags = flags & (WMC_FLAG_FP32_FLUSH | WMC_FLAG_DEVICE_TIMEOUT);
  const double u = st.f64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  const double d = (double)st.max_roundings;
  r->rel_err_bound = d * u / (1.0 - d * u);
  if (st.n_slice_vars > 0) {  // float64 slice factors (s roundings) and the sum of 2^s slices
    const double ds = (double)st.n_slice_vars + std::ldexp(1.0, st.n_slice_vars) - 1.0;
    r->rel_err_bound += ds * std::ldexp(1.0, -53);
  }
  if (negative) r->flags |= WMC_FLAG_NO_BOUND;
  // (a zero count with unit weights is exactly zero: a slice's share that a
  // clause rules out keeps the sum over slices exact)
  if (unit && st.f64 &&
      (mant == 0.0 || (r->exp2 <= 53 && std::ldexp(fr, (int)r->exp2) == std::floor(std::ldexp(fr, (int)r->exp2)))))
    r->flags |= WMC_FLAG_EXACT_INT;
  r->reserved = 0;
}

// ------------------------------------------------------------ C ABI

extern "C" int wmc_plan(const wmc_network_t *net, const wmc_plan_opts *opts, wmc_plan_t **out) {
  if (!net || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  *out = nullptr;
  wmc_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  o.precision = WMC_SCALED_FP32;
  if (opts) o = *opts;
  if (o.precision != WMC_FP64 && o.precision != WMC_SCALED_FP32) { set_error("bad precision %d", o.precision); return WMC_EINVAL; }
  if (o.block_fp < 0 || o.block_fp > 9) { set_error("block_fp must be in [0, 9] (got %d)", o.block_fp); return WMC_EINVAL; }
  if (o.block_fp && (o.precision != WMC_SCALED_FP32 || o.slice_to_rank > 0)) {
    set_error("block floating point needs a scaled-FP32 plan without index slicing");
    return WMC_EINVAL;
  }
  wmc_plan_t *p = new (std::nothrow) wmc_plan_t();
  if (!p) { set_error("out of host memory"); return WMC_ENOMEM; }
  int rc = build_plan(network_of(net), o, *p);
  if (rc) { delete p; return rc; }
  p->bfp_b = o.block_fp - 1;
  if (o.mem_budget_bytes > 0) {
    int64_t ws = plan_workspace_bytes(*p, 1, nullptr);
    if (ws < 0) { delete p; return WMC_EPLAN_TOO_BIG; }
    if (ws > o.mem_budget_bytes) {
      set_error("plan needs %lld bytes at Q=1, budget %lld", (long long)ws, (long long)o.mem_budget_bytes);
      delete p;
      return WMC_EPLAN_TOO_BIG;
    }
  }
  *out = p;
  return WMC_OK;
}

extern "C" void wmc_plan_destroy(wmc_plan_t *plan) { delete plan; }

extern "C" int wmc_plan_info(const wmc_plan_t *cplan, int32_t Q, wmc_plan_info_t *out) {
  if (!cplan || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  wmc_plan_t *plan = const_cast<wmc_plan_t *>(cplan);
  ExecState *st = nullptr;
  int rc = get_state(*plan, Q, &st);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  out->max_rank = plan->max_rank;
  out->max_node_rank = plan->max_node_rank;
  out->n_leaves = plan->n_leaves;
  out->n_nodes = (int64_t)plan->nodes.size();
  out->workspace_bytes = st->ws_bytes;
  out->peak_tensor_bytes = st->arena_bytes;
  out->algorithmic_bytes = st->alg_bytes;
  out->flops = st->flops;
  out->precision = plan->precision;
  out->ordering_used = plan->ordering_used;
  out->max_path_roundings = st->max_roundings;
  out->launches_per_walk = (int32_t)st->kernels_per_run;
  out->n_slice_vars = (int32_t)plan->slice_vars.size();
  for (size_t k = 0; k < plan->slice_vars.size() && k < 24; ++k) out->slice_vars[k] = plan->slice_vars[k];
  out->n_aux_vars = plan->n_aux;
  return WMC_OK;
}

extern "C" int wmc_plan_node(const wmc_plan_t *plan, int64_t node, int64_t *left, int64_t *right,
                             int32_t *n_labels, int32_t *labels) {
  if (!plan || node < 0 || node >= (int64_t)plan->nodes.size()) { set_error("bad node id"); return WMC_EINVAL; }
  const Node &nd = plan->nodes[(size_t)node];
  const TensorInfo &c = plan->tensors[(size_t)nd.c];
  if (left) *left = nd.a;
  if (right) *right = nd.b;
  if (n_labels) *n_labels = (int32_t)c.labels.size();
  if (labels) for (size_t i = 0; i < c.labels.size() && i < 64; ++i) labels[i] = c.labels[i];
  return WMC_OK;
}

extern "C" int wmc_plan_leaf(const wmc_plan_t *plan, int64_t leaf, int32_t *kind, int32_t *n_labels,
                             int32_t *labels, uint64_t *fals) {
  if (!plan || leaf < 0 || leaf >= plan->n_leaves) { set_error("bad leaf id"); return WMC_EINVAL; }
  const TensorInfo &t = plan->tensors[(size_t)leaf];
  if (kind) *kind = t.kind;
  if (n_labels) *n_labels = (int32_t)t.labels.size();
  if (labels) for (size_t i = 0; i < t.labels.size() && i < 64; ++i) labels[i] = t.labels[i];
  if (fals) *fals = t.fals;
  return WMC_OK;
}

extern "C" int wmc_execute_device(wmc_plan_t *plan, int32_t Q, const double *d_w_pos,
                                  const double *d_w_neg, void *d_workspace, size_t workspace_bytes,
                                  double *d_mant, int64_t *d_exp2, uint32_t *d_flags, void *stream) {
  if (!plan || !d_workspace || !d_mant || !d_exp2 || !d_flags) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  if (plan->n_vars > 0 && (!d_w_pos || !d_w_neg)) { set_error("weights are NULL"); return WMC_EINVAL; }
  if ((uintptr_t)d_workspace % kAlign) { set_error("workspace not 256-byte aligned"); return WMC_EINVAL; }
  ExecState *st = nullptr;
  int rc = get_state(*plan, Q, &st);
  if (rc) return rc;
  if ((int64_t)workspace_bytes < st->ws_bytes) {
    set_error("workspace %zu bytes < %lld needed", workspace_bytes, (long long)st->ws_bytes);
    return WMC_EINVAL;
  }
  return run_device(*plan, *st, d_w_pos, d_w_neg, (char *)d_workspace, d_mant, d_exp2, d_flags,
                    (cudaStream_t)stream);
}

extern "C" int wmc_profile_walk(wmc_plan_t *plan, int32_t Q, const double *d_w_pos,
                                const double *d_w_neg, void *d_workspace, size_t workspace_bytes,
                                double *d_mant, int64_t *d_exp2, uint32_t *d_flags, void *stream,
                                int64_t n_max, float *node_ms, int32_t *kind, double *alg_bytes,
                                int64_t *n_launches) {
  if (!plan || !d_workspace || !d_mant || !d_exp2 || !d_flags) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  ExecState *st = nullptr;
  int rc = get_state(*plan, Q, &st);
  if (rc) return rc;
  if ((int64_t)workspace_bytes < st->ws_bytes || (uintptr_t)d_workspace % kAlign) {
    set_error("workspace too small or misaligned");
    return WMC_EINVAL;
  }
  if ((rc = ensure_dev(*st))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nl = st->launches.size();
  std::vector<cudaEvent_t> ev(nl + 1, nullptr);
  for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
  const IoDesc io = io_desc(*plan, d_w_pos, d_w_neg, d_mant, d_exp2, d_flags);  // slice 0
  char *ws = (char *)d_workspace;
  CUDA_TRY(cudaMemcpyAsync(ws + st->off_io, &io, sizeof(io), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaEventRecord(ev[0], s));
  enqueue_walk(*plan, *st, ws, s, ev.data());
  g_launches.fetch_add(st->kernels_per_run);
  CUDA_TRY(cudaStreamSynchronize(s));
  for (size_t i = 0; i < nl && (int64_t)i < n_max; ++i) {
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
    const Launch &l = st->launches[i];
    if (node_ms) node_ms[i] = ms;
    if (kind) kind[i] = l.kind == L_CTA ? 10 : (l.kind == L_K1 || l.kind == L_BFP) ? 0 : l.kind == L_K2 ? 1 : l.kind == L_K2T ? 4 : l.kind == L_K4 ? 5 : l.kind == L_SMALL ? 7 : l.kind == L_K2C ? 8 : l.kind == L_K2CSEQ ? 9 : l.kind == L_K2B ? 11 : l.kind == L_MEMSET ? 3 : 2;
    if (alg_bytes) alg_bytes[i] = l.alg_bytes;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (n_launches) *n_launches = (int64_t)nl;
  return WMC_OK;
}

static int execute_host(wmc_plan_t *plan, int32_t Q, const double *w_pos_q, const double *w_neg_q,
                        int64_t slice_lo, int64_t slice_hi, void *stream, wmc_result *out);

extern "C" int wmc_execute(wmc_plan_t *plan, int32_t Q, const double *w_pos_q, const double *w_neg_q,
                           void *stream, wmc_result *out) {
  if (!plan) { set_error("NULL argument"); return WMC_EINVAL; }
  return execute_host(plan, Q, w_pos_q, w_neg_q, 0, n_slices(*plan), stream, out);
}

extern "C" int wmc_execute_slices(wmc_plan_t *plan, int32_t Q, const double *w_pos_q,
                                  const double *w_neg_q, int64_t slice_lo, int64_t slice_hi,
                                  void *stream, wmc_result *out) {
  if (!plan) { set_error("NULL argument"); return WMC_EINVAL; }
  if (slice_lo < 0 || slice_lo > slice_hi || slice_hi > n_slices(*plan)) {
    set_error("slice range [%lld, %lld) outside [0, %lld]", (long long)slice_lo, (long long)slice_hi,
              (long long)n_slices(*plan));
    return WMC_EINVAL;
  }
  if (slice_lo == slice_hi) {  // an empty range: the sum is 0
    if (!out) { set_error("NULL argument"); return WMC_EINVAL; }
    if (check_q(Q)) return WMC_EINVAL;
    for (int32_t q = 0; q < Q; ++q) {
      std::memset(out + q, 0, sizeof(wmc_result));
      out[q].log10 = -INFINITY;
    }
    return WMC_OK;
  }
  return execute_host(plan, Q, w_pos_q, w_neg_q, slice_lo, slice_hi, stream, out);
}

// One walk of state `st` with host weights, results filled into out[Q].
// pinned staging per execution state: the call descriptor (256-byte slot)
// and up to 64 KB of weights (larger inputs take the pageable path)
static constexpr size_t kStageIoBytes = (sizeof(IoDesc) + 255) / 256 * 256;
static constexpr size_t kStageWeightBytes = size_t(64) << 10;

static int run_host(wmc_plan_t *plan, ExecState *st, int32_t Q, const double *w_pos_q, const double *w_neg_q,
                    int64_t slice_lo, int64_t slice_hi, void *stream, wmc_result *out, int32_t lanes_per_slice = 0,
                    int32_t n_lanes = 0) {
  int rc = WMC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nv = (size_t)plan->n_vars;
  std::lock_guard<std::mutex> run(st->run_mu);  // the owned workspace is single-use at a time
  {
    if (!st->own_ws) {
      if ((rc = dev_alloc(&st->own_ws, (size_t)st->ws_bytes))) return rc;
      if ((rc = dev_alloc((void **)&st->d_w, sizeof(double) * 2 * (size_t)Q * std::max<size_t>(nv, 1)))) return rc;
      const size_t res_bytes = 20 * (size_t)Q;
      if ((rc = dev_alloc((void **)&st->d_res_mant, res_bytes))) return rc;
      st->d_res_exp = (int64_t *)(st->d_res_mant + Q);
      st->d_res_flags = (uint32_t *)(st->d_res_exp + Q);
      CUDA_TRY(cudaMallocHost(&st->h_res_mant, res_bytes));
      st->h_res_exp = (int64_t *)(st->h_res_mant + Q);
      st->h_res_flags = (uint32_t *)(st->h_res_exp + Q);
      if (kStageWeightBytes > 0)
        CUDA_TRY(cudaMallocHost(&st->h_stage, kStageIoBytes + kStageWeightBytes));
    }
  }
  IoDesc *h_io = st->h_stage ? (IoDesc *)st->h_stage : nullptr;
  double *h_w = st->h_stage ? (double *)(st->h_stage + kStageIoBytes) : nullptr;
  const size_t w_bytes = sizeof(double) * 2 * (size_t)Q * nv;  // w_pos then w_neg
  bool unit = true, negative = false;
  if (nv) {
    double *d_wp = st->d_w, *d_wn = st->d_w + (size_t)Q * nv;
    if (w_pos_q && h_w && w_bytes <= kStageWeightBytes) {  // small: one copy from pinned staging
      std::memcpy(h_w, w_pos_q, w_bytes / 2);
      std::memcpy(h_w + (size_t)Q * nv, w_neg_q, w_bytes / 2);
      CUDA_TRY(cudaMemcpyAsync(d_wp, h_w, w_bytes, cudaMemcpyHostToDevice, s));
    } else if (w_pos_q) {
      CUDA_TRY(cudaMemcpyAsync(d_wp, w_pos_q, sizeof(double) * (size_t)Q * nv, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(d_wn, w_neg_q, sizeof(double) * (size_t)Q * nv, cudaMemcpyHostToDevice, s));
    }
    if (w_pos_q) {
      for (size_t i = 0; i < (size_t)Q * nv; ++i) {
        unit &= (w_pos_q[i] == 1.0) & (w_neg_q[i] == 1.0);
        negative |= (w_pos_q[i] < 0.0) | (w_neg_q[i] < 0.0);
      }
    } else {
      for (int32_t q = 0; q < Q; ++q) {
        CUDA_TRY(cudaMemcpyAsync(d_wp + (size_t)q * nv, plan->w_pos.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_wn + (size_t)q * nv, plan->w_neg.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, s));
      }
      unit = plan->unit_weights;
      negative = plan->any_negative;
    }
  }
  rc = run_device(*plan, *st, st->d_w, st->d_w + (size_t)Q * nv, (char *)st->own_ws,
                  st->d_res_mant, st->d_res_exp, st->d_res_flags, s, slice_lo, slice_hi, lanes_per_slice, n_lanes,
                  h_io);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(st->h_res_mant, st->d_res_mant, 20 * (size_t)Q, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));  // (also frees the staging for the next call)
  for (int32_t q = 0; q < Q; ++q)
    if (st->h_res_flags[q] & WMC_FLAG_DEVICE_TIMEOUT) {
      set_error("a bounded wait inside a contraction kernel timed out; results discarded");
      return WMC_ETIMEOUT;
    }
  for (int32_t q = 0; q < Q; ++q)
    fill_result(*st, st->h_res_mant[q], st->h_res_exp[q], st->h_res_flags[q], unit, negative, out + q);
  return WMC_OK;
}

// Index slicing with the slice assignments along the lanes, as queries are
// batched: lane c Q + q is query q under slice lo + c, so one walk of
// Q x C lanes evaluates C slices of every query (the clause tensors with
// sliced literals carry the lanes; every other tensor does already).  Each
// query's partial counts are then summed exponent-aligned (Thm 4.2, as
// wmc_combine_results does).  C: the most slices whose lanes keep every
// tensor within 2^28 entries and at most 256 lanes; returns 1 (nothing
// done) when that is a single slice.
static int execute_slice_lanes(wmc_plan_t *plan, int32_t Q, const double *w_pos_q, const double *w_neg_q,
                               int64_t slice_lo, int64_t slice_hi, void *stream, wmc_result *out) {
  int mq = 0;
  while ((1 << mq) < Q) ++mq;
  const int m_max = std::min(8, std::max(0, 28 - plan->max_rank));
  const int64_t C = std::min<int64_t>(int64_t(1) << std::max(0, m_max - mq), slice_hi - slice_lo);
  if (C < 2) return 1;
  const int32_t Qe = (int32_t)(Q * C);
  ExecState *st = nullptr;
  int rc = get_state(*plan, Qe, &st);
  if (rc) return rc;
  const size_t nv = (size_t)plan->n_vars;
  std::vector<double> wp((size_t)Qe * std::max<size_t>(nv, 1)), wn(wp.size());
  for (int64_t c = 0; c < C; ++c)
    for (int32_t q = 0; q < Q; ++q) {
      const size_t d = ((size_t)c * (size_t)Q + (size_t)q) * nv;
      for (size_t v = 0; v < nv; ++v) {
        wp[d + v] = w_pos_q ? w_pos_q[(size_t)q * nv + v] : plan->w_pos[v];
        wn[d + v] = w_neg_q ? w_neg_q[(size_t)q * nv + v] : plan->w_neg[v];
      }
    }
  std::vector<std::vector<wmc_result>> parts((size_t)Q);
  std::vector<wmc_result> lane_out((size_t)Qe);
  for (int64_t b = slice_lo; b < slice_hi; b += C) {
    const int64_t cnt = std::min<int64_t>(C, slice_hi - b);
    if ((rc = run_host(plan, st, Qe, wp.data(), wn.data(), b, b + 1, stream, lane_out.data(), Q,
                       (int32_t)(Q * cnt))))
      return rc;
    for (int64_t c = 0; c < cnt; ++c)
      for (int32_t q = 0; q < Q; ++q) parts[(size_t)q].push_back(lane_out[(size_t)(c * Q + q)]);
  }
  for (int32_t q = 0; q < Q; ++q)
    if ((rc = wmc_combine_results(parts[(size_t)q].data(), (int64_t)parts[(size_t)q].size(), out + q))) return rc;
  return WMC_OK;
}

static int execute_host(wmc_plan_t *plan, int32_t Q, const double *w_pos_q, const double *w_neg_q,
                        int64_t slice_lo, int64_t slice_hi, void *stream, wmc_result *out) {
  if (!plan || !out) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  if ((w_pos_q == nullptr) != (w_neg_q == nullptr)) { set_error("give both weight arrays or neither"); return WMC_EINVAL; }
  int rc = 1;
  if (!plan->slice_vars.empty() && slice_hi - slice_lo > 1)
    rc = execute_slice_lanes(plan, Q, w_pos_q, w_neg_q, slice_lo, slice_hi, stream, out);
  if (rc == 1) {  // one walk per slice
    ExecState *st = nullptr;
    if ((rc = get_state(*plan, Q, &st))) return rc;
    rc = run_host(plan, st, Q, w_pos_q, w_neg_q, slice_lo, slice_hi, stream, out);
  }
  if (rc || plan->precision == WMC_FP64 || !g_fp64_fallback.load()) return rc;
  // queries whose float32 walk may have flushed run again in float64
  std::vector<int32_t> redo;
  for (int32_t q = 0; q < Q; ++q)
    if (out[q].flags & WMC_FLAG_FP32_FLUSH) redo.push_back(q);
  if (redo.empty()) return WMC_OK;
  const int32_t R = (int32_t)redo.size();
  const size_t nv = (size_t)plan->n_vars;
  std::vector<double> wp, wn;
  if (w_pos_q) {
    wp.resize((size_t)R * nv);
    wn.resize((size_t)R * nv);
    for (int32_t i = 0; i < R; ++i) {
      std::memcpy(wp.data() + (size_t)i * nv, w_pos_q + (size_t)redo[(size_t)i] * nv, sizeof(double) * nv);
      std::memcpy(wn.data() + (size_t)i * nv, w_neg_q + (size_t)redo[(size_t)i] * nv, sizeof(double) * nv);
    }
  }
  ExecState *st64 = nullptr;
  if ((rc = get_state(*plan, R, &st64, false, true))) return rc;
  std::vector<wmc_result> r64((size_t)R);
  rc = run_host(plan, st64, R, w_pos_q ? wp.data() : nullptr, w_neg_q ? wn.data() : nullptr, slice_lo, slice_hi,
                stream, r64.data());
  if (rc) return rc;
  for (int32_t i = 0; i < R; ++i) {
    out[redo[(size_t)i]] = r64[(size_t)i];
    out[redo[(size_t)i]].flags |= WMC_FLAG_FELL_BACK_FP64;
  }
  return WMC_OK;
}

namespace wmc {
int exec_layout(Plan &plan, int32_t Q, LayoutView *out) {
  ExecState *st = nullptr;
  int rc = get_state(plan, Q, &st, true);
  if (rc) return rc;
  out->ws_bytes = st->ws_bytes;
  out->off_io = st->off_io;
  out->off_flags = st->off_flags;
  out->off_err = st->off_err;
  out->off_exp = st->off_exp;
  out->off_max = st->off_max;
  out->off_min = st->off_min;
  out->n_slots = st->n_slots;
  out->arena0 = st->ws_bytes - align_up(st->arena_bytes);
  out->t_off = &st->t_off;
  out->t_meta = &st->t_meta;
  out->t_bytes = &st->t_bytes;
  out->t_dbl = &st->t_dbl;
  return WMC_OK;
}
void k1_bitmaps(const std::vector<int32_t> &LA, const std::vector<int32_t> &LB,
                const std::vector<int32_t> &LC, int32_t *rC, int32_t *k, int8_t *posA,
                int8_t *posB, int8_t *sposA, int8_t *sposB) {
  K1Params p;
  fill_k1(LA, LB, LC, p);
  *rC = p.rC;
  *k = p.k;
  std::memcpy(posA, p.posA, 32);
  std::memcpy(posB, p.posB, 32);
  std::memcpy(sposA, p.sposA, 24);
  std::memcpy(sposB, p.sposB, 24);
}
void count_launches(int64_t n) { g_launches.fetch_add(n); }
int device_alloc(void **p, size_t bytes) { return dev_alloc(p, bytes); }
int exec_state(Plan &plan, int32_t Q, ExecState **out) {
  if (check_q(Q)) return WMC_EINVAL;
  return get_state(plan, Q, out);
}
int64_t exec_ws_bytes(const ExecState *st) { return st->ws_bytes; }
int exec_prepare(Plan &plan, ExecState *st, void *ws) {
  int rc = ensure_dev(*st);
  if (rc) return rc;
  cudaGraphExec_t ge = nullptr;
  std::lock_guard<std::mutex> lk(st->graph_mu);
  return get_graph(plan, *st, (char *)ws, &ge);
}
int exec_run_device(Plan &plan, ExecState *st, const double *d_w_pos, const double *d_w_neg,
                    void *ws, double *d_mant, int64_t *d_exp2, uint32_t *d_flags, void *stream) {
  return run_device(plan, *st, d_w_pos, d_w_neg, (char *)ws, d_mant, d_exp2, d_flags,
                    (cudaStream_t)stream);
}
void exec_fill_result(const ExecState *st, double mant, int64_t exp2, uint32_t flags, bool unit,
                      bool negative, wmc_result *out) {
  fill_result(*st, mant, exp2, flags, unit, negative, out);
}
Plan &plan_of(wmc_plan_t *p) { return *p; }
}  // namespace wmc

// ------------------------------------------------------------ pairwise

namespace {
int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 148;
  return n;
}

// Stream-ordered scratch of pair contractions: a memory pool of the
// library's own per device that keeps up to 8 GiB cached across
// synchronisations (the default pool returns its memory at every one).
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it == pools.end()) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = 8ull << 30;
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
      pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// Packs one K4 operand for k4_tc: rows = its free bits (i of A, j of B).
dev::TcPackParams tc_pack_params(const void *x, float *xp, const dev::Meta &m, const dev::OutMeta &mc,
                                 const dev::K4Params &p4, bool is_a, int rows_log2) {
  dev::TcPackParams q;
  std::memset(&q, 0, sizeof(q));
  q.X = (const float *)x;
  q.Xp = xp;
  q.m = m;
  q.scale_inputs = mc.scale_inputs;
  q.rows_log2 = rows_log2;
  q.nr = is_a ? p4.ni : p4.nj;
  q.ns = p4.ns;
  q.nb = p4.nb;
  std::memcpy(q.r_pos, is_a ? p4.iA : p4.jB, 32);
  std::memcpy(q.s_pos, is_a ? p4.sA : p4.sB, 32);
  std::memcpy(q.b_pos, is_a ? p4.bA : p4.bB, 32);
  std::memcpy(q.bC, p4.bC, 32);
  q.Qc = mc.Qc;
  q.row_fast = is_a ? p4.a_i_fast : p4.b_j_fast;
  return q;
}

template <int N>
cudaError_t launch_k4_tc_n(const dev::K4Params &p4, const float *ap, const float *bp, cudaStream_t s) {
  static bool attr = false;  // opt in to the large dynamic shared memory once
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(dev::k4_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dev::TcShape<N>::smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nlog = N == 256 ? 8 : 7;
  const uint64_t tiles = ((uint64_t)1 << (p4.ni - 7 + p4.nj - nlog)) << p4.nb;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)num_sms());
  dev::k4_tc<N><<<grid, dev::kTcThreads, dev::TcShape<N>::smem, s>>>(p4, ap, bp, nullptr);
  return cudaGetLastError();
}

// C = A.B on the tensor cores: both operands packed (scaled, split into
// TF32 hi and lo) into stream-ordered scratch, then the persistent product.
cudaError_t launch_k4_tc(const dev::K4Params &p4, cudaStream_t s) {
  const int nlog = p4.nj >= 8 ? 8 : 7;
  const size_t a_elems = (size_t)1 << (p4.ni + p4.ns + p4.nb), b_elems = (size_t)1 << (p4.nj + p4.ns + p4.nb);
  float *scratch = nullptr;
  cudaError_t e = scratch_alloc((void **)&scratch, (a_elems + b_elems) * 2 * sizeof(float), s);
  if (e != cudaSuccess) return e;
  float *ap = scratch, *bp = scratch + 2 * a_elems;
  const dev::TcPackParams pa = tc_pack_params(p4.A, ap, p4.ma, p4.mc, p4, true, 7);
  const dev::TcPackParams pb = tc_pack_params(p4.B, bp, p4.mb, p4.mc, p4, false, nlog);
  dev::k4_tc_pack<<<(unsigned)(a_elems / (128 * dev::kTcKC)), 256, 0, s>>>(pa);
  dev::k4_tc_pack<<<(unsigned)(b_elems / ((size_t)(1 << nlog) * dev::kTcKC)), 256, 0, s>>>(pb);
  g_launches.fetch_add(3);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = nlog == 8 ? launch_k4_tc_n<256>(p4, ap, bp, s) : launch_k4_tc_n<128>(p4, ap, bp, s);
  const cudaError_t f = cudaFreeAsync(scratch, s);
  return e != cudaSuccess ? e : f;
}
}  // namespace


// ------------------------------------------------- pairwise contraction
//
// wmc_contract_pair picks one of several kernels for a node.  The fixed
// rule (pair_default) follows the node's shape; with autotuning on
// (wmc_set_autotune), the first call of each shape times every legal
// variant that adds the summed terms in the canonical order (so all give
// the same bits: k1_generic, the streaming kernels at several block counts,
// the TMA-staged streaming kernel at 1..3 blocks per SM, the tiled and the
// outer-product dense kernels) on the call's own buffers and keeps the
// fastest for later calls of that shape.  Variants with another order (the
// tensor-core product, the split summed range) are never swapped in or out.

namespace {

enum PairKind { PK_K1 = 0, PK_K2 = 1, PK_K2T = 2, PK_K4D = 3, PK_K4O = 4, PK_K4TC = 5, PK_K4SPLIT = 6, PK_K2Q = 7 };

struct PairChoice {
  int kind = PK_K1;
  int64_t blocks = 0;  // 0: the kernel's own block count
};

struct PairSetup {
  bool f64 = false;
  const void *a = nullptr, *b = nullptr;
  void *c = nullptr;
  const int64_t *exp_a = nullptr, *exp_b = nullptr;
  int64_t *exp_c = nullptr;
  std::vector<int32_t> LA, LB, LC;
  // streaming form: P (the larger operand, else the other) keeps its order
  bool k2 = false, use_a = true;
  K2Params p2;
  int vmax = 1, kmax = 1, fmax = 1;
  bool quad = false;  // k2_stream_s16q applies (four units per thread)
  bool k2t = false;
  wmc::dev::K2TParams k2tp;
  size_t k2t_smem = 0;
  int k2t_per_sm = 1;
  uint64_t k2t_tiles = 0;
  // dense form
  bool k4 = false;
  wmc::dev::K4Params p4;
  int64_t outer_blocks = 0;
  int split_g = 0;
  int32_t k1_k = 0;
};

void pair_setup(PairSetup &ps) {
  const bool a_first = ps.LA.size() >= ps.LB.size();
  for (int attempt = 0; attempt < 2 && !ps.k2; ++attempt) {
    ps.use_a = (attempt == 0) == a_first;
    ps.k2 = try_k2(ps.use_a ? ps.LA : ps.LB, ps.use_a ? ps.LB : ps.LA, ps.LC, ps.f64, ps.p2, ps.vmax, ps.kmax,
                   ps.fmax);
  }
  dev::Meta ma{ps.exp_a, nullptr, nullptr, 0}, mb{ps.exp_b, nullptr, nullptr, 0};
  dev::OutMeta mc{ps.exp_c, nullptr, nullptr, nullptr, 1, 1, 0};
  if (ps.k2) {
    ps.p2.A = ps.use_a ? ps.a : ps.b; ps.p2.B = ps.use_a ? ps.b : ps.a; ps.p2.C = ps.c;
    ps.p2.ma = ps.use_a ? ma : mb; ps.p2.mb = ps.use_a ? mb : ma; ps.p2.mc = mc;
    ps.k2t = try_k2_tma(ps.p2, ps.use_a ? ps.LA : ps.LB, ps.use_a ? ps.LB : ps.LA, ps.f64, false, false, 1,
                        ps.k2tp, ps.k2t_smem);
    // four units per thread: float32 with S staged, the units' two lowest
    // bits P's and C's two lowest bits, S independent of them
    {
      const K2Params &q = ps.p2;
      bool ok = !ps.f64 && q.s_staged && q.vbits == 0 && q.log2_nu >= 2 && q.f >= 1;
      for (int i = 0; i < q.n_insA && ok; ++i) ok = q.insA[i] >= 2;
      for (int i = 0; i < q.n_insC && ok; ++i) ok = q.insC[i] >= 2;
      for (int i = 0; i < q.n_seg && ok; ++i) ok = q.seg_c[i] >= 2;
      ps.quad = ok && ((uintptr_t)ps.c & 15u) == 0 && (((uintptr_t)ps.p2.A) & 15u) == 0;
    }
    if (ps.k2t) {
      ps.k2t_tiles = 1ull << (ps.p2.log2_nu + ps.p2.vbits - ps.k2tp.tb);
      const int kf = ps.p2.k + ps.p2.f;
      const int per_sm_regs = kf <= 2 ? 3 : (kf <= 4 ? 2 : 1);
      ps.k2t_per_sm = std::min(per_sm_regs, ps.k2t_smem <= 72 * 1024 ? 3 : (ps.k2t_smem <= 108 * 1024 ? 2 : 1));
      ps.k2tp.k = ps.p2;
      ps.k2tp.err = nullptr;
    }
  }
  ps.k4 = try_k4(ps.LA, ps.LB, ps.LC, ps.f64, ps.p4);
  if (ps.k4) {
    ps.p4.A = ps.a; ps.p4.B = ps.b; ps.p4.C = ps.c; ps.p4.ma = ma; ps.p4.mb = mb; ps.p4.mc = mc;
    if (((uintptr_t)ps.c & 15u) == 0) ps.outer_blocks = k4_outer_pick(ps.p4);
    const unsigned tiles = 1u << (ps.p4.ni - 6 + ps.p4.nj - 6 + ps.p4.nb);
    int g = 0;
    while (ps.p4.ns - 8 - g > 0 && (tiles << g) < 2 * 148 && g < 9) ++g;
    if (ps.p4.ns <= 8) g = 0;
    ps.split_g = g;
  }
  K1Params k1;
  fill_k1(ps.LA, ps.LB, ps.LC, k1);
  ps.k1_k = k1.k;
}

PairChoice pair_default(const PairSetup &ps) {
  PairChoice ch;
  if (!ps.k2 && ps.k4) {
    if (!ps.f64 && g_tensor_cores.load() && ps.p4.ni >= 7 && ps.p4.nj >= 7 && ps.p4.ns >= 4) ch.kind = PK_K4TC;
    else if (g_outer.load() && ps.outer_blocks) ch.kind = PK_K4O;
    else ch.kind = ps.split_g ? PK_K4SPLIT : PK_K4D;
  } else if (ps.k2) {
    ch.kind = ps.k2t ? PK_K2T : (ps.quad ? PK_K2Q : PK_K2);
  } else {
    ch.kind = PK_K1;
  }
  return ch;
}

bool pair_canonical(const PairChoice &ch) { return ch.kind != PK_K4TC && ch.kind != PK_K4SPLIT; }

int pair_enqueue(PairSetup &ps, const PairChoice &ch, cudaStream_t s) {
  const bool f64 = ps.f64;
  switch (ch.kind) {
    case PK_K4TC:
      CUDA_TRY(launch_k4_tc(ps.p4, s));
      return WMC_OK;
    case PK_K4O: {
      const unsigned ob = (unsigned)ps.outer_blocks;
      const int ns = ps.p4.ns;  // at most 2 summed bits (k4_outer_pick)
      if (f64) {
        if (ns == 0) dev::k4_outer<double, 1><<<ob, 256, 0, s>>>(ps.p4);
        else if (ns == 1) dev::k4_outer<double, 2><<<ob, 256, 0, s>>>(ps.p4);
        else dev::k4_outer<double, 4><<<ob, 256, 0, s>>>(ps.p4);
      } else {
        if (ns == 0) dev::k4_outer<float, 1><<<ob, 256, 0, s>>>(ps.p4);
        else if (ns == 1) dev::k4_outer<float, 2><<<ob, 256, 0, s>>>(ps.p4);
        else dev::k4_outer<float, 4><<<ob, 256, 0, s>>>(ps.p4);
      }
      g_launches.fetch_add(1);
      break;
    }
    case PK_K4D:
    case PK_K4SPLIT: {
      dev::K4Params p4 = ps.p4;
      const unsigned tiles = 1u << (p4.ni - 6 + p4.nj - 6 + p4.nb);
      const int g = ch.kind == PK_K4SPLIT ? ps.split_g : 0;
      // a long summed range over few output tiles: split into groups of
      // whole 256-term blocks, each group's partials in stream-ordered
      // scratch, then the groups added in order
      p4.groups_log2 = g;
      void *scratch = nullptr;
      if (g) {
        const size_t bytes = ((size_t)tiles << g) * 4096 * (f64 ? 8 : 4);
        CUDA_TRY(scratch_alloc(&scratch, bytes, s));
        p4.partial = scratch;
      }
      if (f64) dev::k4_dense<double><<<tiles << g, 256, 0, s>>>(p4);
      else dev::k4_dense<float><<<tiles << g, 256, 0, s>>>(p4);
      g_launches.fetch_add(1);
      if (g) {
        if (f64) dev::k4_reduce<double><<<tiles * 16, 256, 0, s>>>(p4);
        else dev::k4_reduce<float><<<tiles * 16, 256, 0, s>>>(p4);
        g_launches.fetch_add(1);
        CUDA_TRY(cudaFreeAsync(scratch, s));
      }
      break;
    }
    case PK_K2T: {
      Launch l;
      l.kind = L_K2T; l.ti = f64 ? TD : TF; l.v = ps.vmax; l.kmax = ps.kmax; l.fmax = ps.fmax;
      l.smem = ps.k2t_smem;
      const int per_sm = ch.blocks > 0 ? (int)ch.blocks : ps.k2t_per_sm;
      l.blocks = (int64_t)std::min<uint64_t>(ps.k2t_tiles, (uint64_t)(148 * per_sm));
      l.k2t = ps.k2tp;
      launch_k2t(l, l.k2t, s);
      g_launches.fetch_add(1);
      break;
    }
    case PK_K2Q: {
      const uint64_t nq = 1ull << (ps.p2.log2_nu - 2);
      const int64_t dflt = std::min<int64_t>((int64_t)((nq + dev::kThreads - 1) / dev::kThreads), 148 * 2);
      const unsigned blocks = (unsigned)(ch.blocks > 0 ? std::min<int64_t>(dflt, ch.blocks) : dflt);
      const size_t smem = sizeof(float) << ps.p2.s_log2;
      if (ps.p2.s_contig) dev::k2_stream_s16q<true><<<blocks, dev::kThreads, smem, s>>>(ps.p2);
      else dev::k2_stream_s16q<false><<<blocks, dev::kThreads, smem, s>>>(ps.p2);
      g_launches.fetch_add(1);
      break;
    }
    case PK_K2: {
      Launch l;
      l.kind = L_K2; l.ti = f64 ? TD : TF; l.v = ps.vmax; l.kmax = ps.kmax; l.fmax = ps.fmax;
      const int64_t dflt = grid_for(1ull << ps.p2.log2_nu);
      l.blocks = ch.blocks > 0 ? std::min<int64_t>(dflt, ch.blocks) : dflt;
      launch_k2(l, ps.p2, s);
      g_launches.fetch_add(1);
      break;
    }
    default: {
      Launch l;
      l.kind = L_K1;
      fill_k1(ps.LA, ps.LB, ps.LC, l.k1);
      if (l.k1.k > 24) { set_error("at most 24 summed indices"); return WMC_EINVAL; }
      l.ti = f64 ? TD : TF;
      l.ta = (f64 || l.k1.k > 16) ? TD : TF;
      l.to = f64 ? TD : TF;
      l.blocks = grid_for(1ull << l.k1.rC);
      l.k1.A = ps.a; l.k1.B = ps.b; l.k1.C = ps.c;
      l.k1.ma = dev::Meta{ps.exp_a, nullptr, nullptr, 0};
      l.k1.mb = dev::Meta{ps.exp_b, nullptr, nullptr, 0};
      l.k1.mc = dev::OutMeta{ps.exp_c, nullptr, nullptr, nullptr, 1, 1, 0};
      launch_k1(l, l.k1, s);
      g_launches.fetch_add(1);
      break;
    }
  }
  CUDA_TRY(cudaGetLastError());
  return WMC_OK;
}

// the legal same-order variants of a node, the fixed rule's first
std::vector<PairChoice> pair_candidates(const PairSetup &ps, const PairChoice &dflt) {
  std::vector<PairChoice> v{dflt};
  auto add = [&](int kind, int64_t blocks) {
    for (const PairChoice &c : v)
      if (c.kind == kind && c.blocks == blocks) return;
    v.push_back(PairChoice{kind, blocks});
  };
  if (ps.k2) {
    if (ps.quad) { add(PK_K2Q, 0); add(PK_K2Q, 148); }
    add(PK_K2, 0);
    const int64_t g = grid_for(1ull << ps.p2.log2_nu);
    for (int64_t m : {2, 4, 8})
      if (148 * m < g) add(PK_K2, 148 * m);
    if (ps.k2t)
      for (int per_sm = 1; per_sm <= ps.k2t_per_sm; ++per_sm)
        if (!(dflt.kind == PK_K2T && dflt.blocks == 0 && per_sm == ps.k2t_per_sm)) add(PK_K2T, per_sm);
  }
  if (ps.k4 && ps.split_g == 0) {
    add(PK_K4D, 0);
    if (ps.outer_blocks) add(PK_K4O, 0);
  }
  if (ps.k1_k <= 24) add(PK_K1, 0);
  return v;
}

std::mutex g_tune_mu;
std::map<std::string, PairChoice> g_tune_cache;

std::string pair_key(const PairSetup &ps, int precision) {
  std::string k = std::to_string(precision) + ":" + std::to_string(((uintptr_t)ps.c & 15u) == 0) + ":";
  for (const auto *L : {&ps.LA, &ps.LB, &ps.LC}) {
    for (int32_t x : *L) k += std::to_string(x) + ",";
    k += "|";
  }
  return k;
}

// The tuned choice for this node's shape: cached, or measured now on the
// call's own buffers (each variant once to warm, then three timed runs;
// the fastest minimum wins).  Synchronises the stream while measuring.
int pair_tuned(PairSetup &ps, int precision, PairChoice &ch, cudaStream_t s) {
  const std::string key = pair_key(ps, precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) { ch = it->second; return WMC_OK; }
  }
  const std::vector<PairChoice> cands = pair_candidates(ps, ch);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 0.0f;
  PairChoice pick = ch;
  for (size_t i = 0; i < cands.size(); ++i) {
    int rc = pair_enqueue(ps, cands[i], s);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    float t_min = 0.0f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, s);
      rc = pair_enqueue(ps, cands[i], s);
      cudaEventRecord(e1, s);
      if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0); cudaEventDestroy(e1);
        if (!rc) set_error("timing a variant failed: %s", cudaGetErrorString(cudaGetLastError()));
        return rc ? rc : WMC_ECUDA;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      t_min = r == 0 ? ms : std::min(t_min, ms);
    }
    if (i == 0 || t_min < best) { best = t_min; pick = cands[i]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = pick;
  ch = pick;
  return WMC_OK;
}

}  // namespace

extern "C" void wmc_set_autotune(int32_t on) { g_autotune.store(on ? 1 : 0); }

extern "C" int wmc_pair_variants(int32_t precision, int32_t rank_a, const int32_t *labels_a, int32_t rank_b,
                                 const int32_t *labels_b, int32_t rank_c, const int32_t *labels_c,
                                 int32_t c_aligned16, int32_t max_n, int32_t *kinds, int64_t *blocks,
                                 int32_t *n, int32_t *chosen) {
  if (!n || !chosen || max_n < 0 || (max_n && (!kinds || !blocks)) || rank_a < 0 || rank_b < 0 || rank_c < 0 ||
      rank_a > 31 || rank_b > 31 || rank_c > 31 || (rank_a && !labels_a) || (rank_b && !labels_b) ||
      (rank_c && !labels_c)) {
    set_error("bad argument");
    return WMC_EINVAL;
  }
  PairSetup ps;
  ps.f64 = precision == WMC_FP64;
  ps.c = c_aligned16 ? (void *)(uintptr_t)256 : (void *)(uintptr_t)4;  // only its alignment is read
  ps.LA.assign(labels_a, labels_a + rank_a);
  ps.LB.assign(labels_b, labels_b + rank_b);
  ps.LC.assign(labels_c, labels_c + rank_c);
  pair_setup(ps);
  const PairChoice dflt = pair_default(ps);
  PairChoice cur = dflt;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(pair_key(ps, precision));
    if (g_autotune.load() && it != g_tune_cache.end()) cur = it->second;
  }
  const std::vector<PairChoice> v = pair_canonical(dflt) ? pair_candidates(ps, dflt) : std::vector<PairChoice>{dflt};
  *n = (int32_t)v.size();
  *chosen = 0;
  for (size_t i = 0; i < v.size(); ++i) {
    if (v[i].kind == cur.kind && v[i].blocks == cur.blocks) *chosen = (int32_t)i;
    if ((int32_t)i < max_n) { kinds[i] = v[i].kind; blocks[i] = v[i].blocks; }
  }
  return WMC_OK;
}

extern "C" void wmc_debug_force_pair_variant(int32_t kind, int64_t blocks) {
  g_force_kind.store(kind);
  g_force_blocks.store(blocks);
}

extern "C" int wmc_contract_pair(int32_t precision, int32_t rank_a, const int32_t *labels_a,
                                 const void *a, int32_t rank_b, const int32_t *labels_b,
                                 const void *b, int32_t rank_c, const int32_t *labels_c, void *c,
                                 const int64_t *exp_a, const int64_t *exp_b, int64_t *exp_c,
                                 void *stream) {
  if (precision != WMC_FP64 && precision != WMC_SCALED_FP32) { set_error("bad precision"); return WMC_EINVAL; }
  if (rank_a < 0 || rank_b < 0 || rank_c < 0 || rank_a > 31 || rank_b > 31 || rank_c > 31) {
    set_error("ranks must be in [0, 31]");
    return WMC_EINVAL;
  }
  if (!a || !b || !c || (rank_a && !labels_a) || (rank_b && !labels_b) || (rank_c && !labels_c)) {
    set_error("NULL argument");
    return WMC_EINVAL;
  }
  const bool f64 = precision == WMC_FP64;
  if (!f64 && (!exp_a || !exp_b || !exp_c)) { set_error("scaled FP32 needs exp_a, exp_b, exp_c"); return WMC_EINVAL; }
  std::vector<int32_t> LA(labels_a, labels_a + rank_a), LB(labels_b, labels_b + rank_b),
      LC(labels_c, labels_c + rank_c);
  auto dup = [](std::vector<int32_t> L) {
    std::sort(L.begin(), L.end());
    return std::adjacent_find(L.begin(), L.end()) != L.end();
  };
  if (dup(LA) || dup(LB) || dup(LC)) { set_error("repeated label within a tensor"); return WMC_EINVAL; }
  for (int32_t l : LC)
    if (pos_of(LA, l) < 0 && pos_of(LB, l) < 0) { set_error("label %d of C is in neither A nor B", l); return WMC_EINVAL; }
  PairSetup ps;
  ps.f64 = f64; ps.a = a; ps.b = b; ps.c = c;
  ps.exp_a = exp_a; ps.exp_b = exp_b; ps.exp_c = exp_c;
  ps.LA = LA; ps.LB = LB; ps.LC = LC;
  pair_setup(ps);
  if (ps.k1_k > 24 && !ps.k2 && !ps.k4) { set_error("at most 24 summed indices"); return WMC_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  PairChoice ch = pair_default(ps);
  if (g_force_kind.load() >= 0) {  // test hook: one listed variant
    const std::vector<PairChoice> v = pair_canonical(ch) ? pair_candidates(ps, ch) : std::vector<PairChoice>{ch};
    bool found = false;
    for (const PairChoice &c : v)
      if (c.kind == g_force_kind.load() && c.blocks == g_force_blocks.load()) { ch = c; found = true; }
    if (!found) { set_error("the forced variant is not one of this node's variants"); return WMC_EINVAL; }
    return pair_enqueue(ps, ch, s);
  }
  if (g_autotune.load() && pair_canonical(ch)) {
    int rc = pair_tuned(ps, precision, ch, s);
    if (rc) return rc;
  }
  return pair_enqueue(ps, ch, s);
}

extern "C" int wmc_to_scaled_fp32(const double *x, int64_t n, float *out, int64_t *exp_out,
                                  void *stream) {
  if (!x || !out || !exp_out || n < 0) { set_error("bad argument"); return WMC_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  // the max is accumulated in exp_out's storage (8 bytes) before it is
  // overwritten by the exponent: no scratch allocation
  unsigned long long *maxb = (unsigned long long *)exp_out;
  CUDA_TRY(cudaMemsetAsync(maxb, 0, sizeof(unsigned long long), s));
  const unsigned g = (unsigned)grid_for((uint64_t)std::max<int64_t>(n, 1));
  dev::k_absmax_f64<<<g, dev::kThreads, 0, s>>>(x, n, maxb);
  dev::k_scale_to_f32<<<g, dev::kThreads, 0, s>>>(x, n, maxb, out);
  dev::k_max_to_exp<<<1, 1, 0, s>>>(maxb);
  g_launches.fetch_add(3);
  CUDA_TRY(cudaGetLastError());
  return WMC_OK;
}

// ------------------------------------------------- allocation-free variant
//
// Some callers cannot allocate device memory at the time they run a count:
// a library embedded in a host process whose device memory is entirely
// owned by another allocator (a framework's caching allocator, or a pool
// reserved up front), and code that must not call cudaMalloc/cudaFree once
// it is running (both can synchronise the device).  For them,
// wmc_execute_device_noalloc runs the same walk on a fixed scratch array
// that is part of this library's device image instead of on caller- or
// library-allocated memory.

// The scratch lives for as long as the library stays loaded, on every GPU
// that uses it.  Host code must not take its address directly (that is a
// host-side shadow); the device address comes from cudaGetSymbolAddress.
static constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256];         // device address of the scratch, per device
static uint64_t g_noalloc_tables[256];   // serial of the state whose tables it holds (0: none)

// Looked up once per device, by the first call on that device, with that
// device current.  A cudaDeviceReset of the device invalidates it (as it
// invalidates every plan's cached device state).
static int noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= 256) { set_error("device id %d out of range", dev); return WMC_EINVAL; }
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return WMC_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return WMC_OK;
}

// The call descriptor travels as a kernel argument (copied at launch), so
// nothing reads host memory after the call returns.
__global__ void k_store_io(IoDesc io, IoDesc *dst) { *dst = io; }

extern "C" int wmc_execute_device_noalloc(wmc_plan_t *plan, int32_t Q, const double *d_w_pos,
                                          const double *d_w_neg, double *d_mant, int64_t *d_exp2,
                                          uint32_t *d_flags, void *stream) {
  if (!plan || !d_mant || !d_exp2 || !d_flags) { set_error("NULL argument"); return WMC_EINVAL; }
  if (check_q(Q)) return WMC_EINVAL;
  if (plan->n_vars > 0 && (!d_w_pos || !d_w_neg)) { set_error("weights are NULL"); return WMC_EINVAL; }
  ExecState *st = nullptr;
  int rc = get_state(*plan, Q, &st);  // host-side layout only
  if (rc) return rc;
  // scratch layout: [leaf tables][workspace]
  const size_t b_clause = sizeof(ClauseLeaf) * st->h_clause.size();
  const size_t b_first = sizeof(int64_t) * st->h_first.size();
  const size_t b_woff = sizeof(int64_t) * st->h_woff.size();
  const size_t b_wmeta = sizeof(int64_t) * st->h_wmeta.size();
  const size_t b_sn = sizeof(wmc::dev::SNode) * st->h_snodes.size();
  const size_t b_stk = sizeof(wmc::dev::STask) * st->h_stasks.size();
  const size_t b_seq = sizeof(wmc::dev::K2CParams) * st->h_seq.size();
  const size_t b_cta = sizeof(wmc::dev::CtaLeaf) * st->h_cta.size();
  const size_t o_first = (size_t)align_up((int64_t)b_clause);
  const size_t o_woff = o_first + (size_t)align_up((int64_t)b_first);
  const size_t o_wmeta = o_woff + (size_t)align_up((int64_t)b_woff);
  const size_t o_sn = o_wmeta + (size_t)align_up((int64_t)b_wmeta);
  const size_t o_stk = o_sn + (size_t)align_up((int64_t)b_sn);
  const size_t o_seq = o_stk + (size_t)align_up((int64_t)b_stk);
  const size_t o_cta = o_seq + (size_t)align_up((int64_t)b_seq);
  const size_t o_ws = o_cta + (size_t)align_up((int64_t)b_cta);
  const size_t need = o_ws + (size_t)st->ws_bytes;
  if (need > kNoAllocScratchBytes) {
    set_error("this plan needs %zu bytes of scratch at Q = %d; the static scratch holds %zu",
              need, Q, kNoAllocScratchBytes);
    return WMC_EINVAL;
  }
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  char *base = nullptr;
  if ((rc = noalloc_scratch(dev, (void **)&base))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // The tables depend on the plan and Q alone and the walk never writes
  // them: they are copied only when the scratch holds another state's.
  if (g_noalloc_tables[dev] != st->serial) {
    g_noalloc_tables[dev] = 0;
    auto up = [&](size_t off, const void *src, size_t bytes) {
      return bytes ? cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    if (up(0, st->h_clause.data(), b_clause) || up(o_first, st->h_first.data(), b_first) ||
        up(o_woff, st->h_woff.data(), b_woff) || up(o_wmeta, st->h_wmeta.data(), b_wmeta) ||
        up(o_sn, st->h_snodes.data(), b_sn) || up(o_stk, st->h_stasks.data(), b_stk) ||
        up(o_seq, st->h_seq.data(), b_seq) || up(o_cta, st->h_cta.data(), b_cta)) {
      set_error("copying the leaf tables into the static scratch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
      return WMC_ECUDA;
    }
    g_noalloc_tables[dev] = st->serial;
  }
  char *ws = base + o_ws;
  IoDesc io = io_desc(*plan, d_w_pos, d_w_neg, d_mant, d_exp2, d_flags);
  const LeafTables tables{(const ClauseLeaf *)base, (const int64_t *)(base + o_first),
                          (const int64_t *)(base + o_woff), (const int64_t *)(base + o_wmeta),
                          (const wmc::dev::SNode *)(base + o_sn), (const wmc::dev::STask *)(base + o_stk),
                          (const wmc::dev::K2CParams *)(base + o_seq),
                          (const wmc::dev::CtaLeaf *)(base + o_cta)};
  // the walk's first launch zeroes the flags and metadata it accumulates
  // into; one walk per slice assignment (index slicing), the later ones
  // adding into the outputs
  for (int64_t eta = 0; eta < n_slices(*plan); ++eta) {
    io.slice = (uint64_t)eta;
    io.accumulate = eta != 0;
    k_store_io<<<1, 1, 0, s>>>(io, (IoDesc *)(ws + st->off_io));
    enqueue_walk(*plan, *st, ws, s, nullptr, &tables);
    g_launches.fetch_add(st->kernels_per_run + 1);
  }
  CUDA_TRY(cudaGetLastError());
  return WMC_OK;
}

// ------------------------------------------------------ host bounds check
//
// Replays, on the CPU, the index arithmetic of every contraction launch of
// the walk for batch size Q (every bulk copy of every tile, and the
// per-thread offsets of sampled work units including the first and last)
// and checks each access against the tensor it touches.  Used by the CPU
// test suite before kernels run on a GPU.
namespace {
inline uint32_t h_insert0(uint32_t x, int p) {
  uint32_t lo = x & ((1u << p) - 1u);
  return ((x >> p) << (p + 1)) | lo;
}
}  // namespace

extern "C" int wmc_debug_check_bounds(wmc_plan_t *plan, int32_t Q, int64_t *n_checked) {
  if (!plan) { set_error("NULL argument"); return WMC_EINVAL; }
  ExecState *st = nullptr;
  int rc = get_state(*plan, Q, &st);
  if (rc) return rc;
  int64_t checked = 0;
  // clause leaves: 2^(rank + lane bits) elements and 2^(lane bits) metadata
  // slots inside their tensor's allocation and slots
  for (size_t i = 0; i < st->h_clause.size(); ++i) {
    const ClauseLeaf &L = st->h_clause[i];
    const int64_t es = st->f64 ? 8 : 4;
    bool ok = false;
    for (size_t t = 0; t < st->t_off.size() && !ok; ++t)
      ok = st->t_off[t] == L.off * es && (int64_t(1) << (L.rank + L.lbits)) * es <= st->t_bytes[t] &&
           L.meta + (int64_t(1) << L.lbits) <= st->t_meta[t] + st->t_qc[t] && L.meta >= st->t_meta[t];
    if (!ok) { set_error("clause leaf %zu: elements or metadata slots outside its tensor", i); return WMC_EINVAL; }
    ++checked;
  }
  for (size_t i = 0; i < st->h_snodes.size(); ++i) {
    const wmc::dev::SNode &sn = st->h_snodes[i];
    int64_t ma = 0, mb = 0;
    for (int j = 0; j < sn.rC; ++j) {
      if (sn.posA[j] >= 0) ma |= 1ll << sn.posA[j];
      if (sn.posB[j] >= 0) mb |= 1ll << sn.posB[j];
    }
    for (int j = 0; j < sn.k; ++j) {
      if (sn.sposA[j] >= 0) ma |= 1ll << sn.sposA[j];
      if (sn.sposB[j] >= 0) mb |= 1ll << sn.sposB[j];
    }
    const int64_t esi = sn.ti ? 8 : 4, eso = sn.to ? 8 : 4;
    const bool cta = !st->h_cta.empty();
    const bool cta_root = cta && i + 1 == st->h_snodes.size();
    auto within = [&](int64_t off, int64_t last_elem, int64_t es, bool shared) {
      if (shared) {  // one-block walk: a tensor of the shared-memory arena
        const int64_t arena = st->cta_lut_off - st->cta_meta;  // (the level tables follow it)
        for (size_t t = 0; t < st->cta_off.size(); ++t)
          if (st->cta_off[t] == off && (last_elem + 1) * es <= st->t_bytes[t] && off + st->t_bytes[t] <= arena)
            return true;
        return false;
      }
      for (size_t t = 0; t < st->t_off.size(); ++t)
        if (st->t_off[t] == off && (last_elem + 1) * es <= st->t_bytes[t]) return true;
      return false;
    };
    if (!within(sn.a, ma, esi, cta) || !within(sn.b, mb, esi, cta) ||
        !within(sn.c, (1ll << sn.rC) - 1, eso, cta && !cta_root)) {
      set_error("small-phase node %zu: an offset leaves its tensor", i);
      return WMC_EINVAL;
    }
    if (sn.chunk_log2 > sn.rC || sn.k > 8 || sn.rC > 16) { set_error("small-phase node %zu: bad shape", i); return WMC_EINVAL; }
    ++checked;
  }
  // one-block walk: levels partition the node list, each level's tables
  // and outputs are laid out back to back, the tables fit their region
  if (!st->h_cta.empty()) {
    const size_t n = st->h_snodes.size();
    for (size_t i = 0; i < n;) {
      const size_t e = (size_t)st->h_snodes[i].level_end;
      if (e <= i || e > n) { set_error("one-block walk: level of node %zu ends at %zu", i, e); return WMC_EINVAL; }
      int64_t words = 0, outs = 0;
      for (size_t j = i; j < e; ++j) {
        const wmc::dev::SNode &sn = st->h_snodes[j];
        if (sn.lut_base != words || sn.out_base != outs || (size_t)sn.level_end != e) {
          set_error("one-block walk: node %zu's table or output offset", j);
          return WMC_EINVAL;
        }
        words += 2 * ((1 << std::min<int32_t>(sn.rC, 8)) + (1 << std::max<int32_t>(sn.rC - 8, 0)) + (1 << sn.k));
        outs += int64_t(1) << sn.rC;
      }
      if (words > st->cta_lut_words || st->cta_lut_off + 4 * words > st->cta_smem || outs > (int64_t(1) << 31)) {
        set_error("one-block walk: a level's tables (%lld words) exceed their region", (long long)words);
        return WMC_EINVAL;
      }
      i = e;
      ++checked;
    }
  }
  // weight leaves: every variable's table entry is its own leaf or -1
  {
    std::vector<uint8_t> has_leaf((size_t)plan->n_vars, 0);
    for (int64_t i = 0; i < plan->n_leaves; ++i) {
      const TensorInfo &t = plan->tensors[(size_t)i];
      if (t.kind != LEAF_WEIGHT) continue;
      const size_t v = (size_t)t.labels[0];
      has_leaf[v] = 1;
      const int64_t es = st->f64 ? 8 : 4;
      if (st->h_woff[v] * es != st->t_off[(size_t)i] || 2 * st->Qp * es > st->t_bytes[(size_t)i]) {
        set_error("weight leaf of variable %zu: table offset outside its tensor", v);
        return WMC_EINVAL;
      }
    }
    for (size_t v = 0; v < (size_t)plan->n_vars; ++v)
      if (!has_leaf[v] && (st->h_woff[v] != -1 || st->h_wmeta[v] != -1)) {
        set_error("variable %zu has no weight leaf but a table entry", v);
        return WMC_EINVAL;
      }
    ++checked;
  }
  size_t li = 0;
  std::vector<const Launch *> flat;  // runs of chains checked chain by chain
  for (const Launch &l : st->launches) {
    if (l.kind != L_K2CSEQ) { flat.push_back(&l); continue; }
    if (l.seq_ctr_off + 8 * (int64_t)l.chains.size() > st->off_seqctr + 8 * (int64_t)plan->nodes.size() ||
        l.seq_first + (int64_t)l.chains.size() > (int64_t)st->h_seq.size() || l.smem > 220 * 1024 ||
        l.blocks < 1 || l.blocks > 148) {
      set_error("run of chains: counters, parameter table, shared memory or grid out of range");
      return WMC_EINVAL;
    }
    for (const Launch &c : l.chains) flat.push_back(&c);
  }
  for (const Launch *lp : flat) {
    const Launch &l = *lp;
    ++li;
    // k4 offsets are bit scatters onto each tensor's own positions: in
    // bounds by construction
    if (l.kind == L_K2C) {
      const wmc::dev::K2CParams &cp = l.k2c;
      const int64_t es = l.ti == TD ? 8 : 4;
      const int V = 1 << cp.vbits, D = l.chain_d;
      const int64_t np = st->t_bytes[(size_t)l.id_a] / es, nc = st->t_bytes[(size_t)l.id_c] / es;
      auto badc = [&](const char *what, int64_t o, int64_t n) {
        set_error("launch %zu: chain %s offset %lld outside [0, %lld)", li, what, (long long)o, (long long)n);
        return WMC_EINVAL;
      };
      for (int i = 0; i < D; ++i)
        if (l.id_sc[i] < 0 || st->t_bytes[(size_t)l.id_sc[i]] != (int64_t)es << cp.s_log2[i])
          return badc("S size", i, D);
      const uint64_t nu = 1ull << cp.log2_nu;
      std::vector<uint64_t> us;
      if (nu <= (1u << 14)) for (uint64_t u = 0; u < nu; ++u) us.push_back(u);
      else {
        for (uint64_t u = 0; u < 4096; ++u) { us.push_back(u); us.push_back(nu - 1 - u); }
        uint64_t x = 0x9e3779b97f4a7c15ull;
        for (int i = 0; i < 8192; ++i) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; us.push_back(x % nu); }
      }
      const int NB = D + l.chain_grow;
      uint32_t xmask = 0;
      for (int i = 0; i < cp.n_ins; ++i) xmask |= 1u << cp.ins[i];
      for (uint64_t u : us) {
        const uint32_t w = (uint32_t)(u << cp.vbits);
        uint32_t op = w, oc = w;
        for (int i = 0; i < cp.n_ins; ++i) op = h_insert0(op, cp.ins[i]);
        for (int i = 0; i < cp.n_insc; ++i) oc = h_insert0(oc, cp.insc[i]);
        if (op % (uint32_t)V || oc % (uint32_t)V) return badc("unaligned vector", oc, V);
        if ((int64_t)(op | xmask) + V - 1 >= np) return badc("P", (int64_t)(op | xmask) + V - 1, np);
        for (int i = 0; i < D; ++i) {
          uint32_t g = 0;
          for (int j = 0; j < cp.n_seg[i]; ++j)
            g |= ((oc >> cp.seg_c[i][j]) & ((1u << cp.seg_len[i][j]) - 1u)) << cp.seg_b[i][j];
          const int64_t ns = int64_t(1) << cp.s_log2[i];
          for (int c = 0; c < std::min(4 << NB, wmc::dev::kChainDRow); ++c)
            for (int e = 0; e < V; ++e) {
              const int64_t lane = cp.b_vec[i] == 1 ? e : (cp.b_vec[i] == 2 ? 0 : cp.dv[i][e]);
              const int64_t o = (int64_t)g + cp.d[i][c] / es + lane;
              if (cp.d[i][c] % es || o >= ns) return badc("S", o, ns);
            }
        }
        for (int c = 0; c < (1 << NB); ++c)
          if ((int64_t)(oc | cp.dC[c]) + V - 1 >= nc) return badc("C", (int64_t)(oc | cp.dC[c]) + V - 1, nc);
        ++checked;
      }
      if (D > 4) {  // direct loads: no tiles; staged S_i and per-lane max/min
        for (int i = 0; i < D; ++i)
          if (cp.s_bytes_off[i] % 16 || cp.s_bytes_off[i] + ((size_t)es << cp.s_log2[i]) > cp.s_bytes_off[i + 1])
            return badc("staged S", i, D);
        const size_t need = cp.s_bytes_off[D] + 16 * (size_t)cp.mc.Qc;
        if (V > 2 || l.chain_grow || need > l.smem || l.smem > 220 * 1024 ||
            (l.threads != 0 && (l.threads < 32 || l.threads > wmc::dev::kDirectThreads || l.threads % 32)) ||
            ((uint64_t)l.blocks * (uint64_t)(l.threads ? l.threads : wmc::dev::kDirectThreads) * (uint64_t)V) %
                (uint64_t)cp.mc.Qc)
          return badc("direct chain launch", (int64_t)need, (int64_t)l.smem);
        continue;
      }
      const uint64_t n_tiles = 1ull << (cp.log2_nu + cp.vbits - cp.tb);
      const int64_t run_len = 1ll << cp.run_log2;
      const int64_t tile_elems = (int64_t)cp.nruns * run_len;
      for (uint64_t t = 0; t < n_tiles; ++t) {
        uint32_t base = (uint32_t)(t << cp.tb);
        for (int j = 0; j < cp.n_ins; ++j) base = h_insert0(base, cp.ins[j]);
        for (int r = 0; r < cp.nruns; ++r) {
          const int64_t lo = (int64_t)base + cp.run_off[r];
          if ((lo * es) % 16 || (run_len * es) % 16 || lo + run_len > np) return badc("bulk copy", lo + run_len - 1, np);
        }
        ++checked;
      }
      for (uint32_t wl = 0; wl < (1u << cp.tb); wl += (uint32_t)V) {
        uint32_t la = wl;
        for (int j = 0; j < cp.n_low; ++j) la = h_insert0(la, cp.low[j]);
        for (int c = 0; c < (1 << D); ++c) {
          const int64_t o = (int64_t)cp.pA[c] / es + la + V - 1;
          if (cp.pA[c] % es || o >= tile_elems) return badc("stage", o, tile_elems);
        }
      }
      // shared memory: stages, staged S_i, per-lane max/min and D scales
      size_t need = (size_t)cp.n_stages * (size_t)tile_elems * (size_t)es + cp.s_bytes_off[D] +
                    (16 + (size_t)D * (size_t)es) * (size_t)cp.mc.Qc;
      for (int i = 0; i < D; ++i)
        if (cp.s_bytes_off[i] % 16 || cp.s_bytes_off[i] + ((size_t)es << cp.s_log2[i]) > cp.s_bytes_off[i + 1])
          return badc("staged S", i, D);
      if (need > l.smem || l.smem > 220 * 1024 || cp.n_stages < 2 || cp.n_stages > wmc::dev::kMaxStagesC)
        return badc("shared memory", (int64_t)need, (int64_t)l.smem);
      continue;
    }
    if (l.kind == L_K2B) {
      // every unit's offsets (batch bits deposited) plus the small tables
      const wmc::dev::K2BParams &p = l.k2b;
      const int64_t es = l.ti == TD ? 8 : 4;
      const int64_t na = st->t_bytes[(size_t)l.id_a] / es, nb = st->t_bytes[(size_t)l.id_b] / es,
                    nc = st->t_bytes[(size_t)l.id_c] / es;
      const uint32_t last = (uint32_t)((1ull << p.log2_nu) - 1);
      uint32_t oa = 0, ob = 0, oc = last;
      for (int j = 0; j < p.log2_nu; ++j) {
        if (p.posA[j] >= 0) oa |= 1u << p.posA[j];
        if (p.posB[j] >= 0) ob |= 1u << p.posB[j];
      }
      for (int j = 0; j < p.n_insC; ++j) oc = h_insert0(oc, p.insC[j]);
      bool ok = (int64_t)(oa | p.offA[(1 << (p.fA + p.k)) - 1]) < na && (int64_t)(ob | p.offB[(1 << (p.k + p.fB)) - 1]) < nb &&
                (int64_t)(oc | p.offC[(1 << (p.fA + p.fB)) - 1]) < nc;
      for (int i = 0; i < (1 << (p.fA + p.k)) && ok; ++i) ok = (p.offA[i] & oa) == 0;
      for (int i = 0; i < (1 << (p.k + p.fB)) && ok; ++i) ok = (p.offB[i] & ob) == 0;
      for (int i = 0; i < (1 << (p.fA + p.fB)) && ok; ++i) ok = (p.offC[i] & oc) == 0;
      ok = ok && ((uint64_t)l.blocks * 256) % (uint64_t)p.mc.Qc == 0;
      if (!ok) { set_error("launch %zu: batched contraction offsets outside their tensors", li); return WMC_EINVAL; }
      ++checked;
      continue;
    }
    if (l.kind == L_BFP) {
      // mantissas (all index bits set) and the exponent entry of the last
      // block and lane of each tensor, inside the tensor's allocation
      const K1Params &p = l.k1;
      int64_t ma = 0, mb = 0;
      for (int j = 0; j < p.rC; ++j) {
        if (p.posA[j] >= 0) ma |= 1ll << p.posA[j];
        if (p.posB[j] >= 0) mb |= 1ll << p.posB[j];
      }
      for (int j = 0; j < p.k; ++j) {
        if (p.sposA[j] >= 0) ma |= 1ll << p.sposA[j];
        if (p.sposB[j] >= 0) mb |= 1ll << p.sposB[j];
      }
      const int64_t ids[3] = {l.id_a, l.id_b, l.id_c};
      const int64_t last[3] = {ma, mb, (1ll << p.rC) - 1};
      for (int t = 0; t < 3; ++t) {
        const size_t id = (size_t)ids[t];
        const TensorInfo &T = plan->tensors[id];
        const int mq = T.has_q ? st->m : 0;
        const int64_t es = st->t_dbl[id] ? 8 : 4;
        const int64_t n_el = int64_t(1) << ((int64_t)T.labels.size() + mq);
        const int64_t e_last = ((last[t] >> (mq + st->t_bb[id])) << mq) | (last[t] & ((1ll << mq) - 1));
        if (last[t] >= n_el || st->t_eoff[id] < st->t_off[id] + n_el * es ||
            st->t_eoff[id] + 4 * (e_last + 1) > st->t_off[id] + st->t_bytes[id] ||
            (t == 2 && (mq + st->t_bb[id] > 11))) {
          set_error("launch %zu: block-floating-point tensor %d out of bounds", li, t);
          return WMC_EINVAL;
        }
      }
      ++checked;
      continue;
    }
    if (l.kind != L_K2 && l.kind != L_K2T && l.kind != L_K1) continue;
    const int64_t ta = l.id_a, tb = l.id_b, tc = l.id_c;
    if (ta < 0 || tb < 0 || tc < 0) { set_error("launch %zu: unknown tensor", li); return WMC_EINVAL; }
    const int64_t es_in = l.kind == L_K1 ? (l.ti == TD ? 8 : 4) : (l.ti == TD ? 8 : 4);
    const int64_t es_out = l.kind == L_K1 ? (l.to == TD ? 8 : 4) : es_in;
    const int64_t na = st->t_bytes[(size_t)ta] / es_in, nb = st->t_bytes[(size_t)tb] / es_in,
                  nc = st->t_bytes[(size_t)tc] / es_out;
    auto bad = [&](const char *what, int64_t o, int64_t n) {
      set_error("launch %zu: %s offset %lld outside [0, %lld)", li, what, (long long)o, (long long)n);
      if (getenv("WMC_DEBUG_BOUNDS")) {
        const K2Params &q = l.kind == L_K2T ? l.k2t.k : l.k2;
        fprintf(stderr, "kind %d vbits %d log2_nu %d k %d f %d insA[%d]={%d,%d} insC[%d]={%d,%d} dC={%u,%u} dA={%u,%u} na %lld nb %lld nc %lld\n",
                (int)l.kind, q.vbits, q.log2_nu, q.k, q.f, q.n_insA, q.insA[0], q.insA[1], q.n_insC, q.insC[0], q.insC[1], q.dC[0], q.dC[1], q.dA[0], q.dA[1],
                (long long)na, (long long)nb, (long long)nc);
      }
      return WMC_EINVAL;
    };
    if (l.kind == L_K1) {
      const K1Params &p = l.k1;
      // the largest offsets: all bits set
      int64_t ma = 0, mb = 0;
      for (int j = 0; j < p.rC; ++j) {
        if (p.posA[j] >= 0) ma |= 1ll << p.posA[j];
        if (p.posB[j] >= 0) mb |= 1ll << p.posB[j];
      }
      for (int j = 0; j < p.k; ++j) {
        if (p.sposA[j] >= 0) ma |= 1ll << p.sposA[j];
        if (p.sposB[j] >= 0) mb |= 1ll << p.sposB[j];
      }
      if (ma >= na) return bad("A", ma, na);
      if (mb >= nb) return bad("B", mb, nb);
      if ((1ll << p.rC) > nc) return bad("C", (1ll << p.rC) - 1, nc);
      ++checked;
      continue;
    }
    const K2Params &p = l.kind == L_K2T ? l.k2t.k : l.k2;
    const int V = 1 << p.vbits;
    const uint64_t nu = 1ull << p.log2_nu;
    std::vector<uint64_t> us;
    if (nu <= (1u << 14)) for (uint64_t u = 0; u < nu; ++u) us.push_back(u);
    else {
      for (uint64_t u = 0; u < 4096; ++u) { us.push_back(u); us.push_back(nu - 1 - u); }
      uint64_t x = 0x9e3779b97f4a7c15ull;
      for (int i = 0; i < 8192; ++i) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; us.push_back(x % nu); }
    }
    for (uint64_t u : us) {
      const uint32_t w = (uint32_t)(u << p.vbits);
      uint32_t oa = w, oc = w, gb = 0;
      for (int i = 0; i < p.n_insA; ++i) oa = h_insert0(oa, p.insA[i]);
      for (int i = 0; i < p.n_insC; ++i) oc = h_insert0(oc, p.insC[i]);
      for (int i = 0; i < p.n_seg; ++i)
        gb |= ((oc >> p.seg_c[i]) & ((1u << p.seg_len[i]) - 1u)) << p.seg_b[i];
      if ((oa % (uint32_t)V) || (oc % (uint32_t)V)) return bad("unaligned vector", oa, V);
      for (int s = 0; s < (1 << p.k); ++s) {
        const int64_t o = (int64_t)oa + p.dA[s] + V - 1;
        if (o >= na) return bad("P", o, na);
        for (int f = 0; f < (1 << p.f); ++f) {
          for (int e = 0; e < V; ++e) {
            const int64_t ob = (int64_t)gb + p.dBs[s] + p.dBf[f] + p.dBv[e];
            if (ob >= nb) return bad("S", ob, nb);
          }
          const int64_t o2 = (int64_t)oc + p.dC[f] + V - 1;
          if (o2 >= nc) return bad("C", o2, nc);
        }
      }
      ++checked;
    }
    if (l.kind == L_K2T) {
      const dev::K2TParams &tp = l.k2t;
      const uint64_t n_tiles = 1ull << (p.log2_nu + p.vbits - tp.tb);
      const int64_t run_len = 1ll << tp.run_log2;
      const int64_t tile_elems = (int64_t)tp.nruns * run_len;
      if ((int64_t)l.smem != tile_elems * dev::kStages * es_in + (((es_in << tp.s_log2) + 15) & ~15ll) +
                                 (16 + es_in) * st->Qp)
        return bad("stage bytes", (int64_t)l.smem, tile_elems);
      if ((1ll << tp.s_log2) != nb) return bad("staged S size", 1ll << tp.s_log2, nb);
      for (uint64_t t = 0; t < n_tiles; ++t) {
        uint32_t base = (uint32_t)(t << tp.tb);
        for (int j = 0; j < p.n_insA; ++j) base = h_insert0(base, p.insA[j]);
        for (int r = 0; r < tp.nruns; ++r) {
          const int64_t lo = (int64_t)base + tp.run_off[r];
          if (lo % 4 || lo + run_len > na) return bad("bulk copy", lo + run_len - 1, na);
        }
        ++checked;
      }
      // shared-memory reads of one tile (all local work units)
      for (uint32_t wl = 0; wl < (1u << tp.tb); wl += (uint32_t)V) {
        uint32_t la = wl;
        for (int j = 0; j < tp.n_lowA; ++j) la = h_insert0(la, tp.lowA[j]);
        for (int s = 0; s < (1 << p.k); ++s) {
          const int64_t o = (int64_t)tp.sA_off[s] + la + V - 1;
          if (o >= tile_elems) return bad("stage", o, tile_elems);
        }
      }
    }
  }
  if (n_checked) *n_checked = checked;
  return WMC_OK;
}
