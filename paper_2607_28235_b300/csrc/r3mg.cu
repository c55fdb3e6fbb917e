// libr3mg: hierarchy setup, V-cycle, PCG / flexible CG and the C ABI (include/r3mg.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <limits>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels_dense.cuh"
#include "kernels_krylov.cuh"
#include "kernels_level.cuh"
#include "kernels_level_tma.cuh"
#include "kernels_batch.cuh"
#include "kernels_level_sym.cuh"
#include "kernels_mrhs.cuh"
#include "kernels_setup.cuh"
#include "kernels_vcycle.cuh"
#include "kernels_persistent.cuh"
#include "kernels_tcgen05.cuh"

using namespace r3mg;

namespace {

thread_local std::string g_last_error = "no error";

// Scratch of r3mg_level0_apply_noalloc: the caller-numbered input and output permuted into
// tree order.  It lives in the library image, so every GPU that loads the library holds it
// (16 MiB) until the process exits; no call ever allocates it.
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxN];
constexpr size_t kMaxSmem = 226 * 1024;   // opt-in shared memory per CTA on sm_103a, minus static use

struct Level {
  int64_t n = 0, nbox = 0;
  int b = 0;  // 0 on the fine level
  int64_t *box_row = nullptr, *nbr_ptr = nullptr, *nbr = nullptr, *slot_src = nullptr, *row_ptr = nullptr,
          *pair_box = nullptr;
  int32_t *win_off = nullptr, *win_size = nullptr;
  uint16_t* idx = nullptr;
  int max_slots = 0, win_max = 0, max_box_rows = 0;
  int32_t* row_order = nullptr;   // fine level: per box, local row indices by decreasing length
  int64_t stored = 0, nnz = 0, npairs = 0;
  double* v64 = nullptr;
  float* v32 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double lam_lo = 0.0, lam_hi = 0.0;
  std::vector<std::pair<double, double>> pre, post;  // Chebyshev step coefficients (a, c)
  double c0 = 0.0;                                   // 1/theta: first update of a zero guess
  void *x = nullptr, *r = nullptr, *d[2] = {nullptr, nullptr};
  int G = 8;
  HostPattern pat;
  // TMA-streamed kernel: work items per precision ([0] FP64, [1] FP32)
  struct Items { unsigned char* desc = nullptr; int64_t* desc_off = nullptr; int64_t nitems = 0; int SE = 0; int rmax = 0; int dmax = 0; size_t smem = 0; int grid = 0; };
  Items tma[2];
  // kernel configuration per precision ([0] FP64, [1] FP32): form 0 = register-streamed,
  // 1 = TMA-streamed; G lanes per row; nt threads per CTA (TMA form)
  // form 0 = register, 1 = TMA-streamed, 2 = register persistent (double-buffered window),
  // 3 = register with an L2 bulk prefetch of each box's matrix slice
  struct KConf { int form = 0; int G = 8; int nt = 256; float ms = 0.f; int u = 0; };   // u: 0 = default unroll
  int nsm = 148;
  KConf conf[2];
  int use_tma = 1;   // TMA work items could be built for this level
  // symmetric block form (coarse levels, FP32): upper blocks only
  SymView sym;
  bool sym_ok = false;
  int64_t sym_nnz = 0, sym_tvals = 0;   // stored upper values (padding excluded); transposed-pair values

  float* sym_vals = nullptr;
  float* sym_y = nullptr;
  float* sym_t = nullptr;
  std::vector<int64_t> h_row_ptr;   // host copy of the block-row pointers (symmetric gather)
  std::vector<int64_t> h_box_row;   // host copy of box row offsets (fine) for item building
  std::vector<int32_t> h_win_size;  // host copy of the window lengths (fine) for item building
};

}  // namespace

struct r3mg_hierarchy;
using Hier = r3mg_hierarchy;
struct r3mg_hierarchy {
  r3mg_params prm{};
  int64_t n = 0;
  int dim = 0, L = 0, b = 1, fan = 4;
  HostPartition part;
  std::vector<Level> lv;
  int64_t nnz_csr = 0;
  int64_t *src = nullptr, *diag_src = nullptr, *perm = nullptr;
  int64_t* csr_rowptr = nullptr;   // the caller's CSR structure (adjoint sampled outer product)
  int32_t* csr_col = nullptr;
  int32_t* box_of_tree = nullptr;
  double* coords_tree = nullptr;
  std::vector<double*> P64;
  std::vector<float*> P32;
  int64_t nc = 0, ncp = 0;
  double* Ainv64 = nullptr;
  float* Ainv32 = nullptr;
  double *hb_dev = nullptr, *hx_dev = nullptr;   // device copies for r3mg_pcg_host
  double *cx = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr, *cz = nullptr, *cb = nullptr;
  double *part_a = nullptr, *part_b = nullptr, *scal = nullptr;
  int64_t npart = 0;
  int* status = nullptr;
  double* host_scal = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_state = 0;  // 0 untried, 1 ready, -1 unavailable
  int graph_prof = 0;   // profiling state the graph was captured with
  std::vector<void*> allocs;
  std::string err = "no error";
  // instrumentation: event pairs around level-operator launches, kernel launch counter
  int prof_on = 0;
  struct ProfSlot { int kind; cudaEvent_t e0, e1; };
  std::vector<ProfSlot> slots;        // fixed slots used by the V-cycle body (same in every replay)
  size_t slot_next = 0;
  std::vector<int> pending;           // slots recorded since the last harvest
  std::vector<int> graph_slots;       // slots recorded by one replay of the V-cycle graph
  ProfSlot cg_slot{0, nullptr, nullptr};  // the CG product (launched outside the graph)
  bool cg_pending = false;
  std::vector<double> prof_ms;        // per kind: total milliseconds
  std::vector<int64_t> prof_n;        // per kind: launches
  std::vector<double> prof_bytes;     // per kind: algorithmic bytes per launch
  int64_t launches = 0;               // kernels launched by solve-path calls
  int* tma_err = nullptr;             // bounded-wait expiry flag of the TMA kernels
  // ---- batches of independent problems (nprob > 1): one block-diagonal hierarchy
  int nprob = 1;
  struct BLevel {
    std::vector<int64_t> row_off;                 // nprob + 1 row offsets of the problems
    int32_t* rprob = nullptr;                     // problem of every row
    int64_t* label = nullptr;                     // index of every row inside its problem (Lanczos start)
    int64_t *sb = nullptr, *se = nullptr;         // segments: rows of one problem, at most kSegRows
    int* soff = nullptr;                          // nprob + 1 first segments
    int nseg = 0;
    double *preA = nullptr, *preC = nullptr, *postA = nullptr, *postC = nullptr;   // [step][nprob]
    double* c0 = nullptr;                         // per problem: 1 / theta
    std::vector<double> lam;                      // per problem: upper interval end
    int npre = 0, npost = 0;
  };
  std::vector<BLevel> bl;
  std::vector<int64_t> h_moff, h_mld, h_cof;     // coarsest blocks: offset, leading dim, row offsets
  int64_t *d_moff = nullptr, *d_mld = nullptr, *d_cof = nullptr;
  int64_t batch_ainv_size = 0;
  BatchScal bs{};
  double* seg_part = nullptr;
  double* seg_out = nullptr;                      // nprob scratch for host reads
  std::vector<double> h_seg;
  cudaGraphExec_t bgraph = nullptr;
  int bgraph_state = 0;
  // single-problem loop graph (conditional WHILE node)
  cudaGraphExec_t lgraph = nullptr;
  int lgraph_state = 0;
  int* d_its = nullptr;
  double* d_loop = nullptr;
  int* d_flag = nullptr;              // zero-initial-guess test
  double bgraph_rtol = -1.0;
  int bgraph_maxit = -1;
  // ---- several right-hand sides (row-interleaved blocks of M columns)
  int mr_M = 0;                       // columns of the allocated block vectors (0: none yet)
  std::vector<void*> mr_x, mr_r, mr_d0, mr_d1;   // per level, V-cycle precision
  double *mr_b = nullptr, *mr_xc = nullptr, *mr_rc = nullptr, *mr_p = nullptr, *mr_q = nullptr, *mr_z = nullptr;
  double *mr_scal = nullptr, *mr_pa = nullptr, *mr_pb = nullptr, *mr_lp = nullptr;
  int *mr_its = nullptr, *mr_active = nullptr;
  double* mr_host = nullptr;          // pinned: 2 x 16 doubles + 2 x 16 ints
  int64_t mr_npart = 0;
  std::vector<int> mr_S[2];           // per level: entry slots per row ([0] FP64, [1] FP32)
  cudaGraphExec_t mgraph = nullptr;
  int mgraph_state = 0;
  int prof_cols = 1;                  // columns of the last profiled solve (bytes per launch)
  int64_t mr_graph_kernels = 0;       // kernels in one block V-cycle
  int32_t* mr_gidx = nullptr;         // fine level: global column (tree row) of every stored entry
  // grouped fine level for the block kernels (rows with equal column lists; k_mr_grouped), built
  // on first use: classes of 8, 4, 2 and 1 rows per group, class-major
  bool mrg_built = false;
  int64_t mrg_ng[4] = {0, 0, 0, 0};   // groups per class
  int64_t mrg_g0[4] = {0, 0, 0, 0};   // first group of each class
  int64_t mrg_r0[4] = {0, 0, 0, 0};   // first row slot of each class in mrg_rows
  int64_t* mrg_geoff = nullptr;       // groups + 1 offsets into mrg_col (entries per group)
  int64_t* mrg_gvoff = nullptr;       // groups + 1 offsets into the grouped values
  int32_t* mrg_rows = nullptr;        // R rows per group
  int32_t* mrg_col = nullptr;         // the groups' column lists (global rows of the level)
  void* mrg_vals[2] = {nullptr, nullptr};   // grouped values ([0] FP64, [1] FP32), entry-major
  int nsm = 148;
  int tma_ctas = 1;                   // TMA kernel CTAs per SM
  int64_t graph_kernels = 0;          // kernels in one replay of the V-cycle graph
  // stop test: ||r|| <= max(rtol ||b||, stop_atol, stop_red ||r_0||)  (r3mg_set_stop_rule)
  double stop_atol = 0.0, stop_red = 0.0;
  // mesh statistics of the paper's tables: h = largest distance between two coupled support
  // points, H = largest diameter of a coarsest-level box
  double h_fine = 0.0, H_coarse = 0.0;
  std::vector<double> ritz;           // per smoothed level: the Lanczos Ritz value (before the safety factor)
  int mr_last_m = 0;                  // columns of the last block solve (condition estimates)
  double* noalloc_scratch = nullptr;  // device address of the allocation-free product's static scratch
  // coarsest solve: 0 = explicit inverse (one GEMV), 1 = forward and back substitution with the
  // Cholesky factor (r3mg_set_coarse_mode); the factor is kept for single hierarchies
  int coarse_mode = 0;
  double* L64 = nullptr;
  float* L32 = nullptr;
  double* ctmp = nullptr;             // the forward substitution's result (nc values, either precision)
  // batched solves: 0 = the iteration loop as a graph of per-step kernels, 1 = one persistent
  // cooperative kernel for the whole loop (r3mg_set_batch_mode); 2 = automatic: the first two
  // solves time one form each (per iteration of the loop), later solves take the faster
  int batch_mode = 2;
  float batch_ms_it[2] = {-1.f, -1.f};
  int batch_used = 0;
  unsigned* pbar = nullptr;           // persistent solve: grid-barrier counter and generation
  int* pany = nullptr;                // persistent solve: running problems per iteration
  int pany_cap = 0;
  cudaGraphExec_t pgraph = nullptr;   // persistent solve captured in a graph (memsets + the launch)
  int pgraph_state = 0;
  double pgraph_rtol = -1.0;
  int pgraph_budget = -1;
  long long wait_cycles = 0;          // limit of the streamed kernels' mbarrier waits (0 = about 1 s)
  int withhold_first = 0;             // expiry-path test: withhold CTA 0's first descriptor copy
};

namespace {

struct Fail {
  r3mg_status st;
  std::string msg;
};

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      throw Fail{e_ == cudaErrorMemoryAllocation ? R3MG_E_OOM : R3MG_E_CUDA,                       \
                 std::string(#call) + ": " + cudaGetErrorString(e_)};                              \
  } while (0)

template <typename T>
T* dalloc(r3mg_hierarchy* h, int64_t count) {
  void* p = nullptr;
  if (count <= 0) count = 1;
  CK(cudaMalloc(&p, sizeof(T) * (size_t)count));
  h->allocs.push_back(p);
  return (T*)p;
}

template <typename T>
T* upload(r3mg_hierarchy* h, const std::vector<T>& v) {
  T* p = dalloc<T>(h, (int64_t)v.size());
  if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream));
  return p;
}

inline int grid_for(int64_t work, int threads = 256, int cap = 148 * 32) {
  int64_t g = (work + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

template <typename T>
LevelView<T> view(const Level& L) {
  LevelView<T> v;
  v.nrows = L.n; v.nbox = L.nbox; v.b = L.b;
  v.box_row = L.box_row; v.nbr_ptr = L.nbr_ptr; v.nbr = L.nbr; v.win_off = L.win_off; v.slot_src = L.slot_src;
  v.win_size = L.win_size; v.row_ptr = L.row_ptr; v.idx = L.idx;
  if constexpr (sizeof(T) == 8) { v.vals = (const T*)L.v64; v.dinv = (const T*)L.dinv64; }
  else { v.vals = (const T*)L.v32; v.dinv = (const T*)L.dinv32; }
  v.max_slots = L.max_slots; v.win_max = L.win_max; v.max_box_rows = L.max_box_rows;
  v.row_order = L.row_order;
  // a coarse level whose values fit half of L2 keeps them there between its consecutive steps
  v.keep = (L.b > 0 && L.stored * (int64_t)sizeof(T) <= ((int64_t)64 << 20)) ? 1 : 0;
  return v;
}

// The opt-in dynamic shared-memory limit is an attribute of a kernel on one device: raise it once
// per (kernel, device) to the largest size launched there (before any graph capture: the
// setup's warm-up launches do this).
void ensure_smem(const void* func, size_t sm) {
  if (sm <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[{func, dev}];
  if (sm > cur) {
    CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    cur = sm;
  }
}

// loads in flight per lane: 4 x 16-byte steps (FP32) or 2 x 32-byte steps (FP64)
template <typename T, bool FINE>
constexpr int unroll_for() { return sizeof(T) == 4 ? 4 : 2; }

template <typename T, int G, bool FINE, class Ep, int U>
void launch_level_gu(const LevelView<T>& v, const T* xin, Ep ep, double* part, cudaStream_t s, int pipe, int nsm,
                     int pf, int nt, int sp);

// FP64 rows may use 2 or 4 steps of 32 bytes in flight per lane (autotuned); FP32 uses 4 x 16 bytes
template <typename T, int G, bool FINE, class Ep>
void launch_level_g(const LevelView<T>& v, const T* xin, Ep ep, double* part, cudaStream_t s, int pipe, int nsm,
                    int pf, int nt, int u, int sp) {
  if (sizeof(T) == 8 && u == 4 && !sp) launch_level_gu<T, G, FINE, Ep, 4>(v, xin, ep, part, s, pipe, nsm, pf, nt, 0);
  else launch_level_gu<T, G, FINE, Ep, unroll_for<T, FINE>()>(v, xin, ep, part, s, pipe, nsm, pf, nt, sp);
}

template <typename T, int G, bool FINE, class Ep, int U>
void launch_level_gu(const LevelView<T>& v, const T* xin, Ep ep, double* part, cudaStream_t s, int pipe, int nsm,
                     int pf, int nt, int sp) {
  if constexpr (U == unroll_for<T, FINE>()) {
    if (sp) {   // software-pipelined row loop, with or without the L2 prefetch
      const size_t sm = level_smem_bytes(v);
      auto kern = pf ? level_kernel<T, G, FINE, Ep, U, false, true, true> : level_kernel<T, G, FINE, Ep, U, false, false, true>;
      ensure_smem((const void*)kern, sm);
      kern<<<(int)std::max<int64_t>(1, v.nbox), nt, sm, s>>>(v, xin, ep, part);
      CK(cudaGetLastError());
      return;
    }
  }
  if (pf) {
    const size_t sm = level_smem_bytes(v);
    auto kern = level_kernel<T, G, FINE, Ep, U, false, true, false>;
    ensure_smem((const void*)kern, sm);
    kern<<<(int)std::max<int64_t>(1, v.nbox), nt, sm, s>>>(v, xin, ep, part);
    CK(cudaGetLastError());
    return;
  }
  if (pipe) {
    // persistent form: two windows per CTA, grid sized to the CTAs that fit the SMs
    const size_t sm = 2 * level_smem_bytes(v);
    auto kern = level_kernel<T, G, FINE, Ep, U, true, false, false>;
    ensure_smem((const void*)kern, sm);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2048 / nt, (kMaxSmem + 1024) / (sm + 1024)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(v.nbox, (int64_t)nsm * per_sm));
    kern<<<grid, nt, sm, s>>>(v, xin, ep, part);
    CK(cudaGetLastError());
    return;
  }
  const size_t sm = level_smem_bytes(v);
  auto kern = level_kernel<T, G, FINE, Ep, U, false, false, false>;
  // opt in to more than 48 KB of dynamic shared memory per instantiation (the setup's warm-up
  // V-cycle does this before any graph capture)
  ensure_smem((const void*)kern, sm);
  const int grid = (int)std::max<int64_t>(1, v.nbox);
  kern<<<grid, nt, sm, s>>>(v, xin, ep, part);
  CK(cudaGetLastError());
}

template <typename T, class Ep>
int launch_level(const Level& L, const T* xin, Ep ep, double* part, cudaStream_t s) {
  const LevelView<T> v = view<T>(L);
  const bool fine = (L.b == 0);
  const Level::KConf& c = L.conf[sizeof(T) == 4 ? 1 : 0];

  // forms: 0 register, 2 persistent, 3 L2 prefetch, 5 software-pipelined, 6 pipelined + L2 prefetch
  const int pipe = (c.form == 2), pf = (c.form == 3 || c.form == 6), sp = (c.form == 5 || c.form == 6);
  const int nsm = L.nsm, nt = (c.nt == 128) ? 128 : 256, u = c.u;
  // products on a level whose step takes the staged symmetric form (lanes = CTAs per SM) run on
  // the register form with 16 lanes per row
  switch (c.form == 7 ? 16 : c.G) {
    case 2:   // two lanes per row: fine FP64 rows only (shorter reductions, finer row tails)
      if constexpr (sizeof(T) == 8) {
        if (fine) { launch_level_g<T, 2, true>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp); break; }
      }
      [[fallthrough]];
    case 4: fine ? launch_level_g<T, 4, true>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp) : launch_level_g<T, 4, false>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp); break;
    case 8: fine ? launch_level_g<T, 8, true>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp) : launch_level_g<T, 8, false>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp); break;
    case 16: fine ? launch_level_g<T, 16, true>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp) : launch_level_g<T, 16, false>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp); break;
    default: fine ? launch_level_g<T, 32, true>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp) : launch_level_g<T, 32, false>(v, xin, ep, part, s, pipe, nsm, pf, nt, u, sp); break;
  }
  if (!pipe) return (int)std::max<int64_t>(1, v.nbox);
  const size_t sm = 2 * level_smem_bytes(v);
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2048 / nt, (kMaxSmem + 1024) / (sm + 1024)));
  return (int)std::max<int64_t>(1, std::min<int64_t>(v.nbox, (int64_t)nsm * per_sm));
}

// kinds: 0 = CG product (FP64 fine level), 1 + l = smoother steps on level l
int prof_begin(r3mg_hierarchy* h, int kind, bool capturing) {
  if (!h->prof_on) return -1;
  if (h->slot_next == h->slots.size()) {
    r3mg_hierarchy::ProfSlot s{kind, nullptr, nullptr};
    CK(cudaEventCreate(&s.e0));
    CK(cudaEventCreate(&s.e1));
    h->slots.push_back(s);
  }
  const int id = (int)h->slot_next++;
  h->slots[id].kind = kind;
  CK(cudaEventRecordWithFlags(h->slots[id].e0, h->stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  return id;
}

void prof_end(r3mg_hierarchy* h, int id, bool capturing) {
  if (id < 0) return;
  CK(cudaEventRecordWithFlags(h->slots[id].e1, h->stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  if (capturing) h->graph_slots.push_back(id); else h->pending.push_back(id);
}

// after a host synchronisation: fold the elapsed times of every recorded pair into the totals
void prof_add(r3mg_hierarchy* h, int k, float ms) {
  if ((int)h->prof_ms.size() <= k) { h->prof_ms.resize(k + 1, 0.0); h->prof_n.resize(k + 1, 0); }
  h->prof_ms[k] += ms;
  h->prof_n[k] += 1;
}

void prof_harvest(r3mg_hierarchy* h) {
  if (h->cg_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->cg_slot.e0, h->cg_slot.e1) == cudaSuccess) prof_add(h, 0, ms);
    h->cg_pending = false;
  }
  for (int id : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->slots[id].e0, h->slots[id].e1) == cudaSuccess) {
      prof_add(h, h->slots[id].kind, ms);
    }
  }
  h->pending.clear();
}

// Bounded-wait control of the copy-engine-streamed kernels: the expiry flag, the wait limit and
// the expiry-path test switch (r3mg_set_wait_limit).
struct TmaCtl {
  int* err;
  long long wait;
  int withhold;
};

template <typename T, int G, bool FINE, class Ep>
void launch_tma_g(const Level& A, const Level::Items& it, const T* xin, Ep ep, double* part, cudaStream_t s, TmaCtl ctl) {
  TmaView<T> v;
  v.L = view<T>(A);
  v.desc = it.desc; v.desc_off = it.desc_off; v.nitems = it.nitems; v.stage_entries = it.SE; v.max_item_rows = it.rmax;
  v.desc_max = it.dmax; v.err = ctl.err; v.wait_cycles = ctl.wait; v.withhold_first = ctl.withhold;
  auto kern = level_kernel_tma<T, G, FINE, Ep>;
  ensure_smem((const void*)kern, it.smem);
  kern<<<it.grid, A.conf[sizeof(T) == 4 ? 1 : 0].nt, it.smem, s>>>(v, xin, ep, part);
  CK(cudaGetLastError());
}

template <typename T, class Ep>
void launch_tma(const Level& A, const T* xin, Ep ep, double* part, cudaStream_t s, TmaCtl err) {
  const Level::Items& it = A.tma[sizeof(T) == 4 ? 1 : 0];
  const bool fine = (A.b == 0);
  switch (A.conf[sizeof(T) == 4 ? 1 : 0].G) {
    case 4: fine ? launch_tma_g<T, 4, true>(A, it, xin, ep, part, s, err) : launch_tma_g<T, 4, false>(A, it, xin, ep, part, s, err); break;
    case 8: fine ? launch_tma_g<T, 8, true>(A, it, xin, ep, part, s, err) : launch_tma_g<T, 8, false>(A, it, xin, ep, part, s, err); break;
    case 16: fine ? launch_tma_g<T, 16, true>(A, it, xin, ep, part, s, err) : launch_tma_g<T, 16, false>(A, it, xin, ep, part, s, err); break;
    default: fine ? launch_tma_g<T, 32, true>(A, it, xin, ep, part, s, err) : launch_tma_g<T, 32, false>(A, it, xin, ep, part, s, err); break;
  }
}

TmaCtl tma_ctl(const r3mg_hierarchy* h) {
  return TmaCtl{h->tma_err, h->wait_cycles > 0 ? h->wait_cycles : kWaitCycles, h->withhold_first};
}

// the FP32 step of this level runs on the symmetric (upper-block) storage: form 4 streamed, 7 staged
// (form 7 keeps its resident CTAs per SM in the lanes field)
bool sym_form(const Level& A) { return A.sym_ok && (A.conf[1].form == 4 || A.conf[1].form == 7); }

// Product y = A x (+ partial w . y) on either kernel form; partial count = grid of the kernel.
template <typename T>
bool tma_on(const Level& A) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  return A.conf[pi].form == 1 && A.tma[pi].nitems > 0;   // form 0 / 2: register kernel
}

template <typename T>
int level_apply_dot(r3mg_hierarchy* h, const Level& A, const T* x, T* y, const T* w, double* part) {
  if (tma_on<T>(A)) {
    launch_tma<T>(A, x, TEpApplyDot<T>{y, w}, part, h->stream, tma_ctl(h));
    return A.tma[sizeof(T) == 4 ? 1 : 0].grid;
  }
  return launch_level<T>(A, x, TEpApplyDot<T>{y, w}, part, h->stream);
}

template <typename T>
void level_cheb(r3mg_hierarchy* h, const Level& A, T* x, T* r, T* d, T* dn, const T* dinv, T a, T c) {
  if constexpr (sizeof(T) == 4) {
    if (sym_form(A)) {
      sym_step(h, A, d, SymCheb{x, r, d, dn, dinv, a, c});
      return;
    }
  }
  if (tma_on<T>(A)) launch_tma<T>(A, d, TEpCheb<T>{x, r, d, dn, dinv, a, c}, nullptr, h->stream, tma_ctl(h));
  else launch_level<T>(A, d, TEpCheb<T>{x, r, d, dn, dinv, a, c}, nullptr, h->stream);
}

// Work items of the TMA kernel: each box, split into runs of rows whose entries fit one
// stage buffer; the stage size fills the shared memory of tma_ctas CTAs per SM.  Every item
// gets a descriptor (entry range, window segments, local row offsets) the kernel bulk-copies.
void build_items(r3mg_hierarchy* h, Level& A, int prec_idx, const std::vector<int64_t>& row_ptr,
                 const std::vector<int32_t>& win_off_h, const std::vector<int64_t>& slot_src_h) {
  const bool fine = (A.b == 0);
  const size_t es = prec_idx == 1 ? 4 : 8;
  auto box_rows = [&](int64_t B, int64_t& r0, int64_t& r1) {
    r0 = fine ? A.h_box_row[B] : B * A.b;
    r1 = fine ? A.h_box_row[B + 1] : (B + 1) * A.b;
  };
  int rmax = 0, nnmax = 0;
  for (int64_t B = 0; B < A.nbox; ++B) {
    int64_t r0, r1;
    box_rows(B, r0, r1);
    rmax = std::max<int>(rmax, (int)(r1 - r0));
    nnmax = std::max<int>(nnmax, (int)(A.pat.ptr[B + 1] - A.pat.ptr[B]));
  }
  const int dmax = (int)((sizeof(ItemDesc) + sizeof(SegDesc) * nnmax + 4 * (rmax + 1) + 15) & ~(size_t)15);
  const size_t budget = kMaxSmem / h->tma_ctas - 1024;
  const size_t fixed = 128 + 3 * ((size_t)dmax + 128) + 2 * ((size_t)A.win_max * es + 128) +
                       2 * ((size_t)kAux * rmax * es + 128) + (fine ? 2 * (32 + 128) : 0) + 256;
  if (fixed + 2 * 1024 * (es + 2) > budget) { A.use_tma = 0; return; }
  int SE = (int)((budget - fixed) / (2 * (es + (fine ? 2 : 0))));
  SE = std::min(SE, 1 << 20) & ~7;
  std::vector<unsigned char> blob;
  std::vector<int64_t> off{0};
  for (int64_t B = 0; B < A.nbox; ++B) {
    int64_t r0, r1;
    box_rows(B, r0, r1);
    const int64_t q0 = A.pat.ptr[B], nn = A.pat.ptr[B + 1] - q0;
    int64_t rs = r0;
    while (rs < r1) {
      int64_t re = rs;
      while (re < r1 && row_ptr[re + 1] - row_ptr[rs] <= SE) ++re;
      if (re == rs) { A.use_tma = 0; return; }   // one row longer than a stage: register kernel
      ItemDesc hd{row_ptr[rs], row_ptr[re], rs, (int32_t)(re - rs), (int32_t)nn, 0, 0};
      std::vector<SegDesc> seg(nn);
      int64_t W = 0;
      for (int64_t s = 0; s < nn; ++s) {
        if (fine) {
          const int32_t wend = (s + 1 < nn) ? win_off_h[q0 + s + 1] : A.h_win_size[B];
          seg[s] = SegDesc{slot_src_h[q0 + s], win_off_h[q0 + s], wend - win_off_h[q0 + s]};
        } else {
          seg[s] = SegDesc{A.pat.nbr[q0 + s] * A.b, (int32_t)(s * A.b), A.b};
        }
        W = std::max<int64_t>(W, seg[s].wo + seg[s].len);
      }
      hd.W = (int32_t)W;
      const size_t o = blob.size();
      const size_t sz = (sizeof(ItemDesc) + sizeof(SegDesc) * nn + 4 * (re - rs + 1) + 15) & ~(size_t)15;
      blob.resize(o + sz, 0);
      std::memcpy(blob.data() + o, &hd, sizeof hd);
      std::memcpy(blob.data() + o + sizeof hd, seg.data(), sizeof(SegDesc) * nn);
      int32_t* ro = reinterpret_cast<int32_t*>(blob.data() + o + sizeof hd + sizeof(SegDesc) * nn);
      for (int64_t rr = rs; rr <= re; ++rr) ro[rr - rs] = (int32_t)(row_ptr[rr] - row_ptr[rs]);
      off.push_back((int64_t)blob.size());
      rs = re;
    }
  }
  Level::Items& it = A.tma[prec_idx];
  it.nitems = (int64_t)off.size() - 1;
  it.desc = upload(h, blob);
  it.desc_off = upload(h, off);
  it.SE = SE;
  it.rmax = rmax;
  it.dmax = dmax;
  it.smem = fine ? (es == 4 ? TmaLayout<float, true>(SE, A.win_max, rmax, dmax).total : TmaLayout<double, true>(SE, A.win_max, rmax, dmax).total)
                 : (es == 4 ? TmaLayout<float, false>(SE, A.win_max, rmax, dmax).total : TmaLayout<double, false>(SE, A.win_max, rmax, dmax).total);
  if (it.smem > kMaxSmem / h->tma_ctas) { A.use_tma = 0; return; }
  it.grid = (int)std::max<int64_t>(1, std::min<int64_t>(it.nitems, (int64_t)h->nsm * h->tma_ctas));
}

// Symmetric block form of a coarse level: upper block rows, transposed-pair vectors, lower lists.
void build_sym(r3mg_hierarchy* h, Level& A) {
  const int b = A.b;
  if (b <= 0 || b > kSymMaxB) return;
  const int64_t nb = A.nbox;
  std::vector<int64_t> up_base(nb + 1, 0), tp_off(nb + 1, 0), low_ptr(nb + 1, 0);
  std::vector<int32_t> up_len(nb), dslot(nb);
  std::vector<std::vector<int64_t>> low(nb);
  int wmax = 0;
  int64_t smax = 0;
  for (int64_t B = 0; B < nb; ++B) {
    const int64_t q0 = A.pat.ptr[B], nn = A.pat.ptr[B + 1] - q0;
    int64_t d = -1;
    for (int64_t s = 0; s < nn; ++s) if (A.pat.nbr[q0 + s] == B) { d = s; break; }
    if (d < 0) return;   // no diagonal block: leave the level to the full forms
    const int nup = (int)(nn - d);
    const int len = (nup * b + 3) & ~3;
    dslot[B] = (int32_t)d;
    up_len[B] = len;
    up_base[B + 1] = up_base[B] + (int64_t)b * len;
    tp_off[B + 1] = tp_off[B] + (nup - 1);
    wmax = std::max(wmax, len);
    smax = std::max<int64_t>(smax, (int64_t)b * len);
    for (int64_t s = d + 1; s < nn; ++s) low[A.pat.nbr[q0 + s]].push_back(tp_off[B] + (s - d - 1));
  }
  std::vector<int64_t> low_pair;
  for (int64_t B = 0; B < nb; ++B) {
    low_pair.insert(low_pair.end(), low[B].begin(), low[B].end());
    low_ptr[B + 1] = (int64_t)low_pair.size();
  }
  SymView& V = A.sym;
  V.nbox = nb; V.b = b;
  V.up_base = upload(h, up_base);
  V.up_len = upload(h, up_len);
  V.nbr_ptr = A.nbr_ptr; V.nbr = A.nbr;
  V.dslot = upload(h, dslot);
  V.tp_off = upload(h, tp_off);
  V.low_ptr = upload(h, low_ptr);
  V.low_pair = upload(h, low_pair);
  V.win_max = wmax;
  V.stage_max = (int)std::min<int64_t>(smax, 1 << 30);
  A.sym_vals = dalloc<float>(h, up_base[nb]);
  V.vals = A.sym_vals;
  A.sym_y = dalloc<float>(h, A.n);
  A.sym_t = dalloc<float>(h, std::max<int64_t>(1, tp_off[nb] * b));
  A.sym_nnz = 0;
  for (int64_t B = 0; B < nb; ++B) A.sym_nnz += (int64_t)(A.pat.ptr[B + 1] - A.pat.ptr[B] - dslot[B]) * b * b;
  A.sym_tvals = tp_off[nb] * b;
  A.sym_ok = true;
}

// Shared-memory stage of the staged symmetric kernel for `cps` resident CTAs per SM: the CTA's
// share of the SM's shared memory less the window, capped at the level's largest upper slice
// (floats, multiple of 4; 0 when not even the window fits).
int sym_stage_cap(const Level& A, int cps) {
  const int64_t win = (A.sym.win_max + 3) & ~3;
  const int64_t share = std::min<int64_t>((int64_t)kMaxSmem, (int64_t)228 * 1024 / std::max(1, cps) - 2048) / 4;
  const int64_t cap = std::min<int64_t>(share - win, ((int64_t)A.sym.stage_max + 3) & ~3);
  return cap < 4 * A.b ? 0 : (int)(cap & ~(int64_t)3);
}

void sym_step(r3mg_hierarchy* h, const Level& A, const float* d, SymCheb ep) {
  const int cap = A.conf[1].form == 7 ? sym_stage_cap(A, A.conf[1].G) : 0;
  if (cap > 0) {
    const TmaCtl c = tma_ctl(h);
    const size_t sm = sizeof(float) * ((size_t)cap + (((size_t)A.sym.win_max + 3) & ~(size_t)3));
    ensure_smem((const void*)k_sym_block_staged, sm);
    k_sym_block_staged<<<(int)std::max<int64_t>(1, A.nbox), kSymThreads, sm, h->stream>>>(
        A.sym, d, A.sym_y, A.sym_t, cap, c.err, c.wait, c.withhold);
  } else {
    // form 4: the lanes field selects the load wave (4 rows, else 8), the threads field 96 or 128
    const size_t sm = sizeof(float) * (size_t)A.sym.win_max;
    const bool t96 = A.conf[1].nt == 96;
    auto kern = A.conf[1].G == 4 ? (t96 ? k_sym_block<4, 96> : k_sym_block<4>)
                                 : (t96 ? k_sym_block<8, 96> : k_sym_block<8>);
    ensure_smem((const void*)kern, sm);
    kern<<<(int)std::max<int64_t>(1, A.nbox), t96 ? 96 : kSymThreads, sm, h->stream>>>(A.sym, d, A.sym_y, A.sym_t);
  }
  k_sym_finish<<<grid_for(A.n), 256, 0, h->stream>>>(A.sym, A.sym_y, A.sym_t, ep);
  CK(cudaGetLastError());
}

void read_status(r3mg_hierarchy* h, int& st) {
  CK(cudaMemcpyAsync(&h->host_scal[15], h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(&st, &h->host_scal[15], sizeof(int));
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
}

double reduce_read(r3mg_hierarchy* h, const double* part, int m, int slot, int fin = FIN_NONE) {
  k_reduce<<<1, 1024, 0, h->stream>>>(part, m, h->scal, slot, fin, h->status);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h->host_scal[slot], &h->scal[slot], sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return h->host_scal[slot];
}

void reduce_dev(r3mg_hierarchy* h, const double* part, int m, int slot, int fin) {
  k_reduce<<<1, 1024, 0, h->stream>>>(part, m, h->scal, slot, fin, h->status);
  CK(cudaGetLastError());
}

int auto_lanes(double avg_row) {
  if (avg_row >= 512) return 32;
  if (avg_row >= 160) return 16;
  if (avg_row >= 48) return 8;
  return 4;
}

// Chebyshev coefficient schedule (Saad, Algorithm 12.1) split into fused steps.  Every step
// is  x += d;  r -= A d;  d = a d + c D^{-1} r.  A sweep boundary restarts the recurrence
// (a = 0, c = 1/theta); the last pre-smoothing step only serves the residual.
void make_schedule(Level& L, int k, int nu) {
  const double theta = 0.5 * (L.lam_hi + L.lam_lo), delta = 0.5 * (L.lam_hi - L.lam_lo), sigma = theta / delta;
  L.c0 = 1.0 / theta;
  L.pre.clear(); L.post.clear();
  auto sweep_inner = [&](std::vector<std::pair<double, double>>& out) {
    double rho = 1.0 / sigma;
    for (int i = 1; i < k; ++i) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      out.emplace_back(rn * rho, 2.0 * rn / delta);
      rho = rn;
    }
  };
  for (int j = 0; j < nu; ++j) {
    sweep_inner(L.pre);
    L.pre.emplace_back(0.0, 1.0 / theta);
  }
  L.post.emplace_back(0.0, 1.0 / theta);
  for (int j = 0; j < nu; ++j) {
    sweep_inner(L.post);
    if (j + 1 < nu) L.post.emplace_back(0.0, 1.0 / theta);
  }
}

// ---------------------------------------------------------------- V-cycle
template <typename T>
const T* Pmat(r3mg_hierarchy* h, int l) {
  if constexpr (sizeof(T) == 8) return (const T*)h->P64[l]; else return (const T*)h->P32[l];
}
template <typename T>
const T* Ainv(r3mg_hierarchy* h) {
  if constexpr (sizeof(T) == 8) return (const T*)h->Ainv64; else return (const T*)h->Ainv32;
}
template <typename T>
const T* Lfac(r3mg_hierarchy* h) {
  if constexpr (sizeof(T) == 8) return (const T*)h->L64; else return (const T*)h->L32;
}

// The coarsest solve x = A_c^{-1} r in the configured form: one GEMV with the explicit inverse,
// or forward and back substitution with the Cholesky factor (one CTA each).  Returns launches.
template <typename T>
int coarsest_apply(r3mg_hierarchy* h, const T* r, T* x) {
  cudaStream_t s = h->stream;
  if (h->coarse_mode == 1) {
    const size_t sm = sizeof(T) * (size_t)h->nc;
    k_trsv_lower<T><<<1, 1024, sm, s>>>(Lfac<T>(h), h->ncp, r, (int)h->nc, (T*)h->ctmp);
    k_trsv_lower_t<T><<<1, 1024, sm, s>>>(Lfac<T>(h), h->ncp, (const T*)h->ctmp, (int)h->nc, x);
    CK(cudaGetLastError());
    return 2;
  }
  k_dense_gemv<T><<<grid_for(h->nc * 32), 256, 0, s>>>(Ainv<T>(h), h->ncp, r, h->nc, x);
  CK(cudaGetLastError());
  return 1;
}

template <typename T>
const T* Dinv(const Level& L) {
  if constexpr (sizeof(T) == 8) return (const T*)L.dinv64; else return (const T*)L.dinv32;
}

// Runs the V-cycle on the level vectors.  On entry level 0 holds x = 0, r = b,
// d[0] = D^{-1} b / theta.  Returns the d buffer of level 0 holding the last update:
// the result is z = x_0 + d.
template <typename T>
T* vcycle_body_batch(r3mg_hierarchy* h, bool capturing);

template <typename T>
T* vcycle_body(r3mg_hierarchy* h, bool capturing = false) {
  if (!h->bl.empty()) return vcycle_body_batch<T>(h, capturing);
  cudaStream_t s = h->stream;
  const int L = h->L;
  std::vector<int> cur(L, 0);
  int64_t nk = 0;
  h->slot_next = 0;
  for (int l = 0; l < L - 1; ++l) {
    Level& A = h->lv[l];
    T* x = (T*)A.x; T* r = (T*)A.r;
    for (auto& ac : A.pre) {
      T* d = (T*)A.d[cur[l]]; T* dn = (T*)A.d[cur[l] ^ 1];
      const int ps = prof_begin(h, 1 + l, capturing);
      level_cheb<T>(h, A, x, r, d, dn, Dinv<T>(A), (T)ac.first, (T)ac.second);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
    Level& C = h->lv[l + 1];
    const bool coarsest = (l + 1 == L - 1);
    NextInit<T> nx{(T*)C.r, coarsest ? nullptr : (T*)C.x, coarsest ? nullptr : (T*)C.d[0], Dinv<T>(C), (T)C.c0};
    if (l == 0)
      k_restrict_fine<T, NextInit<T>><<<(int)std::min<int64_t>(C.nbox, 148 * 64), 256, 0, s>>>(Pmat<T>(h, 0), r, A.box_row, C.nbox, h->b, nx);
    else
      k_restrict_coarse_box<T, NextInit<T>><<<(int)std::min<int64_t>(C.nbox, (int64_t)h->nsm * 8), 256,
                                              sizeof(T) * h->fan * h->b, s>>>(Pmat<T>(h, l), r, C.nbox, h->b, h->fan, nx);
    CK(cudaGetLastError());
    ++nk;
  }
  {
    Level& C = h->lv[L - 1];
    nk += coarsest_apply<T>(h, (const T*)C.r, (T*)C.x);
  }
  for (int l = L - 2; l >= 0; --l) {
    Level& A = h->lv[l];
    Level& C = h->lv[l + 1];
    const bool coarsest = (l + 1 == L - 1);
    const T* x1 = (const T*)C.x;
    const T* d1 = coarsest ? nullptr : (const T*)C.d[cur[l + 1]];
    T* d = (T*)A.d[cur[l]];
    if (l == 0)
      {
        const size_t sm = sizeof(T) * 4 * 32 * h->b;   // four warps of 32 rows
        ensure_smem((const void*)k_prolong_fine_staged<T>, sm);
        k_prolong_fine_staged<T><<<(int)std::max<int64_t>(1, std::min<int64_t>((h->n + 127) / 128, (int64_t)h->nsm * 16)),
                                   128, sm, s>>>(Pmat<T>(h, 0), h->box_of_tree, x1, d1, h->n, h->b, d);
      }
    else
      k_prolong_coarse<T><<<grid_for(A.nbox * h->b), 256, 0, s>>>(Pmat<T>(h, l), x1, d1, A.nbox, h->b, h->fan, d);
    CK(cudaGetLastError());
    ++nk;
    T* x = (T*)A.x; T* r = (T*)A.r;
    for (auto& ac : A.post) {
      T* dd = (T*)A.d[cur[l]]; T* dn = (T*)A.d[cur[l] ^ 1];
      const int ps = prof_begin(h, 1 + l, capturing);
      level_cheb<T>(h, A, x, r, dd, dn, Dinv<T>(A), (T)ac.first, (T)ac.second);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
  }
  if (capturing) h->graph_kernels = nk; else h->launches += nk;
  return (T*)h->lv[0].d[cur[0]];
}

template <typename T>
T* run_vcycle(r3mg_hierarchy* h) {
  // capture once into a CUDA graph; the buffers never move, so the graph is reusable.
  // Switching profiling on or off recaptures (event-record nodes are part of the graph).
  if (h->graph_state == 1 && h->graph_prof != h->prof_on) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_state = 0;
  }
  if (h->graph_state == 0) {
    cudaGraph_t g = nullptr;
    h->graph_slots.clear();
    bool ok = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try { vcycle_body<T>(h, true); } catch (Fail&) { ok = false; }
      if (cudaStreamEndCapture(h->stream, &g) != cudaSuccess) ok = false;
    }
    if (ok && cudaGraphInstantiate(&h->graph, g, 0) == cudaSuccess) { h->graph_state = 1; h->graph_prof = h->prof_on; }
    else { h->graph_state = -1; h->graph_slots.clear(); cudaGetLastError(); }
    if (g) cudaGraphDestroy(g);
  }
  if (h->graph_state == 1) {
    CK(cudaGraphLaunch(h->graph, h->stream));
    h->launches += h->graph_kernels;
    for (int id : h->graph_slots) h->pending.push_back(id);
    // the body is deterministic: the result sits in d[(pre + post) % 2] of level 0
    const int steps0 = !h->bl.empty() ? h->bl[0].npre + h->bl[0].npost
                                    : (int)(h->lv[0].pre.size() + h->lv[0].post.size());
    return (T*)h->lv[0].d[steps0 & 1];
  }
  return vcycle_body<T>(h);
}

template <typename T>
void vcycle_apply(r3mg_hierarchy* h, const double* r_tree, double* z_tree, bool use_graph = true) {
  Level& F = h->lv[0];
  if (!h->bl.empty())
    k_bvc_init<T><<<grid_for(h->n), 256, 0, h->stream>>>(r_tree, h->n, (T*)F.r, (T*)F.x, (T*)F.d[0], Dinv<T>(F),
                                                         h->bl[0].c0, h->bl[0].rprob);
  else
    k_vc_init<T><<<grid_for(h->n), 256, 0, h->stream>>>(r_tree, h->n, (T*)F.r, (T*)F.x, (T*)F.d[0], Dinv<T>(F), (T)F.c0);
  CK(cudaGetLastError());
  T* d = use_graph ? run_vcycle<T>(h) : vcycle_body<T>(h);
  k_vc_final_dot<T><<<grid_for(h->n), 256, 0, h->stream>>>((const T*)F.x, d, z_tree, nullptr, h->n, nullptr);
  CK(cudaGetLastError());
  h->launches += 2;
}

// ---------------------------------------------------------------- setup
void lanczos(r3mg_hierarchy* h, int l) {
  Level& A = h->lv[l];
  const int64_t n = A.n;
  cudaStream_t s = h->stream;
  double *r = h->cr, *z = h->cz, *p = h->cp, *q = h->cq;
  const int gv = grid_for(n);
  k_splitmix_vec<<<gv, 256, 0, s>>>(h->prm.seed + (uint64_t)l, l == 0 ? h->perm : nullptr, r, n);
  k_jacobi_dot<<<gv, 256, 0, s>>>(A.dinv64, r, z, n, h->part_a);
  CK(cudaGetLastError());
  double rz = reduce_read(h, h->part_a, gv, S_TMP);
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  std::vector<double> al, be;
  const int steps = (int)std::min<int64_t>(h->prm.lanczos_steps, n);
  for (int j = 0; j < steps; ++j) {
    const int npq = level_apply_dot<double>(h, A, p, q, p, h->part_a);
    const double pq = reduce_read(h, h->part_a, npq, S_TMP);
    const double alpha = rz / pq;
    k_axpy<<<gv, 256, 0, s>>>(-alpha, q, r, n);
    k_jacobi_dot<<<gv, 256, 0, s>>>(A.dinv64, r, z, n, h->part_a);
    CK(cudaGetLastError());
    const double rzn = reduce_read(h, h->part_a, gv, S_TMP);
    al.push_back(alpha);
    const double beta = rzn / rz;
    be.push_back(beta);
    if (rzn == 0.0) break;
    k_xpay<<<gv, 256, 0, s>>>(z, beta, p, n);
    CK(cudaGetLastError());
    rz = rzn;
  }
  const int k = (int)al.size();
  std::vector<double> dg(k), off(k > 0 ? k - 1 : 0);
  for (int j = 0; j < k; ++j) {
    dg[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < k) off[j] = std::sqrt(be[j]) / al[j];
  }
  const double lmax = tridiag_max_eig(dg, off);
  if (!(lmax > 0.0) || !std::isfinite(lmax)) throw Fail{R3MG_E_NOT_SPD, "Lanczos estimate non-positive on level " + std::to_string(l)};
  if ((int)h->ritz.size() < h->L) h->ritz.resize(h->L, 0.0);
  h->ritz[l] = lmax;
  A.lam_hi = h->prm.eig_safety * lmax;
  A.lam_lo = A.lam_hi / h->prm.eig_ratio;
  make_schedule(A, h->prm.cheb_degree, h->prm.sweeps);
}

// Dense Cholesky, triangular inverse and symmetric inverse of the boxes [B0, B0 + nbox) of the
// coarsest block level, written to out (ncp x ncp, leading dimension ncp, identity padding).
void dense_block(r3mg_hierarchy* h, Level& C, int64_t B0, int64_t nbox, double* out, int64_t ncp,
                 double* keep_factor = nullptr) {
  cudaStream_t s = h->stream;
  const int64_t nc = nbox * h->b;
  const int nb = (int)(ncp / kTile);
  double* D = dalloc<double>(h, ncp * ncp);
  double* Li = dalloc<double>(h, ncp * ncp);
  CK(cudaMemsetAsync(D, 0, sizeof(double) * ncp * ncp, s));
  CK(cudaMemsetAsync(Li, 0, sizeof(double) * ncp * ncp, s));
  std::vector<double> one(1, 1.0);
  for (int64_t i = nc; i < ncp; ++i) CK(cudaMemcpyAsync(D + i * ncp + i, one.data(), sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  k_blocks_to_dense<<<(int)std::min<int64_t>(nc, 65535), 256, 0, s>>>(C.nbr_ptr, C.nbr, C.row_ptr, C.v64, nbox, h->b, D, ncp, B0);
  CK(cudaGetLastError());
  for (int k = 0; k < nb; ++k) {
    k_potrf_diag<<<1, 256, 0, s>>>(D, ncp, k, Li, h->status);
    if (nb - k - 1 > 0) {
      k_trsm_panel<<<nb - k - 1, 256, 0, s>>>(D, ncp, k, Li);
      const int m = nb - k - 1;
      k_syrk_update<<<m * (m + 1) / 2, 256, 0, s>>>(D, ncp, k, nb);
    }
    CK(cudaGetLastError());
  }
  int st = 0;
  read_status(h, st);
  if (st) throw Fail{R3MG_E_NOT_SPD, "coarsest level: Cholesky pivot <= 0 (A_c not SPD)"};
  for (int t = 1; t < nb; ++t) {
    k_trtri_step<<<nb - t, 256, 0, s>>>(D, Li, ncp, t, nb);
    CK(cudaGetLastError());
  }
  k_lauum<<<nb * (nb + 1) / 2, 256, 0, s>>>(Li, out, ncp, nb);
  CK(cudaGetLastError());
  // the factor itself (lower triangle of D) for the substitution form of the coarsest solve
  if (keep_factor) CK(cudaMemcpyAsync(keep_factor, D, sizeof(double) * ncp * ncp, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaFree(D)); CK(cudaFree(Li));
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)D), h->allocs.end());
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)Li), h->allocs.end());
}

void dense_coarsest(r3mg_hierarchy* h) {
  Level& C = h->lv[h->L - 1];
  if (!h->Ainv64) h->Ainv64 = dalloc<double>(h, h->ncp * h->ncp);
  if (!h->L64) h->L64 = dalloc<double>(h, h->ncp * h->ncp);
  dense_block(h, C, 0, C.nbox, h->Ainv64, h->ncp, h->L64);
}

// Autotuner: times one fused level step (or the FP64 product for the fine level of the mixed
// solver) for every candidate kernel shape and keeps the fastest.  Candidates: the
// register-streamed kernel with 4..32 lanes per row, and the TMA-streamed kernel with 8..32
// lanes per row and 256, 512 or 1024 threads per CTA.
template <typename T>
void autotune_level(r3mg_hierarchy* h, Level& A, bool product) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  cudaStream_t s = h->stream;
  T *x, *r, *d, *dn;
  if (product) { x = (T*)h->cb; r = (T*)h->cz; d = (T*)h->cp; dn = nullptr; }
  else { x = (T*)A.x; r = (T*)A.r; d = (T*)A.d[0]; dn = (T*)A.d[1]; }
  const int64_t nb = A.n * (int64_t)sizeof(T);
  CK(cudaMemsetAsync(x, 0, nb, s)); CK(cudaMemsetAsync(r, 0, nb, s)); CK(cudaMemsetAsync(d, 0, nb, s));
  if (dn) CK(cudaMemsetAsync(dn, 0, nb, s));
  const bool fine = (A.b == 0);
  std::vector<Level::KConf> cand;
  for (int G : {2, 4, 8, 16, 32}) {
    if (G == 2 && !(fine && sizeof(T) == 8)) continue;
    if (fine && G == 32) continue;
    if (!fine && G < 8 && sizeof(T) == 4) continue;   // coarse FP32 rows keep 16-byte loads per 8+ lanes
    for (int nt : {128, 256})
      for (int u : {0, 4}) {
        if (nt / G < 2) continue;
        if (u == 4 && sizeof(T) != 8) continue;   // deeper unroll is an FP64 option
        cand.push_back({0, G, nt, 0.f, u});
        if (2 * level_smem_bytes(view<T>(A)) <= kMaxSmem) cand.push_back({2, G, nt, 0.f, u});
        cand.push_back({3, G, nt, 0.f, u});
        if (u == 0) { cand.push_back({5, G, nt, 0.f, 0}); cand.push_back({6, G, nt, 0.f, 0}); }
      }
    if (A.tma[pi].nitems > 0)
      for (int nt : {256, 512, 1024}) if (G >= 8) cand.push_back({1, G, nt, 0.f, 0});
    if (sizeof(T) == 4 && A.sym_ok && G == 16 && !product) {
      cand.push_back({4, G, 128, 0.f, 0});
      cand.push_back({4, 4, 128, 0.f, 0});   // symmetric form with 4-row load waves
      cand.push_back({4, G, 96, 0.f, 0});    // ... with 96 threads (no idle column group at b = 27)
      cand.push_back({4, 4, 96, 0.f, 0});
      for (int cps : {2, 3, 4, 5})   // staged form: the lanes field holds the resident CTAs per SM
        if (sym_stage_cap(A, cps) > 0) cand.push_back({7, cps, 128, 0.f, 0});
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  Level::KConf best = A.conf[pi];
  float best_ms = 1e30f;
  for (auto& c : cand) {
    A.conf[pi] = c;
    auto once = [&] {
      if (product) level_apply_dot<T>(h, A, x, r, d, h->part_a);
      else level_cheb<T>(h, A, x, r, d, dn, Dinv<T>(A), T(0), T(0));
    };
    once();
    CK(cudaEventRecord(e0, s));
    for (int k = 0; k < 3; ++k) once();
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 3.f;
    if (ms < best_ms) { best_ms = ms; best = c; best.ms = ms; }
  }
  CK(cudaEventDestroy(e0)); CK(cudaEventDestroy(e1));
  A.conf[pi] = best;
  int terr = 0;
  CK(cudaMemcpy(&terr, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (terr) throw Fail{R3MG_E_TIMEOUT, "autotuner: a bounded wait of the TMA-streamed kernel expired"};
}

// Numeric setup from CSR values on the device (setup and r3mg_update_values).
void lanczos_batch(r3mg_hierarchy* h, int l);
void dense_batch(r3mg_hierarchy* h);
template <typename T>
T* vcycle_body_batch(r3mg_hierarchy* h, bool capturing);

// Captured graphs hold the Chebyshev coefficients, c0 and kernel configurations as launch
// arguments: drop them whenever those change; the next solve recaptures.
void drop_graphs(r3mg_hierarchy* h) {
  if (h->pgraph) cudaGraphExecDestroy(h->pgraph);
  h->pgraph = nullptr;
  h->pgraph_state = 0;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  if (h->lgraph) cudaGraphExecDestroy(h->lgraph);
  if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
  h->graph = h->bgraph = h->lgraph = h->mgraph = nullptr;
  h->graph_state = h->bgraph_state = h->lgraph_state = h->mgraph_state = 0;
}

void mr_regroup(r3mg_hierarchy* h);

void numeric(r3mg_hierarchy* h, const double* vals_dev) {
  cudaStream_t s = h->stream;
  CK(cudaStreamSynchronize(s));
  drop_graphs(h);
  Level& F = h->lv[0];
  k_gather_vals<<<grid_for(F.stored), 256, 0, s>>>(h->src, vals_dev, F.v64, F.stored);
  k_dinv_fine<<<grid_for(h->n), 256, 0, s>>>(h->diag_src, vals_dev, F.dinv64, h->n, h->status);
  CK(cudaGetLastError());
  int st = 0;
  read_status(h, st);
  if (st) throw Fail{R3MG_E_NOT_SPD, "fine level: non-positive or non-finite diagonal entry"};
  const int b = h->b;
  // Galerkin products, level by level
  {
    Level& C = h->lv[1];
    const size_t sm = sizeof(double) * 2 * kRapRows * b;
    k_rap_fine<<<(int)std::min<int64_t>(C.npairs, 1 << 30), 256, sm, s>>>(
        F.pair_box, F.nbr_ptr, F.nbr, F.win_off, F.slot_src, F.win_size, F.box_row, F.row_ptr, F.idx, F.v64, h->P64[0], b,
        F.npairs, C.row_ptr,
        C.v64);
    CK(cudaGetLastError());
  }
  for (int l = 1; l + 1 < h->L; ++l) {
    Level& A = h->lv[l];
    Level& C = h->lv[l + 1];
    const size_t sm = sizeof(double) * 4 * b * b;
    if (sm > 48 * 1024) CK(cudaFuncSetAttribute(k_rap_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_rap_coarse<<<(int)std::min<int64_t>(C.npairs, 1 << 30), 256, sm, s>>>(
        C.pair_box, C.nbr_ptr, C.nbr, A.nbr_ptr, A.nbr, A.row_ptr, A.v64, h->P64[l], b, h->fan, C.npairs, C.row_ptr, C.v64);
    CK(cudaGetLastError());
  }
  for (int l = 1; l < h->L; ++l) {
    Level& A = h->lv[l];
    k_dinv_coarse<<<grid_for(A.n), 256, 0, s>>>(A.nbr_ptr, A.nbr, A.row_ptr, A.v64, A.dinv64, A.nbox, b, h->status);
    CK(cudaGetLastError());
  }
  read_status(h, st);
  if (st) throw Fail{R3MG_E_NOT_SPD, "coarse level: non-positive diagonal entry"};
  if (!h->bl.empty()) {
    for (int l = 0; l + 1 < h->L; ++l) lanczos_batch(h, l);
    dense_batch(h);
  } else {
    for (int l = 0; l + 1 < h->L; ++l) lanczos(h, l);
    dense_coarsest(h);
  }
  if (h->prm.precision == 1) {
    for (int l = 0; l < h->L; ++l) {
      Level& A = h->lv[l];
      if (l + 1 < h->L) {
        k_convert<double, float><<<grid_for(A.stored), 256, 0, s>>>(A.v64, A.v32, A.stored);
        k_convert<double, float><<<grid_for(A.n), 256, 0, s>>>(A.dinv64, A.dinv32, A.n);
      }
    }
    for (int l = 1; l + 1 < h->L; ++l) {
      Level& A = h->lv[l];
      if (!A.sym_ok) continue;
      k_sym_gather<<<(int)std::min<int64_t>(A.n, 1 << 20), 128, 0, s>>>(A.sym, A.row_ptr, A.v32, A.sym_vals);
      CK(cudaGetLastError());
    }
    const int64_t na = !h->bl.empty() ? h->batch_ainv_size : h->ncp * h->ncp;
    k_convert<double, float><<<grid_for(na), 256, 0, s>>>(h->Ainv64, h->Ainv32, na);
    CK(cudaGetLastError());
    if (h->L64) {
      if (!h->L32) h->L32 = dalloc<float>(h, h->ncp * h->ncp);
      k_convert<double, float><<<grid_for(h->ncp * h->ncp), 256, 0, s>>>(h->L64, h->L32, h->ncp * h->ncp);
      CK(cudaGetLastError());
    }
  }
  mr_regroup(h);   // the grouped fine level's own copy of the values, if the block path built one
  CK(cudaStreamSynchronize(s));
}

// Host analysis of one problem: CSR checks, R-tree partition, admissibility, block adjacency
// of every level and the fine windowed layout.
struct ProbHost {
  HostPartition P;
  std::vector<HostPattern> pats;
  HostFineLayout lay;
  double hmax = 0.0;   // largest distance between two coupled support points (the mesh size h)
};

// Cells of a problem for cell-based agglomeration (null: point-based).
struct CellsIn {
  int64_t ncells;
  const int64_t* ptr;
  const int64_t* pts;
};

void analyse_problem(const r3mg_params& prm, int dim, int b, int fan, int64_t n, const double* coords,
                     const int64_t* rowptr, const int32_t* colidx, const double* vals, ProbHost& out,
                     const CellsIn* cells = nullptr) {
  Error err;
  if (!validate_csr(n, rowptr, colidx, err)) throw Fail{err.status, err.msg};
  for (int64_t k = 0; k < rowptr[n]; ++k)
    if (!std::isfinite(vals[k])) throw Fail{R3MG_E_ARG, "CSR: non-finite value"};
  if (cells) {
    if (!partition_cells(n, dim, coords, cells->ncells, cells->ptr, cells->pts, prm.leaf_size, prm.levels, out.P, err))
      throw Fail{err.status, err.msg};
  } else if (!partition_points(n, dim, coords, prm.leaf_size, prm.levels, out.P, err)) {
    throw Fail{err.status, err.msg};
  }
  HostPartition& P = out.P;
  const int L = prm.levels;
  // admissibility (Section 4, Remark on (m, M)): enough points and non-degenerate boxes
  for (int64_t B = 0; B < P.nbox(1); ++B) {
    if (P.box_off[1][B + 1] - P.box_off[1][B] < b)
      throw Fail{R3MG_E_UNISOLVENT, "level-1 box " + std::to_string(B) + " owns fewer points than (p'+1)^d"};
  }
  if (prm.pprime >= 1)
    for (int l = 1; l < L; ++l)
      for (int64_t B = 0; B < P.nbox(l); ++B)
        for (int a = 0; a < dim; ++a)
          if (!(P.hi[l][B * dim + a] > P.lo[l][B * dim + a]))
            throw Fail{R3MG_E_UNISOLVENT, "level-" + std::to_string(l) + " box " + std::to_string(B) + " has zero extent"};
  out.pats.assign(L, HostPattern());
  fine_pattern(P, rowptr, colidx, out.pats[1]);
  for (int l = 2; l < L; ++l) coarse_pattern(out.pats[l - 1], fan, P.nbox(l), out.pats[l]);
  if (!fine_layout(P, out.pats[1], rowptr, colidx, out.lay, err)) throw Fail{err.status, err.msg};
  out.hmax = max_coupled_distance(n, dim, coords, rowptr, colidx);
}

void batch_levels_upload(r3mg_hierarchy* h);

// Device structures and numeric setup from the (possibly concatenated) host analysis.
//   coords: caller-numbered coordinates (h->n x dim); rowptr/colidx: the caller's CSR when the
//   adjoint product is wanted (single problems), else null; vals: pieces of the caller's CSR
//   values in order (one per problem).
void build_device(r3mg_hierarchy* h, std::vector<HostPattern>& pats, HostFineLayout& lay, const double* coords,
                  const int64_t* rowptr, const int32_t* colidx,
                  const std::vector<std::pair<const double*, int64_t>>& vals) {
  const r3mg_params& prm = h->prm;
  const int dim = h->dim;
  cudaStream_t s = h->stream;
  const int b = h->b;
  HostPartition& P = h->part;
  const int L = prm.levels;
  h->L = L;
  h->lv.assign(L, Level());
  // H: the largest diameter (MBR diagonal) of a coarsest-level box
  h->H_coarse = 0.0;
  for (int64_t B = 0; B < P.nbox(L - 1); ++B) {
    double s2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double e = P.hi[L - 1][B * dim + a] - P.lo[L - 1][B * dim + a];
      s2 += e * e;
    }
    h->H_coarse = std::max(h->H_coarse, std::sqrt(s2));
  }
  h->nnz_csr = 0;
  for (auto& pc : vals) h->nnz_csr += pc.second;
  // ---- fine level
  {
    Level& F = h->lv[0];
    F.n = h->n; F.nbox = P.nbox(1); F.b = 0;
    F.box_row = upload(h, P.box_off[1]);
    F.nbr_ptr = upload(h, pats[1].ptr);
    F.nbr = upload(h, pats[1].nbr);
    F.win_off = upload(h, lay.win_off);
    F.win_size = upload(h, lay.win_size);
    std::vector<int64_t> ss(pats[1].nbr.size()), pb(pats[1].nbr.size());
    int ms = 0;
    for (int64_t B = 0; B < F.nbox; ++B) {
      ms = std::max<int>(ms, (int)(pats[1].ptr[B + 1] - pats[1].ptr[B]));
      for (int64_t e = pats[1].ptr[B]; e < pats[1].ptr[B + 1]; ++e) { ss[e] = lay.win_src[e]; pb[e] = B; }
    }
    F.slot_src = upload(h, ss);
    F.pair_box = upload(h, pb);
    F.npairs = (int64_t)pb.size();
    F.max_slots = ms;
    F.win_max = (lay.win_max + 3) & ~3;
    std::vector<int32_t> ord(h->n);
    for (int64_t B = 0; B < F.nbox; ++B) {
      const int64_t r0 = P.box_off[1][B], r1 = P.box_off[1][B + 1];
      F.max_box_rows = std::max<int>(F.max_box_rows, (int)(r1 - r0));
      for (int64_t k = r0; k < r1; ++k) ord[k] = (int32_t)(k - r0);
      std::stable_sort(ord.begin() + r0, ord.begin() + r1, [&](int32_t a, int32_t c) {
        return lay.row_ptr[r0 + a + 1] - lay.row_ptr[r0 + a] > lay.row_ptr[r0 + c + 1] - lay.row_ptr[r0 + c];
      });
    }
    F.row_order = upload(h, ord);
    F.row_ptr = upload(h, lay.row_ptr);

    lay.idx.resize(lay.idx.size() + 16, 0);   // bulk copies of index runs round up to 16 bytes
    F.idx = upload(h, lay.idx);
    F.stored = lay.row_ptr[h->n];
    F.nnz = lay.nnz;
    F.v64 = dalloc<double>(h, F.stored);
    F.dinv64 = dalloc<double>(h, F.n);
    F.pat = pats[1];
    for (auto& c : F.conf) {
      c.G = prm.group_lanes ? prm.group_lanes : auto_lanes((double)F.nnz / (double)F.n);
      c.form = (prm.kernel_form == 2) ? 1 : 0;
      c.nt = 512;
    }
    F.h_box_row = P.box_off[1];
    F.h_win_size = lay.win_size;
    F.use_tma = (prm.kernel_form != 1) && h->bl.empty();
    if (F.use_tma) build_items(h, F, 0, lay.row_ptr, lay.win_off, ss);
    if (F.use_tma && prm.precision == 1) build_items(h, F, 1, lay.row_ptr, lay.win_off, ss);
    h->src = upload(h, lay.src);
    h->diag_src = upload(h, lay.diag_src);
    h->perm = upload(h, P.perm);
    std::vector<int32_t> bot(h->n);
    for (int64_t B = 0; B < F.nbox; ++B)
      for (int64_t k = P.box_off[1][B]; k < P.box_off[1][B + 1]; ++k) bot[k] = (int32_t)B;
    h->box_of_tree = upload(h, bot);
    std::vector<double> ct(h->n * dim);
    for (int64_t k = 0; k < h->n; ++k)
      for (int a = 0; a < dim; ++a) ct[k * dim + a] = coords[P.perm[k] * dim + a];
    h->coords_tree = upload(h, ct);
  }
  // ---- coarse levels (block layout)
  for (int l = 1; l < L; ++l) {
    Level& C = h->lv[l];
    const HostPattern& pt = pats[l];
    C.nbox = P.nbox(l); C.b = b; C.n = C.nbox * b;
    C.pat = pt;
    C.nbr_ptr = upload(h, pt.ptr);
    C.nbr = upload(h, pt.nbr);
    std::vector<int64_t> rp(C.n + 1, 0), pb(pt.nbr.size());
    int ms = 0;
    for (int64_t B = 0; B < C.nbox; ++B) {
      const int64_t nn = pt.ptr[B + 1] - pt.ptr[B];
      ms = std::max<int>(ms, (int)nn);
      const int64_t len = (nn * b + kPad - 1) / kPad * kPad;
      for (int q = 0; q < b; ++q) rp[B * b + q + 1] = rp[B * b + q] + len;
      for (int64_t e = pt.ptr[B]; e < pt.ptr[B + 1]; ++e) pb[e] = B;
    }
    C.row_ptr = upload(h, rp);
    C.pair_box = upload(h, pb);
    C.npairs = (int64_t)pb.size();
    C.max_slots = ms;
    C.win_max = (ms * b + 3) & ~3;
    C.max_box_rows = b;
    C.stored = rp[C.n];
    C.nnz = (int64_t)pt.nbr.size() * b * b;
    C.v64 = dalloc<double>(h, C.stored);
    CK(cudaMemsetAsync(C.v64, 0, sizeof(double) * C.stored, s));
    C.dinv64 = dalloc<double>(h, C.n);
    for (auto& c : C.conf) {
      c.G = prm.group_lanes ? prm.group_lanes : auto_lanes((double)C.nnz / (double)C.n);
      c.form = (prm.kernel_form == 2) ? 1 : 0;
      c.nt = 512;
    }
    C.use_tma = (prm.kernel_form != 1) && h->bl.empty();
    if (prm.precision == 1 && l + 1 < L) { C.h_row_ptr = rp; build_sym(h, C); }
    if (C.use_tma) build_items(h, C, 0, rp, {}, {});
    if (C.use_tma && prm.precision == 1 && l + 1 < L) build_items(h, C, 1, rp, {}, {});
  }
  for (auto& A : h->lv) A.nsm = h->nsm;
  // ---- transfers (geometry only: computed once)
  GLLTable g{};
  g.pp = prm.pprime;
  gll_nodes01(prm.pprime, g.z);
  h->P64.assign(L - 1, nullptr);
  h->P32.assign(L - 1, nullptr);
  {
    std::vector<double> lo = P.lo[1], hi = P.hi[1];
    double* dlo = upload(h, lo); double* dhi = upload(h, hi);
    h->P64[0] = dalloc<double>(h, h->n * b);
    k_p0_eval<<<grid_for(h->n * b), 256, 0, s>>>(h->coords_tree, h->box_of_tree, dlo, dhi, g, dim, b, h->P64[0], h->n);
    CK(cudaGetLastError());
    if (prm.pprime >= 1) {
      k_unisolvent<<<(int)std::min<int64_t>(P.nbox(1), 148 * 16), 128, sizeof(double) * b * b, s>>>(
          h->P64[0], h->lv[0].box_row, P.nbox(1), b, h->status);
      CK(cudaGetLastError());
      int st = 0;
      read_status(h, st);
      if (st) throw Fail{R3MG_E_UNISOLVENT, "a level-1 box's points cannot carry Q^{p'} (rank-deficient evaluation)"};
    }
  }
  for (int l = 1; l + 1 < L; ++l) {
    double* lc = upload(h, P.lo[l]); double* hc = upload(h, P.hi[l]);
    double* lp = upload(h, P.lo[l + 1]); double* hp = upload(h, P.hi[l + 1]);
    h->P64[l] = dalloc<double>(h, P.nbox(l) * b * b);
    k_ptilde_eval<<<grid_for(P.nbox(l) * b * b), 256, 0, s>>>(lc, hc, lp, hp, g, dim, b, h->fan, h->P64[l], P.nbox(l));
    CK(cudaGetLastError());
  }
  // ---- coarsest and Krylov work space
  h->nc = h->lv[L - 1].n;
  h->ncp = (h->nc + kTile - 1) / kTile * kTile;
  int64_t np = kVecBlocks;
  for (int l = 0; l < L; ++l) np = std::max(np, h->lv[l].nbox);
  np = std::max<int64_t>(np, 148 * 32);
  h->npart = np;
  h->part_a = dalloc<double>(h, np);
  h->part_b = dalloc<double>(h, np);
  h->scal = dalloc<double>(h, kScalTotal);
  CK(cudaMemsetAsync(h->scal, 0, sizeof(double) * kScalTotal, s));
  int64_t nmax = h->n;
  for (int l = 1; l < L; ++l) nmax = std::max(nmax, h->lv[l].n);
  h->cx = dalloc<double>(h, nmax); h->cr = dalloc<double>(h, nmax); h->cp = dalloc<double>(h, nmax);
  h->cq = dalloc<double>(h, nmax); h->cz = dalloc<double>(h, nmax); h->cb = dalloc<double>(h, nmax);
  // V-cycle vectors in the V-cycle precision
  const size_t es = prm.precision == 1 ? sizeof(float) : sizeof(double);
  for (int l = 0; l < L; ++l) {
    Level& A = h->lv[l];
    A.x = dalloc<char>(h, A.n * es);
    A.r = dalloc<char>(h, A.n * es);
    if (l + 1 < L) { A.d[0] = dalloc<char>(h, A.n * es); A.d[1] = dalloc<char>(h, A.n * es); }
  }
  if (prm.precision == 1) {
    for (int l = 0; l < L; ++l) {
      Level& A = h->lv[l];
      if (l + 1 < L) { A.v32 = dalloc<float>(h, A.stored); A.dinv32 = dalloc<float>(h, A.n); }
    }
    for (int l = 0; l + 1 < L; ++l) {
      const int64_t m = (l == 0) ? h->n * b : P.nbox(l) * b * b;
      h->P32[l] = dalloc<float>(h, m);
      k_convert<double, float><<<grid_for(m), 256, 0, s>>>(h->P64[l], h->P32[l], m);
    }
    h->Ainv32 = dalloc<float>(h, !h->bl.empty() ? h->batch_ainv_size : h->ncp * h->ncp);
    CK(cudaGetLastError());
  }
  // ---- shared-memory limits of the level kernels
  for (int l = 0; l + 1 < L; ++l) {
    const size_t es2 = prm.precision == 1 ? sizeof(float) : sizeof(double);
    const Level& A = h->lv[l];
    const size_t need = std::max(level_smem_bytes(view<double>(A)),
                                 es2 * (size_t)A.win_max + 12 * (size_t)(A.max_slots + 2));
    if (need > kMaxSmem)
      throw Fail{R3MG_E_LIMIT, "level " + std::to_string(l) + " window needs " + std::to_string(need) +
                                   " bytes of shared memory (> 227 KB): use a smaller leaf_size"};
  }
  // ---- the caller's CSR structure, for the sampled outer product of the adjoint
  if (rowptr && colidx) {
    h->csr_rowptr = upload(h, std::vector<int64_t>(rowptr, rowptr + h->n + 1));
    h->csr_col = upload(h, std::vector<int32_t>(colidx, colidx + h->nnz_csr));
  }
  if (!h->bl.empty()) batch_levels_upload(h);
  // ---- numeric setup from the caller's values
  double* dvals = dalloc<double>(h, h->nnz_csr);
  {
    int64_t o = 0;
    for (auto& pc : vals) {
      CK(cudaMemcpyAsync(dvals + o, pc.first, sizeof(double) * pc.second, cudaMemcpyHostToDevice, s));
      o += pc.second;
    }
  }
  numeric(h, dvals);
  CK(cudaFree(dvals));
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)dvals), h->allocs.end());
  if (prm.kernel_form == 0) {
    for (int l = 0; l + 1 < L; ++l) {
      if (prm.precision == 1) autotune_level<float>(h, h->lv[l], false);
      else autotune_level<double>(h, h->lv[l], false);
    }
    if (prm.precision == 1) autotune_level<double>(h, h->lv[0], true);   // the FP64 CG product
  }
  // one direct V-cycle so every kernel instantiation is configured before graph capture
  CK(cudaMemsetAsync(h->cb, 0, sizeof(double) * h->n, s));
  if (prm.precision == 1) vcycle_apply<float>(h, h->cb, h->cz, false);
  else vcycle_apply<double>(h, h->cb, h->cz, false);
  CK(cudaStreamSynchronize(s));
}

void build(r3mg_hierarchy* h, const double* coords, const int64_t* rowptr, const int32_t* colidx, const double* vals,
           const CellsIn* cells = nullptr) {
  const r3mg_params& prm = h->prm;
  h->b = 1;
  for (int a = 0; a < h->dim; ++a) h->b *= (prm.pprime + 1);
  h->fan = 1 << h->dim;
  ProbHost ph;
  analyse_problem(prm, h->dim, h->b, h->fan, h->n, coords, rowptr, colidx, vals, ph, cells);
  h->part = std::move(ph.P);
  h->h_fine = ph.hmax;
  build_device(h, ph.pats, ph.lay, coords, rowptr, colidx, {{vals, rowptr[h->n]}});
}

template <typename F>
r3mg_status guarded(r3mg_hierarchy* h, F&& f) {
  try {
    f();
    return R3MG_OK;
  } catch (Fail& e) {
    if (h) h->err = e.msg;
    g_last_error = e.msg;
    return e.st;
  } catch (std::bad_alloc&) {
    if (h) h->err = "host allocation failed";
    g_last_error = "host allocation failed";
    return R3MG_E_OOM;
  }
}

struct StreamJoin {  // run the hierarchy's work after the caller's stream, and vice versa
  r3mg_hierarchy* h;
  cudaStream_t user;
  StreamJoin(r3mg_hierarchy* hh, void* st) : h(hh), user((cudaStream_t)st) {
    CK(cudaEventRecord(h->ev_in, user));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  }
  ~StreamJoin() {
    if (cudaEventRecord(h->ev_out, h->stream) == cudaSuccess) cudaStreamWaitEvent(user, h->ev_out, 0);
  }
};

// Capture one CG/FCG iteration into a WHILE-loop graph (see krylov); lgraph_state -1 on failure,
// after which solves use the host-driven loop.
template <typename T>
void build_loop_graph(r3mg_hierarchy* h) {
  cudaStream_t s = h->stream;
  Level& F = h->lv[0];
  const int64_t n = h->n;
  const bool fcg = (h->prm.precision == 1);
  const int gv = grid_for(n);
  if (!h->d_its) h->d_its = dalloc<int>(h, 1);
  if (!h->d_loop) h->d_loop = dalloc<double>(h, 2);
  cudaGraph_t g = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle wh{}, ih{};
  cudaGraph_t body = nullptr, rest = nullptr;
  if (ok) ok = cudaGraphConditionalHandleCreate(&wh, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = wh;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    ok = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp) == cudaSuccess;
    if (ok) body = wp.conditional.phGraph_out[0];
  }
  if (ok) ok = cudaGraphConditionalHandleCreate(&ih, body, 0, 0) == cudaSuccess;
  if (ok) ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    bool cap_ok = true;
    try {
      const int nb0 = level_apply_dot<double>(h, F, h->cp, h->cq, h->cp, h->part_a);
      reduce_dev(h, h->part_a, nb0, S_PQ, fcg ? FIN_ALPHA_FCG : FIN_ALPHA_PCG);
      k_cg_update<T><<<gv, 256, 0, s>>>(h->cx, h->cr, h->cp, h->cq, h->scal, n, h->part_a, (T*)F.r, (T*)F.x,
                                        (T*)F.d[0], Dinv<T>(F), (T)F.c0);
      CK(cudaGetLastError());
      reduce_dev(h, h->part_a, gv, S_RR, FIN_NONE);
      k_converge1<<<1, 32, 0, s>>>(h->scal, h->d_loop, h->d_its, h->status, wh, ih);
      CK(cudaGetLastError());
      cudaStreamCaptureStatus cs;
      cudaGraph_t capg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, nullptr, &nd));
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = ih;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t inode;
      CK(cudaGraphAddNode(&inode, capg, deps, nullptr, nd, &ip));
      rest = ip.conditional.phGraph_out[0];
      CK(cudaStreamUpdateCaptureDependencies(s, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    } catch (Fail&) { cap_ok = false; }
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(s, &out) != cudaSuccess || !cap_ok) ok = false;
  }
  if (ok) ok = cudaStreamBeginCaptureToGraph(s, rest, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    bool cap_ok = true;
    try {
      T* d = vcycle_body<T>(h, true);
      k_vc_final_dot<T><<<gv, 256, 0, s>>>((const T*)F.x, d, h->cz, fcg ? h->cq : h->cr, n, h->part_a);
      CK(cudaGetLastError());
      reduce_dev(h, h->part_a, gv, fcg ? S_ZQ : S_RZNEW, fcg ? FIN_BETA_FCG : FIN_BETA_PCG);
      k_p_update<<<gv, 256, 0, s>>>(h->cp, h->cz, h->cr, h->scal, n, fcg ? 1 : 0, fcg ? h->part_a : nullptr);
      CK(cudaGetLastError());
      if (fcg) reduce_dev(h, h->part_a, gv, S_PR, FIN_NONE);
    } catch (Fail&) { cap_ok = false; }
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(s, &out) != cudaSuccess || !cap_ok) ok = false;
  }
  if (ok) ok = cudaGraphInstantiate(&h->lgraph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  h->lgraph_state = ok ? 1 : -1;
  if (!ok) { h->lgraph = nullptr; cudaGetLastError(); }
}

// True when the n FP64 entries of x are all zero: the initial residual is then b itself, and
// the product A x0 (a full pass over the fine matrix) is skipped.
bool all_zero(r3mg_hierarchy* h, const double* x, int64_t n) {
  if (!h->d_flag) h->d_flag = dalloc<int>(h, 1);
  CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
  k_any_nonzero<<<grid_for(n), 256, 0, h->stream>>>(x, n, h->d_flag);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h->host_scal[13], h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int f = 0;
  std::memcpy(&f, &h->host_scal[13], sizeof(int));
  h->launches += 1;
  return f == 0;
}

// PCG (FP64 V-cycle) or flexible CG (FP32 V-cycle) on tree-ordered b (cb) and x (cx).
template <typename T>
r3mg_status krylov(r3mg_hierarchy* h, double rtol, int maxit, int* iters, double* relres) {
  cudaStream_t s = h->stream;
  Level& F = h->lv[0];
  const int64_t n = h->n;
  const bool fcg = (h->prm.precision == 1);
  const int gv = grid_for(n);
  auto true_residual = [&](double& rr, double* bb, bool x_zero = false) {
    // with x = 0, A x = 0 = x: the residual takes x itself in place of the product
    if (!x_zero) level_apply_dot<double>(h, F, h->cx, h->cq, nullptr, nullptr);
    k_residual<<<gv, 256, 0, s>>>(h->cb, x_zero ? h->cx : h->cq, h->cr, n, h->part_a, bb ? h->part_b : nullptr);
    CK(cudaGetLastError());
    rr = reduce_read(h, h->part_a, gv, S_RR);
    if (bb) *bb = reduce_read(h, h->part_b, gv, S_BB);
  };
  auto precondition_restart = [&]() {
    // z = M r; p = z; (PCG) rz = r.z ; (FCG) pr = p.r.  A restart begins a new Lanczos
    // sequence: the coefficient history of the condition estimate starts over.
    CK(cudaMemsetAsync(h->scal + S_NA, 0, 2 * sizeof(double), s));
    k_vc_init<T><<<gv, 256, 0, s>>>(h->cr, n, (T*)F.r, (T*)F.x, (T*)F.d[0], Dinv<T>(F), (T)F.c0);
    CK(cudaGetLastError());
    T* d = run_vcycle<T>(h);
    k_vc_final_dot<T><<<gv, 256, 0, s>>>((const T*)F.x, d, h->cz, h->cr, n, h->part_a);
    CK(cudaGetLastError());
    reduce_dev(h, h->part_a, gv, fcg ? S_PR : S_RZ, FIN_NONE);
    CK(cudaMemcpyAsync(h->cp, h->cz, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  };
  double rr = 0.0, bb = 0.0;
  CK(cudaMemsetAsync(h->scal + S_NA, 0, 2 * sizeof(double), s));   // no coefficients recorded yet
  true_residual(rr, &bb, all_zero(h, h->cx, n));
  const double bnorm = std::sqrt(bb);
  *iters = 0;
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(h->cx, 0, sizeof(double) * n, s));
    *relres = 0.0;
    return R3MG_OK;
  }
  double rel = std::sqrt(rr) / bnorm;
  *relres = rel;
  // stop when ||r|| <= max(rtol ||b||, atol, reduction ||r_0||); with atol = reduction = 0 (the
  // default) this is the relative test, with rtol = 0, atol = 1e-9, reduction = 1e-6 Section 6's
  const double thr = std::max(rtol * bnorm, std::max(h->stop_atol, h->stop_red * std::sqrt(rr)));
  const double thr2 = thr * thr;
  if (rr <= thr2) return R3MG_OK;
  precondition_restart();
  if (!h->prof_on && h->lgraph_state >= 0) {
    // The whole iteration loop as one graph launch.  A conditional WHILE node repeats one
    // iteration; inside it, the product, alpha, the x/r update and ||r||^2 run first, the stop test
    // sets both the loop condition and an IF node's condition, and the IF node holds the rest of
    // the iteration (V-cycle, beta, new direction), so the last iteration does no V-cycle.
    // Profiled solves keep the host loop below (events time each launch).
    if (h->lgraph_state == 0) build_loop_graph<T>(h);
    if (h->lgraph_state == 1) {
      int done_its = 0;
      while (done_its < maxit) {
        k_loop_init<<<1, 32, 0, s>>>(h->d_loop, h->d_its, h->status, thr2, maxit - done_its);
        CK(cudaGetLastError());
        CK(cudaGraphLaunch(h->lgraph, s));
        int its = 0, st = 0;
        CK(cudaMemcpyAsync(&h->host_scal[14], h->d_its, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&h->host_scal[15], h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::memcpy(&its, &h->host_scal[14], sizeof(int));
        std::memcpy(&st, &h->host_scal[15], sizeof(int));
        // per iteration: product, 2 or 3 reductions, update, stop test, V-cycle graph, final dot, p update
        h->launches += 1 + (int64_t)its * (h->graph_kernels + (fcg ? 8 : 7));
        if (st) {
          CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
          throw Fail{R3MG_E_BREAKDOWN, "CG breakdown: p^T A p <= 0 or non-finite scalar"};
        }
        done_its += its;
        *iters = done_its;
        double rt = 0.0;
        true_residual(rt, nullptr);
        *relres = std::sqrt(rt) / bnorm;
        if (!std::isfinite(*relres)) throw Fail{R3MG_E_BREAKDOWN, "CG breakdown: non-finite residual"};
        if (rt <= thr2) return R3MG_OK;
        if (done_its >= maxit) break;
        precondition_restart();   // recursive residual drifted: restart from the true residual
      }
      return R3MG_E_NOCONV;
    }
  }
  for (int it = 1; it <= maxit; ++it) {
    if (h->prof_on) {
      if (!h->cg_slot.e0) { CK(cudaEventCreate(&h->cg_slot.e0)); CK(cudaEventCreate(&h->cg_slot.e1)); }
      CK(cudaEventRecord(h->cg_slot.e0, s));
    }
    const int nb0 = level_apply_dot<double>(h, F, h->cp, h->cq, h->cp, h->part_a);
    if (h->prof_on) { CK(cudaEventRecord(h->cg_slot.e1, s)); h->cg_pending = true; }
    h->launches += 3;   // product, reduction, update
    reduce_dev(h, h->part_a, nb0, S_PQ, fcg ? FIN_ALPHA_FCG : FIN_ALPHA_PCG);
    k_cg_update<T><<<gv, 256, 0, s>>>(h->cx, h->cr, h->cp, h->cq, h->scal, n, h->part_a, (T*)F.r, (T*)F.x,
                                      (T*)F.d[0], Dinv<T>(F), (T)F.c0);
    CK(cudaGetLastError());
    k_reduce<<<1, 1024, 0, s>>>(h->part_a, gv, h->scal, S_RR, FIN_NONE, h->status);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&h->host_scal[S_RR], &h->scal[S_RR], sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h->host_scal[15], h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rr = h->host_scal[S_RR];
    h->launches += 1;
    prof_harvest(h);
    int st = 0;
    std::memcpy(&st, &h->host_scal[15], sizeof(int));
    if (st) {
      CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
      throw Fail{R3MG_E_BREAKDOWN, "CG breakdown: p^T A p <= 0 or non-finite scalar"};
    }
    *iters = it;
    rel = std::sqrt(rr) / bnorm;
    *relres = rel;
    if (!std::isfinite(rel)) throw Fail{R3MG_E_BREAKDOWN, "CG breakdown: non-finite residual"};
    if (rr <= thr2) {
      double rt = 0.0;
      true_residual(rt, nullptr);
      *relres = std::sqrt(rt) / bnorm;
      if (rt <= thr2) return R3MG_OK;
      precondition_restart();   // recursive residual drifted: restart from the true residual
      continue;
    }
    T* d = run_vcycle<T>(h);
    k_vc_final_dot<T><<<gv, 256, 0, s>>>((const T*)F.x, d, h->cz, fcg ? h->cq : h->cr, n, h->part_a);
    CK(cudaGetLastError());
    reduce_dev(h, h->part_a, gv, fcg ? S_ZQ : S_RZNEW, fcg ? FIN_BETA_FCG : FIN_BETA_PCG);
    k_p_update<<<gv, 256, 0, s>>>(h->cp, h->cz, h->cr, h->scal, n, fcg ? 1 : 0, fcg ? h->part_a : nullptr);
    CK(cudaGetLastError());
    if (fcg) reduce_dev(h, h->part_a, gv, S_PR, FIN_NONE);
    h->launches += fcg ? 4 : 3;
  }
  return R3MG_E_NOCONV;
}



// ================================================================ batches of problems
constexpr int64_t kSegRows = 8192;

// per-level batch arrays: problem of every row, in-problem index, segments, scalars
void batch_levels_upload(r3mg_hierarchy* h) {
  const int np = h->nprob;
  int maxseg = 1;
  for (int l = 0; l < h->L; ++l) {
    auto& B = h->bl[l];
    const int64_t n = B.row_off[np];
    std::vector<int32_t> rp(n);
    std::vector<int64_t> lab(n), sb, se;
    std::vector<int> soff{0};
    for (int q = 0; q < np; ++q) {
      for (int64_t k = B.row_off[q]; k < B.row_off[q + 1]; ++k) { rp[k] = q; lab[k] = k - B.row_off[q]; }
      for (int64_t k = B.row_off[q]; k < B.row_off[q + 1]; k += kSegRows) {
        sb.push_back(k);
        se.push_back(std::min(k + kSegRows, B.row_off[q + 1]));
      }
      soff.push_back((int)sb.size());
    }
    if (l == 0)   // fine level: the caller's index inside the problem (tree rows stay in their problem)
      for (int64_t k = 0; k < n; ++k) lab[k] = h->part.perm[k] - B.row_off[rp[k]];
    B.rprob = upload(h, rp);
    B.label = upload(h, lab);
    B.sb = upload(h, sb);
    B.se = upload(h, se);
    B.soff = upload(h, soff);
    B.nseg = (int)sb.size();
    maxseg = std::max(maxseg, B.nseg);
  }
  h->seg_part = dalloc<double>(h, maxseg);
  h->seg_out = dalloc<double>(h, np);
  h->h_seg.assign(np, 0.0);
  BatchScal& S = h->bs;
  S.pq = dalloc<double>(h, np); S.pr = dalloc<double>(h, np); S.zq = dalloc<double>(h, np);
  S.rz = dalloc<double>(h, np); S.rzn = dalloc<double>(h, np); S.rr = dalloc<double>(h, np);
  S.bb = dalloc<double>(h, np); S.alpha = dalloc<double>(h, np); S.beta = dalloc<double>(h, np);
  S.active = dalloc<int>(h, np); S.its = dalloc<int>(h, np); S.any = dalloc<int>(h, 1); S.err = dalloc<int>(h, 1);
  CK(cudaMemsetAsync(S.err, 0, sizeof(int), h->stream));
  h->d_moff = upload(h, h->h_moff);
  h->d_mld = upload(h, h->h_mld);
  h->d_cof = upload(h, h->h_cof);
}

// per-problem dots on level l: out[q] = sum over problem q's rows of x y (y null: x x)
template <typename T>
void seg_dot(r3mg_hierarchy* h, int l, const T* x, const T* y, double* out) {
  auto& B = h->bl[l];
  k_seg_dot<T><<<std::min(B.nseg, 148 * 8), 256, 0, h->stream>>>(x, y, B.sb, B.se, B.nseg, h->seg_part);
  k_seg_reduce<<<(h->nprob + 255) / 256, 256, 0, h->stream>>>(h->seg_part, B.soff, h->nprob, out);
  CK(cudaGetLastError());
}

const std::vector<double>& seg_dot_read(r3mg_hierarchy* h, int l, const double* x, const double* y) {
  seg_dot<double>(h, l, x, y, h->seg_out);
  CK(cudaMemcpyAsync(h->h_seg.data(), h->seg_out, sizeof(double) * h->nprob, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return h->h_seg;
}

// Lanczos estimate of every problem's lambda_max(D^-1 A_l) at once (Section 6; same reading as
// the single-problem estimate, each problem with its own CG scalars and start vector).
void lanczos_batch(r3mg_hierarchy* h, int l) {
  Level& A = h->lv[l];
  auto& B = h->bl[l];
  const int np = h->nprob;
  const int64_t n = A.n;
  cudaStream_t s = h->stream;
  double *r = h->cr, *z = h->cz, *p = h->cp, *q = h->cq;
  const int gv = grid_for(n);
  k_splitmix_vec<<<gv, 256, 0, s>>>(h->prm.seed + (uint64_t)l, B.label, r, n);
  k_jacobi<<<gv, 256, 0, s>>>(A.dinv64, r, z, n);
  CK(cudaGetLastError());
  std::vector<double> rz = seg_dot_read(h, l, r, z);
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  std::vector<std::vector<double>> al(np), be(np);
  std::vector<char> alive(np, 1);
  std::vector<int> steps(np);
  int maxsteps = 0;
  for (int k = 0; k < np; ++k) {
    steps[k] = (int)std::min<int64_t>(h->prm.lanczos_steps, B.row_off[k + 1] - B.row_off[k]);
    maxsteps = std::max(maxsteps, steps[k]);
  }
  std::vector<double> sa(np), sbv(np);
  for (int j = 0; j < maxsteps; ++j) {
    level_apply_dot<double>(h, A, p, q, nullptr, nullptr);
    const std::vector<double> pq = seg_dot_read(h, l, p, q);
    for (int k = 0; k < np; ++k) sa[k] = (alive[k] && j < steps[k]) ? -(rz[k] / pq[k]) : 0.0;
    CK(cudaMemcpyAsync(h->bs.alpha, sa.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    k_baxpy<<<gv, 256, 0, s>>>(h->bs.alpha, B.rprob, q, r, n);
    k_jacobi<<<gv, 256, 0, s>>>(A.dinv64, r, z, n);
    CK(cudaGetLastError());
    const std::vector<double> rzn = seg_dot_read(h, l, r, z);
    for (int k = 0; k < np; ++k) {
      sbv[k] = 0.0;
      if (!(alive[k] && j < steps[k])) continue;
      al[k].push_back(-sa[k]);
      const double beta = rzn[k] / rz[k];
      be[k].push_back(beta);
      if (rzn[k] == 0.0) { alive[k] = 0; continue; }
      sbv[k] = beta;
      rz[k] = rzn[k];
    }
    CK(cudaMemcpyAsync(h->bs.beta, sbv.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    k_bxpay<<<gv, 256, 0, s>>>(z, h->bs.beta, B.rprob, p, n);
    CK(cudaGetLastError());
  }
  // per-problem interval and Chebyshev schedule
  const int kdeg = h->prm.cheb_degree, nu = h->prm.sweeps;
  std::vector<double> preA, preC, postA, postC, c0(np);
  B.lam.assign(np, 0.0);
  Level tmp;
  for (int k = 0; k < np; ++k) {
    const int m = (int)al[k].size();
    std::vector<double> dg(m), off(m > 0 ? m - 1 : 0);
    for (int j = 0; j < m; ++j) {
      dg[j] = 1.0 / al[k][j] + (j > 0 ? be[k][j - 1] / al[k][j - 1] : 0.0);
      if (j + 1 < m) off[j] = std::sqrt(be[k][j]) / al[k][j];
    }
    const double lmax = tridiag_max_eig(dg, off);
    if (!(lmax > 0.0) || !std::isfinite(lmax))
      throw Fail{R3MG_E_NOT_SPD, "Lanczos estimate non-positive on level " + std::to_string(l) + ", problem " + std::to_string(k)};
    tmp.lam_hi = h->prm.eig_safety * lmax;
    tmp.lam_lo = tmp.lam_hi / h->prm.eig_ratio;
    make_schedule(tmp, kdeg, nu);
    B.lam[k] = tmp.lam_hi;
    c0[k] = tmp.c0;
    if (k == 0) { preA.assign(tmp.pre.size() * np, 0); preC = preA; postA.assign(tmp.post.size() * np, 0); postC = postA; }
    for (size_t st = 0; st < tmp.pre.size(); ++st) { preA[st * np + k] = tmp.pre[st].first; preC[st * np + k] = tmp.pre[st].second; }
    for (size_t st = 0; st < tmp.post.size(); ++st) { postA[st * np + k] = tmp.post[st].first; postC[st * np + k] = tmp.post[st].second; }
  }
  // the level keeps problem 0's scalar schedule (step counts; reported interval)
  A.lam_hi = B.lam[0];
  A.lam_lo = A.lam_hi / h->prm.eig_ratio;
  make_schedule(A, kdeg, nu);
  B.npre = (int)A.pre.size();
  B.npost = (int)A.post.size();
  auto put = [&](double*& dst, const std::vector<double>& v) {
    if (!dst) dst = dalloc<double>(h, (int64_t)v.size());
    CK(cudaMemcpyAsync(dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s));
  };
  put(B.preA, preA); put(B.preC, preC); put(B.postA, postA); put(B.postC, postC); put(B.c0, c0);
  CK(cudaStreamSynchronize(s));
}

// every problem's coarsest block: Cholesky, inverse, stored at its own offset
void dense_batch(r3mg_hierarchy* h) {
  Level& C = h->lv[h->L - 1];
  if (!h->Ainv64) h->Ainv64 = dalloc<double>(h, h->batch_ainv_size);
  const int np = h->nprob;
  const auto& ro = h->bl[h->L - 1].row_off;
  for (int k = 0; k < np; ++k) {
    const int64_t B0 = ro[k] / h->b, nb = (ro[k + 1] - ro[k]) / h->b;
    dense_block(h, C, B0, nb, h->Ainv64 + h->h_moff[k], h->h_mld[k]);
  }
}

// fused Chebyshev step with the per-problem coefficients of step st (register kernels)
template <typename T>
void level_cheb_b(r3mg_hierarchy* h, const Level& A, int l, T* x, T* r, T* d, T* dn, bool post, int st) {
  auto& B = h->bl[l];
  const int np = h->nprob;
  const double* ta = (post ? B.postA : B.preA) + (int64_t)st * np;
  const double* tc = (post ? B.postC : B.preC) + (int64_t)st * np;
  if constexpr (sizeof(T) == 4) {
    if (sym_form(A)) {
      SymCheb ep{x, r, d, dn, Dinv<T>(A), 0.f, 0.f};
      ep.A = ta; ep.C = tc; ep.rprob = B.rprob;
      sym_step(h, A, d, ep);
      return;
    }
  }
  launch_level<T>(A, d, TEpChebB<T>{x, r, d, dn, Dinv<T>(A), ta, tc, B.rprob}, nullptr, h->stream);
}

template <typename T>
T* vcycle_body_batch(r3mg_hierarchy* h, bool capturing) {
  cudaStream_t s = h->stream;
  const int L = h->L;
  std::vector<int> cur(L, 0);
  int64_t nk = 0;
  h->slot_next = 0;
  for (int l = 0; l < L - 1; ++l) {
    Level& A = h->lv[l];
    T* x = (T*)A.x; T* r = (T*)A.r;
    for (int st = 0; st < h->bl[l].npre; ++st) {
      T* d = (T*)A.d[cur[l]]; T* dn = (T*)A.d[cur[l] ^ 1];
      const int ps = prof_begin(h, 1 + l, capturing);
      level_cheb_b<T>(h, A, l, x, r, d, dn, false, st);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
    Level& C = h->lv[l + 1];
    const bool coarsest = (l + 1 == L - 1);
    NextInitB<T> nx{(T*)C.r, coarsest ? nullptr : (T*)C.x, coarsest ? nullptr : (T*)C.d[0], Dinv<T>(C),
                    h->bl[l + 1].c0, h->bl[l + 1].rprob};
    if (l == 0)
      k_restrict_fine<T, NextInitB<T>><<<(int)std::min<int64_t>(C.nbox, 148 * 64), 256, 0, s>>>(Pmat<T>(h, 0), r, A.box_row, C.nbox, h->b, nx);
    else
      k_restrict_coarse<T, NextInitB<T>><<<grid_for(C.nbox * h->b), 256, 0, s>>>(Pmat<T>(h, l), r, C.nbox, h->b, h->fan, nx);
    CK(cudaGetLastError());
    ++nk;
  }
  {
    Level& C = h->lv[L - 1];
    k_block_gemv<T><<<grid_for(C.n * 32), 256, 0, s>>>(Ainv<T>(h), h->d_moff, h->d_mld, h->d_cof, h->bl[L - 1].rprob,
                                                       (const T*)C.r, C.n, (T*)C.x);
    CK(cudaGetLastError());
    ++nk;
  }
  for (int l = L - 2; l >= 0; --l) {
    Level& A = h->lv[l];
    Level& C = h->lv[l + 1];
    const bool coarsest = (l + 1 == L - 1);
    const T* x1 = (const T*)C.x;
    const T* d1 = coarsest ? nullptr : (const T*)C.d[cur[l + 1]];
    T* d = (T*)A.d[cur[l]];
    if (l == 0)
      k_prolong_fine<T><<<grid_for(h->n), 256, 0, s>>>(Pmat<T>(h, 0), h->box_of_tree, x1, d1, h->n, h->b, d);
    else
      k_prolong_coarse<T><<<grid_for(A.nbox * h->b), 256, 0, s>>>(Pmat<T>(h, l), x1, d1, A.nbox, h->b, h->fan, d);
    CK(cudaGetLastError());
    ++nk;
    T* x = (T*)A.x; T* r = (T*)A.r;
    for (int st = 0; st < h->bl[l].npost; ++st) {
      T* dd = (T*)A.d[cur[l]]; T* dn = (T*)A.d[cur[l] ^ 1];
      const int ps = prof_begin(h, 1 + l, capturing);
      level_cheb_b<T>(h, A, l, x, r, dd, dn, true, st);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
  }
  if (capturing) h->graph_kernels = nk; else h->launches += nk;
  return (T*)h->lv[0].d[cur[0]];
}

// The batched iteration loop as ONE cooperative launch (see kernels_persistent.cuh): the same
// phases as the loop graph, separated by bounded grid barriers, skipping stopped problems.
template <typename T>
void launch_persistent_batch(r3mg_hierarchy* h, double rtol, int budget) {
  cudaStream_t s = h->stream;
  const int L = h->L;
  if (L > kPMaxLevels) throw Fail{R3MG_E_LIMIT, "persistent batched solve: more than 8 levels"};
  const int pi = sizeof(T) == 4 ? 1 : 0;
  PBatchArgs<T> A{};
  A.L = L; A.np = h->nprob; A.fcg = (h->prm.precision == 1) ? 1 : 0; A.b = h->b; A.fan = h->fan; A.maxit = budget;
  A.n = h->n; A.rtol2 = rtol * rtol;
  size_t smem = 0;
  for (int l = 0; l < L; ++l) {
    Level& V = h->lv[l];
    A.lv[l] = view<T>(V);
    // form 7 keeps CTAs per SM in the lanes field; the persistent kernel has no 2-lane rows
    A.G[l] = V.conf[pi].form == 7 ? 16 : std::max(4, V.conf[pi].G);
    A.x[l] = (T*)V.x; A.r[l] = (T*)V.r; A.d[l][0] = (T*)V.d[0]; A.d[l][1] = (T*)V.d[1];
    A.dinv[l] = Dinv<T>(V);
    A.P[l] = (l + 1 < L) ? Pmat<T>(h, l) : nullptr;
    auto& B = h->bl[l];
    A.rprob[l] = B.rprob;
    A.preA[l] = B.preA; A.preC[l] = B.preC; A.postA[l] = B.postA; A.postC[l] = B.postC;
    A.c0[l] = B.c0; A.npre[l] = B.npre; A.npost[l] = B.npost;
    if (l + 1 < L) smem = std::max(smem, level_smem_bytes(view<T>(V)));
  }
  Level& F = h->lv[0];
  A.box_of_tree = h->box_of_tree;
  A.Ainv = Ainv<T>(h); A.moff = h->d_moff; A.mld = h->d_mld; A.cof = h->d_cof;
  A.f64 = view<double>(F); A.G64 = std::max(4, F.conf[0].G);
  smem = std::max(smem, level_smem_bytes(view<double>(F)));
  A.cx = h->cx; A.cr = h->cr; A.cp = h->cp; A.cq = h->cq; A.cz = h->cz;
  A.S = h->bs;
  A.sb = h->bl[0].sb; A.se = h->bl[0].se; A.soff = h->bl[0].soff; A.nseg = h->bl[0].nseg; A.seg_part = h->seg_part;
  if (!h->pbar) h->pbar = dalloc<unsigned>(h, 2);
  if (h->pany_cap < budget + 1) {
    h->pany = dalloc<int>(h, budget + 1);
    h->pany_cap = budget + 1;
    if (h->pgraph) { cudaGraphExecDestroy(h->pgraph); h->pgraph = nullptr; h->pgraph_state = 0; }
  }
  A.any_count = h->pany;
  A.bar = GridBar{h->pbar, h->pbar + 1, h->tma_err, h->wait_cycles > 0 ? h->wait_cycles : kWaitCycles,
                  h->withhold_first};
  auto kern = k_batch_persistent<T>;
  ensure_smem((const void*)kern, smem);
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem));
  if (per_sm < 1) throw Fail{R3MG_E_LIMIT, "persistent batched solve: the kernel does not fit an SM"};
  const int grid = h->nsm * per_sm;   // every CTA resident at once (cooperative launch)
  auto enqueue = [&]() {
    CK(cudaMemsetAsync(h->pbar, 0, 2 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(h->pany, 0, sizeof(int) * (budget + 1), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident at once (the kernel's grid barrier)
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, kern, A));
  };
  // the launch (with the resets of its barrier and counters) captured once per (rtol, budget,
  // wait setting) into a graph; the direct launch if the capture is not possible
  if (h->pgraph_state == 1 && (h->pgraph_rtol != rtol || h->pgraph_budget != budget)) {
    cudaGraphExecDestroy(h->pgraph);
    h->pgraph = nullptr;
    h->pgraph_state = 0;
  }
  if (h->pgraph_state == 0) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try { enqueue(); } catch (Fail&) { ok = false; }
      if (cudaStreamEndCapture(s, &g) != cudaSuccess) ok = false;
    }
    if (ok && cudaGraphInstantiate(&h->pgraph, g, 0) == cudaSuccess) {
      h->pgraph_state = 1;
      h->pgraph_rtol = rtol;
      h->pgraph_budget = budget;
    } else {
      h->pgraph_state = -1;
      h->pgraph = nullptr;
      cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
  }
  if (h->pgraph_state == 1) CK(cudaGraphLaunch(h->pgraph, s));
  else enqueue();
  h->launches += 1;
}

// Batched PCG (FP64 V-cycle) or flexible CG (FP32 V-cycle) on tree-ordered cb / cx.  After a
// host-launched start (residuals, activity flags, first V-cycle entry), the whole iteration loop
// runs as one CUDA graph launch: a conditional WHILE node repeats one batched iteration until
// every problem has converged or reached maxit.
template <typename T>
r3mg_status krylov_batch(r3mg_hierarchy* h, double rtol, int maxit, int* iters, double* relres) {
  cudaStream_t s = h->stream;
  Level& F = h->lv[0];
  const int64_t n = h->n;
  const int np = h->nprob;
  const bool fcg = (h->prm.precision == 1);
  const int gv = grid_for(n);
  BatchScal& S = h->bs;
  auto& B0 = h->bl[0];
  std::vector<int> its_total(np, 0), done(np, 0);
  std::vector<double> bbh(np), rel(np, 0.0);
  for (int attempt = 0; attempt < 3; ++attempt) {
    // start: r = b - A x, per-problem norms, activity
    level_apply_dot<double>(h, F, h->cx, h->cq, nullptr, nullptr);
    k_residual<<<gv, 256, 0, s>>>(h->cb, h->cq, h->cr, n, h->part_a, nullptr);
    CK(cudaGetLastError());
    seg_dot<double>(h, 0, h->cb, nullptr, S.bb);
    seg_dot<double>(h, 0, h->cr, nullptr, S.rr);
    std::vector<double> rrh(np);
    CK(cudaMemcpyAsync(bbh.data(), S.bb, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rrh.data(), S.rr, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int> act(np, 0);
    int nact = 0;
    for (int k = 0; k < np; ++k) {
      rel[k] = bbh[k] > 0.0 ? std::sqrt(rrh[k] / bbh[k]) : 0.0;
      act[k] = (bbh[k] > 0.0 && rel[k] > rtol && its_total[k] < maxit) ? 1 : 0;
      nact += act[k];
    }
    if (nact == 0) break;
    std::vector<int> zero(np, 0);
    std::vector<double> ones(np, 1.0), infs(np, std::numeric_limits<double>::infinity());
    CK(cudaMemcpyAsync(S.active, act.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(S.its, zero.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(S.pq, ones.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(S.rz, infs.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(S.zq, 0, sizeof(double) * np, s));
    CK(cudaMemsetAsync(h->cp, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(h->cq, 0, sizeof(double) * n, s));
    k_bvc_init<T><<<gv, 256, 0, s>>>(h->cr, n, (T*)F.r, (T*)F.x, (T*)F.d[0], Dinv<T>(F), B0.c0, B0.rprob);
    CK(cudaGetLastError());
    const int budget = maxit - *std::min_element(its_total.begin(), its_total.end());
    int mode = h->batch_mode;
    if (mode == 2) {   // automatic: time each form once, then keep the faster
      if (h->L > kPMaxLevels || h->batch_ms_it[0] < 0.f) mode = 0;
      else if (h->batch_ms_it[1] < 0.f) mode = 1;
      else mode = h->batch_ms_it[1] < h->batch_ms_it[0] ? 1 : 0;
    }
    const bool timing = h->batch_mode == 2 && h->batch_ms_it[mode] < 0.f;
    cudaEvent_t te0 = nullptr, te1 = nullptr;
    if (timing) {
      CK(cudaEventCreate(&te0)); CK(cudaEventCreate(&te1));
      CK(cudaEventRecord(te0, s));
    }
    h->batch_used = mode;
    if (mode == 1) {
      launch_persistent_batch<T>(h, rtol, budget);
    } else {
    // the loop graph, captured once per (rtol, maxit)
    if (h->bgraph_state == 1 && (h->bgraph_rtol != rtol || h->bgraph_maxit != budget)) {
      cudaGraphExecDestroy(h->bgraph);
      h->bgraph = nullptr;
      h->bgraph_state = 0;
    }
    if (h->bgraph_state == 0) {
      cudaGraph_t g = nullptr;
      CK(cudaGraphCreate(&g, 0));
      cudaGraphConditionalHandle hdl;
      CK(cudaGraphConditionalHandleCreate(&hdl, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = hdl;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      bool ok = true;
      try {
        T* d = vcycle_body_batch<T>(h, true);
        k_bvc_final<T><<<gv, 256, 0, s>>>((const T*)F.x, d, h->cz, n);
        if (fcg) { seg_dot<double>(h, 0, h->cz, h->cq, S.zq); k_bscal<<<(np + 255) / 256, 256, 0, s>>>(S, np, BF_BETA_FCG); }
        else { seg_dot<double>(h, 0, h->cz, h->cr, S.rzn); k_bscal<<<(np + 255) / 256, 256, 0, s>>>(S, np, BF_BETA_PCG); }
        k_bp_update<<<gv, 256, 0, s>>>(h->cp, h->cz, S.beta, B0.rprob, n, fcg ? 1 : 0);
        level_apply_dot<double>(h, F, h->cp, h->cq, nullptr, nullptr);
        seg_dot<double>(h, 0, h->cp, h->cq, S.pq);
        if (fcg) seg_dot<double>(h, 0, h->cp, h->cr, S.pr);
        k_bscal<<<(np + 255) / 256, 256, 0, s>>>(S, np, fcg ? BF_ALPHA_FCG : BF_ALPHA_PCG);
        k_bcg_update<T><<<gv, 256, 0, s>>>(h->cx, h->cr, h->cp, h->cq, S.alpha, B0.rprob, n, (T*)F.r, (T*)F.x,
                                           (T*)F.d[0], Dinv<T>(F), B0.c0);
        seg_dot<double>(h, 0, h->cr, nullptr, S.rr);
        k_bconverge<<<1, 1024, 0, s>>>(S, np, rtol * rtol, budget);
        k_set_condition<<<1, 32, 0, s>>>(hdl, S.any);
        CK(cudaGetLastError());
      } catch (Fail&) { ok = false; }
      cudaGraph_t cap = body;
      const bool ended = cudaStreamEndCapture(s, &cap) == cudaSuccess;
      if (!ok || !ended || cudaGraphInstantiate(&h->bgraph, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        throw Fail{R3MG_E_CUDA, "batched solve: the conditional loop graph could not be built"};
      }
      cudaGraphDestroy(g);
      h->bgraph_state = 1;
      h->bgraph_rtol = rtol;
      h->bgraph_maxit = budget;
    }
    CK(cudaGraphLaunch(h->bgraph, s));
    }
    if (timing) CK(cudaEventRecord(te1, s));
    std::vector<int> itsh(np);
    int err = 0;
    CK(cudaMemcpyAsync(itsh.data(), S.its, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, S.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (timing) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, te0, te1));
      const int itmax = *std::max_element(itsh.begin(), itsh.end());
      if (itmax > 0) h->batch_ms_it[mode] = ms / (float)itmax;
      cudaEventDestroy(te0); cudaEventDestroy(te1);
    }
    if (err) {
      CK(cudaMemsetAsync(S.err, 0, sizeof(int), s));
      throw Fail{R3MG_E_BREAKDOWN, "batched CG breakdown: p^T A p <= 0 or non-finite scalar"};
    }
    if (mode == 1) {
      int terr = 0;
      CK(cudaMemcpy(&terr, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (terr) {
        CK(cudaMemset(h->tma_err, 0, sizeof(int)));
        throw Fail{R3MG_E_TIMEOUT, "persistent batched solve: a bounded grid-barrier wait expired"};
      }
    }
    for (int k = 0; k < np; ++k) its_total[k] += itsh[k];
  }
  // confirmed (true) residuals
  level_apply_dot<double>(h, F, h->cx, h->cq, nullptr, nullptr);
  k_residual<<<gv, 256, 0, s>>>(h->cb, h->cq, h->cr, n, h->part_a, nullptr);
  CK(cudaGetLastError());
  const std::vector<double>& rrt = seg_dot_read(h, 0, h->cr, nullptr);
  bool all = true;
  for (int k = 0; k < np; ++k) {
    relres[k] = bbh[k] > 0.0 ? std::sqrt(rrt[k] / bbh[k]) : 0.0;
    iters[k] = its_total[k];
    if (relres[k] > rtol) all = false;
  }
  return all ? R3MG_OK : R3MG_E_NOCONV;
}

void build_batch(r3mg_hierarchy* h, int np, const int64_t* n, const double* const* coords,
                 const int64_t* const* rowptr, const int32_t* const* colidx, const double* const* vals) {
  const r3mg_params& prm = h->prm;
  const int dim = h->dim;
  h->b = 1;
  for (int a = 0; a < dim; ++a) h->b *= (prm.pprime + 1);
  h->fan = 1 << dim;
  h->nprob = np;
  const int b = h->b, L = prm.levels;
  std::vector<ProbHost> ph(np);
  for (int k = 0; k < np; ++k) {
    try {
      analyse_problem(prm, dim, b, h->fan, n[k], coords[k], rowptr[k], colidx[k], vals[k], ph[k]);
    } catch (Fail& f) {
      throw Fail{f.st, "problem " + std::to_string(k) + ": " + f.msg};
    }
  }
  // offsets of every problem at every level
  std::vector<int64_t> row0(np + 1, 0), nnz0(np + 1, 0), st0(np + 1, 0);
  std::vector<std::vector<int64_t>> box0(L, std::vector<int64_t>(np + 1, 0)), pat0(L, std::vector<int64_t>(np + 1, 0));
  for (int k = 0; k < np; ++k) {
    row0[k + 1] = row0[k] + n[k];
    nnz0[k + 1] = nnz0[k] + rowptr[k][n[k]];
    st0[k + 1] = st0[k] + ph[k].lay.row_ptr[n[k]];
    for (int l = 1; l < L; ++l) {
      box0[l][k + 1] = box0[l][k] + ph[k].P.nbox(l);
      pat0[l][k + 1] = pat0[l][k] + (int64_t)ph[k].pats[l].nbr.size();
    }
  }
  const int64_t N = row0[np];
  h->n = N;
  for (int k = 0; k < np; ++k) h->h_fine = std::max(h->h_fine, ph[k].hmax);
  // combined partition: every problem's boxes, in problem order
  HostPartition& P = h->part;
  P.n = N; P.dim = dim; P.levels = L; P.depth = 0;
  P.perm.resize(N);
  P.iperm.resize(N);
  P.box_off.assign(L, {});
  P.lo.assign(L, {});
  P.hi.assign(L, {});
  for (int k = 0; k < np; ++k) {
    P.depth = std::max(P.depth, ph[k].P.depth);
    for (int64_t t = 0; t < n[k]; ++t) P.perm[row0[k] + t] = ph[k].P.perm[t] + row0[k];
  }
  for (int64_t t = 0; t < N; ++t) P.iperm[P.perm[t]] = t;
  for (int l = 1; l < L; ++l) {
    P.box_off[l].push_back(0);
    for (int k = 0; k < np; ++k) {
      const auto& bo = ph[k].P.box_off[l];
      for (size_t B = 1; B < bo.size(); ++B) P.box_off[l].push_back(bo[B] + row0[k]);
      P.lo[l].insert(P.lo[l].end(), ph[k].P.lo[l].begin(), ph[k].P.lo[l].end());
      P.hi[l].insert(P.hi[l].end(), ph[k].P.hi[l].begin(), ph[k].P.hi[l].end());
    }
  }
  // combined block adjacency
  std::vector<HostPattern> pats(L);
  for (int l = 1; l < L; ++l) {
    pats[l].ptr.push_back(0);
    for (int k = 0; k < np; ++k) {
      const auto& pt = ph[k].pats[l];
      for (size_t B = 1; B < pt.ptr.size(); ++B) pats[l].ptr.push_back(pt.ptr[B] + pat0[l][k]);
      for (int64_t c : pt.nbr) pats[l].nbr.push_back(c + box0[l][k]);
    }
  }
  // combined fine layout
  HostFineLayout lay;
  lay.row_ptr.push_back(0);
  for (int k = 0; k < np; ++k) {
    const HostFineLayout& a = ph[k].lay;
    for (int64_t t = 1; t <= n[k]; ++t) lay.row_ptr.push_back(a.row_ptr[t] + st0[k]);
    lay.idx.insert(lay.idx.end(), a.idx.begin(), a.idx.end());
    for (int64_t v : a.src) lay.src.push_back(v >= 0 ? v + nnz0[k] : -1);
    for (int64_t v : a.diag_src) lay.diag_src.push_back(v + nnz0[k]);
    lay.win_off.insert(lay.win_off.end(), a.win_off.begin(), a.win_off.end());
    for (int64_t v : a.win_src) lay.win_src.push_back(v + row0[k]);
    lay.win_size.insert(lay.win_size.end(), a.win_size.begin(), a.win_size.end());
    lay.win_max = std::max(lay.win_max, a.win_max);
    lay.nnz += a.nnz;
  }
  std::vector<double> cc(N * dim);
  for (int k = 0; k < np; ++k) std::memcpy(cc.data() + row0[k] * dim, coords[k], sizeof(double) * n[k] * dim);
  // per-level problem offsets and the coarsest blocks
  h->bl.assign(L, Hier::BLevel());
  h->bl[0].row_off = row0;
  for (int l = 1; l < L; ++l) {
    h->bl[l].row_off.resize(np + 1);
    for (int k = 0; k <= np; ++k) h->bl[l].row_off[k] = box0[l][k] * b;
  }
  h->h_moff.assign(np + 1, 0);
  h->h_mld.assign(np, 0);
  h->h_cof = h->bl[L - 1].row_off;
  for (int k = 0; k < np; ++k) {
    const int64_t nc = h->h_cof[k + 1] - h->h_cof[k];
    const int64_t ncp = (nc + kTile - 1) / kTile * kTile;
    h->h_mld[k] = ncp;
    h->h_moff[k + 1] = h->h_moff[k] + ncp * ncp;
  }
  h->batch_ainv_size = h->h_moff[np];
  std::vector<std::pair<const double*, int64_t>> pieces;
  for (int k = 0; k < np; ++k) pieces.emplace_back(vals[k], rowptr[k][n[k]]);
  build_device(h, pats, lay, cc.data(), nullptr, nullptr, pieces);
}

// ================================================================ several right-hand sides
// M columns per block vector (M in {4, 8, 16}; a caller's m columns are padded with zero
// columns).  The hierarchy is shared; only the vectors and the per-column CG scalars are new.

int mr_cols(int m) { return m <= 4 ? 4 : m <= 8 ? 8 : 16; }

void mr_free(r3mg_hierarchy* h, void* p) {
  if (!p) return;
  cudaFree(p);
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
}

// Block vectors for M columns on every level (V-cycle precision) and the FP64 CG blocks.
void mr_alloc(r3mg_hierarchy* h, int M) {
  if (h->mr_M == M) return;
  CK(cudaStreamSynchronize(h->stream));
  for (auto* v : {&h->mr_x, &h->mr_r, &h->mr_d0, &h->mr_d1})
    for (void* p : *v) mr_free(h, p);
  for (double* p : {h->mr_b, h->mr_xc, h->mr_rc, h->mr_p, h->mr_q, h->mr_z, h->mr_scal, h->mr_pa, h->mr_pb, h->mr_lp})
    mr_free(h, p);
  mr_free(h, h->mr_its);
  mr_free(h, h->mr_active);
  if (h->mgraph) { cudaGraphExecDestroy(h->mgraph); h->mgraph = nullptr; }
  h->mgraph_state = 0;
  h->mr_M = 0;
  h->mr_S[0].clear();   // kernel choices were tuned for the old column count
  h->mr_S[1].clear();
  const size_t es = (h->prm.precision == 1) ? 4 : 8;
  const int L = h->L;
  h->mr_x.assign(L, nullptr); h->mr_r.assign(L, nullptr); h->mr_d0.assign(L, nullptr); h->mr_d1.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const int64_t cnt = h->lv[l].n * M * (int64_t)es;
    h->mr_x[l] = dalloc<unsigned char>(h, cnt);
    h->mr_r[l] = dalloc<unsigned char>(h, cnt);
    if (l + 1 < L) {
      h->mr_d0[l] = dalloc<unsigned char>(h, cnt);
      h->mr_d1[l] = dalloc<unsigned char>(h, cnt);
    }
  }
  const int64_t nm = h->n * M;
  h->mr_b = dalloc<double>(h, nm); h->mr_xc = dalloc<double>(h, nm); h->mr_rc = dalloc<double>(h, nm);
  h->mr_p = dalloc<double>(h, nm); h->mr_q = dalloc<double>(h, nm); h->mr_z = dalloc<double>(h, nm);
  h->mr_scal = dalloc<double>(h, (int64_t)(S_COUNT + 2 * kHist) * M);   // slots, then per-column histories
  CK(cudaMemsetAsync(h->mr_scal, 0, sizeof(double) * (S_COUNT + 2 * kHist) * M, h->stream));
  h->mr_npart = std::max<int64_t>(grid_for(nm), (int64_t)h->nsm * 8);
  h->mr_pa = dalloc<double>(h, h->mr_npart * M);
  h->mr_pb = dalloc<double>(h, h->mr_npart * M);
  h->mr_lp = dalloc<double>(h, 2);
  h->mr_its = dalloc<int>(h, M + 1);   // + the host-driven loop's continue flag
  h->mr_active = dalloc<int>(h, M);
  if (!h->mr_host) CK(cudaMallocHost(&h->mr_host, sizeof(double) * 128));
  h->mr_M = M;
}

// Global column indices of the fine level for the flat block sweep (built once, kept).
void mr_build_gidx(r3mg_hierarchy* h) {
  if (h->mr_gidx) return;
  Level& F = h->lv[0];
  h->mr_gidx = dalloc<int32_t>(h, F.stored);
  const LevelView<double> v = view<double>(F);
  const size_t sm = sizeof(int32_t) * (((size_t)v.win_max + 7) & ~(size_t)3);
  ensure_smem((const void*)k_mr_build_gidx<double>, sm);
  k_mr_build_gidx<double><<<(int)std::min<int64_t>(F.nbox, (int64_t)h->nsm * 8), 256, sm, h->stream>>>(v, h->mr_gidx);
  CK(cudaGetLastError());
}

// The grouped fine level (k_mr_grouped): within each box, rows are keyed by (length, FNV-1a
// hash of the window index list) and sorted; runs of rows whose lists are equal (compared entry
// by entry; equal lists have equal padding) are split into groups of 8, 4, 2 and 1 rows.  Built
// once on the host from the per-row layout's window indices.
constexpr int kMrGrouped = 20;          // block-config code of the grouped fine level
constexpr int kMrGroupR[4] = {8, 4, 2, 1};

// Host grouping of a windowed per-row layout (rows of box B: box_row[B] .. box_row[B+1]-1, row
// r's window indices idx[row_ptr[r] .. row_ptr[r+1])): per box, rows keyed by (length, hash),
// sorted by (length, hash, row); each run of rows with equal lists, in increasing row order, is
// cut into groups of 8, then 4, 2 and 1.  Output class-major (8, 4, 2, 1), boxes in order within a
// class: the rows group by group, each group's entry count, and per class its group count, first
// group and first row slot.
struct RowGroups {
  int64_t ng[4] = {0, 0, 0, 0}, g0[4] = {0, 0, 0, 0}, r0[4] = {0, 0, 0, 0};
  std::vector<int32_t> rows;
  std::vector<int64_t> len;
};

RowGroups group_rows_host(const int64_t* rp, int64_t nbox, const int64_t* br, const uint16_t* ix) {
  auto same = [&](int64_t a, int64_t b) {
    return rp[a + 1] - rp[a] == rp[b + 1] - rp[b] && std::equal(ix + rp[a], ix + rp[a + 1], ix + rp[b]);
  };
  // per box: its rows group by group, class by class, and its group count per class
  std::vector<std::vector<int32_t>> order(nbox);
  std::vector<int64_t> cnt(nbox * 4, 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t B = 0; B < nbox; ++B) {
    struct Key { int64_t len; uint64_t hash; int64_t row; };
    std::vector<Key> key;
    for (int64_t r = br[B]; r < br[B + 1]; ++r) {
      uint64_t hsh = 1469598103934665603ull;
      for (int64_t k = rp[r]; k < rp[r + 1]; ++k) { hsh ^= ix[k]; hsh *= 1099511628211ull; }
      key.push_back({rp[r + 1] - rp[r], hsh, r});
    }
    std::sort(key.begin(), key.end(), [](const Key& a, const Key& b) {
      return a.len != b.len ? a.len < b.len : a.hash != b.hash ? a.hash < b.hash : a.row < b.row;
    });
    std::vector<int32_t> cls[4];
    auto emit = [&](const std::vector<int64_t>& run) {
      size_t i = 0;
      for (int c = 0; c < 4; ++c)
        for (; run.size() - i >= (size_t)kMrGroupR[c]; i += kMrGroupR[c])
          for (int q = 0; q < kMrGroupR[c]; ++q) cls[c].push_back((int32_t)run[i + q]);
    };
    for (size_t i = 0; i < key.size();) {
      size_t j = i;
      while (j < key.size() && key[j].len == key[i].len && key[j].hash == key[i].hash) ++j;
      // rows [i, j) share the key; split them into lists that are really equal
      std::vector<char> used(j - i, 0);
      for (size_t a = i; a < j; ++a) {
        if (used[a - i]) continue;
        std::vector<int64_t> run{key[a].row};
        for (size_t b = a + 1; b < j; ++b)
          if (!used[b - i] && same(key[a].row, key[b].row)) { used[b - i] = 1; run.push_back(key[b].row); }
        emit(run);
      }
      i = j;
    }
    for (int c = 0; c < 4; ++c) {
      cnt[B * 4 + c] = (int64_t)cls[c].size() / kMrGroupR[c];
      order[B].insert(order[B].end(), cls[c].begin(), cls[c].end());
    }
  }
  // class-major numbering, boxes in order within a class
  RowGroups out;
  std::vector<int64_t> boff(nbox * 4);
  int64_t g = 0, rows = 0;
  for (int c = 0; c < 4; ++c) {
    out.g0[c] = g;
    out.r0[c] = rows;
    for (int64_t B = 0; B < nbox; ++B) { boff[B * 4 + c] = g; g += cnt[B * 4 + c]; }
    out.ng[c] = g - out.g0[c];
    rows += out.ng[c] * kMrGroupR[c];
  }
  out.rows.assign(rows, 0);
  out.len.assign(g, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t B = 0; B < nbox; ++B) {
    size_t p = 0;
    for (int c = 0; c < 4; ++c) {
      const int R = kMrGroupR[c];
      for (int64_t q = 0; q < cnt[B * 4 + c]; ++q, p += R) {
        const int64_t gg = boff[B * 4 + c] + q;
        for (int t = 0; t < R; ++t) out.rows[out.r0[c] + (gg - out.g0[c]) * R + t] = order[B][p + t];
        out.len[gg] = rp[order[B][p] + 1] - rp[order[B][p]];
      }
    }
  }
  return out;
}

void mr_build_groups(r3mg_hierarchy* h) {
  if (h->mrg_built) return;
  mr_build_gidx(h);
  const Level& F = h->lv[0];
  const LevelView<double> v = view<double>(F);
  const int64_t n = F.n, nbox = F.nbox;
  std::vector<int64_t> rp(n + 1), br(nbox + 1);
  std::vector<uint16_t> ix(F.stored);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(rp.data(), v.row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(br.data(), v.box_row, sizeof(int64_t) * (nbox + 1), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ix.data(), v.idx, sizeof(uint16_t) * F.stored, cudaMemcpyDeviceToHost));
  const RowGroups grp = group_rows_host(rp.data(), nbox, br.data(), ix.data());
  for (int c = 0; c < 4; ++c) { h->mrg_ng[c] = grp.ng[c]; h->mrg_g0[c] = grp.g0[c]; h->mrg_r0[c] = grp.r0[c]; }
  const int64_t NG = (int64_t)grp.len.size(), rows = (int64_t)grp.rows.size();
  // entry offsets, and value offsets with every class starting on a 16-value boundary (the
  // kernels read a group entry's R values with 16-byte loads)
  std::vector<int64_t> geoff(NG + 1), gvoff(NG + 1);
  geoff[0] = gvoff[0] = 0;
  int64_t ev = 0;
  for (int c = 0; c < 4; ++c) {
    ev = (ev + 15) & ~(int64_t)15;
    for (int64_t q = grp.g0[c]; q < grp.g0[c] + grp.ng[c]; ++q) {
      gvoff[q] = ev;
      ev += grp.len[q] * kMrGroupR[c];
      geoff[q + 1] = geoff[q] + grp.len[q];
    }
  }
  gvoff[NG] = ev;
  h->mrg_geoff = dalloc<int64_t>(h, NG + 1);
  h->mrg_gvoff = dalloc<int64_t>(h, NG + 1);
  h->mrg_rows = dalloc<int32_t>(h, std::max<int64_t>(1, rows));
  h->mrg_col = dalloc<int32_t>(h, std::max<int64_t>(1, geoff[NG]));
  CK(cudaMemcpy(h->mrg_geoff, geoff.data(), sizeof(int64_t) * (NG + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->mrg_gvoff, gvoff.data(), sizeof(int64_t) * (NG + 1), cudaMemcpyHostToDevice));
  if (rows > 0) CK(cudaMemcpy(h->mrg_rows, grp.rows.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice));
  h->mrg_built = true;
}

// The grouped values of the fine level in precision T (and, with cols, the column lists),
// gathered on the device from the per-row layout into dst.
template <typename T>
void mr_group_gather(r3mg_hierarchy* h, T* dst, bool cols) {
  const LevelView<T> v = view<T>(h->lv[0]);
  for (int c = 0; c < 4; ++c) {
    if (h->mrg_ng[c] == 0) continue;
    const int grid = (int)std::min<int64_t>((h->mrg_ng[c] + 7) / 8, (int64_t)h->nsm * 16);
    k_mr_group_gather<T><<<grid, 256, 0, h->stream>>>(kMrGroupR[c], h->mrg_ng[c], h->mrg_geoff + h->mrg_g0[c],
                                                      h->mrg_gvoff + h->mrg_g0[c], h->mrg_rows + h->mrg_r0[c],
                                                      v.row_ptr, h->mr_gidx, v.vals, cols ? h->mrg_col : nullptr, dst);
    CK(cudaGetLastError());
  }
}

// Built on first use (the block tuner runs it before any graph capture), in place afterwards.
template <typename T>
void mr_group_vals(r3mg_hierarchy* h) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  if (h->mrg_vals[pi]) return;
  mr_build_groups(h);
  const int64_t NG = h->mrg_g0[3] + h->mrg_ng[3];
  int64_t nvals = 0;
  CK(cudaMemcpy(&nvals, h->mrg_gvoff + NG, sizeof(int64_t), cudaMemcpyDeviceToHost));
  T* gv = dalloc<T>(h, std::max<int64_t>(1, nvals));
  mr_group_gather<T>(h, gv, h->mrg_vals[1 - pi] == nullptr);   // column lists are gathered once
  h->mrg_vals[pi] = gv;
}

// New matrix values (numeric setup again): the grouped copies are gathered again in place, so
// pointers held by launch arguments stay valid.
void mr_regroup(r3mg_hierarchy* h) {
  if (h->mrg_vals[0]) mr_group_gather<double>(h, (double*)h->mrg_vals[0], false);
  if (h->mrg_vals[1]) mr_group_gather<float>(h, (float*)h->mrg_vals[1], false);
}

template <typename T, int M, int R, class Ep>
int mr_launch_grouped(r3mg_hierarchy* h, int c, const T* x, Ep ep, double* part) {
  constexpr int CL = M / Slice<T>::V, GPW = 32 / (CL * mr_group_slots(R, CL));
  const int64_t ng = h->mrg_ng[c];
  if (ng == 0) return 0;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ng + 8 * GPW - 1) / (8 * GPW), (int64_t)h->nsm * 2));
  k_mr_grouped<T, M, R, Ep><<<grid, 256, 0, h->stream>>>(ng, h->mrg_geoff + h->mrg_g0[c], h->mrg_gvoff + h->mrg_g0[c],
                                                         h->mrg_rows + h->mrg_r0[c], h->mrg_col,
                                                         (const T*)h->mrg_vals[sizeof(T) == 4 ? 1 : 0], x, ep, part);
  CK(cudaGetLastError());
  return grid;
}

template <typename T, int M, int S, bool FINE, class Ep>
void mr_launch(const Level& A, const T* x, Ep ep, double* part, cudaStream_t s, int grid) {
  const LevelView<T> v = view<T>(A);
  auto kern = k_mr_level<T, M, S, FINE, Ep>;
  const size_t sm = sizeof(int32_t) * (((size_t)v.win_max + 7) & ~(size_t)3);
  ensure_smem((const void*)kern, sm);
  kern<<<grid, 256, sm, s>>>(v, x, ep, part);
  CK(cudaGetLastError());
}

// Rows per lane of the staged coarse kernel (a power of two with ceil(b/R) * CL <= 32), 0 when
// the level cannot use it (row groups too long, or the window does not fit in shared memory).
template <typename T, int M>
int mr_coarse_rows(const Level& A) {
  if (A.b == 0) return 0;
  constexpr int CL = M / Slice<T>::V;
  int R = 1;
  while ((A.b + R - 1) / R * CL > 32) R *= 2;
  if (R > 16) return 0;
  if (mr_coarse_smem<T, M>(view<T>(A)) > kMaxSmem) return 0;
  return R;
}

template <typename T, int M, int R, class Ep>
void mr_launch_coarse(const Level& A, const T* x, Ep ep, double* part, cudaStream_t s, int grid) {
  const LevelView<T> v = view<T>(A);
  auto kern = k_mr_coarse<T, M, R, Ep>;
  const size_t sm = mr_coarse_smem<T, M>(v);
  ensure_smem((const void*)kern, sm);
  kern<<<grid, 256, sm, s>>>(v, x, ep, part);
  CK(cudaGetLastError());
}

// Streamed coarse block kernel: rows per chunk so that the window, two chunk buffers and the
// partial sums fit the shared memory (0: does not fit), and rows per lane.
template <typename T, int M>
MrStreamLayout mr_stream_layout(const Level& A) {
  for (int rc = A.b; rc >= 1; --rc) {
    MrStreamLayout lay(A.win_max, A.b, M, (int)sizeof(T), rc);
    if (lay.total <= kMaxSmem) return lay;
  }
  return MrStreamLayout();
}

template <typename T, int M>
int mr_stream_rows(int RC) {
  constexpr int CL = M / Slice<T>::V;
  int R = 1;
  while ((RC + R - 1) / R * CL > 32) R *= 2;
  return R;
}

template <typename T, int M, int R, class Ep>
void mr_launch_stream(r3mg_hierarchy* h, const Level& A, const T* x, Ep ep, double* part, const MrStreamLayout& lay,
                      int grid) {
  const LevelView<T> v = view<T>(A);
  auto kern = k_mr_coarse_stream<T, M, R, Ep>;
  ensure_smem((const void*)kern, lay.total);
  kern<<<grid, 256, lay.total, h->stream>>>(v, x, ep, part, lay, h->tma_err);
  CK(cudaGetLastError());
}

// Tensor-core coarse block kernel: FP32, M = 8 or 16, products without dot partials.
template <typename T, int M, class Ep>
constexpr bool mr_mma_ok() { return sizeof(T) == 4 && (M == 8 || M == 16); }

template <typename T, int M, class Ep>
void mr_launch_mma(r3mg_hierarchy* h, const Level& A, const T* x, Ep ep) {
  if constexpr (mr_mma_ok<T, M, Ep>()) {
    const LevelView<float> v = view<float>(A);
    auto kern = k_mr_coarse_mma<M, Ep>;
    const size_t sm = sizeof(int32_t) * (((size_t)v.win_max + 31) & ~(size_t)15);
    ensure_smem((const void*)kern, sm);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm * 16));
    kern<<<grid, 128, sm, h->stream>>>(v, x, ep);
    CK(cudaGetLastError());
  }
}

// 5th-generation tensor-core coarse block kernel (tcgen05, TMEM accumulator): FP32, 16 columns,
// boxes of at most 32 rows, products without dot partials.
template <typename T, int M, class Ep>
constexpr bool mr_tc_ok() { return sizeof(T) == 4 && M == 16; }

template <typename T, int M, class Ep>
bool mr_tc_fits(const Level& A) { return mr_tc_ok<T, M, Ep>() && A.b > 0 && A.b <= kTcRows; }

template <typename T, int M, class Ep>
void mr_launch_tc(r3mg_hierarchy* h, const Level& A, const T* x, Ep ep) {
  if constexpr (mr_tc_ok<T, M, Ep>()) {
    const LevelView<float> v = view<float>(A);
    auto kern = k_mr_coarse_tc<M, Ep>;
    const size_t sm = TcLayout<M>::kTotal;
    ensure_smem((const void*)kern, sm);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (kMaxSmem + 1024) / (sm + 1024)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm * per_sm));
    kern<<<grid, 128, sm, h->stream>>>(v, x, ep, h->tma_err, tma_ctl(h).wait);
    CK(cudaGetLastError());
  }
}

template <typename T, int M, class Ep>
void mr_launch_tc2(r3mg_hierarchy* h, const Level& A, const T* x, Ep ep) {
  if constexpr (mr_tc_ok<T, M, Ep>()) {
    const LevelView<float> v = view<float>(A);
    auto kern = k_mr_coarse_tc2<Ep>;
    ensure_smem((const void*)kern, kT2SmemLaunch);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm));
    kern<<<grid, kT2Warps * 32, kT2SmemLaunch, h->stream>>>(v, x, ep, h->tma_err, tma_ctl(h).wait);
    CK(cudaGetLastError());
  }
}

// One level operator on M columns with S entry slots per row (on a coarse level S = 0: the
// staged-window kernel, S = 1: the streamed kernel, S = 3: the mma.sync tensor-core kernel,
// S = 5: the tcgen05 tensor-core kernel, S = 6: the warp-specialised tcgen05 kernel with A in
// TMEM); returns the partial count.
template <typename T, int M, class Ep>
int mr_level(r3mg_hierarchy* h, const Level& A, const T* x, Ep ep, double* part, int S) {
  const bool fine = (A.b == 0);
  cudaStream_t s = h->stream;
  constexpr int CL = M / Slice<T>::V;
  if (!fine && S == 6) {
    if (mr_tc_fits<T, M, Ep>(A) && part == nullptr) {
      mr_launch_tc2<T, M, Ep>(h, A, x, ep);
      return 1;
    }
    S = 5;
  }
  if (!fine && S == 5) {
    if (mr_tc_fits<T, M, Ep>(A) && part == nullptr) {
      mr_launch_tc<T, M, Ep>(h, A, x, ep);
      return 1;
    }
    S = 3;
  }
  if (!fine && S == 3) {
    if (mr_mma_ok<T, M, Ep>() && part == nullptr) {
      mr_launch_mma<T, M, Ep>(h, A, x, ep);
      return 1;
    }
    S = 2;
  }
  if (fine && S == kMrGrouped) {   // groups of rows with equal column lists, one launch per group size
    mr_group_vals<T>(h);
    int np = 0;
    np += mr_launch_grouped<T, M, 8, Ep>(h, 0, x, ep, part ? part + (int64_t)np * M : nullptr);
    np += mr_launch_grouped<T, M, 4, Ep>(h, 1, x, ep, part ? part + (int64_t)np * M : nullptr);
    np += mr_launch_grouped<T, M, 2, Ep>(h, 2, x, ep, part ? part + (int64_t)np * M : nullptr);
    np += mr_launch_grouped<T, M, 1, Ep>(h, 3, x, ep, part ? part + (int64_t)np * M : nullptr);
    return std::max(np, 1);
  }
  if (fine && S > 8) {   // 10 + slots: the flat row sweep on global column indices
    mr_build_gidx(h);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((A.n + 7) / 8, (int64_t)h->nsm * 8));
    const LevelView<T> v = view<T>(A);
    const int Sr = S - 10;
    if (Sr == 2 && CL * 2 <= 32) {
      if constexpr (CL * 2 <= 32) k_mr_rows<T, M, 2, Ep><<<grid, 256, 0, s>>>(v.row_ptr, h->mr_gidx, v.vals, A.n, x, ep, part);
    } else if (Sr == 8 && CL * 8 <= 32) {
      if constexpr (CL * 8 <= 32) k_mr_rows<T, M, 8, Ep><<<grid, 256, 0, s>>>(v.row_ptr, h->mr_gidx, v.vals, A.n, x, ep, part);
    } else {
      if constexpr (CL * 4 <= 32) k_mr_rows<T, M, 4, Ep><<<grid, 256, 0, s>>>(v.row_ptr, h->mr_gidx, v.vals, A.n, x, ep, part);
    }
    CK(cudaGetLastError());
    return grid;
  }
  if (!fine && S == 1) {
    const MrStreamLayout lay = mr_stream_layout<T, M>(A);
    const int R = lay.RC > 0 ? mr_stream_rows<T, M>(lay.RC) : 0;
    if (R > 0 && R <= 16) {
      const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (kMaxSmem + 1024) / (lay.total + 1024)));
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm * per_sm));
      switch (R) {
        case 1: mr_launch_stream<T, M, 1>(h, A, x, ep, part, lay, grid); break;
        case 2: mr_launch_stream<T, M, 2>(h, A, x, ep, part, lay, grid); break;
        case 4: mr_launch_stream<T, M, 4>(h, A, x, ep, part, lay, grid); break;
        case 8: mr_launch_stream<T, M, 8>(h, A, x, ep, part, lay, grid); break;
        default: mr_launch_stream<T, M, 16>(h, A, x, ep, part, lay, grid); break;
      }
      return grid;
    }
    S = 0;
  }
  if (!fine && S == 0) {
    const int R = mr_coarse_rows<T, M>(A);
    if (R > 0) {
      const size_t sm = mr_coarse_smem<T, M>(view<T>(A));
      const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (kMaxSmem + 1024) / (sm + 1024)));
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm * per_sm));
      switch (R) {
        case 1: mr_launch_coarse<T, M, 1>(A, x, ep, part, s, grid); break;
        case 2: mr_launch_coarse<T, M, 2>(A, x, ep, part, s, grid); break;
        case 4: mr_launch_coarse<T, M, 4>(A, x, ep, part, s, grid); break;
        case 8: mr_launch_coarse<T, M, 8>(A, x, ep, part, s, grid); break;
        default: mr_launch_coarse<T, M, 16>(A, x, ep, part, s, grid); break;
      }
      return grid;
    }
    S = 4;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.nbox, (int64_t)h->nsm * 8));
  if (S == 2 && CL * 2 <= 32) {
    if constexpr (CL * 2 <= 32) { if (fine) mr_launch<T, M, 2, true>(A, x, ep, part, s, grid); else mr_launch<T, M, 2, false>(A, x, ep, part, s, grid); }
  } else if (S == 8 && CL * 8 <= 32) {
    if constexpr (CL * 8 <= 32) { if (fine) mr_launch<T, M, 8, true>(A, x, ep, part, s, grid); else mr_launch<T, M, 8, false>(A, x, ep, part, s, grid); }
  } else {
    if constexpr (CL * 4 <= 32) { if (fine) mr_launch<T, M, 4, true>(A, x, ep, part, s, grid); else mr_launch<T, M, 4, false>(A, x, ep, part, s, grid); }
  }
  return grid;
}

// Entry slots per row, per level: the fastest of S in {2, 4, 8} (as far as the lanes allow) for
// one Chebyshev step on the block vectors, timed with events at setup of the block path.
template <typename T, int M>
void mr_tune(r3mg_hierarchy* h) {
  const int pi = sizeof(T) == 4 ? 1 : 0;
  std::vector<int>& Sv = h->mr_S[pi];
  if ((int)Sv.size() == h->L) return;
  Sv.assign(h->L, 4);
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  constexpr int CL = M / Slice<T>::V;
  for (int l = 0; l + 1 < h->L; ++l) {
    Level& A = h->lv[l];
    T* x = (T*)h->mr_x[l]; T* r = (T*)h->mr_r[l]; T* d = (T*)h->mr_d0[l]; T* dn = (T*)h->mr_d1[l];
    CK(cudaMemsetAsync(x, 0, sizeof(T) * A.n * M, s));
    CK(cudaMemsetAsync(r, 0, sizeof(T) * A.n * M, s));
    CK(cudaMemsetAsync(d, 0, sizeof(T) * A.n * M, s));
    float best = 1e30f;
    for (int S : {6, 5, 3, 1, 0, 2, 4, 8, 12, 14, 18, kMrGrouped}) {
      if (S == kMrGrouped) {
        if (A.b != 0) continue;
      } else if (S == 5 || S == 6) {
        if (!mr_tc_fits<T, M, MEpCheb<T, M>>(A)) continue;
      } else if (S == 3) {
        if (A.b == 0 || !mr_mma_ok<T, M, MEpCheb<T, M>>()) continue;
      } else if (S > 8) {
        if (A.b != 0 || CL * (S - 10) > 32) continue;
      } else if (CL * S > 32) {
        continue;
      }
      if (S == 0 && mr_coarse_rows<T, M>(A) == 0) continue;
      if (S == 1 && (A.b == 0 || mr_stream_layout<T, M>(A).RC == 0)) continue;
      MEpCheb<T, M> ep{x, r, d, dn, Dinv<T>(A), T(0), T(0)};
      mr_level<T, M>(h, A, d, ep, nullptr, S);
      CK(cudaEventRecord(e0, s));
      for (int k = 0; k < 3; ++k) mr_level<T, M>(h, A, d, ep, nullptr, S);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; Sv[l] = S; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// The FP64 fine product's slot count (CG product and true residual).
template <int M>
int mr_S64(r3mg_hierarchy* h) {
  if (h->mr_S[0].empty()) {
    // FP64 blocks: tuned on level 0 only when the V-cycle itself is FP32
    if (h->prm.precision == 1) {
      std::vector<int> keep = h->mr_S[1];
      h->mr_S[0].assign(h->L, 4);
      constexpr int CL = M / Slice<double>::V;
      cudaStream_t s = h->stream;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      float best = 1e30f;
      for (int S : {2, 4, 8, 12, 14, 18, kMrGrouped}) {
        if (S != kMrGrouped && CL * (S > 8 ? S - 10 : S) > 32) continue;
        mr_level<double, M>(h, h->lv[0], h->mr_p, MEpApply<double, M>{h->mr_q, nullptr}, nullptr, S);
        CK(cudaEventRecord(e0, s));
        for (int k = 0; k < 3; ++k) mr_level<double, M>(h, h->lv[0], h->mr_p, MEpApply<double, M>{h->mr_q, nullptr}, nullptr, S);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; h->mr_S[0][0] = S; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    } else {
      mr_tune<double, M>(h);
    }
  }
  return h->mr_S[0][0];
}

template <typename T, int M>
T* mr_vcycle_body(r3mg_hierarchy* h, bool capturing) {
  cudaStream_t s = h->stream;
  const int L = h->L, b = h->b;
  const int pi = sizeof(T) == 4 ? 1 : 0;
  std::vector<int> cur(L, 0);
  auto dbuf = [&](int l, int k) { return (T*)(k == 0 ? h->mr_d0[l] : h->mr_d1[l]); };
  int64_t nk = 0;
  h->slot_next = 0;
  for (int l = 0; l < L - 1; ++l) {
    Level& A = h->lv[l];
    T* x = (T*)h->mr_x[l]; T* r = (T*)h->mr_r[l];
    for (auto& ac : A.pre) {
      T* d = dbuf(l, cur[l]); T* dn = dbuf(l, cur[l] ^ 1);
      const int ps = prof_begin(h, 1 + l, capturing);
      mr_level<T, M>(h, A, d, MEpCheb<T, M>{x, r, d, dn, Dinv<T>(A), (T)ac.first, (T)ac.second}, nullptr, h->mr_S[pi][l]);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
    Level& C = h->lv[l + 1];
    const bool coarsest = (l + 1 == L - 1);
    MNextInit<T, M> nx{(T*)h->mr_r[l + 1], coarsest ? nullptr : (T*)h->mr_x[l + 1],
                       coarsest ? nullptr : dbuf(l + 1, 0), Dinv<T>(C), (T)C.c0};
    if (l == 0)
      k_mr_restrict_fine<T, M, MNextInit<T, M>><<<(int)std::min<int64_t>(C.nbox, 148 * 64), 256, 0, s>>>(
          Pmat<T>(h, 0), r, A.box_row, C.nbox, b, nx);
    else
      k_mr_restrict_coarse<T, M, MNextInit<T, M>><<<grid_for(C.nbox * b * M), 256, 0, s>>>(Pmat<T>(h, l), r, C.nbox,
                                                                                         b, h->fan, nx);
    CK(cudaGetLastError());
    ++nk;
  }
  k_mr_dense<T, M><<<grid_for(h->nc * 32), 256, 0, s>>>(Ainv<T>(h), h->ncp, (const T*)h->mr_r[L - 1], h->nc,
                                                        (T*)h->mr_x[L - 1]);
  CK(cudaGetLastError());
  ++nk;
  for (int l = L - 2; l >= 0; --l) {
    Level& A = h->lv[l];
    const bool coarsest = (l + 1 == L - 1);
    const T* x1 = (const T*)h->mr_x[l + 1];
    const T* d1 = coarsest ? nullptr : dbuf(l + 1, cur[l + 1]);
    T* d = dbuf(l, cur[l]);
    if (l == 0)
      k_mr_prolong_fine<T, M><<<grid_for(h->n * M), 256, 0, s>>>(Pmat<T>(h, 0), h->box_of_tree, x1, d1, h->n, b, d);
    else
      k_mr_prolong_coarse<T, M><<<grid_for(A.nbox * b * M), 256, 0, s>>>(Pmat<T>(h, l), x1, d1, A.nbox, b, h->fan, d);
    CK(cudaGetLastError());
    ++nk;
    T* x = (T*)h->mr_x[l]; T* r = (T*)h->mr_r[l];
    for (auto& ac : A.post) {
      T* dd = dbuf(l, cur[l]); T* dn = dbuf(l, cur[l] ^ 1);
      const int ps = prof_begin(h, 1 + l, capturing);
      mr_level<T, M>(h, A, dd, MEpCheb<T, M>{x, r, dd, dn, Dinv<T>(A), (T)ac.first, (T)ac.second}, nullptr, h->mr_S[pi][l]);
      prof_end(h, ps, capturing);
      cur[l] ^= 1;
      ++nk;
    }
  }
  if (capturing) h->mr_graph_kernels = nk; else h->launches += nk;
  return dbuf(0, cur[0]);
}

// One V-cycle on M columns of the FP64 block r_blk (tree order, interleaved) into z_blk.
template <typename T, int M>
void mr_vcycle_apply(r3mg_hierarchy* h, const double* r_blk, double* z_blk) {
  Level& F = h->lv[0];
  const int64_t nm = h->n * M;
  mr_tune<T, M>(h);
  k_mr_vc_init<T, M><<<grid_for(nm), 256, 0, h->stream>>>(r_blk, nm, (T*)h->mr_r[0], (T*)h->mr_x[0],
                                                         (T*)h->mr_d0[0], Dinv<T>(F), (T)F.c0);
  CK(cudaGetLastError());
  T* d = mr_vcycle_body<T, M>(h, false);
  k_mr_vc_final_dot<T, M><<<grid_for(nm), 256, 0, h->stream>>>((const T*)h->mr_x[0], d, z_blk, r_blk, nm, h->mr_pa);
  CK(cudaGetLastError());
}

template <int M>
void mr_reduce(r3mg_hierarchy* h, const double* part, int nb, int slot, int fin) {
  k_mr_reduce<M><<<1, 32 * M, 0, h->stream>>>(part, nb, h->mr_scal, slot, fin, h->mr_active, h->status);
  CK(cudaGetLastError());
}

// The multi-column CG/FCG loop as one graph: WHILE { product, alpha, update, ||r||, stop test,
// IF { V-cycle, beta, direction } } (the single-vector loop's structure, per column).
template <typename T, int M>
void mr_build_graph(r3mg_hierarchy* h) {
  cudaStream_t s = h->stream;
  Level& F = h->lv[0];
  const int64_t nm = h->n * M;
  const bool fcg = (h->prm.precision == 1);
  const int gv = grid_for(nm);
  const int S64 = mr_S64<M>(h);
  cudaGraph_t g = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle wh{}, ih{};
  cudaGraph_t body = nullptr, rest = nullptr;
  if (ok) ok = cudaGraphConditionalHandleCreate(&wh, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = wh;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    ok = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp) == cudaSuccess;
    if (ok) body = wp.conditional.phGraph_out[0];
  }
  if (ok) ok = cudaGraphConditionalHandleCreate(&ih, body, 0, 0) == cudaSuccess;
  if (ok) ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    bool cap_ok = true;
    try {
      const int nb = mr_level<double, M>(h, F, h->mr_p, MEpApply<double, M>{h->mr_q, h->mr_p}, h->mr_pa, S64);
      mr_reduce<M>(h, h->mr_pa, nb, S_PQ, fcg ? FIN_ALPHA_FCG : FIN_ALPHA_PCG);
      k_mr_cg_update<T, M><<<gv, 256, 0, s>>>(h->mr_xc, h->mr_rc, h->mr_p, h->mr_q, h->mr_scal, nm, h->mr_pa,
                                              (T*)h->mr_r[0], (T*)h->mr_x[0], (T*)h->mr_d0[0], Dinv<T>(F), (T)F.c0);
      CK(cudaGetLastError());
      mr_reduce<M>(h, h->mr_pa, gv, S_RR, FIN_NONE);
      k_mr_converge<M><<<1, 32, 0, s>>>(h->mr_scal, h->mr_lp, h->mr_its, h->mr_active, h->status, wh, ih, 1, nullptr);
      CK(cudaGetLastError());
      cudaStreamCaptureStatus cs;
      cudaGraph_t capg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, nullptr, &nd));
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = ih;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t inode;
      CK(cudaGraphAddNode(&inode, capg, deps, nullptr, nd, &ip));
      rest = ip.conditional.phGraph_out[0];
      CK(cudaStreamUpdateCaptureDependencies(s, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    } catch (Fail&) { cap_ok = false; }
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(s, &out) != cudaSuccess || !cap_ok) ok = false;
  }
  if (ok) ok = cudaStreamBeginCaptureToGraph(s, rest, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    bool cap_ok = true;
    try {
      T* d = mr_vcycle_body<T, M>(h, true);
      k_mr_vc_final_dot<T, M><<<gv, 256, 0, s>>>((const T*)h->mr_x[0], d, h->mr_z, fcg ? h->mr_q : h->mr_rc, nm,
                                                  h->mr_pa);
      CK(cudaGetLastError());
      mr_reduce<M>(h, h->mr_pa, gv, fcg ? S_ZQ : S_RZNEW, fcg ? FIN_BETA_FCG : FIN_BETA_PCG);
      k_mr_p_update<M><<<gv, 256, 0, s>>>(h->mr_p, h->mr_z, h->mr_rc, h->mr_scal, nm, fcg ? 1 : 0,
                                          fcg ? h->mr_pa : nullptr);
      CK(cudaGetLastError());
      if (fcg) mr_reduce<M>(h, h->mr_pa, gv, S_PR, FIN_NONE);
    } catch (Fail&) { cap_ok = false; }
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(s, &out) != cudaSuccess || !cap_ok) ok = false;
  }
  if (ok) ok = cudaGraphInstantiate(&h->mgraph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  h->mgraph_state = ok ? 1 : -1;
  if (!ok) { h->mgraph = nullptr; cudaGetLastError(); }
}

__global__ void k_mr_set_loop(double* lp, double rtol2, int budget) {
  if (threadIdx.x == 0) { lp[0] = rtol2; lp[1] = (double)budget; }
}

// Zero the columns of x whose right-hand side is zero (their solution is x = 0).
__global__ void k_mr_zero_cols(double* x, int64_t nm, int M, unsigned mask) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nm; t += (int64_t)gridDim.x * blockDim.x)
    if ((mask >> (t % M)) & 1u) x[t] = 0.0;
}

// PCG / FCG on m <= M columns at once: b and x in mr_b / mr_xc (tree order, interleaved).
template <typename T, int M>
r3mg_status mr_krylov(r3mg_hierarchy* h, int m, double rtol, int maxit, int* its_out, double* rel_out) {
  cudaStream_t s = h->stream;
  Level& F = h->lv[0];
  const int64_t nm = h->n * M;
  const bool fcg = (h->prm.precision == 1);
  const int gv = grid_for(nm);
  mr_tune<T, M>(h);
  const int S64 = mr_S64<M>(h);
  double* hs = h->mr_host;                       // [0, 16) rr, [16, 32) bb, [32, 48) its / active
  int* hi = reinterpret_cast<int*>(hs + 32);     // its: hi[0..16), active: hi[16..32)
  auto true_residual = [&](bool with_bb, bool x_zero = false) {
    // with X = 0 the residual takes X itself in place of the product A X
    if (!x_zero) mr_level<double, M>(h, F, h->mr_xc, MEpApply<double, M>{h->mr_q, nullptr}, nullptr, S64);
    k_mr_residual<M><<<gv, 256, 0, s>>>(h->mr_b, x_zero ? h->mr_xc : h->mr_q, h->mr_rc, nm, h->mr_pa,
                                        with_bb ? h->mr_pb : nullptr);
    CK(cudaGetLastError());
    k_mr_reduce<M><<<1, 32 * M, 0, s>>>(h->mr_pa, gv, h->mr_scal, S_RR, FIN_NONE, nullptr, nullptr);
    if (with_bb) k_mr_reduce<M><<<1, 32 * M, 0, s>>>(h->mr_pb, gv, h->mr_scal, S_BB, FIN_NONE, nullptr, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hs, h->mr_scal + S_RR * M, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
    if (with_bb) CK(cudaMemcpyAsync(hs + 16, h->mr_scal + S_BB * M, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->launches += with_bb ? 4 : 3;
  };
  auto restart = [&]() {   // z = M r; p = z; per column rz (PCG) or pr (FCG)
    k_mr_hist_reset<M><<<1, 32, 0, s>>>(h->mr_scal, h->mr_active);   // new Lanczos sequences
    mr_vcycle_apply<T, M>(h, h->mr_rc, h->mr_z);
    mr_reduce<M>(h, h->mr_pa, gv, fcg ? S_PR : S_RZ, FIN_NONE);
    CK(cudaMemcpyAsync(h->mr_p, h->mr_z, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    h->launches += 3;
  };
  h->mr_last_m = m;
  CK(cudaMemsetAsync(h->mr_scal + S_NA * M, 0, 2 * M * sizeof(double), s));   // no coefficients yet
  true_residual(true, all_zero(h, h->mr_xc, nm));
  std::vector<double> bb(M), rel(M, 0.0), thr2(M, 0.0);
  std::vector<int> its(M, 0), act(M, 0);
  unsigned zero_mask = 0;
  double* hthr = hs + 64;   // pinned: the per-column thresholds uploaded to mscal[S_THR]
  for (int c = 0; c < M; ++c) {
    bb[c] = hs[16 + c];
    if (c < m && bb[c] == 0.0) zero_mask |= 1u << c;
    rel[c] = (bb[c] > 0.0) ? std::sqrt(hs[c] / bb[c]) : 0.0;
    // ||r_c|| <= max(rtol ||b_c||, atol, reduction ||r_c,0||), as in the single-vector solve
    const double t = std::max(rtol * std::sqrt(bb[c]), std::max(h->stop_atol, h->stop_red * std::sqrt(hs[c])));
    thr2[c] = t * t;
    hthr[c] = thr2[c];
    act[c] = (c < m && bb[c] > 0.0 && !(hs[c] <= thr2[c]) && maxit > 0) ? 1 : 0;
  }
  CK(cudaMemcpyAsync(h->mr_scal + S_THR * M, hthr, sizeof(double) * M, cudaMemcpyHostToDevice, s));
  if (zero_mask) {
    k_mr_zero_cols<<<gv, 256, 0, s>>>(h->mr_xc, nm, M, zero_mask);
    CK(cudaGetLastError());
  }
  auto upload_active = [&]() {
    for (int c = 0; c < M; ++c) { hi[c] = its[c]; hi[16 + c] = act[c]; }
    CK(cudaMemcpyAsync(h->mr_its, hi, sizeof(int) * M, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->mr_active, hi + 16, sizeof(int) * M, cudaMemcpyHostToDevice, s));
  };
  bool any = false;
  std::vector<char> conv_c(M, 0);
  for (int c = 0; c < M; ++c) { any = any || act[c]; conv_c[c] = (c < m && !act[c] && hs[c] <= thr2[c]); }
  if (any) {
    upload_active();
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    restart();
    if (!h->prof_on) {
      if (h->mgraph_state == 0) mr_build_graph<T, M>(h);
      if (h->mgraph_state != 1) throw Fail{R3MG_E_CUDA, "pcg_multi: the conditional loop graph could not be built"};
    }
    while (true) {
      k_mr_set_loop<<<1, 32, 0, s>>>(h->mr_lp, rtol * rtol, maxit);
      CK(cudaGetLastError());
      if (!h->prof_on) {
        CK(cudaGraphLaunch(h->mgraph, s));
      } else {
        // profiled solves: the same iteration driven from the host, events around the level
        // operators (kind 0: the FP64 block product, kind 1 + l: Chebyshev steps on level l)
        const cudaGraphConditionalHandle none{};
        int* go = h->mr_its + M;
        for (int it = 0; it < maxit; ++it) {
          if (!h->cg_slot.e0) { CK(cudaEventCreate(&h->cg_slot.e0)); CK(cudaEventCreate(&h->cg_slot.e1)); }
          CK(cudaEventRecord(h->cg_slot.e0, s));
          const int nb = mr_level<double, M>(h, F, h->mr_p, MEpApply<double, M>{h->mr_q, h->mr_p}, h->mr_pa, S64);
          CK(cudaEventRecord(h->cg_slot.e1, s));
          h->cg_pending = true;
          mr_reduce<M>(h, h->mr_pa, nb, S_PQ, fcg ? FIN_ALPHA_FCG : FIN_ALPHA_PCG);
          k_mr_cg_update<T, M><<<gv, 256, 0, s>>>(h->mr_xc, h->mr_rc, h->mr_p, h->mr_q, h->mr_scal, nm, h->mr_pa,
                                                  (T*)h->mr_r[0], (T*)h->mr_x[0], (T*)h->mr_d0[0], Dinv<T>(F), (T)F.c0);
          CK(cudaGetLastError());
          mr_reduce<M>(h, h->mr_pa, gv, S_RR, FIN_NONE);
          k_mr_converge<M><<<1, 32, 0, s>>>(h->mr_scal, h->mr_lp, h->mr_its, h->mr_active, h->status, none, none, 0, go);
          CK(cudaGetLastError());
          CK(cudaMemcpyAsync(hi + 48, go, sizeof(int), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          prof_harvest(h);
          h->launches += 5;
          if (!hi[48]) break;
          T* d = mr_vcycle_body<T, M>(h, false);
          k_mr_vc_final_dot<T, M><<<gv, 256, 0, s>>>((const T*)h->mr_x[0], d, h->mr_z, fcg ? h->mr_q : h->mr_rc, nm,
                                                      h->mr_pa);
          CK(cudaGetLastError());
          mr_reduce<M>(h, h->mr_pa, gv, fcg ? S_ZQ : S_RZNEW, fcg ? FIN_BETA_FCG : FIN_BETA_PCG);
          k_mr_p_update<M><<<gv, 256, 0, s>>>(h->mr_p, h->mr_z, h->mr_rc, h->mr_scal, nm, fcg ? 1 : 0,
                                              fcg ? h->mr_pa : nullptr);
          CK(cudaGetLastError());
          if (fcg) mr_reduce<M>(h, h->mr_pa, gv, S_PR, FIN_NONE);
          h->launches += fcg ? 5 : 4;
        }
      }
      CK(cudaMemcpyAsync(hi, h->mr_its, sizeof(int) * M, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hi + 32, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int added = 0;
      for (int c = 0; c < M; ++c) { added = std::max(added, hi[c] - its[c]); its[c] = hi[c]; }
      if (!h->prof_on) h->launches += 1 + (int64_t)added * (h->mr_graph_kernels + (fcg ? 9 : 8));
      if (hi[32]) {
        CK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
        throw Fail{R3MG_E_BREAKDOWN, "pcg_multi: breakdown (p^T A p <= 0 or non-finite scalar) in a column"};
      }
      true_residual(false);
      bool again = false;
      for (int c = 0; c < M; ++c) {
        if (c >= m || bb[c] == 0.0) { act[c] = 0; continue; }
        rel[c] = std::sqrt(hs[c] / bb[c]);
        if (!std::isfinite(rel[c])) throw Fail{R3MG_E_BREAKDOWN, "pcg_multi: non-finite residual"};
        act[c] = (hs[c] > thr2[c] && its[c] < maxit) ? 1 : 0;
        conv_c[c] = hs[c] <= thr2[c];
        again = again || act[c];
      }
      if (!again) break;
      upload_active();   // recursive residual drifted in some column: restart those from the true residual
      restart();
    }
  }
  bool conv = true;
  for (int c = 0; c < m; ++c) {
    its_out[c] = its[c];
    rel_out[c] = rel[c];
    conv = conv && (bb[c] == 0.0 || conv_c[c]);
  }
  return conv ? R3MG_OK : R3MG_E_NOCONV;
}

template <int M>
r3mg_status mr_dispatch_solve(r3mg_hierarchy* h, int m, double rtol, int maxit, int* its, double* rel) {
  mr_alloc(h, M);
  return (h->prm.precision == 1) ? mr_krylov<float, M>(h, m, rtol, maxit, its, rel)
                                 : mr_krylov<double, M>(h, m, rtol, maxit, its, rel);
}

template <int M>
void mr_dispatch_vcycle(r3mg_hierarchy* h) {
  mr_alloc(h, M);
  if (h->prm.precision == 1) mr_vcycle_apply<float, M>(h, h->mr_b, h->mr_z);
  else mr_vcycle_apply<double, M>(h, h->mr_b, h->mr_z);
}

// Y = A_l X on M columns: FP64 values (fp32 = 0) or the FP32 V-cycle values (fp32 = 1).
template <typename T, int M>
void mr_apply_level(r3mg_hierarchy* h, int level, const double* x_blk, double* y_blk) {
  Level& A = h->lv[level];
  const int pi = sizeof(T) == 4 ? 1 : 0;
  if (pi == 1) mr_tune<float, M>(h); else mr_S64<M>(h);
  // the configured choice of this level (FP64 blocks of a mixed hierarchy are tuned on level 0 only)
  const int lv = std::min(level, h->L - 2);
  const int S = pi == 1 ? h->mr_S[1][lv] : (h->prm.precision == 0 || level == 0 ? h->mr_S[0][lv] : 4);
  const int64_t nm = A.n * M;
  // scratch of level 0's size in the right precision (level 0 is the largest level)
  T* xt = pi == 1 ? (T*)h->mr_d0[0] : (T*)h->mr_p;
  T* yt = pi == 1 ? (T*)h->mr_d1[0] : (T*)h->mr_q;
  k_convert<double, T><<<grid_for(nm), 256, 0, h->stream>>>(x_blk, xt, nm);
  mr_level<T, M>(h, A, xt, MEpApply<T, M>{yt, nullptr}, nullptr, S);
  k_convert<T, double><<<grid_for(nm), 256, 0, h->stream>>>(yt, y_blk, nm);
  CK(cudaGetLastError());
}

}  // namespace

// ================================================================ C ABI
extern "C" {

void r3mg_default_params(r3mg_params* p) {
  if (!p) return;
  p->leaf_size = 64; p->pprime = 1; p->levels = 3; p->cheb_degree = 3; p->sweeps = 2; p->lanczos_steps = 10;
  p->eig_safety = 1.1; p->eig_ratio = 30.0; p->precision = 0; p->group_lanes = 0; p->seed = 0x5EED;
  p->kernel_form = 0;
}

r3mg_status r3mg_partition(int64_t n, int dim, const double* coords_host, int leaf_size, int levels, int64_t* perm_out,
                           int64_t* leaf_offsets_out, int* depth_out) {
  if (!coords_host || !perm_out) { g_last_error = "partition: null pointer"; return R3MG_E_ARG; }
  HostPartition P;
  Error err;
  try {
    if (!partition_points(n, dim, coords_host, leaf_size, levels, P, err)) { g_last_error = err.msg; return err.status; }
  } catch (std::bad_alloc&) { g_last_error = "host allocation failed"; return R3MG_E_OOM; }
  std::memcpy(perm_out, P.perm.data(), sizeof(int64_t) * n);
  if (leaf_offsets_out) std::memcpy(leaf_offsets_out, P.leaf_off.data(), sizeof(int64_t) * P.leaf_off.size());
  if (depth_out) *depth_out = P.depth;
  return R3MG_OK;
}

r3mg_status r3mg_group_rows(int64_t n, const int64_t* row_ptr, int64_t nbox, const int64_t* box_row,
                            const uint16_t* idx, int64_t* counts_out, int32_t* rows_out) {
  if (!row_ptr || !box_row || !counts_out || (n > 0 && !rows_out)) { g_last_error = "group_rows: null pointer"; return R3MG_E_ARG; }
  if (n < 0 || nbox < 1 || n > INT32_MAX || row_ptr[0] != 0 || box_row[0] != 0 || box_row[nbox] != n) {
    g_last_error = "group_rows: need n >= 0 rows (below 2^31), nbox >= 1, row_ptr[0] = 0 and box_row from 0 to n";
    return R3MG_E_ARG;
  }
  for (int64_t B = 0; B < nbox; ++B)
    if (box_row[B + 1] < box_row[B]) { g_last_error = "group_rows: box_row must not decrease"; return R3MG_E_ARG; }
  for (int64_t r = 0; r < n; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) { g_last_error = "group_rows: row_ptr must not decrease"; return R3MG_E_ARG; }
  if (row_ptr[n] > 0 && !idx) { g_last_error = "group_rows: null pointer"; return R3MG_E_ARG; }
  try {
    const RowGroups grp = group_rows_host(row_ptr, nbox, box_row, idx);
    for (int c = 0; c < 4; ++c) counts_out[c] = grp.ng[c];
    if (n > 0) std::memcpy(rows_out, grp.rows.data(), sizeof(int32_t) * n);
  } catch (std::bad_alloc&) { g_last_error = "host allocation failed"; return R3MG_E_OOM; }
  return R3MG_OK;
}

static r3mg_status setup_common(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                                const int32_t* colidx_host, const double* vals_host, const CellsIn* cells,
                                const r3mg_params* params, void* stream, r3mg_hierarchy** out);

r3mg_status r3mg_setup(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                       const int32_t* colidx_host, const double* vals_host, const r3mg_params* params, void* stream,
                       r3mg_hierarchy** out) {
  return setup_common(n, dim, coords_host, rowptr_host, colidx_host, vals_host, nullptr, params, stream, out);
}

r3mg_status r3mg_setup_cells(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                             const int32_t* colidx_host, const double* vals_host, int64_t ncells,
                             const int64_t* cell_ptr_host, const int64_t* cell_pts_host, const r3mg_params* params,
                             void* stream, r3mg_hierarchy** out) {
  if (ncells < 1 || !cell_ptr_host || !cell_pts_host) {
    g_last_error = "setup_cells: need ncells >= 1 and non-null cell arrays";
    if (out) *out = nullptr;
    return R3MG_E_ARG;
  }
  const CellsIn cells{ncells, cell_ptr_host, cell_pts_host};
  return setup_common(n, dim, coords_host, rowptr_host, colidx_host, vals_host, &cells, params, stream, out);
}

r3mg_status r3mg_partition_cells(int64_t n, int dim, const double* coords_host, int64_t ncells,
                                 const int64_t* cell_ptr_host, const int64_t* cell_pts_host, int leaf_size, int levels,
                                 int64_t* perm_out, int64_t* box_offsets_out, double* box_lo_out, double* box_hi_out,
                                 int* depth_out) {
  if (!coords_host || !cell_ptr_host || !cell_pts_host || !perm_out) {
    g_last_error = "partition_cells: null pointer";
    return R3MG_E_ARG;
  }
  HostPartition P;
  Error err;
  try {
    if (!partition_cells(n, dim, coords_host, ncells, cell_ptr_host, cell_pts_host, leaf_size, levels, P, err)) {
      g_last_error = err.msg;
      return err.status;
    }
  } catch (std::bad_alloc&) { g_last_error = "host allocation failed"; return R3MG_E_OOM; }
  std::memcpy(perm_out, P.perm.data(), sizeof(int64_t) * n);
  if (box_offsets_out) std::memcpy(box_offsets_out, P.box_off[1].data(), sizeof(int64_t) * P.box_off[1].size());
  if (box_lo_out) std::memcpy(box_lo_out, P.lo[1].data(), sizeof(double) * P.lo[1].size());
  if (box_hi_out) std::memcpy(box_hi_out, P.hi[1].data(), sizeof(double) * P.hi[1].size());
  if (depth_out) *depth_out = P.depth;
  return R3MG_OK;
}

static r3mg_status setup_common(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_host,
                                const int32_t* colidx_host, const double* vals_host, const CellsIn* cells,
                                const r3mg_params* params, void* stream, r3mg_hierarchy** out) {
  if (!out) { g_last_error = "setup: null output"; return R3MG_E_ARG; }
  *out = nullptr;
  if (!coords_host || !rowptr_host || !colidx_host || !vals_host || n < 1 || (dim != 2 && dim != 3)) {
    g_last_error = "setup: null pointer, n < 1 or dim not in {2,3}";
    return R3MG_E_ARG;
  }
  r3mg_hierarchy* h = new (std::nothrow) r3mg_hierarchy();
  if (!h) return R3MG_E_OOM;
  if (params) h->prm = *params; else r3mg_default_params(&h->prm);
  const r3mg_params& p = h->prm;
  int b = 1;
  for (int a = 0; a < dim; ++a) b *= (p.pprime + 1);
  // leaf_size counts points (>= (p'+1)^d) for point-based agglomeration, cells (>= 2) for cell-based
  const bool leaf_ok = cells ? p.leaf_size >= 2 : p.leaf_size >= b;
  if (p.pprime < 0 || p.pprime > 8 || b > 64 || !leaf_ok || p.levels < 2 || p.cheb_degree < 1 || p.sweeps < 1 ||
      p.lanczos_steps < 1 || !(p.eig_safety > 0) || !(p.eig_ratio > 1) || (p.precision != 0 && p.precision != 1) ||
      (p.group_lanes != 0 && p.group_lanes != 4 && p.group_lanes != 8 && p.group_lanes != 16 && p.group_lanes != 32) ||
      p.kernel_form < 0 || p.kernel_form > 2) {
    g_last_error = "setup: invalid parameters (need 0 <= p' <= 8, (p'+1)^d <= 64, leaf >= (p'+1)^d points or >= 2 cells, levels >= 2, "
                   "degree >= 1, sweeps >= 1, lanes in {0,4,8,16,32}, precision in {0,1})";
    delete h;
    return R3MG_E_ARG;
  }
  h->n = n; h->dim = dim;
  r3mg_status st = guarded(h, [&] {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CK(cudaMallocHost(&h->host_scal, sizeof(double) * 16));
    h->status = dalloc<int>(h, 1);
    h->tma_err = dalloc<int>(h, 1);
    // the allocation-free product's static scratch: its device address on this device
    CK(cudaGetSymbolAddress((void**)&h->noalloc_scratch, g_noalloc_scratch));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(h->tma_err, 0, sizeof(int), h->stream));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
    StreamJoin j(h, stream);
    build(h, coords_host, rowptr_host, colidx_host, vals_host, cells);
    CK(cudaStreamSynchronize(h->stream));
  });
  if (st != R3MG_OK) {
    g_last_error = h->err;
    r3mg_destroy(h);
    return st;
  }
  *out = h;
  return R3MG_OK;
}

r3mg_status r3mg_batch_setup(int nprob, int dim, const int64_t* n, const double* const* coords_host,
                             const int64_t* const* rowptr_host, const int32_t* const* colidx_host,
                             const double* const* vals_host, const r3mg_params* params, void* stream,
                             r3mg_hierarchy** out) {
  if (!out) { g_last_error = "batch_setup: null output"; return R3MG_E_ARG; }
  *out = nullptr;
  if (nprob < 1 || (dim != 2 && dim != 3) || !n || !coords_host || !rowptr_host || !colidx_host || !vals_host) {
    g_last_error = "batch_setup: need nprob >= 1, dim in {2,3} and non-null arrays";
    return R3MG_E_ARG;
  }
  for (int k = 0; k < nprob; ++k)
    if (n[k] < 1 || !coords_host[k] || !rowptr_host[k] || !colidx_host[k] || !vals_host[k]) {
      g_last_error = "batch_setup: problem " + std::to_string(k) + " is empty or has a null array";
      return R3MG_E_ARG;
    }
  r3mg_hierarchy* h = new (std::nothrow) r3mg_hierarchy();
  if (!h) return R3MG_E_OOM;
  if (params) h->prm = *params; else r3mg_default_params(&h->prm);
  const r3mg_params& p = h->prm;
  int b = 1;
  for (int a = 0; a < dim; ++a) b *= (p.pprime + 1);
  if (p.pprime < 0 || p.pprime > 8 || b > 64 || p.leaf_size < b || p.levels < 2 || p.cheb_degree < 1 || p.sweeps < 1 ||
      p.lanczos_steps < 1 || !(p.eig_safety > 0) || !(p.eig_ratio > 1) || (p.precision != 0 && p.precision != 1) ||
      (p.group_lanes != 0 && p.group_lanes != 4 && p.group_lanes != 8 && p.group_lanes != 16 && p.group_lanes != 32) ||
      p.kernel_form < 0 || p.kernel_form > 2) {
    g_last_error = "batch_setup: invalid parameters";
    delete h;
    return R3MG_E_ARG;
  }
  h->dim = dim;
  r3mg_status st = guarded(h, [&] {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CK(cudaMallocHost(&h->host_scal, sizeof(double) * 16));
    h->status = dalloc<int>(h, 1);
    h->tma_err = dalloc<int>(h, 1);
    // the allocation-free product's static scratch: its device address on this device
    CK(cudaGetSymbolAddress((void**)&h->noalloc_scratch, g_noalloc_scratch));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(h->tma_err, 0, sizeof(int), h->stream));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
    StreamJoin j(h, stream);
    build_batch(h, nprob, n, coords_host, rowptr_host, colidx_host, vals_host);
    CK(cudaStreamSynchronize(h->stream));
  });
  if (st != R3MG_OK) {
    g_last_error = h->err;
    r3mg_destroy(h);
    return st;
  }
  *out = h;
  return R3MG_OK;
}

r3mg_status r3mg_batch_pcg(r3mg_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit,
                           int* iters_out, double* relres_out, void* stream) {
  if (!h || !b_dev || !x_dev || maxit < 0 || !(rtol >= 0.0) || !iters_out || !relres_out) return R3MG_E_ARG;
  if (h->bl.empty()) {
    int it = 0; double rel = 0.0;
    r3mg_status s1 = r3mg_pcg(h, b_dev, x_dev, rtol, maxit, &it, &rel, stream);
    iters_out[0] = it; relres_out[0] = rel;
    return s1;
  }
  r3mg_status res = R3MG_OK;
  r3mg_status st = guarded(h, [&] {
    StreamJoin j(h, stream);
    const int gv = grid_for(h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(b_dev, h->perm, h->cb, h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(x_dev, h->perm, h->cx, h->n);
    CK(cudaGetLastError());
    if (h->prof_on) h->prof_cols = 1;
    res = (h->prm.precision == 1) ? krylov_batch<float>(h, rtol, maxit, iters_out, relres_out)
                                  : krylov_batch<double>(h, rtol, maxit, iters_out, relres_out);
    k_scatter_perm<double, double><<<gv, 256, 0, h->stream>>>(h->cx, h->perm, x_dev, h->n);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
  });
  if (st != R3MG_OK) return st;
  if (res == R3MG_E_NOCONV) h->err = "batched PCG: a problem reached maxit";
  return res;
}

r3mg_status r3mg_batch_offsets(const r3mg_hierarchy* h, int level, int* nprob_out, int64_t* row_off_host) {
  if (!h || level < 0 || level >= h->L) return R3MG_E_ARG;
  if (nprob_out) *nprob_out = h->nprob;
  if (row_off_host) {
    if (!h->bl.empty()) {
      std::memcpy(row_off_host, h->bl[level].row_off.data(), sizeof(int64_t) * (h->nprob + 1));
    } else {
      row_off_host[0] = 0;
      row_off_host[1] = h->lv[level].n;
    }
  }
  return R3MG_OK;
}

r3mg_status r3mg_update_values(r3mg_hierarchy* h, const double* vals_dev, void* stream) {
  if (!h || !vals_dev) return R3MG_E_ARG;
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    numeric(h, vals_dev);
  });
}

r3mg_status r3mg_vcycle(r3mg_hierarchy* h, const double* r_dev, double* z_dev, void* stream) {
  if (!h || !r_dev || !z_dev) return R3MG_E_ARG;
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    const int gv = grid_for(h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(r_dev, h->perm, h->cb, h->n);
    CK(cudaGetLastError());
    if (h->prm.precision == 1) vcycle_apply<float>(h, h->cb, h->cz);
    else vcycle_apply<double>(h, h->cb, h->cz);
    k_scatter_perm<double, double><<<gv, 256, 0, h->stream>>>(h->cz, h->perm, z_dev, h->n);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_pcg(r3mg_hierarchy* h, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters_out,
                     double* relres_out, void* stream) {
  if (!h || !b_dev || !x_dev || maxit < 0 || !(rtol >= 0.0)) return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "pcg: batched hierarchy, use r3mg_batch_pcg"; return R3MG_E_ARG; }
  int it = 0;
  double rel = 0.0;
  r3mg_status res = R3MG_OK;
  r3mg_status st = guarded(h, [&] {
    StreamJoin j(h, stream);
    const int gv = grid_for(h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(b_dev, h->perm, h->cb, h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(x_dev, h->perm, h->cx, h->n);
    CK(cudaGetLastError());
    if (h->prof_on) h->prof_cols = 1;
    res = (h->prm.precision == 1) ? krylov<float>(h, rtol, maxit, &it, &rel) : krylov<double>(h, rtol, maxit, &it, &rel);
    k_scatter_perm<double, double><<<gv, 256, 0, h->stream>>>(h->cx, h->perm, x_dev, h->n);
    CK(cudaGetLastError());
    h->launches += 3;
    CK(cudaStreamSynchronize(h->stream));
    prof_harvest(h);
    int terr = 0;
    CK(cudaMemcpy(&terr, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (terr) {
      CK(cudaMemset(h->tma_err, 0, sizeof(int)));
      throw Fail{R3MG_E_TIMEOUT, "a bounded wait of the TMA-streamed level kernel expired"};
    }
  });
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = rel;
  if (st != R3MG_OK) return st;
  if (res == R3MG_E_NOCONV) h->err = "PCG: maximum iterations reached";
  return res;
}

r3mg_status r3mg_pcg_multi(r3mg_hierarchy* h, int m, const double* b_dev, double* x_dev, double rtol, int maxit,
                           int* iters_out, double* relres_out, void* stream) {
  if (!h || m < 1 || m > 16 || !b_dev || !x_dev || !iters_out || !relres_out || maxit < 0 || !(rtol >= 0.0))
    return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "pcg_multi: batched hierarchy"; return R3MG_E_ARG; }
  r3mg_status res = R3MG_OK;
  for (int c = 0; c < m; ++c) { iters_out[c] = 0; relres_out[c] = 0.0; }
  r3mg_status st = guarded(h, [&] {
    StreamJoin j(h, stream);
    const int M = mr_cols(m);
    mr_alloc(h, M);
    const int64_t nm = h->n * M;
    k_mr_gather<<<grid_for(nm), 256, 0, h->stream>>>(b_dev, h->perm, h->n, m, M, h->mr_b);
    k_mr_gather<<<grid_for(nm), 256, 0, h->stream>>>(x_dev, h->perm, h->n, m, M, h->mr_xc);
    CK(cudaGetLastError());
    if (h->prof_on) h->prof_cols = M;
    res = M == 4 ? mr_dispatch_solve<4>(h, m, rtol, maxit, iters_out, relres_out)
        : M == 8 ? mr_dispatch_solve<8>(h, m, rtol, maxit, iters_out, relres_out)
                 : mr_dispatch_solve<16>(h, m, rtol, maxit, iters_out, relres_out);
    k_mr_scatter<<<grid_for(nm), 256, 0, h->stream>>>(h->mr_xc, h->perm, h->n, m, M, x_dev);
    CK(cudaGetLastError());
    h->launches += 3;
    CK(cudaStreamSynchronize(h->stream));
    prof_harvest(h);
    int terr = 0;
    CK(cudaMemcpy(&terr, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (terr) {
      CK(cudaMemset(h->tma_err, 0, sizeof(int)));
      throw Fail{R3MG_E_TIMEOUT, "a bounded wait of the streamed block kernel expired"};
    }
  });
  if (st != R3MG_OK) return st;
  if (res == R3MG_E_NOCONV) h->err = "pcg_multi: maximum iterations reached in some column";
  return res;
}

r3mg_status r3mg_vcycle_multi(r3mg_hierarchy* h, int m, const double* r_dev, double* z_dev, void* stream) {
  if (!h || m < 1 || m > 16 || !r_dev || !z_dev) return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "vcycle_multi: batched hierarchy"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    const int M = mr_cols(m);
    mr_alloc(h, M);
    const int64_t nm = h->n * M;
    k_mr_gather<<<grid_for(nm), 256, 0, h->stream>>>(r_dev, h->perm, h->n, m, M, h->mr_b);
    CK(cudaGetLastError());
    if (M == 4) mr_dispatch_vcycle<4>(h); else if (M == 8) mr_dispatch_vcycle<8>(h); else mr_dispatch_vcycle<16>(h);
    k_mr_scatter<<<grid_for(nm), 256, 0, h->stream>>>(h->mr_z, h->perm, h->n, m, M, z_dev);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_block_config(r3mg_hierarchy* h, int level, int fp32, int* slots) {
  if (!h || level < 0 || level >= h->L || !slots) return R3MG_E_ARG;
  const auto& Sv = h->mr_S[fp32 ? 1 : 0];
  *slots = level < (int)Sv.size() ? Sv[level] : -1;
  return R3MG_OK;
}

r3mg_status r3mg_set_block_config(r3mg_hierarchy* h, int level, int fp32, int slots) {
  if (!h || level < 0 || level >= h->L) return R3MG_E_ARG;
  if (!(slots == 0 || slots == 1 || slots == 2 || slots == 3 || slots == 4 || slots == 5 || slots == 6 ||
        slots == 8 || slots == 12 || slots == 14 || slots == 18 || slots == kMrGrouped)) {
    h->err = "set_block_config: slots must be 0, 1, 2, 3, 4, 5, 6, 8, 12, 14, 18 or 20";
    return R3MG_E_ARG;
  }
  if (slots > 8 && h->lv[level].b != 0) {
    h->err = "set_block_config: the flat row sweep and the grouped rows are for the fine level";
    return R3MG_E_ARG;
  }
  if ((slots <= 1 || slots == 3 || slots == 5 || slots == 6) && h->lv[level].b == 0) {
    h->err = "set_block_config: the staged, streamed and tensor-core forms are for coarse levels";
    return R3MG_E_ARG;
  }
  if (slots == 3 && (!fp32 || (h->mr_M != 8 && h->mr_M != 16))) {
    h->err = "set_block_config: the tensor-core form is FP32 with 8 or 16 columns";
    return R3MG_E_ARG;
  }
  if (fp32 && h->prm.precision != 1) { h->err = "set_block_config: the hierarchy has no FP32 V-cycle"; return R3MG_E_ARG; }
  if (h->mr_M == 0) { h->err = "set_block_config: no block solve has run yet (nothing tuned)"; return R3MG_E_ARG; }
  auto& Sv = h->mr_S[fp32 ? 1 : 0];
  if ((int)Sv.size() != h->L) { h->err = "set_block_config: this precision is not tuned yet"; return R3MG_E_ARG; }
  if ((slots == 5 || slots == 6) && (!fp32 || h->mr_M != 16 || h->lv[level].b > kTcRows)) {
    h->err = "set_block_config: the tcgen05 form is FP32 with 16 columns and boxes of at most 32 rows";
    return R3MG_E_ARG;
  }
  const int CL = h->mr_M / (fp32 ? 4 : 2);
  if (slots != 3 && slots != 5 && slots != 6 && slots != kMrGrouped && CL * (slots > 8 ? slots - 10 : slots) > 32) {
    h->err = "set_block_config: too many slots for the column count";
    return R3MG_E_ARG;
  }
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    Sv[level] = slots;
    drop_graphs(h);
  });
}

r3mg_status r3mg_level_apply_multi(r3mg_hierarchy* h, int level, int m, int fp32, const double* x_dev, double* y_dev,
                                   void* stream) {
  if (!h || level < 0 || level >= h->L || m < 1 || m > 16 || !x_dev || !y_dev) return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "level_apply_multi: batched hierarchy"; return R3MG_E_ARG; }
  if (fp32 && h->prm.precision != 1) { h->err = "level_apply_multi: the hierarchy has no FP32 values"; return R3MG_E_ARG; }
  if (fp32 && level == h->L - 1) {
    h->err = "level_apply_multi: the coarsest level has no FP32 values (it is solved with its inverse)";
    return R3MG_E_ARG;
  }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    const int M = mr_cols(m);
    mr_alloc(h, M);
    const int64_t nl = h->lv[level].n, nm = nl * M;
    // caller columns -> interleaved block (level 0: caller numbering -> tree order)
    double* xb = h->mr_b;
    double* yb = h->mr_z;
    k_mr_gather<<<grid_for(nm), 256, 0, h->stream>>>(x_dev, level == 0 ? h->perm : nullptr, nl, m, M, xb);
    CK(cudaGetLastError());
    auto run = [&](auto tag) {
      constexpr int MM = decltype(tag)::value;
      if (fp32) mr_apply_level<float, MM>(h, level, xb, yb); else mr_apply_level<double, MM>(h, level, xb, yb);
    };
    if (M == 4) run(std::integral_constant<int, 4>{});
    else if (M == 8) run(std::integral_constant<int, 8>{});
    else run(std::integral_constant<int, 16>{});
    k_mr_scatter<<<grid_for(nm), 256, 0, h->stream>>>(yb, level == 0 ? h->perm : nullptr, nl, m, M, y_dev);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_pcg_host(r3mg_hierarchy* h, const double* b_host, double* x_host, double rtol, int maxit,
                          int* iters_out, double* relres_out, void* stream) {
  if (!h || !b_host || !x_host) return R3MG_E_ARG;
  r3mg_status st = guarded(h, [&] {
    if (!h->hb_dev) { h->hb_dev = dalloc<double>(h, h->n); h->hx_dev = dalloc<double>(h, h->n); }
    cudaStream_t us = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h->hb_dev, b_host, sizeof(double) * h->n, cudaMemcpyHostToDevice, us));
    CK(cudaMemcpyAsync(h->hx_dev, x_host, sizeof(double) * h->n, cudaMemcpyHostToDevice, us));
  });
  if (st != R3MG_OK) return st;
  r3mg_status res = r3mg_pcg(h, h->hb_dev, h->hx_dev, rtol, maxit, iters_out, relres_out, stream);
  r3mg_status st2 = guarded(h, [&] {
    CK(cudaMemcpyAsync(x_host, h->hx_dev, sizeof(double) * h->n, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
  });
  return res == R3MG_OK ? st2 : res;
}

r3mg_status r3mg_coarse_solve(r3mg_hierarchy* h, const double* r_dev, double* z_dev, void* stream) {
  if (!h || !r_dev || !z_dev) return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "coarse_solve: batched hierarchy"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    coarsest_apply<double>(h, r_dev, z_dev);
  });
}

r3mg_status r3mg_level_apply(r3mg_hierarchy* h, int level, const double* x_dev, double* y_dev, void* stream) {
  if (!h || level < 0 || level >= h->L || !x_dev || !y_dev) return R3MG_E_ARG;
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    Level& A = h->lv[level];
    if (level == 0) {
      const int gv = grid_for(h->n);
      k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(x_dev, h->perm, h->cb, h->n);
      level_apply_dot<double>(h, A, h->cb, h->cz, nullptr, nullptr);
      k_scatter_perm<double, double><<<gv, 256, 0, h->stream>>>(h->cz, h->perm, y_dev, h->n);
    } else {
      level_apply_dot<double>(h, A, x_dev, y_dev, nullptr, nullptr);
    }
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_info(const r3mg_hierarchy* h, int* levels_out, int* depth_out, int64_t* n_out, int64_t* nnz_out,
                      int64_t* nbox_out, double* lam_out) {
  if (!h) return R3MG_E_ARG;
  if (levels_out) *levels_out = h->L;
  if (depth_out) *depth_out = h->part.depth;
  for (int l = 0; l < h->L; ++l) {
    if (n_out) n_out[l] = h->lv[l].n;
    if (nnz_out) nnz_out[l] = h->lv[l].nnz;
    if (nbox_out) nbox_out[l] = h->lv[l].nbox;
    if (lam_out) lam_out[l] = h->lv[l].lam_hi;
  }
  return R3MG_OK;
}

r3mg_status r3mg_get_agglomerates(const r3mg_hierarchy* h, int level, int64_t* box_of_point_host) {
  if (!h || level < 1 || level >= h->L || !box_of_point_host) return R3MG_E_ARG;
  const std::vector<int64_t>& off = h->part.box_off[level];
  for (int64_t B = 0; B + 1 < (int64_t)off.size(); ++B)
    for (int64_t k = off[B]; k < off[B + 1]; ++k) box_of_point_host[h->part.perm[k]] = B;
  return R3MG_OK;
}

r3mg_status r3mg_get_level_pattern(const r3mg_hierarchy* h, int level, int64_t* nbr_ptr_host, int64_t* nbr_host) {
  if (!h || level < 1 || level >= h->L || !nbr_ptr_host) return R3MG_E_ARG;
  const HostPattern& pt = h->lv[level].pat;
  std::memcpy(nbr_ptr_host, pt.ptr.data(), sizeof(int64_t) * pt.ptr.size());
  if (nbr_host) std::memcpy(nbr_host, pt.nbr.data(), sizeof(int64_t) * pt.nbr.size());
  return R3MG_OK;
}

r3mg_status r3mg_get_level_blocks(r3mg_hierarchy* h, int level, double* vals_host) {
  if (!h || level < 1 || level >= h->L || !vals_host) return R3MG_E_ARG;
  return guarded(h, [&] {
    Level& C = h->lv[level];
    double* tmp = dalloc<double>(h, C.npairs * h->b * h->b);
    k_blocks_export<<<grid_for(C.npairs * h->b * h->b), 256, 0, h->stream>>>(C.pair_box, C.nbr_ptr, C.row_ptr, C.v64,
                                                                              C.npairs, h->b, tmp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(vals_host, tmp, sizeof(double) * C.npairs * h->b * h->b, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaFree(tmp));
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)tmp), h->allocs.end());
  });
}

r3mg_status r3mg_get_prolongation(r3mg_hierarchy* h, int level, double* p_host) {
  if (!h || level < 0 || level + 1 >= h->L || !p_host) return R3MG_E_ARG;
  return guarded(h, [&] {
    const int b = h->b;
    if (level == 0) {
      std::vector<double> t(h->n * b);
      CK(cudaMemcpyAsync(t.data(), h->P64[0], sizeof(double) * t.size(), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int64_t k = 0; k < h->n; ++k) std::memcpy(p_host + h->part.perm[k] * b, t.data() + k * b, sizeof(double) * b);
    } else {
      CK(cudaMemcpyAsync(p_host, h->P64[level], sizeof(double) * h->lv[level].nbox * b * b, cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
  });
}

r3mg_status r3mg_profile_enable(r3mg_hierarchy* h, int on) {
  if (!h) return R3MG_E_ARG;
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    prof_harvest(h);
    h->prof_on = on ? 1 : 0;
    h->prof_ms.clear();
    h->prof_n.clear();
    h->launches = 0;
  });
}

r3mg_status r3mg_profile_read(r3mg_hierarchy* h, int kind, double* total_ms, int64_t* count, double* bytes_per_launch,
                              int64_t* kernel_launches) {
  if (!h || kind < 0 || kind > h->L) return R3MG_E_ARG;
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    prof_harvest(h);
    if (total_ms) *total_ms = kind < (int)h->prof_ms.size() ? h->prof_ms[kind] : 0.0;
    if (count) *count = kind < (int)h->prof_n.size() ? h->prof_n[kind] : 0;
    if (kernel_launches) *kernel_launches = h->launches;
    if (bytes_per_launch) {
      // algorithmic bytes: stored nonzeros (padding excluded) x (value + index bytes), one
      // 8-byte row pointer per row, and every vector read or written once
      const bool f32 = (h->prm.precision == 1);
      // (block solves: cols vectors of every kind; the matrix is read once for all of them)
      const double cols = (double)h->prof_cols;
      if (kind == 0) {
        const Level& F = h->lv[0];
        *bytes_per_launch = (double)F.nnz * (8 + 2) + 8.0 * (F.n + 1) + 2.0 * 8.0 * F.n * cols;
      } else {
        const Level& A = h->lv[kind - 1];
        const double es = f32 ? 4.0 : 8.0;
        const double ib = (A.b == 0) ? 2.0 : 0.0;
        if (f32 && cols == 1.0 && sym_form(A)) {
          // symmetric block form: the upper blocks once, the transposed-pair values and the row
          // sums written and read back, and the step's vectors
          *bytes_per_launch = (double)A.sym_nnz * es + 2.0 * es * (double)A.sym_tvals + 2.0 * es * A.n +
                              7.0 * es * A.n + 8.0 * (double)A.npairs;
        } else {
          *bytes_per_launch = (double)A.nnz * (es + ib) + 8.0 * (A.n + 1) + (6.0 * cols + 1.0) * es * A.n +
                              (A.b == 0 ? 0.0 : 8.0 * (double)A.npairs);
        }
      }
    }
  });
}

r3mg_status r3mg_sampled_outer(r3mg_hierarchy* h, const double* lam_dev, const double* u_dev, double alpha,
                               double* out_dev, void* stream) {
  if (!h || !lam_dev || !u_dev || !out_dev) return R3MG_E_ARG;
  if (!h->csr_rowptr) { h->err = "sampled_outer: not available on batched hierarchies"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    k_sampled_outer<<<grid_for(h->n * 32), 256, 0, h->stream>>>(h->csr_rowptr, h->csr_col, lam_dev, u_dev, alpha,
                                                                  out_dev, h->n);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_set_kernel_config(r3mg_hierarchy* h, int level, int fp32, int form, int lanes, int threads) {
  return r3mg_set_kernel_config2(h, level, fp32, form, lanes, threads, 0);
}

r3mg_status r3mg_set_kernel_config2(r3mg_hierarchy* h, int level, int fp32, int form, int lanes, int threads, int unroll) {
  if (unroll != 0 && !(unroll == 4 && !fp32)) {
    if (h) h->err = "set_kernel_config: unroll 4 is an FP64 option (0 = default)";
    return R3MG_E_ARG;
  }
  if (h && level >= 0 && level < h->L && form == 7) {   // staged symmetric form: lanes = CTAs per SM
    Level& A = h->lv[level];
    if (!fp32 || !A.sym_ok || lanes < 1 || lanes > 8 || threads != 128 || sym_stage_cap(A, lanes) == 0) {
      h->err = "set_kernel_config: the staged symmetric form is FP32 on a symmetric coarse level, lanes = 1..8 "
               "resident CTAs per SM (the stage sizing), 128 threads";
      return R3MG_E_ARG;
    }
    if (h->prm.precision != 1) { h->err = "set_kernel_config: the hierarchy has no FP32 V-cycle"; return R3MG_E_ARG; }
    return guarded(h, [&] {
      CK(cudaStreamSynchronize(h->stream));
      A.conf[1] = Level::KConf{form, lanes, threads, 0.f, 0};
      drop_graphs(h);
    });
  }
  const bool two = lanes == 2 && level == 0 && !fp32 && (form == 0 || form == 2 || form == 3 || form == 5 || form == 6);
  if (!h || level < 0 || level >= h->L || form < 0 || form > 6 || (lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32 && !two) ||
      (threads != 128 && threads != 256 && threads != 512 && threads != 1024 && !(threads == 96 && form == 4)) ||
      (form == 1 && threads == 128)) {
    if (h) h->err = "set_kernel_config: invalid level, form (0..7), lanes (4,8,16,32; 2 on the FP64 fine level's register forms; 1..8 for form 7) or threads (128 register forms only, 256, 512, 1024; 96 or 128 for form 4)";
    return R3MG_E_ARG;
  }
  Level& A = h->lv[level];
  const int pi = fp32 ? 1 : 0;
  if (fp32 && h->prm.precision != 1) { h->err = "set_kernel_config: the hierarchy has no FP32 V-cycle"; return R3MG_E_ARG; }
  if (form == 1 && A.tma[pi].nitems == 0) { h->err = "set_kernel_config: no TMA work items on this level"; return R3MG_E_ARG; }
  if (form == 4 && (!fp32 || !A.sym_ok)) { h->err = "set_kernel_config: no symmetric block form on this level"; return R3MG_E_ARG; }
  if (form == 2 && 2 * level_smem_bytes(view<double>(A)) > kMaxSmem) { h->err = "set_kernel_config: windows too large"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    A.conf[pi] = Level::KConf{form, lanes, threads, 0.f, unroll};
    drop_graphs(h);   // recaptured at the next V-cycle / solve
  });
}

r3mg_status r3mg_kernel_config(const r3mg_hierarchy* h, int level, int fp32, int* form, int* lanes, int* threads,
                               float* tuned_ms) {
  if (!h || level < 0 || level >= h->L) return R3MG_E_ARG;
  const Level::KConf& c = h->lv[level].conf[fp32 ? 1 : 0];
  const bool tma = c.form == 1 && h->lv[level].tma[fp32 ? 1 : 0].nitems > 0;
  if (form)
    *form = tma ? 1
                : (c.form == 2 || c.form == 3 || c.form == 5 || c.form == 6 ||
                           ((c.form == 4 || c.form == 7) && h->lv[level].sym_ok)
                       ? c.form
                       : 0);
  if (lanes) *lanes = c.G;
  if (threads) *threads = tma ? c.nt : (c.nt == 128 ? 128 : (c.nt == 96 && c.form == 4) ? 96 : 256);
  if (tuned_ms) *tuned_ms = c.ms;
  return R3MG_OK;
}

r3mg_status r3mg_kernel_unroll(const r3mg_hierarchy* h, int level, int fp32, int* unroll) {
  if (!h || level < 0 || level >= h->L || !unroll) return R3MG_E_ARG;
  *unroll = h->lv[level].conf[fp32 ? 1 : 0].u;
  return R3MG_OK;
}

const char* r3mg_last_error(const r3mg_hierarchy* h) { return h ? h->err.c_str() : g_last_error.c_str(); }

void r3mg_destroy(r3mg_hierarchy* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  if (h->lgraph) cudaGraphExecDestroy(h->lgraph);
  if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
  if (h->pgraph) cudaGraphExecDestroy(h->pgraph);
  if (h->mr_host) cudaFreeHost(h->mr_host);
  for (auto& sl : h->slots) { cudaEventDestroy(sl.e0); cudaEventDestroy(sl.e1); }
  if (h->cg_slot.e0) { cudaEventDestroy(h->cg_slot.e0); cudaEventDestroy(h->cg_slot.e1); }
  for (void* p : h->allocs) cudaFree(p);
  if (h->host_scal) cudaFreeHost(h->host_scal);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// ---------------------------------------------------------------- single steps, statistics, exports
r3mg_status r3mg_level_apply_prec(r3mg_hierarchy* h, int level, int fp32, const double* x_dev, double* y_dev,
                                  void* stream) {
  if (!h || level < 0 || level >= h->L || !x_dev || !y_dev || (fp32 != 0 && fp32 != 1)) return R3MG_E_ARG;
  if (!fp32) return r3mg_level_apply(h, level, x_dev, y_dev, stream);
  if (h->prm.precision != 1 || level == h->L - 1) {
    h->err = "level_apply_prec: FP32 values exist only on the smoothed levels of an FP32 V-cycle hierarchy";
    return R3MG_E_ARG;
  }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    Level& A = h->lv[level];
    float* xs = (float*)A.x;   // the level's V-cycle vectors serve as FP32 scratch
    float* ys = (float*)A.r;
    const int gv = grid_for(A.n);
    k_gather_perm<double, float><<<gv, 256, 0, h->stream>>>(x_dev, level == 0 ? h->perm : nullptr, xs, A.n);
    CK(cudaGetLastError());
    level_apply_dot<float>(h, A, xs, ys, nullptr, nullptr);
    k_scatter_perm<float, double><<<gv, 256, 0, h->stream>>>(ys, level == 0 ? h->perm : nullptr, y_dev, A.n);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_level_cheb_step(r3mg_hierarchy* h, int level, const double* x_dev, const double* r_dev,
                                 const double* d_dev, double a, double c, double* x_out, double* r_out,
                                 double* d_out, void* stream) {
  if (!h || level < 0 || level + 1 >= h->L || !x_dev || !r_dev || !d_dev || !x_out || !r_out || !d_out)
    return R3MG_E_ARG;
  if (!h->bl.empty()) { h->err = "level_cheb_step: batched hierarchy"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    Level& A = h->lv[level];
    const int64_t* perm = level == 0 ? h->perm : nullptr;
    const int gv = grid_for(A.n);
    auto run = [&](auto zero) {
      using T = decltype(zero);
      T *x = (T*)A.x, *r = (T*)A.r, *d = (T*)A.d[0], *dn = (T*)A.d[1];
      k_gather_perm<double, T><<<gv, 256, 0, h->stream>>>(x_dev, perm, x, A.n);
      k_gather_perm<double, T><<<gv, 256, 0, h->stream>>>(r_dev, perm, r, A.n);
      k_gather_perm<double, T><<<gv, 256, 0, h->stream>>>(d_dev, perm, d, A.n);
      CK(cudaGetLastError());
      level_cheb<T>(h, A, x, r, d, dn, Dinv<T>(A), (T)a, (T)c);
      k_scatter_perm<T, double><<<gv, 256, 0, h->stream>>>(x, perm, x_out, A.n);
      k_scatter_perm<T, double><<<gv, 256, 0, h->stream>>>(r, perm, r_out, A.n);
      k_scatter_perm<T, double><<<gv, 256, 0, h->stream>>>(dn, perm, d_out, A.n);
      CK(cudaGetLastError());
    };
    if (h->prm.precision == 1) run(0.0f); else run(0.0);
  });
}

r3mg_status r3mg_coarse_solve_prec(r3mg_hierarchy* h, int fp32, const double* r_dev, double* z_dev, void* stream) {
  if (!h || !r_dev || !z_dev || (fp32 != 0 && fp32 != 1)) return R3MG_E_ARG;
  if (!fp32) return r3mg_coarse_solve(h, r_dev, z_dev, stream);
  if (!h->bl.empty() || h->prm.precision != 1) {
    h->err = "coarse_solve_prec: the FP32 inverse exists only on single FP32 V-cycle hierarchies";
    return R3MG_E_ARG;
  }
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    Level& C = h->lv[h->L - 1];
    float* rs = (float*)C.r;
    float* zs = (float*)C.x;
    k_convert<double, float><<<grid_for(h->nc), 256, 0, h->stream>>>(r_dev, rs, h->nc);
    coarsest_apply<float>(h, rs, zs);
    k_convert<float, double><<<grid_for(h->nc), 256, 0, h->stream>>>(zs, z_dev, h->nc);
    CK(cudaGetLastError());
  });
}

r3mg_status r3mg_set_stop_rule(r3mg_hierarchy* h, double atol, double reduction) {
  if (!h) return R3MG_E_ARG;
  if (!(atol >= 0.0) || !(reduction >= 0.0) || !std::isfinite(atol) || !std::isfinite(reduction)) {
    h->err = "set_stop_rule: atol and reduction must be finite and >= 0";
    return R3MG_E_ARG;
  }
  h->stop_atol = atol;
  h->stop_red = reduction;
  return R3MG_OK;
}

r3mg_status r3mg_cond_estimate(r3mg_hierarchy* h, int column, double* cond_out, double* lmin_out, double* lmax_out,
                               int* steps_out) {
  if (!h) return R3MG_E_ARG;
  if (column >= 0 && (column >= h->mr_last_m || !h->mr_scal)) {
    h->err = "cond_estimate: no such column in the last block solve";
    return R3MG_E_ARG;
  }
  if (!h->bl.empty()) { h->err = "cond_estimate: not kept for batched solves"; return R3MG_E_ARG; }
  return guarded(h, [&] {
    double* hs = h->host_scal;   // pinned, 16 doubles
    const double* hist;
    double* cnt_a;
    double* cnt_b;
    if (column < 0) {
      cnt_a = h->scal + S_NA; cnt_b = h->scal + S_NB; hist = h->scal + S_COUNT;
    } else {
      const int M = h->mr_M;
      cnt_a = h->mr_scal + S_NA * M + column; cnt_b = h->mr_scal + S_NB * M + column;
      hist = h->mr_scal + S_COUNT * M + (int64_t)column * 2 * kHist;
    }
    CK(cudaMemcpyAsync(&hs[10], cnt_a, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&hs[11], cnt_b, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int na = std::min((int)hs[10], kHist), nb = std::min((int)hs[11], kHist);
    const int k = std::min(na, nb + 1);
    std::vector<double> al(kHist), be(kHist);
    if (k > 0) {
      CK(cudaMemcpy(al.data(), hist, sizeof(double) * k, cudaMemcpyDeviceToHost));
      if (k > 1) CK(cudaMemcpy(be.data(), hist + kHist, sizeof(double) * (k - 1), cudaMemcpyDeviceToHost));
    }
    // Lanczos tridiagonal of the CG iteration: T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    // T_{j,j+1} = sqrt(beta_j)/alpha_j; its extreme eigenvalues estimate those of M^{-1} A
    double lmin = 0.0, lmax = 0.0, cond = 1.0;
    if (k > 0) {
      std::vector<double> dg(k), off(k > 1 ? k - 1 : 0);
      for (int i = 0; i < k; ++i) {
        dg[i] = 1.0 / al[i] + (i > 0 ? be[i - 1] / al[i - 1] : 0.0);
        if (i + 1 < k) off[i] = std::sqrt(std::max(be[i], 0.0)) / al[i];
      }
      lmin = tridiag_kth_eig(dg, off, 0);
      lmax = tridiag_kth_eig(dg, off, k - 1);
      cond = lmax / lmin;
    }
    if (cond_out) *cond_out = cond;
    if (lmin_out) *lmin_out = lmin;
    if (lmax_out) *lmax_out = lmax;
    if (steps_out) *steps_out = k;
  });
}

r3mg_status r3mg_stats(r3mg_hierarchy* h, double* H_out, double* h_out, double* ratio_out, double* ritz_out) {
  if (!h) return R3MG_E_ARG;
  if (H_out) *H_out = h->H_coarse;
  if (h_out) *h_out = h->h_fine;
  if (ratio_out) *ratio_out = h->h_fine > 0.0 ? h->H_coarse / h->h_fine : 0.0;
  if (ritz_out) {
    for (int l = 0; l < h->L; ++l) {
      double v = 0.0;
      if (l + 1 < h->L) {
        if (h->bl.empty()) v = l < (int)h->ritz.size() ? h->ritz[l] : 0.0;
        else for (double lam : h->bl[l].lam) v = std::max(v, lam / h->prm.eig_safety);
      }
      ritz_out[l] = v;
    }
  }
  return R3MG_OK;
}

r3mg_status r3mg_get_transfer_pattern(r3mg_hierarchy* h, int level, int64_t* rowptr_host, int32_t* cols_host,
                                      double* vals_host) {
  if (!h || level < 0 || level + 1 >= h->L || !rowptr_host) return R3MG_E_ARG;
  return guarded(h, [&] {
    const int b = h->b;
    const int64_t nl = h->lv[level].n;
    for (int64_t i = 0; i <= nl; ++i) rowptr_host[i] = i * b;
    std::vector<int64_t> box;   // level 0: level-1 box of every tree position
    if (level == 0) {
      box.resize(h->n);
      const auto& off = h->part.box_off[1];
      for (int64_t B = 0; B + 1 < (int64_t)off.size(); ++B)
        for (int64_t k = off[B]; k < off[B + 1]; ++k) box[k] = B;
    }
    if (cols_host) {
      for (int64_t i = 0; i < nl; ++i) {
        const int64_t parent = (level == 0) ? box[h->part.iperm[i]] : (i / b) / h->fan;
        for (int q = 0; q < b; ++q) cols_host[i * b + q] = (int32_t)(parent * b + q);
      }
    }
    if (vals_host) {
      const int64_t cnt = nl * b;
      std::vector<double> t(cnt);
      CK(cudaMemcpyAsync(t.data(), h->P64[level], sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (level == 0) {
        for (int64_t k = 0; k < h->n; ++k) std::memcpy(vals_host + h->part.perm[k] * b, t.data() + k * b, sizeof(double) * b);
      } else {
        std::memcpy(vals_host, t.data(), sizeof(double) * cnt);   // rows (c, q') already in level order
      }
    }
  });
}

r3mg_status r3mg_get_level_matrix(r3mg_hierarchy* h, int level, int64_t* rowptr_host, int32_t* cols_host,
                                  double* vals_host) {
  if (!h || level < 1 || level >= h->L || !rowptr_host) return R3MG_E_ARG;
  return guarded(h, [&] {
    const int b = h->b;
    const Level& C = h->lv[level];
    const HostPattern& pt = C.pat;
    rowptr_host[0] = 0;
    for (int64_t B = 0; B < C.nbox; ++B) {
      const int64_t len = (pt.ptr[B + 1] - pt.ptr[B]) * b;
      for (int q = 0; q < b; ++q) rowptr_host[B * b + q + 1] = rowptr_host[B * b + q] + len;
    }
    if (cols_host) {
      for (int64_t B = 0; B < C.nbox; ++B)
        for (int q1 = 0; q1 < b; ++q1) {
          int64_t o = rowptr_host[B * b + q1];
          for (int64_t e = pt.ptr[B]; e < pt.ptr[B + 1]; ++e)
            for (int q = 0; q < b; ++q) cols_host[o++] = (int32_t)(pt.nbr[e] * b + q);
        }
    }
    if (vals_host) {
      std::vector<double> blk((size_t)C.npairs * b * b);
      CK(cudaStreamSynchronize(h->stream));
      r3mg_status st = r3mg_get_level_blocks(h, level, blk.data());
      if (st != R3MG_OK) throw Fail{st, h->err};
      for (int64_t B = 0; B < C.nbox; ++B)
        for (int q1 = 0; q1 < b; ++q1) {
          int64_t o = rowptr_host[B * b + q1];
          for (int64_t e = pt.ptr[B]; e < pt.ptr[B + 1]; ++e)
            for (int q = 0; q < b; ++q) vals_host[o++] = blk[(size_t)e * b * b + q1 * b + q];
        }
    }
  });
}

r3mg_status r3mg_device_status(r3mg_hierarchy* h, void* stream) {
  if (!h) return R3MG_E_ARG;
  return guarded(h, [&] {
    StreamJoin j(h, stream);
    int terr = 0;
    CK(cudaMemcpyAsync(&h->host_scal[15], h->tma_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(&terr, &h->host_scal[15], sizeof(int));
    if (terr) {
      CK(cudaMemsetAsync(h->tma_err, 0, sizeof(int), h->stream));
      CK(cudaStreamSynchronize(h->stream));
      throw Fail{R3MG_E_TIMEOUT, "a bounded wait of a copy-engine-streamed kernel expired since the last check"};
    }
  });
}

r3mg_status r3mg_set_coarse_mode(r3mg_hierarchy* h, int mode) {
  if (!h || (mode != 0 && mode != 1)) return R3MG_E_ARG;
  if (mode == 1 && (!h->bl.empty() || !h->L64)) {
    h->err = "set_coarse_mode: the substitution form needs a single (not batched) hierarchy";
    return R3MG_E_ARG;
  }
  const size_t sm = sizeof(double) * (size_t)h->nc;
  if (mode == 1 && sm + 16 * 1024 > kMaxSmem) {   // dynamic solution vector + the kernels' static arrays
    h->err = "set_coarse_mode: the coarsest level (" + std::to_string(h->nc) + " rows) does not fit one CTA's shared memory";
    return R3MG_E_LIMIT;
  }
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    if (mode == 1) {
      if (!h->ctmp) h->ctmp = dalloc<double>(h, h->nc);
      ensure_smem((const void*)k_trsv_lower<double>, sm);
      ensure_smem((const void*)k_trsv_lower_t<double>, sm);
      ensure_smem((const void*)k_trsv_lower<float>, sm / 2);
      ensure_smem((const void*)k_trsv_lower_t<float>, sm / 2);
    }
    h->coarse_mode = mode;
    drop_graphs(h);   // captured V-cycles hold the old form
  });
}

r3mg_status r3mg_get_batch_mode(const r3mg_hierarchy* h, int* mode, int* used, float* ms_graph, float* ms_persistent) {
  if (!h) return R3MG_E_ARG;
  if (mode) *mode = h->batch_mode;
  if (used) *used = h->batch_used;
  if (ms_graph) *ms_graph = h->batch_ms_it[0];
  if (ms_persistent) *ms_persistent = h->batch_ms_it[1];
  return R3MG_OK;
}

r3mg_status r3mg_set_batch_mode(r3mg_hierarchy* h, int mode) {
  if (!h || mode < 0 || mode > 2) return R3MG_E_ARG;
  if (h->bl.empty()) { h->err = "set_batch_mode: not a batched hierarchy"; return R3MG_E_ARG; }
  if (mode == 1 && h->L > kPMaxLevels) { h->err = "set_batch_mode: more than 8 levels"; return R3MG_E_LIMIT; }
  h->batch_mode = mode;
  if (mode == 2) h->batch_ms_it[0] = h->batch_ms_it[1] = -1.f;   // measure both forms again
  return R3MG_OK;
}

r3mg_status r3mg_set_wait_limit(r3mg_hierarchy* h, long long cycles, int withhold_first_copy) {
  if (!h || cycles < 0 || cycles > 4000000000LL || (withhold_first_copy != 0 && withhold_first_copy != 1)) return R3MG_E_ARG;
  return guarded(h, [&] {
    CK(cudaStreamSynchronize(h->stream));
    h->wait_cycles = cycles;
    h->withhold_first = withhold_first_copy;
    drop_graphs(h);   // captured graphs hold the old setting as launch arguments
  });
}

r3mg_status r3mg_setup_device(int64_t n, int dim, const double* coords_host, const int64_t* rowptr_dev,
                              const int32_t* colidx_dev, const double* vals_dev, const r3mg_params* params,
                              void* stream, r3mg_hierarchy** out) {
  if (!out) { g_last_error = "setup_device: null output"; return R3MG_E_ARG; }
  *out = nullptr;
  if (n < 1 || !rowptr_dev || !colidx_dev || !vals_dev) { g_last_error = "setup_device: null pointer or n < 1"; return R3MG_E_ARG; }
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
  cudaStream_t us = (cudaStream_t)stream;
  try {
    rp.resize(n + 1);
    if (cudaMemcpyAsync(rp.data(), rowptr_dev, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, us) != cudaSuccess ||
        cudaStreamSynchronize(us) != cudaSuccess) {
      g_last_error = "setup_device: reading the row pointers failed";
      return R3MG_E_CUDA;
    }
    const int64_t nnz = rp[n];
    if (nnz < 0 || rp[0] != 0) { g_last_error = "setup_device: malformed row pointers"; return R3MG_E_ARG; }
    ci.resize(nnz);
    va.resize(nnz);
    if (cudaMemcpyAsync(ci.data(), colidx_dev, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, us) != cudaSuccess ||
        cudaMemcpyAsync(va.data(), vals_dev, sizeof(double) * nnz, cudaMemcpyDeviceToHost, us) != cudaSuccess ||
        cudaStreamSynchronize(us) != cudaSuccess) {
      g_last_error = "setup_device: reading the CSR arrays failed";
      return R3MG_E_CUDA;
    }
  } catch (std::bad_alloc&) { g_last_error = "host allocation failed"; return R3MG_E_OOM; }
  return setup_common(n, dim, coords_host, rp.data(), ci.data(), va.data(), nullptr, params, stream, out);
}

// ---------------------------------------------------------------- allocation-free product
r3mg_status r3mg_level0_apply_noalloc(r3mg_hierarchy* h, const double* x_dev, double* y_dev, void* stream) {
  if (!h || !x_dev || !y_dev) return R3MG_E_ARG;
  if (h->n > kNoAllocMaxN) {
    h->err = "level0_apply_noalloc: n = " + std::to_string(h->n) + " exceeds the static scratch limit of " +
             std::to_string(kNoAllocMaxN) + " DoFs";
    return R3MG_E_LIMIT;
  }
  if (!h->noalloc_scratch) { h->err = "level0_apply_noalloc: no scratch address"; return R3MG_E_CUDA; }
  return guarded(h, [&] {
    // the device address of the static array was looked up by the setup call, on the
    // hierarchy's device (host code may not use the symbol itself as a device pointer)
    double* scratch = h->noalloc_scratch;
    double* xt = scratch;                  // x in tree order
    double* yt = scratch + kNoAllocMaxN;   // y in tree order
    StreamJoin j(h, stream);
    const int gv = grid_for(h->n);
    k_gather_perm<double, double><<<gv, 256, 0, h->stream>>>(x_dev, h->perm, xt, h->n);
    CK(cudaGetLastError());
    level_apply_dot<double>(h, h->lv[0], xt, yt, nullptr, nullptr);
    k_scatter_perm<double, double><<<gv, 256, 0, h->stream>>>(yt, h->perm, y_dev, h->n);
    CK(cudaGetLastError());
  });
}

}  // extern "C"
