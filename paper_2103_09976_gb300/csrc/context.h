// Library context: one CUDA device, one stream, the current two-site problem
// and its device-resident operators and work lists.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dmrg.h"
#include "kernels.h"
#include "model.h"

namespace dmrg {

#define DMRG_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::dmrg::Error(e_ == cudaErrorMemoryAllocation ? DMRG_ENOMEM : DMRG_ECUDA,      \
                          std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

// Stream that this thread's device allocations are ordered on: set by the
// library's entry points (the context's stream) and by serving workers.
// With a stream set, DevBuf uses the stream-ordered allocator
// (cudaMallocAsync / cudaFreeAsync on that stream), so allocating or freeing
// never synchronizes the device with work on other streams; without one it
// falls back to cudaMalloc / cudaFree.
extern thread_local cudaStream_t t_alloc_stream;
struct AllocStreamScope {
  cudaStream_t prev;
  explicit AllocStreamScope(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
  ~AllocStreamScope() { t_alloc_stream = prev; }
  AllocStreamScope(const AllocStreamScope&) = delete;
  AllocStreamScope& operator=(const AllocStreamScope&) = delete;
};

// Owning device allocation. A stream-ordered buffer is freed on the stream
// it was allocated on, which must outlive it (contexts free their buffers
// before destroying their stream).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  bool async = false;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) {
      if (async)
        cudaFreeAsync(p, st);
      else
        cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    async = false;
  }
  void alloc(size_t n) {
    if (n <= bytes && p) return;
    reset();
    if (n == 0) n = 16;
    if (t_alloc_stream) {
      DMRG_CUDA(cudaMallocAsync(&p, n, t_alloc_stream));
      st = t_alloc_stream;
      async = true;
    } else {
      DMRG_CUDA(cudaMalloc(&p, n));
    }
    bytes = n;
  }
  // Take over o's allocation (o becomes empty).
  void take(DevBuf& o) {
    reset();
    p = o.p;
    bytes = o.bytes;
    st = o.st;
    async = o.async;
    o.p = nullptr;
    o.bytes = 0;
    o.async = false;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
  template <class T, class A>
  void upload(const std::vector<T, A>& v, cudaStream_t s) {
    alloc(v.size() * sizeof(T));
    if (!v.empty())
      DMRG_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

// A two-site problem: left/right operator tables over one FP64 store
// (left ops first), the psi layout, NC terms and the sigma work list.
// Instantiated sigma graphs of a problem, keyed by (precision, psi, sigma).
struct GraphKey {
  int prec;
  const void* psi;
  const void* sigma;
  bool operator<(const GraphKey& o) const {
    if (prec != o.prec) return prec < o.prec;
    if (psi != o.psi) return psi < o.psi;
    return sigma < o.sigma;
  }
};
struct GraphCache {
  std::map<GraphKey, cudaGraphExec_t> m;
  unsigned warm = 0;  // bit p: precision p has run once directly
  GraphCache() = default;
  GraphCache(const GraphCache&) = delete;
  GraphCache& operator=(const GraphCache&) = delete;
  void clear() {
    for (auto& kv : m) cudaGraphExecDestroy(kv.second);
    m.clear();
  }
  ~GraphCache() { clear(); }
};

// A work list and its device copies (the full sigma, or one sub-Hamiltonian part).
struct DevWork {
  WorkList wl;
  DevBuf d_tasks, d_items, d_groups, d_sched, d_scratch, d_counter;
};

struct Problem {
  int nL = 0, n = 0;
  bool cn = false;           // terms of the CN partition (App. B, Eq. h-cn) instead of NC
  int part_rank = 0, part_n = 1;  // sub-Hamiltonian held (Sec. II.B); part_n = 1: the whole H
  QN Q;
  OpSet L, R;
  std::vector<PsiBlock> blocks;
  long long psi_size = 0;
  std::vector<Term> terms;
  WorkList wl;
  DevBuf store;              // FP64 operator store
  DevBuf d_tasks, d_items, d_groups, d_sched, d_blocks, d_scratch, d_counter;
  bool ready = false;
  // tensor-core path (built on first mixed-precision sigma): the plan, and
  // the split of the operators for the precision in use (bf16 for BF16X3 /
  // BF16X2, fp16 for FP16X2; one at a time)
  TcPlan tc;
  bool tc_plan_ready = false;
  long long tc_plan_gen = 0;       // plan builds so far
  bool bf16_split_ready = false;
  long long f16_gen = -1;          // plan build the FP16X2 records were made for; -1: no fp16 split
  // Davidson workspace (built on first use)
  bool dav_ready = false;
  int dav_space = 0;
  DevBuf dav_V, dav_AV, dav_diag, dav_x, dav_ax, dav_r, dav_t, dav_partial, dav_H, dav_w, dav_Y, dav_s;
  DevBuf d_dstart, d_dtask;
  DevBuf split, psi_split;         // slice-interleaved bf16 tiles of the operators / of psi
  DevBuf split16, psi_split16;     // FP16X2: slice-interleaved fp16 tiles of the scaled operators / psi
  DevBuf d_exps, d_psi_exp;        // FP16X2: block exponents (per split job), exponent of max |psi|
  DevBuf d_tc_recs16, d_tc_small16;  // FP16X2: records and small terms with coefficients for the scaled split
  DevBuf d_tc_recs, d_tc_items, d_tc_small, d_tc_small_sched, d_tc_groups, d_tc_sched, d_tc_pblk, d_tc_scratch, d_err;
  GraphCache graphs;
  // FP64 work-list tuning (dmrg_autotune): items per SM and per-task cost term
  int items_per_sm = 8;
  double per_task_cost = 16384.0;
  // tensor-core plan tuning (dmrg_autotune at a mixed precision): items per SM
  int tc_items_per_sm = 4;
  double tc_unit_cost = 128.0 * 128 * 64;  // fixed cost of a unit of stacked terms in the item split
  // producer warps of the tensor-core kernel per tile geometry (bf16, fp16):
  // the plan's default (tc_default_producers) or the autotuner's choice
  int tc_producers[2] = {1, 1};
  // sub-Hamiltonian parts: (n_ranks, rank) -> work list of that rank's terms
  std::map<std::pair<int, int>, std::unique_ptr<DevWork>> parts;
};

// CUDA-event timing of kernel launches (dmrg_profile).
struct Profiler {
  static constexpr int kKinds = 5;
  bool on = false;
  bool waits = false;   // also run the tensor-core kernel's wait accounting
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[kKinds];
  std::vector<cudaEvent_t> pool;
  double ms[kKinds] = {0, 0, 0, 0, 0};
  long long launches[kKinds] = {0, 0, 0, 0, 0};
  cudaEvent_t get();
  void begin(int kind, cudaStream_t st, cudaEvent_t* a);
  void end(int kind, cudaStream_t st, cudaEvent_t a);
  void collect();
  void clear();
  ~Profiler();
};

// RAII scope: records a start/stop event pair around the launches inside it.
struct ProfScope {
  Profiler& p;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(Profiler& p_, int k, cudaStream_t s) : p(p_), kind(k), st(s) {
    if (p.on) p.begin(kind, st, &a);
  }
  ~ProfScope() {
    if (p.on && a) p.end(kind, st, a);
  }
};

struct SweepState;

struct Context {
  dmrg_opts opts;
  int device = 0;
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::unique_ptr<Problem> prob;   // synthetic or current sweep step
  std::shared_ptr<SweepState> sweep;  // blocks of a problem built from integrals
  DevBuf d_psi, d_sigma;           // staging for host psi / sigma
  Profiler prof;
  DevBuf d_wait_prof;              // tensor-core kernel wait accounting (profiling only)
  // Pinned host scalars for the few device-to-host reads of the Davidson
  // loop (a pageable destination would stage every copy).
  struct PinnedScalars {
    double* p = nullptr;
    PinnedScalars() = default;
    PinnedScalars(const PinnedScalars&) = delete;
    PinnedScalars& operator=(const PinnedScalars&) = delete;
    double* get() {
      if (!p && cudaMallocHost(&p, 8 * sizeof(double)) != cudaSuccess) p = nullptr;
      return p;
    }
    ~PinnedScalars() {
      if (p) cudaFreeHost(p);
    }
  } h_scalars;
};

// Free every device buffer of the context (in stream order) and wait for the
// frees; the stream itself stays.
void release_context_buffers(Context& c);
void prepare_worklist(Context& c, Problem& p);
Basis parse_sectors(int n, const int* s);
// Synthetic middle-bond problem; with n_ranks > 1 only sub-Hamiltonian
// `rank` (its terms and the operators they use).
void load_synthetic(Context& c, int nL, int n, int N, int two_sz, const Basis& bL, const Basis& bR,
                    unsigned long long seed, int rank, int n_ranks);
// Device bytes a synthetic problem needs for one Davidson solve (an upper estimate).
long long synthetic_footprint(int nL, int n, int N, int two_sz, const Basis& bL, const Basis& bR, int prec,
                              int dav_space, int n_sm);
void prepare_tc(Context& c, Problem& p);
// The tensor-core plan and the split for precision `prec` are on the device.
bool tc_ready_for(const Problem& p, int prec);
void check_device_error(Context& c, Problem& p);
void sigma_noalloc(Context& c, Problem& p, const double* psi, double* sigma);
void sweep_problem(Context& c, int site);
// True when the context's resident problem is bond `site` of its sweep state.
bool sweep_problem_ready(const Context& c, int site);
// True for device or managed memory on device `dev`, false for host memory;
// throws DMRG_EINVAL for device memory of another GPU.
bool is_device_ptr(const void* p, int dev);
void sweep_build_blocks(Context& c, const double* t, const double* v, int K, int N, int two_sz, int M_init);
void sweep_run(Context& c, const int* Ms, int n_sweeps, double tol, double* energies, double* max_discard);
const std::vector<dmrg_step_log>& sweep_log(const Context& c);
void sweep_block_info(const Context& c, int side, int j, int* n_sectors, int* q, int* dims, int* n_ops);
void sweep_block_read(Context& c, int side, int j, int op, double* dense);
// Davidson on the device: x0 (device, may be null = seeded random) -> energy,
// eigenvector in x_out (device, may be null). Returns false if not converged.
void ensure_davidson_workspace(Context& c, Problem& p);
bool run_davidson(Context& c, Problem& p, const double* x0, double tol, double* energy, double* x_out,
                  int* iters, unsigned long long guess_counter_base);
void run_sigma(Context& c, Problem& p, const double* d_psi, double* d_sigma);      // context precision
void run_sigma_tc_direct(Context& c, Problem& p, const double* d_psi, double* d_sigma);  // mixed, no graph
void run_sigma_f64(Context& c, Problem& p, const double* d_psi, double* d_sigma);  // always FP64
// FP64 sigma of the terms that sub-Hamiltonian rank `rank` of n_ranks owns
void run_sigma_part(Context& c, Problem& p, int rank, int n_ranks, const double* d_psi, double* d_sigma);

}  // namespace dmrg

struct dmrg_ctx {
  dmrg::Context c;
};
