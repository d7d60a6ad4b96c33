// C ABI entry points (include/dmrg.h). Each call catches every exception and
// turns it into a status code plus a message on the context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include <cmath>

#include "context.h"

using namespace dmrg;

Basis dmrg::parse_sectors(int n, const int* s) {
  if (n <= 0 || !s) throw Error(DMRG_EINVAL, "empty sector list");
  Basis b;
  for (int i = 0; i < n; ++i) {
    b.q.push_back({s[3 * i], s[3 * i + 1]});
    b.dim.push_back(s[3 * i + 2]);
    if ((s[3 * i + 1] - s[3 * i]) % 2 != 0) throw Error(DMRG_EINVAL, "2Sz parity must match N");
  }
  b.finish();
  return b;
}


namespace {

thread_local std::string g_noctx_err = "no error";

template <class F>
dmrg_status guarded(dmrg_ctx* ctx, F&& f) {
  try {
    AllocStreamScope scope(ctx ? ctx->c.stream : nullptr);
    f();
    if (ctx) ctx->c.err.clear();
    return DMRG_OK;
  } catch (const Error& e) {
    if (ctx) ctx->c.err = e.what(); else g_noctx_err = e.what();
    return (dmrg_status)e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->c.err = "host allocation failed"; else g_noctx_err = "host allocation failed";
    return DMRG_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->c.err = e.what(); else g_noctx_err = e.what();
    return DMRG_EINVAL;
  }
}

}  // namespace

// True for device or managed memory, false for host memory (pageable or
// pinned). Device memory of another GPU is refused: the context's kernels
// run on its own device and would fault on, or silently read across, a peer
// GPU's memory.
bool dmrg::is_device_ptr(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) {
    if (at.device != dev)
      throw Error(DMRG_EINVAL, "buffer is device memory of GPU " + std::to_string(at.device) +
                                   " but the context runs on GPU " + std::to_string(dev));
    return true;
  }
  return at.type == cudaMemoryTypeManaged;
}

namespace {


Problem& need_problem(Context& c, int site) {
  if (c.sweep) {
    if (site < 0) throw Error(DMRG_EINVAL, "site must be a bond index (0 .. K-2) for a context built from integrals");
    sweep_problem(c, site);
    return *c.prob;
  }
  if (!c.prob) throw Error(DMRG_ESTATE, "no operators loaded (call dmrg_load_synthetic or dmrg_build_blocks)");
  if (site != -1) throw Error(DMRG_EINVAL, "site must be -1 for a synthetic context");
  return *c.prob;
}

}  // namespace

namespace dmrg {

// Items, groups and scratch of the FP64 work list for the problem's tuning.
static void prepare_items(Context& c, Problem& p) {
  TileShape ts{F64_TM, F64_TN, 2e6, p.per_task_cost};
  build_items(p.blocks, p.wl, ts, c.n_sm * p.items_per_sm);
  cudaStream_t st = c.stream;
  p.d_items.upload(p.wl.items, st);
  p.d_groups.upload(p.wl.groups, st);
  p.d_sched.upload(p.wl.schedule, st);
  p.d_scratch.alloc(std::max<long long>(1, p.wl.scratch_elems) * sizeof(double));
  DMRG_CUDA(cudaStreamSynchronize(st));
  p.graphs.clear();
}

void prepare_worklist(Context& c, Problem& p) {
  build_tasks(p.blocks, p.L, p.R, p.terms, p.wl);
  TileShape ts{F64_TM, F64_TN, 2e6, p.per_task_cost};
  build_items(p.blocks, p.wl, ts, c.n_sm * p.items_per_sm);
  cudaStream_t st = c.stream;
  p.d_tasks.upload(p.wl.tasks, st);
  p.d_items.upload(p.wl.items, st);
  p.d_groups.upload(p.wl.groups, st);
  p.d_sched.upload(p.wl.schedule, st);
  p.d_blocks.upload(p.blocks, st);
  p.d_scratch.alloc(std::max<long long>(1, p.wl.scratch_elems) * sizeof(double));
  p.d_counter.alloc(16);
  DMRG_CUDA(cudaStreamSynchronize(st));
  p.ready = true;
}

static_assert(sizeof(TcItem) == sizeof(Item), "reduction reads TcItem as Item");

// Work records of the tensor-core path for the problem's tuning (the split
// operator store is unchanged by it).
static void prepare_tc_plan(Context& c, Problem& p) {
  cudaStream_t st = c.stream;
  build_tc_plan(p.blocks, p.L, p.R, p.wl, p.tc, TcShape{c.n_sm * p.tc_items_per_sm, p.tc_unit_cost});
  p.tc_producers[0] = tc_default_producers(p.tc, false);
  p.tc_producers[1] = tc_default_producers(p.tc, true);
  p.d_tc_recs.upload(p.tc.recs, st);
  p.d_tc_items.upload(p.tc.items, st);
  p.d_tc_small.upload(p.tc.small, st);
  p.d_tc_small_sched.upload(p.tc.small_schedule, st);
  p.d_tc_groups.upload(p.tc.groups, st);
  p.d_tc_sched.upload(p.tc.schedule, st);
  p.d_tc_pblk.upload(p.tc.psi, st);
  p.d_tc_scratch.alloc(std::max<long long>(1, p.tc.scratch_elems) * sizeof(double));
  if (!p.d_err.p) {
    p.d_err.alloc(16);
    DMRG_CUDA(cudaMemsetAsync(p.d_err.p, 0, 16, st));
  }
  DMRG_CUDA(cudaStreamSynchronize(st));
  p.graphs.clear();
  p.tc_plan_ready = true;
  ++p.tc_plan_gen;
}

// Split jobs: every stored block in store order, then the identity blocks of
// the left and of the right sectors (the order of the plan's split-block
// indices).
static std::vector<SplitJob> split_jobs(const Problem& p) {
  std::vector<SplitJob> jobs;
  jobs.reserve(p.tc.opblocks.size() + p.tc.identL.size() + p.tc.identR.size());
  size_t k = 0;
  for (const OpSet* set : {&p.L, &p.R})
    for (const OpDesc& o : set->ops)
      for (const OpBlock& b : o.blocks) {
        const TcBlock& t = p.tc.opblocks[k++];
        jobs.push_back({b.off, b.rows, b.cols, t.tile, t.R8, t.C8});
      }
  for (int side = 0; side < 2; ++side) {
    const Basis& B = side == 0 ? p.L.basis : p.R.basis;
    const auto& id = side == 0 ? p.tc.identL : p.tc.identR;
    for (int i = 0; i < B.size(); ++i) jobs.push_back({-1, B.dim[i], B.dim[i], id[i].tile, id[i].R8, id[i].C8});
  }
  return jobs;
}

static void check_split_fits(Context& c, size_t bytes, const char* what) {
  // buffers freed on the stream (a split just dropped) stay in the device's
  // memory pool until trimmed; return them before asking what is free
  DMRG_CUDA(cudaStreamSynchronize(c.stream));
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess && pool) DMRG_CUDA(cudaMemPoolTrimTo(pool, 0));
  cudaGetLastError();
  size_t freeb = 0, totb = 0;
  DMRG_CUDA(cudaMemGetInfo(&freeb, &totb));
  if ((double)bytes > 0.92 * (double)freeb)
    throw Error(DMRG_ENOMEM, std::string(what) + " does not fit in free device memory");
}

// bf16 split of the operators (BF16X3 / BF16X2); drops an fp16 split.
static void ensure_split_bf16(Context& c, Problem& p) {
  if (p.bf16_split_ready) return;
  cudaStream_t st = c.stream;
  if (p.f16_gen >= 0) {
    p.graphs.clear();
    p.split16.reset();
    p.psi_split16.reset();
    p.d_tc_recs16.reset();
    p.d_tc_small16.reset();
    p.f16_gen = -1;
  }
  const size_t split_bytes = (size_t)p.tc.n_tiles * 384;
  check_split_fits(c, split_bytes, "bf16 split operator store");
  p.split.alloc(split_bytes);
  DMRG_CUDA(cudaMemsetAsync(p.split.p, 0, split_bytes, st));
  p.psi_split.alloc((size_t)p.tc.psi_tiles * 384);
  DMRG_CUDA(cudaMemsetAsync(p.psi_split.p, 0, (size_t)p.tc.psi_tiles * 384, st));
  const std::vector<SplitJob> jobs = split_jobs(p);
  DevBuf d_jobs;
  d_jobs.upload(jobs, st);
  launch_split_ops(p.store.as<double>(), d_jobs.as<SplitJob>(), (long long)jobs.size(), p.split.p, st);
  DMRG_CUDA(cudaGetLastError());
  DMRG_CUDA(cudaStreamSynchronize(st));
  p.bf16_split_ready = true;
}

// fp16 split of the scaled operators (FP16X2) and the records and small
// terms of the current plan with coefficients for it; drops a bf16 split.
static void ensure_split_f16(Context& c, Problem& p) {
  cudaStream_t st = c.stream;
  if (p.f16_gen < 0) {
    if (p.bf16_split_ready) {
      p.graphs.clear();
      p.split.reset();
      p.psi_split.reset();
      p.bf16_split_ready = false;
    }
    const size_t split_bytes = (size_t)p.tc.n_tiles * 256;
    check_split_fits(c, split_bytes, "fp16 split operator store");
    p.split16.alloc(split_bytes);
    DMRG_CUDA(cudaMemsetAsync(p.split16.p, 0, split_bytes, st));
    p.psi_split16.alloc((size_t)p.tc.psi_tiles * 256);
    DMRG_CUDA(cudaMemsetAsync(p.psi_split16.p, 0, (size_t)p.tc.psi_tiles * 256, st));
    const std::vector<SplitJob> jobs = split_jobs(p);
    DevBuf d_jobs;
    d_jobs.upload(jobs, st);
    p.d_exps.alloc(std::max<size_t>(1, jobs.size()) * sizeof(int));
    launch_block_exp(p.store.as<double>(), d_jobs.as<SplitJob>(), (long long)jobs.size(), p.d_exps.as<int>(), st);
    launch_split_ops16(p.store.as<double>(), d_jobs.as<SplitJob>(), (long long)jobs.size(), p.d_exps.as<int>(),
                       p.split16.p, st);
    DMRG_CUDA(cudaGetLastError());
    p.d_psi_exp.alloc(16);
    DMRG_CUDA(cudaStreamSynchronize(st));
    p.f16_gen = 0;
  }
  if (p.f16_gen != p.tc_plan_gen) {
    DevBuf d_tb, d_sb;
    d_tb.upload(p.tc.term_blk, st);
    d_sb.upload(p.tc.small_blk, st);
    p.d_tc_recs16.alloc(std::max<size_t>(1, p.tc.recs.size()) * sizeof(TcUnitRec));
    p.d_tc_small16.alloc(std::max<size_t>(1, p.tc.small.size()) * sizeof(SmallTerm));
    launch_fix_recs16(p.d_tc_recs.as<TcUnitRec>(), (long long)p.tc.recs.size(), d_tb.as<int>(), p.d_exps.as<int>(),
                      p.d_tc_recs16.as<TcUnitRec>(), st);
    launch_fix_small16(p.d_tc_small.as<SmallTerm>(), (long long)p.tc.small.size(), d_sb.as<int>(),
                       p.d_exps.as<int>(), p.d_tc_small16.as<SmallTerm>(), st);
    DMRG_CUDA(cudaGetLastError());
    DMRG_CUDA(cudaStreamSynchronize(st));
    p.graphs.clear();
    p.f16_gen = p.tc_plan_gen;
  }
}

bool tc_ready_for(const Problem& p, int prec) {
  if (!p.tc_plan_ready) return false;
  return prec == DMRG_FP16X2 ? p.f16_gen == p.tc_plan_gen : p.bf16_split_ready;
}

void prepare_tc(Context& c, Problem& p) {
  if (!p.tc_plan_ready) prepare_tc_plan(c, p);
  if (c.opts.sigma_prec == DMRG_FP16X2)
    ensure_split_f16(c, p);
  else
    ensure_split_bf16(c, p);
}

void check_device_error(Context& c, Problem& p) {
  DMRG_CUDA(cudaStreamSynchronize(c.stream));
  if (!p.tc_plan_ready) return;
  int e = 0;
  DMRG_CUDA(cudaMemcpy(&e, p.d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    DMRG_CUDA(cudaMemset(p.d_err.p, 0, sizeof(int)));
    throw Error(DMRG_ETIMEOUT, "tensor-core sigma: a bounded wait gave up (code " + std::to_string(e) +
                                   "); the last sigma result is invalid");
  }
}

static void run_sigma_tc(Context& c, Problem& p, const double* d_psi, double* d_sigma);
void run_sigma_tc_direct(Context& c, Problem& p, const double* d_psi, double* d_sigma) { run_sigma_tc(c, p, d_psi, d_sigma); }

static void run_sigma_tc(Context& c, Problem& p, const double* d_psi, double* d_sigma) {
  const int prec = c.opts.sigma_prec;
  if (!tc_ready_for(p, prec)) prepare_tc(c, p);
  const bool f16 = prec == DMRG_FP16X2;
  {
    ProfScope ps_(c.prof, 2, c.stream);
    if (f16)
      launch_split_psi16(d_psi, p.psi_size, p.d_blocks.as<PsiBlock>(), p.d_tc_pblk.as<TcPsiBlock>(),
                         (int)p.blocks.size(), p.d_psi_exp.as<int>(), p.psi_split16.p, c.stream);
    else
      launch_split_psi(d_psi, p.d_blocks.as<PsiBlock>(), p.d_tc_pblk.as<TcPsiBlock>(), (int)p.blocks.size(),
                       p.psi_split.p, c.stream);
  }
  DMRG_CUDA(cudaGetLastError());
  TcDev t;
  t.op = f16 ? p.split16.p : p.split.p;
  t.psi = f16 ? p.psi_split16.p : p.psi_split.p;
  t.psi_exp = p.d_psi_exp.as<int>();
  t.f16 = f16 ? 1 : 0;
  t.recs = f16 ? p.d_tc_recs16.as<TcUnitRec>() : p.d_tc_recs.as<TcUnitRec>();
  t.items = p.d_tc_items.as<TcItem>();
  t.schedule = p.d_tc_sched.as<int>();
  t.n_items = (int)p.tc.schedule.size();
  t.counter = p.d_counter.as<unsigned int>();
  t.scratch = p.d_tc_scratch.as<double>();
  t.err = p.d_err.as<int>();
  t.nprod = prec == DMRG_BF16X3 ? 6 : 3;
  // by default BF16X3 and FP16X2 bound each FP32 accumulation to 8 main MMA
  // steps (128 products along K); BF16X2, whose slices carry 16 bits,
  // flushes once per half of every unit
  const int chain = c.opts.tc_chain;
  t.max_chain = chain > 0 ? chain : (chain == 0 && prec != DMRG_BF16X2 ? 8 : 0);
  t.producers = c.opts.tc_producers > 0 ? c.opts.tc_producers : p.tc_producers[f16 ? 1 : 0];
  t.wait_prof = nullptr;
  if (c.prof.on && c.prof.waits) {
    if (!c.d_wait_prof.p) {
      c.d_wait_prof.alloc(32 * sizeof(unsigned long long));
      DMRG_CUDA(cudaMemsetAsync(c.d_wait_prof.p, 0, 32 * sizeof(unsigned long long), c.stream));
    }
    t.wait_prof = c.d_wait_prof.as<unsigned long long>();
  }
  DMRG_CUDA(cudaMemsetAsync(p.d_counter.p, 0, sizeof(unsigned int), c.stream));
  {
    ProfScope ps_(c.prof, 0, c.stream);
    SmallDev sd;
    sd.op = t.op;
    sd.psi = t.psi;
    sd.psi_exp = t.psi_exp;
    sd.f16 = t.f16;
    sd.pblk = p.d_tc_pblk.as<TcPsiBlock>();
    sd.terms = f16 ? p.d_tc_small16.as<SmallTerm>() : p.d_tc_small.as<SmallTerm>();
    sd.items = p.d_tc_items.as<TcItem>();
    sd.schedule = p.d_tc_small_sched.as<int>();
    sd.n_items = (int)p.tc.small_schedule.size();
    sd.n_mid = p.tc.n_small_mid;
    sd.scratch = p.d_tc_scratch.as<double>();
    {
      ProfScope ps4_(c.prof, 4, c.stream);  // the small classes alone (also inside kind 0)
      launch_sigma_small(sd, c.n_sm, c.stream);
    }
    launch_sigma_tc(t, c.n_sm, c.stream);
  }
  DMRG_CUDA(cudaGetLastError());
  SigmaDev r;
  r.sigma = d_sigma;
  r.items = reinterpret_cast<const Item*>(p.d_tc_items.p);
  r.groups = p.d_tc_groups.as<Group>();
  r.n_groups = (int)p.tc.groups.size();
  r.blocks = p.d_blocks.as<PsiBlock>();
  r.scratch = p.d_tc_scratch.as<double>();
  {
    ProfScope ps_(c.prof, 1, c.stream);
    launch_reduce(r, c.stream);
  }
  DMRG_CUDA(cudaGetLastError());
}

// One sigma at the context's precision. With graphs on, the launch sequence
// for a given (precision, psi, sigma) is captured once (on its second use;
// the first runs directly so that one-time setup such as kernel attributes
// happens outside a capture) and replayed as one graph launch afterwards.
void run_sigma(Context& c, Problem& p, const double* d_psi, double* d_sigma) {
  const int prec = c.opts.sigma_prec;
  auto direct = [&] {
    if (prec != DMRG_FP64)
      run_sigma_tc(c, p, d_psi, d_sigma);
    else
      run_sigma_f64(c, p, d_psi, d_sigma);
  };
  if (!c.opts.graphs || c.prof.on) {
    direct();
    return;
  }
  if (prec != DMRG_FP64 && !tc_ready_for(p, prec)) prepare_tc(c, p);  // allocations stay outside any capture
  const GraphKey key{prec, d_psi, d_sigma};
  auto it = p.graphs.m.find(key);
  if (it == p.graphs.m.end()) {
    if (!(p.graphs.warm & (1u << prec))) {
      direct();
      p.graphs.warm |= 1u << prec;
      return;
    }
    cudaGraph_t g = nullptr;
    DMRG_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
    try {
      direct();
    } catch (...) {
      cudaStreamEndCapture(c.stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    DMRG_CUDA(cudaStreamEndCapture(c.stream, &g));
    cudaGraphExec_t e = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&e, g, 0);
    cudaGraphDestroy(g);
    DMRG_CUDA(ie);
    it = p.graphs.m.emplace(key, e).first;
  }
  DMRG_CUDA(cudaGraphLaunch(it->second, c.stream));
}

void run_sigma_f64(Context& c, Problem& p, const double* d_psi, double* d_sigma) {
  SigmaDev a;
  a.store = p.store.as<double>();
  a.psi = d_psi;
  a.sigma = d_sigma;
  a.tasks = p.d_tasks.as<Task>();
  a.items = p.d_items.as<Item>();
  a.schedule = p.d_sched.as<int>();
  a.n_items = (int)p.wl.items.size();
  a.groups = p.d_groups.as<Group>();
  a.n_groups = (int)p.wl.groups.size();
  a.blocks = p.d_blocks.as<PsiBlock>();
  a.scratch = p.d_scratch.as<double>();
  a.counter = p.d_counter.as<unsigned int>();
  cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), c.stream);
  {
    ProfScope ps(c.prof, 0, c.stream);
    launch_sigma_f64(a, c.n_sm, c.stream);
  }
  DMRG_CUDA(cudaGetLastError());
  {
    ProfScope ps(c.prof, 1, c.stream);
    launch_reduce(a, c.stream);
  }
  DMRG_CUDA(cudaGetLastError());
}

void run_sigma_part(Context& c, Problem& p, int rank, int n_ranks, const double* d_psi, double* d_sigma) {
  auto& slot = p.parts[{n_ranks, rank}];
  cudaStream_t st = c.stream;
  if (!slot) {
    auto w = std::make_unique<DevWork>();
    const std::vector<int> ranks = p.cn ? cn_term_ranks(p.nL, p.n, n_ranks) : nc_term_ranks(p.nL, p.n, n_ranks);
    if (ranks.size() != p.terms.size()) throw Error(DMRG_EINVAL, "internal: term rank count");
    std::vector<Term> mine;
    for (size_t t = 0; t < p.terms.size(); ++t)
      if (ranks[t] == rank) mine.push_back(p.terms[t]);
    build_tasks(p.blocks, p.L, p.R, mine, w->wl);
    build_items(p.blocks, w->wl, TileShape{F64_TM, F64_TN, 2e6}, c.n_sm * 8);
    w->d_tasks.upload(w->wl.tasks, st);
    w->d_items.upload(w->wl.items, st);
    w->d_groups.upload(w->wl.groups, st);
    w->d_sched.upload(w->wl.schedule, st);
    w->d_scratch.alloc(std::max<long long>(1, w->wl.scratch_elems) * sizeof(double));
    w->d_counter.alloc(16);
    DMRG_CUDA(cudaStreamSynchronize(st));
    slot = std::move(w);
  }
  DevWork& w = *slot;
  SigmaDev a;
  a.store = p.store.as<double>();
  a.psi = d_psi;
  a.sigma = d_sigma;
  a.tasks = w.d_tasks.as<Task>();
  a.items = w.d_items.as<Item>();
  a.schedule = w.d_sched.as<int>();
  a.n_items = (int)w.wl.items.size();
  a.groups = w.d_groups.as<Group>();
  a.n_groups = (int)w.wl.groups.size();
  a.blocks = p.d_blocks.as<PsiBlock>();
  a.scratch = w.d_scratch.as<double>();
  a.counter = w.d_counter.as<unsigned int>();
  DMRG_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st));
  {
    ProfScope ps(c.prof, 0, st);
    launch_sigma_f64(a, c.n_sm, st);
  }
  DMRG_CUDA(cudaGetLastError());
  {
    ProfScope ps(c.prof, 1, st);
    launch_reduce(a, st);
  }
  DMRG_CUDA(cudaGetLastError());
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  DMRG_CUDA(cudaEventCreate(&e));
  return e;
}

void Profiler::begin(int kind, cudaStream_t st, cudaEvent_t* a) {
  *a = get();
  DMRG_CUDA(cudaEventRecord(*a, st));
}

void Profiler::end(int kind, cudaStream_t st, cudaEvent_t a) {
  cudaEvent_t b = get();
  cudaEventRecord(b, st);
  pending[kind].push_back({a, b});
}

void Profiler::collect() {
  for (int k = 0; k < kKinds; ++k) {
    for (auto& pr : pending[k]) {
      float t = 0;
      cudaEventSynchronize(pr.second);
      cudaEventElapsedTime(&t, pr.first, pr.second);
      ms[k] += t;
      launches[k] += 1;
      pool.push_back(pr.first);
      pool.push_back(pr.second);
    }
    pending[k].clear();
  }
}

void Profiler::clear() {
  collect();
  for (int k = 0; k < kKinds; ++k) {
    ms[k] = 0;
    launches[k] = 0;
  }
}

Profiler::~Profiler() {
  for (int k = 0; k < kKinds; ++k)
    for (auto& pr : pending[k]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace dmrg

namespace dmrg {
namespace {
// Host/device marshalling shared by the sigma entry points: stage host
// buffers through the context's device copies around `compute`.
template <class F>
void sigma_call(Context& c, Problem& p, const double* psi, double* sigma, F compute) {
  if (!psi || !sigma) throw Error(DMRG_EINVAL, "psi and sigma must not be NULL");
  const size_t bytes = (size_t)p.psi_size * sizeof(double);
  const char* a0 = (const char*)psi;
  const char* b0 = (const char*)sigma;
  if (a0 < b0 + bytes && b0 < a0 + bytes) throw Error(DMRG_EINVAL, "psi and sigma overlap");
  bool dpsi = is_device_ptr(psi, c.device), dsig = is_device_ptr(sigma, c.device);
  const double* xin = psi;
  double* yout = sigma;
  if (!dpsi) {
    c.d_psi.alloc(bytes);
    DMRG_CUDA(cudaMemcpyAsync(c.d_psi.p, psi, bytes, cudaMemcpyHostToDevice, c.stream));
    xin = c.d_psi.as<double>();
  }
  if (!dsig) {
    c.d_sigma.alloc(bytes);
    yout = c.d_sigma.as<double>();
  }
  compute(xin, yout);
  if (!dsig) {
    DMRG_CUDA(cudaMemcpyAsync(sigma, yout, bytes, cudaMemcpyDeviceToHost, c.stream));
    check_device_error(c, p);
  }
}
}  // namespace
}  // namespace dmrg

namespace dmrg {

// Middle-bond problem with synthetic operators: sector tables, NC operator
// tables and terms on the host, every stored block drawn on the device.
static void build_synthetic_tables(Problem& p, int nL, int n, int N, int two_sz, const Basis& bL,
                                   const Basis& bR) {
  if (nL <= 0 || n <= nL || nL % 2 || n % 2)
    throw Error(DMRG_EINVAL, "mode counts must be even with 0 < n_left_modes < n_modes");
  p.nL = nL;
  p.n = n;
  p.Q = {N, two_sz};
  build_nc_opset(p.L, bL, nL, n, true, 0);
  build_nc_opset(p.R, bR, nL, n, false, p.L.elements);
  p.terms = nc_terms(nL, n);
  p.blocks = psi_layout(bL, bR, p.Q, &p.psi_size);
  if (p.blocks.empty()) throw Error(DMRG_EINVAL, "no psi block: sectors cannot form the target");
  for (auto& b : p.blocks)
    if (b.mR > F64_TN * 64 || b.mL > (1 << 20)) throw Error(DMRG_EINVAL, "block too large");
}

void load_synthetic(Context& c, int nL, int n, int N, int two_sz, const Basis& bL, const Basis& bR,
                    unsigned long long seed, int rank, int n_ranks) {
  auto p = std::make_unique<Problem>();
  build_synthetic_tables(*p, nL, n, N, two_sz, bL, bR);
  // canonical store offset of every block: the generator's counter base
  std::vector<long long> canon;
  if (n_ranks > 1) {  // one sub-Hamiltonian: its terms and only the operators they use
    Partition part;
    partition_nc(p->L, p->R, nL, n, rank, n_ranks, part);
    p->terms = std::move(part.terms);
    canon = std::move(part.canon_off);
    p->part_rank = rank;
    p->part_n = n_ranks;
  }
  long long elems = p->L.elements + p->R.elements;
  size_t freeb = 0, totb = 0;
  DMRG_CUDA(cudaMemGetInfo(&freeb, &totb));
  if ((double)elems * 8.0 > 0.92 * (double)freeb)
    throw Error(DMRG_ENOMEM, "operator store (" + std::to_string(elems * 8.0 / 1e9) +
                                 " GB) does not fit in free device memory");
  c.prob.reset();
  c.sweep.reset();
  p->store.alloc((size_t)elems * sizeof(double));
  // generate every stored block on the device
  std::vector<GenBlock> gb;
  for (const OpSet* s : {&p->L, &p->R})
    for (const OpDesc& o : s->ops)
      for (const OpBlock& b : o.blocks) {
        const long long ctr = canon.empty() ? b.off : canon[gb.size()];
        gb.push_back({b.off, ctr, b.rows, b.cols, o.sym ? 1 : 0, 0});
      }
  DevBuf d_gb;
  d_gb.upload(gb, c.stream);
  launch_gen_blocks(p->store.as<double>(), d_gb.as<GenBlock>(), (long long)gb.size(), (uint64_t)seed, c.stream);
  DMRG_CUDA(cudaGetLastError());
  DMRG_CUDA(cudaStreamSynchronize(c.stream));
  prepare_worklist(c, *p);
  c.prob = std::move(p);
}

long long synthetic_footprint(int nL, int n, int N, int two_sz, const Basis& bL, const Basis& bR, int prec,
                              int dav_space, int n_sm) {
  Problem p;
  build_synthetic_tables(p, nL, n, N, two_sz, bL, bR);
  const double elems = (double)(p.L.elements + p.R.elements);
  const double psi = (double)p.psi_size;
  double bytes = 8.0 * elems;                                  // FP64 store
  bytes += 8.0 * (2.0 * psi + (double)F64_TM * F64_TN * n_sm * 8);  // partial-tile scratch (bound)
  bytes += 8.0 * psi * (2.0 * dav_space + 8.0);               // Davidson vectors and staging
  if (prec != DMRG_FP64) bytes += 6.0 * elems * 1.5 + 6.0 * psi * 2.0 + 8.0 * psi * 4.0;  // bf16 slices
  bytes += 64.0 * (1 << 20);                                   // tables, work lists, slack
  return (long long)bytes;
}

}  // namespace dmrg

namespace dmrg {
thread_local cudaStream_t t_alloc_stream = nullptr;

void release_context_buffers(Context& c) {
  if (c.stream) cudaStreamSynchronize(c.stream);
  c.prob.reset();
  c.sweep.reset();
  c.d_psi.reset();
  c.d_sigma.reset();
  c.d_wait_prof.reset();
  if (c.stream) cudaStreamSynchronize(c.stream);
}
}  // namespace dmrg

extern "C" {

void dmrg_default_opts(dmrg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->sigma_prec = DMRG_FP64;
  o->dav_max_space = 24;
  o->dav_max_iter = 200;
  o->keep_one_per_q = 0;
  o->noise = 0.0;
  o->seed = 0;
  o->device = 0;
  o->graphs = 1;
  o->mixed_cut = -1;
  o->tc_chain = 0;
  o->tc_producers = 0;
}

dmrg_status dmrg_create(dmrg_ctx** out, const dmrg_opts* opts) {
  if (!out) {
    g_noctx_err = "dmrg_create: out is NULL";
    return DMRG_EINVAL;
  }
  *out = nullptr;
  dmrg_ctx* ctx = nullptr;
  dmrg_status st = guarded(nullptr, [&] {
    dmrg_opts o;
    dmrg_default_opts(&o);
    if (opts) o = *opts;
    if (o.dav_max_space < 3) throw Error(DMRG_EINVAL, "dav_max_space must be >= 3");
    if (o.dav_max_iter < 1) throw Error(DMRG_EINVAL, "dav_max_iter must be >= 1");
    if (o.keep_one_per_q != 0 && o.keep_one_per_q != 1) throw Error(DMRG_EINVAL, "keep_one_per_q must be 0 or 1");
    if (!(o.noise >= 0.0) || !std::isfinite(o.noise)) throw Error(DMRG_EINVAL, "noise must be finite and >= 0");
    if (o.mixed_cut < -1) throw Error(DMRG_EINVAL, "mixed_cut must be -1 (NC everywhere) or >= 0");
    if (o.tc_chain < -1) throw Error(DMRG_EINVAL, "tc_chain must be -1 (unbounded), 0 (default) or >= 1");
    if (o.tc_producers != 0 && o.tc_producers != 1 && o.tc_producers != 3)
      throw Error(DMRG_EINVAL, "tc_producers must be 0 (by the plan or the autotuner), 1 or 3");
    if (o.sigma_prec < DMRG_FP64 || o.sigma_prec > DMRG_FP16X2)
      throw Error(DMRG_EINVAL, "unknown sigma precision");
    int ndev = 0;
    DMRG_CUDA(cudaGetDeviceCount(&ndev));
    if (o.device < 0 || o.device >= ndev) throw Error(DMRG_EINVAL, "device ordinal out of range");
    DMRG_CUDA(cudaSetDevice(o.device));
    ctx = new dmrg_ctx();
    ctx->c.opts = o;
    ctx->c.device = o.device;
    DMRG_CUDA(cudaDeviceGetAttribute(&ctx->c.n_sm, cudaDevAttrMultiProcessorCount, o.device));
    DMRG_CUDA(cudaStreamCreateWithFlags(&ctx->c.stream, cudaStreamNonBlocking));
  });
  if (st != DMRG_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return DMRG_OK;
}

void dmrg_destroy(dmrg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->c.device);
  release_context_buffers(ctx->c);
  if (ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
  ctx->c.stream = nullptr;
  delete ctx;
}

const char* dmrg_last_error(const dmrg_ctx* ctx) {
  if (!ctx) return g_noctx_err.c_str();
  return ctx->c.err.c_str();
}

void* dmrg_stream(dmrg_ctx* ctx) { return ctx ? (void*)ctx->c.stream : nullptr; }

dmrg_status dmrg_set_precision(dmrg_ctx* ctx, int prec) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (prec < DMRG_FP64 || prec > DMRG_FP16X2) throw Error(DMRG_EINVAL, "unknown sigma precision");
    ctx->c.opts.sigma_prec = prec;
  });
}

dmrg_status dmrg_load_synthetic(dmrg_ctx* ctx, int n_left_modes, int n_modes, int N, int two_sz,
                                int n_sec_left, const int* sec_left, int n_sec_right,
                                const int* sec_right, unsigned long long seed) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    DMRG_CUDA(cudaSetDevice(c.device));
    load_synthetic(c, n_left_modes, n_modes, N, two_sz, parse_sectors(n_sec_left, sec_left),
                   parse_sectors(n_sec_right, sec_right), seed, 0, 1);
  });
}

dmrg_status dmrg_load_synthetic_part(dmrg_ctx* ctx, int n_left_modes, int n_modes, int N, int two_sz,
                                     int n_sec_left, const int* sec_left, int n_sec_right,
                                     const int* sec_right, unsigned long long seed, int rank, int n_ranks) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (n_ranks < 1 || rank < 0 || rank >= n_ranks) throw Error(DMRG_EINVAL, "need 0 <= rank < n_ranks");
    Context& c = ctx->c;
    DMRG_CUDA(cudaSetDevice(c.device));
    load_synthetic(c, n_left_modes, n_modes, N, two_sz, parse_sectors(n_sec_left, sec_left),
                   parse_sectors(n_sec_right, sec_right), seed, rank, n_ranks);
  });
}

dmrg_status dmrg_partition_info(int n_left_modes, int n_modes, int N, int two_sz, int n_sec_left,
                                const int* sec_left, int n_sec_right, const int* sec_right, int rank,
                                int n_ranks, long long* n_terms, long long* op_elements, long long* total_elements,
                                int* term_ids, int max_ids) {
  return guarded(nullptr, [&] {
    if (n_ranks < 1 || rank < 0 || rank >= n_ranks) throw Error(DMRG_EINVAL, "need 0 <= rank < n_ranks");
    if (max_ids < 0 || (max_ids > 0 && !term_ids)) throw Error(DMRG_EINVAL, "term_ids must hold max_ids entries");
    Problem p;
    build_synthetic_tables(p, n_left_modes, n_modes, N, two_sz, parse_sectors(n_sec_left, sec_left),
                           parse_sectors(n_sec_right, sec_right));
    if (total_elements) *total_elements = p.L.elements + p.R.elements;
    Partition part;
    partition_nc(p.L, p.R, n_left_modes, n_modes, rank, n_ranks, part);
    if (n_terms) *n_terms = (long long)part.terms.size();
    if (op_elements) *op_elements = part.elements;
    for (int i = 0; i < max_ids && i < (int)part.term_ids.size(); ++i) term_ids[i] = part.term_ids[i];
  });
}

dmrg_status dmrg_psi_layout(dmrg_ctx* ctx, int site, int* n_blk, int* q_l, int* m_l, int* m_r,
                            long long* offset, long long* size) {
  if (!ctx || !n_blk) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Problem& p = need_problem(ctx->c, site);
    *n_blk = (int)p.blocks.size();
    if (size) *size = p.psi_size;
    for (size_t i = 0; i < p.blocks.size(); ++i) {
      const PsiBlock& b = p.blocks[i];
      if (q_l) {
        q_l[2 * i] = p.L.basis.q[b.qL].n;
        q_l[2 * i + 1] = p.L.basis.q[b.qL].s;
      }
      if (m_l) m_l[i] = b.mL;
      if (m_r) m_r[i] = b.mR;
      if (offset) offset[i] = b.off;
    }
  });
}

dmrg_status dmrg_get_sigma_info(dmrg_ctx* ctx, int site, dmrg_sigma_info* info) {
  if (!ctx || !info) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Problem& p = need_problem(ctx->c, site);
    info->n_terms = (long long)p.terms.size();
    info->n_products = (long long)p.wl.tasks.size();
    info->flops = p.wl.flops;
    info->op_elements = p.L.elements + p.R.elements;
    info->op_bytes_read = p.wl.bytes_ops;
    info->psi_size = p.psi_size;
    info->tc_items_per_sm = p.tc_items_per_sm;
    info->tc_producers = ctx->c.opts.tc_producers > 0 ? ctx->c.opts.tc_producers
                                                       : p.tc_producers[ctx->c.opts.sigma_prec == DMRG_FP16X2 ? 1 : 0];
    info->tc_unit_cost = p.tc_unit_cost;
  });
}


dmrg_status dmrg_sigma(dmrg_ctx* ctx, int site, const double* psi, double* sigma) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    DMRG_CUDA(cudaSetDevice(c.device));
    Problem& p = need_problem(c, site);
    sigma_call(c, p, psi, sigma, [&](const double* x, double* y) { run_sigma(c, p, x, y); });
  });
}

dmrg_status dmrg_autotune(dmrg_ctx* ctx, int site, int* items_per_sm, double* per_task_cost, double* best_ms) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    DMRG_CUDA(cudaSetDevice(c.device));
    Problem& p = need_problem(c, site);
    const size_t bytes = (size_t)p.psi_size * sizeof(double);
    c.d_psi.alloc(bytes);
    c.d_sigma.alloc(bytes);
    launch_gen_vector(c.d_psi.as<double>(), p.psi_size, 0x54554E45ull ^ c.opts.seed, 0ull, c.stream);
    DMRG_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    DMRG_CUDA(cudaEventCreate(&e0));
    DMRG_CUDA(cudaEventCreate(&e1));
    if (c.opts.sigma_prec != DMRG_FP64) {
      // tensor-core path: items per SM of the persistent kernel (the split
      // of each output tile's units into items, largest first)
      if (!tc_ready_for(p, c.opts.sigma_prec)) prepare_tc(c, p);
      // items per SM x fixed unit cost (in multiply-adds: 1 / 4 / 16 MMAs of
      // 128 x 128 x 64) of the item split
      const int cand[4] = {4, 8, 16, 32};
      const double ucand[3] = {128.0 * 128 * 64, 4 * 128.0 * 128 * 64, 16 * 128.0 * 128 * 64};
      const int g = c.opts.sigma_prec == DMRG_FP16X2 ? 1 : 0;
      double best = 1e300;
      int bi = p.tc_items_per_sm;
      double bu = p.tc_unit_cost;
      auto time_one = [&]() -> float {  // one warm-up, one timed sigma
        run_sigma_tc_direct(c, p, c.d_psi.as<double>(), c.d_sigma.as<double>());
        DMRG_CUDA(cudaEventRecord(e0, c.stream));
        run_sigma_tc_direct(c, p, c.d_psi.as<double>(), c.d_sigma.as<double>());
        DMRG_CUDA(cudaEventRecord(e1, c.stream));
        DMRG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        DMRG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
      };
      try {
        for (double uc : ucand)
          for (int wi : cand) {
            p.tc_items_per_sm = wi;
            p.tc_unit_cost = uc;
            prepare_tc_plan(c, p);
            prepare_tc(c, p);  // FP16X2: records of the new plan
            const float ms = time_one();
            if (ms < best) {
              best = ms;
              bi = wi;
              bu = uc;
            }
          }
        p.tc_items_per_sm = bi;
        p.tc_unit_cost = bu;
        prepare_tc_plan(c, p);
        prepare_tc(c, p);
        // then the other producer setting on the chosen plan (unless fixed by
        // the options)
        if (c.opts.tc_producers == 0) {
          const int d = p.tc_producers[g];
          p.tc_producers[g] = d == 1 ? 3 : 1;
          const float ms = time_one();
          if (ms < best)
            best = ms;
          else
            p.tc_producers[g] = d;
        }
      } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      check_device_error(c, p);
      if (items_per_sm) *items_per_sm = bi;
      if (per_task_cost) *per_task_cost = bu;
      if (best_ms) *best_ms = best;
      return;
    }
    const int cand_items[3] = {8, 16, 32};
    const double cand_cost[3] = {4096.0, 16384.0, 65536.0};
    double best = 1e300;
    int bi = p.items_per_sm;
    double bc = p.per_task_cost;
    try {
      for (int wi : cand_items)
        for (double cc : cand_cost) {
          p.items_per_sm = wi;
          p.per_task_cost = cc;
          prepare_items(c, p);
          run_sigma_f64(c, p, c.d_psi.as<double>(), c.d_sigma.as<double>());  // warm-up
          DMRG_CUDA(cudaEventRecord(e0, c.stream));
          run_sigma_f64(c, p, c.d_psi.as<double>(), c.d_sigma.as<double>());
          DMRG_CUDA(cudaEventRecord(e1, c.stream));
          DMRG_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          DMRG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            bi = wi;
            bc = cc;
          }
        }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p.items_per_sm = bi;
    p.per_task_cost = bc;
    prepare_items(c, p);
    if (items_per_sm) *items_per_sm = bi;
    if (per_task_cost) *per_task_cost = bc;
    if (best_ms) *best_ms = best;
  });
}

dmrg_status dmrg_sigma_part(dmrg_ctx* ctx, int site, int rank, int n_ranks, const double* psi, double* sigma) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    if (n_ranks < 1 || rank < 0 || rank >= n_ranks) throw Error(DMRG_EINVAL, "need 0 <= rank < n_ranks");
    DMRG_CUDA(cudaSetDevice(c.device));
    Problem& p = need_problem(c, site);
    if (p.part_n > 1)
      throw Error(DMRG_EINVAL, "the context already holds one sub-Hamiltonian (dmrg_load_synthetic_part); "
                               "use dmrg_sigma");
    sigma_call(c, p, psi, sigma, [&](const double* x, double* y) { run_sigma_part(c, p, rank, n_ranks, x, y); });
  });
}

dmrg_status dmrg_sigma_noalloc(dmrg_ctx* ctx, int site, const double* psi, double* sigma) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    // a context built from integrals keeps one bond's operators resident;
    // building another bond's would allocate, so it is refused here
    if (c.sweep && !sweep_problem_ready(c, site))
      throw Error(DMRG_ESTATE, "dmrg_sigma_noalloc: the operators of bond " + std::to_string(site) +
                                   " are not resident (call dmrg_sigma or dmrg_davidson at this bond first)");
    sigma_noalloc(c, need_problem(c, site), psi, sigma);
  });
}

dmrg_status dmrg_davidson(dmrg_ctx* ctx, int site, const double* psi0, double tol, double* energy,
                          double* psi_out, int* iters) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    Context& c = ctx->c;
    DMRG_CUDA(cudaSetDevice(c.device));
    Problem& p = need_problem(c, site);
    if (!energy || !iters) throw Error(DMRG_EINVAL, "energy and iters must not be NULL");
    if (!(tol > 0.0)) throw Error(DMRG_EINVAL, "tol must be positive");
    if (c.opts.dav_max_space > 32) throw Error(DMRG_EINVAL, "dav_max_space must be <= 32");
    const size_t bytes = (size_t)p.psi_size * sizeof(double);
    const double* x0 = psi0;
    if (psi0 && !is_device_ptr(psi0, c.device)) {
      c.d_psi.alloc(bytes);
      DMRG_CUDA(cudaMemcpyAsync(c.d_psi.p, psi0, bytes, cudaMemcpyHostToDevice, c.stream));
      x0 = c.d_psi.as<double>();
    }
    double* xo = psi_out;
    const bool host_out = psi_out && !is_device_ptr(psi_out, c.device);
    if (host_out) {
      c.d_sigma.alloc(bytes);
      xo = c.d_sigma.as<double>();
    }
    const bool conv = run_davidson(c, p, x0, tol, energy, xo, iters, 0ull);
    if (host_out) {
      DMRG_CUDA(cudaMemcpyAsync(psi_out, xo, bytes, cudaMemcpyDeviceToHost, c.stream));
      DMRG_CUDA(cudaStreamSynchronize(c.stream));
    }
    if (!conv) throw Error(DMRG_ENOCONV, "Davidson reached dav_max_iter before the residual tolerance");
  });
}

dmrg_status dmrg_build_blocks(dmrg_ctx* ctx, const double* t, const double* v, int K, int N,
                              int two_sz, int M_init) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (!t || !v) throw Error(DMRG_EINVAL, "t and v must not be NULL");
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    ctx->c.prob.reset();
    ctx->c.sweep.reset();
    sweep_build_blocks(ctx->c, t, v, K, N, two_sz, M_init);
  });
}

dmrg_status dmrg_sweep(dmrg_ctx* ctx, const int* M_schedule, int n_sweeps, double tol,
                       double* energies, double* max_discard) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (!M_schedule || n_sweeps < 1) throw Error(DMRG_EINVAL, "empty M schedule");
    if (!(tol > 0.0)) throw Error(DMRG_EINVAL, "tol must be positive");
    if (ctx->c.opts.dav_max_space > 32) throw Error(DMRG_EINVAL, "dav_max_space must be <= 32");
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    sweep_run(ctx->c, M_schedule, n_sweeps, tol, energies, max_discard);
  });
}

dmrg_status dmrg_block_info(dmrg_ctx* ctx, int side, int j, int* n_sectors, int* q, int* dims, int* n_ops) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (!n_sectors) throw Error(DMRG_EINVAL, "n_sectors must not be NULL");
    sweep_block_info(ctx->c, side, j, n_sectors, q, dims, n_ops);
  });
}

dmrg_status dmrg_block_read(dmrg_ctx* ctx, int side, int j, int op, double* dense) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (!dense) throw Error(DMRG_EINVAL, "dense must not be NULL");
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    sweep_block_read(ctx->c, side, j, op, dense);
  });
}

dmrg_status dmrg_sweep_log(dmrg_ctx* ctx, dmrg_step_log* out, int max_steps, int* n_steps) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (!n_steps) throw Error(DMRG_EINVAL, "n_steps must not be NULL");
    if (max_steps < 0 || (max_steps > 0 && !out)) throw Error(DMRG_EINVAL, "out must hold max_steps records");
    const std::vector<dmrg_step_log>& log = sweep_log(ctx->c);
    const int n = (int)log.size();
    for (int k = 0; k < n && k < max_steps; ++k) out[k] = log[k];
    *n_steps = n;
  });
}

dmrg_status dmrg_sync(dmrg_ctx* ctx) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    DMRG_CUDA(cudaStreamSynchronize(ctx->c.stream));
    if (ctx->c.prob) check_device_error(ctx->c, *ctx->c.prob);
  });
}

dmrg_status dmrg_profile_waits(dmrg_ctx* ctx, double* cycles, int n) {
  if (!ctx || !cycles || n <= 0) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    DMRG_CUDA(cudaStreamSynchronize(ctx->c.stream));
    unsigned long long h[32] = {0};
    if (ctx->c.d_wait_prof.p)
      DMRG_CUDA(cudaMemcpy(h, ctx->c.d_wait_prof.p, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n && i < 32; ++i) cycles[i] = (double)h[i];
  });
}

dmrg_status dmrg_profile(dmrg_ctx* ctx, int enable) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    if (enable && ctx->c.d_wait_prof.p)
      DMRG_CUDA(cudaMemsetAsync(ctx->c.d_wait_prof.p, 0, 32 * sizeof(unsigned long long), ctx->c.stream));
    if (enable < 0 || enable > 2) throw Error(DMRG_EINVAL, "enable must be 0, 1 or 2");
    if (enable) ctx->c.prof.clear();
    ctx->c.prof.on = enable != 0;
    ctx->c.prof.waits = enable == 2;
  });
}

dmrg_status dmrg_profile_read(dmrg_ctx* ctx, int kernel, double* total_ms, long long* launches) {
  if (!ctx) return DMRG_EINVAL;
  return guarded(ctx, [&] {
    if (kernel < 0 || kernel >= Profiler::kKinds) throw Error(DMRG_EINVAL, "unknown kernel id");
    DMRG_CUDA(cudaSetDevice(ctx->c.device));
    ctx->c.prof.collect();
    if (total_ms) *total_ms = ctx->c.prof.ms[kernel];
    if (launches) *launches = ctx->c.prof.launches[kernel];
  });
}

}  // extern "C"
