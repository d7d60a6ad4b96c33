// Serving loop: continuous batching of Davidson solves on one GPU.
//
// Requests (a middle-bond problem given by its sector tables, a seed, a
// precision and a tolerance) enter a queue. n_slots worker threads each own
// a context (own CUDA stream); a free worker admits the oldest queued
// request whose device footprint fits in what the budget has left, builds
// its operators on the device, keeps them there for the whole solve, runs
// the device Davidson and frees them. Solves of different sizes therefore
// run side by side on separate streams, and a request that arrives while
// others run is admitted as soon as a slot and memory are free. A request
// passed over four times blocks later ones until it fits, so a large
// request is not starved by a stream of small ones. All kernels reduce in a
// fixed order, so a result does not depend on what else was running.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>

#include "context.h"

using namespace dmrg;

namespace {

struct Job {
  dmrg_request r;
  std::vector<int> left, right;
  long long bytes = 0;
  double t_submit = 0.0;
  int passed_over = 0;
};

}  // namespace

struct dmrg_server {
  int device = 0;
  int n_sm = 0;
  long long budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::deque<dmrg_result> done;
  long long in_use = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  std::string err = "no error";

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // Index of the job to admit, or -1. Caller holds mu.
  int pick() {
    const long long free_bytes = budget - in_use;
    for (size_t i = 0; i < queue.size(); ++i) {
      if (queue[i].bytes <= free_bytes) {
        for (size_t k = 0; k < i; ++k) queue[k].passed_over++;
        return (int)i;
      }
      if (queue[i].passed_over >= 4) return -1;  // reserve memory for a starved request
    }
    return -1;
  }

  void worker(int slot) {
    cudaSetDevice(device);
    Context c;
    dmrg_default_opts(&c.opts);
    c.device = device;
    c.n_sm = n_sm;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) return;
    AllocStreamScope scope(c.stream);
    for (;;) {
      Job job;
      {
        std::unique_lock<std::mutex> lk(mu);
        int idx = -1;
        cv_work.wait(lk, [&] { return stop || (idx = pick()) >= 0; });
        if (stop) break;
        job = std::move(queue[idx]);
        queue.erase(queue.begin() + idx);
        in_use += job.bytes;
        ++running;
      }
      dmrg_result res{};
      res.id = job.r.id;
      res.slot = slot;
      res.bytes = job.bytes;
      res.t_submit = job.t_submit;
      res.t_admit = now();
      res.energy = 0.0;
      try {
        c.opts.sigma_prec = job.r.sigma_prec;
        c.opts.dav_max_iter = job.r.max_iter;
        c.opts.seed = job.r.seed;
        load_synthetic(c, job.r.n_left_modes, job.r.n_modes, job.r.N, job.r.two_sz,
                       parse_sectors((int)job.left.size() / 3, job.left.data()),
                       parse_sectors((int)job.right.size() / 3, job.right.data()), job.r.seed, 0, 1);
        res.t_loaded = now();
        double e = 0.0;
        int it = 0;
        const bool conv = run_davidson(c, *c.prob, nullptr, job.r.tol, &e, nullptr, &it, 0ull);
        res.energy = e;
        res.iters = it;
        res.converged = conv ? 1 : 0;
        res.status = DMRG_OK;
      } catch (const Error& ex) {
        res.status = ex.code;
        std::lock_guard<std::mutex> lk(mu);
        err = ex.what();
      } catch (const std::exception& ex) {
        res.status = DMRG_ECUDA;
        std::lock_guard<std::mutex> lk(mu);
        err = ex.what();
      }
      c.prob.reset();
      cudaStreamSynchronize(c.stream);
      res.t_done = now();
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= job.bytes;
        --running;
        done.push_back(res);
      }
      cv_work.notify_all();
      cv_done.notify_all();
    }
    release_context_buffers(c);
    cudaStreamDestroy(c.stream);
    c.stream = nullptr;
  }
};

extern "C" {

dmrg_status dmrg_server_create(dmrg_server** out, int device, int n_slots, long long budget_bytes) {
  if (!out || n_slots < 1 || n_slots > 64 || budget_bytes <= 0) return DMRG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return DMRG_ECUDA;
  auto* s = new dmrg_server();
  s->device = device;
  s->budget = budget_bytes;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete s;
    return DMRG_ECUDA;
  }
  for (int k = 0; k < n_slots; ++k) s->workers.emplace_back([s, k] { s->worker(k); });
  *out = s;
  return DMRG_OK;
}

dmrg_status dmrg_server_submit(dmrg_server* s, const dmrg_request* r) {
  if (!s || !r) return DMRG_EINVAL;
  Job job;
  job.r = *r;
  try {
    if (r->n_sec_left <= 0 || r->n_sec_right <= 0 || !r->sec_left || !r->sec_right)
      throw Error(DMRG_EINVAL, "empty sector list");
    if (!(r->tol > 0.0) || r->max_iter < 1) throw Error(DMRG_EINVAL, "tol must be positive, max_iter >= 1");
    if (r->sigma_prec < DMRG_FP64 || r->sigma_prec > DMRG_FP16X2) throw Error(DMRG_EINVAL, "unknown precision");
    job.left.assign(r->sec_left, r->sec_left + 3 * r->n_sec_left);
    job.right.assign(r->sec_right, r->sec_right + 3 * r->n_sec_right);
    job.r.sec_left = nullptr;
    job.r.sec_right = nullptr;
    dmrg_opts o;
    dmrg_default_opts(&o);
    job.bytes = synthetic_footprint(r->n_left_modes, r->n_modes, r->N, r->two_sz,
                                    parse_sectors(r->n_sec_left, job.left.data()),
                                    parse_sectors(r->n_sec_right, job.right.data()), r->sigma_prec,
                                    o.dav_max_space, s->n_sm);
    if (job.bytes > s->budget) throw Error(DMRG_ENOMEM, "request footprint exceeds the server's memory budget");
  } catch (const Error& ex) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = ex.what();
    return (dmrg_status)ex.code;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    job.t_submit = s->now();
    s->queue.push_back(std::move(job));
  }
  s->cv_work.notify_all();
  return DMRG_OK;
}

int dmrg_server_poll(dmrg_server* s, dmrg_result* out, int max_results, int wait_ms) {
  if (!s || !out || max_results <= 0) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < max_results && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

dmrg_status dmrg_server_pending(dmrg_server* s, int* queued, int* running, long long* bytes_in_use) {
  if (!s) return DMRG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->queue.size();
  if (running) *running = s->running;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  return DMRG_OK;
}

const char* dmrg_server_last_error(dmrg_server* s) {
  if (!s) return "server is NULL";
  std::lock_guard<std::mutex> lk(s->mu);
  thread_local std::string copy;
  copy = s->err;
  return copy.c_str();
}

void dmrg_server_destroy(dmrg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
