// Allocation-free FP64 sigma (dmrg_sigma_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// sigma: a serving process that reserved all of its HBM for operators up
// front, or a latency-critical loop that must not call cudaMalloc/cudaFree
// because those calls can block on, or synchronize with, other work on the
// device. For them this entry point runs the FP64 sigma kernel with its
// scratch (the per-item partial tiles and the work counter) in the
// fixed-size arrays below instead of buffers owned by the context. The
// operators, work lists, psi and sigma are still provided by the caller's
// context and arguments; nothing is allocated during the call.
//
// The arrays are file-scope __device__ variables: every GPU that loads this
// library holds them (32 MiB + 256 B) until the process exits, and every call
// on a device shares them. Calls whose partial tiles need more than
// kScratchDoubles doubles are rejected. Two calls that overlap on the GPU
// (different streams or contexts on the same device) race on the arrays.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "context.h"

namespace dmrg {

constexpr long long kScratchDoubles = 4ll << 20;  // 32 MiB of FP64 partial tiles

static __device__ __align__(256) double g_sigma_scratch[kScratchDoubles];
static __device__ __align__(256) unsigned int g_sigma_counter[64];

namespace {

struct SymbolAddrs {
  double* scratch = nullptr;
  unsigned int* counter = nullptr;
};

std::mutex g_mu;
SymbolAddrs g_addr[64];  // per device ordinal, filled on first use

// Host code cannot use g_sigma_scratch directly (in host code it names a
// host-side stand-in): look up its device address once per device, with
// that device current. The addresses stay valid for the life of the
// device's primary context; the library must not be used across a reset of
// that context (cudaDeviceReset) in the same process.
SymbolAddrs device_addrs(int dev) {
  if (dev < 0 || dev >= 64) throw Error(DMRG_EINVAL, "device ordinal out of range for dmrg_sigma_noalloc");
  std::lock_guard<std::mutex> lk(g_mu);
  SymbolAddrs& a = g_addr[dev];
  if (!a.scratch) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sigma_scratch);
    if (e != cudaSuccess)
      throw Error(DMRG_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&q, g_sigma_counter);
    if (e != cudaSuccess)
      throw Error(DMRG_ECUDA, std::string("cudaGetSymbolAddress(counter): ") + cudaGetErrorString(e));
    a.scratch = static_cast<double*>(p);
    a.counter = static_cast<unsigned int*>(q);
  }
  return a;
}

}  // namespace

void sigma_noalloc(Context& c, Problem& p, const double* psi, double* sigma) {
  DMRG_CUDA(cudaSetDevice(c.device));
  if (!psi || !sigma) throw Error(DMRG_EINVAL, "psi and sigma must not be NULL");
  if (!is_device_ptr(psi, c.device) || !is_device_ptr(sigma, c.device))
    throw Error(DMRG_EINVAL, "dmrg_sigma_noalloc needs device pointers for psi and sigma");
  const size_t bytes = (size_t)p.psi_size * sizeof(double);
  const char* a0 = (const char*)psi;
  const char* b0 = (const char*)sigma;
  if (a0 < b0 + bytes && b0 < a0 + bytes) throw Error(DMRG_EINVAL, "psi and sigma overlap");
  if (p.wl.scratch_elems > kScratchDoubles)
    throw Error(DMRG_EINVAL, "dmrg_sigma_noalloc: this problem needs " + std::to_string(p.wl.scratch_elems) +
                                 " doubles of scratch, the fixed maximum is " + std::to_string(kScratchDoubles) +
                                 " (32 MiB); use dmrg_sigma");
  const SymbolAddrs s = device_addrs(c.device);
  SigmaDev a;
  a.store = p.store.as<double>();
  a.psi = psi;
  a.sigma = sigma;
  a.tasks = p.d_tasks.as<Task>();
  a.items = p.d_items.as<Item>();
  a.schedule = p.d_sched.as<int>();
  a.n_items = (int)p.wl.items.size();
  a.groups = p.d_groups.as<Group>();
  a.n_groups = (int)p.wl.groups.size();
  a.blocks = p.d_blocks.as<PsiBlock>();
  a.scratch = s.scratch;
  a.counter = s.counter;
  // the work counter must start at zero; the partial tiles are fully written
  DMRG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(unsigned int), c.stream));
  launch_sigma_f64(a, c.n_sm, c.stream);
  DMRG_CUDA(cudaGetLastError());
  launch_reduce(a, c.stream);
  DMRG_CUDA(cudaGetLastError());
}

}  // namespace dmrg
