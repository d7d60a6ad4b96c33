// Host control of the device Davidson solver (FP64 vectors on the device).
//
// Appendix A names the Davidson method for the solving step (Eq. eff-eigsh);
// the steps follow E. R. Davidson (J. Comput. Phys. 17, 87 (1975)) with the
// choices stated in include/dmrg.h: diagonal preconditioner clamped at 1e-8,
// classical Gram-Schmidt applied twice, thick restart from the two lowest
// Ritz vectors, convergence when the squared residual norm is below tol.
#include <cmath>
#include <cstring>

#include "context.h"

namespace dmrg {

namespace {

constexpr uint64_t KEY_GUESS = 0x4755455353505349ull;  // "GUESSPSI" stream of the seed
constexpr int LDH = 32;                                // leading dimension of the projected matrix

}  // namespace

// Davidson buffers of a problem and the diagonal of H_eff (built once).
void ensure_davidson_workspace(Context& c, Problem& p) {
  const int S = c.opts.dav_max_space;
  if (p.dav_ready && p.dav_space == S) return;
  const long long n = p.psi_size;
  cudaStream_t st = c.stream;
  p.dav_V.alloc((size_t)S * n * sizeof(double));
  p.dav_AV.alloc((size_t)S * n * sizeof(double));
  p.dav_diag.alloc(n * sizeof(double));
  p.dav_x.alloc(n * sizeof(double));
  p.dav_ax.alloc(n * sizeof(double));
  p.dav_r.alloc(n * sizeof(double));
  p.dav_t.alloc(n * sizeof(double));
  p.dav_partial.alloc((size_t)(S + 2) * 256 * sizeof(double));
  p.dav_H.alloc(LDH * LDH * sizeof(double));
  p.dav_w.alloc(LDH * sizeof(double));
  p.dav_Y.alloc(LDH * LDH * sizeof(double));
  p.dav_s.alloc(64 * sizeof(double));
  // diagonal of H_eff: the tasks whose output block is their input block
  std::vector<int> dstart(p.blocks.size() + 1, 0), dtask;
  for (size_t b = 0; b < p.blocks.size(); ++b) {
    for (int t = p.wl.out_start[b]; t < p.wl.out_start[b + 1]; ++t)
      if (p.wl.tasks[t].in_blk == (int)b) dtask.push_back(t);
    dstart[b + 1] = (int)dtask.size();
  }
  if (dtask.empty()) dtask.push_back(0);
  p.d_dstart.upload(dstart, st);
  p.d_dtask.upload(dtask, st);
  {
    ProfScope ps(c.prof, 2, st);
    launch_heff_diag(p.store.as<double>(), p.d_tasks.as<Task>(), p.d_dstart.as<int>(), p.d_dtask.as<int>(),
                     p.d_blocks.as<PsiBlock>(), (int)p.blocks.size(), p.dav_diag.as<double>(), st);
  }
  DMRG_CUDA(cudaGetLastError());
  DMRG_CUDA(cudaStreamSynchronize(st));
  p.dav_space = S;
  p.dav_ready = true;
}

namespace {

}  // namespace

bool run_davidson(Context& c, Problem& p, const double* x0, double tol, double* energy, double* x_out,
                  int* iters, unsigned long long guess_counter_base) {
  ensure_davidson_workspace(c, p);
  const long long n = p.psi_size;
  const int S = c.opts.dav_max_space;
  const int max_iter = c.opts.dav_max_iter;
  cudaStream_t st = c.stream;
  double* V = p.dav_V.as<double>();
  double* AV = p.dav_AV.as<double>();
  double* H = p.dav_H.as<double>();
  double* w = p.dav_w.as<double>();
  double* Y = p.dav_Y.as<double>();
  double* s = p.dav_s.as<double>();       // s[0..31]: coefficients, s[40..]: scalars
  double* part = p.dav_partial.as<double>();
  double* x = p.dav_x.as<double>();
  double* ax = p.dav_ax.as<double>();
  double* r = p.dav_r.as<double>();
  double* t = p.dav_t.as<double>();
  auto row = [&](double* M, int i) { return M + (long long)i * n; };
  double host[2];

  auto sigma = [&](const double* in, double* out) { run_sigma(c, p, in, out); };
  double* pinned = c.h_scalars.get();
  auto read2 = [&](const double* a, const double* b) {
    double* dst = pinned ? pinned : host;
    DMRG_CUDA(cudaMemcpyAsync(&dst[0], a, sizeof(double), cudaMemcpyDeviceToHost, st));
    DMRG_CUDA(cudaMemcpyAsync(&dst[1], b, sizeof(double), cudaMemcpyDeviceToHost, st));
    DMRG_CUDA(cudaStreamSynchronize(st));
    host[0] = dst[0];
    host[1] = dst[1];
  };
  // projected-matrix entries of the newest vector j: H[i][j] = V_i . AV_j, H[j][i] = V_j . AV_i
  auto update_H = [&](int k) {
    const int j = k - 1;
    dav_dots(V, n, k, row(AV, j), n, part, H + j, LDH, st);
    dav_dots(AV, n, k, row(V, j), n, part, H + (long long)j * LDH, 1, st);
  };

  ProfScope prof_all(c.prof, 2, st);
  // initial vector, normalised
  if (x0)
    DMRG_CUDA(cudaMemcpyAsync(row(V, 0), x0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else
    launch_gen_vector(row(V, 0), n, (uint64_t)(c.opts.seed ^ KEY_GUESS), guess_counter_base, st);
  dav_dots(V, n, 1, row(V, 0), n, part, s + 42, 1, st);
  dav_scale(row(V, 0), s + 42, n, st);
  sigma(row(V, 0), row(AV, 0));
  int k = 1, nmv = 1;
  update_H(k);
  bool converged = false;
  double theta = 0.0;
  int warm = 0;  // size of the projected matrix whose eigenvectors Y holds
  for (;;) {
    dav_eigh(H, k, LDH, w, Y, warm, st);
    warm = k;
    dav_lincomb(V, n, k, Y, LDH, 1.0, x, n, false, st);
    dav_lincomb(AV, n, k, Y, LDH, 1.0, ax, n, false, st);
    dav_residual(x, ax, p.dav_diag.as<double>(), w, r, t, n, st);
    dav_dots(r, n, 1, r, n, part, s + 40, 1, st);
    read2(w, s + 40);
    theta = host[0];
    const double rr = host[1];
    if (!(rr == rr)) throw Error(DMRG_ECUDA, "Davidson: residual is not a number");
    if (rr < tol) {
      converged = true;
      break;
    }
    if (nmv >= max_iter) break;
    if (k >= S) {  // thick restart from the two lowest Ritz vectors
      dav_lincomb(V, n, k, Y + 1, LDH, 1.0, r, n, false, st);   // r <- second Ritz vector
      DMRG_CUDA(cudaMemcpyAsync(row(V, 0), x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA(cudaMemcpyAsync(row(V, 1), r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      dav_lincomb(AV, n, k, Y + 1, LDH, 1.0, r, n, false, st);  // r <- H times it
      DMRG_CUDA(cudaMemcpyAsync(row(AV, 0), ax, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA(cudaMemcpyAsync(row(AV, 1), r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      k = 2;
      warm = 0;
      update_H(1);
      update_H(2);
    }
    // new direction: classical Gram-Schmidt twice against V, then normalise
    double* vk = row(V, k);
    DMRG_CUDA(cudaMemcpyAsync(vk, t, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int pass = 0; pass < 2; ++pass) {
      dav_dots(V, n, k, vk, n, part, s, 1, st);
      dav_lincomb(V, n, k, s, 1, -1.0, vk, n, true, st);
    }
    dav_dots(V + (long long)k * n, n, 1, vk, n, part, s + 41, 1, st);
    read2(s + 41, s + 41);
    if (std::sqrt(host[0]) < 1e-14) break;
    dav_scale(vk, s + 41, n, st);
    sigma(vk, row(AV, k));
    ++nmv;
    ++k;
    update_H(k);
  }
  if (c.opts.sigma_prec != DMRG_FP64) {
    // The mixed-precision operator differs from H by a relative 1e-5 or so,
    // which moves its eigenvalue at first order. The Rayleigh quotient of
    // the final vector with the FP64 sigma is off only at second order in
    // the vector's error, so it is the energy returned.
    run_sigma_f64(c, p, x, ax);
    dav_dots(x, n, 1, ax, n, part, s + 43, 1, st);
    dav_dots(x, n, 1, x, n, part, s + 44, 1, st);
    read2(s + 43, s + 44);
    theta = host[0] / host[1];
  }
  if (x_out) DMRG_CUDA(cudaMemcpyAsync(x_out, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DMRG_CUDA(cudaStreamSynchronize(st));
  check_device_error(c, p);
  *energy = theta;
  *iters = nmv;
  return converged;
}

}  // namespace dmrg
