// Host-logic check of the wavefunction carry between sweep steps (CPU only,
// no CUDA calls): builds the two GEMM passes with the library's own
// carry_jobs (terms.h) from the bases of the previous and the next bond and
// the stored bases of the two blocks involved, applies them with a plain CPU
// loop (the strided GEMM semantics of the device kernel), and writes psi'.
//
//   carry_check <in file> <out file>
//   in (int32 unless noted): forward, N, 2Sz; four bases (previous left,
//   previous right, next left, next right block), each nsec then nsec x
//   (N, 2Sz, dim); then for the left and the right block with stored states:
//   nsec, nsec x (N, 2Sz, k), float64 matrices d x k row-major in sector
//   order; then float64 previous psi (its layout's length)
//   out: int64 count, then that many float64 (psi' over the next bond)
#include <cstdio>
#include <vector>

#include "model.h"
#include "terms.h"

using namespace dmrg;
using namespace dmrg::terms;

static bool read_basis(FILE* f, Basis& b) {
  int ns = 0;
  if (std::fread(&ns, sizeof(int), 1, f) != 1) return false;
  for (int i = 0; i < ns; ++i) {
    int q[3];
    if (std::fread(q, sizeof(int), 3, f) != 3) return false;
    b.q.push_back({q[0], q[1]});
    b.dim.push_back(q[2]);
  }
  b.finish();
  return true;
}

static void apply(const std::vector<GJob>& jobs, const double* A, const double* B, double* C) {
  for (const GJob& g : jobs)
    for (int i = 0; i < g.m; ++i)
      for (int j = 0; j < g.n; ++j) {
        double acc = 0.0;
        for (int k = 0; k < g.kk; ++k) {
          const double a = A[g.a + (g.ta ? (long long)k * g.lda + i : (long long)i * g.lda + k)];
          const double b = B[g.b + (g.tb ? (long long)j * g.ldb + k : (long long)k * g.ldb + j)];
          acc += a * b;
        }
        C[g.c + (long long)i * g.ldc + j] = acc;
      }
}

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 3;
  int hdr[3];
  if (std::fread(hdr, sizeof(int), 3, f) != 3) return 4;
  const bool forward = hdr[0] != 0;
  const QN Q{hdr[1], hdr[2]};
  Basis pL, pR, nL, nR;
  if (!read_basis(f, pL) || !read_basis(f, pR) || !read_basis(f, nL) || !read_basis(f, nR)) return 4;
  const Enlarged prev_EL = enlarge(pL), prev_ER = enlarge(pR), EL = enlarge(nL), ER = enlarge(nR);
  // blocks with stored states and the enlarged bases they were made from
  Basis lb, rb;
  std::vector<long long> luoff, ruoff;
  std::vector<int> lesec, resec;
  std::vector<double> lu, ru;
  const Enlarged& lpar = forward ? prev_EL : EL;
  const Enlarged& rpar = forward ? ER : prev_ER;
  for (int side = 0; side < 2; ++side) {
    Basis& b = side == 0 ? lb : rb;
    std::vector<long long>& uoff = side == 0 ? luoff : ruoff;
    std::vector<int>& esec = side == 0 ? lesec : resec;
    std::vector<double>& u = side == 0 ? lu : ru;
    const Enlarged& par = side == 0 ? lpar : rpar;
    if (!read_basis(f, b)) return 4;
    long long off = 0;
    for (int s = 0; s < b.size(); ++s) {
      const int e = par.basis.find(b.q[s]);
      if (e < 0) return 5;
      esec.push_back(e);
      uoff.push_back(off);
      off += (long long)par.basis.dim[e] * b.dim[s];
    }
    u.resize((size_t)off);
    if (std::fread(u.data(), sizeof(double), u.size(), f) != u.size()) return 4;
  }
  long long prev_size = 0, size = 0;
  const std::vector<PsiBlock> prev_blocks = psi_layout(prev_EL.basis, prev_ER.basis, Q, &prev_size);
  const std::vector<PsiBlock> blocks = psi_layout(EL.basis, ER.basis, Q, &size);
  std::vector<double> psi((size_t)prev_size);
  if (std::fread(psi.data(), sizeof(double), psi.size(), f) != psi.size()) return 4;
  std::fclose(f);

  std::vector<GJob> j1, j2;
  long long phi_size = 0;
  carry_jobs(forward, prev_blocks, prev_EL, prev_ER, EL, ER, blocks, {&lb, &luoff, &lesec}, {&rb, &ruoff, &resec}, j1,
             j2, phi_size);
  std::vector<double> phi((size_t)phi_size, 0.0), out((size_t)size, 0.0);
  if (forward) {
    apply(j1, lu.data(), psi.data(), phi.data());
    apply(j2, phi.data(), ru.data(), out.data());
  } else {
    apply(j1, psi.data(), ru.data(), phi.data());
    apply(j2, lu.data(), phi.data(), out.data());
  }
  FILE* g = std::fopen(argv[2], "wb");
  std::fwrite(&size, sizeof(size), 1, g);
  std::fwrite(out.data(), sizeof(double), out.size(), g);
  std::fclose(g);
  return 0;
}
