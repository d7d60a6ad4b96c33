// Host-logic check of the global truncation (CPU only): reads singular values
// per psi block with the block's left quantum numbers, applies the library's
// select_kept (terms.h) and prints the kept count per block and the
// discarded weight as JSON.
//
//   truncation_check <M> <keep_one_per_q> < input
//   input: nb, then per block: N 2Sz count v_1 ... v_count (descending)
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "model.h"
#include "terms.h"

using namespace dmrg;

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  const int M = std::atoi(argv[1]);
  const bool keep_one = std::atoi(argv[2]) != 0;
  int nb = 0;
  if (std::scanf("%d", &nb) != 1) return 3;
  std::vector<std::vector<double>> sv(nb);
  std::vector<QN> qL(nb);
  for (int b = 0; b < nb; ++b) {
    int n, s, c;
    if (std::scanf("%d %d %d", &n, &s, &c) != 3) return 3;
    qL[b] = {n, s};
    sv[b].resize(c);
    for (int i = 0; i < c; ++i)
      if (std::scanf("%lf", &sv[b][i]) != 1) return 3;
  }
  double disc = 0.0;
  const std::vector<int> kept = terms::select_kept(sv, qL, M, keep_one, &disc);
  std::printf("{\"kept\": [");
  for (int b = 0; b < nb; ++b) std::printf("%s%d", b ? ", " : "", kept[b]);
  std::printf("], \"discarded\": %.17g}\n", disc);
  return 0;
}
