// Host check of the decision-path schedule of the decoder (path_split,
// path_reinit, path_at in gdg_kernel.cuh), built with g++ by
// tests/test_layout_host.py.
//
// usage: tree_check k side_max reinit nb dmax_main dmax_other
// Prints one line per queue position: "pos id split reinit dmax".
#define __host__
#define __device__
#define __align__(n) alignas(n)
#include "../paper_2403_18901_gb300/csrc/gdg_kernel.cuh"

#include <cstdio>
#include <cstdlib>

int main(int argc, char** argv) {
  if (argc != 7) {
    std::printf("usage: tree_check k side_max reinit nb dmax_main dmax_other\n");
    return 2;
  }
  qd::KParams P{};
  P.k = std::atoi(argv[1]);
  P.side_max = std::atoi(argv[2]);
  P.reinit = std::atoi(argv[3]);
  P.nb = std::atoi(argv[4]);
  P.dmax_main = std::atoi(argv[5]);
  P.dmax_other = std::atoi(argv[6]);
  for (int pos = 0; pos < P.nb; ++pos) {
    const int id = qd::path_at(P, pos);
    const int split = qd::path_split(P, id);
    const int dmax = qd::path_dmax(P, id, split);
    std::printf("%d %d %d %d %d\n", pos, id, split, qd::path_reinit(P, id, split), dmax);
  }
  return 0;
}
