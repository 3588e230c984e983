// Host check of the decoder's shared-memory layout (make_layout in
// gdg_kernel.cuh), built with g++ by tests/test_layout_host.py.
//
// usage: layout_check nr nc ne ns es nb nslots stage_graph ranker
// Prints "ok" or the first violated invariant:
//   * every region starts on a 16-byte boundary (bulk copies and 16-byte
//     vector loads need it) and regions of one part do not overlap;
//   * the persistent part ends at U; the union holds the pre-BP scratch and
//     nslots path slots; total = U + union;
//   * the window graph staged for the pre-BP lies after the arrays the pre-BP
//     writes (post, key, check states, signs, parity words) and inside the
//     union;
//   * the sort buffer holds a power of two >= nc keys, and the shortened-graph
//     build's scratch (n_short + 1 ints) fits in it.
#define __host__
#define __device__
#define __align__(n) alignas(n)
#include "../paper_2403_18901_gb300/csrc/gdg_kernel.cuh"

#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {
struct Region {
  const char* name;
  unsigned off, bytes;
};

bool check(const std::vector<Region>& rs, unsigned lo, unsigned hi, const char* part) {
  unsigned end = lo;
  for (const Region& r : rs) {
    if (r.off % 16u) {
      std::printf("%s.%s at %u: not 16-byte aligned\n", part, r.name, r.off);
      return false;
    }
    if (r.off < end) {
      std::printf("%s.%s at %u overlaps the region before (ends %u)\n", part, r.name, r.off, end);
      return false;
    }
    end = r.off + r.bytes;
    if (end > hi) {
      std::printf("%s.%s ends at %u past %u\n", part, r.name, end, hi);
      return false;
    }
  }
  return true;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 10) {
    std::printf("usage: layout_check nr nc ne ns es nb nslots stage_graph ranker\n");
    return 2;
  }
  const int nr = std::atoi(argv[1]), nc = std::atoi(argv[2]), ne = std::atoi(argv[3]), ns = std::atoi(argv[4]);
  const int es = std::atoi(argv[5]), nb = std::atoi(argv[6]), nslots = std::atoi(argv[7]);
  const bool stage = std::atoi(argv[8]) != 0, ranker = std::atoi(argv[9]) != 0;
  const qd::Layout L = qd::make_layout(nr, nc, ne, ns, es, nb, nslots, stage, ranker);
  const unsigned rw = L.rw, sw = L.sw;
  std::vector<Region> pers = {
      {"sbits", L.sbits, 4u * rw},           {"cbits", L.cbits, 4u * L.cw},
      {"sel", L.sel, 2u * ns},               {"s_colptr", L.s_colptr, 2u * (ns + 1)},
      {"s_colrows", L.s_colrows, 2u * es},   {"s_rowptr", L.s_rowptr, 2u * (nr + 1)},
      {"s_rowent", L.s_rowent, 4u * es},     {"s_llr", L.s_llr, 4u * ns},
      {"s_vdeg", L.s_vdeg, 1u * ns},         {"s_efull", L.s_efull, 2u * es},
      {"s_cperm", L.s_cperm, 2u * nr},       {"s_vperm", L.s_vperm, 2u * ns},
      {"rowcnt", L.rowcnt, 4u * (nr + 1)},   {"res_status", L.res_status, 4u * nb},
      {"res_pm", L.res_pm, 8u * nb},         {"res_ebits", L.res_ebits, 4u * sw * nb},
      {"red", L.red, 16u * 32},              {"misc", L.misc, 64u}};
  if (stage) {
    pers.push_back({"g_colptr", L.g_colptr, 2u * (nc + 1)});
    pers.push_back({"g_colrows", L.g_colrows, 2u * ne});
    pers.push_back({"g_rowptr", L.g_rowptr, 2u * (nr + 1)});
    pers.push_back({"g_rowent", L.g_rowent, 4u * ne});
    pers.push_back({"g_llr", L.g_llr, 4u * nc});
  }
  if (!check(pers, 0, L.U, "persistent")) return 1;
  if (L.U % 16u) {
    std::printf("U = %u not 16-byte aligned\n", L.U);
    return 1;
  }
  const unsigned ub = L.total - L.U;
  const std::vector<Region> pre = {{"p_post", L.p_post, 4u * nc}, {"p_key", L.p_key, 4u * nc},
                                   {"p_cns", L.p_cns, 16u * nr},  {"p_sign", L.p_sign, 1u * ne},
                                   {"p_par", L.p_par, 8u * rw},   {"p_sort", L.p_sort, 8u * L.sortn}};
  if (!check(pre, 0, ub, "pre-BP")) return 1;
  if (L.p_end > ub) {
    std::printf("pre-BP scratch (%u) larger than the union (%u)\n", L.p_end, ub);
    return 1;
  }
  const std::vector<Region> slot = {
      {"b_post", L.b_post, 4u * ns},     {"b_acc", L.b_acc, 4u * ns},   {"b_hfl", L.b_hfl, 1u * ns},
      {"b_status", L.b_status, 1u * ns}, {"b_sign", L.b_sign, 1u * es}, {"b_cns", L.b_cns, 16u * nr},
      {"b_deg", L.b_deg, 4u * nr},       {"b_sp", L.b_sp, 4u * rw},     {"b_unsat", L.b_unsat, 4u * rw},
      {"b_hq", L.b_hq, ranker ? 4u * ns : 0u}};
  if (!check(slot, 0, L.b_size, "slot")) return 1;
  if (L.b_size % 16u || (unsigned long long)L.b_size * (unsigned)nslots > ub) {
    std::printf("slots: %d x %u bytes in a union of %u\n", nslots, L.b_size, ub);
    return 1;
  }
  if (L.pre_stage) {
    const std::vector<Region> q = {{"q_colptr", L.q_colptr, 2u * (nc + 1)}, {"q_colrows", L.q_colrows, 2u * ne},
                                   {"q_rowptr", L.q_rowptr, 2u * (nr + 1)}, {"q_rowent", L.q_rowent, 4u * ne},
                                   {"q_llr", L.q_llr, 4u * nc},             {"q_vperm", L.q_vperm, 2u * nc}};
    if (!check(q, L.p_sort, ub, "staged graph")) return 1;
  }
  if (L.sortn < nc || (L.sortn & (L.sortn - 1))) {
    std::printf("sort buffer of %d keys for %d columns\n", L.sortn, nc);
    return 1;
  }
  if (4ull * (ns + 1) > 8ull * L.sortn) {
    std::printf("shortening scratch (%d ints) larger than the sort buffer\n", ns + 1);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
