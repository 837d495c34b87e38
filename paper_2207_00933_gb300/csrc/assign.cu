// States assignment (Section 4, Algorithm 2) and the qubit roles of one
// recursion (Algorithm 1).  Host code only: no device work.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/sqc.h"

extern "C" {

SQC_API sqc_status sqc_assign_states(int32_t n_subcircuits, const uint64_t* l, uint64_t M, uint64_t* l_out) {
  if (n_subcircuits < 1 || !l || !l_out || M < 1) return SQC_EINVAL;
  std::vector<uint64_t> lp(l, l + n_subcircuits);
  auto product_exceeds = [&]() {
    // product > M, without overflowing: p * v > M  <=>  p > floor(M / v)
    uint64_t p = 1;
    for (uint64_t v : lp) {
      if (v == 0) return false;
      if (p > M / v) return true;
      p *= v;
    }
    return false;
  };
  while (product_exceeds()) {
    int best = 0;
    for (int i = 1; i < n_subcircuits; ++i)
      if (lp[i] > lp[best]) best = i;           // ties: lowest index
    if (lp[best] <= 1) break;
    lp[best] = (lp[best] + 1) / 2;              // ceil(l / 2)
  }
  std::copy(lp.begin(), lp.end(), l_out);
  return SQC_OK;
}

SQC_API sqc_status sqc_recursion_roles(const sqc_graph* g, const int8_t* zoom, uint64_t M, int8_t* roles) {
  if (!g || !zoom || !roles || g->n_subcircuits < 1 || !g->n_data || !g->data_qubit) return SQC_EINVAL;
  const int nq = g->n_qubits, nc = g->n_subcircuits;
  std::vector<std::vector<int>> free(nc);
  int off = 0;
  for (int i = 0; i < nc; ++i) {
    for (int t = 0; t < g->n_data[i]; ++t) {
      const int q = g->data_qubit[off + t];
      if (q < 0 || q >= nq) return SQC_EINVAL;
      if (zoom[q] != SQC_ROLE_ZOOM0 && zoom[q] != SQC_ROLE_ZOOM1) free[i].push_back(q);
    }
    off += g->n_data[i];
  }
  std::vector<uint64_t> l(nc), lp(nc);
  for (int i = 0; i < nc; ++i) {
    if (free[i].size() > 62) return SQC_ESHAPE;
    l[i] = uint64_t(1) << free[i].size();
  }
  sqc_status st = sqc_assign_states(nc, l.data(), M, lp.data());
  if (st != SQC_OK) return st;
  for (int q = 0; q < nq; ++q)
    roles[q] = (zoom[q] == SQC_ROLE_ZOOM0 || zoom[q] == SQC_ROLE_ZOOM1) ? zoom[q] : int8_t(SQC_ROLE_MERGED);
  for (int i = 0; i < nc; ++i) {
    int a = 0;
    while ((uint64_t(1) << a) < lp[i]) ++a;     // l'_i is a power of two
    for (int t = 0; t < a && t < int(free[i].size()); ++t) roles[free[i][t]] = SQC_ROLE_ACTIVE;
  }
  return SQC_OK;
}

}  // extern "C"
