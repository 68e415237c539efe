// Instantiations of the fused normal-operator kernel for Q = 16.
#include "normal_lines.cuh"

namespace nl {

NLKernel pick_q16(int P, int jmax, int mode, int ns) {
  if (ns == 1) {
    if (P == 16) return pick_j<16, 16, 1>(jmax, mode);
    if (P == 20) return pick_j<16, 20, 1>(jmax, mode);
    if (P == 23) return pick_j<16, 23, 1>(jmax, mode);
  } else if (ns == 2) {
    if (P == 20) return pick_j<16, 20, 2>(jmax, mode);
    if (P == 23) return pick_j<16, 23, 2>(jmax, mode);
  }
  return nullptr;
}

CgKernel pick_cg_q16(int P, int jmax, int ns) {
  if (ns == 1) {
    if (P == 16) return pick_cg_j<16, 16, 1>(jmax);
    if (P == 20) return pick_cg_j<16, 20, 1>(jmax);
    if (P == 23) return pick_cg_j<16, 23, 1>(jmax);
  } else if (ns == 2) {
    if (P == 20) return pick_cg_j<16, 20, 2>(jmax);
    if (P == 23) return pick_cg_j<16, 23, 2>(jmax);
  }
  return nullptr;
}

}  // namespace nl
