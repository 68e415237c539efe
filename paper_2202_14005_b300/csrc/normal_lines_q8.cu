// Instantiations of the fused normal-operator kernel for Q = 8.
#include "normal_lines.cuh"

namespace nl {

NLKernel pick_q8(int P, int jmax, int mode, int ns) {
  if (ns == 1) {
    if (P == 8) return pick_j<8, 8, 1>(jmax, mode);
    if (P == 16) return pick_j<8, 16, 1>(jmax, mode);
    if (P == 29) return pick_j<8, 29, 1>(jmax, mode);
  } else if (ns == 2) {
    if (P == 16) return pick_j<8, 16, 2>(jmax, mode);
    if (P == 29) return pick_j<8, 29, 2>(jmax, mode);
  }
  return nullptr;
}

CgKernel pick_cg_q8(int P, int jmax, int ns) {
  if (ns == 1) {
    if (P == 8) return pick_cg_j<8, 8, 1>(jmax);
    if (P == 16) return pick_cg_j<8, 16, 1>(jmax);
    if (P == 29) return pick_cg_j<8, 29, 1>(jmax);
  } else if (ns == 2) {
    if (P == 16) return pick_cg_j<8, 16, 2>(jmax);
    if (P == 29) return pick_cg_j<8, 29, 2>(jmax);
  }
  return nullptr;
}

}  // namespace nl
