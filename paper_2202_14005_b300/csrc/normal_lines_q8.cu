// Instantiations of the fused normal-operator kernel for Q = 8.
#include "normal_lines.cuh"

namespace nl {

NLKernel pick_q8(int P, int jmax, int mode) {
  if (P == 8) return pick_j<8, 8>(jmax, mode);
  if (P == 16) return pick_j<8, 16>(jmax, mode);
  if (P == 29) return pick_j<8, 29>(jmax, mode);
  return nullptr;
}

}  // namespace nl
