// Instantiations of the fused normal-operator kernel for Q = 16.
#include "normal_lines.cuh"

namespace nl {

NLKernel pick_q16(int P, int jmax, int mode) {
  if (P == 16) return pick_j<16, 16>(jmax, mode);
  if (P == 20) return pick_j<16, 20>(jmax, mode);
  if (P == 23) return pick_j<16, 23>(jmax, mode);
  return nullptr;
}

}  // namespace nl
