// hop_f32r12.cu -- FP32 hopping block with SU(3) links stored as two rows
// (Sec. II-B "Dphi"): 12 instead of 18 reals per link, the third row rebuilt
// in registers, a quarter less memory traffic per output site.
#include "hop.cuh"

namespace bsm {

int launch_hop_f32r12(int d, bool real, const HopArgs& A, cudaStream_t s) {
  if (d == 3 && !real) return launch_hop_t<F32R12, 3, false>(A, s);
  return -1;
}

}  // namespace bsm
