// hop_f32.cu -- FP32 instantiations of the hopping block (Sec. II-B).
#include "hop.cuh"

namespace bsm {

int launch_hop_f32(int d, bool real, const HopArgs& A, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: return launch_hop_t<F32, 3, true>(A, s);
      case 8: return launch_hop_t<F32, 8, true>(A, s);
      default: return -1;
    }
  }
  switch (d) {
    case 2: return launch_hop_t<F32, 2, false>(A, s);
    case 3: return launch_hop_t<F32, 3, false>(A, s);
    case 4: return launch_hop_t<F32, 4, false>(A, s);
    case 6: return launch_hop_t<F32, 6, false>(A, s);
    case 8: return launch_hop_t<F32, 8, false>(A, s);
    default: return -1;
  }
}

}  // namespace bsm
