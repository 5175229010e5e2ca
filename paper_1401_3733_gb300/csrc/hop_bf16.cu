// hop_bf16.cu -- BF16-storage (FP32 arithmetic) instantiations of the hopping block (Sec. II-B).
#include "hop.cuh"

namespace bsm {

int launch_hop_bf16(int d, bool real, const HopArgs& A, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: return launch_hop_t<BF16, 3, true>(A, s);
      case 8: return launch_hop_t<BF16, 8, true>(A, s);
      default: return -1;
    }
  }
  switch (d) {
    case 2: return launch_hop_t<BF16, 2, false>(A, s);
    case 3: return launch_hop_t<BF16, 3, false>(A, s);
    case 4: return launch_hop_t<BF16, 4, false>(A, s);
    case 6: return launch_hop_t<BF16, 6, false>(A, s);
    case 8: return launch_hop_t<BF16, 8, false>(A, s);
    default: return -1;
  }
}

}  // namespace bsm
