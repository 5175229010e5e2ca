// hop_df64.cu -- DF64 (double-float) instantiations of the hopping block (Sec. II-B).
#include "hop.cuh"

namespace bsm {

int launch_hop_df64(int d, bool real, const HopArgs& A, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: return launch_hop_t<DF64, 3, true>(A, s);
      case 8: return launch_hop_t<DF64, 8, true>(A, s);
      default: return -1;
    }
  }
  switch (d) {
    case 2: return launch_hop_t<DF64, 2, false>(A, s);
    case 3: return launch_hop_t<DF64, 3, false>(A, s);
    case 4: return launch_hop_t<DF64, 4, false>(A, s);
    case 6: return launch_hop_t<DF64, 6, false>(A, s);
    case 8: return launch_hop_t<DF64, 8, false>(A, s);
    default: return -1;
  }
}

}  // namespace bsm
