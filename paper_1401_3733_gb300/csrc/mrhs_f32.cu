// mrhs_f32.cu -- FP32 instantiations of the multi-RHS hopping block (Sec. II-B).
#include "mrhs.cuh"

namespace bsm {

bool launch_mrhs_f32(int d, bool real, int rb, const MrhsArgs& A, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: return launch_mrhs_rb<F32, 3, true>(rb, A, s);
      case 8: return launch_mrhs_rb<F32, 8, true>(rb, A, s);
      default: return false;
    }
  }
  switch (d) {
    case 2: return launch_mrhs_rb<F32, 2, false>(rb, A, s);
    case 3: return launch_mrhs_rb<F32, 3, false>(rb, A, s);
    case 4: return launch_mrhs_rb<F32, 4, false>(rb, A, s);
    case 6: return launch_mrhs_rb<F32, 6, false>(rb, A, s);
    case 8: return launch_mrhs_rb<F32, 8, false>(rb, A, s);
    default: return false;
  }
}

}  // namespace bsm
