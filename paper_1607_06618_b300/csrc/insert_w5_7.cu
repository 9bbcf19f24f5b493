// insert_w5_7.cu -- instantiations of the insert kernel (insert.cuh) for keys of five to seven words (129 <= k <= 224).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w5_7(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 5 * 32 + 4: return launch_insert_w<5, 4>(p, need, persistent, nsm, st);
    case 5 * 32 + 5: return launch_insert_w<5, 5>(p, need, persistent, nsm, st);
    case 6 * 32 + 5: return launch_insert_w<6, 5>(p, need, persistent, nsm, st);
    case 6 * 32 + 6: return launch_insert_w<6, 6>(p, need, persistent, nsm, st);
    case 7 * 32 + 6: return launch_insert_w<7, 6>(p, need, persistent, nsm, st);
    case 7 * 32 + 7: return launch_insert_w<7, 7>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
