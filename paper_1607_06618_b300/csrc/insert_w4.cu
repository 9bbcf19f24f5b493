// insert_w4.cu -- instantiations of the insert kernel (insert.cuh) for keys of four words (97 <= k <= 128).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w4(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 4 * 32 + 3: return launch_insert_w<4, 3>(p, need, persistent, nsm, st);
    case 4 * 32 + 4: return launch_insert_w<4, 4>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
