// insert_w1_2.cu -- instantiations of the insert kernel (insert.cuh) for keys of one or two words (k <= 64).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w1_2(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 1 * 32 + 1: return launch_insert_w<1, 1>(p, need, persistent, nsm, st);
    case 2 * 32 + 1: return launch_insert_w<2, 1>(p, need, persistent, nsm, st);
    case 2 * 32 + 2: return launch_insert_w<2, 2>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
