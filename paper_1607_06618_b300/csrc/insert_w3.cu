// insert_w3.cu -- instantiations of the insert kernel (insert.cuh) for keys of three words (65 <= k <= 96).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w3(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 3 * 32 + 2: return launch_insert_w<3, 2>(p, need, persistent, nsm, st);
    case 3 * 32 + 3: return launch_insert_w<3, 3>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
