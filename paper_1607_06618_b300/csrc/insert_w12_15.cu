// insert_w12_15.cu -- instantiations of the insert kernel (insert.cuh) for keys of twelve to fifteen words (353 <= k <= 479).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w12_15(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 12 * 32 + 11: return launch_insert_w<12, 11>(p, need, persistent, nsm, st);
    case 12 * 32 + 12: return launch_insert_w<12, 12>(p, need, persistent, nsm, st);
    case 13 * 32 + 12: return launch_insert_w<13, 12>(p, need, persistent, nsm, st);
    case 13 * 32 + 13: return launch_insert_w<13, 13>(p, need, persistent, nsm, st);
    case 14 * 32 + 13: return launch_insert_w<14, 13>(p, need, persistent, nsm, st);
    case 14 * 32 + 14: return launch_insert_w<14, 14>(p, need, persistent, nsm, st);
    case 15 * 32 + 14: return launch_insert_w<15, 14>(p, need, persistent, nsm, st);
    case 15 * 32 + 15: return launch_insert_w<15, 15>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
