// insert_w8_11.cu -- instantiations of the insert kernel (insert.cuh) for keys of eight to eleven words (225 <= k <= 352).
#include "insert.cuh"

namespace gerbil {

cudaError_t launch_insert_w8_11(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st) {
  switch (W * 32 + WS) {
    case 8 * 32 + 7: return launch_insert_w<8, 7>(p, need, persistent, nsm, st);
    case 8 * 32 + 8: return launch_insert_w<8, 8>(p, need, persistent, nsm, st);
    case 9 * 32 + 8: return launch_insert_w<9, 8>(p, need, persistent, nsm, st);
    case 9 * 32 + 9: return launch_insert_w<9, 9>(p, need, persistent, nsm, st);
    case 10 * 32 + 9: return launch_insert_w<10, 9>(p, need, persistent, nsm, st);
    case 10 * 32 + 10: return launch_insert_w<10, 10>(p, need, persistent, nsm, st);
    case 11 * 32 + 10: return launch_insert_w<11, 10>(p, need, persistent, nsm, st);
    case 11 * 32 + 11: return launch_insert_w<11, 11>(p, need, persistent, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gerbil
