// membench.cu -- throughput of the memory operations the counting kernel is built from, on the
// GPU at hand: the ceilings that the insert kernel's rate is compared with (besides HBM copy
// bandwidth).  Every thread performs `per_thread` operations at pseudo-random 32-byte-aligned
// slots of an array of `bytes` bytes (L2-resident or not, by size).
#include <algorithm>

#include "../../include/gerbil.h"
#include "common.cuh"
#include "kernels.h"

namespace gerbil {

__device__ __forceinline__ unsigned long long mb_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// op 0: red.add.u64 on slot word 0; 1: 32-byte relaxed load of the slot; 2: 32-byte load then
// red.add on the same slot (a found-key insert); 3: CAS on slot word 0 (a new-key claim).
__global__ void __launch_bounds__(256) membench_kernel(unsigned long long* arr, unsigned long long nslots,
                                                       int op, unsigned long long per_thread,
                                                       unsigned long long* sink) {
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  unsigned long long acc = 0;
  for (unsigned long long i = 0; i < per_thread; ++i) {
    const unsigned long long s = mb_mix(tid * 0x9E3779B97F4A7C15ull + i) % nslots;
    unsigned long long* slot = arr + s * 4;
    if (op == 0) {
      red_add(slot, 1ull);
    } else if (op == 1) {
      unsigned long long a, b, c, d;
      ld_relaxed_v2(slot, a, b);
      ld_relaxed_v2(slot + 2, c, d);
      acc += a ^ b ^ c ^ d;
    } else if (op == 2) {
      unsigned long long a, b, c, d;
      ld_relaxed_v2(slot, a, b);
      ld_relaxed_v2(slot + 2, c, d);
      if ((a ^ b ^ c ^ d) != 1ull) red_add(slot, 1ull);  // data-dependent, as in a probe
    } else {
      acc += cas_relaxed(slot, acc, acc + 1);
    }
  }
  if (acc == 0x123456789ull) *sink = acc;  // keeps the loads alive
}

}  // namespace gerbil

// The context struct is private to runtime.cu; these two helpers live there.
extern "C" int gerbil_internal_alloc(gerbil_ctx* ctx, void** p, size_t bytes, void** stream, int* nsm);
extern "C" void gerbil_internal_free(gerbil_ctx* ctx, void* p, size_t bytes);

extern "C" int gerbil_membench(gerbil_ctx* ctx, uint64_t bytes, int op, uint64_t per_thread,
                               double* gops) {
  if (!ctx || !gops || op < 0 || op > 3 || bytes < 4096 || per_thread < 1) return GERBIL_E_INVAL;
  void* mem = nullptr;
  void* stream = nullptr;
  int nsm = 0;
  int rc = gerbil_internal_alloc(ctx, &mem, bytes + 256, &stream, &nsm);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* arr = (unsigned long long*)mem;
  const unsigned long long nslots = bytes / 32;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  const unsigned grid = (unsigned)nsm * 8;
  bool ok = cudaMemsetAsync(mem, 0, bytes + 256, st) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (ok) {
    gerbil::membench_kernel<<<grid, 256, 0, st>>>(arr, nslots, op, std::min<uint64_t>(per_thread, 64),
                                                  arr + nslots * 4);  // warm-up
    cudaEventRecord(e0, st);
    gerbil::membench_kernel<<<grid, 256, 0, st>>>(arr, nslots, op, per_thread, arr + nslots * 4);
    cudaEventRecord(e1, st);
    ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  gerbil_internal_free(ctx, mem, bytes + 256);
  if (!ok || ms <= 0.f) {
    cudaGetLastError();
    return GERBIL_E_CUDA;
  }
  *gops = (double)grid * 256.0 * (double)per_thread / (ms * 1e-3) / 1e9;
  return GERBIL_OK;
}
