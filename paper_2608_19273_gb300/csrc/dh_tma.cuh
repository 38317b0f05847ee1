// TMA helpers of the finite-volume stage: 5-D tensor maps over an arena level
// (x, y, z, patch, variable), bulk tensor copies into shared memory that complete
// on an mbarrier, and a bounded wait.  Every copy reads this GPU's own memory; no
// cluster multicast is used.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "dh_internal.cuh"

namespace dh {
namespace fvtma {

// An encoded tensor map (CUtensorMap: 128 bytes, 64-byte aligned), passed to the kernel as
// part of a __grid_constant__ parameter.
struct alignas(64) Map {
  unsigned long long v[16];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// The arrival of the issuing thread, announcing `bytes` of copies that complete on `bar`.
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One 5-D tile copy into shared memory (dst 128-byte aligned; c0 * 8 bytes a multiple of 16).
__device__ __forceinline__ void load5(void* dst, const Map* map, int c0, int c1, int c2, int c3, int c4,
                                      uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of `bar`, giving up after ~2^27 SM clocks (about 65 ms) or as
// soon as `*abort` is set (by another thread that gave up, or on entry).  Returns false if
// it gave up.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort || clock64() - t0 > (1ll << 27)) return false;
  }
}

// Host: encode the tiled 5-D map of one arena level (patches of p^3 voxels stored back to
// back from `base`, nv variables var_stride apart) with box {bx, by, 1, 1, nv}.
dh_status encode_level(const double* base, int p, int K, int nv, int64_t var_stride, int bx, int by, Map* out);

}  // namespace fvtma
}  // namespace dh
