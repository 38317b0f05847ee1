// AoAoS <-> SoA arena: the gather prologue K~^(0) and the scatter epilogue
// K~^(S+1) that embed the batched kernel (paper Sec. III-C, Eq. 4).
//
// The paper's input is K separately allocated patches, each one array of
// structs (Sec. II-B): voxel after voxel, the nq quantities of a voxel next to
// each other, over the p^ = p + 2h voxels per dimension of the patch and its
// halo (Sec. II, Eq. 2).  The kernels of this library work on the SoA arena
// (one contiguous run per variable and patch), so these two kernels convert:
//
//   gather : arena[v*vs + off_k + (z*p + y)*p + x] = blk_k[(((z+h)*p^ + y+h)*p^ + x+h)*nq + v]
//   scatter: the reverse assignment
//
// for the interior voxels only; halo entries of the blocks are never read or
// written (halos come from the face neighbours inside the stage kernels).
//
// Design (an HBM-bound permutation, 16 bytes of traffic per element):
//   * A CTA takes one unit of the plan's unit list: up to AO_UNIT_VOXELS
//     consecutive interior voxels (arena order) of one patch; units of the
//     largest patches come first.
//   * A warp takes one segment of SEG consecutive interior voxels of the unit.
//     In the arena a segment is one contiguous run per variable; in the AoS
//     block it is SEG*nq doubles per row, rows separated by the halo.  The
//     warp first tabulates the block position of each of its voxels, then
//     reads the segment with coalesced loads (four in flight per lane) into
//     its own shared-memory slice (voxel-major, pitch nq|1 so that the
//     transposed reads are free of bank conflicts) and writes it out
//     coalesced in the other order.  Only __syncwarp is needed.
//   * Index splits j -> (voxel, quantity) and x -> (row, x) multiply by a
//     float reciprocal of the divisor; every quotient involved is below 2^9
//     and every dividend below 2^15, so the result is the exact quotient.
#include <algorithm>

#include "dh_internal.cuh"

namespace dh {
namespace {

constexpr int AO_WARPS = 8;
constexpr int AO_MAX_NQ = 256;
constexpr int AO_BATCH = 4;                   // loads in flight per lane
constexpr size_t AO_SMEM_TARGET = 96 * 1024;  // two CTAs per SM up to this size

struct AoArgs {
  const dh_patch* patches;
  const int2* units;      // (patch, first voxel)
  const double* const* src_blocks;
  double* const* dst_blocks;
  const double* src_arena;
  double* dst_arena;
  int64_t vs;
  int nq;        // quantities per voxel in a block (its struct size in doubles)
  int v0, nv;    // quantities v0 .. v0+nv-1 of a voxel <-> arena variables 0 .. nv-1
  int nvp;       // shared-memory pitch nv | 1
  int halo, dim, seg;
  float inv_nv;
};

// Shared memory of one warp: SEG x nvp doubles, then SEG ints (block voxel index of each voxel).
__host__ __device__ inline size_t ao_warp_bytes(int seg, int nvp) {
  return (size_t)seg * nvp * sizeof(double) + (size_t)seg * sizeof(int);
}

__device__ __forceinline__ int fdiv_small(int a, float inv_b) { return (int)(((float)a + 0.5f) * inv_b); }

template <bool GATHER>
__global__ void __launch_bounds__(AO_WARPS * 32) k_aoas(const __grid_constant__ AoArgs A) {
  extern __shared__ double ao_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = A.nq, nv = A.nv, nvp = A.nvp, seg = A.seg, h = A.halo;
  unsigned char* wbase = reinterpret_cast<unsigned char*>(ao_smem) + (size_t)warp * ao_warp_bytes(seg, nvp);
  double* s = reinterpret_cast<double*>(wbase);
  int* tab = reinterpret_cast<int*>(wbase + (size_t)seg * nvp * sizeof(double));
  const int2 u = A.units[blockIdx.x];
  const int k = u.x;
  const int p = A.patches[k].p;
  const int64_t off = A.patches[k].offset;
  const int ph = p + 2 * h;
  const int nvox = A.dim == 3 ? p * p * p : p * p;
  const int uvox = min(AO_UNIT_VOXELS, nvox - u.y);
  const int nsegs = (uvox + seg - 1) / seg;
  const float inv_p = 1.0f / (float)p;
  const double* __restrict__ blk_in = GATHER ? A.src_blocks[k] + A.v0 : nullptr;
  double* __restrict__ blk_out = GATHER ? nullptr : A.dst_blocks[k] + A.v0;
  for (int sg = warp; sg < nsegs; sg += AO_WARPS) {
    const int i0 = u.y + sg * seg;               // first voxel of the segment (patch-local, arena order)
    const int n = min(seg, u.y + uvox - i0);
    // block voxel index of every voxel of the segment
    const int row0 = i0 / p, x0 = i0 - row0 * p;
    const int z0 = A.dim == 3 ? row0 / p : 0, y0 = row0 - z0 * p;
    for (int lv = lane; lv < n; lv += 32) {
      const int t = x0 + lv;
      const int dr = fdiv_small(t, inv_p);       // rows advanced (t < p + seg)
      const int x = t - dr * p;
      int y = y0 + dr, z = z0;
      if (A.dim == 3) {
        const int dz = fdiv_small(y, inv_p);     // y < p + seg
        y -= dz * p;
        z += dz;
      }
      tab[lv] = A.dim == 3 ? ((z + h) * ph + (y + h)) * ph + (x + h) : (y + h) * ph + (x + h);
    }
    __syncwarp();
    const int64_t soff = off + i0;
    const int tot = n * nv;
    const float inv_n = 1.0f / (float)n;
    if (GATHER) {
      for (int jb = lane; jb < tot; jb += 32 * AO_BATCH) {
        double r[AO_BATCH];
#pragma unroll
        for (int b = 0; b < AO_BATCH; ++b) {
          const int j = jb + 32 * b;
          if (j < tot) {
            const int lv = fdiv_small(j, A.inv_nv);
            r[b] = __ldg(blk_in + (int64_t)tab[lv] * nq + (j - lv * nv));
          }
        }
#pragma unroll
        for (int b = 0; b < AO_BATCH; ++b) {
          const int j = jb + 32 * b;
          if (j < tot) {
            const int lv = fdiv_small(j, A.inv_nv);
            s[lv * nvp + (j - lv * nv)] = r[b];
          }
        }
      }
      __syncwarp();
      for (int e = lane; e < tot; e += 32) {
        const int v = fdiv_small(e, inv_n);
        const int lv = e - v * n;
        A.dst_arena[v * A.vs + soff + lv] = s[lv * nvp + v];
      }
    } else {
      for (int eb = lane; eb < tot; eb += 32 * AO_BATCH) {
        double r[AO_BATCH];
#pragma unroll
        for (int b = 0; b < AO_BATCH; ++b) {
          const int e = eb + 32 * b;
          if (e < tot) {
            const int v = fdiv_small(e, inv_n);
            r[b] = __ldg(A.src_arena + v * A.vs + soff + (e - v * n));
          }
        }
#pragma unroll
        for (int b = 0; b < AO_BATCH; ++b) {
          const int e = eb + 32 * b;
          if (e < tot) {
            const int v = fdiv_small(e, inv_n);
            s[(e - v * n) * nvp + v] = r[b];
          }
        }
      }
      __syncwarp();
      for (int j = lane; j < tot; j += 32) {
        const int lv = fdiv_small(j, A.inv_nv);
        blk_out[(int64_t)tab[lv] * nq + (j - lv * nv)] = s[lv * nvp + (j - lv * nv)];
      }
    }
    __syncwarp();
  }
}

// Segment length: the longest of 64, 32, 16, 8 voxels whose per-CTA slices fit the target.
int ao_seg(int nvp) {
  int seg = 64;
  while (seg > 8 && AO_WARPS * ao_warp_bytes(seg, nvp) > AO_SMEM_TARGET) seg >>= 1;
  return seg;
}

template <bool GATHER>
dh_status ao_launch(dh_plan* plan, const AoArgs& A, cudaStream_t s) {
  const size_t smem = AO_WARPS * ao_warp_bytes(A.seg, A.nvp);
  static int configured_device = -1;
  if (configured_device != plan->device) {
    const size_t mx = AO_WARPS * ao_warp_bytes(ao_seg(AO_MAX_NQ | 1), AO_MAX_NQ | 1);
    cudaError_t e = cudaFuncSetAttribute(k_aoas<GATHER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_aoas)");
    configured_device = plan->device;
  }
  k_aoas<GATHER><<<plan->n_aunits, AO_WARPS * 32, smem, s>>>(A);
  return cuda_error(cudaGetLastError(), GATHER ? "dh_gather_aoas launch" : "dh_scatter_aoas launch");
}

dh_status ao_check(const dh_plan* plan, const void* blocks, const void* arena, int32_t nq, int32_t aos_halo,
                   const char* who) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (!blocks || !arena) { set_error("%s: the block pointer array and the arena are required", who); return DH_EINVAL; }
  if (nq < 1 || nq > AO_MAX_NQ) { set_error("%s: nq = %d outside [1, %d]", who, nq, AO_MAX_NQ); return DH_EINVAL; }
  if (aos_halo < 0 || aos_halo > 8) { set_error("%s: aos_halo = %d outside [0, 8]", who, aos_halo); return DH_EINVAL; }
  if (((uintptr_t)arena & 7) != 0 || ((uintptr_t)blocks & 7) != 0) {
    set_error("%s: arena and block pointer array must be 8-byte aligned", who);
    return DH_EINVAL;
  }
  if (plan->n_aunits <= 0 || !plan->d_aunits) { set_error("%s: plan has no unit list", who); return DH_EINVAL; }
  return DH_OK;
}

AoArgs ao_args(const dh_plan* plan, int nq, int v0, int nv, int halo) {
  AoArgs A{};
  A.patches = plan->d_patches;
  A.units = plan->d_aunits;
  A.vs = plan->var_stride;
  A.nq = nq;
  A.v0 = v0;
  A.nv = nv;
  A.nvp = nv | 1;
  A.halo = halo;
  A.dim = plan->dim;
  A.seg = ao_seg(A.nvp);
  A.inv_nv = 1.0f / (float)nv;
  return A;
}

}  // namespace

// Quantities v0 .. v0+nv-1 of every interior voxel of the blocks <-> arena
// variables 0 .. nv-1 (validated by the callers).
dh_status aoas_move(dh_plan* plan, bool gather, const double* const* blocks, int nq, int v0, int nv, int halo,
                    double* arena, cudaStream_t s) {
  AoArgs A = ao_args(plan, nq, v0, nv, halo);
  if (gather) {
    A.src_blocks = blocks;
    A.dst_arena = arena;
    return ao_launch<true>(plan, A, s);
  }
  A.dst_blocks = const_cast<double* const*>(blocks);
  A.src_arena = arena;
  return ao_launch<false>(plan, A, s);
}

// Unit list of the plan: up to AO_UNIT_VOXELS voxels of one patch per CTA,
// units of the largest p first.
std::vector<int2> aoas_units(const dh_patch* patches, int K, int dim) {
  std::vector<int> idx(K);
  for (int k = 0; k < K; ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return patches[a].p > patches[b].p; });
  std::vector<int2> units;
  for (int k : idx) {
    const int p = patches[k].p, nvox = dim == 3 ? p * p * p : p * p;
    for (int i = 0; i < nvox; i += AO_UNIT_VOXELS) units.push_back(make_int2(k, i));
  }
  return units;
}

}  // namespace dh

using namespace dh;

extern "C" {

dh_status dh_gather_aoas(dh_plan* plan, const double* const* aos_patches_dev, int32_t nq, int32_t aos_halo,
                         double* arena, void* stream) {
  dh_status st = ao_check(plan, aos_patches_dev, arena, nq, aos_halo, "dh_gather_aoas");
  if (st != DH_OK) return st;
  return aoas_move(plan, true, aos_patches_dev, nq, 0, nq, aos_halo, arena, (cudaStream_t)stream);
}

dh_status dh_scatter_aoas(dh_plan* plan, const double* arena, double* const* aos_patches_dev, int32_t nq,
                          int32_t aos_halo, void* stream) {
  dh_status st = ao_check(plan, aos_patches_dev, arena, nq, aos_halo, "dh_scatter_aoas");
  if (st != DH_OK) return st;
  return aoas_move(plan, false, aos_patches_dev, nq, 0, nq, aos_halo, const_cast<double*>(arena),
                   (cudaStream_t)stream);
}

}  // extern "C"
