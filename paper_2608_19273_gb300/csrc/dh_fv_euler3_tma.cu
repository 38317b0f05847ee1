// Instantiation of the TMA-staged finite-volume stage kernels (3D Euler) and the tensor
// maps they read: per arena level of back-to-back patches, 5-D maps (x, y, z, patch,
// variable) over the stage input with the boxes of one z-plane of a 16x16 or 32x8 column
// and of its ring strips.
#include <cstring>

#include "dh_fv_stage.cuh"

namespace dh {
namespace fvtma {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

dh_status encode_level(const double* base, int p, int K, int nv, int64_t var_stride, int bx, int by, Map* out) {
  static_assert(sizeof(Map) == sizeof(CUtensorMap), "tensor map size");
  EncodeTiledFn fn = encode_fn();
  if (!fn) { set_error("k_fv_stage: cuTensorMapEncodeTiled is unavailable"); return DH_EUNSUPPORTED; }
  const uint64_t pp = (uint64_t)p;
  const cuuint64_t dims[5] = {pp, pp, pp, (cuuint64_t)K, (cuuint64_t)nv};
  const cuuint64_t strides[4] = {pp * 8, pp * pp * 8, pp * pp * pp * 8, (cuuint64_t)var_stride * 8};
  const cuuint32_t box[5] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1, (cuuint32_t)nv};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUtensorMap m;
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("k_fv_stage: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DH_ECUDA;
  }
  std::memcpy(out, &m, sizeof(m));
  return DH_OK;
}

}  // namespace fvtma

template <int BASE, int WM, bool T32>
static dh_status tma_launch(dh_plan* plan, const FvArgs& A, cudaStream_t stream, const FvMaps<true>& M) {
  return launch_var<PdeEuler3, 64 | BASE | (WM << 2) | (T32 ? 32 : 0)>(plan, A, stream, M);
}

template <int BASE, bool T32>
static dh_status tma_launch_wm(dh_plan* plan, const FvArgs& A, int wm, cudaStream_t stream, const FvMaps<true>& M) {
  switch (wm) {
    case 0: return tma_launch<BASE, 0, T32>(plan, A, stream, M);
    case 1: return tma_launch<BASE, 1, T32>(plan, A, stream, M);
    case 2: return tma_launch<BASE, 2, T32>(plan, A, stream, M);
    default: return tma_launch<BASE, 3, T32>(plan, A, stream, M);
  }
}

dh_status fv_launch_euler3_tma(dh_plan* plan, const FvArgs& A, int wm, cudaStream_t stream) {
  const int v = plan->fv_var, tile = (v >> 3) & 3;
  if (!plan->tma_ok || plan->coupled || plan->n_lvl > FV_TMA_LEVELS || !(v & 2) || (v & 4) || tile > 1) {
    set_error("k_fv_stage: the TMA-staged variant needs levels of back-to-back patches (no coupled levels), the "
              "register cap, one CTA per tile and tile shape 0 or 1");
    return DH_EUNSUPPORTED;
  }
  FvMaps<true> M;
  std::memset(&M, 0, sizeof(M));
  static const int shape[FVB_N][2] = {{16, 16}, {2, 16}, {16, 1}, {32, 8}, {2, 8}, {32, 1}};
  for (int l = 0; l < plan->n_lvl; ++l) {
    const int p = plan->lvl_p[l];
    for (int b = 0; b < FVB_N; ++b) {
      if (shape[b][0] > p || shape[b][1] > p) continue;  // a column shape this level's patches cannot hold
      dh_status st = fvtma::encode_level(A.qs + plan->lvl_off[l], p, plan->lvl_K[l], plan->nq, plan->var_stride,
                                         shape[b][0], shape[b][1], &M.m[l][b]);
      if (st != DH_OK) return st;
    }
  }
  const bool t32 = tile == 1;
  if (v & 1) return t32 ? tma_launch_wm<3, true>(plan, A, wm, stream, M) : tma_launch_wm<3, false>(plan, A, wm, stream, M);
  return t32 ? tma_launch_wm<2, true>(plan, A, wm, stream, M) : tma_launch_wm<2, false>(plan, A, wm, stream, M);
}

}  // namespace dh
