// Autotuner: picks, per plan (PDE x patch mix x GPU), the fastest compiled
// variant of the stage kernel by timing every candidate with CUDA events on
// the caller's own buffers, and remembers the choice in a small JSON-lines
// cache file.
//
// Candidates
//   FV stage: halo ring before / after the mid-plane barrier
//             x register cap (1 or 2 CTAs per SM)
//             x grid: one CTA per tile, or persistent (SMs x resident CTAs taking tiles
//               from an atomic queue)
//             x tile shape: 16x16 columns (256 threads per column), 32x8 columns for
//               32^3 patches, 8x8 columns (64 threads) grouped four to a CTA (up to
//               four patches per CTA) -- tile sets that give the same list as the
//               first one are skipped -- or one 8x8 column per 64-thread CTA
//             x z-march of whole patches or chunks of <= 16 planes
//             x loads: plain (L2-prefetched) or, for 3D Euler, TMA tensor copies of every
//               column plane and its ring strips into a double-buffered shared ring
//   second-order FV stage: z-march of whole patches or in chunks of <= 16 planes, or the 8x8x4
//             tile kernel;
//   FD stage: register cap (1 or 2 CTAs per SM) x staging (plain loads or TMA);
//             with TMA staging of one group (systems of <= 5 variables) also
//             caps for 3 and 4 CTAs per SM
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "dh_internal.cuh"

namespace dh {

static std::string tune_key(const dh_plan* plan, int scheme) {
  std::map<int, int> mix;
  for (const dh_patch& p : plan->h_patches) mix[p.p]++;
  cudaDeviceProp prop;
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&prop, plan->device) == cudaSuccess) dev = prop.name;
  std::string k = dev + "|pde=" + std::to_string(plan->pde) + "|scheme=" + std::to_string(scheme) +
                  "|dim=" + std::to_string(plan->dim) + "|mix=";
  for (auto& kv : mix) k += std::to_string(kv.first) + "x" + std::to_string(kv.second) + ",";
  return k;
}

// Looks for `"key": "<key>"` in the cache and reads the three integers after it.
static bool cache_lookup(const char* path, const std::string& key, int* fv_var, int* fv_zs, int* fd_var) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[4096];
  bool found = false;
  const std::string needle = "\"key\": \"" + key + "\"";
  while (fgets(line, sizeof(line), f)) {
    if (!strstr(line, needle.c_str())) continue;
    const char* a = strstr(line, "\"fv_var\": ");
    const char* b = strstr(line, "\"fv_zs\": ");
    const char* c = strstr(line, "\"fd_var\": ");
    if (a && b && c && sscanf(a, "\"fv_var\": %d", fv_var) == 1 && sscanf(b, "\"fv_zs\": %d", fv_zs) == 1 &&
        sscanf(c, "\"fd_var\": %d", fd_var) == 1)
      found = true;  // the last matching line wins
  }
  fclose(f);
  return found;
}

static bool fv_tma_ok(const dh_plan* plan) {
  return plan->pde == DH_PDE_EULER3D && plan->tma_ok && !plan->coupled && plan->n_lvl <= 8;
}

// The candidates of a plan (see the top of this file), in the order the timings are reported.
struct Cand {
  int v, z, f;
};

static int tune_candidates(const dh_plan* plan, int scheme, Cand* cands) {
  int nc = 0;
  if (scheme == 2) {
    // second-order FV: z-march of whole patches, z-march in chunks of <= 16 planes, 8x8x4 tiles
    for (int v = 0; v < 3; ++v) cands[nc++] = {v, plan->fv_zs, plan->fd_var};
    return nc;
  }
  if (scheme == 0) {
    // a tile set is a candidate only where it changes the work list
    bool has32 = false, has16 = false;
    for (const dh_patch& p : plan->h_patches) {
      has32 |= p.p % 32 == 0;
      has16 |= p.p % 16 == 0;
    }
    // (the persistent grid and the 32x8 columns come with the register cap, fv_var bit 1)
    for (int tile = 0; tile < 3; ++tile) {
      if ((tile == 1 && !has32) || (tile == 2 && !has16)) continue;
      for (int pers = 0; pers < 2; ++pers)
        for (int zz = 0; zz < 2; ++zz)
          for (int vv = 0; vv < 4; ++vv) {
            if ((pers || tile == 1) && !(vv & 2)) continue;
            cands[nc++] = {vv | (pers << 2) | (tile << 3), zz, plan->fd_var};
          }
    }
    // one 8x8 column per 64-thread CTA (every kernel form)
    for (int zz = 0; zz < 2; ++zz)
      for (int vv = 0; vv < 4; ++vv) cands[nc++] = {vv | (3 << 3), zz, plan->fd_var};
    // TMA staging of the column planes (3D Euler), with the register cap, one CTA per tile
    if (fv_tma_ok(plan))
      for (int tile = 0; tile < 2; ++tile) {
        if (tile == 1 && !has32) continue;
        for (int zz = 0; zz < 2; ++zz)
          for (int vv = 2; vv < 4; ++vv) cands[nc++] = {32 | vv | (tile << 3), zz, plan->fd_var};
      }
  } else {
    cands[nc++] = {plan->fv_var, plan->fv_zs, 0};
    cands[nc++] = {plan->fv_var, plan->fv_zs, 2};
    if (plan->tma_ok) {
      cands[nc++] = {plan->fv_var, plan->fv_zs, 4};
      cands[nc++] = {plan->fv_var, plan->fv_zs, 6};
      if (plan->pde != DH_PDE_GW59) {
        cands[nc++] = {plan->fv_var, plan->fv_zs, 12};
        cands[nc++] = {plan->fv_var, plan->fv_zs, 20};
      }
    }
  }
  return nc;
}

// Look the choice up in the cache, else time `launch` for every candidate (one warm-up, then
// `reps` timed calls with CUDA events on s), keep the fastest and append it to the cache.
template <class Launch>
static dh_status tune_run(dh_plan* plan, int scheme, const std::string& key, int reps, const char* cache_path,
                          int32_t* choice_out, float* times_out, cudaStream_t s, Launch launch) {
  if (plan->fv_generic) {
    // patch sizes that are not all multiples of 8: one FV kernel (no variants); FD and MUSCL
    // refuse such plans
    if (scheme != 0) {
      set_error("dh_autotune: FD and MUSCL stages need patch sizes that are multiples of 8");
      return DH_EUNSUPPORTED;
    }
    if (choice_out) { choice_out[0] = plan->fv_var; choice_out[1] = plan->fv_zs; choice_out[2] = plan->fd_var; choice_out[3] = 0; }
    return DH_OK;
  }
  if (!cache_path) cache_path = std::getenv("DH_TUNE_CACHE");  // NULL and unset: no cache
  int v = 0, z = 0, f = 0;
  if (cache_path && cache_lookup(cache_path, key, &v, &z, &f)) {
    dh_status st = scheme == 2 ? dh_plan_set_variant_muscl(plan, v) : dh_plan_set_variant(plan, v, z, f);
    if (st == DH_OK && choice_out) { choice_out[0] = v; choice_out[1] = z; choice_out[2] = f; choice_out[3] = 1; }
    return st;
  }
  Cand cands[DH_TUNE_MAX_CANDIDATES];
  const int nc = tune_candidates(plan, scheme, cands);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("dh_autotune: cudaEventCreate failed");
    return DH_ECUDA;
  }
  float best = 1e30f;
  int bi = 0;
  dh_status st = DH_OK;
  auto apply = [&](const Cand& c) {
    if (scheme == 2) {
      plan->fv2_var = c.v;
    } else {
      plan->fv_var = c.v;
      plan->fv_zs = c.z;
      plan->fd_var = c.f;
    }
  };
  for (int i = 0; i < nc && st == DH_OK; ++i) {
    apply(cands[i]);
    st = launch();  // warm-up (also sets the kernel's shared-memory attribute)
    if (st != DH_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == DH_OK; ++r) st = launch();
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) { st = cuda_error(ce, "dh_autotune"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (times_out) times_out[i] = ms;
    if (ms < best) { best = ms; bi = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DH_OK) return st;
  apply(cands[bi]);
  if (choice_out) { choice_out[0] = cands[bi].v; choice_out[1] = cands[bi].z; choice_out[2] = cands[bi].f; choice_out[3] = 0; }
  if (cache_path) {
    FILE* fo = fopen(cache_path, "a");
    if (fo) {
      fprintf(fo, "{\"key\": \"%s\", \"fv_var\": %d, \"fv_zs\": %d, \"fd_var\": %d, \"ms\": %.6f, \"candidates\": %d}\n",
              key.c_str(), cands[bi].v, cands[bi].z, cands[bi].f, best, nc);
      fclose(fo);
    }
  }
  return DH_OK;
}

}  // namespace dh

using namespace dh;

extern "C" {

dh_status dh_plan_set_variant(dh_plan* plan, int32_t fv_var, int32_t fv_zs, int32_t fd_var) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  const bool fd_ok = fd_var == 0 || fd_var == 2 || fd_var == 4 || fd_var == 6 ||
                     ((fd_var == 12 || fd_var == 20) && plan->pde != DH_PDE_GW59);
  const int tile = (fv_var >> 3) & 3;
  const bool fv_ok = fv_var >= 0 && fv_var <= 63 &&
                     (!((fv_var & 4) || tile == 1 || (fv_var & 32)) || (fv_var & 2)) &&
                     (!(fv_var & 32) || (!(fv_var & 4) && tile <= 1)) && (tile != 3 || !(fv_var & 4));
  if (!fv_ok || fv_zs < 0 || fv_zs > 1 || !fd_ok) {
    set_error("dh_plan_set_variant: fv_var in 0..63 (bit 2, tile set 1 and bit 5 need bit 1; bit 5 excludes bit 2 "
              "and tile sets 2, 3; tile set 3 excludes bit 2), fv_zs in 0..1, fd_var in {0, 2, 4, 6} (and 12, 20 "
              "except for GW59)");
    return DH_EINVAL;
  }
  if ((fv_var & 32) && !fv_tma_ok(plan)) {
    set_error("dh_plan_set_variant: the TMA-staged FV stage needs 3D Euler on levels of back-to-back patches whose "
              "neighbours stay in the level (at most 8 levels, no coupled levels)");
    return DH_EUNSUPPORTED;
  }
  if ((fd_var & 4) && !plan->tma_ok) {
    set_error("dh_plan_set_variant: TMA staging needs levels of back-to-back patches whose neighbours stay in the level");
    return DH_EUNSUPPORTED;
  }
  plan->fv_var = fv_var;
  plan->fv_zs = fv_zs;
  plan->fd_var = fd_var;
  return DH_OK;
}

dh_status dh_plan_set_variant_muscl(dh_plan* plan, int32_t fv2_var) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (fv2_var < 0 || fv2_var > 2) { set_error("dh_plan_set_variant_muscl: fv2_var in 0..2"); return DH_EINVAL; }
  plan->fv2_var = fv2_var;
  return DH_OK;
}

dh_status dh_autotune(dh_plan* plan, int32_t scheme, const double* qs, double* out, const double* mat,
                      const double* dt_dev, int32_t reps, const char* cache_path, int32_t* choice_out,
                      float* times_out, void* stream) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (scheme < 0 || scheme > 2) { set_error("dh_autotune: scheme must be 0 (FV), 1 (FD) or 2 (FV, MUSCL)"); return DH_EINVAL; }
  if (!qs || !out || !dt_dev || reps < 1 || reps > 1000) { set_error("dh_autotune: bad arguments"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  auto launch = [&]() {
    return scheme == 0   ? patch_update_fv(plan, qs, nullptr, out, nullptr, mat, dt_dev, 0, 1, 1, 0, nullptr, s)
           : scheme == 2 ? patch_update_fv_muscl(plan, qs, nullptr, out, nullptr, mat, dt_dev, 0, 1, 1, 0, nullptr, s)
                         : patch_update_fd_ko(plan, qs, nullptr, out, nullptr, mat, dt_dev, 0, 1, 1, 0, 0.1, nullptr, s);
  };
  return tune_run(plan, scheme, tune_key(plan, scheme), reps, cache_path, choice_out, times_out, s, launch);
}

dh_status dh_autotune_steps(dh_plan* plan, int32_t scheme, int32_t rk, int32_t n_steps, double* q, double* u1,
                            double* u2, double* acc, const double* mat, double* dt_dev, double* lam_dev, double cfl,
                            double sigma_ko, int32_t reps, const char* cache_path, int32_t* choice_out,
                            float* times_out, void* stream) {
  if (!plan) { set_error("plan is NULL"); return DH_EINVAL; }
  if (scheme < 0 || scheme > 2) {
    set_error("dh_autotune_steps: scheme must be 0 (FV), 1 (FD) or 2 (FV, MUSCL)");
    return DH_EINVAL;
  }
  if (n_steps < 1 || n_steps > 1000 || reps < 1 || reps > 1000) {
    set_error("dh_autotune_steps: n_steps and reps must lie in [1, 1000]");
    return DH_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto launch = [&]() { return rk_steps(plan, scheme, rk, n_steps, q, u1, u2, acc, mat, dt_dev, lam_dev, cfl, sigma_ko, s); };
  // the buffers are checked by the first launch (as dh_rk_step checks them)
  const std::string key = tune_key(plan, scheme) + "|steps=rk" + std::to_string(rk) + (acc ? "+acc" : "") +
                          (cfl > 0 ? "+cfl" : "");
  return tune_run(plan, scheme, key, reps, cache_path, choice_out, times_out, s, launch);
}

}  // extern "C"
