// Small FP32 MLP (3 -> 32 tanh -> 32 tanh -> 1) that seeds the SRHD pressure
// Newton iteration.  Weight vector layout (floats), shared by inference and
// training:
//   W1[32][3] (0..95), b1[32] (96..127), W2[32][32] (128..1151), b2[32]
//   (1152..1183), W3[32] (1184..1215), b3 (1216), then the z-score
//   statistics of the inputs: mean[3] (1217..1219), std[3] (1220..1222), pad.
// Inputs: x = (|S|/E, D/E, ln(E/D)) with E = tau + D; target y = ln(p/E).
// tanh is CUDA's tanhf.
#pragma once

#include "dh_internal.cuh"

namespace dh {

constexpr int MLP_NW = 1217;       // trainable parameters
constexpr int MLP_LEN = 1224;      // parameters + statistics + pad
constexpr int MLP_W1 = 0, MLP_B1 = 96, MLP_W2 = 128, MLP_B2 = 1152, MLP_W3 = 1184, MLP_B3 = 1216;
constexpr int MLP_MEAN = 1217, MLP_STD = 1220;

// Invariants of a conserved SRHD state in FP64.
__device__ __forceinline__ void srhd_invariants(const double* q, double* x) {
  const double D = q[0], E = q[4] + q[0];
  const double S = sqrt(fma(q[1], q[1], fma(q[2], q[2], q[3] * q[3])));
  x[0] = S / E;
  x[1] = D / E;
  x[2] = log(E / D);
}

// z-scored FP32 input from FP64 invariants (statistics in the weight vector).
__device__ __forceinline__ void mlp_normalize(const float* w, const double* xd, float* x) {
#pragma unroll
  for (int j = 0; j < 3; ++j) x[j] = (float)((xd[j] - (double)w[MLP_MEAN + j]) / (double)w[MLP_STD + j]);
}

// Conversions between FP64 and FP32 on the integer pipes.  On this GPU the hardware
// conversions run on the FP64 pipe at the FP64 rate (measured: a double -> float -> double
// round trip costs as much as two FMAs and does not overlap with FMAs), so the FP32 seed
// paths convert with bit operations.  Both give IEEE round-to-nearest-even results, so they
// are bitwise the hardware conversions (tested over all exponent ranges); operands whose
// float result would be zero, subnormal, infinite or NaN take the hardware path (a call, so
// that it never executes on the common path).
static __device__ __noinline__ float f32_rn_slow(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double f64_of_f32_slow(float f) { return (double)f; }

// double -> float, round to nearest even: the 52-bit fraction keeps its top 23 bits and rounds
// on the remaining 29 (a carry out of the fraction moves into the exponent, and past the largest
// finite float into infinity, as IEEE rounding does).
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // float biased exponent (1023 - 127 = 896)
  if (e < 1 || e > 254) return f32_rn_slow(x);
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem + (frac & 1u)) > 0x10000000u ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | (((unsigned)e << 23) + frac + up));
}

// float -> double (exact): exponent rebiased, fraction shifted into place.
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return f64_of_f32_slow(f);
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// z-scored FP32 network input formed in FP32 from D, E = tau + D and |S|
// (the seed path of con2prim: the network is FP32, so its inputs need no FP64
// divides or logarithm on the FP64 pipe).
__device__ __forceinline__ void mlp_inputs_f32(const float* w, double D, double E, double S, float* x) {
  const float rE = 1.0f / f32_rn(E);
  const float dE = f32_rn(D) * rE;
  const float raw[3] = {f32_rn(S) * rE, dE, -logf(dE)};  // |S|/E, D/E, ln(E/D)
#pragma unroll
  for (int j = 0; j < 3; ++j) x[j] = (raw[j] - w[MLP_MEAN + j]) / w[MLP_STD + j];
}

// Forward pass; h1/h2 receive the hidden activations.  w must be 16-byte
// aligned: the rows of W2 are read as float4.
__device__ __forceinline__ float mlp_forward(const float* w, const float* x, float* h1, float* h2) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float s = w[MLP_B1 + i];
#pragma unroll
    for (int j = 0; j < 3; ++j) s = fmaf(w[MLP_W1 + 3 * i + j], x[j], s);
    h1[i] = tanhf(s);
  }
  float y = w[MLP_B3];
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    float s = w[MLP_B2 + i];
    const float4* row = reinterpret_cast<const float4*>(w + MLP_W2 + 32 * i);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 r = row[j];
      s = fmaf(r.x, h1[4 * j], s);
      s = fmaf(r.y, h1[4 * j + 1], s);
      s = fmaf(r.z, h1[4 * j + 2], s);
      s = fmaf(r.w, h1[4 * j + 3], s);
    }
    h2[i] = tanhf(s);
    y = fmaf(w[MLP_W3 + i], h2[i], y);
  }
  return y;
}

}  // namespace dh
