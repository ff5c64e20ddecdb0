// darts_device.cuh -- device-side building blocks of libdarts (sm_103a).
//
// Philox4x32-10 (Salmon et al., SC'11), the uniform mapping, the HG phase
// function, the orthonormal frame of Duff et al. (JCGT 2017) and the few
// elementary functions the path kernels need at FP32 accuracy without the
// cost of the full-range library routines.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#error "CUDA translation units only"
#endif

namespace darts {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInv4Pi = 0.0795774715459476678844f;

struct U4 {
  uint32_t x, y, z, w;
};

// Philox4x32-10: ten rounds of two 32x32 -> 64-bit multiplies, Weyl key bumps.
// UNROLL: rounds per iteration of the round loop in the generated code (the
// same ten rounds and the same result for every value; kernels short of
// instruction cache take a shorter body).
template <int UNROLL = 10>
__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                      uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll UNROLL
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0, p1 = uint64_t(0xCD9E8D57u) * c2;
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Two Philox4x32-10 blocks whose counters differ only in the last word,
// advanced in one loop: two independent chains in one loop body (the same
// results as two calls).
template <int UNROLL = 10>
__host__ __device__ __forceinline__ void philox4x32_10_pair(uint32_t c0, uint32_t c1, uint32_t c2,
                                                           uint32_t c3a, uint32_t c3b, uint32_t k0,
                                                           uint32_t k1, U4* a, U4* b) {
  uint32_t a0 = c0, a1 = c1, a2 = c2, a3 = c3a;
  uint32_t b0 = c0, b1 = c1, b2 = c2, b3 = c3b;
#pragma unroll UNROLL
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t ha0 = __umulhi(0xD2511F53u, a0), la0 = 0xD2511F53u * a0;
    const uint32_t ha1 = __umulhi(0xCD9E8D57u, a2), la1 = 0xCD9E8D57u * a2;
    const uint32_t hb0 = __umulhi(0xD2511F53u, b0), lb0 = 0xD2511F53u * b0;
    const uint32_t hb1 = __umulhi(0xCD9E8D57u, b2), lb1 = 0xCD9E8D57u * b2;
#else
    const uint64_t pa0 = uint64_t(0xD2511F53u) * a0, pa1 = uint64_t(0xCD9E8D57u) * a2;
    const uint64_t pb0 = uint64_t(0xD2511F53u) * b0, pb1 = uint64_t(0xCD9E8D57u) * b2;
    const uint32_t ha0 = uint32_t(pa0 >> 32), la0 = uint32_t(pa0), ha1 = uint32_t(pa1 >> 32), la1 = uint32_t(pa1);
    const uint32_t hb0 = uint32_t(pb0 >> 32), lb0 = uint32_t(pb0), hb1 = uint32_t(pb1 >> 32), lb1 = uint32_t(pb1);
#endif
    const uint32_t na0 = ha1 ^ a1 ^ k0, na2 = ha0 ^ a3 ^ k1;
    const uint32_t nb0 = hb1 ^ b1 ^ k0, nb2 = hb0 ^ b3 ^ k1;
    a0 = na0; a1 = la1; a2 = na2; a3 = la0;
    b0 = nb0; b1 = lb1; b2 = nb2; b3 = lb0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  *a = U4{a0, a1, a2, a3};
  *b = U4{b0, b1, b2, b3};
}

// Counter layout shared by every kernel: (path lo, path hi, stream,
// vertex << 8 | group); group 0 = distance step, group 1 = direction and
// control vertex; vertex 0xFFFFFE = per sensor element.
constexpr uint32_t kVertexElement = 0xFFFFFEu;

// 24 random bits -> [0, 1): exact in FP32.
__host__ __device__ __forceinline__ float u01(uint32_t x) {
  return float(x >> 8) * 5.9604644775390625e-08f;
}

// log(1 - x) for x in [0, 1).  For x < 1/4 through log(1-x) = -2 atanh(x/(2-x))
// and the odd series of atanh (|z| <= 1/7: six terms reach ~1e-9 relative);
// above that 1 - x is exact enough for the hardware logarithm.
__device__ __forceinline__ float log1m(float x) {
  const float z = __fdividef(x, 2.0f - x);
  const float z2 = z * z;
  float s = fmaf(z2, 1.0f / 11.0f, 1.0f / 9.0f);
  s = fmaf(z2, s, 1.0f / 7.0f);
  s = fmaf(z2, s, 1.0f / 5.0f);
  s = fmaf(z2, s, 1.0f / 3.0f);
  s = fmaf(z2, s, 1.0f);
  const float small = -2.0f * z * s;
  const float large = __logf(1.0f - x);
  return x < 0.25f ? small : large;
}

// exp(x) - 1 for x <= 0: Taylor series (Horner) for x > -1/2, else exp - 1.
__device__ __forceinline__ float expm1_neg(float x) {
  float s = fmaf(x, 1.0f / 40320.0f, 1.0f / 5040.0f);
  s = fmaf(x, s, 1.0f / 720.0f);
  s = fmaf(x, s, 1.0f / 120.0f);
  s = fmaf(x, s, 1.0f / 24.0f);
  s = fmaf(x, s, 1.0f / 6.0f);
  s = fmaf(x, s, 0.5f);
  s = fmaf(x, s, 1.0f);
  const float small = x * s;
  const float large = __expf(x) - 1.0f;
  return x > -0.5f ? small : large;
}

// Henyey-Greenstein density per steradian: a * (b - c mu)^(-3/2) with
// a = (1 - g^2)/(4 pi), b = 1 + g^2, c = 2 g.
__device__ __forceinline__ float hg_eval(float mu, float a, float b, float c) {
  const float r = rsqrtf(fmaf(-c, mu, b));
  return a * r * r * r;
}

// HG inversion written without the cancellation of the textbook form at small
// |g|: with h = 1 - 2 xi and e = 1 - g h,
// mu = (-h + g (3 + h^2)/2 - g^2 h + g^3 (h^2 - 1)/2) / e^2   (exact identity).
__device__ __forceinline__ float hg_sample(float g, float xi) {
  const float h = fmaf(-2.0f, xi, 1.0f);
  const float h2 = h * h;
  const float e = fmaf(-g, h, 1.0f);
  float num = fmaf(0.5f * g * g * g, h2 - 1.0f, -g * g * h);
  num = fmaf(0.5f * g, 3.0f + h2, num) - h;
  const float mu = __fdividef(num, e * e);
  return fminf(1.0f, fmaxf(-1.0f, mu));
}

// sin(theta) of the HG sample of the same xi, free of the cancellation of
// sqrt(1 - mu^2) near mu = +-1 (strongly forward or backward g): with
// e = 1 - g + 2 g xi,
//   1 - mu = 2 (1 - g)^2 (1 - xi) (1 + g xi) / e^2,
//   1 + mu = 2 (1 + g)^2 xi (1 - g + g xi) / e^2,
// so sin = 2 (1 - g^2) sqrt(xi (1 - xi) (1 + g xi) (1 - g + g xi)) / e^2,
// a product of positive factors.
__device__ __forceinline__ float hg_sin(float g, float xi) {
  const float e = fmaf(2.0f * g, xi, 1.0f - g);
  const float q = xi * (1.0f - xi) * fmaf(g, xi, 1.0f) * fmaf(g, xi, 1.0f - g);
  return fminf(1.0f, __fdividef(2.0f * (1.0f - g * g) * sqrtf(q), e * e));
}

// cos/sin of 2 pi u for u in [0, 1), with the argument kept in [-pi, pi).
__device__ __forceinline__ void sincos_2pi(float u, float* s, float* c) {
  float ss, cc;
  __sincosf(kTwoPi * (u - 0.5f), &ss, &cc);
  *s = -ss;
  *c = -cc;
}

// dir = mu n + sin_t (cos phi b1 + sin phi b2), frame of Duff et al.; the
// caller passes sin_t = sqrt(1 - mu^2) in a form accurate near mu = +-1.
__device__ __forceinline__ void frame_dir(float nx, float ny, float nz, float mu, float sin_t,
                                          float sphi, float cphi, float* ox, float* oy, float* oz) {
  const float sign = nz >= 0.0f ? 1.0f : -1.0f;
  const float a = -__fdividef(1.0f, sign + nz);  // |sign + nz| >= 1
  const float b = nx * ny * a;
  const float b1x = fmaf(sign * nx * nx, a, 1.0f), b1y = sign * b, b1z = -sign * nx;
  const float b2x = b, b2y = fmaf(ny * ny, a, sign), b2z = -ny;
  const float p = sin_t * cphi, q = sin_t * sphi;
  *ox = fmaf(mu, nx, fmaf(p, b1x, q * b2x));
  *oy = fmaf(mu, ny, fmaf(p, b1y, q * b2y));
  *oz = fmaf(mu, nz, fmaf(p, b1z, q * b2z));
}

}  // namespace darts
