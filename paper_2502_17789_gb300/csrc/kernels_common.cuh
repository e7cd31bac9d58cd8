// Device helpers shared by the libidg kernels.
#pragma once

#include <cuda_runtime.h>

#include "idg_internal.h"

namespace idg {

constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr double kTwoPi = 6.28318530717958647692;
// adding and subtracting 1.5 * 2^23 rounds a float with |x| < 2^22 to the
// nearest integer (round-half-even) using two plain adds
constexpr float kRoundMagic = 12582912.0f;

// Packed two-lane FMA (sm_100+ f32x2): d = a * b + c per lane.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

__device__ __forceinline__ float round_nearest(float x) {
  return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic);
}

struct cf {
  float re, im;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cmulc(cf a, cf b) {  // conj(a) * b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
__device__ __forceinline__ cf cadd(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }

// 2x2 complex Jones matrix, row-major [00 01; 10 11].
struct Jones {
  cf m[4];
};

// C = A * B
__device__ __forceinline__ Jones jmul(const Jones& A, const Jones& B) {
  Jones C;
  C.m[0] = cadd(cmul(A.m[0], B.m[0]), cmul(A.m[1], B.m[2]));
  C.m[1] = cadd(cmul(A.m[0], B.m[1]), cmul(A.m[1], B.m[3]));
  C.m[2] = cadd(cmul(A.m[2], B.m[0]), cmul(A.m[3], B.m[2]));
  C.m[3] = cadd(cmul(A.m[2], B.m[1]), cmul(A.m[3], B.m[3]));
  return C;
}
// C = A^H * B
__device__ __forceinline__ Jones jmul_ah(const Jones& A, const Jones& B) {
  Jones C;
  C.m[0] = cadd(cmulc(A.m[0], B.m[0]), cmulc(A.m[2], B.m[2]));
  C.m[1] = cadd(cmulc(A.m[0], B.m[1]), cmulc(A.m[2], B.m[3]));
  C.m[2] = cadd(cmulc(A.m[1], B.m[0]), cmulc(A.m[3], B.m[2]));
  C.m[3] = cadd(cmulc(A.m[1], B.m[1]), cmulc(A.m[3], B.m[3]));
  return C;
}
// C = A * B^H
__device__ __forceinline__ Jones jmul_bh(const Jones& A, const Jones& B) {
  auto mc = [](cf a, cf b) {  // a * conj(b)
    return cf{a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
  };
  Jones C;
  C.m[0] = cadd(mc(A.m[0], B.m[0]), mc(A.m[1], B.m[1]));
  C.m[1] = cadd(mc(A.m[0], B.m[2]), mc(A.m[1], B.m[3]));
  C.m[2] = cadd(mc(A.m[2], B.m[0]), mc(A.m[3], B.m[1]));
  C.m[3] = cadd(mc(A.m[2], B.m[2]), mc(A.m[3], B.m[3]));
  return C;
}

// Bilinear interpolation weights of pixel index i on `nodes` A-term samples:
// pixel i sits at fractional node (nodes - 1) * i / L.
struct NodeWeight {
  int a;
  float f;
};
__device__ __forceinline__ NodeWeight node_weight(int i, int nodes, int L) {
  const int num = (nodes - 1) * i;
  int a = num / L;
  float f = float(num - a * L) / float(L);
  if (a > nodes - 2) {
    f += float(a - (nodes - 2));
    a = nodes - 2;
  }
  return {a, f};
}

// Interpolated Jones matrix from node samples A[a_m][a_l][4] held in shared memory.
__device__ __forceinline__ Jones interp_jones(const float2* A, int nodes, NodeWeight wx, NodeWeight wy) {
  const float2* r0 = A + (size_t(wy.a) * nodes + wx.a) * 4;
  const float2* r1 = r0 + size_t(nodes) * 4;
  const float w00 = (1.f - wx.f) * (1.f - wy.f), w01 = wx.f * (1.f - wy.f);
  const float w10 = (1.f - wx.f) * wy.f, w11 = wx.f * wy.f;
  Jones J;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 a = r0[e], b = r0[4 + e], c = r1[e], d = r1[4 + e];
    J.m[e].re = w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x;
    J.m[e].im = w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y;
  }
  return J;
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

}  // namespace idg
