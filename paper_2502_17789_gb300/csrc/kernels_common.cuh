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

// packed f32x2 multiply, round to nearest
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
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

// Same interpolation reading the node samples from global memory through the
// read-only cache (16-byte loads: a node's 4 entries are 2 float4).
__device__ __forceinline__ Jones interp_jones_ldg(const float2* A, int nodes, NodeWeight wx, NodeWeight wy) {
  const float4* r0 = reinterpret_cast<const float4*>(A + (size_t(wy.a) * nodes + wx.a) * 4);
  const float4* r1 = r0 + size_t(nodes) * 2;
  const float w00 = (1.f - wx.f) * (1.f - wy.f), w01 = wx.f * (1.f - wy.f);
  const float w10 = (1.f - wx.f) * wy.f, w11 = wx.f * wy.f;
  Jones J;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float4 a = __ldg(r0 + h), b = __ldg(r0 + 2 + h), c = __ldg(r1 + h), d = __ldg(r1 + 2 + h);
    J.m[2 * h].re = w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x;
    J.m[2 * h].im = w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y;
    J.m[2 * h + 1].re = w00 * a.z + w01 * b.z + w10 * c.z + w11 * d.z;
    J.m[2 * h + 1].im = w00 * a.w + w01 * b.w + w10 * c.w + w11 * d.w;
  }
  return J;
}

// Diagonal entries (XX, YY) of the interpolated Jones matrix, for A-terms
// flagged diagonal (off-diagonal node samples all zero).
struct JonesDiag {
  cf d0, d1;
};
__device__ __forceinline__ JonesDiag interp_diag(const float2* A, int nodes, NodeWeight wx, NodeWeight wy) {
  const float2* r0 = A + (size_t(wy.a) * nodes + wx.a) * 4;
  const float2* r1 = r0 + size_t(nodes) * 4;
  const float w00 = (1.f - wx.f) * (1.f - wy.f), w01 = wx.f * (1.f - wy.f);
  const float w10 = (1.f - wx.f) * wy.f, w11 = wx.f * wy.f;
  JonesDiag J;
  {
    const float2 a = r0[0], b = r0[4], c = r1[0], d = r1[4];
    J.d0 = {w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y};
  }
  {
    const float2 a = r0[3], b = r0[7], c = r1[3], d = r1[7];
    J.d1 = {w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y};
  }
  return J;
}
__device__ __forceinline__ JonesDiag interp_diag_ldg(const float2* A, int nodes, NodeWeight wx, NodeWeight wy) {
  const float2* r0 = A + (size_t(wy.a) * nodes + wx.a) * 4;
  const float2* r1 = r0 + size_t(nodes) * 4;
  const float w00 = (1.f - wx.f) * (1.f - wy.f), w01 = wx.f * (1.f - wy.f);
  const float w10 = (1.f - wx.f) * wy.f, w11 = wx.f * wy.f;
  JonesDiag J;
  {
    const float2 a = __ldg(r0), b = __ldg(r0 + 4), c = __ldg(r1), d = __ldg(r1 + 4);
    J.d0 = {w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y};
  }
  {
    const float2 a = __ldg(r0 + 3), b = __ldg(r0 + 7), c = __ldg(r1 + 3), d = __ldg(r1 + 7);
    J.d1 = {w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y};
  }
  return J;
}
// E = Ap^H X Aq for diagonal Ap, Aq: E_rc = conj(p_r) X_rc q_c
__device__ __forceinline__ Jones jdiag_ah_x_b(const JonesDiag& P, const Jones& X, const JonesDiag& Q) {
  Jones E;
  E.m[0] = cmul(cmulc(P.d0, X.m[0]), Q.d0);
  E.m[1] = cmul(cmulc(P.d0, X.m[1]), Q.d1);
  E.m[2] = cmul(cmulc(P.d1, X.m[2]), Q.d0);
  E.m[3] = cmul(cmulc(P.d1, X.m[3]), Q.d1);
  return E;
}
// Z = Ap Y Aq^H for diagonal Ap, Aq: Z_rc = p_r Y_rc conj(q_c)
__device__ __forceinline__ Jones jdiag_a_y_bh(const JonesDiag& P, const Jones& Y, const JonesDiag& Q) {
  Jones Z;
  Z.m[0] = cmulc(Q.d0, cmul(P.d0, Y.m[0]));
  Z.m[1] = cmulc(Q.d1, cmul(P.d0, Y.m[1]));
  Z.m[2] = cmulc(Q.d0, cmul(P.d1, Y.m[2]));
  Z.m[3] = cmulc(Q.d1, cmul(P.d1, Y.m[3]));
  return Z;
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// V -> V^H for a visibility stored as 2 float4 (XX, XY) (YX, YY): the value a
// mirrored row carries (Section 2.4 footnote, V(u,v,w) = V(-u,-v,-w)^H)
__device__ __forceinline__ void mirror_values(float4& v0, float4& v1) {
  const float4 a = v0, b = v1;
  v0 = make_float4(a.x, -a.y, b.x, -b.y);
  v1 = make_float4(a.z, -a.w, b.z, -b.w);
}

// ---------------------------------------------------------------- async bulk copies (TMA, 1-D)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// arrive once and announce `bytes` of transaction for the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy completing on `bar`; addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar` to complete; gives up after `limit_ns`
// nanoseconds (returns false) so a lost transaction cannot hang the GPU.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// status word bits written by kernels (read back by idg_synchronize)
constexpr int kStatusTimeout = 1;

}  // namespace idg
