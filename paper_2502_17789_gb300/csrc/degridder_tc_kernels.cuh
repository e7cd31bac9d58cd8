// Degridder on the tensor cores (templates), included by the per-subgrid-size
// translation units next to degridder_kernels.cuh.
//
// The same item as the FP32 degridder (Eq. 13 read as the adjoint of the
// gridder, one or two A-term segments of one subgrid, one visibility per
// row), with the sum V_k = sum_{ij} Z(i,j) e^{-2 pi i phi_k(i,j)} taken as a
// real matrix product D = A B: the rows of A are visibilities, its columns
// the pairs (cos, sin) of the phase at 4 pixels per step, and B holds Z at
// those pixels so that column 2p of D is Re V_p and column 2p+1 is Im V_p:
//   re:  B[(q, cos)] = Zr_p(q),  B[(q, sin)] = Zi_p(q)
//   im:  B[(q, cos)] = Zi_p(q),  B[(q, sin)] = -Zr_p(q).
// One mma.sync m16n8k8 (TF32 operands, FP32 accumulator) takes 16
// visibilities x 4 pixels.  TF32 keeps 10 explicit mantissa bits, so each
// operand is split into hi (its top 19 bits) and lo (the rest, exact in
// FP32) and the product is taken as A_hi B_hi + A_lo B_hi + A_hi B_lo (the
// dropped A_lo B_lo is ~2^-21 of a term): about FP32 accuracy, with the
// phasors computed by the CUDA cores (phase in FP32 from the exact anchor
// reduction, __sincosf) and the multiply-accumulate on the tensor pipe.  The
// accumulators run over the 64 pixels of one chunk (48 MMAs) and are then
// added into shared memory in FP32, which bounds the tensor core's
// accumulation rounding.
//
// Layout: the chunk of 512 pixels is split into 8 groups of 64, one per
// warp; lane (g, t) of a warp evaluates rows g and g+8 of each 16-row tile
// at pixels 16 t .. 16 t + 15 of its group (one phase anchor per 16 pixels,
// as in the FP32 kernel), pixel 16 t + k in step k.  Z is stored per chunk
// as [group][k][t][pol] complex values (rows of 16 values padded to 18 so
// that the prologue's stores spread over the banks), so the B fragment of
// a step is one contiguous 128-byte row.  Rows of the second segment start
// at the next multiple of 16, so no tile mixes the two segments' Z.
#pragma once

#include "degridder_kernels.cuh"

namespace idg {

constexpr int kTcRows = kTcItemRows;  // rows (visibilities) per item, 16 tiles of 16
constexpr int kTcGroup = 4;         // tiles per warp pass
constexpr int kTcZRow = 18;         // complex values per (group, step) row of the Z layout
constexpr int kTcChunkPixels = 512;
constexpr uint32_t kTf32Mask = 0xffffe000u;

struct DegridTcSmem {
  float2 z[2][kDegridSegs][8 * 16 * kTcZRow];  // [buf][segment][group][step][t * 4 + pol]
  float4 g[2][kTcChunkPixels / 16][5];         // geometry of the 16-pixel phase-anchor blocks
  float4 coef[2][kTcRows];                     // per row: (ah, bh, al, bl), (w, 2 pi a, 2 pi w, 0)
  float out[8][kTcRows + 4];                   // [component][row], padded against bank conflicts
};

__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// (hi, lo) split of x for TF32 operands: hi = x with the low 13 mantissa bits cleared, lo = x - hi (exact)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & kTf32Mask;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// the same for a pair: two masks and one packed FMA, lo = x - hi
__device__ __forceinline__ void tf32_split2(float2 x, uint32_t& hi0, uint32_t& hi1, uint32_t& lo0, uint32_t& lo1) {
  hi0 = __float_as_uint(x.x) & kTf32Mask;
  hi1 = __float_as_uint(x.y) & kTf32Mask;
  const float2 lo = ffma2(make_float2(__uint_as_float(hi0), __uint_as_float(hi1)), make_float2(-1.f, -1.f), x);
  lo0 = __float_as_uint(lo.x);
  lo1 = __float_as_uint(lo.y);
}

// Row of the item (tile layout) for lane l: segment 1 starts at row r1
__device__ __forceinline__ int tc_row(int l, int n0, int r1, int n_seg) {
  return (n_seg == 2 && l >= n0) ? r1 + (l - n0) : l;
}

// The sums of CNT tiles (tiles gb .. gb + CNT - 1) over this lane's 16-pixel
// run of the chunk, added into S.out.  CNT is a compile-time count so that
// the tiles' independent sine/cosine, split and MMA chains interleave.
template <int CNT>
__device__ __forceinline__ void tc_group_sum(DegridTcSmem& S, const float2* zs, const float* dn, const float4 g0,
                                             int gb, int g, int t) {
  const bool odd = g & 1;
  float2 R0[CNT], AR[CNT], CR[CNT];
#pragma unroll
  for (int m = 0; m < CNT; ++m) {
    const int ra = 16 * (gb + m) + g;
    const float4 c1a = S.coef[1][ra], c1b = S.coef[1][ra + 8];
    R0[m] = make_float2(anchor_phase(S.coef[0][ra], c1a, g0.x, g0.y, g0.z),
                        anchor_phase(S.coef[0][ra + 8], c1b, g0.x, g0.y, g0.z));
    AR[m] = make_float2(c1a.y, c1b.y);
    CR[m] = make_float2(c1a.z, c1b.z);
  }
  float acc[CNT][4];
#pragma unroll
  for (int m = 0; m < CNT; ++m) acc[m][0] = acc[m][1] = acc[m][2] = acc[m][3] = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    // B fragment of step k: this lane's column is pol g/2, re (g even) or im (g odd)
    const float2 z = zs[k * kTcZRow];
    uint32_t Bh[2], Bl[2];
    tf32_split2(make_float2(odd ? z.y : z.x, odd ? -z.x : z.y), Bh[0], Bh[1], Bl[0], Bl[1]);
    const float dnk = dn[k];
    const float2 DN = make_float2(dnk, dnk);
    const float2 DI = make_float2(float(k - 8), float(k - 8));
#pragma unroll
    for (int m = 0; m < CNT; ++m) {
      const float2 ph = ffma2(CR[m], DN, ffma2(AR[m], DI, R0[m]));
      float ca, sa, cb, sb;
      __sincosf(ph.x, &sa, &ca);
      __sincosf(ph.y, &sb, &cb);
      // A fragment: (row g, col t) cos, (row g+8, col t) cos, (row g, col t+4) sin, (row g+8, col t+4) sin
      uint32_t Ah[4], Al[4];
      tf32_split2(make_float2(ca, cb), Ah[0], Ah[1], Al[0], Al[1]);
      tf32_split2(make_float2(sa, sb), Ah[2], Ah[3], Al[2], Al[3]);
      mma_tf32_16x8x8(acc[m], Ah, Bh);
      mma_tf32_16x8x8(acc[m], Al, Bh);
      mma_tf32_16x8x8(acc[m], Ah, Bl);
    }
  }
  // D fragment: (row g, cols 2t, 2t+1) and (row g+8, cols 2t, 2t+1) = pol t (re, im)
#pragma unroll
  for (int m = 0; m < CNT; ++m) {
    const int ra = 16 * (gb + m) + g;
    atomicAdd(&S.out[2 * t][ra], acc[m][0]);
    atomicAdd(&S.out[2 * t + 1][ra], acc[m][1]);
    atomicAdd(&S.out[2 * t][ra + 8], acc[m][2]);
    atomicAdd(&S.out[2 * t + 1][ra + 8], acc[m][3]);
  }
}

template <int L>
__device__ __forceinline__ void degridder_tc_item(const DegridArgs& a, int item_idx, DegridTcSmem& S, float2* s_A) {
  constexpr int TPR = L / 8;
  constexpr int NBLK = L * L / 8;      // 8-pixel blocks of the subgrid
  constexpr int CB = kTcChunkPixels / 8;
  constexpr int NCH = NBLK / CB;
  constexpr int NT = 256;
  static_assert(NBLK % CB == 0, "chunking");
  const DegridItem item = a.items[item_idx];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int nl = item.k_end - item.k_begin;
  const int n0 = item.k_mid - item.k_begin;
  const int n_seg = item.k_mid < item.k_end ? 2 : 1;
  const int r1 = (n0 + 15) & ~15;                       // first row of segment 1
  const int T0 = n_seg == 2 ? r1 >> 4 : (nl + 15) >> 4;  // tiles of segment 0
  const int T1 = n_seg == 2 ? (nl - n0 + 15) >> 4 : 0;   // tiles of segment 1
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;
  const int nc = sd.c1 - sd.c0;
  unsigned diag = 0;
#pragma unroll
  for (int s = 0; s < kDegridSegs; ++s) {
    if (s < n_seg) {
      const SegmentDesc seg = a.seg[item.segment + s];
      if (a.adiag[seg.interval * a.g.n_st + sd.p] && a.adiag[seg.interval * a.g.n_st + sd.q]) diag |= 1u << s;
      const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
      const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
      for (int e = tid; e < nA; e += NT) {
        s_A[2 * s * nA + e] = Ap[e];
        s_A[(2 * s + 1) * nA + e] = Aq[e];
      }
    }
  }
  // row tid: phase coefficients of its visibility (zeros for padding rows)
  {
    int l = tid;
    if (n_seg == 2) l = tid < r1 ? (tid < n0 ? tid : -1) : tid - r1 + n0;
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
    if (l >= 0 && l < nl) {
      const int gidx = item.k_begin + l;
      const int row = gidx / nc;
      double aa, bb, w;
      degrid_slopes(a, sd, L, sd.t0 + row, sd.c0 + (gidx - row * nc), aa, bb, w);
      degrid_coef(aa, bb, w, c0, c1);
    }
    S.coef[0][tid] = c0;
    S.coef[1][tid] = c1;
#pragma unroll
    for (int c = 0; c < 8; ++c) S.out[c][tid] = 0.f;
  }
  const float2* Y = a.scratch + size_t(item.sg) * 4 * L * L;

  // prologue geometry: each thread builds one pixel pair per chunk
  const int pb = tid >> 2;
  const int pq = tid & 3;
  float2 ya[4], yb[4];
  auto load_y = [&](int chunk) {
    const int bidx = chunk * CB + pb;
    const int j = bidx / TPR, i = (bidx % TPR) * 8 + 2 * pq;
    if (a.g.npol == 1) {
      const float4 v = *reinterpret_cast<const float4*>(Y + size_t(j) * L + i);
      ya[0] = ya[3] = make_float2(v.x, v.y);
      yb[0] = yb[3] = make_float2(v.z, v.w);
      ya[1] = ya[2] = yb[1] = yb[2] = make_float2(0.f, 0.f);
      return;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float4 v = *reinterpret_cast<const float4*>(Y + (size_t(p) * L + j) * L + i);
      ya[p] = make_float2(v.x, v.y);
      yb[p] = make_float2(v.z, v.w);
    }
  };
  auto build_z = [&](int chunk, int buf) {
    const int bidx = chunk * CB + pb;
    const int j = bidx / TPR, i = (bidx % TPR) * 8 + 2 * pq;
    const NodeWeight wy = node_weight(j, nodes, L);
    const float tj = a.taper[j];
#pragma unroll 1
    for (int s = 0; s < n_seg; ++s) {
      const float2* sAp = s_A + 2 * s * nA;
      const float2* sAq = sAp + nA;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ii = i + h;
        Jones Yp;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 y = h ? yb[p] : ya[p];
          Yp.m[p] = {y.x, y.y};
        }
        const NodeWeight wx = node_weight(ii, nodes, L);
        Jones Z;
        if (diag >> s & 1u) {
          Z = jdiag_a_y_bh(interp_diag(sAp, nodes, wx, wy), Yp, interp_diag(sAq, nodes, wx, wy));
        } else {
          const Jones Apj = interp_jones(sAp, nodes, wx, wy);
          const Jones Aqj = interp_jones(sAq, nodes, wx, wy);
          Z = jmul_bh(jmul(Apj, Yp), Aqj);
        }
        const float wgt = a.taper[ii] * tj * (((ii + j) & 1) ? -1.f : 1.f);
        // chunk pixel -> (group, step, t) of the tensor-core layout
        const int px = pb * 8 + 2 * pq + h;
        const int zi = ((px >> 6) * 16 + (px & 15)) * kTcZRow + ((px >> 4) & 3) * 4;
        float4* dst = reinterpret_cast<float4*>(&S.z[buf][s][zi]);
        dst[0] = make_float4(wgt * Z.m[0].re, wgt * Z.m[0].im, wgt * Z.m[1].re, wgt * Z.m[1].im);
        dst[1] = make_float4(wgt * Z.m[2].re, wgt * Z.m[2].im, wgt * Z.m[3].re, wgt * Z.m[3].im);
      }
    }
    if (tid < CB / 2 * 5) {
      const int b = tid / 5, c = tid % 5;
      S.g[buf][b][c] = a.blk16[size_t(chunk * (CB / 2) + b) * 5 + c];
    }
  };

  load_y(0);
  __syncthreads();  // s_A and the coefficient table visible
  build_z(0, 0);
  __syncthreads();

  for (int chunk = 0; chunk < NCH; ++chunk) {
    const int buf = chunk & 1;
    const bool more = chunk + 1 < NCH;
    const float4* Gm = S.g[buf][4 * warp + t];  // this lane's 16-pixel anchor block
    const float4 g0 = Gm[0];
    const float* dn = reinterpret_cast<const float*>(Gm + 1);  // n' increments of its 16 pixels
#pragma unroll 1
    for (int s = 0; s < n_seg; ++s) {
      const float2* zs = &S.z[buf][s][warp * 16 * kTcZRow + t * 4 + (g >> 1)];
      const int tb = s == 0 ? 0 : T0, te = s == 0 ? T0 : T0 + T1;
#pragma unroll 1
      for (int gb = tb; gb < te; gb += kTcGroup) {
        switch (imin(kTcGroup, te - gb)) {
          case 4: tc_group_sum<4>(S, zs, dn, g0, gb, g, t); break;
          case 3: tc_group_sum<3>(S, zs, dn, g0, gb, g, t); break;
          case 2: tc_group_sum<2>(S, zs, dn, g0, gb, g, t); break;
          default: tc_group_sum<1>(S, zs, dn, g0, gb, g, t); break;
        }
      }
    }
    if (more) {
      load_y(chunk + 1);
      build_z(chunk + 1, buf ^ 1);
    }
    __syncthreads();
  }

  // ---- write the visibilities of this item
  if (tid < nl) {
    const int r = tc_row(tid, n0, r1, n_seg);
    const int gidx = item.k_begin + tid;
    const int row = gidx / nc;
    const size_t vrow = (size_t(sd.b) * a.g.n_t + sd.t0 + row) * a.g.n_ch + sd.c0 + (gidx - row * nc);
    float4 v0 = make_float4(S.out[0][r], S.out[1][r], S.out[2][r], S.out[3][r]);
    float4 v1 = make_float4(S.out[4][r], S.out[5][r], S.out[6][r], S.out[7][r]);
    if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);
    a.vis[2 * vrow] = v0;
    a.vis[2 * vrow + 1] = v1;
  }
}

template <int L, bool PERSIST>
__global__ void __launch_bounds__(256, 2) degridder_tc_kernel(const DegridArgs a) {
  extern __shared__ float4 smem_raw[];
  DegridTcSmem& S = *reinterpret_cast<DegridTcSmem*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);  // [segment][station p, q][nodes*nodes*4]
  __shared__ int s_item;
  if constexpr (!PERSIST) {
    degridder_tc_item<L>(a, blockIdx.x, S, s_A);
  } else {
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
      __syncthreads();
      const int it = s_item;
      if (it >= a.n_items) return;
      degridder_tc_item<L>(a, it, S, s_A);
      __syncthreads();
    }
  }
}

template <int L>
__global__ void __launch_bounds__(256, 2) degridder_tc_multi_kernel(const DegridArgs* args, const int2* items) {
  extern __shared__ float4 smem_raw[];
  DegridTcSmem& S = *reinterpret_cast<DegridTcSmem*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);
  __shared__ __align__(16) unsigned char s_args_raw[sizeof(DegridArgs)];
  const int2 it = items[blockIdx.x];
  if (threadIdx.x == 0) memcpy(s_args_raw, args + it.x, sizeof(DegridArgs));
  __syncthreads();
  degridder_tc_item<L>(*reinterpret_cast<const DegridArgs*>(s_args_raw), it.y, S, s_A);
}

inline size_t degridder_tc_smem(int nodes) {
  return sizeof(DegridTcSmem) + sizeof(float2) * 2 * kDegridSegs * nodes * nodes * 4;
}

template <int L>
int configure_degridder_tc_l(int nodes, int* persistent_blocks) {
  const int smem_max = int(degridder_tc_smem(kMaxAtermNodes));
  cudaError_t e = cudaFuncSetAttribute(degridder_tc_kernel<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_max);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(degridder_tc_kernel<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(degridder_tc_multi_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, degridder_tc_kernel<L, true>, 256,
                                                      degridder_tc_smem(nodes));
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L>
int launch_degridder_tc_l(const DegridArgs& a, int n_items, int persistent_blocks, void* stream) {
  if (n_items <= 0) return 0;
  const size_t smem = degridder_tc_smem(a.g.nodes);
  if (persistent_blocks > 0)
    degridder_tc_kernel<L, true><<<persistent_blocks < n_items ? persistent_blocks : n_items, 256, smem,
                                   cudaStream_t(stream)>>>(a);
  else
    degridder_tc_kernel<L, false><<<n_items, 256, smem, cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

template <int L>
int launch_degridder_tc_multi_l(const DegridArgs* args, const int2* items, int n_items, int max_nodes,
                                void* stream) {
  if (n_items <= 0) return 0;
  cudaError_t e = cudaFuncSetAttribute(degridder_tc_multi_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(degridder_tc_smem(kMaxAtermNodes)));
  if (e != cudaSuccess) return int(e);
  degridder_tc_multi_kernel<L><<<n_items, 256, degridder_tc_smem(max_nodes), cudaStream_t(stream)>>>(args, items);
  return int(cudaGetLastError());
}

}  // namespace idg
