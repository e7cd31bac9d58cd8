// Degridder kernel: Section 2.5 prediction step 3c (Eq. 13), read as the
// exact adjoint of the gridder:
//   Z(i,j) = (-1)^(i+j) T_i T_j A_p(i,j) Y(i,j) A_q(i,j)^H
//   V_k    = sum_{ij} Z(i,j) e^{-2 pi i phi_k(i,j)}
// where Y is the uncentred inverse subgrid FFT of the split-out grid
// footprint (the splitter applied (-1)^(x+y)).
//
// Work item = up to 256 visibilities of one or two consecutive segments of
// a subgrid (one A-term each), in groups of 32 (one per lane); pairing
// segments fills the lanes that a lone segment of, say, 40 visibilities
// would leave idle.  The block walks the subgrid in chunks of 64 pixel
// blocks (8 consecutive pixels of a row each, 512 pixels).  Within a chunk,
// warp w sums pixel blocks [8w, 8w+8) for every visibility group in turn and
// adds its partial sums into a shared-memory accumulator with shared-memory
// atomics, so all warps stay busy whatever the segment size.  Z of the next
// chunk is built while the current chunk is summed: its Y values are loaded
// into registers before the phasor sum and turned into Z (A-term prologue)
// after it, into the other half of a double buffer, one barrier per chunk;
// with two segments, each pixel pair gets one Z per segment and every lane
// reads the Z of its own visibility's segment.
// Phases use the same FP64 offset / exact anchor reduction / FP32 increment
// scheme as the gridder, with one anchor per 16 pixels of a row.
#include <type_traits>

#include "kernels_common.cuh"

namespace idg {

constexpr int kDegridThreads = 256;
constexpr int kChunkBlocks = 64;  // pixel blocks (of 8) per chunk = 512 pixels
constexpr int kRangeBlocks = 8;   // pixel blocks per work unit (one per warp per visibility group)

template <int L>
struct DegridSmem {
  // [buf][segment][pol][block][pixel pair] {Zr_a, Zr_b, Zi_a, Zi_b}: the prologue's thread t writes
  // element t of each pol plane, so a warp's stores are contiguous (no bank conflicts)
  float4 z[2][kDegridSegs][4][kChunkBlocks][4];
  float4 g[2][kChunkBlocks / 2][5]; // geometry of the 16-pixel phase-anchor blocks
  float4 coef[8][2][32];            // [vis group][half][lane]: (ah, bh, al, bl), (w, 2 pi a, 2 pi w, 0)
  float out[8][kDegridThreads];     // [component][visibility slot], accumulated with shared atomics
};

template <int L>
__device__ __forceinline__ void degridder_item(const DegridArgs& a, int item_idx, DegridSmem<L>& S, float2* s_A) {
  constexpr int TPR = L / 8;
  constexpr int NBLK = L * L / 8;
  constexpr int NCH = NBLK / kChunkBlocks;
  static_assert(NBLK % kChunkBlocks == 0 && kChunkBlocks == 8 * kRangeBlocks, "chunking");
  const DegridItem item = a.items[item_idx];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nv = item.k_end - item.k_begin;
  const int n0 = item.k_mid - item.k_begin;          // visibilities of the first segment
  const int n_seg = item.k_mid < item.k_end ? 2 : 1;
  const int n_vg = (nv + 31) >> 5;  // groups of 32 visibilities, 1..8
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;
  // per segment, uniform over the block: both stations' A-terms diagonal -> quarter of the Jones work
  unsigned diag = 0;  // bit s: segment s
#pragma unroll
  for (int s = 0; s < kDegridSegs; ++s) {
    if (s < n_seg) {
      const SegmentDesc seg = a.seg[item.segment + s];
      if (a.adiag[seg.interval * a.g.n_st + sd.p] && a.adiag[seg.interval * a.g.n_st + sd.q]) diag |= 1u << s;
      const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
      const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
      for (int e = tid; e < nA; e += kDegridThreads) {
        s_A[2 * s * nA + e] = Ap[e];
        s_A[(2 * s + 1) * nA + e] = Aq[e];
      }
    }
  }
  const unsigned all_segs = n_seg == 2 ? 3u : 1u;
  const bool two_pol = a.g.npol == 1 && (diag & all_segs) == all_segs;
  // visibility slot tid: FP64 offsets -> FP32 phase coefficients (zeros for empty slots)
  {
    const int nc = sd.c1 - sd.c0;
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
    if (tid < nv) {
      const int k = item.k_begin + tid;
      const int t = sd.t0 + k / nc, ch = sd.c0 + k % nc;
      const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
      const double fs = subgrid_sign(sd) * a.fscale[ch];  // a mirrored subgrid predicts (-u, -v, -w)
      const double inv_l = 1.0 / double(L);
      const double dx = (r[0] * fs) * a.g.fov - double(sd.x0 + L / 2 - a.g.N / 2);
      const double dy = (r[1] * fs) * a.g.fov - double(sd.y0 + L / 2 - a.g.N / 2);
      const double w = r[2] * fs - subgrid_w0(a.g, sd);  // w - w0 (Section 2.4)
      const double aa = dx * inv_l, bb = dy * inv_l;
      const double dah = rint(aa * 65536.0) * (1.0 / 65536.0);
      const double dbh = rint(bb * 65536.0) * (1.0 / 65536.0);
      c0 = make_float4(float(dah), float(dbh), float(aa - dah), float(bb - dbh));
      c1 = make_float4(float(w), float(kTwoPi * aa), float(kTwoPi * w), 0.f);
    }
    S.coef[tid >> 5][0][tid & 31] = c0;
    S.coef[tid >> 5][1][tid & 31] = c1;
#pragma unroll
    for (int c = 0; c < 8; ++c) S.out[c][tid] = 0.f;
  }
  const float2* Y = a.scratch + size_t(item.sg) * 4 * L * L;

  // prologue geometry: each thread builds one pixel pair (2 consecutive pixels) per chunk
  const int pb = tid >> 2;          // block within the chunk, 0..63
  const int pq = tid & 3;           // pixel pair within the block
  float2 ya[4], yb[4];              // Y of the pair, prefetched

  auto load_y = [&](int chunk) {
    const int bidx = chunk * kChunkBlocks + pb;
    const int j = bidx / TPR, i = (bidx % TPR) * 8 + 2 * pq;
    if (a.g.npol == 1) {
      // Stokes-I model: Y = Y_I times the 2x2 identity (XX = YY = I)
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
    const int bidx = chunk * kChunkBlocks + pb;
    const int j = bidx / TPR, i = (bidx % TPR) * 8 + 2 * pq;
    const NodeWeight wy = node_weight(j, nodes, L);
    const float tj = a.taper[j];
#pragma unroll 1
    for (int s = 0; s < n_seg; ++s) {
    const float2* sAp = s_A + 2 * s * nA;
    const float2* sAq = sAp + nA;
    float4 zo[4];
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
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (h == 0) {
          zo[p].x = wgt * Z.m[p].re;
          zo[p].z = wgt * Z.m[p].im;
        } else {
          zo[p].y = wgt * Z.m[p].re;
          zo[p].w = wgt * Z.m[p].im;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) S.z[buf][s][p][pb][pq] = zo[p];
    }
    if (tid < kChunkBlocks / 2 * 5) {
      const int b = tid / 5, c = tid % 5;
      S.g[buf][b][c] = a.blk16[size_t(chunk * (kChunkBlocks / 2) + b) * 5 + c];
    }
  };

  load_y(0);
  __syncthreads();  // s_A and the coefficient table visible
  build_z(0, 0);
  __syncthreads();

  for (int chunk = 0; chunk < NCH; ++chunk) {
    const int buf = chunk & 1;
    const bool more = chunk + 1 < NCH;
    if (more) load_y(chunk + 1);
    // warp `warp` sums pixel blocks [warp*8, warp*8+8) of the chunk for every
    // visibility group, over all four correlations (NP = 4) or, for a
    // Stokes-I model seen through diagonal A-terms, XX and YY only (NP = 2:
    // Z01 = Z10 = 0, so the predicted XY and YX are zero)
    auto sum_chunk = [&](auto np_tag) {
    constexpr int NP = decltype(np_tag)::value;
    for (int g = 0; g < n_vg; ++g) {
      const float4 c0 = S.coef[g][0][lane], c1 = S.coef[g][1][lane];
      // Z of this lane's segment (lanes of one group may straddle the two segments)
      const float4(*zs)[kChunkBlocks][4] = S.z[buf][g * 32 + lane >= n0 ? 1 : 0];
      const float2 ARR = make_float2(c1.y, c1.y), CRR = make_float2(c1.z, c1.z);
      float2 RE[4], IM[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        RE[p] = make_float2(0.f, 0.f);
        IM[p] = make_float2(0.f, 0.f);
      }
#pragma unroll 1
      for (int b2 = warp * (kRangeBlocks / 2); b2 < (warp + 1) * (kRangeBlocks / 2); ++b2) {
        // one phase anchor per 16 pixels (pixel 8 of the block): exact reduction there, FP32 increments
        const float4* G = S.g[buf][b2];
        const float4 g0 = G[0];
        const float n0 = g0.x, di0 = g0.y, dj0 = g0.z;
        const float sh = fmaf(c0.x, di0, c0.y * dj0);
        const float d1 = __fsub_rn(sh, round_nearest(sh));
        const float lo = fmaf(c1.x, n0, fmaf(c0.z, di0, c0.w * dj0));
        float rr = __fadd_rn(d1, lo);
        rr = __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
        const float2 R0 = make_float2(rr, rr);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 dn4 = G[1 + (q >> 1)];  // n' increments of pixels 4(q/2) .. 4(q/2)+3
          const float2 DN = (q & 1) ? make_float2(dn4.z, dn4.w) : make_float2(dn4.x, dn4.y);
          const float2 DI = make_float2(float(2 * q - 8), float(2 * q - 7));
          const float2 ph = ffma2(CRR, DN, ffma2(ARR, DI, R0));
          float2 Cs, Sn;
          __sincosf(ph.x, &Sn.x, &Cs.x);
          __sincosf(ph.y, &Sn.y, &Cs.y);
          const float2 NS = make_float2(-Sn.x, -Sn.y);
#pragma unroll
          for (int pi = 0; pi < NP; ++pi) {
            const int p = NP == 4 ? pi : 3 * pi;
            const float4 z = zs[p][2 * b2 + (q >> 2)][q & 3];
            const float2 ZR = make_float2(z.x, z.y), ZI = make_float2(z.z, z.w);
            // V += Z conj(e): re += Zr c + Zi s, im += Zi c - Zr s
            RE[p] = ffma2(ZR, Cs, RE[p]);
            RE[p] = ffma2(ZI, Sn, RE[p]);
            IM[p] = ffma2(ZI, Cs, IM[p]);
            IM[p] = ffma2(ZR, NS, IM[p]);
          }
        }
      }
      const int slot = g * 32 + lane;
#pragma unroll
      for (int pi = 0; pi < NP; ++pi) {
        const int p = NP == 4 ? pi : 3 * pi;
        atomicAdd(&S.out[2 * p][slot], RE[p].x + RE[p].y);
        atomicAdd(&S.out[2 * p + 1][slot], IM[p].x + IM[p].y);
      }
    }
    };
    if (two_pol)
      sum_chunk(std::integral_constant<int, 2>{});
    else
      sum_chunk(std::integral_constant<int, 4>{});
    if (more) build_z(chunk + 1, buf ^ 1);
    __syncthreads();
  }

  // ---- write the visibilities of this item
  if (tid < nv) {
    const int nc = sd.c1 - sd.c0;
    const int k = item.k_begin + tid;
    const int t = sd.t0 + k / nc, ch = sd.c0 + k % nc;
    const size_t vidx = (size_t(sd.b) * a.g.n_t + t) * a.g.n_ch + ch;
    float4 v0 = make_float4(S.out[0][tid], S.out[1][tid], S.out[2][tid], S.out[3][tid]);
    float4 v1 = make_float4(S.out[4][tid], S.out[5][tid], S.out[6][tid], S.out[7][tid]);
    if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);  // the visibility is the mirror's V^H
    a.vis[2 * vidx] = v0;
    a.vis[2 * vidx + 1] = v1;
  }
}

// PERSIST = false: one item per block; true: blocks drain the a.queue counter.
template <int L, bool PERSIST>
__global__ void __launch_bounds__(kDegridThreads, 2) degridder_kernel(const DegridArgs a) {
  extern __shared__ float4 smem_raw[];
  DegridSmem<L>& S = *reinterpret_cast<DegridSmem<L>*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);  // [segment][station p, q][nodes*nodes*4]
  __shared__ int s_item;
  if constexpr (!PERSIST) {
    degridder_item<L>(a, blockIdx.x, S, s_A);
  } else {
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) return;
    degridder_item<L>(a, it, S, s_A);
    __syncthreads();  // shared memory and s_item free for the next item
  }
  }
}

template <int L>
static size_t degridder_smem(int nodes) {
  return sizeof(DegridSmem<L>) + sizeof(float2) * 2 * kDegridSegs * nodes * nodes * 4;
}

// The shared-memory limit is set for the largest node count any plan may
// use, so plans with different node counts can share the kernels; the
// occupancy (persistent grid size) follows this plan's own footprint.
template <int L>
static int configure_degridder_t(int nodes, int* persistent_blocks) {
  const int smem_max = int(degridder_smem<L>(kMaxAtermNodes));
  const int smem = int(degridder_smem<L>(nodes));
  cudaError_t e =
      cudaFuncSetAttribute(degridder_kernel<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(degridder_kernel<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, degridder_kernel<L, true>, kDegridThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L>
static int launch_degridder_t(const DegridArgs& a, int n_items, int persistent_blocks, void* stream) {
  const size_t smem = degridder_smem<L>(a.g.nodes);
  if (n_items <= 0) return 0;
  if (persistent_blocks > 0)
    degridder_kernel<L, true><<<persistent_blocks < n_items ? persistent_blocks : n_items, kDegridThreads, smem,
                                cudaStream_t(stream)>>>(a);
  else
    degridder_kernel<L, false><<<n_items, kDegridThreads, smem, cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

int launch_degridder(int L, const DegridArgs& a, int n_items, int persistent_blocks, void* stream) {
  switch (L) {
    case 32: return launch_degridder_t<32>(a, n_items, persistent_blocks, stream);
    case 64: return launch_degridder_t<64>(a, n_items, persistent_blocks, stream);
    case 96: return launch_degridder_t<96>(a, n_items, persistent_blocks, stream);
    case 128: return launch_degridder_t<128>(a, n_items, persistent_blocks, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int configure_degridder(int L, int nodes, int* persistent_blocks) {
  switch (L) {
    case 32: return configure_degridder_t<32>(nodes, persistent_blocks);
    case 64: return configure_degridder_t<64>(nodes, persistent_blocks);
    case 96: return configure_degridder_t<96>(nodes, persistent_blocks);
    case 128: return configure_degridder_t<128>(nodes, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}

}  // namespace idg
