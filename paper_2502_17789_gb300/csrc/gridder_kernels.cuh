// Gridder kernels (templates), included by one translation unit per subgrid
// size (gridder_l32.cu ... gridder_l128.cu) so the instantiations compile in
// parallel; gridder.cu dispatches to them.  The algorithm is described at the
// top of gridder.cu.
#pragma once

#include <type_traits>

#include "kernels_common.cuh"

namespace idg {

// ------------------------------------------------------------------ gridder

template <int L, int ROWS>
struct GridCfg {
  static constexpr int PX = 8;           // consecutive pixels of a row per thread
  static constexpr int QN = PX / 2;      // pixel pairs per thread
  static constexpr int TPR = L / PX;     // threads per row
  static constexpr int NT = ROWS * TPR;  // threads per block
  static constexpr int MINB = NT <= 128 ? 3 : (NT <= 192 ? 2 : 1);
  static_assert(L % 8 == 0 && L % ROWS == 0 && (PX == 4 || PX == 8), "gridder shape");
};

// Position of chunk `c` of a subgrid: chunks never straddle segments.
struct ChunkCursor {
  int seg;    // segment index within the subgrid
  int k;      // first member of the chunk
  int end;    // end of the segment
};

__device__ __forceinline__ void cursor_advance(ChunkCursor& cur, int vc, const SegmentDesc* seg, int seg_begin,
                                               int seg_count) {
  cur.k += vc;
  if (cur.k >= cur.end) {
    ++cur.seg;
    if (cur.seg < seg_count) {
      const SegmentDesc s = seg[seg_begin + cur.seg];
      cur.k = s.k_begin;
      cur.end = s.k_end;
    }
  }
}

// One work item.  `cg` counts the chunks this block has consumed so far (it
// selects the buffer and the mbarrier phase, and carries over between the
// items of a persistent block).  Returns false if a bounded wait expired.
// NORM: A-term power normalisation (a.aweights set).  VC: staged records per
// chunk (a compile-time constant: with it the shared-memory layout has fixed
// offsets, which the measured kernel time depends on).
template <int L, int ROWS, bool NORM, int VC>
__device__ __forceinline__ bool gridder_item(const GridArgs& a, int item_idx, uint32_t& cg, float4* s_rec,
                                             float* s_acc, float* s_w, uint64_t* s_bar) {
  using C = GridCfg<L, ROWS>;
  const GridItem item = a.items[item_idx];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x;
  const int j = item.tile * ROWS + tid / C::TPR;
  const int i0 = (tid % C::TPR) * C::PX;
  const int hq = (i0 & 7) >> 1;  // first pixel pair of this thread within its 8-pixel geometry block
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;

  // number of chunks
  int n_chunks = 0;
  for (int g = 0; g < sd.seg_count; ++g) {
    const SegmentDesc s = a.seg[sd.seg_begin + g];
    n_chunks += (s.k_end - s.k_begin + VC - 1) / VC;
  }
  const float4* rec_base = a.records + size_t(sd.rec_offset) * kRecordFloat4;

  // producer (thread 0): issue the copy of the chunk at `pc` into buffer `buf`
  ChunkCursor pc{0, 0, 0};
  if (tid == 0) {
    const SegmentDesc s0 = a.seg[sd.seg_begin];
    pc = {0, s0.k_begin, s0.k_end};
  }
  auto issue = [&](int buf) {
    const int nv = imin(VC, pc.end - pc.k);
    const uint32_t bytes = uint32_t(nv) * kRecordFloat4 * 16;
    mbar_arrive_expect_tx(&s_bar[buf], bytes);
    bulk_copy_g2s(s_rec + buf * VC * kRecordFloat4, rec_base + size_t(pc.k) * kRecordFloat4, bytes, &s_bar[buf]);
    cursor_advance(pc, VC, a.seg, sd.seg_begin, sd.seg_count);
  };
  if (tid == 0) {
    issue(int(cg & 1));
    if (n_chunks > 1) issue(int((cg + 1) & 1));
  }

  // geometry of the 8-pixel block holding this thread's pixels (anchor at
  // its pixel 4), read where phases are evaluated; DI = pixel offsets from the anchor
  const float4* bg = a.blk + (size_t(j) * (L / 8) + (i0 >> 3)) * 3;
  float2 DI[C::QN];
#pragma unroll
  for (int q = 0; q < C::QN; ++q) DI[q] = make_float2(float(2 * (hq + q) - 4), float(2 * (hq + q) - 3));

  float2 RE[4][C::QN], IM[4][C::QN];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < C::QN; ++q) {
      RE[p][q] = make_float2(0.f, 0.f);
      IM[p][q] = make_float2(0.f, 0.f);
    }
  // phasors of the current visibility and of the current channel step; every
  // row of channels starts with a kind-1 record, so none is read unset
  float2 Cs[C::QN], Sn[C::QN], Rc[C::QN], Rs[C::QN];
#pragma unroll
  for (int q = 0; q < C::QN; ++q) Cs[q] = Sn[q] = Rc[q] = Rs[q] = make_float2(0.f, 0.f);

  ChunkCursor cc;
  {
    const SegmentDesc s0 = a.seg[sd.seg_begin];
    cc = {0, s0.k_begin, s0.k_end};
  }
  bool first_seg = true;
  if constexpr (NORM) {
#pragma unroll
    for (int px = 0; px < C::PX; ++px) s_w[px * C::NT + tid] = 0.f;
  }
  for (int c = 0; c < n_chunks; ++c) {
    const uint32_t cc_g = cg + uint32_t(c);
    const int buf = int(cc_g & 1);
    const bool ok = mbar_wait_bounded(&s_bar[buf], (cc_g >> 1) & 1);
    const int nv = imin(VC, cc.end - cc.k);
    // Stokes I with both stations' A-terms of this chunk's segment diagonal:
    // I = (conj(p0) X00 q0 + conj(p1) X11 q1) / 2 needs only the XX and YY sums
    bool two_pol = false;
    if (a.g.npol == 1) {
      const SegmentDesc sg = a.seg[sd.seg_begin + cc.seg];
      two_pol = a.adiag[sg.interval * a.g.n_st + sd.p] && a.adiag[sg.interval * a.g.n_st + sd.q];
    }
    // the record loop, for all four correlations (NP = 4) or XX and YY only (NP = 2)
    auto records = [&](auto np_tag) {
      constexpr int NP = decltype(np_tag)::value;
      const float4* rb = s_rec + buf * VC * kRecordFloat4;
#pragma unroll 1
      for (int v = 0; v < nv; ++v) {
        const float4* rec = rb + v * kRecordFloat4;
        const float4 cw = rec[7];
        const bool base = cw.w == kKindBase;
        if (cw.w != kKindRotate) {
          // phases from the record's slopes: anchor phase in turns (head part
          // exact, then two range reductions) plus FP32 per-pixel increments
          const float4 cf = rec[6];
          const float4 g0 = __ldg(bg), g1 = __ldg(bg + 1), g2 = __ldg(bg + 2);
          const float n0 = g0.x, di0 = g0.y, dj0 = g0.z;
          const float2 DNB[4] = {{g1.x, g1.y}, {g1.z, g1.w}, {g2.x, g2.y}, {g2.z, g2.w}};
          float2 DN[C::QN];
#pragma unroll
          for (int q = 0; q < C::QN; ++q) DN[q] = C::PX == 8 ? DNB[q] : (hq ? DNB[q + 2] : DNB[q]);
          const float sh = fmaf(cf.x, di0, cf.y * dj0);
          const float d1 = __fsub_rn(sh, round_nearest(sh));
          const float lo = fmaf(cw.x, n0, fmaf(cf.z, di0, cf.w * dj0));
          float rr = __fadd_rn(d1, lo);
          rr = __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
          const float2 R0 = make_float2(rr, rr);
          const float2 ARR = make_float2(cw.y, cw.y), CRR = make_float2(cw.z, cw.z);
#pragma unroll
          for (int q = 0; q < C::QN; ++q) {
            const float2 ph = ffma2(CRR, DN[q], ffma2(ARR, DI[q], R0));
            float2 c, s;
            __sincosf(ph.x, &s.x, &c.x);
            __sincosf(ph.y, &s.y, &c.y);
            if (base) {
              Cs[q] = c;
              Sn[q] = s;
            } else {
              Rc[q] = c;
              Rs[q] = s;
            }
          }
        }
        if (!base) {
          // advance by one channel step: e^{i phi} <- e^{i phi} e^{i dphi}
#pragma unroll
          for (int q = 0; q < C::QN; ++q) {
            const float2 c = ffma2(make_float2(-Sn[q].x, -Sn[q].y), Rs[q], fmul2(Cs[q], Rc[q]));
            Sn[q] = ffma2(Sn[q], Rc[q], fmul2(Cs[q], Rs[q]));
            Cs[q] = c;
          }
        }
        const float4 f0 = rec[0], f1 = rec[1], f2 = rec[2], f3 = rec[3], f4 = rec[4], f5 = rec[5];
        const float2 VRR[4] = {{f0.x, f0.y}, {f1.z, f1.w}, {f3.x, f3.y}, {f4.z, f4.w}};
        const float2 VII[4] = {{f0.z, f0.w}, {f2.x, f2.y}, {f3.z, f3.w}, {f5.x, f5.y}};
        const float2 NVI[4] = {{f1.x, f1.y}, {f2.z, f2.w}, {f4.x, f4.y}, {f5.z, f5.w}};
#pragma unroll
        for (int pi = 0; pi < NP; ++pi)
#pragma unroll
          for (int q = 0; q < C::QN; ++q) {
            const int p = NP == 4 ? pi : 3 * pi;  // NP = 2: correlations 0 (XX) and 3 (YY)
            RE[p][q] = ffma2(VRR[p], Cs[q], RE[p][q]);
            IM[p][q] = ffma2(VRR[p], Sn[q], IM[p][q]);
          }
#pragma unroll
        for (int pi = 0; pi < NP; ++pi)
#pragma unroll
          for (int q = 0; q < C::QN; ++q) {
            const int p = NP == 4 ? pi : 3 * pi;
            RE[p][q] = ffma2(NVI[p], Sn[q], RE[p][q]);
            IM[p][q] = ffma2(VII[p], Cs[q], IM[p][q]);
          }
      }
    };
    if (ok) {
      if (two_pol)
        records(std::integral_constant<int, 2>{});
      else
        records(std::integral_constant<int, 4>{});
    }
    // every thread is done with this buffer: refill it with chunk c + 2
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, kStatusTimeout);
        // let copies in flight land before the block's shared memory is released
        mbar_wait_bounded(&s_bar[buf], (cc_g >> 1) & 1);
        mbar_wait_bounded(&s_bar[buf ^ 1], ((cc_g + 1) >> 1) & 1);
      }
      return false;
    }
    if (tid == 0 && c + 2 < n_chunks) {
      fence_proxy_async();
      issue(buf);
    }
    const bool seg_done = cc.k + VC >= cc.end;
    if (seg_done) {
      // ---- epilogue of segment cc.seg: A_p^H X A_q, taper, centring sign (Section 3.3)
      const SegmentDesc seg = a.seg[sd.seg_begin + cc.seg];
      const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
      const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
      const NodeWeight wy = node_weight(j, nodes, L);
      const float tj = a.taper[j];
      // uniform over the block: both stations' A-terms diagonal -> quarter of the Jones work
      const bool diag = a.adiag[seg.interval * a.g.n_st + sd.p] && a.adiag[seg.interval * a.g.n_st + sd.q];
#pragma unroll
      for (int px = 0; px < C::PX; ++px) {
        const int i = i0 + px;
        const int q = px >> 1;
        const NodeWeight wx = node_weight(i, nodes, L);
        Jones X;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          X.m[p].re = (px & 1) ? RE[p][q].y : RE[p][q].x;
          X.m[p].im = (px & 1) ? IM[p][q].y : IM[p][q].x;
        }
        // f2 = ||A_p^H A_q||_F^2 for the A-term power normalisation (Section 3.3),
        // from the same interpolated A-terms
        Jones E;
        float f2 = 0.f;
        if (diag) {
          const JonesDiag P = interp_diag_ldg(Ap, nodes, wx, wy), Q = interp_diag_ldg(Aq, nodes, wx, wy);
          E = jdiag_ah_x_b(P, X, Q);
          if constexpr (NORM)
            f2 = (P.d0.re * P.d0.re + P.d0.im * P.d0.im) * (Q.d0.re * Q.d0.re + Q.d0.im * Q.d0.im) +
                 (P.d1.re * P.d1.re + P.d1.im * P.d1.im) * (Q.d1.re * Q.d1.re + Q.d1.im * Q.d1.im);
        } else {
          const Jones Apj = interp_jones_ldg(Ap, nodes, wx, wy);
          const Jones Aqj = interp_jones_ldg(Aq, nodes, wx, wy);
          E = jmul_ah(Apj, jmul(X, Aqj));
          if constexpr (NORM) {
            const Jones M = jmul_ah(Apj, Aqj);
#pragma unroll
            for (int e = 0; e < 4; ++e) f2 += M.m[e].re * M.m[e].re + M.m[e].im * M.m[e].im;
          }
        }
        float wgt = a.taper[i] * tj * (((i + j) & 1) ? -1.f : 1.f);
        if constexpr (NORM) {
          // divide by f = ||A_p^H A_q||_F
          const float inv_f = f2 > 0.f ? rsqrtf(f2) : 0.f;
          wgt *= inv_f;
          s_w[px * C::NT + tid] += float(seg.k_end - seg.k_begin) * inv_f;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          float* acc = s_acc + (px * 8 + 2 * p) * C::NT + tid;
          if (first_seg) {
            acc[0] = wgt * E.m[p].re;
            acc[C::NT] = wgt * E.m[p].im;
          } else {
            acc[0] += wgt * E.m[p].re;
            acc[C::NT] += wgt * E.m[p].im;
          }
        }
      }
      first_seg = false;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < C::QN; ++q) {
          RE[p][q] = make_float2(0.f, 0.f);
          IM[p][q] = make_float2(0.f, 0.f);
        }
    }
    cursor_advance(cc, VC, a.seg, sd.seg_begin, sd.seg_count);
  }

  // ---- A-term weights of this thread's pixels, and the subgrid's visibility count once
  if (NORM && n_chunks > 0) {
#pragma unroll 1
    for (int px = 0; px < C::PX; ++px) atomicAdd(&a.aweights[size_t(j) * L + i0 + px], double(s_w[px * C::NT + tid]));
    if (item.tile == 0 && tid == 0) atomicAdd(&a.aweights[size_t(L) * L], double(sd.n_vis));
  }
  // ---- write the subgrid image rows: [sg][pol][j][i]; in Stokes-I mode only
  // plane 0, I = (XX + YY) / 2
  if (n_chunks > 0 && a.g.npol == 1) {
    float4* dst = reinterpret_cast<float4*>(a.scratch + (size_t(item.sg) * 4 * L + j) * L + i0);
#pragma unroll
    for (int h = 0; h < C::QN; ++h) {
      const int px = 2 * h;
      auto half_trace = [&](int q, int c) {
        return 0.5f * (s_acc[(q * 8 + c) * C::NT + tid] + s_acc[(q * 8 + 6 + c) * C::NT + tid]);
      };
      dst[h] = make_float4(half_trace(px, 0), half_trace(px, 1), half_trace(px + 1, 0), half_trace(px + 1, 1));
    }
  } else if (n_chunks > 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float4* dst = reinterpret_cast<float4*>(a.scratch + ((size_t(item.sg) * 4 + p) * L + j) * L + i0);
#pragma unroll
      for (int h = 0; h < C::QN; ++h) {
        const int px = 2 * h;
        dst[h] = make_float4(s_acc[(px * 8 + 2 * p) * C::NT + tid], s_acc[(px * 8 + 2 * p + 1) * C::NT + tid],
                             s_acc[((px + 1) * 8 + 2 * p) * C::NT + tid],
                             s_acc[((px + 1) * 8 + 2 * p + 1) * C::NT + tid]);
      }
    }
  }
  cg += uint32_t(n_chunks);
  return true;
}

// PERSIST = false: one item per block (block index, LPT order).
// PERSIST = true: #SMs x occupancy blocks pull items from the work-queue
// counter a.queue until the n_items are drained.
// NORM: with the A-term power normalisation.
template <int L, int ROWS, bool PERSIST, bool NORM, int VC>
__global__ void __launch_bounds__(GridCfg<L, ROWS>::NT, GridCfg<L, ROWS>::MINB)
    gridder_kernel(const GridArgs a) {
  using C = GridCfg<L, ROWS>;
  extern __shared__ float4 smem[];
  float4* s_rec = smem;                                                      // [2][VC][8]
  float* s_acc = reinterpret_cast<float*>(s_rec + 2 * VC * kRecordFloat4);   // [8 PX][NT]
  float* s_w = s_acc + 8 * C::PX * C::NT;                                    // [PX][NT] A-term weights
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_w + C::PX * C::NT);        // [2]
  int* s_item = reinterpret_cast<int*>(s_bar + 2);
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  if constexpr (!PERSIST) {
    gridder_item<L, ROWS, NORM, VC>(a, blockIdx.x, cg, s_rec, s_acc, s_w, s_bar);
  } else {
  for (;;) {
    if (threadIdx.x == 0) *s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= a.n_items) return;
    if (!gridder_item<L, ROWS, NORM, VC>(a, it, cg, s_rec, s_acc, s_w, s_bar)) return;
    __syncthreads();  // shared buffers and s_item free for the next item
  }
  }
}

// One launch over the work items of several plans (the serving loop's
// shared work queue): block b runs item items[b] = (plan slot, item index
// in that slot's batch), with the slot's arguments copied to shared memory
// first.  One item per block, in the order given (longest first).
template <int L, int ROWS, bool NORM, int VC>
__global__ void __launch_bounds__(GridCfg<L, ROWS>::NT, GridCfg<L, ROWS>::MINB)
    gridder_multi_kernel(const GridArgs* args, const int2* items) {
  using C = GridCfg<L, ROWS>;
  // raw storage: the argument struct is trivially copyable, copied in by one thread
  __shared__ __align__(16) unsigned char s_args_raw[sizeof(GridArgs)];
  extern __shared__ float4 smem[];
  const int2 it = items[blockIdx.x];
  if (threadIdx.x == 0) memcpy(s_args_raw, args + it.x, sizeof(GridArgs));
  __syncthreads();
  const GridArgs& a = *reinterpret_cast<const GridArgs*>(s_args_raw);
  float4* s_rec = smem;                                                      // [2][VC][8]
  float* s_acc = reinterpret_cast<float*>(s_rec + 2 * VC * kRecordFloat4);   // [8 PX][NT]
  float* s_w = s_acc + 8 * C::PX * C::NT;                                    // [PX][NT]
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_w + C::PX * C::NT);        // [2]
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  gridder_item<L, ROWS, NORM, VC>(a, it.y, cg, s_rec, s_acc, s_w, s_bar);
}

template <int L, int ROWS>
size_t gridder_smem(int vc) {
  using C = GridCfg<L, ROWS>;
  return sizeof(float4) * 2 * vc * kRecordFloat4 + sizeof(float) * 9 * C::PX * C::NT + 2 * sizeof(uint64_t) + 16;
}

// Calls f(std::integral_constant<int, VC>) for the chunk sizes the kernels
// are instantiated for; false for any other.
template <typename F>
bool with_chunk(int vc, F&& f) {
  switch (vc) {
    case 32: f(std::integral_constant<int, 32>{}); return true;
    case 48: f(std::integral_constant<int, 48>{}); return true;
    case 64: f(std::integral_constant<int, 64>{}); return true;
    default: return false;
  }
}


template <int L, int ROWS>
int configure_gridder_t(int vc, int* persistent_blocks) {
  using C = GridCfg<L, ROWS>;
  cudaError_t e = cudaSuccess;
  int per_sm = 0;
  const bool ok = with_chunk(vc, [&](auto tag) {
    constexpr int VC = decltype(tag)::value;
    const int smem = int(gridder_smem<L, ROWS>(VC));
    const void* fns[6] = {reinterpret_cast<const void*>(gridder_kernel<L, ROWS, false, false, VC>),
                          reinterpret_cast<const void*>(gridder_kernel<L, ROWS, true, false, VC>),
                          reinterpret_cast<const void*>(gridder_kernel<L, ROWS, false, true, VC>),
                          reinterpret_cast<const void*>(gridder_kernel<L, ROWS, true, true, VC>),
                          reinterpret_cast<const void*>(gridder_multi_kernel<L, ROWS, false, VC>),
                          reinterpret_cast<const void*>(gridder_multi_kernel<L, ROWS, true, VC>)};
    for (const void* fn : fns)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gridder_kernel<L, ROWS, true, false, VC>, C::NT,
                                                        smem);
  });
  if (!ok) return int(cudaErrorInvalidValue);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L, int ROWS>
int launch_gridder_t(const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
  using C = GridCfg<L, ROWS>;
  if (n_items <= 0) return 0;
  const int pb = persistent_blocks < n_items ? persistent_blocks : n_items;
  cudaStream_t st = cudaStream_t(stream);
  const bool ok = with_chunk(a.vc, [&](auto tag) {
    constexpr int VC = decltype(tag)::value;
    const size_t smem = gridder_smem<L, ROWS>(VC);
    if (a.aweights) {
      if (persistent_blocks > 0)
        gridder_kernel<L, ROWS, true, true, VC><<<pb, C::NT, smem, st>>>(a);
      else
        gridder_kernel<L, ROWS, false, true, VC><<<n_items, C::NT, smem, st>>>(a);
    } else {
      if (persistent_blocks > 0)
        gridder_kernel<L, ROWS, true, false, VC><<<pb, C::NT, smem, st>>>(a);
      else
        gridder_kernel<L, ROWS, false, false, VC><<<n_items, C::NT, smem, st>>>(a);
    }
  });
  if (!ok) return int(cudaErrorInvalidValue);
  return int(cudaGetLastError());
}

template <int L, int ROWS>
int launch_gridder_multi_t(const GridArgs* args, const int2* items, int n_items, bool norm, int vc,
                                  void* stream) {
  using C = GridCfg<L, ROWS>;
  if (n_items <= 0) return 0;
  const bool ok = with_chunk(vc, [&](auto tag) {
    constexpr int VC = decltype(tag)::value;
    const size_t smem = gridder_smem<L, ROWS>(VC);
    if (norm)
      gridder_multi_kernel<L, ROWS, true, VC><<<n_items, C::NT, smem, cudaStream_t(stream)>>>(args, items);
    else
      gridder_multi_kernel<L, ROWS, false, VC><<<n_items, C::NT, smem, cudaStream_t(stream)>>>(args, items);
  });
  if (!ok) return int(cudaErrorInvalidValue);
  return int(cudaGetLastError());
}

// rows per pixel tile of the gridder for subgrid size L (0: unsupported)
constexpr int gridder_rows_for(int L) { return L == 32 ? 32 : L == 64 ? 16 : (L == 96 || L == 128) ? 8 : 0; }

template <int L>
int gridder_launch(const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
  return launch_gridder_t<L, gridder_rows_for(L)>(a, n_items, persistent_blocks, stream);
}
template <int L>
int gridder_configure(int vc, int* persistent_blocks) {
  return configure_gridder_t<L, gridder_rows_for(L)>(vc, persistent_blocks);
}
template <int L>
int gridder_launch_multi(const GridArgs* args, const int2* items, int n_items, bool norm, int vc, void* stream) {
  return launch_gridder_multi_t<L, gridder_rows_for(L)>(args, items, n_items, norm, vc, stream);
}

}  // namespace idg
