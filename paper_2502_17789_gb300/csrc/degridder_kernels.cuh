// Degridder kernels (templates), included by one translation unit per subgrid
// size (degridder_l32.cu ... degridder_l128.cu) so the instantiations compile
// in parallel; degridder.cu dispatches to them.  The algorithm is described at
// the top of degridder.cu.
#pragma once

#include <type_traits>

#include "kernels_common.cuh"

namespace idg {

constexpr int kRangeBlocks = 8;   // pixel blocks (of 8 pixels) per work unit (one per warp per lane group)

// Launch shape per channels-per-lane C: W warps per block, each summing 8
// pixel blocks of every chunk, so a chunk is 8 W blocks (64 W pixels).  With
// C = 4 the 4 sets of accumulators need more registers than 16 warps per SM
// leave, so that variant runs 4-warp blocks, 3 per SM (12 warps).
__host__ __device__ constexpr int degrid_warps(int C) { return C >= 4 ? 4 : 8; }
__host__ __device__ constexpr int degrid_threads(int C) { return 32 * degrid_warps(C); }
__host__ __device__ constexpr int degrid_min_blocks(int C) { return C >= 4 ? 3 : 2; }

template <int C>
struct DegridSmem {
  static constexpr int LN = degrid_lanes(C);         // lanes per item
  static constexpr int CB = 8 * degrid_warps(C);     // pixel blocks per chunk
  // [buf][segment][pol][block][pixel pair] {Zr_a, Zr_b, Zi_a, Zi_b}: the prologue's thread t writes
  // element t of each pol plane, so a warp's stores are contiguous (no bank conflicts)
  float4 z[2][kDegridSegs][4][CB][4];
  float4 g[2][CB / 2][5];  // geometry of the 16-pixel phase-anchor blocks
  // [lane group][k][lane]: k = 0, 1 first channel (ah, bh, al, bl), (w, 2 pi a, 2 pi w, 0);
  // k = 2, 3 the channel step in the same form (C > 1)
  float4 coef[LN / 32][C > 1 ? 4 : 2][32];
  float out[8][C][LN];  // [component][channel of the group][lane], accumulated with shared atomics
};

// Phase slopes of (row t, channel ch) of a subgrid in turns per pixel, and
// w - w0 in turns (Section 2.4), from FP64 uvw (negated on a mirrored subgrid)
__device__ __forceinline__ void degrid_slopes(const DegridArgs& a, const SubgridDesc& sd, int L, int t, int ch,
                                              double& aa, double& bb, double& w) {
  const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
  const double fs = subgrid_sign(sd) * a.fscale[ch];  // a mirrored subgrid predicts (-u, -v, -w)
  const double inv_l = 1.0 / double(L);
  aa = ((r[0] * fs) * a.g.fov - double(sd.x0 + L / 2 - a.g.N / 2)) * inv_l;
  bb = ((r[1] * fs) * a.g.fov - double(sd.y0 + L / 2 - a.g.N / 2)) * inv_l;
  w = r[2] * fs - subgrid_w0(a.g, sd);
}

// (head, tail) split of the slopes for the exact anchor reduction
__device__ __forceinline__ void degrid_coef(double aa, double bb, double w, float4& c0, float4& c1) {
  const double ah = rint(aa * 65536.0) * (1.0 / 65536.0);
  const double bh = rint(bb * 65536.0) * (1.0 / 65536.0);
  c0 = make_float4(float(ah), float(bh), float(aa - ah), float(bb - bh));
  c1 = make_float4(float(w), float(kTwoPi * aa), float(kTwoPi * w), 0.f);
}

// anchor phase in radians, reduced to [-pi, pi]: head part exact, then two range reductions
__device__ __forceinline__ float anchor_phase(float4 c0, float4 c1, float n0, float di0, float dj0) {
  const float sh = fmaf(c0.x, di0, c0.y * dj0);
  const float d1 = __fsub_rn(sh, round_nearest(sh));
  const float lo = fmaf(c1.x, n0, fmaf(c0.z, di0, c0.w * dj0));
  const float rr = __fadd_rn(d1, lo);
  return __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
}

// A lane's phase anchor at one 16-pixel block: reduced phase and slopes of its
// first channel, and of the channel step (C > 1)
struct Anchor {
  float r0, d0;
  float2 arr, crr, darr, dcrr;
};

template <int C>
__device__ __forceinline__ Anchor lane_anchor(const DegridSmem<C>& S, int g, int sl, const float4 g0) {
  Anchor an;
  const float4 c1 = S.coef[g][1][sl];
  an.r0 = anchor_phase(S.coef[g][0][sl], c1, g0.x, g0.y, g0.z);
  an.arr = make_float2(c1.y, c1.y);
  an.crr = make_float2(c1.z, c1.z);
  an.d0 = 0.f;
  an.darr = an.dcrr = make_float2(0.f, 0.f);
  if constexpr (C > 1) {
    const float4 c3 = S.coef[g][3][sl];
    an.d0 = anchor_phase(S.coef[g][2][sl], c3, g0.x, g0.y, g0.z);
    an.darr = make_float2(c3.y, c3.y);
    an.dcrr = make_float2(c3.z, c3.z);
  }
  return an;
}

// Phasor sum of pixel pair q of 16-pixel block b2 into a lane's C x NP
// accumulators (NP = 4 correlations, or 2: XX and YY)
template <int C, int NP, int CB>
__device__ __forceinline__ void mac_pair(const float4* Gm, const Anchor& an, const float4* zs, int b2, int q,
                                         float2* RE, float2* IM) {
  const float4 dn4 = Gm[1 + (q >> 1)];  // n' increments of pixels 4(q/2) .. 4(q/2)+3
  const float2 DN = (q & 1) ? make_float2(dn4.z, dn4.w) : make_float2(dn4.x, dn4.y);
  const float2 DI = make_float2(float(2 * q - 8), float(2 * q - 7));
  const float2 ph = ffma2(an.crr, DN, ffma2(an.arr, DI, make_float2(an.r0, an.r0)));
  float2 Cs, Sn;
  __sincosf(ph.x, &Sn.x, &Cs.x);
  __sincosf(ph.y, &Sn.y, &Cs.y);
  float2 Rc = make_float2(1.f, 1.f), Rs = make_float2(0.f, 0.f);
  if constexpr (C > 1) {
    // phasor of the channel step at these pixels
    const float2 dph = ffma2(an.dcrr, DN, ffma2(an.darr, DI, make_float2(an.d0, an.d0)));
    __sincosf(dph.x, &Rs.x, &Rc.x);
    __sincosf(dph.y, &Rs.y, &Rc.y);
  }
  float2 ZR[NP], ZI[NP];
#pragma unroll
  for (int pi = 0; pi < NP; ++pi) {
    const int p = NP == 4 ? pi : 3 * pi;
    const float4 z = zs[(p * CB + 2 * b2 + (q >> 2)) * 4 + (q & 3)];  // Z[pol][block][pair]
    ZR[pi] = make_float2(z.x, z.y);
    ZI[pi] = make_float2(z.z, z.w);
  }
#pragma unroll
  for (int h = 0; h < C; ++h) {
    if (h > 0) {
      // next channel: e^{i phi} <- e^{i phi} e^{i dphi}
      const float2 c = ffma2(make_float2(-Sn.x, -Sn.y), Rs, fmul2(Cs, Rc));
      Sn = ffma2(Sn, Rc, fmul2(Cs, Rs));
      Cs = c;
    }
    const float2 NS = make_float2(-Sn.x, -Sn.y);
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      const int p = NP == 4 ? pi : 3 * pi;
      // V += Z conj(e): re += Zr c + Zi s, im += Zi c - Zr s
      float2& re = RE[h * 4 + p];
      float2& im = IM[h * 4 + p];
      re = ffma2(ZR[pi], Cs, re);
      re = ffma2(ZI[pi], Sn, re);
      im = ffma2(ZI[pi], Cs, im);
      im = ffma2(ZR[pi], NS, im);
    }
  }
}

// SPLIT: an item of at most kSplitLanes lanes, run by its own kernel (see below)
template <int L, int C, bool SPLIT>
__device__ __forceinline__ void degridder_item(const DegridArgs& a, int item_idx, DegridSmem<C>& S, float2* s_A) {
  constexpr int TPR = L / 8;
  constexpr int NBLK = L * L / 8;
  constexpr int NT = degrid_threads(C);
  constexpr int kChunkBlocks = DegridSmem<C>::CB;
  constexpr int NCH = NBLK / kChunkBlocks;
  constexpr int LN = DegridSmem<C>::LN;
  static_assert(NBLK % kChunkBlocks == 0 && kChunkBlocks == degrid_warps(C) * kRangeBlocks, "chunking");
  static_assert(LN <= NT && NT == 4 * kChunkBlocks, "one thread per lane and per pixel pair in the prologue");
  const DegridItem item = a.items[item_idx];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nl = item.k_end - item.k_begin;          // lanes (channel groups) of the item
  const int n0 = item.k_mid - item.k_begin;          // lanes of the first segment
  const int n_seg = item.k_mid < item.k_end ? 2 : 1;
  const int n_vg = (nl + 31) >> 5;  // groups of 32 lanes
  // lanes per slot: an item of at most kSplitLanes lanes spreads each slot over R = 32 / 2^ceil(log2 nl)
  // lanes of a warp
  int R = 1;
  if constexpr (SPLIT)
    while (R * 2 * nl <= 32 && R < 32) R *= 2;
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;
  const int nc = sd.c1 - sd.c0;
  const int G = (nc + C - 1) / C;  // channel groups per row
  // per segment, uniform over the block: both stations' A-terms diagonal -> quarter of the Jones work
  unsigned diag = 0;  // bit s: segment s
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
  const unsigned all_segs = n_seg == 2 ? 3u : 1u;
  const bool two_pol = a.g.npol == 1 && (diag & all_segs) == all_segs;
  // lane tid: row and channel range of its group; FP64 offsets -> FP32 phase
  // coefficients of its first channel and of the channel step (zeros for empty lanes)
  int my_t = 0, my_c = 0, my_n = 0;
  if (tid < LN) {
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0, c2 = c0, c3 = c0;
    if (tid < nl) {
      const int gidx = item.k_begin + tid;
      const int row = gidx / G, gi = gidx - row * G;
      my_t = sd.t0 + row;
      my_c = sd.c0 + (gi * nc) / G;
      my_n = sd.c0 + ((gi + 1) * nc) / G - my_c;
      double aa, bb, w;
      degrid_slopes(a, sd, L, my_t, my_c, aa, bb, w);
      degrid_coef(aa, bb, w, c0, c1);
      if (C > 1 && my_n > 1) {
        double a2, b2, w2;
        degrid_slopes(a, sd, L, my_t, my_c + 1, a2, b2, w2);
        degrid_coef(a2 - aa, b2 - bb, w2 - w, c2, c3);
      }
    }
    S.coef[tid >> 5][0][tid & 31] = c0;
    S.coef[tid >> 5][1][tid & 31] = c1;
    if constexpr (C > 1) {
      S.coef[tid >> 5][2][tid & 31] = c2;
      S.coef[tid >> 5][3][tid & 31] = c3;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
      for (int h = 0; h < C; ++h) S.out[c][h][tid] = 0.f;
  }
  const float2* Y = a.scratch + size_t(item.sg) * 4 * L * L;

  // prologue geometry: each thread builds one pixel pair (2 consecutive pixels) per chunk
  const int pb = tid >> 2;          // block within the chunk
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
    // lane group, over all four correlations (NP = 4) or, for a Stokes-I
    // model seen through diagonal A-terms, XX and YY only (NP = 2: Z01 =
    // Z10 = 0, so the predicted XY and YX are zero)
    auto sum_chunk = [&](auto np_tag) {
    constexpr int NP = decltype(np_tag)::value;
    if constexpr (SPLIT) {
      // few lanes in the item (low occupancy, Section 3.2): the R lanes of
      // slot lane / R take every R-th pixel pair of the warp's range and
      // their partial sums are added with warp shuffles, instead of one
      // lane per slot and the other lanes idle
      const int sl = lane / R, sub = lane % R;
      const float4* zs = &S.z[buf][sl >= n0 ? 1 : 0][0][0][0];
      float2 RE[C * 4], IM[C * 4];
#pragma unroll
      for (int h = 0; h < C; ++h)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          RE[h * 4 + p] = make_float2(0.f, 0.f);
          IM[h * 4 + p] = make_float2(0.f, 0.f);
        }
#pragma unroll 1
      for (int pp = sub; pp < 4 * kRangeBlocks; pp += R) {
        const int b2 = warp * (kRangeBlocks / 2) + (pp >> 3), q = pp & 7;
        const float4* Gm = S.g[buf][b2];
        mac_pair<C, NP, DegridSmem<C>::CB>(Gm, lane_anchor<C>(S, 0, sl, Gm[0]), zs, b2, q, RE, IM);
      }
#pragma unroll
      for (int h = 0; h < C; ++h)
#pragma unroll
        for (int pi = 0; pi < NP; ++pi) {
          const int p = NP == 4 ? pi : 3 * pi;
          float re = RE[h * 4 + p].x + RE[h * 4 + p].y, im = IM[h * 4 + p].x + IM[h * 4 + p].y;
          for (int off = R >> 1; off > 0; off >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, off);
            im += __shfl_xor_sync(0xffffffffu, im, off);
          }
          if (sub == 0) {
            atomicAdd(&S.out[2 * p][h][sl], re);
            atomicAdd(&S.out[2 * p + 1][h][sl], im);
          }
        }
    } else {
    for (int g = 0; g < n_vg; ++g) {
      // Z of this lane's segment (lanes of one group may straddle the two segments)
      const float4(*zs)[kChunkBlocks][4] = S.z[buf][g * 32 + lane >= n0 ? 1 : 0];
      float2 RE[C][4], IM[C][4];
#pragma unroll
      for (int h = 0; h < C; ++h)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          RE[h][p] = make_float2(0.f, 0.f);
          IM[h][p] = make_float2(0.f, 0.f);
        }
#pragma unroll 1
      for (int b2 = warp * (kRangeBlocks / 2); b2 < (warp + 1) * (kRangeBlocks / 2); ++b2) {
        // one phase anchor per 16 pixels (pixel 8 of the block): exact reduction there, FP32 increments
        // the lane's coefficients are re-read from shared memory per anchor (registers go to the sums)
        const float4* Gm = S.g[buf][b2];
        const float4 g0 = Gm[0];
        const float4 c1 = S.coef[g][1][lane];
        const float2 R0 = make_float2(anchor_phase(S.coef[g][0][lane], c1, g0.x, g0.y, g0.z), 0.f);
        const float2 ARR = make_float2(c1.y, c1.y), CRR = make_float2(c1.z, c1.z);
        float2 D0 = make_float2(0.f, 0.f);
        [[maybe_unused]] float2 DARR = D0, DCRR = D0;
        if constexpr (C > 1) {
          const float4 c3 = S.coef[g][3][lane];
          D0.x = anchor_phase(S.coef[g][2][lane], c3, g0.x, g0.y, g0.z);
          DARR = make_float2(c3.y, c3.y);
          DCRR = make_float2(c3.z, c3.z);
        }
#pragma unroll(C > 2 ? 2 : 8)
        for (int q = 0; q < 8; ++q) {
          const float4 dn4 = Gm[1 + (q >> 1)];  // n' increments of pixels 4(q/2) .. 4(q/2)+3
          const float2 DN = (q & 1) ? make_float2(dn4.z, dn4.w) : make_float2(dn4.x, dn4.y);
          const float2 DI = make_float2(float(2 * q - 8), float(2 * q - 7));
          const float2 ph = ffma2(CRR, DN, ffma2(ARR, DI, make_float2(R0.x, R0.x)));
          float2 Cs, Sn;
          __sincosf(ph.x, &Sn.x, &Cs.x);
          __sincosf(ph.y, &Sn.y, &Cs.y);
          float2 Rc = make_float2(1.f, 1.f), Rs = make_float2(0.f, 0.f);
          if constexpr (C > 1) {
            // phasor of the channel step at these pixels
            const float2 dph = ffma2(DCRR, DN, ffma2(DARR, DI, make_float2(D0.x, D0.x)));
            __sincosf(dph.x, &Rs.x, &Rc.x);
            __sincosf(dph.y, &Rs.y, &Rc.y);
          }
          float2 ZR[NP], ZI[NP];
#pragma unroll
          for (int pi = 0; pi < NP; ++pi) {
            const int p = NP == 4 ? pi : 3 * pi;
            const float4 z = zs[p][2 * b2 + (q >> 2)][q & 3];
            ZR[pi] = make_float2(z.x, z.y);
            ZI[pi] = make_float2(z.z, z.w);
          }
#pragma unroll
          for (int h = 0; h < C; ++h) {
            if (h > 0) {
              // next channel: e^{i phi} <- e^{i phi} e^{i dphi}
              const float2 c = ffma2(make_float2(-Sn.x, -Sn.y), Rs, fmul2(Cs, Rc));
              Sn = ffma2(Sn, Rc, fmul2(Cs, Rs));
              Cs = c;
            }
            const float2 NS = make_float2(-Sn.x, -Sn.y);
#pragma unroll
            for (int pi = 0; pi < NP; ++pi) {
              const int p = NP == 4 ? pi : 3 * pi;
              // V += Z conj(e): re += Zr c + Zi s, im += Zi c - Zr s
              RE[h][p] = ffma2(ZR[pi], Cs, RE[h][p]);
              RE[h][p] = ffma2(ZI[pi], Sn, RE[h][p]);
              IM[h][p] = ffma2(ZI[pi], Cs, IM[h][p]);
              IM[h][p] = ffma2(ZR[pi], NS, IM[h][p]);
            }
          }
        }
      }
      const int slot = g * 32 + lane;
#pragma unroll
      for (int h = 0; h < C; ++h)
#pragma unroll
        for (int pi = 0; pi < NP; ++pi) {
          const int p = NP == 4 ? pi : 3 * pi;
          atomicAdd(&S.out[2 * p][h][slot], RE[h][p].x + RE[h][p].y);
          atomicAdd(&S.out[2 * p + 1][h][slot], IM[h][p].x + IM[h][p].y);
        }
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

  // ---- write the visibilities of this item: lane tid's my_n channels
  if (tid < nl) {
    const size_t vrow = (size_t(sd.b) * a.g.n_t + my_t) * a.g.n_ch + my_c;
#pragma unroll
    for (int h = 0; h < C; ++h) {
      if (h < my_n) {
        float4 v0 = make_float4(S.out[0][h][tid], S.out[1][h][tid], S.out[2][h][tid], S.out[3][h][tid]);
        float4 v1 = make_float4(S.out[4][h][tid], S.out[5][h][tid], S.out[6][h][tid], S.out[7][h][tid]);
        if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);  // the visibility is the mirror's V^H
        a.vis[2 * (vrow + h)] = v0;
        a.vis[2 * (vrow + h) + 1] = v1;
      }
    }
  }
}

// PERSIST = false: one item per block; true: blocks drain the a.queue counter.
// C: channels per lane.
template <int L, int C, bool PERSIST>
__global__ void __launch_bounds__(degrid_threads(C), degrid_min_blocks(C)) degridder_kernel(const DegridArgs a) {
  extern __shared__ float4 smem_raw[];
  DegridSmem<C>& S = *reinterpret_cast<DegridSmem<C>*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);  // [segment][station p, q][nodes*nodes*4]
  __shared__ int s_item;
  if constexpr (!PERSIST) {
    degridder_item<L, C, false>(a, blockIdx.x, S, s_A);
  } else {
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) return;
    degridder_item<L, C, false>(a, it, S, s_A);
    __syncthreads();  // shared memory and s_item free for the next item
  }
  }
}

// Items of at most kSplitLanes lanes (subgrids of few visibilities, the low
// occupancy of Section 3.2) in a kernel of their own, one item per block:
// each visibility's pixels are spread over several lanes.  A separate
// instantiation keeps the code of the regular kernel exactly as it is.
template <int L, int C>
__global__ void __launch_bounds__(degrid_threads(C), degrid_min_blocks(C)) degridder_split_kernel(const DegridArgs a) {
  extern __shared__ float4 smem_raw[];
  DegridSmem<C>& S = *reinterpret_cast<DegridSmem<C>*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);
  degridder_item<L, C, true>(a, blockIdx.x, S, s_A);
}

// One launch over the work items of several plans (the serving loop's
// shared work queue): block b runs item items[b] = (plan slot, item index
// in that slot's batch) with the slot's arguments copied to shared memory.
template <int L, int C, bool SPLIT>
__global__ void __launch_bounds__(degrid_threads(C), degrid_min_blocks(C))
    degridder_multi_kernel(const DegridArgs* args, const int2* items) {
  extern __shared__ float4 smem_raw[];
  DegridSmem<C>& S = *reinterpret_cast<DegridSmem<C>*>(smem_raw);
  float2* s_A = reinterpret_cast<float2*>(&S + 1);
  // raw storage: the argument struct is trivially copyable, copied in by one thread
  __shared__ __align__(16) unsigned char s_args_raw[sizeof(DegridArgs)];
  const int2 it = items[blockIdx.x];
  if (threadIdx.x == 0) memcpy(s_args_raw, args + it.x, sizeof(DegridArgs));
  __syncthreads();
  degridder_item<L, C, SPLIT>(*reinterpret_cast<const DegridArgs*>(s_args_raw), it.y, S, s_A);
}

template <int C>
size_t degridder_smem(int nodes) {
  return sizeof(DegridSmem<C>) + sizeof(float2) * 2 * kDegridSegs * nodes * nodes * 4;
}

// The shared-memory limit is set for the largest node count any plan may
// use, so plans with different node counts can share the kernels; the
// occupancy (persistent grid size) follows this plan's own footprint.
template <int L, int C>
int configure_degridder_t(int nodes, int* persistent_blocks) {
  const int smem_max = int(degridder_smem<C>(kMaxAtermNodes));
  const int smem = int(degridder_smem<C>(nodes));
  cudaError_t e =
      cudaFuncSetAttribute(degridder_kernel<L, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(degridder_kernel<L, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(degridder_split_kernel<L, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, degridder_kernel<L, C, true>, degrid_threads(C), smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L, int C>
int launch_degridder_t(const DegridArgs& a, int n_items, int persistent_blocks, void* stream, bool split) {
  const size_t smem = degridder_smem<C>(a.g.nodes);
  if (n_items <= 0) return 0;
  if (split)
    degridder_split_kernel<L, C><<<n_items, degrid_threads(C), smem, cudaStream_t(stream)>>>(a);
  else if (persistent_blocks > 0)
    degridder_kernel<L, C, true><<<persistent_blocks < n_items ? persistent_blocks : n_items, degrid_threads(C),
                                   smem, cudaStream_t(stream)>>>(a);
  else
    degridder_kernel<L, C, false><<<n_items, degrid_threads(C), smem, cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

template <int L>
int launch_degridder_l(const DegridArgs& a, int channels, int n_items, int persistent_blocks, void* stream,
                              bool split) {
  switch (channels) {
    case 1: return launch_degridder_t<L, 1>(a, n_items, persistent_blocks, stream, split);
    case 2: return launch_degridder_t<L, 2>(a, n_items, persistent_blocks, stream, split);
    case 4: return launch_degridder_t<L, 4>(a, n_items, persistent_blocks, stream, split);
    default: return int(cudaErrorInvalidValue);
  }
}

template <int L>
int configure_degridder_l(int nodes, int channels, int* persistent_blocks) {
  switch (channels) {
    case 1: return configure_degridder_t<L, 1>(nodes, persistent_blocks);
    case 2: return configure_degridder_t<L, 2>(nodes, persistent_blocks);
    case 4: return configure_degridder_t<L, 4>(nodes, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}


template <int L, int C, bool SPLIT>
int launch_degridder_multi_t(const DegridArgs* args, const int2* items, int n_items, int max_nodes,
                                    void* stream) {
  if (n_items <= 0) return 0;
  cudaError_t e = cudaFuncSetAttribute(degridder_multi_kernel<L, C, SPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(degridder_smem<C>(kMaxAtermNodes)));
  if (e != cudaSuccess) return int(e);
  degridder_multi_kernel<L, C, SPLIT><<<n_items, degrid_threads(C), degridder_smem<C>(max_nodes),
                                        cudaStream_t(stream)>>>(args, items);
  return int(cudaGetLastError());
}

template <int L, int C>
int launch_degridder_multi_s(bool split, const DegridArgs* args, const int2* items, int n_items, int max_nodes,
                                    void* stream) {
  return split ? launch_degridder_multi_t<L, C, true>(args, items, n_items, max_nodes, stream)
               : launch_degridder_multi_t<L, C, false>(args, items, n_items, max_nodes, stream);
}

template <int L>
int launch_degridder_multi_l(int channels, bool split, const DegridArgs* args, const int2* items, int n_items,
                                    int max_nodes, void* stream) {
  switch (channels) {
    case 1: return launch_degridder_multi_s<L, 1>(split, args, items, n_items, max_nodes, stream);
    case 2: return launch_degridder_multi_s<L, 2>(split, args, items, n_items, max_nodes, stream);
    case 4: return launch_degridder_multi_s<L, 4>(split, args, items, n_items, max_nodes, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

}  // namespace idg
