// Gridder on the tensor cores (templates), included by the per-subgrid-size
// translation units gridder_tc_l32.cu ... gridder_tc_l128.cu.
//
// Eq. 10's direct sum X_p(i,j) = sum_k V_{k,p} e^{+2 pi i phi_k(i,j)} of one
// A-term segment taken as a real matrix product D = A B: the rows of A are
// pixels, its columns (cos, sin) of the phase of 4 visibilities per step,
// and B holds the visibilities so that column 2p of D is Re X_p and column
// 2p+1 is Im X_p:
//   re:  B[(k, cos)] = Re V_{k,p},  B[(k, sin)] = -Im V_{k,p}
//   im:  B[(k, cos)] = Im V_{k,p},  B[(k, sin)] = Re V_{k,p}.
// One mma.sync m16n8k8 (TF32 operands split into hi + lo as in the
// tensor-core degridder, three products, FP32 accumulation) takes 16
// pixels x 4 visibilities.
//
// The 4 visibilities of a step are 4 rows (timesteps) of the segment at one
// channel, so lane (g, t) follows row t along its channels.  The channels of
// a row group are taken in runs of kGtcRun (the last run holds the rest):
// the phasors of the lane's two pixels start from an exact
// anchor at the run's first channel (__sincosf) and advance by the phasor of
// the channel step for the others (the phase is linear in frequency; the plan
// uses this kernel only for uniform channel spacing).  Rows are taken in
// groups of 4 per segment, the last group padded with zero visibilities.
//
// Staged records (stage_tc_kernel), per subgrid from rec_offset: for every
// row group and run, a header of 16 float4 -- for rows t = 0..3 the phase
// coefficients of the run's first channel at [2t, 2t+1] and of the channel
// step at [8 + 2t, 9 + 2t], in the (head, tail) slope format of the exact
// reduction -- then one step of 32 float4 per channel of the run: column n
// of row t at [4n + t], holding (b0_hi, b1_hi, b0_lo, b1_lo), so that lane
// 4g + t reads its B fragment from float4 number lane of the step
// (conflict-free).  Runs are packed without padding (tc_run_offset).
//
// Item = (subgrid, block of 512 pixels): warp w owns pixels 64 w .. 64 w + 63
// of the block as 4 tiles of 16 (pixels g and g+8 of a tile are rows g and
// g+8 of A).  Runs stream through a double buffer in shared memory by bulk
// copies, two runs per chunk (a whole run of kGtcRun channels fully
// unrolled, a shorter last run in a loop); after every run the accumulators
// are added into an FP32 sum in shared memory (this bounds the tensor core's
// accumulation rounding); after each segment a warp applies A_p^H X A_q, the
// taper and the centring sign to its 64 pixels and adds them to the image
// sum.
#pragma once

#include "kernels_common.cuh"

namespace idg {

constexpr int kGtcChunkRuns = 2;  // runs per staged chunk
// pol planes of the per-pixel sums, padded so that the flush (lanes g, t ->
// pixel g, pol t) and the epilogue (lane -> pixel) both access distinct banks
constexpr int kGtcPolStride = kGtcPixels + 8;
constexpr uint32_t kGtcMask = 0xffffe000u;

__device__ __forceinline__ void tc_split_store(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & kGtcMask);
  lo = x - hi;
}

// The subgrid row of slot t of row group G (-1 for a padding slot)
__device__ __forceinline__ int tc_slot_row(const SegmentDesc* seg, int seg_begin, int seg_count, int nc, int G,
                                           int t) {
  for (int s = 0; s < seg_count; ++s) {
    const SegmentDesc d = seg[seg_begin + s];
    const int r0 = d.k_begin / nc, rows = (d.k_end - d.k_begin) / nc;
    const int ng = (rows + 3) / 4;
    if (G < ng) {
      const int r = 4 * G + t;
      return r < rows ? r0 + r : -1;
    }
    G -= ng;
  }
  return -1;
}

struct TcSlopes {
  double a, b, w;
};

__device__ __forceinline__ TcSlopes tc_slopes(const StageArgs& a, const SubgridDesc& sd, int t, int ch, int L) {
  const double inv_l = 1.0 / double(L);
  const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
  const double fs = subgrid_sign(sd) * a.fscale[ch];
  const double dx = (r[0] * fs) * a.g.fov - double(sd.x0 + L / 2 - a.g.N / 2);
  const double dy = (r[1] * fs) * a.g.fov - double(sd.y0 + L / 2 - a.g.N / 2);
  return {dx * inv_l, dy * inv_l, r[2] * fs - subgrid_w0(a.g, sd)};
}

__device__ __forceinline__ void tc_put_coef(float4* dst, double aa, double bb, double w) {
  const double ah = rint(aa * 65536.0) * (1.0 / 65536.0);
  const double bh = rint(bb * 65536.0) * (1.0 / 65536.0);
  dst[0] = make_float4(float(ah), float(bh), float(aa - ah), float(bb - bh));
  dst[1] = make_float4(float(w), float(kTwoPi * aa), float(kTwoPi * w), 0.f);
}

// One block per subgrid of the batch: run headers and visibility records
template <int L>
__global__ void __launch_bounds__(256) stage_tc_kernel(const StageArgs a, const SegmentDesc* seg) {
  const SubgridDesc sd = a.sg[blockIdx.x];
  const int nc = sd.c1 - sd.c0;
  const int R = tc_runs(nc);
  const int NG = tc_row_groups(seg, sd.seg_begin, sd.seg_count, nc);
  const int NR = NG * R;
  float4* base = a.records + size_t(sd.rec_offset) * kRecordFloat4;
  // one thread per (row group, channel, row slot): the 8 columns of one visibility
  const int n_vrec = NG * nc * 4;
  for (int idx = threadIdx.x; idx < n_vrec; idx += blockDim.x) {
    const int G = idx / (nc * 4), rem = idx - G * (nc * 4), s = rem >> 2, t = rem & 3;
    const int u = s / kGtcRun, st = s - u * kGtcRun;
    const int row = tc_slot_row(seg, sd.seg_begin, sd.seg_count, nc, G, t);
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (row >= 0) {
      const size_t vidx = (size_t(sd.b) * a.g.n_t + sd.t0 + row) * a.g.n_ch + sd.c0 + s;
      v0 = a.vis[2 * vidx];
      v1 = a.vis[2 * vidx + 1];
      if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);
    }
    const float vr[4] = {v0.x, v0.z, v1.x, v1.z}, vi[4] = {v0.y, v0.w, v1.y, v1.w};
    float4* step = base + tc_run_offset(nc, G * R + u) + kGtcHeaderFloat4 + st * kGtcStepFloat4;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int p = n >> 1;
      const float b0 = (n & 1) ? vi[p] : vr[p];
      const float b1 = (n & 1) ? vr[p] : -vi[p];
      float4 f;
      tc_split_store(b0, f.x, f.z);
      tc_split_store(b1, f.y, f.w);
      step[4 * n + t] = f;
    }
  }
  // one thread per (run, row slot): the phase coefficients of the run's first channel and of the channel step
  for (int idx = threadIdx.x; idx < NR * 4; idx += blockDim.x) {
    const int r = idx >> 2, t = idx & 3, G = r / R, u = r - G * R;
    const int row = tc_slot_row(seg, sd.seg_begin, sd.seg_count, nc, G, t);
    float4* hdr = base + tc_run_offset(nc, r);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    hdr[2 * t] = hdr[2 * t + 1] = hdr[8 + 2 * t] = hdr[9 + 2 * t] = z;
    if (row < 0) continue;
    const TcSlopes cu = tc_slopes(a, sd, sd.t0 + row, sd.c0 + u * kGtcRun, L);
    tc_put_coef(hdr + 2 * t, cu.a, cu.b, cu.w);
    if (nc > 1) {
      const TcSlopes c0 = tc_slopes(a, sd, sd.t0 + row, sd.c0, L);
      const TcSlopes c1 = tc_slopes(a, sd, sd.t0 + row, sd.c0 + 1, L);
      tc_put_coef(hdr + 8 + 2 * t, c1.a - c0.a, c1.b - c0.b, c1.w - c0.w);
    }
  }
}

struct GtcSmem {
  float4 rec[2][kGtcChunkRuns * kGtcRunFloat4];  // staged runs, double buffered
  float2 x[4 * kGtcPolStride];                    // [pol][pixel] FP32 sums of the current segment
  float2 img[4 * kGtcPolStride];                  // [pol][pixel] corrected image sum over segments
  float4 geo[8][4][8];                            // [warp][tile][g]: (n0, di0, dj0, dn) of pixel g's 8-block
  float dnd[8][4][8];                             // n'(pixel g + 8) - n'(pixel g)
  uint64_t bar[2];
};

__device__ __forceinline__ void mma_tf32_m16n8k8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Phases (radians) of pixel g (block geometry ga, offset g from the block's
// first pixel) and of pixel g + 8 for the coefficients (c0, c1): the exact
// reduction at the block's anchor, then FP32 increments
__device__ __forceinline__ float2 gtc_phase(float4 c0, float4 c1, float4 ga, float dnd, int g) {
  const float sh = fmaf(c0.x, ga.y, c0.y * ga.z);
  const float d1 = __fsub_rn(sh, round_nearest(sh));
  const float lo = fmaf(c1.x, ga.x, fmaf(c0.z, ga.y, c0.w * ga.z));
  const float rr = __fadd_rn(d1, lo);
  const float r0 = __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
  const float pa = fmaf(c1.z, ga.w, fmaf(c1.y, float(g - 4), r0));
  return make_float2(pa, fmaf(c1.z, dnd, fmaf(c1.y, 8.f, pa)));
}

template <int L>
__device__ __forceinline__ bool gridder_tc_item(const GridArgs& a, int item_idx, uint32_t& cg, GtcSmem& S) {
  const GridItem item = a.items[item_idx];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int nc = sd.c1 - sd.c0;
  const int R = tc_runs(nc);
  const int NR = tc_row_groups(a.seg, sd.seg_begin, sd.seg_count, nc) * R;  // runs
  const int n_chunks = (NR + kGtcChunkRuns - 1) / kGtcChunkRuns;
  const float4* rec_base = a.records + size_t(sd.rec_offset) * kRecordFloat4;
  const int P0 = item.tile * kGtcPixels;
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;

  auto issue = [&](int chunk, int buf) {
    const int r0 = chunk * kGtcChunkRuns, r1 = imin(r0 + kGtcChunkRuns, NR);
    const int64_t o0 = tc_run_offset(nc, r0);
    const uint32_t bytes = uint32_t(tc_run_offset(nc, r1) - o0) * 16;
    mbar_arrive_expect_tx(&S.bar[buf], bytes);
    bulk_copy_g2s(S.rec[buf], rec_base + o0, bytes, &S.bar[buf]);
  };
  if (tid == 0) {
    issue(0, int(cg & 1));
    if (n_chunks > 1) issue(1, int((cg + 1) & 1));
  }
  for (int e = tid; e < 4 * kGtcPolStride; e += 256) S.x[e] = S.img[e] = make_float2(0.f, 0.f);
  {
    // pixel geometry of the tiles: tid -> (warp, tile, g)
    const int w = tid >> 5, m = (tid >> 3) & 3, gg = tid & 7;
    const int pix = P0 + 64 * w + 16 * m + gg;
    const int j = pix / L, i = pix - j * L;
    const float4* bA = a.blk + (size_t(j) * (L / 8) + (i >> 3)) * 3;
    const float4 g0 = bA[0], dA4 = bA[1 + (gg >> 2)], g0b = bA[3], dB4 = bA[4 + (gg >> 2)];
    const float dnA = (gg & 3) == 0 ? dA4.x : (gg & 3) == 1 ? dA4.y : (gg & 3) == 2 ? dA4.z : dA4.w;
    const float dnB = (gg & 3) == 0 ? dB4.x : (gg & 3) == 1 ? dB4.y : (gg & 3) == 2 ? dB4.z : dB4.w;
    S.geo[w][m][gg] = make_float4(g0.x, g0.y, g0.z, dnA);
    S.dnd[w][m][gg] = (g0b.x + dnB) - (g0.x + dnA);
  }
  __syncthreads();

  float2 Cs[4], Sn[4], Rc[4], Rs[4];  // phasors of pixels (g, g + 8) of each tile, and of the channel step
  float acc[4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    Cs[m] = Rc[m] = make_float2(1.f, 1.f);
    Sn[m] = Rs[m] = make_float2(0.f, 0.f);
    acc[m][0] = acc[m][1] = acc[m][2] = acc[m][3] = 0.f;
  }
  auto flush = [&]() {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int pl = 64 * warp + 16 * m + g;
      float2& xa = S.x[t * kGtcPolStride + pl];
      float2& xb = S.x[t * kGtcPolStride + pl + 8];
      xa = make_float2(xa.x + acc[m][0], xa.y + acc[m][1]);
      xb = make_float2(xb.x + acc[m][2], xb.y + acc[m][3]);
      acc[m][0] = acc[m][1] = acc[m][2] = acc[m][3] = 0.f;
    }
  };
  // A_p^H X A_q, taper and centring sign of one segment, added to the image sum (warp `warp`'s 64 pixels)
  auto epilogue = [&](int seg_idx) {
    __syncwarp();
    const SegmentDesc seg = a.seg[sd.seg_begin + seg_idx];
    const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
    const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
    const bool diag = a.adiag[seg.interval * a.g.n_st + sd.p] && a.adiag[seg.interval * a.g.n_st + sd.q];
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int pl = 64 * warp + 32 * h + lane;
      const int pix = P0 + pl;
      const int j = pix / L, i = pix - j * L;
      Jones X;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float2 v = S.x[p * kGtcPolStride + pl];
        X.m[p] = {v.x, v.y};
        S.x[p * kGtcPolStride + pl] = make_float2(0.f, 0.f);
      }
      const NodeWeight wx = node_weight(i, nodes, L), wy = node_weight(j, nodes, L);
      Jones E;
      if (diag) {
        E = jdiag_ah_x_b(interp_diag_ldg(Ap, nodes, wx, wy), X, interp_diag_ldg(Aq, nodes, wx, wy));
      } else {
        const Jones Apj = interp_jones_ldg(Ap, nodes, wx, wy);
        const Jones Aqj = interp_jones_ldg(Aq, nodes, wx, wy);
        E = jmul_ah(Apj, jmul(X, Aqj));
      }
      const float wgt = a.taper[i] * a.taper[j] * (((i + j) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float2& o = S.img[p * kGtcPolStride + pl];
        o = make_float2(fmaf(wgt, E.m[p].re, o.x), fmaf(wgt, E.m[p].im, o.y));
      }
    }
    __syncwarp();
  };

  int seg_i = 0;
  int seg_gend = 0;  // first row group after segment seg_i
  {
    const SegmentDesc d0 = a.seg[sd.seg_begin];
    seg_gend = ((d0.k_end - d0.k_begin) / nc + 3) / 4;
  }
  int G = 0, u = 0;  // row group and run (within the row group) of the next run
  for (int c = 0; c < n_chunks; ++c) {
    const uint32_t cc_g = cg + uint32_t(c);
    const int buf = int(cc_g & 1);
    const bool ok = mbar_wait_bounded(&S.bar[buf], (cc_g >> 1) & 1);
    if (ok) {
      const int nr = imin(kGtcChunkRuns, NR - c * kGtcChunkRuns);
      const float4* run = S.rec[buf];
#pragma unroll 1
      for (int h = 0; h < nr; ++h) {
        const int len = tc_run_len(nc, u);
        if (u == 0 && G == seg_gend) {  // the previous segment is complete
          flush();
          epilogue(seg_i);
          ++seg_i;
          const SegmentDesc d = a.seg[sd.seg_begin + seg_i];
          seg_gend += ((d.k_end - d.k_begin) / nc + 3) / 4;
        }
        {
          // exact anchors at the run's first channel; the channel step's phasor once per row group
          const float4 a0 = run[2 * t], a1 = run[2 * t + 1];
          const bool first = u == 0;
          const float4 s0 = run[8 + 2 * t], s1 = run[9 + 2 * t];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float4 ga = S.geo[warp][m][g];
            const float dd = S.dnd[warp][m][g];
            const float2 ph = gtc_phase(a0, a1, ga, dd, g);
            __sincosf(ph.x, &Sn[m].x, &Cs[m].x);
            __sincosf(ph.y, &Sn[m].y, &Cs[m].y);
            if (first) {
              const float2 dph = gtc_phase(s0, s1, ga, dd, g);
              __sincosf(dph.x, &Rs[m].x, &Rc[m].x);
              __sincosf(dph.y, &Rs[m].y, &Rc[m].y);
            }
          }
        }
        const float4* steps = run + kGtcHeaderFloat4;
        auto step = [&](int st) {
          if (st > 0) {
            // next channel: e^{i phi} <- e^{i phi} e^{i dphi}
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const float2 cn = ffma2(make_float2(-Sn[m].x, -Sn[m].y), Rs[m], fmul2(Cs[m], Rc[m]));
              Sn[m] = ffma2(Sn[m], Rc[m], fmul2(Cs[m], Rs[m]));
              Cs[m] = cn;
            }
          }
          // B fragment: visibility t of the step, column g
          const float4 bf = steps[st * kGtcStepFloat4 + lane];
          const uint32_t Bh[2] = {__float_as_uint(bf.x), __float_as_uint(bf.y)};
          const uint32_t Bl[2] = {__float_as_uint(bf.z), __float_as_uint(bf.w)};
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            // A fragment: (row g, col t) cos, (row g+8, col t) cos, (row g, col t+4) sin, (row g+8, col t+4) sin
            uint32_t Ah[4], Al[4];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float2 x = e ? Sn[m] : Cs[m];
              Ah[2 * e] = __float_as_uint(x.x) & kGtcMask;
              Ah[2 * e + 1] = __float_as_uint(x.y) & kGtcMask;
              const float2 lo = ffma2(make_float2(__uint_as_float(Ah[2 * e]), __uint_as_float(Ah[2 * e + 1])),
                                      make_float2(-1.f, -1.f), x);  // x - hi
              Al[2 * e] = __float_as_uint(lo.x);
              Al[2 * e + 1] = __float_as_uint(lo.y);
            }
            mma_tf32_m16n8k8(acc[m], Ah, Bh);
            mma_tf32_m16n8k8(acc[m], Al, Bh);
            mma_tf32_m16n8k8(acc[m], Ah, Bl);
          }
        };
        if (len == kGtcRun) {  // a whole run, fully unrolled
#pragma unroll
          for (int st = 0; st < kGtcRun; ++st) step(st);
        } else {  // the last run of a row group: the remaining channels
#pragma unroll 1
          for (int st = 0; st < len; ++st) step(st);
        }
        run += kGtcHeaderFloat4 + len * kGtcStepFloat4;
        flush();  // every run: bounds the MMA accumulation chains
        if (++u == R) {
          u = 0;
          ++G;
        }
      }
    }
    // every thread is done with this buffer: refill it with chunk c + 2
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.status, kStatusTimeout);
        mbar_wait_bounded(&S.bar[buf], (cc_g >> 1) & 1);
        mbar_wait_bounded(&S.bar[buf ^ 1], ((cc_g + 1) >> 1) & 1);
      }
      return false;
    }
    if (tid == 0 && c + 2 < n_chunks) {
      fence_proxy_async();
      issue(c + 2, buf);
    }
  }
  epilogue(seg_i);

  // ---- write this block's pixels of the subgrid image: [sg][pol][j][i]; Stokes I: plane 0, (XX + YY) / 2
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int pl = 64 * warp + 32 * h + lane;
    const int pix = P0 + pl;
    float2* dst = a.scratch + size_t(item.sg) * 4 * L * L + pix;
    if (a.g.npol == 1) {
      const float2 xx = S.img[pl], yy = S.img[3 * kGtcPolStride + pl];
      dst[0] = make_float2(0.5f * (xx.x + yy.x), 0.5f * (xx.y + yy.y));
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) dst[size_t(p) * L * L] = S.img[p * kGtcPolStride + pl];
    }
  }
  cg += uint32_t(n_chunks);
  return true;
}

template <int L, bool PERSIST>
__global__ void __launch_bounds__(256, 2) gridder_tc_kernel(const GridArgs a) {
  extern __shared__ float4 smem_raw[];
  GtcSmem& S = *reinterpret_cast<GtcSmem*>(smem_raw);
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  if constexpr (!PERSIST) {
    gridder_tc_item<L>(a, blockIdx.x, cg, S);
  } else {
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
      __syncthreads();
      const int it = s_item;
      if (it >= a.n_items) return;
      if (!gridder_tc_item<L>(a, it, cg, S)) return;
      __syncthreads();  // shared memory and s_item free for the next item
    }
  }
}

// One launch over the items of several plans (items = (plan slot, item index))
template <int L>
__global__ void __launch_bounds__(256, 2) gridder_tc_multi_kernel(const GridArgs* args, const int2* items) {
  __shared__ __align__(16) unsigned char s_args_raw[sizeof(GridArgs)];
  extern __shared__ float4 smem_raw[];
  GtcSmem& S = *reinterpret_cast<GtcSmem*>(smem_raw);
  const int2 it = items[blockIdx.x];
  if (threadIdx.x == 0) {
    memcpy(s_args_raw, args + it.x, sizeof(GridArgs));
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  gridder_tc_item<L>(*reinterpret_cast<const GridArgs*>(s_args_raw), it.y, cg, S);
}

template <int L>
int configure_gridder_tc_l(int* persistent_blocks) {
  const int smem = int(sizeof(GtcSmem));
  cudaError_t e = cudaFuncSetAttribute(gridder_tc_kernel<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gridder_tc_kernel<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gridder_tc_multi_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gridder_tc_kernel<L, true>, 256, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L>
int launch_gridder_tc_l(const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
  if (n_items <= 0) return 0;
  const size_t smem = sizeof(GtcSmem);
  if (persistent_blocks > 0)
    gridder_tc_kernel<L, true><<<persistent_blocks < n_items ? persistent_blocks : n_items, 256, smem,
                                 cudaStream_t(stream)>>>(a);
  else
    gridder_tc_kernel<L, false><<<n_items, 256, smem, cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

template <int L>
int launch_gridder_tc_multi_l(const GridArgs* args, const int2* items, int n_items, void* stream) {
  if (n_items <= 0) return 0;
  gridder_tc_multi_kernel<L><<<n_items, 256, sizeof(GtcSmem), cudaStream_t(stream)>>>(args, items);
  return int(cudaGetLastError());
}

template <int L>
int launch_stage_tc_l(const StageArgs& a, const SegmentDesc* seg, int n_subgrids, void* stream) {
  if (n_subgrids <= 0) return 0;
  stage_tc_kernel<L><<<n_subgrids, 256, 0, cudaStream_t(stream)>>>(a, seg);
  return int(cudaGetLastError());
}

}  // namespace idg

