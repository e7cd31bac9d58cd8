// Gridder: Section 2.5 imaging step 2a (Eq. 10) plus the deferred A-term of
// Section 3.3.
//
// For subgrid s with corner (x0, y0) and pixel (i, j):
//   X(i,j) = (-1)^(i+j) T_i T_j sum_g A_p,g(i,j)^H [ sum_{k in g} V_k e^{2 pi i phi_k(i,j)} ] A_q,g(i,j)
//   phi_k  = a_k (i - L/2) + b_k (j - L/2) + w_k n'(i,j)            (turns)
//   a_k    = (xi_k - x0 - L/2) / L = (u_k - u0) FOV / L,  b_k likewise
// The (-1)^(i+j) factor lets the subgrid FFT run uncentred.
//
// Two kernels per batch of subgrids:
//  * stage_records_kernel writes every member visibility of the batch, in
//    subgrid member order, as a 128-byte record: the 4 complex values as the
//    operand pairs of the packed multiply-accumulate, and the phase slopes
//    computed in FP64 from uvw and the subgrid offset.  a_k and b_k are split
//    into a head with 16 fractional bits and a tail, so a thread's anchor
//    phase a_k di0 + b_k dj0 is range-reduced exactly in FP32.
//  * gridder_kernel: work item = (subgrid, tile of ROWS rows), each thread
//    owns 8 consecutive pixels of one row.  Records stream into a double
//    buffer in shared memory by 1-D bulk copies (cp.async.bulk, completion on
//    an mbarrier), one chunk ahead of the phasor sum.  The 8 pixel phases are
//    the reduced anchor plus FP32 increments and the phasors come from
//    __sincosf, for the first channel of each run of kRotateRun channels of a
//    (baseline, time) row.  phi is linear in frequency, so the other channels
//    of the run rotate the previous phasors by the phasor of the channel step
//    (itself evaluated once per row the same way): one complex multiply per
//    pixel instead of a sine and a cosine.  The 4-polarisation complex
//    multiply-accumulate runs as packed f32x2 FMAs over pixel pairs.  After each A-term segment the
//    thread applies A_p^H X A_q, the taper and the centring sign and adds
//    the result into its private columns of a shared-memory image sum
//    (with the A-term power normalisation, divided by ||A_p^H A_q||_F per
//    pixel, whose weights n_seg / f go to the plan's weight map).
#include <type_traits>

#include "kernels_common.cuh"

namespace idg {

// ------------------------------------------------------------------ staging

// Phase slopes of a visibility: a = (xi - x0 - L/2) / L, b likewise, w (turns).
struct Slopes {
  double a, b, w;
};

__device__ __forceinline__ Slopes vis_slopes(const StageArgs& a, const SubgridDesc& sd, int t, int ch, int L) {
  const double inv_l = 1.0 / double(L);
  const double off_x = double(sd.x0 + L / 2 - a.g.N / 2);
  const double off_y = double(sd.y0 + L / 2 - a.g.N / 2);
  const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
  const double fs = subgrid_sign(sd) * a.fscale[ch];  // a mirrored subgrid sees (-u, -v, -w)
  const double dx = (r[0] * fs) * a.g.fov - off_x;
  const double dy = (r[1] * fs) * a.g.fov - off_y;
  return {dx * inv_l, dy * inv_l, r[2] * fs - subgrid_w0(a.g, sd)};  // w - w0 (Section 2.4)
}

// (head, tail) split of the slopes for the exact anchor reduction, plus the
// FP32 slopes of the per-pixel increments, and the record kind.
__device__ __forceinline__ void put_slopes(float4* rec, const Slopes& s, float kind) {
  const double ah = rint(s.a * 65536.0) * (1.0 / 65536.0);
  const double bh = rint(s.b * 65536.0) * (1.0 / 65536.0);
  rec[6] = make_float4(float(ah), float(bh), float(s.a - ah), float(s.b - bh));
  rec[7] = make_float4(float(s.w), float(kTwoPi * s.a), float(kTwoPi * s.w), kind);
}

__global__ void __launch_bounds__(256) stage_records_kernel(const StageArgs a, int L) {
  const SubgridDesc sd = a.sg[blockIdx.x];
  const int nc = sd.c1 - sd.c0;
  // channels c0 + 1 .. c0 + s_uniform all follow the same step as channel c0 + 1
  __shared__ int s_uniform;
  if (threadIdx.x == 0) {
    int u = nc > 1 ? 1 : 0;
    if (nc > 1) {
      const double step1 = a.fscale[sd.c0 + 1] - a.fscale[sd.c0];
      while (u + 1 < nc) {
        const double st = a.fscale[sd.c0 + u + 1] - a.fscale[sd.c0 + u];
        if (fabs(st - step1) > 1e-12 * fabs(step1)) break;
        ++u;
      }
    }
    s_uniform = u;
  }
  __syncthreads();
  const int uniform = s_uniform;
  for (int k = threadIdx.x; k < sd.n_vis; k += blockDim.x) {
    const int t = sd.t0 + k / nc, cc = k % nc, ch = sd.c0 + cc;
    const size_t vidx = (size_t(sd.b) * a.g.n_t + t) * a.g.n_ch + ch;
    float4 v0 = a.vis[2 * vidx], v1 = a.vis[2 * vidx + 1];
    if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);
    float4* rec = a.records + (size_t(sd.rec_offset) + k) * kRecordFloat4;
    rec[0] = make_float4(v0.x, v0.x, v0.y, v0.y);
    rec[1] = make_float4(-v0.y, -v0.y, v0.z, v0.z);
    rec[2] = make_float4(v0.w, v0.w, -v0.w, -v0.w);
    rec[3] = make_float4(v1.x, v1.x, v1.y, v1.y);
    rec[4] = make_float4(-v1.y, -v1.y, v1.z, v1.z);
    rec[5] = make_float4(v1.w, v1.w, -v1.w, -v1.w);
    // Phasors along a row of channels (fixed baseline and time) advance by
    // a constant factor while the channel step is constant: phi is linear in
    // frequency.  The first channel of every run of kRotateRun starts from
    // its own phase (kind 1).  The first step of a row carries the step's
    // slopes (kind 2), later steps equal to it repeat it (kind 0), and past
    // the first step that differs every step carries its own slopes.
    const Slopes cur = vis_slopes(a, sd, t, ch, L);
    if (cc % kRotateRun == 0) {
      put_slopes(rec, cur, kKindBase);
    } else if (cc >= 2 && cc <= uniform) {
      rec[6] = make_float4(0.f, 0.f, 0.f, 0.f);
      rec[7] = make_float4(0.f, 0.f, 0.f, kKindRotate);
    } else {
      const Slopes prev = vis_slopes(a, sd, t, ch - 1, L);
      put_slopes(rec, {cur.a - prev.a, cur.b - prev.b, cur.w - prev.w}, kKindStep);
    }
  }
}

// one warp per (interval, station): are all off-diagonal node entries zero?
__global__ void aterm_flags_kernel(const float2* aterms, uint8_t* flags, int n_pairs, int nodes) {
  const int pair = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= n_pairs) return;
  const float2* A = aterms + size_t(pair) * nodes * nodes * 4;
  bool diag = true;
  for (int n = lane; n < nodes * nodes; n += 32) {
    const float2 b = A[n * 4 + 1], c = A[n * 4 + 2];
    diag = diag && b.x == 0.f && b.y == 0.f && c.x == 0.f && c.y == 0.f;
  }
  diag = __all_sync(0xffffffffu, diag);
  if (lane == 0) flags[pair] = diag ? 1 : 0;
}

int launch_aterm_flags(const float2* aterms, uint8_t* flags, int n_int, int n_st, int nodes, void* stream) {
  const int n = n_int * n_st;
  if (n <= 0) return 0;
  aterm_flags_kernel<<<(n + 7) / 8, 256, 0, cudaStream_t(stream)>>>(aterms, flags, n, nodes);
  return int(cudaGetLastError());
}

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives on; when the limit passes it reports kStatusTimeout, as a kernel
// whose bulk copy never landed would.  No copy is in flight, so returning is
// safe.
__global__ void wait_selftest_kernel(int* status, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

int launch_wait_selftest(int* status, int64_t limit_ns, void* stream) {
  wait_selftest_kernel<<<1, 32, 0, cudaStream_t(stream)>>>(status, uint64_t(limit_ns));
  return int(cudaGetLastError());
}

int launch_stage_records(int L, const StageArgs& a, int n_subgrids, void* stream) {
  if (n_subgrids <= 0) return 0;
  stage_records_kernel<<<n_subgrids, 256, 0, cudaStream_t(stream)>>>(a, L);
  return int(cudaGetLastError());
}

// ------------------------------------------------------------------ gridder

template <int L, int ROWS>
struct GridCfg {
  static constexpr int PX = 8;           // consecutive pixels of a row per thread
  static constexpr int QN = PX / 2;      // pixel pairs per thread
  static constexpr int TPR = L / PX;     // threads per row
  static constexpr int NT = ROWS * TPR;  // threads per block
  static constexpr int VC_MAX = 64;      // records per chunk at most (the plan's grid_chunk, GridArgs::vc)
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
// NORM: A-term power normalisation (a.aweights set)
template <int L, int ROWS, bool NORM>
__device__ __forceinline__ bool gridder_item(const GridArgs& a, int item_idx, uint32_t& cg, float4* s_rec,
                                             float* s_acc, float* s_w, uint64_t* s_bar) {
  using C = GridCfg<L, ROWS>;
  const GridItem item = a.items[item_idx];
  const int VC = a.vc;  // records per chunk
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
template <int L, int ROWS, bool PERSIST, bool NORM>
__global__ void __launch_bounds__(GridCfg<L, ROWS>::NT, GridCfg<L, ROWS>::MINB)
    gridder_kernel(const GridArgs a) {
  using C = GridCfg<L, ROWS>;
  extern __shared__ float4 smem[];
  float4* s_rec = smem;                                                      // [2][vc][8]
  float* s_acc = reinterpret_cast<float*>(s_rec + 2 * a.vc * kRecordFloat4);  // [8 PX][NT]
  float* s_w = s_acc + 8 * C::PX * C::NT;                                      // [PX][NT] A-term weights
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_w + C::PX * C::NT);          // [2]
  int* s_item = reinterpret_cast<int*>(s_bar + 2);
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  if constexpr (!PERSIST) {
    gridder_item<L, ROWS, NORM>(a, blockIdx.x, cg, s_rec, s_acc, s_w, s_bar);
  } else {
  for (;;) {
    if (threadIdx.x == 0) *s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= a.n_items) return;
    if (!gridder_item<L, ROWS, NORM>(a, it, cg, s_rec, s_acc, s_w, s_bar)) return;
    __syncthreads();  // shared buffers and s_item free for the next item
  }
  }
}

// One launch over the work items of several plans (the serving loop's
// shared work queue): block b runs item items[b] = (plan slot, item index
// in that slot's batch), with the slot's arguments copied to shared memory
// first.  One item per block, in the order given (longest first).
template <int L, int ROWS, bool NORM>
__global__ void __launch_bounds__(GridCfg<L, ROWS>::NT, GridCfg<L, ROWS>::MINB)
    gridder_multi_kernel(const GridArgs* args, const int2* items) {
  using C = GridCfg<L, ROWS>;
  __shared__ GridArgs s_args;
  extern __shared__ float4 smem[];
  const int2 it = items[blockIdx.x];
  if (threadIdx.x == 0) s_args = args[it.x];
  __syncthreads();
  const GridArgs& a = s_args;
  float4* s_rec = smem;                                                      // [2][vc][8]
  float* s_acc = reinterpret_cast<float*>(s_rec + 2 * a.vc * kRecordFloat4);  // [8 PX][NT]
  float* s_w = s_acc + 8 * C::PX * C::NT;                                    // [PX][NT]
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_w + C::PX * C::NT);        // [2]
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t cg = 0;
  gridder_item<L, ROWS, NORM>(a, it.y, cg, s_rec, s_acc, s_w, s_bar);
}

template <int L, int ROWS>
static size_t gridder_smem(int vc) {
  using C = GridCfg<L, ROWS>;
  return sizeof(float4) * 2 * vc * kRecordFloat4 + sizeof(float) * 9 * C::PX * C::NT + 2 * sizeof(uint64_t) + 16;
}

// The shared-memory limit is set for the largest chunk, so plans with
// different chunks share the kernels; the occupancy (persistent grid size)
// follows this plan's chunk.
template <int L, int ROWS>
static int configure_gridder_t(int vc, int* persistent_blocks) {
  using C = GridCfg<L, ROWS>;
  const int smem_max = int(gridder_smem<L, ROWS>(C::VC_MAX));
  const int smem = int(gridder_smem<L, ROWS>(vc));
  const void* fns[4] = {reinterpret_cast<const void*>(gridder_kernel<L, ROWS, false, false>),
                        reinterpret_cast<const void*>(gridder_kernel<L, ROWS, true, false>),
                        reinterpret_cast<const void*>(gridder_kernel<L, ROWS, false, true>),
                        reinterpret_cast<const void*>(gridder_kernel<L, ROWS, true, true>)};
  cudaError_t e = cudaSuccess;
  for (const void* fn : fns)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gridder_kernel<L, ROWS, true, false>, C::NT, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *persistent_blocks = per_sm * sms;
  return int(e);
}

template <int L, int ROWS>
static int launch_gridder_t(const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
  using C = GridCfg<L, ROWS>;
  const size_t smem = gridder_smem<L, ROWS>(a.vc);
  if (n_items <= 0) return 0;
  const int pb = persistent_blocks < n_items ? persistent_blocks : n_items;
  cudaStream_t st = cudaStream_t(stream);
  if (a.aweights) {
    if (persistent_blocks > 0)
      gridder_kernel<L, ROWS, true, true><<<pb, C::NT, smem, st>>>(a);
    else
      gridder_kernel<L, ROWS, false, true><<<n_items, C::NT, smem, st>>>(a);
  } else {
    if (persistent_blocks > 0)
      gridder_kernel<L, ROWS, true, false><<<pb, C::NT, smem, st>>>(a);
    else
      gridder_kernel<L, ROWS, false, false><<<n_items, C::NT, smem, st>>>(a);
  }
  return int(cudaGetLastError());
}

template <int L, int ROWS>
static int launch_gridder_multi_t(const GridArgs* args, const int2* items, int n_items, bool norm, int max_vc,
                                  void* stream) {
  using C = GridCfg<L, ROWS>;
  if (n_items <= 0) return 0;
  const size_t smem = gridder_smem<L, ROWS>(max_vc);
  const auto fn = norm ? gridder_multi_kernel<L, ROWS, true> : gridder_multi_kernel<L, ROWS, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(gridder_smem<L, ROWS>(C::VC_MAX)));
  if (e != cudaSuccess) return int(e);
  fn<<<n_items, C::NT, smem, cudaStream_t(stream)>>>(args, items);
  return int(cudaGetLastError());
}

int launch_gridder_multi(int L, const GridArgs* args, const int2* items, int n_items, bool norm, int max_vc,
                         void* stream) {
  switch (L) {
    case 32: return launch_gridder_multi_t<32, 32>(args, items, n_items, norm, max_vc, stream);
    case 64: return launch_gridder_multi_t<64, 16>(args, items, n_items, norm, max_vc, stream);
    case 96: return launch_gridder_multi_t<96, 8>(args, items, n_items, norm, max_vc, stream);
    case 128: return launch_gridder_multi_t<128, 8>(args, items, n_items, norm, max_vc, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

// rows per gridder tile for each supported subgrid size
int gridder_rows(int L) {
  switch (L) {
    case 32: return 32;
    case 64: return 16;
    case 96: return 8;
    case 128: return 8;
    default: return 0;
  }
}

int launch_gridder(int L, const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
  switch (L) {
    case 32: return launch_gridder_t<32, 32>(a, n_items, persistent_blocks, stream);
    case 64: return launch_gridder_t<64, 16>(a, n_items, persistent_blocks, stream);
    case 96: return launch_gridder_t<96, 8>(a, n_items, persistent_blocks, stream);
    case 128: return launch_gridder_t<128, 8>(a, n_items, persistent_blocks, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int configure_gridder(int L, int vc, int* persistent_blocks) {
  switch (L) {
    case 32: return configure_gridder_t<32, 32>(vc, persistent_blocks);
    case 64: return configure_gridder_t<64, 16>(vc, persistent_blocks);
    case 96: return configure_gridder_t<96, 8>(vc, persistent_blocks);
    case 128: return configure_gridder_t<128, 8>(vc, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}

bool supported_subgrid_size(int L) { return gridder_rows(L) > 0; }

}  // namespace idg
