// Gridder kernel: Section 2.5 imaging step 2a (Eq. 10) plus the deferred
// A-term of Section 3.3.
//
// For subgrid s with corner (x0, y0) and pixel (i, j):
//   X(i,j) = (-1)^(i+j) T_i T_j sum_g A_p,g(i,j)^H [ sum_{k in g} V_k e^{2 pi i phi_k(i,j)} ] A_q,g(i,j)
//   phi_k  = a_k (i - L/2) + b_k (j - L/2) + w_k n'(i,j)            (turns)
//   a_k    = (xi_k - x0 - L/2) / L = (u_k - u0) FOV / L,  b_k likewise
// The (-1)^(i+j) factor lets the subgrid FFT run uncentred.
//
// Work item = (subgrid, tile of ROWS rows).  Each thread owns 8 consecutive
// pixels of one row.  Visibilities are staged in shared memory in chunks;
// staging computes a_k, b_k, w_k in FP64 (the per-visibility subgrid offset)
// and splits a_k, b_k into a 16-fractional-bit head and a small tail, so
// that the anchor phase a_k di0 + b_k dj0 of a thread is range-reduced
// exactly in FP32.  The 8 pixel phases are anchor + FP32 increments, the
// phasors come from __sincosf, and the 4-polarisation complex
// multiply-accumulate runs as packed f32x2 FMAs over pixel pairs.
#include "kernels_common.cuh"

namespace idg {

template <int L, int ROWS>
struct GridCfg {
  static constexpr int TPR = L / 8;         // threads per row
  static constexpr int NT = ROWS * TPR;     // threads per block
  static constexpr int VC = 64;             // visibilities per staged chunk
  static constexpr int REC = 9;             // float4 per staged visibility
  static constexpr int MINB = NT <= 128 ? 3 : (NT <= 192 ? 2 : 1);
  static_assert(L % 8 == 0 && L % ROWS == 0 && NT >= VC, "gridder shape");
};

template <int L, int ROWS>
__global__ void __launch_bounds__(GridCfg<L, ROWS>::NT, GridCfg<L, ROWS>::MINB)
    gridder_kernel(const GridArgs a) {
  using C = GridCfg<L, ROWS>;
  extern __shared__ float4 smem[];
  float4* s_vis = smem;                                      // [VC][REC]
  float* s_acc = reinterpret_cast<float*>(s_vis + C::VC * C::REC);  // [64][NT]
  float2* s_A = reinterpret_cast<float2*>(s_acc + 64 * C::NT);      // [2][nodes*nodes*4]

  const GridItem item = a.items[blockIdx.x];
  const SubgridDesc sd = a.sg[item.sg];
  const int tid = threadIdx.x;
  const int j = item.tile * ROWS + tid / C::TPR;
  const int ib = tid % C::TPR;
  const int i0 = ib * 8;
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;

  // pixel geometry of this thread's block: anchor at i0 + 4
  const float4* bg = a.blk + (size_t(j) * C::TPR + ib) * 3;
  const float4 g0 = bg[0], g1 = bg[1], g2 = bg[2];
  const float n0 = g0.x;
  const float2 DN[4] = {{g0.y, g0.z}, {g0.w, g1.x}, {g1.y, g1.z}, {g1.w, g2.x}};
  const float di0 = g2.y, dj0 = g2.z;
  const float2 DI[4] = {{-4.f, -3.f}, {-2.f, -1.f}, {0.f, 1.f}, {2.f, 3.f}};

  const int nc = sd.c1 - sd.c0;
  const double inv_l = 1.0 / double(L);
  const double off_x = double(sd.x0 + L / 2 - a.g.N / 2);
  const double off_y = double(sd.y0 + L / 2 - a.g.N / 2);

  for (int gi = 0; gi < sd.seg_count; ++gi) {
    const SegmentDesc seg = a.seg[sd.seg_begin + gi];
    float2 RE[4][4], IM[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        RE[p][q] = make_float2(0.f, 0.f);
        IM[p][q] = make_float2(0.f, 0.f);
      }

    for (int kc = seg.k_begin; kc < seg.k_end; kc += C::VC) {
      const int nv = imin(C::VC, seg.k_end - kc);
      if (tid < nv) {
        // ---- stage one visibility (FP64 offset, FP32 record)
        const int k = kc + tid;
        const int t = sd.t0 + k / nc, ch = sd.c0 + k % nc;
        const size_t vidx = (size_t(sd.b) * a.g.n_t + t) * a.g.n_ch + ch;
        const float4 v0 = a.vis[2 * vidx], v1 = a.vis[2 * vidx + 1];
        const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
        const double fs = a.fscale[ch];
        const double dx = (r[0] * fs) * a.g.fov - off_x;
        const double dy = (r[1] * fs) * a.g.fov - off_y;
        const double w = r[2] * fs;
        const double aa = dx * inv_l, bb = dy * inv_l;
        const double ah = rint(aa * 65536.0) * (1.0 / 65536.0);
        const double bh = rint(bb * 65536.0) * (1.0 / 65536.0);
        float4* rec = s_vis + tid * C::REC;
        rec[0] = make_float4(v0.x, v0.x, v0.y, v0.y);
        rec[1] = make_float4(-v0.y, -v0.y, v0.z, v0.z);
        rec[2] = make_float4(v0.w, v0.w, -v0.w, -v0.w);
        rec[3] = make_float4(v1.x, v1.x, v1.y, v1.y);
        rec[4] = make_float4(-v1.y, -v1.y, v1.z, v1.z);
        rec[5] = make_float4(v1.w, v1.w, -v1.w, -v1.w);
        rec[6] = make_float4(float(ah), float(bh), float(aa - ah), float(bb - bh));
        rec[7] = make_float4(float(w), 0.f, 0.f, 0.f);
        const float ar = float(kTwoPi * aa), cr = float(kTwoPi * w);
        rec[8] = make_float4(ar, ar, cr, cr);
      }
      __syncthreads();

      // ---- phasor sum over the chunk
#pragma unroll 1
      for (int v = 0; v < nv; ++v) {
        const float4* rec = s_vis + v * C::REC;
        const float4 cf = rec[6];
        const float cw = rec[7].x;
        const float4 cr = rec[8];
        // anchor phase in turns: head part exact, then two range reductions
        const float sh = fmaf(cf.x, di0, cf.y * dj0);
        const float d1 = __fsub_rn(sh, round_nearest(sh));
        const float lo = fmaf(cw, n0, fmaf(cf.z, di0, cf.w * dj0));
        float rr = __fadd_rn(d1, lo);
        rr = __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
        const float2 R0 = make_float2(rr, rr);
        const float2 ARR = make_float2(cr.x, cr.y), CRR = make_float2(cr.z, cr.w);
        float2 Cs[4], Sn[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 ph = ffma2(CRR, DN[q], ffma2(ARR, DI[q], R0));
          __sincosf(ph.x, &Sn[q].x, &Cs[q].x);
          __sincosf(ph.y, &Sn[q].y, &Cs[q].y);
        }
        const float4 f0 = rec[0], f1 = rec[1], f2 = rec[2], f3 = rec[3], f4 = rec[4], f5 = rec[5];
        const float2 VRR[4] = {{f0.x, f0.y}, {f1.z, f1.w}, {f3.x, f3.y}, {f4.z, f4.w}};
        const float2 VII[4] = {{f0.z, f0.w}, {f2.x, f2.y}, {f3.z, f3.w}, {f5.x, f5.y}};
        const float2 NVI[4] = {{f1.x, f1.y}, {f2.z, f2.w}, {f4.x, f4.y}, {f5.z, f5.w}};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            RE[p][q] = ffma2(VRR[p], Cs[q], RE[p][q]);
            RE[p][q] = ffma2(NVI[p], Sn[q], RE[p][q]);
            IM[p][q] = ffma2(VRR[p], Sn[q], IM[p][q]);
            IM[p][q] = ffma2(VII[p], Cs[q], IM[p][q]);
          }
      }
      __syncthreads();
    }

    // ---- epilogue: A_p^H X A_q, taper, centring sign (Section 3.3)
    {
      const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
      const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
      for (int e = tid; e < nA; e += C::NT) {
        s_A[e] = Ap[e];
        s_A[nA + e] = Aq[e];
      }
    }
    __syncthreads();
    const NodeWeight wy = node_weight(j, nodes, L);
    const float tj = a.taper[j];
#pragma unroll
    for (int px = 0; px < 8; ++px) {
      const int i = i0 + px;
      const int q = px >> 1;
      Jones X;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        X.m[p].re = (px & 1) ? RE[p][q].y : RE[p][q].x;
        X.m[p].im = (px & 1) ? IM[p][q].y : IM[p][q].x;
      }
      const NodeWeight wx = node_weight(i, nodes, L);
      const Jones Apj = interp_jones(s_A, nodes, wx, wy);
      const Jones Aqj = interp_jones(s_A + nA, nodes, wx, wy);
      const Jones E = jmul_ah(Apj, jmul(X, Aqj));
      const float wgt = a.taper[i] * tj * (((i + j) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float* acc = s_acc + (px * 8 + 2 * p) * C::NT + tid;
        if (gi == 0) {
          acc[0] = wgt * E.m[p].re;
          acc[C::NT] = wgt * E.m[p].im;
        } else {
          acc[0] += wgt * E.m[p].re;
          acc[C::NT] += wgt * E.m[p].im;
        }
      }
    }
    __syncthreads();
  }

  // ---- write the subgrid image rows: [sg][pol][j][i]
  if (sd.seg_count > 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float4* dst = reinterpret_cast<float4*>(a.scratch + ((size_t(item.sg) * 4 + p) * L + j) * L + i0);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int px = 2 * h;
        dst[h] = make_float4(s_acc[(px * 8 + 2 * p) * C::NT + tid], s_acc[(px * 8 + 2 * p + 1) * C::NT + tid],
                             s_acc[((px + 1) * 8 + 2 * p) * C::NT + tid],
                             s_acc[((px + 1) * 8 + 2 * p + 1) * C::NT + tid]);
      }
    }
  }
}

template <int L, int ROWS>
static size_t gridder_smem(int nodes) {
  using C = GridCfg<L, ROWS>;
  return sizeof(float4) * C::VC * C::REC + sizeof(float) * 64 * C::NT + sizeof(float2) * 2 * nodes * nodes * 4;
}

template <int L, int ROWS>
static int launch_gridder_t(const GridArgs& a, int n_items, void* stream) {
  using C = GridCfg<L, ROWS>;
  const size_t smem = gridder_smem<L, ROWS>(a.g.nodes);
  cudaError_t e = cudaFuncSetAttribute(gridder_kernel<L, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  if (n_items <= 0) return 0;
  gridder_kernel<L, ROWS><<<n_items, C::NT, smem, cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

// rows per gridder tile for each supported subgrid size
int gridder_rows(int L) {
  switch (L) {
    case 32: return 32;
    case 64: return 16;
    case 96: return 16;
    case 128: return 8;
    default: return 0;
  }
}

int launch_gridder(int L, const GridArgs& a, int n_items, void* stream) {
  switch (L) {
    case 32: return launch_gridder_t<32, 32>(a, n_items, stream);
    case 64: return launch_gridder_t<64, 16>(a, n_items, stream);
    case 96: return launch_gridder_t<96, 16>(a, n_items, stream);
    case 128: return launch_gridder_t<128, 8>(a, n_items, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

bool supported_subgrid_size(int L) { return gridder_rows(L) > 0; }

}  // namespace idg
