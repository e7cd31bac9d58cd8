// idg_grid_noalloc: gridding that allocates no memory per call.
//
// Some callers cannot allocate device memory at the point where they grid:
// real-time pipelines that reserve all memory at start-up and forbid
// allocation afterwards (cudaMalloc and cudaFree may synchronise the device
// and take unbounded time), and hosts whose device memory is owned by
// another allocator (a framework's caching pool) with no room left for a
// second one.  This entry point grids with an existing device plan but keeps
// its subgrid images in a fixed static device buffer instead of plan- or
// call-owned scratch; it calls no cudaMalloc, cudaFree or other allocating
// routine.
//
// The buffer (kNoAllocScratchBytes) lives as long as the library is loaded
// on every GPU that loads it.  Subgrids are gridded in sub-batches whose
// images fit the buffer.  Every call uses the same buffer and leaves its last
// sub-batch in it; each sub-batch overwrites every image element before the
// FFT reads it, so nothing needs clearing.  Two calls that overlap on the GPU
// (different streams, or different host threads) race on the buffer.
//
// Host code must not use the array's name as a device address (in host code
// it names a host-side stand-in); the device address is obtained once per
// device with cudaGetSymbolAddress, with that device current, during the
// first call on it -- so make that first call before any stream capture.
#include <mutex>

#include "kernels_common.cuh"

namespace idg {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB of subgrid images
static __device__ __align__(256) float2 g_noalloc_images[kNoAllocScratchBytes / sizeof(float2)];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_images on the current device (set-up once per device).
idg_status noalloc_scratch(void** out, std::string* err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = std::string("idg_grid_noalloc: no usable current device: ") + cudaGetErrorString(e);
    return IDG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_images);
    if (e != cudaSuccess || !ptr) {
      *err = std::string("idg_grid_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return IDG_ERR_CUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return IDG_OK;
}

}  // namespace

// Gridder variant: one block per (subgrid of the sub-batch, row tile), taken
// from the block index; visibilities are staged into shared memory by the
// block itself; images go to g_noalloc_images.  The arithmetic is the same as
// gridder_kernel's (phasor sum per Eq. 10, A-term per segment per Section 3.3).
template <int L, int ROWS>
__global__ void __launch_bounds__(ROWS * L / 8, (ROWS * L / 8) <= 128 ? 3 : 2)
    noalloc_gridder_kernel(const GridArgs a, int tiles) {
  constexpr int TPR = L / 8, NT = ROWS * TPR, VC = 64, REC = 8;
  extern __shared__ float4 smem[];
  float4* s_vis = smem;                                           // [VC][8]
  float* s_acc = reinterpret_cast<float*>(s_vis + VC * REC);      // [64][NT]

  const int sgi = blockIdx.x / tiles, tile = blockIdx.x % tiles;
  const SubgridDesc sd = a.sg[sgi];
  const int tid = threadIdx.x;
  const int j = tile * ROWS + tid / TPR;
  const int ib = tid % TPR;
  const int i0 = ib * 8;
  const int nodes = a.g.nodes;
  const int nA = nodes * nodes * 4;
  const float4* bg = a.blk + (size_t(j) * TPR + ib) * 3;
  const float4 g0 = bg[0], g1 = bg[1], g2 = bg[2];
  const float n0 = g0.x;
  const float2 DN[4] = {{g1.x, g1.y}, {g1.z, g1.w}, {g2.x, g2.y}, {g2.z, g2.w}};
  const float di0 = g0.y, dj0 = g0.z;
  const float2 DI[4] = {{-4.f, -3.f}, {-2.f, -1.f}, {0.f, 1.f}, {2.f, 3.f}};
  const int nc = sd.c1 - sd.c0;
  const double inv_l = 1.0 / double(L);
  const double off_x = double(sd.x0 + L / 2 - a.g.N / 2);
  const double off_y = double(sd.y0 + L / 2 - a.g.N / 2);

  // this thread's column of the image sums starts at zero, so a subgrid without segments writes zeros
#pragma unroll
  for (int e = 0; e < 64; ++e) s_acc[e * NT + tid] = 0.f;
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
    for (int kc = seg.k_begin; kc < seg.k_end; kc += VC) {
      const int nv = imin(VC, seg.k_end - kc);
      if (tid < nv) {
        const int k = kc + tid;
        const int t = sd.t0 + k / nc, ch = sd.c0 + k % nc;
        const size_t vidx = (size_t(sd.b) * a.g.n_t + t) * a.g.n_ch + ch;
        float4 v0 = a.vis[2 * vidx], v1 = a.vis[2 * vidx + 1];
        if (sd.flags & kSubgridMirrored) mirror_values(v0, v1);
        const double* r = a.uvw + (size_t(sd.b) * a.g.n_t + t) * 3;
        const double fs = subgrid_sign(sd) * a.fscale[ch];  // a mirrored subgrid sees (-u, -v, -w)
        const double dx = (r[0] * fs) * a.g.fov - off_x;
        const double dy = (r[1] * fs) * a.g.fov - off_y;
        const double w = r[2] * fs - subgrid_w0(a.g, sd);  // w - w0 (Section 2.4)
        const double aa = dx * inv_l, bb = dy * inv_l;
        const double ah = rint(aa * 65536.0) * (1.0 / 65536.0);
        const double bh = rint(bb * 65536.0) * (1.0 / 65536.0);
        float4* rec = s_vis + tid * REC;
        rec[0] = make_float4(v0.x, v0.x, v0.y, v0.y);
        rec[1] = make_float4(-v0.y, -v0.y, v0.z, v0.z);
        rec[2] = make_float4(v0.w, v0.w, -v0.w, -v0.w);
        rec[3] = make_float4(v1.x, v1.x, v1.y, v1.y);
        rec[4] = make_float4(-v1.y, -v1.y, v1.z, v1.z);
        rec[5] = make_float4(v1.w, v1.w, -v1.w, -v1.w);
        rec[6] = make_float4(float(ah), float(bh), float(aa - ah), float(bb - bh));
        rec[7] = make_float4(float(w), float(kTwoPi * aa), float(kTwoPi * w), 0.f);
      }
      __syncthreads();
#pragma unroll 1
      for (int v = 0; v < nv; ++v) {
        const float4* rec = s_vis + v * REC;
        const float4 cf = rec[6], cw = rec[7];
        const float sh = fmaf(cf.x, di0, cf.y * dj0);
        const float d1 = __fsub_rn(sh, round_nearest(sh));
        const float lo = fmaf(cw.x, n0, fmaf(cf.z, di0, cf.w * dj0));
        float rr = __fadd_rn(d1, lo);
        rr = __fmul_rn(__fsub_rn(rr, round_nearest(rr)), kTwoPiF);
        const float2 R0 = make_float2(rr, rr);
        const float2 ARR = make_float2(cw.y, cw.y), CRR = make_float2(cw.z, cw.z);
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
    const float2* Ap = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.p) * nA;
    const float2* Aq = a.aterms + (size_t(seg.interval) * a.g.n_st + sd.q) * nA;
    const NodeWeight wy = node_weight(j, nodes, L);
    const float tj = a.taper[j];
#pragma unroll
    for (int px = 0; px < 8; ++px) {
      const int i = i0 + px;
      const int q = px >> 1;
      const NodeWeight wx = node_weight(i, nodes, L);
      const Jones Apj = interp_jones_ldg(Ap, nodes, wx, wy);
      const Jones Aqj = interp_jones_ldg(Aq, nodes, wx, wy);
      Jones X;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        X.m[p].re = (px & 1) ? RE[p][q].y : RE[p][q].x;
        X.m[p].im = (px & 1) ? IM[p][q].y : IM[p][q].x;
      }
      const Jones E = jmul_ah(Apj, jmul(X, Aqj));
      const float wgt = a.taper[i] * tj * (((i + j) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float* acc = s_acc + (px * 8 + 2 * p) * NT + tid;
        acc[0] += wgt * E.m[p].re;
        acc[NT] += wgt * E.m[p].im;
      }
    }
  }
  // the sub-batch's images live in the static buffer, named directly here
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float4* dst = reinterpret_cast<float4*>(g_noalloc_images + ((size_t(sgi) * 4 + p) * L + j) * L + i0);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int px = 2 * h;
      dst[h] = make_float4(s_acc[(px * 8 + 2 * p) * NT + tid], s_acc[(px * 8 + 2 * p + 1) * NT + tid],
                           s_acc[((px + 1) * 8 + 2 * p) * NT + tid], s_acc[((px + 1) * 8 + 2 * p + 1) * NT + tid]);
    }
  }
}

template <int L, int ROWS>
static int noalloc_grid_t(const PlanDeviceView& v, const void* vis, const void* aterms, void* grid, void* scratch) {
  constexpr int NT = ROWS * L / 8;
  constexpr int tiles = L / ROWS;
  const size_t per_sg = size_t(4) * L * L * sizeof(float2);
  const int cap = int(kNoAllocScratchBytes / per_sg);
  const size_t smem = sizeof(float4) * 64 * 8 + sizeof(float) * 64 * NT;
  cudaError_t e = cudaFuncSetAttribute(noalloc_gridder_kernel<L, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return int(e);
  const cudaStream_t st = cudaStream_t(v.stream);
  for (int s0 = 0; s0 < v.n_sg; s0 += cap) {
    const int n = cap < v.n_sg - s0 ? cap : v.n_sg - s0;
    GridArgs ga{};
    ga.vis = static_cast<const float4*>(vis);
    ga.uvw = v.uvw;
    ga.fscale = v.fscale;
    ga.aterms = static_cast<const float2*>(aterms);
    ga.sg = v.sg + s0;
    ga.seg = v.seg;
    ga.taper = v.taper;
    ga.blk = v.blk;
    ga.g = v.g;
    noalloc_gridder_kernel<L, ROWS><<<n * tiles, NT, smem, st>>>(ga, tiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) return int(e);
    FftArgs fa{v.sg + s0, static_cast<float2*>(scratch), static_cast<double2*>(grid), v.twiddle, v.g.N};
    const int r = launch_fft_adder(L, fa, n, 0, v.stream);
    if (r) return r;
  }
  return 0;
}

}  // namespace idg

using namespace idg;

extern "C" idg_status idg_grid_noalloc(idg_plan* plan, const void* vis_c64, const void* aterms_c64,
                                       void* grid_c128) {
  PlanDeviceView v{};
  if (!plan_device_view(plan, &v))
    return plan ? plan_set_error(plan, IDG_ERR_INVALID_ARG, "idg_grid_noalloc needs a device plan")
                : plan_set_error(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  const void* ptrs[3] = {vis_c64, aterms_c64, grid_c128};
  for (const void* p : ptrs)
    if (!p || reinterpret_cast<uintptr_t>(p) % 16)
      return plan_set_error(plan, IDG_ERR_INVALID_ARG, "idg_grid_noalloc: NULL or misaligned buffer");
  if (v.flags & (IDG_NORMALIZE_ATERM | IDG_STOKES_I))
    return plan_set_error(plan, IDG_ERR_UNSUPPORTED,
                          "idg_grid_noalloc grids the 4 correlation planes without A-term normalisation");
  const size_t per_sg = size_t(4) * v.g.L * v.g.L * sizeof(float2);
  if (per_sg > kNoAllocScratchBytes)
    return plan_set_error(plan, IDG_ERR_UNSUPPORTED,
                          "idg_grid_noalloc: one subgrid image exceeds the 32 MiB static scratch buffer");
  void* scratch = nullptr;
  std::string err;
  const idg_status st = noalloc_scratch(&scratch, &err);
  if (st != IDG_OK) return plan_set_error(plan, st, err.c_str());
  int e = 0;
  switch (v.g.L) {
    case 32: e = noalloc_grid_t<32, 32>(v, vis_c64, aterms_c64, grid_c128, scratch); break;
    case 64: e = noalloc_grid_t<64, 16>(v, vis_c64, aterms_c64, grid_c128, scratch); break;
    case 96: e = noalloc_grid_t<96, 16>(v, vis_c64, aterms_c64, grid_c128, scratch); break;
    case 128: e = noalloc_grid_t<128, 8>(v, vis_c64, aterms_c64, grid_c128, scratch); break;
    default: return plan_set_error(plan, IDG_ERR_UNSUPPORTED, "idg_grid_noalloc: unsupported subgrid size");
  }
  if (e) {
    const std::string msg = std::string("idg_grid_noalloc: ") + cudaGetErrorName(cudaError_t(e)) + " (" +
                            cudaGetErrorString(cudaError_t(e)) + ")";
    return plan_set_error(plan, IDG_ERR_CUDA, msg.c_str());
  }
  return IDG_OK;
}
