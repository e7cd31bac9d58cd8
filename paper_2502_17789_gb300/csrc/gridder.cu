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

// ------------------------------------------------------------------ gridder dispatch

// the tensor-core gridder lives in gridder_tc_kernels.cuh, instantiated in gridder_tc_lNN.cu
template <int L>
int configure_gridder_tc_l(int* persistent_blocks);
template <int L>
int launch_gridder_tc_l(const GridArgs& a, int n_items, int persistent_blocks, void* stream);
template <int L>
int launch_gridder_tc_multi_l(const GridArgs* args, const int2* items, int n_items, void* stream);
template <int L>
int launch_stage_tc_l(const StageArgs& a, const SegmentDesc* seg, int n_subgrids, void* stream);
#define IDG_GRID_TC_EXTERN(L)                                                                                    \
  extern template int configure_gridder_tc_l<L>(int*);                                                          \
  extern template int launch_gridder_tc_l<L>(const GridArgs&, int, int, void*);                                 \
  extern template int launch_gridder_tc_multi_l<L>(const GridArgs*, const int2*, int, void*);                   \
  extern template int launch_stage_tc_l<L>(const StageArgs&, const SegmentDesc*, int, void*);
IDG_GRID_TC_EXTERN(32)
IDG_GRID_TC_EXTERN(64)
IDG_GRID_TC_EXTERN(96)
IDG_GRID_TC_EXTERN(128)
#undef IDG_GRID_TC_EXTERN

#define IDG_SWITCH_L(CALL)                 \
  switch (L) {                             \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 96: return CALL(96);              \
    case 128: return CALL(128);            \
    default: return int(cudaErrorInvalidValue); \
  }

int configure_gridder_tc(int L, int* persistent_blocks) {
#define C_(X) configure_gridder_tc_l<X>(persistent_blocks)
  IDG_SWITCH_L(C_)
#undef C_
}
int launch_gridder_tc(int L, const GridArgs& a, int n_items, int persistent_blocks, void* stream) {
#define C_(X) launch_gridder_tc_l<X>(a, n_items, persistent_blocks, stream)
  IDG_SWITCH_L(C_)
#undef C_
}
int launch_gridder_tc_multi(int L, const GridArgs* args, const int2* items, int n_items, void* stream) {
#define C_(X) launch_gridder_tc_multi_l<X>(args, items, n_items, stream)
  IDG_SWITCH_L(C_)
#undef C_
}
int launch_stage_tc(int L, const StageArgs& a, const SegmentDesc* seg, int n_subgrids, void* stream) {
#define C_(X) launch_stage_tc_l<X>(a, seg, n_subgrids, stream)
  IDG_SWITCH_L(C_)
#undef C_
}
#undef IDG_SWITCH_L

// the kernels live in gridder_kernels.cuh, instantiated per subgrid size in gridder_lNN.cu
template <int L>
int gridder_launch(const GridArgs& a, int n_items, int persistent_blocks, void* stream);
template <int L>
int gridder_configure(int vc, int* persistent_blocks);
template <int L>
int gridder_launch_multi(const GridArgs* args, const int2* items, int n_items, bool norm, int vc, void* stream);
extern template int gridder_launch<32>(const GridArgs&, int, int, void*);
extern template int gridder_launch<64>(const GridArgs&, int, int, void*);
extern template int gridder_launch<96>(const GridArgs&, int, int, void*);
extern template int gridder_launch<128>(const GridArgs&, int, int, void*);
extern template int gridder_configure<32>(int, int*);
extern template int gridder_configure<64>(int, int*);
extern template int gridder_configure<96>(int, int*);
extern template int gridder_configure<128>(int, int*);
extern template int gridder_launch_multi<32>(const GridArgs*, const int2*, int, bool, int, void*);
extern template int gridder_launch_multi<64>(const GridArgs*, const int2*, int, bool, int, void*);
extern template int gridder_launch_multi<96>(const GridArgs*, const int2*, int, bool, int, void*);
extern template int gridder_launch_multi<128>(const GridArgs*, const int2*, int, bool, int, void*);

bool supported_grid_chunk(int vc) { return vc == 32 || vc == 48 || vc == 64; }

int launch_gridder_multi(int L, const GridArgs* args, const int2* items, int n_items, bool norm, int vc,
                         void* stream) {
  switch (L) {
    case 32: return gridder_launch_multi<32>(args, items, n_items, norm, vc, stream);
    case 64: return gridder_launch_multi<64>(args, items, n_items, norm, vc, stream);
    case 96: return gridder_launch_multi<96>(args, items, n_items, norm, vc, stream);
    case 128: return gridder_launch_multi<128>(args, items, n_items, norm, vc, stream);
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
    case 32: return gridder_launch<32>(a, n_items, persistent_blocks, stream);
    case 64: return gridder_launch<64>(a, n_items, persistent_blocks, stream);
    case 96: return gridder_launch<96>(a, n_items, persistent_blocks, stream);
    case 128: return gridder_launch<128>(a, n_items, persistent_blocks, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int configure_gridder(int L, int vc, int* persistent_blocks) {
  switch (L) {
    case 32: return gridder_configure<32>(vc, persistent_blocks);
    case 64: return gridder_configure<64>(vc, persistent_blocks);
    case 96: return gridder_configure<96>(vc, persistent_blocks);
    case 128: return gridder_configure<128>(vc, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}

bool supported_subgrid_size(int L) { return gridder_rows(L) > 0; }

}  // namespace idg
