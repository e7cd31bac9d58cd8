// Internal types of libidg shared by the host planner, the API layer and the
// CUDA kernels.  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/idg.h"

namespace idg {

constexpr double kSpeedOfLight = 299792458.0;

// One subgrid (Section 2.2): the subtable [t0,t1) x [c0,c1) of baseline b,
// placed with corner (x0, y0) on the master grid.  64 bytes.
struct SubgridDesc {
  int32_t b, p, q;
  int32_t t0, t1, c0, c1;
  int32_t x0, y0;
  int32_t seg_begin, seg_count;  // into the segment table
  int32_t n_vis;
  int32_t flags;                 // kSubgridDropped | kSubgridMirrored
  int32_t plan_index;            // position in plan order
  int32_t rec_offset;            // first staged record of this subgrid within its batch
  int32_t layer;                 // w layer: k (w0 = (k + 1/2) w_step) in the partition, k - k_min on the device
};
static_assert(sizeof(SubgridDesc) == 64, "SubgridDesc layout");

// SubgridDesc::flags
constexpr int32_t kSubgridDropped = 1;   // outside the grid (IDG_DROP_OUT_OF_GRID): not gridded, degrids to 0
// w layers (Section 2.4, footnote): the subgrid holds rows with w < 0, taken
// as their mirrors V^H at (-u, -v, -w) on baseline (q, p); p and q of the
// descriptor are already swapped, the kernels negate uvw and conjugate-
// transpose the values they read (gridder) or write (degridder)
constexpr int32_t kSubgridMirrored = 2;

// The part of a subgrid that shares one A-term interval (Section 3.3).
// Members are enumerated t-major: k = (t - t0) * (c1 - c0) + (c - c0).
struct SegmentDesc {
  int32_t subgrid;   // plan index
  int32_t interval;
  int32_t k_begin, k_end;
};

// Gridder work item: one pixel tile of one subgrid of the current batch.
struct GridItem {
  int32_t sg;    // index into the batch's device subgrid table
  int32_t tile;  // row tile
};

// Degridder work item: up to degrid_lanes(C) lanes of one or two segments,
// a lane being a channel group -- up to C consecutive channels of one
// timestep row.  A subgrid row of nc channels has G = ceil(nc / C) groups,
// numbered row-major over the subgrid (group g = row * G + gi covers channels
// c0 + gi nc / G .. c0 + (gi + 1) nc / G - 1).  Groups [k_begin, k_mid) belong
// to segment `segment`, [k_mid, k_end) (if any) to segment `segment` + 1 of
// the same subgrid.  With C = 1 a group is one visibility.
struct DegridItem {
  int32_t sg;       // index into the batch's device subgrid table
  int32_t segment;  // global index of the first segment
  int32_t k_begin, k_mid, k_end;
  int32_t pad;
};

// lanes (channel groups) per degridder work item for C channels per lane
__host__ __device__ constexpr int degrid_lanes(int C) { return C == 1 ? 256 : 128; }
constexpr int kDefaultDegridChannels = 1;  // channels per degridder lane when the geometry leaves it 0
// staged visibility records per gridder chunk (bulk copy into shared memory):
// 32, 48 or 64 (supported_grid_chunk), one kernel instantiation each
constexpr int kDefaultGridChunk = 48;
constexpr int kMaxAtermNodes = 25;  // A-term samples per axis (bounds the degridder's shared memory)
constexpr int kDegridSegs = 2;  // segments per degridder work item
// degridder items of at most this many lanes run in the kernel that spreads a
// visibility over several lanes (low occupancy)
constexpr int kSplitLanes = 8;
constexpr int kTcItemRows = 256;  // rows (16-row tiles) per item of the tensor-core degridder

// channels per run of rotated phasors (one fresh evaluation per run bounds
// the growth of the rotation's rounding error)
constexpr int kRotateRun = 8;

// Tensor-core gridder: work items of kGtcPixels pixels; the staged records of
// a subgrid are its row groups (4 rows of one segment) times the runs of up
// to kGtcRun channels of a row group (the last run holds the remaining
// channels); a run is a header (the phase coefficients of the run's first
// channel and of the channel step for the 4 rows, 2 float4 each) followed by
// one step of 4 visibilities x 8 columns (one float4 per column) per channel
constexpr int kGtcPixels = 512;  // pixels per work item

// channels per run of rotated phasors in the tensor-core gridder: longer
// runs than the FP32 gridder's (fewer anchor evaluations per step), for a
// larger but bounded rotation error
constexpr int kGtcRun = 16;
__host__ __device__ constexpr int tc_runs(int nc) { return (nc + kGtcRun - 1) / kGtcRun; }
constexpr int kGtcHeaderFloat4 = 16;                                 // run header
constexpr int kGtcStepFloat4 = 32;                                   // one step: 8 columns x 4 rows
constexpr int kGtcRunFloat4 = kGtcHeaderFloat4 + kGtcRun * kGtcStepFloat4;  // the longest run
// float4s of one row group: a header per run and a step per channel (a multiple of 16)
__host__ __device__ constexpr int tc_group_float4(int nc) {
  return kGtcHeaderFloat4 * tc_runs(nc) + kGtcStepFloat4 * nc;
}
// channels of run u of a row group
__host__ __device__ constexpr int tc_run_len(int nc, int u) {
  return nc - u * kGtcRun < kGtcRun ? nc - u * kGtcRun : kGtcRun;
}
// float4 offset of run r (row group r / runs, run r % runs) in a subgrid's records;
// r = row groups x runs gives the end of the records
__host__ __device__ inline int64_t tc_run_offset(int nc, int r) {
  const int R = tc_runs(nc), G = r / R, u = r - G * R;
  return int64_t(G) * tc_group_float4(nc) + int64_t(u) * kGtcRunFloat4;
}

// Row groups of a subgrid: segments contribute ceil(rows / 4) each
__host__ __device__ inline int tc_row_groups(const SegmentDesc* seg, int seg_begin, int seg_count, int nc) {
  int n = 0;
  for (int s = 0; s < seg_count; ++s) {
    const int rows = (seg[seg_begin + s].k_end - seg[seg_begin + s].k_begin) / nc;
    n += (rows + 3) / 4;
  }
  return n;
}

// Staged 128-byte records of a subgrid in the tensor-core layout
__host__ __device__ inline int64_t tc_records(int n_groups, int nc) {
  return int64_t(n_groups) * tc_group_float4(nc) / 8;
}


// ---------------------------------------------------------------- planner

struct PlanInput {
  int32_t N, L, P;
  double fov;
  int32_t flags;
  int32_t n_st, n_bl, n_t, n_ch, n_int;
  const int32_t* baselines;
  const double* uvw;
  const double* freqs;
  const int32_t* aterm_offsets;
};

struct Partition {
  std::vector<SubgridDesc> subgrids;  // plan order
  std::vector<SegmentDesc> segments;
  double w_step = 0.0;                // w layer width 2 w_max (wavelengths)
};

// Returns IDG_OK or an error status with a message in `err`.
idg_status partition(const PlanInput& in, Partition* out, std::string* err);

// Kaiser-Bessel taper samples T_i, i in [0,L), at x = (2i - L)/L.
std::vector<double> kaiser_bessel_taper(int L, double beta);

// ---------------------------------------------------------------- kernels

struct KernelGeom {
  int32_t N, L, n_t, n_ch, n_st, nodes;
  double fov;
  double w_step;   // w layer width 2 w_max; a subgrid's w0 = (k_min + layer + 1/2) * w_step
  int32_t k_min;
  int32_t npol = 4;  // master-grid planes: 4 correlations, or 1 (Stokes I = (XX + YY) / 2)
};

// w0 of a subgrid: (2k+1) w_max on layer k, one of {w_max, 3 w_max, ...}
// (Section 2.4); 0 without layers (w_step = 0)
__host__ __device__ inline double subgrid_w0(const KernelGeom& g, const SubgridDesc& d) {
  return (double(g.k_min + d.layer) + 0.5) * g.w_step;
}
// -1 for a mirrored subgrid (its members' uvw are negated), else +1
__host__ __device__ inline double subgrid_sign(const SubgridDesc& d) {
  return (d.flags & kSubgridMirrored) ? -1.0 : 1.0;
}

// Staged visibility record, 8 float4 = 128 bytes (written by the staging
// kernel, streamed by the gridder with bulk copies):
//   [0..5] value pairs per polarisation p: (Vr,Vr) (Vi,Vi) (-Vi,-Vi)
//   [6]    (a_head, b_head, a_tail, b_tail)  phase slopes in turns per pixel
//   [7]    (w, 2 pi a, 2 pi w, kind)
constexpr int kRecordFloat4 = 8;
// Gridder record kinds (record float 31): phasors from the record's own slopes,
// rotate by the last channel step, or new channel-step slopes then rotate.
constexpr float kKindRotate = 0.f;
constexpr float kKindBase = 1.f;
constexpr float kKindStep = 2.f;

struct StageArgs {
  const float4* vis;
  const double* uvw;
  const double* fscale;
  const SubgridDesc* sg;      // batch subgrid table
  float4* records;            // [batch records][8]
  KernelGeom g;
};

struct GridArgs {
  const uint8_t* adiag;       // [n_int][n_st]: 1 if that station's A-term nodes are diagonal
  const float4* records;      // staged visibility records of the batch
  int* status;                // device status word (kStatusTimeout)
  int* queue;                 // work-queue counter (persistent launches), zero before the launch
  int n_items;
  const float4* vis;          // [bl][t][ch][4] complex64, 2 float4 per visibility
  const double* uvw;          // [bl][t][3] metres
  const double* fscale;       // [ch] f / c
  const float2* aterms;       // [n_int][n_st][nodes][nodes][4]
  const SubgridDesc* sg;      // batch subgrid table
  const SegmentDesc* seg;     // global segment table
  const GridItem* items;
  const float* taper;         // [L]
  const float4* blk;          // [L][L/8][3] block geometry (n0, anchor offsets) (dn[0..3]) (dn[4..7])
  float2* scratch;            // [batch][4][L][L]
  double* aweights;           // A-term power weights [L*L + 1] (IDG_NORMALIZE_ATERM), else NULL
  int vc = kDefaultGridChunk;  // staged records per chunk: 32, 48 or 64
  KernelGeom g;
};

struct DegridArgs {
  const uint8_t* adiag;       // [n_int][n_st]: 1 if that station's A-term nodes are diagonal
  int* queue;                 // work-queue counter (persistent launches), zero before the launch
  int n_items;
  float4* vis;
  const double* uvw;
  const double* fscale;
  const float2* aterms;
  const SubgridDesc* sg;
  const SegmentDesc* seg;
  const DegridItem* items;
  const float* taper;
  const float4* blk16;        // [L][L/16][5] 16-pixel block geometry (n0, anchor offsets) (dn[0..15])
  const float2* scratch;      // [batch][4][L][L] subgrid images Y
  KernelGeom g;
};

struct FftArgs {
  const SubgridDesc* sg;   // batch subgrid table
  float2* scratch;         // [batch][4][L][L]
  double2* grid;           // [layers][npol][N][N] (adder: +=, splitter: read)
  const float2* twiddle;   // [L] e^{-2 pi i m / L}
  int32_t N;
  int32_t npol = 4;        // planes per subgrid transformed and added / split (4, or 1 for Stokes I)
};

// Launchers (return cudaError_t as int).  `n` is the item or subgrid count.
// persistent_blocks > 0: persistent launch of that many blocks draining a.queue
int launch_gridder(int L, const GridArgs& a, int n_items, int persistent_blocks, void* stream);
// one launch over the items of several plans: args[slot] in device memory, items (slot, item index) in
// launch order; vc the slots' common records per chunk
int launch_gridder_multi(int L, const GridArgs* args, const int2* items, int n_items, bool norm, int vc,
                         void* stream);
bool supported_grid_chunk(int vc);
int configure_gridder(int L, int vc, int* persistent_blocks);   // attributes + persistent grid size
// channels: channels per degridder lane (1, 2 or 4; > 1 needs uniform channel spacing)
int configure_degridder(int L, int nodes, int channels, int* persistent_blocks);
bool supported_degrid_channels(int channels);
int launch_stage_records(int L, const StageArgs& a, int n_subgrids, void* stream);
// element-wise pass over the 4 N x N complex128 planes of one w layer (image-domain wrapper):
// out (+)= in * c * w[x] w[y] * (-1)^(x+y) * e^{i 2 pi w0 n'(x,y)}; w may be null
constexpr int kPassSign = 1;        // apply (-1)^(x+y)
constexpr int kPassAccumulate = 2;  // add into out
// image /= W(p, q) with W the A-term weight map [L*L + 1] (sum n_seg / f,
// then sum n_seg) averaged and interpolated bilinearly from the subgrid lattice
int launch_weight_correction(int npol, double2* image, const double* aweights, int N, int L, void* stream);
int launch_image_pass(int npol, const double2* in, double2* out, const double* w, double c, double w0, double fov, int N,
                      int flags, void* stream);
// one warp waits, bounded by limit_ns, on an mbarrier nothing completes; sets kStatusTimeout bit in *status
int launch_wait_selftest(int* status, int64_t limit_ns, void* stream);
// flags[i][s] = 1 when every node of A-term (interval i, station s) has zero off-diagonal entries
int launch_aterm_flags(const float2* aterms, uint8_t* flags, int n_int, int n_st, int nodes, void* stream);
// split: the items are of at most kSplitLanes lanes and run in the kernel that spreads each
// visibility's pixels over several lanes (one block per item; persistent_blocks is ignored)
int launch_degridder(int L, int channels, const DegridArgs& a, int n_items, int persistent_blocks, void* stream,
                     bool split);
int launch_degridder_multi(int L, int channels, bool split, const DegridArgs* args, const int2* items, int n_items,
                           int max_nodes, void* stream);
// the degridder on the tensor cores (split-TF32 mma.sync, one visibility per row); its items may hold
// two segments only when the first, rounded up to 16 rows, and the second fit in kTcItemRows rows
int launch_degridder_tc(int L, const DegridArgs& a, int n_items, int persistent_blocks, void* stream);
// the gridder on the tensor cores (records staged by launch_stage_tc; uniform channel spacing)
int launch_stage_tc(int L, const StageArgs& a, const SegmentDesc* seg, int n_subgrids, void* stream);
int launch_gridder_tc(int L, const GridArgs& a, int n_items, int persistent_blocks, void* stream);
int configure_gridder_tc(int L, int* persistent_blocks);
int launch_gridder_tc_multi(int L, const GridArgs* args, const int2* items, int n_items, void* stream);
int configure_degridder_tc(int L, int nodes, int* persistent_blocks);
int launch_degridder_tc_multi(int L, const DegridArgs* args, const int2* items, int n_items, int max_nodes,
                              void* stream);
// mode 0: FFT + add into grid; mode 1: FFT in place in scratch (inspection)
int launch_fft_adder(int L, const FftArgs& a, int n_subgrids, int mode, void* stream);
int launch_splitter_ifft(int L, const FftArgs& a, int n_subgrids, void* stream);
// copy a batch of subgrid images to plan order with the (-1)^(x+y) centring undone
int launch_export_subgrids(int L, const SubgridDesc* sg, const float2* scratch, float2* out, int n_subgrids,
                           int npol, void* stream);
int configure_kernels(int L);  // one-time attributes (dynamic shared memory opt-in)

// Read-only view of a device plan's tables, for entry points defined outside
// the API translation unit.  Returns false for host-only plans.
struct PlanDeviceView {
  KernelGeom g;
  void* stream;
  const double* uvw;
  const double* fscale;
  const float* taper;
  const float4* blk;
  const float2* twiddle;
  const SubgridDesc* sg;   // non-dropped subgrids, execution order
  int32_t n_sg;
  const SegmentDesc* seg;
  int32_t flags;           // the plan's IDG_* flags
};
bool plan_device_view(const idg_plan* plan, PlanDeviceView* out);
idg_status plan_set_error(const idg_plan* plan, idg_status st, const char* msg);
bool supported_subgrid_size(int L);
int gridder_rows(int L);  // rows per gridder pixel tile (0 if unsupported)

}  // namespace idg
