// C ABI of libidg (include/idg.h): plan creation, gridding, degridding.
//
// A plan holds the partition (Section 3.1) and everything the kernels need
// on the device.  Subgrids run in batches whose subgrid images fit the
// plan's scratch buffer (Section 3.4 batches by memory; here the batch is a
// set of subgrids, ordered so that neighbouring subgrids of the uv plane run
// together and their adds into the master grid stay in L2).  Within a batch
// the work items are ordered longest-first so the tail of the launch is
// short.
#include <cufft.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "idg_internal.h"

using namespace idg;

namespace {

thread_local std::string g_thread_error;
constexpr double kPi = 3.14159265358979323846;

struct Batch {
  int32_t sg_offset, sg_count;
  int32_t gi_offset, gi_count;
  int32_t di_offset, di_count;  // degridder items; then ds_count items of at most kSplitLanes lanes
  int32_t ds_count;
};

template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
};

}  // namespace

struct idg_plan {
  idg_geometry geom{};
  int32_t n_st = 0, n_bl = 0, n_t = 0, n_ch = 0, n_int = 0;
  int32_t L = 0, N = 0;
  int32_t k_min = 0, n_layers = 1;  // w layers of the master grid
  int32_t npol = 4;                  // master-grid planes per layer: 4, or 1 with IDG_STOKES_I
  int32_t degrid_channels = 1;       // channels per degridder lane
  int32_t grid_chunk = kDefaultGridChunk;  // staged records per gridder chunk
  int32_t mac = IDG_MAC_FP32;        // multiply-accumulate unit of the degridder
  bool grid_tc = false;              // gridder on the tensor cores (mac, uniform channels, no A-term normalisation)
  cudaStream_t stream = nullptr;
  bool host_only = false;
  Partition part;
  std::vector<SubgridDesc> exec;  // non-dropped subgrids in execution order
  std::vector<Batch> batches;
  int32_t batch_cap = 0;
  int64_t n_grid_items = 0, n_degrid_items = 0;
  // work estimate per item, host copies (the order of the items of several plans in one launch)
  std::vector<int32_t> gcost, dcost;
  int64_t n_vis_dropped = 0, n_sg_dropped = 0;
  int64_t vis_pixels = 0;
  int64_t device_bytes = 0;
  std::string last_error;
  // device
  double* d_uvw = nullptr;
  double* d_fscale = nullptr;
  float* d_taper = nullptr;
  float4* d_blk = nullptr;
  float4* d_blk16 = nullptr;
  float2* d_twiddle = nullptr;
  SubgridDesc* d_sg = nullptr;
  SegmentDesc* d_seg = nullptr;
  GridItem* d_gitems = nullptr;
  DegridItem* d_ditems = nullptr;
  float2* d_scratch = nullptr;
  float4* d_records = nullptr;  // staged visibility records of one batch
  int* d_status = nullptr;      // kernel status word (timeouts)
  int* d_queue = nullptr;       // work-queue counters, 2 per batch (gridder, degridder)
  uint8_t* d_adiag = nullptr;   // [n_int][n_st] diagonal-A-term flags of the current call
  double* d_aweights = nullptr; // [L*L + 1] A-term power weights (IDG_NORMALIZE_ATERM)
  // image-domain wrapper, made at its first use
  cufftHandle fft = 0;
  bool fft_ready = false;
  double* d_inv_t = nullptr;    // [N] 1 / T(l_p), l_p = (p - N/2) FOV/N
  int64_t max_batch_vis = 0;
  int persistent_grid_blocks = 0, persistent_degrid_blocks = 0;  // > 0: persistent launches
  struct GraphCache {
    const void* x = nullptr;
    const void* y = nullptr;
    const void* z = nullptr;
    cudaGraphExec_t exec = nullptr;
  } graph_grid, graph_degrid;
  // profiling: event pairs recorded around launches, per kernel class
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

namespace {

idg_status set_err(idg_plan* p, idg_status st, const std::string& msg) {
  if (p)
    p->last_error = msg;
  else
    g_thread_error = msg;
  return st;
}

idg_status cuda_err(idg_plan* p, int code, const char* where) {
  if (code == 0) return IDG_OK;
  const cudaError_t e = cudaError_t(code);
  std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(p, e == cudaErrorMemoryAllocation ? IDG_ERR_OOM : IDG_ERR_CUDA, msg);
}

template <typename T>
int upload(idg_plan* p, T** dst, const T* src, size_t n) {
  if (n == 0) {
    *dst = nullptr;
    return 0;
  }
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(dst), n * sizeof(T), p->stream);
  if (e != cudaSuccess) return int(e);
  p->device_bytes += int64_t(n * sizeof(T));
  return int(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, p->stream));
}

enum KernelClass { kGridder = 0, kFftAdder = 1, kSplitter = 2, kDegridder = 3, kStage = 4, kFlags = 5, kClasses = 6 };

cudaEvent_t take_event(idg_plan* p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch `fn` (returning a cudaError_t as int), bracketed by events when profiling.
template <typename F>
int timed(idg_plan* p, int cls, F&& fn) {
  if (!p->profiling) return fn();
  cudaEvent_t a = take_event(p), b = take_event(p);
  if (a) cudaEventRecord(a, p->stream);
  const int e = fn();
  if (b) cudaEventRecord(b, p->stream);
  if (a && b) p->ev_pending.push_back({cls, {a, b}});
  return e;
}

void release_events(idg_plan* p) {
  for (auto& pe : p->ev_pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pending.clear();
  p->ev_pool.clear();
}

void free_device(idg_plan* p) {
  if (p->graph_grid.exec) cudaGraphExecDestroy(p->graph_grid.exec);
  if (p->graph_degrid.exec) cudaGraphExecDestroy(p->graph_degrid.exec);
  p->graph_grid = {};
  p->graph_degrid = {};
  void* ptrs[] = {p->d_uvw,    p->d_fscale, p->d_taper,   p->d_blk,     p->d_twiddle, p->d_sg,     p->d_seg,
                  p->d_gitems, p->d_ditems, p->d_scratch, p->d_records, p->d_status,  p->d_queue,
                  p->d_adiag,  p->d_blk16, p->d_inv_t, p->d_aweights};
  // stream-ordered frees: no device-wide synchronisation, so plans of other
  // streams keep running while this one is released
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, p->stream);
  p->d_uvw = nullptr;
  p->d_fscale = nullptr;
  p->d_taper = nullptr;
  p->d_blk = nullptr;
  p->d_blk16 = nullptr;
  p->d_inv_t = nullptr;
  p->d_twiddle = nullptr;
  p->d_sg = nullptr;
  p->d_seg = nullptr;
  p->d_gitems = nullptr;
  p->d_ditems = nullptr;
  p->d_scratch = nullptr;
  p->d_records = nullptr;
  p->d_status = nullptr;
  p->d_queue = nullptr;
  p->d_adiag = nullptr;
  p->d_aweights = nullptr;
}

// Block geometry table, FP64 -> FP32: for each row j and block ib of 8
// pixels, n'(anchor) and n'(pixel) - n'(anchor) (anchor = pixel 4 of the
// block), plus the anchor offsets (i_a - L/2, j - L/2):
// [j][ib][3] = (n0, i_a - L/2, j - L/2, 0) (dn[0..3]) (dn[4..7]).
std::vector<float4> block_geometry(int L, double fov) {
  const int tpr = L / 8;
  std::vector<float4> t(size_t(L) * tpr * 3);
  auto nprime = [&](int i, int j) {
    const double l = double(i - L / 2) * fov / double(L), m = double(j - L / 2) * fov / double(L);
    return std::sqrt(1.0 - l * l - m * m) - 1.0;
  };
  for (int j = 0; j < L; ++j)
    for (int ib = 0; ib < tpr; ++ib) {
      const int ia = ib * 8 + 4;
      const double n0 = nprime(ia, j);
      float dn[8];
      for (int k = 0; k < 8; ++k) dn[k] = float(nprime(ib * 8 + k, j) - n0);
      float4* g = &t[(size_t(j) * tpr + ib) * 3];
      g[0] = make_float4(float(n0), float(ia - L / 2), float(j - L / 2), 0.f);
      g[1] = make_float4(dn[0], dn[1], dn[2], dn[3]);
      g[2] = make_float4(dn[4], dn[5], dn[6], dn[7]);
    }
  return t;
}

// Same for blocks of 16 pixels (the degridder's phase anchors), anchor at pixel 8:
// [j][m][5] = (n0, i_a - L/2, j - L/2, 0) (dn[0..3]) (dn[4..7]) (dn[8..11]) (dn[12..15]): the
// increments sit in aligned float4s so pixel pairs load as register pairs
std::vector<float4> block_geometry16(int L, double fov) {
  const int bpr = L / 16;
  std::vector<float4> t(size_t(L) * bpr * 5);
  auto nprime = [&](int i, int j) {
    const double l = double(i - L / 2) * fov / double(L), m = double(j - L / 2) * fov / double(L);
    return std::sqrt(1.0 - l * l - m * m) - 1.0;
  };
  for (int j = 0; j < L; ++j)
    for (int mb = 0; mb < bpr; ++mb) {
      const int ia = mb * 16 + 8;
      const double n0 = nprime(ia, j);
      float dn[16];
      for (int k = 0; k < 16; ++k) dn[k] = float(nprime(mb * 16 + k, j) - n0);
      float4* g = &t[(size_t(j) * bpr + mb) * 5];
      g[0] = make_float4(float(n0), float(ia - L / 2), float(j - L / 2), 0.f);
      for (int q = 0; q < 4; ++q) g[1 + q] = make_float4(dn[4 * q], dn[4 * q + 1], dn[4 * q + 2], dn[4 * q + 3]);
    }
  return t;
}

size_t scratch_budget_bytes() {
  const char* s = std::getenv("IDG_SCRATCH_BYTES");
  if (s && *s) {
    const double v = std::atof(s);
    if (v >= 1.0) return size_t(v);
  }
  return size_t(1) << 30;  // 1 GiB of subgrid images per batch
}

idg_status check_buffer(idg_plan* p, const void* ptr, const char* name) {
  if (!ptr) return set_err(p, IDG_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(ptr) % 16) return set_err(p, IDG_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return IDG_OK;
}

}  // namespace

namespace idg {

bool plan_device_view(const idg_plan* p, PlanDeviceView* v) {
  if (!p || p->host_only || !v) return false;
  v->g = KernelGeom{p->N, p->L, p->n_t, p->n_ch, p->n_st, p->geom.aterm_nodes, p->geom.image_size,
                    p->part.w_step, p->k_min};
  v->stream = p->stream;
  v->uvw = p->d_uvw;
  v->fscale = p->d_fscale;
  v->taper = p->d_taper;
  v->blk = p->d_blk;
  v->twiddle = p->d_twiddle;
  v->sg = p->d_sg;
  v->n_sg = int32_t(p->exec.size());
  v->seg = p->d_seg;
  v->flags = p->geom.flags;
  return true;
}

idg_status plan_set_error(const idg_plan* p, idg_status st, const char* msg) {
  return set_err(const_cast<idg_plan*>(p), st, msg);
}

}  // namespace idg

extern "C" {

int32_t idg_abi_version(void) { return IDG_ABI_VERSION; }

const char* idg_last_error(const idg_plan* plan) {
  return plan ? plan->last_error.c_str() : g_thread_error.c_str();
}

idg_status idg_plan_create(idg_plan** out, const idg_geometry* g, int32_t n_stations, int32_t n_baselines,
                           int32_t n_timesteps, int32_t n_channels, const int32_t* baselines, const double* uvw_m,
                           const double* freqs_hz, const int32_t* aterm_offsets, int32_t n_intervals,
                           void* cuda_stream) {
  if (!out) return set_err(nullptr, IDG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!g) return set_err(nullptr, IDG_ERR_INVALID_ARG, "geometry is NULL");
  if (n_baselines < 0 || n_timesteps < 0 || n_channels < 0 || n_stations < 0 || n_intervals < 1)
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "negative size or n_intervals < 1");
  if (!aterm_offsets) return set_err(nullptr, IDG_ERR_INVALID_ARG, "aterm_offsets is NULL");
  if ((n_baselines > 0 && !baselines) || (n_baselines > 0 && n_timesteps > 0 && !uvw_m) || (n_channels > 0 && !freqs_hz))
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL input table");
  if (g->aterm_nodes < 2 || g->aterm_nodes > kMaxAtermNodes)
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "aterm_nodes must be in [2, 25]");
  const bool host_only = (g->flags & IDG_HOST_ONLY) != 0;
  if (!host_only && !supported_subgrid_size(g->subgrid_size))
    return set_err(nullptr, IDG_ERR_UNSUPPORTED, "device plans support subgrid_size 32, 64, 96 or 128");
  if (g->taper_kind != IDG_TAPER_KB && g->taper_kind != IDG_TAPER_USER)
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "unknown taper_kind");
  if (g->taper_kind == IDG_TAPER_USER && !g->taper_user)
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "taper_user is NULL");
  if (g->degrid_channels != 0 && !supported_degrid_channels(g->degrid_channels))
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "degrid_channels must be 0, 1, 2 or 4");
  if (g->grid_chunk != 0 && !supported_grid_chunk(g->grid_chunk))
    return set_err(nullptr, IDG_ERR_INVALID_ARG, "grid_chunk must be 0, 32, 48 or 64");
  if (g->mac_unit < IDG_MAC_DEFAULT || g->mac_unit > IDG_MAC_TENSOR_DEGRID)
    return set_err(nullptr, IDG_ERR_INVALID_ARG,
                   "mac_unit must be IDG_MAC_DEFAULT, IDG_MAC_FP32, IDG_MAC_TENSOR or IDG_MAC_TENSOR_DEGRID");

  idg_plan* p = new (std::nothrow) idg_plan();
  if (!p) return set_err(nullptr, IDG_ERR_OOM, "host allocation failed");
  p->geom = *g;
  p->geom.taper_user = nullptr;
  p->n_st = n_stations;
  p->n_bl = n_baselines;
  p->n_t = n_timesteps;
  p->n_ch = n_channels;
  p->n_int = n_intervals;
  p->L = g->subgrid_size;
  p->N = g->grid_size;
  p->stream = cudaStream_t(cuda_stream);
  p->host_only = host_only;

  PlanInput in{g->grid_size, g->subgrid_size, g->kernel_padding, g->image_size, g->flags, n_stations,
               n_baselines, n_timesteps, n_channels, n_intervals, baselines, uvw_m, freqs_hz, aterm_offsets};
  std::string err;
  idg_status st = partition(in, &p->part, &err);
  if (st != IDG_OK) {
    set_err(nullptr, st, err);
    delete p;
    return st;
  }
  const int L = p->L;
  // w layers held by the master grid: k_min .. k_min + n_layers - 1 over the kept subgrids
  bool any = false;
  int32_t k_lo = 0, k_hi = 0;
  for (const SubgridDesc& d : p->part.subgrids) {
    if (d.flags & kSubgridDropped) {
      ++p->n_sg_dropped;
      p->n_vis_dropped += d.n_vis;
    } else {
      // the kernels write a subgrid's image after its last segment: every
      // kept subgrid has members and at least one segment
      if (d.seg_count < 1 || d.n_vis < 1) {
        set_err(nullptr, IDG_ERR_INVALID_ARG, "internal: a subgrid without members or segments");
        delete p;
        return IDG_ERR_INVALID_ARG;
      }
      p->exec.push_back(d);
      p->vis_pixels += int64_t(d.n_vis) * L * L;
      k_lo = any ? std::min(k_lo, d.layer) : d.layer;
      k_hi = any ? std::max(k_hi, d.layer) : d.layer;
      any = true;
    }
  }
  p->k_min = k_lo;
  p->n_layers = k_hi - k_lo + 1;
  p->npol = (g->flags & IDG_STOKES_I) ? 1 : 4;
  // channel groups per degridder lane: rotation by the channel-step phasor
  // needs one step along the whole band (equal to 1e-12 relative)
  {
    bool uniform = true;
    for (int c = 2; c < n_channels && uniform; ++c) {
      const double s1 = freqs_hz[1] - freqs_hz[0], sc = freqs_hz[c] - freqs_hz[c - 1];
      uniform = std::fabs(sc - s1) <= 1e-12 * std::fabs(s1);
    }
    const int want = g->degrid_channels > 0 ? g->degrid_channels : kDefaultDegridChannels;
    p->degrid_channels = uniform ? want : 1;
  }
  // the default: gridder and degridder on the tensor cores (the gridder falls back to FP32 below where it
  // cannot run); both on FP32 when channel groups were asked for, and for Stokes I (the FP32 kernels' sums
  // over XX and YY alone, with diagonal A-terms, do half the multiply-adds of the four correlations)
  p->mac = g->mac_unit != IDG_MAC_DEFAULT ? g->mac_unit
           : (g->degrid_channels > 1 || (g->flags & IDG_STOKES_I)) ? IDG_MAC_FP32 : IDG_MAC_TENSOR;
  if (p->mac != IDG_MAC_FP32) p->degrid_channels = 1;  // one visibility per row of the tensor-core product
  {
    // the tensor-core gridder rotates phasors by one channel step along each row
    bool uniform = true;
    for (int c = 2; c < n_channels && uniform; ++c) {
      const double s1 = freqs_hz[1] - freqs_hz[0], sc = freqs_hz[c] - freqs_hz[c - 1];
      uniform = std::fabs(sc - s1) <= 1e-12 * std::fabs(s1);
    }
    p->grid_tc = p->mac == IDG_MAC_TENSOR && uniform && !(g->flags & IDG_NORMALIZE_ATERM);
    if (p->mac == IDG_MAC_TENSOR && !p->grid_tc) p->mac = IDG_MAC_TENSOR_DEGRID;  // the units in use
  }
  p->grid_chunk = g->grid_chunk > 0 ? g->grid_chunk : kDefaultGridChunk;
  for (SubgridDesc& d : p->exec) d.layer -= k_lo;  // device tables hold the grid plane set
  if (host_only) {
    *out = p;
    return IDG_OK;
  }

  // execution order: row-major position on the uv plane (adder locality)
  std::stable_sort(p->exec.begin(), p->exec.end(), [](const SubgridDesc& x, const SubgridDesc& y) {
    if (x.y0 != y.y0) return x.y0 < y.y0;
    return x.x0 < y.x0;
  });
  const size_t per_sg = size_t(4) * L * L * sizeof(float2);
  const size_t cap = std::max<size_t>(1, scratch_budget_bytes() / per_sg);
  p->batch_cap = int32_t(std::min<size_t>(cap, std::max<size_t>(1, p->exec.size())));
  const int rows = gridder_rows(L);
  const int tiles = L / rows;
  std::vector<GridItem> gitems;
  std::vector<DegridItem> ditems;
  for (size_t s0 = 0; s0 < p->exec.size(); s0 += p->batch_cap) {
    const int32_t cnt = int32_t(std::min<size_t>(p->batch_cap, p->exec.size() - s0));
    Batch b{int32_t(s0), cnt, int32_t(gitems.size()), 0, int32_t(ditems.size()), 0, 0};
    // staged records of the batch, in batch order
    int64_t recs = 0;
    for (int32_t o = 0; o < cnt; ++o) {
      SubgridDesc& d = p->exec[s0 + o];
      d.rec_offset = int32_t(recs);
      const int nc = d.c1 - d.c0;
      recs += p->grid_tc ? tc_records(tc_row_groups(p->part.segments.data(), d.seg_begin, d.seg_count, nc), nc)
                         : d.n_vis;
    }
    p->max_batch_vis = std::max(p->max_batch_vis, recs);
    // longest first: order batch subgrids by visibility count; the items of
    // one subgrid stay adjacent so its data is reused from L2
    std::vector<int32_t> order(cnt);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
      return p->exec[s0 + x].n_vis > p->exec[s0 + y].n_vis;
    });
    for (int32_t o : order)
      for (int t = 0; t < (p->grid_tc ? L * L / kGtcPixels : tiles); ++t) gitems.push_back(GridItem{o, t});
    // degridder items: pieces of <= `lanes` channel groups of one segment
    // (a segment's rows times G groups per row); a piece that ends its
    // segment shares its item with the first piece of the next segment when
    // both fit
    const int lanes = degrid_lanes(p->degrid_channels);
    const size_t d_first = ditems.size();
    for (int32_t o : order) {
      const SubgridDesc& d = p->exec[s0 + o];
      const int width = d.c1 - d.c0;
      const int G = (width + p->degrid_channels - 1) / p->degrid_channels;
      bool open = false;  // the last item can take a piece of the next segment
      for (int gidx = d.seg_begin; gidx < d.seg_begin + d.seg_count; ++gidx) {
        const SegmentDesc& sgd = p->part.segments[gidx];
        const int g_begin = sgd.k_begin / width * G, g_end = sgd.k_end / width * G;
        for (int k = g_begin; k < g_end; k += lanes) {
          const int ke = std::min(k + lanes, g_end);
          // the tensor-core degridder starts the second segment at the next 16-row tile
          const int first = ditems.empty() ? 0 : ditems.back().k_end - ditems.back().k_begin;
          const int held = p->mac != IDG_MAC_FP32 ? (first + 15) / 16 * 16 : first;
          if (open && k == g_begin && held + (ke - k) <= lanes) {
            ditems.back().k_end = ke;  // second segment of the item
            open = false;
          } else {
            ditems.push_back(DegridItem{o, gidx, k, ke, ke, 0});
            open = ke == g_end;
          }
        }
      }
    }
    // items of at most kSplitLanes lanes go last, for the kernel that spreads a visibility over
    // several lanes; both parts keep the longest-first order
    std::stable_partition(ditems.begin() + d_first, ditems.end(),
                          [](const DegridItem& it) { return it.k_end - it.k_begin > kSplitLanes; });
    size_t n_small = 0;
    for (size_t i = d_first; i < ditems.size(); ++i) n_small += ditems[i].k_end - ditems[i].k_begin <= kSplitLanes;
    b.gi_count = int32_t(gitems.size()) - b.gi_offset;
    b.ds_count = int32_t(n_small);
    b.di_count = int32_t(ditems.size()) - b.di_offset - b.ds_count;
    p->batches.push_back(b);
  }
  p->n_grid_items = int64_t(gitems.size());
  p->n_degrid_items = int64_t(ditems.size());
  p->gcost.resize(gitems.size());
  for (size_t i = 0; i < gitems.size(); ++i) {
    const Batch& bb = *std::upper_bound(p->batches.begin(), p->batches.end(), int32_t(i),
                                        [](int32_t v, const Batch& x) { return v < x.gi_offset + x.gi_count; });
    p->gcost[i] = p->exec[bb.sg_offset + gitems[i].sg].n_vis;
  }
  p->dcost.resize(ditems.size());
  for (size_t i = 0; i < ditems.size(); ++i) p->dcost[i] = ditems[i].k_end - ditems[i].k_begin;

  // device tables
  std::vector<double> fscale(n_channels);
  for (int c = 0; c < n_channels; ++c) fscale[c] = freqs_hz[c] / kSpeedOfLight;
  std::vector<double> taper_d;
  if (g->taper_kind == IDG_TAPER_USER)
    taper_d.assign(g->taper_user, g->taper_user + L);
  else
    taper_d = kaiser_bessel_taper(L, g->taper_beta > 0.0 ? g->taper_beta : 0.35 * kPi * g->kernel_padding);
  std::vector<float> taper_f(taper_d.begin(), taper_d.end());
  std::vector<float4> blk = block_geometry(L, g->image_size);
  std::vector<float4> blk16 = block_geometry16(L, g->image_size);
  std::vector<float2> tw(L);
  for (int m = 0; m < L; ++m) {
    const double ang = -2.0 * kPi * double(m) / double(L);
    tw[m] = make_float2(float(std::cos(ang)), float(std::sin(ang)));
  }
  int pg = 0, pd = 0;
  int e = configure_kernels(L);
  if (!e) e = configure_gridder(L, p->grid_chunk, &pg);
  if (!e && p->grid_tc) e = configure_gridder_tc(L, &pg);
  // the FP32 kernels serve the items of few visibilities in either mode
  if (!e) e = configure_degridder(L, g->aterm_nodes, p->degrid_channels, &pd);
  if (!e && p->mac != IDG_MAC_FP32) e = configure_degridder_tc(L, g->aterm_nodes, &pd);
  if (g->flags & IDG_PERSISTENT) {
    p->persistent_grid_blocks = pg;
    p->persistent_degrid_blocks = pd;
  }
  if (!e) e = upload(p, &p->d_uvw, uvw_m, size_t(n_baselines) * n_timesteps * 3);
  if (!e) e = upload(p, &p->d_fscale, fscale.data(), fscale.size());
  if (!e) e = upload(p, &p->d_taper, taper_f.data(), taper_f.size());
  if (!e) e = upload(p, &p->d_blk, blk.data(), blk.size());
  if (!e) e = upload(p, &p->d_blk16, blk16.data(), blk16.size());
  if (!e) e = upload(p, &p->d_twiddle, tw.data(), tw.size());
  if (!e) e = upload(p, &p->d_sg, p->exec.data(), p->exec.size());
  if (!e) e = upload(p, &p->d_seg, p->part.segments.data(), p->part.segments.size());
  if (!e) e = upload(p, &p->d_gitems, gitems.data(), gitems.size());
  if (!e) e = upload(p, &p->d_ditems, ditems.data(), ditems.size());
  if (!e && !p->exec.empty()) {
    e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_scratch), per_sg * p->batch_cap, p->stream));
    if (!e) p->device_bytes += int64_t(per_sg * p->batch_cap);
  }
  if (!e && p->max_batch_vis > 0) {
    const size_t rb = size_t(p->max_batch_vis) * kRecordFloat4 * sizeof(float4);
    e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_records), rb, p->stream));
    if (!e) p->device_bytes += int64_t(rb);
  }
  if (!e) e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_status), sizeof(int), p->stream));
  if (!e) e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_adiag), size_t(n_intervals) * std::max(1, n_stations),
                                  p->stream));
  if (!e && !p->batches.empty()) {
    e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_queue), sizeof(int) * 2 * p->batches.size(), p->stream));
    if (!e) p->device_bytes += int64_t(sizeof(int) * 2 * p->batches.size());
  }
  if (!e && (g->flags & IDG_NORMALIZE_ATERM)) {
    const size_t wb = (size_t(L) * L + 1) * sizeof(double);
    e = int(cudaMallocAsync(reinterpret_cast<void**>(&p->d_aweights), wb, p->stream));
    if (!e) e = int(cudaMemsetAsync(p->d_aweights, 0, wb, p->stream));
    if (!e) p->device_bytes += int64_t(wb);
  }
  if (!e) e = int(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
  if (!e) e = int(cudaStreamSynchronize(p->stream));
  if (e) {
    st = cuda_err(nullptr, e, "idg_plan_create");
    free_device(p);
    delete p;
    return st;
  }
  *out = p;
  return IDG_OK;
}

idg_status idg_plan_destroy(idg_plan* plan) {
  if (!plan) return IDG_OK;
  if (!plan->host_only) cudaStreamSynchronize(plan->stream);
  if (plan->fft_ready) cufftDestroy(plan->fft);
  plan->fft_ready = false;
  release_events(plan);
  free_device(plan);
  if (!plan->host_only) cudaStreamSynchronize(plan->stream);
  delete plan;
  return IDG_OK;
}

idg_status idg_set_stream(idg_plan* plan, void* cuda_stream) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  plan->stream = cudaStream_t(cuda_stream);
  return IDG_OK;
}

static KernelGeom kgeom(const idg_plan* p) {
  KernelGeom g{p->N, p->L, p->n_t, p->n_ch, p->n_st, p->geom.aterm_nodes, p->geom.image_size, p->part.w_step,
               p->k_min};
  g.npol = p->npol;
  return g;
}

static StageArgs stage_args(const idg_plan* p, const Batch& b, const void* vis) {
  StageArgs sa{};
  sa.vis = static_cast<const float4*>(vis);
  sa.uvw = p->d_uvw;
  sa.fscale = p->d_fscale;
  sa.sg = p->d_sg + b.sg_offset;
  sa.records = p->d_records;
  sa.g = kgeom(p);
  return sa;
}

static GridArgs grid_args(const idg_plan* p, const Batch& b, const void* vis, const void* aterms) {
  GridArgs ga{};
  ga.adiag = p->d_adiag;
  ga.records = p->d_records;
  ga.status = p->d_status;
  ga.vis = static_cast<const float4*>(vis);
  ga.uvw = p->d_uvw;
  ga.fscale = p->d_fscale;
  ga.aterms = static_cast<const float2*>(aterms);
  ga.sg = p->d_sg + b.sg_offset;
  ga.seg = p->d_seg;
  ga.items = p->d_gitems + b.gi_offset;
  ga.taper = p->d_taper;
  ga.blk = p->d_blk;
  ga.scratch = p->d_scratch;
  ga.aweights = p->d_aweights;
  ga.vc = p->grid_chunk;
  ga.g = kgeom(p);
  return ga;
}

// record staging and the gridder of the plan's kind (FP32 pipe or tensor cores)
static int stage_any(const idg_plan* p, const Batch& b, const void* vis, cudaStream_t strm) {
  return p->grid_tc ? launch_stage_tc(p->L, stage_args(p, b, vis), p->d_seg, b.sg_count, strm)
                    : launch_stage_records(p->L, stage_args(p, b, vis), b.sg_count, strm);
}

static int gridder_any(const idg_plan* p, const GridArgs& ga, int n_items, int persistent_blocks, cudaStream_t strm) {
  return p->grid_tc ? launch_gridder_tc(p->L, ga, n_items, persistent_blocks, strm)
                    : launch_gridder(p->L, ga, n_items, persistent_blocks, strm);
}

idg_status idg_grid(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->host_only) return set_err(plan, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  idg_status st;
  if ((st = check_buffer(plan, vis_c64, "vis")) || (st = check_buffer(plan, aterms_c64, "aterms")) ||
      (st = check_buffer(plan, grid_c128, "grid")))
    return st;
  const int L = plan->L;
  {
    const int e = timed(plan, kFlags, [&] {
      return launch_aterm_flags(static_cast<const float2*>(aterms_c64), plan->d_adiag, plan->n_int, plan->n_st,
                                plan->geom.aterm_nodes, plan->stream);
    });
    if (e) return cuda_err(plan, e, "A-term flag launch");
  }
  if (plan->persistent_grid_blocks > 0 && plan->d_queue) {
    const int e = int(cudaMemsetAsync(plan->d_queue, 0, sizeof(int) * 2 * plan->batches.size(), plan->stream));
    if (e) return cuda_err(plan, e, "work-queue reset");
  }
  for (size_t bi = 0; bi < plan->batches.size(); ++bi) {
    const Batch& b = plan->batches[bi];
    GridArgs ga = grid_args(plan, b, vis_c64, aterms_c64);
    ga.queue = plan->d_queue + 2 * bi;
    ga.n_items = b.gi_count;
    int es = timed(plan, kStage, [&] { return stage_any(plan, b, vis_c64, plan->stream); });
    if (es) return cuda_err(plan, es, "staging launch");
    int e = timed(plan, kGridder, [&] {
      return gridder_any(plan, ga, b.gi_count, plan->persistent_grid_blocks, plan->stream);
    });
    if (e) return cuda_err(plan, e, "gridder launch");
    FftArgs fa{plan->d_sg + b.sg_offset, plan->d_scratch, static_cast<double2*>(grid_c128), plan->d_twiddle, plan->N,
               plan->npol};
    e = timed(plan, kFftAdder, [&] { return launch_fft_adder(L, fa, b.sg_count, 0, plan->stream); });
    if (e) return cuda_err(plan, e, "fft/adder launch");
  }
  return IDG_OK;
}

idg_status idg_degrid(idg_plan* plan, const void* grid_c128, const void* aterms_c64, void* vis_c64) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->host_only) return set_err(plan, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  idg_status st;
  if ((st = check_buffer(plan, vis_c64, "vis")) || (st = check_buffer(plan, aterms_c64, "aterms")) ||
      (st = check_buffer(plan, grid_c128, "grid")))
    return st;
  const int L = plan->L;
  if (plan->n_vis_dropped > 0) {
    const size_t bytes = size_t(plan->n_bl) * plan->n_t * plan->n_ch * 4 * sizeof(float2);
    const int e = int(cudaMemsetAsync(vis_c64, 0, bytes, plan->stream));
    if (e) return cuda_err(plan, e, "zeroing dropped visibilities");
  }
  {
    const int e = timed(plan, kFlags, [&] {
      return launch_aterm_flags(static_cast<const float2*>(aterms_c64), plan->d_adiag, plan->n_int, plan->n_st,
                                plan->geom.aterm_nodes, plan->stream);
    });
    if (e) return cuda_err(plan, e, "A-term flag launch");
  }
  if (plan->persistent_degrid_blocks > 0 && plan->d_queue) {
    const int e = int(cudaMemsetAsync(plan->d_queue, 0, sizeof(int) * 2 * plan->batches.size(), plan->stream));
    if (e) return cuda_err(plan, e, "work-queue reset");
  }
  for (size_t bi = 0; bi < plan->batches.size(); ++bi) {
    const Batch& b = plan->batches[bi];
    FftArgs fa{plan->d_sg + b.sg_offset, plan->d_scratch, const_cast<double2*>(static_cast<const double2*>(grid_c128)),
               plan->d_twiddle, plan->N, plan->npol};
    int e = timed(plan, kSplitter, [&] { return launch_splitter_ifft(L, fa, b.sg_count, plan->stream); });
    if (e) return cuda_err(plan, e, "splitter/ifft launch");
    DegridArgs da{};
    da.adiag = plan->d_adiag;
    da.queue = plan->d_queue + 2 * bi + 1;
    da.n_items = b.di_count;
    da.vis = static_cast<float4*>(vis_c64);
    da.uvw = plan->d_uvw;
    da.fscale = plan->d_fscale;
    da.aterms = static_cast<const float2*>(aterms_c64);
    da.sg = plan->d_sg + b.sg_offset;
    da.seg = plan->d_seg;
    da.items = plan->d_ditems + b.di_offset;
    da.taper = plan->d_taper;
    da.blk16 = plan->d_blk16;
    da.scratch = plan->d_scratch;
    da.g = kgeom(plan);
    e = timed(plan, kDegridder, [&] {
      if (plan->mac != IDG_MAC_FP32)
        return launch_degridder_tc(L, da, b.di_count, plan->persistent_degrid_blocks, plan->stream);
      return launch_degridder(L, plan->degrid_channels, da, b.di_count, plan->persistent_degrid_blocks,
                              plan->stream, false);
    });
    if (e) return cuda_err(plan, e, "degridder launch");
    if (b.ds_count > 0) {  // items of few lanes (low occupancy)
      DegridArgs ds = da;
      ds.items = plan->d_ditems + b.di_offset + b.di_count;
      ds.n_items = b.ds_count;
      e = timed(plan, kDegridder, [&] {
        return launch_degridder(L, plan->degrid_channels, ds, b.ds_count, 0, plan->stream, true);
      });
      if (e) return cuda_err(plan, e, "degridder launch (items of few lanes)");
    }
  }
  return IDG_OK;
}

idg_status idg_subgrid_images(idg_plan* plan, const void* vis_c64, const void* aterms_c64, int32_t stage,
                              void* out_c64) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->host_only) return set_err(plan, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  if (stage != 0 && stage != 1) return set_err(plan, IDG_ERR_INVALID_ARG, "stage must be 0 or 1");
  idg_status st;
  if ((st = check_buffer(plan, vis_c64, "vis")) || (st = check_buffer(plan, aterms_c64, "aterms")) ||
      (st = check_buffer(plan, out_c64, "out")))
    return st;
  const int L = plan->L;
  const size_t total = plan->part.subgrids.size() * size_t(plan->npol) * L * L * sizeof(float2);
  int e = int(cudaMemsetAsync(out_c64, 0, total, plan->stream));
  if (e) return cuda_err(plan, e, "zeroing output");
  e = timed(plan, kFlags, [&] {
    return launch_aterm_flags(static_cast<const float2*>(aterms_c64), plan->d_adiag, plan->n_int, plan->n_st,
                              plan->geom.aterm_nodes, plan->stream);
  });
  if (e) return cuda_err(plan, e, "A-term flag launch");
  for (const Batch& b : plan->batches) {
    GridArgs ga = grid_args(plan, b, vis_c64, aterms_c64);
    int es = timed(plan, kStage, [&] { return stage_any(plan, b, vis_c64, plan->stream); });
    if (es) return cuda_err(plan, es, "staging launch");
    e = gridder_any(plan, ga, b.gi_count, 0, plan->stream);
    if (e) return cuda_err(plan, e, "gridder launch");
    if (stage == 1) {
      FftArgs fa{plan->d_sg + b.sg_offset, plan->d_scratch, nullptr, plan->d_twiddle, plan->N, plan->npol};
      e = launch_fft_adder(L, fa, b.sg_count, 1, plan->stream);
      if (e) return cuda_err(plan, e, "fft launch");
    }
    e = launch_export_subgrids(L, plan->d_sg + b.sg_offset, plan->d_scratch, static_cast<float2*>(out_c64),
                               b.sg_count, plan->npol, plan->stream);
    if (e) return cuda_err(plan, e, "export launch");
  }
  return IDG_OK;
}

// Capture one whole grid or degrid call into a CUDA graph (once per buffer
// set) and replay it.
static idg_status run_graph(idg_plan* p, bool degrid, const void* x, const void* y, void* z) {
  if (!p) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return set_err(p, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  if (!p->stream) return set_err(p, IDG_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  idg_plan::GraphCache& gc = degrid ? p->graph_degrid : p->graph_grid;
  if (!(gc.exec && gc.x == x && gc.y == y && gc.z == z)) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc = {};
    const bool prof = p->profiling;
    p->profiling = false;
    int e = int(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    if (e) {
      p->profiling = prof;
      return cuda_err(p, e, "cudaStreamBeginCapture");
    }
    const idg_status st = degrid ? idg_degrid(p, x, y, z) : idg_grid(p, x, y, z);
    cudaGraph_t graph = nullptr;
    e = int(cudaStreamEndCapture(p->stream, &graph));
    p->profiling = prof;
    if (st != IDG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e) return cuda_err(p, e, "cudaStreamEndCapture");
    e = int(cudaGraphInstantiate(&gc.exec, graph, 0));
    cudaGraphDestroy(graph);
    if (e) {
      gc.exec = nullptr;
      return cuda_err(p, e, "cudaGraphInstantiate");
    }
    gc.x = x;
    gc.y = y;
    gc.z = z;
  }
  const int e = int(cudaGraphLaunch(gc.exec, p->stream));
  if (e) return cuda_err(p, e, "cudaGraphLaunch");
  return IDG_OK;
}

idg_status idg_grid_graph(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128) {
  return run_graph(plan, false, vis_c64, aterms_c64, grid_c128);
}

idg_status idg_degrid_graph(idg_plan* plan, const void* grid_c128, const void* aterms_c64, void* vis_c64) {
  return run_graph(plan, true, grid_c128, aterms_c64, vis_c64);
}

// ------------------------------------------------------------------ several plans, one launch per wave

}  // extern "C"

namespace {

// The plans of one grid_many / degrid_many call must share the kernel
// instantiation: subgrid size, planes per layer, normalisation, degridder
// channels per lane.
idg_status check_many(int32_t n, idg_plan* const* plans, const void* const* a, const void* const* b,
                      void* const* c, const char* an, const char* bn, const char* cn) {
  if (n < 1 || !plans || !a || !b || !c) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL array or n < 1");
  for (int32_t k = 0; k < n; ++k) {
    idg_plan* p = plans[k];
    if (!p) return set_err(nullptr, IDG_ERR_INVALID_ARG, "a plan is NULL");
    if (p->host_only) return set_err(p, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
    idg_status st;
    if ((st = check_buffer(p, a[k], an)) || (st = check_buffer(p, b[k], bn)) || (st = check_buffer(p, c[k], cn)))
      return st;
    const idg_plan* p0 = plans[0];
    if (p->L != p0->L || p->npol != p0->npol || (p->d_aweights != nullptr) != (p0->d_aweights != nullptr) ||
        p->degrid_channels != p0->degrid_channels || p->grid_chunk != p0->grid_chunk || p->mac != p0->mac ||
        p->grid_tc != p0->grid_tc)
      return set_err(p, IDG_ERR_INVALID_ARG,
                     "plans of one call must share subgrid size, Stokes-I mode, normalisation, grid_chunk, "
                     "degrid_channels, mac_unit and the gridder kind");
    for (int32_t j = 0; j < k; ++j)
      if (plans[j] == p) return set_err(p, IDG_ERR_INVALID_ARG, "a plan appears twice");
  }
  return IDG_OK;
}

// Items of several plans' batches merged longest first (each plan's batch is
// already in that order): (slot, item index within the slot's batch).
std::vector<int2> merge_items(const std::vector<const int32_t*>& cost, const std::vector<int32_t>& count) {
  std::vector<int2> out;
  size_t total = 0;
  for (int32_t c : count) total += size_t(c);
  out.reserve(total);
  std::vector<int32_t> pos(count.size(), 0);
  while (out.size() < total) {
    int best = -1;
    for (size_t s = 0; s < count.size(); ++s)
      if (pos[s] < count[s] && (best < 0 || cost[s][pos[s]] > cost[best][pos[best]])) best = int(s);
    out.push_back(make_int2(best, pos[best]++));
  }
  return out;
}

// device copies of the wave's argument table and item list (stream-ordered, freed after the launch)
template <typename A>
int upload_wave(cudaStream_t st, const std::vector<A>& args, const std::vector<int2>& items, A** d_args,
                int2** d_items) {
  int e = int(cudaMallocAsync(reinterpret_cast<void**>(d_args), sizeof(A) * args.size(), st));
  if (!e) e = int(cudaMallocAsync(reinterpret_cast<void**>(d_items), sizeof(int2) * std::max<size_t>(1, items.size()), st));
  if (!e) e = int(cudaMemcpyAsync(*d_args, args.data(), sizeof(A) * args.size(), cudaMemcpyHostToDevice, st));
  if (!e && !items.empty())
    e = int(cudaMemcpyAsync(*d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
  return e;
}

}  // namespace

extern "C" {

idg_status idg_grid_many(int32_t n, idg_plan* const* plans, const void* const* vis_c64,
                         const void* const* aterms_c64, void* const* grid_c128, void* cuda_stream) {
  idg_status st = check_many(n, plans, vis_c64, aterms_c64, grid_c128, "vis", "aterms", "grid");
  if (st) return st;
  cudaStream_t strm = cudaStream_t(cuda_stream);
  const int L = plans[0]->L;
  size_t n_waves = 0;
  for (int32_t k = 0; k < n; ++k) {
    idg_plan* p = plans[k];
    n_waves = std::max(n_waves, p->batches.size());
    const int e = launch_aterm_flags(static_cast<const float2*>(aterms_c64[k]), p->d_adiag, p->n_int, p->n_st,
                                     p->geom.aterm_nodes, strm);
    if (e) return cuda_err(p, e, "A-term flag launch");
  }
  for (size_t w = 0; w < n_waves; ++w) {
    std::vector<GridArgs> args;
    std::vector<const int32_t*> cost;
    std::vector<int32_t> count;
    std::vector<int32_t> slot_plan;
    for (int32_t k = 0; k < n; ++k) {
      idg_plan* p = plans[k];
      if (w >= p->batches.size()) continue;
      const Batch& b = p->batches[w];
      const int e = stage_any(p, b, vis_c64[k], strm);
      if (e) return cuda_err(p, e, "staging launch");
      GridArgs ga = grid_args(p, b, vis_c64[k], aterms_c64[k]);
      ga.n_items = b.gi_count;
      args.push_back(ga);
      cost.push_back(p->gcost.data() + b.gi_offset);
      count.push_back(b.gi_count);
      slot_plan.push_back(k);
    }
    const std::vector<int2> items = merge_items(cost, count);
    GridArgs* d_args = nullptr;
    int2* d_items = nullptr;
    int e = upload_wave(strm, args, items, &d_args, &d_items);
    if (!e)
      e = plans[0]->grid_tc ? launch_gridder_tc_multi(L, d_args, d_items, int(items.size()), strm)
                            : launch_gridder_multi(L, d_args, d_items, int(items.size()),
                                                   plans[0]->d_aweights != nullptr, plans[0]->grid_chunk, strm);
    if (d_args) cudaFreeAsync(d_args, strm);
    if (d_items) cudaFreeAsync(d_items, strm);
    if (e) return cuda_err(plans[0], e, "gridder launch (several plans)");
    for (size_t s = 0; s < slot_plan.size(); ++s) {
      idg_plan* p = plans[slot_plan[s]];
      const Batch& b = p->batches[w];
      FftArgs fa{p->d_sg + b.sg_offset, p->d_scratch, static_cast<double2*>(grid_c128[slot_plan[s]]), p->d_twiddle,
                 p->N, p->npol};
      e = launch_fft_adder(L, fa, b.sg_count, 0, strm);
      if (e) return cuda_err(p, e, "fft/adder launch");
    }
  }
  return IDG_OK;
}

idg_status idg_degrid_many(int32_t n, idg_plan* const* plans, const void* const* grid_c128,
                           const void* const* aterms_c64, void* const* vis_c64, void* cuda_stream) {
  idg_status st = check_many(n, plans, grid_c128, aterms_c64, vis_c64, "grid", "aterms", "vis");
  if (st) return st;
  if (!vis_c64) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL array");
  cudaStream_t strm = cudaStream_t(cuda_stream);
  const int L = plans[0]->L;
  size_t n_waves = 0;
  int max_nodes = 2;
  for (int32_t k = 0; k < n; ++k) {
    idg_plan* p = plans[k];
    n_waves = std::max(n_waves, p->batches.size());
    max_nodes = std::max(max_nodes, int(p->geom.aterm_nodes));
    if (p->n_vis_dropped > 0) {
      const size_t bytes = size_t(p->n_bl) * p->n_t * p->n_ch * 4 * sizeof(float2);
      const int e = int(cudaMemsetAsync(vis_c64[k], 0, bytes, strm));
      if (e) return cuda_err(p, e, "zeroing dropped visibilities");
    }
    const int e = launch_aterm_flags(static_cast<const float2*>(aterms_c64[k]), p->d_adiag, p->n_int, p->n_st,
                                     p->geom.aterm_nodes, strm);
    if (e) return cuda_err(p, e, "A-term flag launch");
  }
  for (size_t w = 0; w < n_waves; ++w) {
    std::vector<DegridArgs> args;
    std::vector<const int32_t*> cost, cost_s;
    std::vector<int32_t> count, count_s;
    for (int32_t k = 0; k < n; ++k) {
      idg_plan* p = plans[k];
      if (w >= p->batches.size()) continue;
      const Batch& b = p->batches[w];
      FftArgs fa{p->d_sg + b.sg_offset, p->d_scratch,
                 const_cast<double2*>(static_cast<const double2*>(grid_c128[k])), p->d_twiddle, p->N, p->npol};
      const int e = launch_splitter_ifft(L, fa, b.sg_count, strm);
      if (e) return cuda_err(p, e, "splitter/ifft launch");
      DegridArgs da{};
      da.adiag = p->d_adiag;
      da.n_items = b.di_count;
      da.vis = static_cast<float4*>(vis_c64[k]);
      da.uvw = p->d_uvw;
      da.fscale = p->d_fscale;
      da.aterms = static_cast<const float2*>(aterms_c64[k]);
      da.sg = p->d_sg + b.sg_offset;
      da.seg = p->d_seg;
      da.items = p->d_ditems + b.di_offset;
      da.taper = p->d_taper;
      da.blk16 = p->d_blk16;
      da.scratch = p->d_scratch;
      da.g = kgeom(p);
      args.push_back(da);
      cost.push_back(p->dcost.data() + b.di_offset);
      count.push_back(b.di_count);
      cost_s.push_back(p->dcost.data() + b.di_offset + b.di_count);
      count_s.push_back(b.ds_count);
    }
    // regular items, then the items of few lanes; the latter index their plan's item table past
    // the regular ones
    std::vector<int2> items = merge_items(cost, count);
    const size_t n_regular = items.size();
    for (int2 it : merge_items(cost_s, count_s)) items.push_back(make_int2(it.x, count[it.x] + it.y));
    DegridArgs* d_args = nullptr;
    int2* d_items = nullptr;
    int e = upload_wave(strm, args, items, &d_args, &d_items);
    if (!e)
      e = plans[0]->mac != IDG_MAC_FP32
              ? launch_degridder_tc_multi(L, d_args, d_items, int(n_regular), max_nodes, strm)
              : launch_degridder_multi(L, plans[0]->degrid_channels, false, d_args, d_items, int(n_regular),
                                       max_nodes, strm);
    if (!e && items.size() > n_regular)
      e = launch_degridder_multi(L, plans[0]->degrid_channels, true, d_args, d_items + n_regular,
                                 int(items.size() - n_regular), max_nodes, strm);
    if (d_args) cudaFreeAsync(d_args, strm);
    if (d_items) cudaFreeAsync(d_items, strm);
    if (e) return cuda_err(plans[0], e, "degridder launch (several plans)");
  }
  return IDG_OK;
}

// ------------------------------------------------------------------ image-domain wrapper

static idg_status fft_err(idg_plan* p, cufftResult r, const char* what) {
  return set_err(p, IDG_ERR_CUDA, std::string(what) + ": cuFFT error " + std::to_string(int(r)));
}

// cuFFT plan for the 4 master-grid planes and the image taper table, made once per plan
static idg_status ensure_image(idg_plan* p) {
  if (p->host_only) return set_err(p, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  if (p->geom.taper_kind != IDG_TAPER_KB)
    return set_err(p, IDG_ERR_UNSUPPORTED, "the image-domain wrapper needs the Kaiser-Bessel taper");
  if (p->N % 2) return set_err(p, IDG_ERR_UNSUPPORTED, "the image-domain wrapper needs an even grid size");
  if (!p->fft_ready) {
    int n[2] = {p->N, p->N};
    cufftResult r =
        cufftPlanMany(&p->fft, 2, n, nullptr, 1, p->N * p->N, nullptr, 1, p->N * p->N, CUFFT_Z2Z, p->npol);
    if (r != CUFFT_SUCCESS) return fft_err(p, r, "cufftPlanMany");
    p->fft_ready = true;
    const double beta = p->geom.taper_beta > 0.0 ? p->geom.taper_beta : 0.35 * kPi * p->geom.kernel_padding;
    std::vector<double> inv = kaiser_bessel_taper(p->N, beta);
    for (double& v : inv) v = 1.0 / v;
    const int e = upload(p, &p->d_inv_t, inv.data(), inv.size());
    if (e) return cuda_err(p, e, "image taper table");
  }
  const cufftResult r = cufftSetStream(p->fft, p->stream);
  if (r != CUFFT_SUCCESS) return fft_err(p, r, "cufftSetStream");
  return IDG_OK;
}

idg_status idg_invert(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128,
                      void* image_c128) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  idg_status st;
  if ((st = check_buffer(plan, grid_c128, "grid")) || (st = check_buffer(plan, image_c128, "image")) ||
      (st = ensure_image(plan)))
    return st;
  const int N = plan->N;
  const size_t plane_set = size_t(plan->npol) * N * N;
  const double inv_l2 = 1.0 / (double(plan->L) * double(plan->L));
  const double fov = plan->geom.image_size;
  int e = int(cudaMemsetAsync(grid_c128, 0, plane_set * plan->n_layers * sizeof(double2), plan->stream));
  if (e) return cuda_err(plan, e, "zeroing the grid");
  if (plan->d_aweights) {
    e = int(cudaMemsetAsync(plan->d_aweights, 0, (size_t(plan->L) * plan->L + 1) * sizeof(double), plan->stream));
    if (e) return cuda_err(plan, e, "zeroing the A-term weights");
  }
  if ((st = idg_grid(plan, vis_c64, aterms_c64, grid_c128))) return st;
  // A-term power correction (Section 3.3), after the taper correction
  auto weight_correction = [&]() -> idg_status {
    if (!plan->d_aweights) return IDG_OK;
    const int ew = launch_weight_correction(plan->npol, static_cast<double2*>(image_c128), plan->d_aweights, N, plan->L,
                                            plan->stream);
    return ew ? cuda_err(plan, ew, "A-term weight correction") : IDG_OK;
  };
  double2* img = static_cast<double2*>(image_c128);
  double2* grid = static_cast<double2*>(grid_c128);
  auto inverse = [&](double2* x) {
    return cufftExecZ2Z(plan->fft, reinterpret_cast<cufftDoubleComplex*>(x), reinterpret_cast<cufftDoubleComplex*>(x),
                        CUFFT_INVERSE);
  };
  const bool single = (plan->geom.flags & IDG_W_LAYERS) == 0;
  if (single) {
    // one layer at w0 = 0: transform a signed copy, the gridded plane stays in `grid`
    e = launch_image_pass(plan->npol, grid, img, nullptr, 1.0, 0.0, fov, N, kPassSign, plan->stream);
    if (e) return cuda_err(plan, e, "centring signs");
    const cufftResult r = inverse(img);
    if (r != CUFFT_SUCCESS) return fft_err(plan, r, "cufftExecZ2Z");
    e = launch_image_pass(plan->npol, img, img, plan->d_inv_t, inv_l2, 0.0, fov, N, kPassSign, plan->stream);
    if (e) return cuda_err(plan, e, "taper correction");
    return weight_correction();
  }
  // w-stacking (Eq. 11): transform every layer in place, shift it from w0 to w = 0, sum
  for (int li = 0; li < plan->n_layers; ++li) {
    double2* gl = grid + plane_set * li;
    const double w0 = (double(plan->k_min + li) + 0.5) * plan->part.w_step;
    e = launch_image_pass(plan->npol, gl, gl, nullptr, 1.0, 0.0, fov, N, kPassSign, plan->stream);
    if (e) return cuda_err(plan, e, "centring signs");
    const cufftResult r = inverse(gl);
    if (r != CUFFT_SUCCESS) return fft_err(plan, r, "cufftExecZ2Z");
    e = launch_image_pass(plan->npol, gl, img, nullptr, 1.0, w0, fov, N, kPassSign | (li ? kPassAccumulate : 0), plan->stream);
    if (e) return cuda_err(plan, e, "w-stacking");
  }
  e = launch_image_pass(plan->npol, img, img, plan->d_inv_t, inv_l2, 0.0, fov, N, 0, plan->stream);
  if (e) return cuda_err(plan, e, "taper correction");
  return weight_correction();
}

idg_status idg_predict(idg_plan* plan, const void* image_c128, const void* aterms_c64, void* grid_c128,
                       void* vis_c64) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  idg_status st;
  if ((st = check_buffer(plan, grid_c128, "grid")) || (st = check_buffer(plan, image_c128, "image")) ||
      (st = ensure_image(plan)))
    return st;
  const int N = plan->N;
  const size_t plane_set = size_t(plan->npol) * N * N;
  const double inv_l2 = 1.0 / (double(plan->L) * double(plan->L));
  const double fov = plan->geom.image_size;
  const double2* img = static_cast<const double2*>(image_c128);
  double2* grid = static_cast<double2*>(grid_c128);
  // inverse w-stacking (Eq. 12): each layer's model grid from the image shifted to its w0
  for (int li = 0; li < plan->n_layers; ++li) {
    double2* gl = grid + plane_set * li;
    const double w0 = (double(plan->k_min + li) + 0.5) * plan->part.w_step;
    int e = launch_image_pass(plan->npol, img, gl, plan->d_inv_t, inv_l2, -w0, fov, N, kPassSign, plan->stream);
    if (e) return cuda_err(plan, e, "taper correction");
    const cufftResult r = cufftExecZ2Z(plan->fft, reinterpret_cast<cufftDoubleComplex*>(gl),
                                       reinterpret_cast<cufftDoubleComplex*>(gl), CUFFT_FORWARD);
    if (r != CUFFT_SUCCESS) return fft_err(plan, r, "cufftExecZ2Z");
    e = launch_image_pass(plan->npol, gl, gl, nullptr, 1.0, 0.0, fov, N, kPassSign, plan->stream);
    if (e) return cuda_err(plan, e, "centring signs");
  }
  return idg_degrid(plan, grid_c128, aterms_c64, vis_c64);
}

idg_status idg_aterm_weights(idg_plan* plan, double* out, int32_t reset) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->d_aweights || !out)
    return set_err(plan, IDG_ERR_INVALID_ARG, "idg_aterm_weights needs a plan made with IDG_NORMALIZE_ATERM and an output");
  const size_t bytes = (size_t(plan->L) * plan->L + 1) * sizeof(double);
  int e = int(cudaMemcpyAsync(out, plan->d_aweights, bytes, cudaMemcpyDeviceToHost, plan->stream));
  if (!e && reset) e = int(cudaMemsetAsync(plan->d_aweights, 0, bytes, plan->stream));
  if (!e) e = int(cudaStreamSynchronize(plan->stream));
  return e ? cuda_err(plan, e, "idg_aterm_weights") : IDG_OK;
}

idg_status idg_synchronize(idg_plan* plan) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->host_only) return IDG_OK;
  int e = int(cudaStreamSynchronize(plan->stream));
  if (e) return cuda_err(plan, e, "idg_synchronize");
  // stream-ordered read (and reset) of the status word: no device-wide synchronisation
  int status = 0;
  e = int(cudaMemcpyAsync(&status, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, plan->stream));
  if (!e) e = int(cudaStreamSynchronize(plan->stream));
  if (e) return cuda_err(plan, e, "idg_synchronize");
  if (status) {
    e = int(cudaMemsetAsync(plan->d_status, 0, sizeof(int), plan->stream));
    if (!e) e = int(cudaStreamSynchronize(plan->stream));
    if (e) return cuda_err(plan, e, "idg_synchronize");
    return set_err(plan, IDG_ERR_TIMEOUT, "a kernel gave up waiting for a bulk copy (bounded wait expired)");
  }
  return IDG_OK;
}

idg_status idg_wait_selftest(idg_plan* plan, int32_t limit_us) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->host_only) return set_err(plan, IDG_ERR_INVALID_ARG, "plan was created with IDG_HOST_ONLY");
  if (limit_us < 1 || limit_us > 2000000) return set_err(plan, IDG_ERR_INVALID_ARG, "limit_us must be in [1, 2e6]");
  const int e = launch_wait_selftest(plan->d_status, int64_t(limit_us) * 1000, plan->stream);
  if (e) return cuda_err(plan, e, "wait self-test launch");
  return IDG_OK;
}

idg_status idg_profile_enable(idg_plan* plan, int32_t on) {
  if (!plan) return set_err(nullptr, IDG_ERR_INVALID_ARG, "plan is NULL");
  plan->profiling = on != 0;
  return IDG_OK;
}

idg_status idg_profile_read(idg_plan* plan, double* ms, int64_t* launches) {
  if (!plan || !ms || !launches) return set_err(plan, IDG_ERR_INVALID_ARG, "NULL argument");
  for (int c = 0; c < kClasses; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  if (plan->host_only) return IDG_OK;
  const int e = int(cudaStreamSynchronize(plan->stream));
  if (e) return cuda_err(plan, e, "idg_profile_read");
  for (auto& pe : plan->ev_pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) ms[pe.first] += double(t);
    launches[pe.first] += 1;
    plan->ev_pool.push_back(pe.second.first);
    plan->ev_pool.push_back(pe.second.second);
  }
  plan->ev_pending.clear();
  return IDG_OK;
}

idg_status idg_plan_stats(const idg_plan* plan, idg_plan_stats_t* out) {
  if (!plan || !out) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->n_subgrids = int64_t(plan->part.subgrids.size());
  out->n_segments = int64_t(plan->part.segments.size());
  out->n_vis = int64_t(plan->n_bl) * plan->n_t * plan->n_ch;
  out->n_vis_dropped = plan->n_vis_dropped;
  out->n_subgrids_dropped = plan->n_sg_dropped;
  out->n_grid_items = plan->n_grid_items;
  out->n_degrid_items = plan->n_degrid_items;
  out->n_batches = int64_t(plan->batches.size());
  for (const SubgridDesc& d : plan->part.subgrids) {
    int k = 0;
    while (k < 15 && (int64_t(1) << (k + 1)) <= d.n_vis) ++k;
    out->occupancy_hist[k] += 1;
  }
  out->device_bytes = plan->device_bytes;
  out->vis_pixels = plan->vis_pixels;
  out->subgrid_size = plan->L;
  out->batch_capacity = plan->batch_cap;
  out->n_w_layers = plan->n_layers;
  out->n_pol = plan->npol;
  out->w_layer_min = plan->k_min;
  out->w_layer_step = plan->part.w_step;
  out->degrid_channels = plan->degrid_channels;
  out->grid_chunk = plan->grid_chunk;
  out->mac_unit = plan->mac;
  return IDG_OK;
}

idg_status idg_plan_layers(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n) {
  if (!plan || !n || (cap > 0 && !out)) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL argument");
  *n = int64_t(plan->part.subgrids.size());
  for (int64_t s = 0; s < std::min<int64_t>(cap, *n); ++s) {
    const SubgridDesc& d = plan->part.subgrids[s];
    out[2 * s] = d.layer;
    out[2 * s + 1] = (d.flags & kSubgridMirrored) ? 1 : 0;
  }
  return IDG_OK;
}

idg_status idg_plan_subgrids(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n) {
  if (!plan || !n || (cap > 0 && !out)) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL argument");
  *n = int64_t(plan->part.subgrids.size());
  for (int64_t s = 0; s < std::min<int64_t>(cap, *n); ++s) {
    const SubgridDesc& d = plan->part.subgrids[s];
    const int32_t row[8] = {d.b, d.t0, d.t1, d.c0, d.c1, d.x0, d.y0, (d.flags & kSubgridDropped) ? 1 : 0};
    std::memcpy(out + s * 8, row, sizeof row);
  }
  return IDG_OK;
}

idg_status idg_plan_segments(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n) {
  if (!plan || !n || (cap > 0 && !out)) return set_err(nullptr, IDG_ERR_INVALID_ARG, "NULL argument");
  *n = int64_t(plan->part.segments.size());
  for (int64_t s = 0; s < std::min<int64_t>(cap, *n); ++s) {
    const SegmentDesc& g = plan->part.segments[s];
    const SubgridDesc& d = plan->part.subgrids[g.subgrid];
    const int width = d.c1 - d.c0;
    const int32_t row[4] = {g.subgrid, g.interval, d.t0 + g.k_begin / width, d.t0 + g.k_end / width};
    std::memcpy(out + s * 4, row, sizeof row);
  }
  return IDG_OK;
}

}  // extern "C"
