/*
 * idg.h -- C ABI of libidg, a GB300 (sm_103a) implementation of the
 * image-domain gridding (IDG) hot path of arXiv 2502.17789 ("That pesky
 * A-term", the Pigi imager).
 *
 * The library partitions visibilities into subgrids (Section 3.1), grids
 * them (Section 2.5 imaging steps 2a-2c: direct phasor sum per subgrid with
 * the A-term and taper applied afterwards, subgrid FFT, add into the master
 * uv grid) and degrids them (Section 2.5 prediction steps 3a-3c: split,
 * inverse subgrid FFT, A-term and taper, direct phasor sum per visibility).
 *
 * Conventions (all sizes in elements unless stated):
 *   visibility    complex64 [n_baselines][n_timesteps][n_channels][4]; the 4
 *                 entries are the 2x2 Jones matrix [XX XY; YX YY] row-major.
 *   uvw           float64 [n_baselines][n_timesteps][3], metres; u,v,w in
 *                 wavelengths are uvw * f / c.
 *   A-terms       complex64 [n_intervals][n_stations][nodes][nodes][4]: each
 *                 station's 2x2 Jones matrix sampled on a nodes x nodes grid
 *                 of directions l,m = -FOV/2 + a FOV/(nodes-1), indexed
 *                 [a_m][a_l], bilinearly interpolated to subgrid pixels.
 *   master grid   complex128 [4][N][N] = [pol][y][x]; cell x holds
 *                 u = (x - N/2) / FOV wavelengths.
 * Gridding applies A_p^H X A_q per pixel and degridding A_p Y A_q^H (the
 * adjoint pair of the paper's A^{-1} / A, Eq. 10 and Eq. 13); both multiply
 * by the taper T(l) T(m), so idg_degrid is the exact adjoint of idg_grid.
 *
 * Ownership: the caller owns every buffer it passes and the CUDA stream.
 * A plan owns copies of the baseline table, uvw, frequencies and interval
 * offsets, the subgrid and work tables, and its device scratch.
 *
 * Errors: every function returns an idg_status and never aborts or traps.
 * idg_last_error() gives a message for the last failure on a plan (or, for
 * a NULL plan, for the calling thread).
 *
 * Threading: calls on one plan are asynchronous on the plan's stream; a plan
 * must not be used from two host threads at once.
 */
#ifndef IDG_H
#define IDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IDG_ABI_VERSION 3

typedef struct idg_plan idg_plan; /* opaque, owned by the library */

typedef enum {
  IDG_OK = 0,
  IDG_ERR_INVALID_ARG = 1,   /* bad geometry, sizes, NULL pointer, mismatched plan */
  IDG_ERR_UNSORTED_FREQ = 2, /* channel frequencies not strictly ascending */
  IDG_ERR_UV_OUT_OF_GRID = 3,/* a subgrid would leave the master grid (without IDG_DROP_OUT_OF_GRID) */
  IDG_ERR_W_TOO_LARGE = 4,   /* |w| fringe across a subgrid exceeds P/2 - 1 pixels (Section 2.4) */
  IDG_ERR_OOM = 5,           /* device or host allocation failed */
  IDG_ERR_CUDA = 6,          /* a CUDA runtime call failed; see idg_last_error */
  IDG_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
  IDG_ERR_UNSUPPORTED = 8    /* valid request this build does not implement (e.g. subgrid size) */
} idg_status;

enum { IDG_TAPER_KB = 0, IDG_TAPER_USER = 1 };

/* Units that take the phasor sums' multiply-accumulate (idg_geometry.mac_unit).  On the tensor cores the
   operands are split into TF32 hi and lo parts (A_hi B_hi + A_lo B_hi + A_hi B_lo, about FP32 accuracy) and
   accumulated in FP32; the tensor-core degridder takes one visibility per row (one channel per lane whatever
   degrid_channels asks), the tensor-core gridder needs uniformly spaced channels and no A-term normalisation
   (the plan keeps the FP32 gridder otherwise). */
enum {
  IDG_MAC_DEFAULT = 0,       /* IDG_MAC_TENSOR (IDG_MAC_TENSOR_DEGRID where the tensor-core gridder cannot
                                run); IDG_MAC_FP32 when degrid_channels asks for 2 or 4 and with IDG_STOKES_I
                                (the FP32 kernels then sum XX and YY alone) */
  IDG_MAC_FP32 = 1,          /* gridder and degridder on the FP32 FMA pipe of the CUDA cores */
  IDG_MAC_TENSOR = 2,        /* gridder and degridder on the tensor cores */
  IDG_MAC_TENSOR_DEGRID = 3  /* degridder on the tensor cores, gridder on the FP32 pipe */
};

enum {
  IDG_DROP_OUT_OF_GRID = 1,         /* drop subgrids that leave the grid instead of failing */
  IDG_SPLIT_AT_ATERM_INTERVALS = 2, /* never let a subgrid span two A-term intervals (Section 3.3 as written) */
  IDG_HOST_ONLY = 4,                /* plan on the host only: no device memory, grid/degrid refused */
  IDG_PERSISTENT = 8,               /* persistent launches: #SMs x occupancy blocks drain a work queue */
  IDG_W_LAYERS = 16,                /* w layers (Section 2.4): rows (baseline, timestep) with w < 0 are taken
                                       as their mirrors V^H of baseline (q, p) at (-u, -v, -w) (the footnote's
                                       V(u,v,w) = V(-u,-v,-w)^H), and each subgrid sits on one layer
                                       w0 in {w_max, 3 w_max, 5 w_max, ...} instead of rejecting
                                       |w| > w_max; grids hold one [n_pol][N][N] plane set per layer */
  IDG_NORMALIZE_ATERM = 32,         /* A-term power normalisation (Section 3.3): the gridder divides each
                                       segment's corrected image by ||A_p^H A_q||_F per pixel and the plan
                                       accumulates the weights idg_invert corrects the image with */
  IDG_STOKES_I = 64                 /* Stokes-I imaging: grids and images hold one plane, I = (XX + YY)/2 of
                                       each corrected subgrid image; prediction takes an unpolarised model
                                       (XX = YY = I, XY = YX = 0); the grid, FFT, adder and splitter work
                                       on a quarter of the planes */
};

typedef struct {
  int32_t grid_size;      /* N: even, > 0 */
  int32_t subgrid_size;   /* L: one of 32, 64, 96, 128 for device plans (even, <= N for host plans) */
  int32_t kernel_padding; /* P: even, L - P - 4 >= 1 */
  double image_size;      /* FOV in direction cosines; du = 1/FOV; FOV^2/2 < 1 */
  int32_t taper_kind;     /* IDG_TAPER_KB (beta = taper_beta, or 0.35*pi*P when <= 0) or IDG_TAPER_USER */
  double taper_beta;
  const double* taper_user; /* host [L] taper samples at l_i = (i - L/2) FOV/L (IDG_TAPER_USER), copied */
  int32_t aterm_nodes;    /* nodes per axis of the A-term samples, 2 .. 25 */
  int32_t flags;          /* IDG_DROP_OUT_OF_GRID | IDG_SPLIT_AT_ATERM_INTERVALS | IDG_HOST_ONLY | IDG_PERSISTENT
                             | IDG_W_LAYERS | IDG_NORMALIZE_ATERM | IDG_STOKES_I */
  int32_t degrid_channels; /* degridder channels per lane: 1, 2 or 4, or 0 for the default.  With C > 1 a
                              lane predicts C consecutive channels of one timestep, the first by sine and
                              cosine, the others by rotation with the channel-step phasor (the phase is
                              linear in frequency, Eq. 7); it needs uniformly spaced channels and falls back
                              to 1 otherwise (idg_plan_stats reports the value in use) */
  int32_t grid_chunk;      /* gridder: staged visibility records per chunk copied to shared memory, 32, 48 or
                              64, or 0 for the default (48); a tuning choice, the results do not depend on it */
  int32_t mac_unit;        /* IDG_MAC_DEFAULT, IDG_MAC_FP32, IDG_MAC_TENSOR or IDG_MAC_TENSOR_DEGRID: a tuning
                              choice; the results agree to FP32 rounding */
} idg_geometry;

typedef struct {
  int64_t n_subgrids;         /* all subgrids of the partition, dropped ones included */
  int64_t n_segments;         /* (subgrid, A-term interval) pieces */
  int64_t n_vis;              /* n_baselines * n_timesteps * n_channels */
  int64_t n_vis_dropped;      /* visibilities of dropped subgrids */
  int64_t n_subgrids_dropped;
  int64_t n_grid_items;       /* gridder work items (subgrid, pixel tile) */
  int64_t n_degrid_items;     /* degridder work items (<= 256 visibilities of one or two segments) */
  int64_t n_batches;          /* device batches the subgrids are processed in */
  int64_t occupancy_hist[16]; /* subgrids with visibility count in [2^k, 2^(k+1)), last bin open */
  int64_t device_bytes;       /* device memory held by the plan */
  int64_t vis_pixels;         /* sum over non-dropped subgrids of n_vis * L^2 */
  int32_t subgrid_size;
  int32_t batch_capacity;     /* subgrids per batch */
  int32_t n_w_layers;         /* w layers of the master grid (1 without IDG_W_LAYERS) */
  int32_t w_layer_min;        /* layer k of grid plane set 0; plane set i has w0 = (w_layer_min + i + 1/2)
                                 w_layer_step, i.e. layer k sits at w0 = (2k + 1) w_max */
  double w_layer_step;        /* layer width 2 w_max in wavelengths, w_max = (P/2 - 1) / (max|grad n'| FOV) */
  int32_t n_pol;              /* planes per layer of grids and images: 4, or 1 with IDG_STOKES_I */
  int32_t degrid_channels;    /* channels per degridder lane in use */
  int32_t grid_chunk;         /* gridder records per chunk in use */
  int32_t mac_unit;           /* in use: IDG_MAC_FP32, IDG_MAC_TENSOR (both kernels on the tensor cores) or
                                 IDG_MAC_TENSOR_DEGRID */
} idg_plan_stats_t;

/*
 * idg_plan_create -- partition and prepare one observation (Section 3.1, 3.3).
 *   out            receives the plan (NULL on failure)
 *   g              geometry, copied
 *   n_stations     stations referenced by `baselines`
 *   baselines      host int32 [n_baselines][2] station pairs (p, q), copied
 *   uvw_m          host float64 [n_baselines][n_timesteps][3] metres, copied
 *   freqs_hz       host float64 [n_channels], strictly ascending, copied
 *   aterm_offsets  host int32 [n_intervals + 1] timestep boundaries of the
 *                  A-term intervals: [0] = 0, last = n_timesteps, ascending
 *   cuda_stream    cudaStream_t every later call runs on (NULL = legacy default)
 * Every visibility lands in exactly one subgrid; subgrids share one baseline
 * and carry one segment per A-term interval they cover.  Fails with
 * IDG_ERR_UNSORTED_FREQ, IDG_ERR_UV_OUT_OF_GRID, IDG_ERR_W_TOO_LARGE,
 * IDG_ERR_INVALID_ARG, IDG_ERR_UNSUPPORTED, IDG_ERR_OOM or IDG_ERR_CUDA.
 * Device memory comes from the stream-ordered allocator (cudaMallocAsync on
 * cuda_stream).  Synchronises the stream (uploads the plan tables).
 * Subgrids run in batches whose subgrid images fit a scratch buffer of
 * 1 GiB, or of the byte count in the environment variable
 * IDG_SCRATCH_BYTES read at plan creation (the plan's statistics give the
 * batch count and its device bytes).
 */
idg_status idg_plan_create(idg_plan** out, const idg_geometry* g, int32_t n_stations, int32_t n_baselines,
                           int32_t n_timesteps, int32_t n_channels, const int32_t* baselines,
                           const double* uvw_m, const double* freqs_hz, const int32_t* aterm_offsets,
                           int32_t n_intervals, void* cuda_stream);

/*
 * idg_grid -- imaging direction (Section 2.5 steps 2a-2c, Eq. 10, Eq. 6).
 *   vis_c64     device complex64 [n_baselines][n_timesteps][n_channels][4]
 *   aterms_c64  device complex64 [n_intervals][n_stations][nodes][nodes][4]
 *   grid_c128   device complex128 [n_w_layers][n_pol][N][N] (see idg_plan_stats;
 *               [n_pol][N][N] without IDG_W_LAYERS; n_pol = 4, or 1 with
 *               IDG_STOKES_I), ACCUMULATED INTO (+=)
 * Dropped subgrids contribute nothing.  Asynchronous on the plan's stream.
 * With IDG_STOKES_I the one plane receives I = (XX + YY) / 2 of every
 * corrected subgrid image (the visibilities still carry 4 correlations).
 * Buffers must be 16-byte aligned.
 * With IDG_NORMALIZE_ATERM (Section 3.3) each segment's corrected image
 * A_p^H X A_q is divided, at every subgrid pixel, by f = ||A_p^H A_q||_F of
 * the two interpolated matrices (a pixel with f = 0 contributes nothing),
 * and the plan's weights (idg_aterm_weights) accumulate n_seg / f there.
 */
idg_status idg_grid(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128);

/*
 * idg_degrid -- prediction direction (Section 2.5 steps 3a-3c, Eq. 13 read
 * as the adjoint of idg_grid).
 *   grid_c128   device complex128 [n_w_layers][n_pol][N][N], read only; with
 *               IDG_STOKES_I an unpolarised model, XX = YY = I, XY = YX = 0
 *   aterms_c64  device complex64 [n_intervals][n_stations][nodes][nodes][4]
 *   vis_c64     device complex64 [n_baselines][n_timesteps][n_channels][4],
 *               OVERWRITTEN; visibilities of dropped subgrids are set to 0
 * Asynchronous on the plan's stream.  Buffers must be 16-byte aligned.
 */
idg_status idg_degrid(idg_plan* plan, const void* grid_c128, const void* aterms_c64, void* vis_c64);

/*
 * idg_grid_graph / idg_degrid_graph -- the same operations replayed from a
 * CUDA graph (Section 3.4 batches, all captured as one graph): the first call
 * with a given set of buffers captures the whole call on the plan's stream
 * and instantiates it; later calls with the same buffers launch the graph.
 * Different buffers trigger a new capture.  The plan's stream must not be the
 * legacy default stream (IDG_ERR_INVALID_ARG).  Profiling does not see
 * graph replays.
 */
idg_status idg_grid_graph(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128);
idg_status idg_degrid_graph(idg_plan* plan, const void* grid_c128, const void* aterms_c64, void* vis_c64);

/* Set the stream later calls run on (cudaStream_t; NULL = legacy default). */
idg_status idg_set_stream(idg_plan* plan, void* cuda_stream);

/* Plan statistics (host only, no device work). */
idg_status idg_plan_stats(const idg_plan* plan, idg_plan_stats_t* out);

/*
 * idg_plan_subgrids -- copy the partition, in plan order, to host memory.
 *   out   host int32 [cap][8] rows {baseline, t0, t1, c0, c1, x0, y0, dropped}
 *         (member timesteps [t0,t1), channels [c0,c1), corner (x0,y0))
 *   n     receives the number of subgrids; rows beyond cap are not written
 */
idg_status idg_plan_subgrids(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n);

/*
 * idg_plan_layers -- per subgrid, in plan order, its w layer (Section 2.4).
 *   out   host int32 [cap][2] rows {k, mirrored}: w0 = (k + 1/2) w_layer_step
 *         = (2k + 1) w_max, and mirrored = 1 when the subgrid holds rows of
 *         w < 0 gridded as their mirrors (V^H of baseline (q, p) at -uvw);
 *         {0, 0} for every subgrid without IDG_W_LAYERS (w0 = 0 then)
 *   n     receives the number of subgrids; rows beyond cap are not written
 */
idg_status idg_plan_layers(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n);

/*
 * idg_plan_segments -- copy the segments to host memory.
 *   out   host int32 [cap][4] rows {subgrid, interval, t_begin, t_end}
 */
idg_status idg_plan_segments(const idg_plan* plan, int32_t* out, int64_t cap, int64_t* n);

/*
 * idg_subgrid_images -- stage output of the gridder for inspection
 * (Section 2.5 step 2a, or 2a+2b with stage = 1).
 *   stage 0: subgrid images X(i,j) after the phasor sum, A-term and taper
 *   stage 1: the same after the centred subgrid FFT, Vhat(x,y)
 *   out_c64: device complex64 [n_subgrids][n_pol][L][L] in plan order, written;
 *            rows of dropped subgrids are zero
 * Does not touch any grid.  Asynchronous on the plan's stream.
 */
idg_status idg_subgrid_images(idg_plan* plan, const void* vis_c64, const void* aterms_c64, int32_t stage,
                              void* out_c64);

/*
 * idg_aterm_weights -- the A-term power weights of a plan made with
 * IDG_NORMALIZE_ATERM (Section 3.3: the image is corrected by the weighted
 * average of the normalisation factor over all subgrids).
 *   out    host float64 [L*L + 1]: at subgrid pixel (i, j), out[j*L + i] =
 *          sum over the gridded segments of n_seg / ||A_p^H A_q||_F at
 *          (l_i, m_j); out[L*L] = sum of n_seg (the gridded visibilities).
 *          Accumulated by every idg_grid (and idg_invert) since the last reset.
 *   reset  != 0: zero the weights after reading them
 * The image correction is out / out[L*L] interpolated to the image pixels,
 * as idg_invert applies it.  Synchronises the plan's stream.
 * IDG_ERR_INVALID_ARG for plans without the flag or a NULL out.
 */
idg_status idg_aterm_weights(idg_plan* plan, double* out, int32_t reset);

/*
 * idg_synchronize -- wait for the plan's stream and report device-side
 * failures of earlier calls: IDG_ERR_TIMEOUT if a kernel gave up a bounded
 * wait (the call's results are then incomplete), IDG_ERR_CUDA on an
 * asynchronous CUDA error.  Clears the recorded status.
 */
idg_status idg_synchronize(idg_plan* plan);

/*
 * idg_profile_enable -- time every later kernel launch of the plan with CUDA
 * events recorded on the plan's stream around it (on != 0), or stop (0).
 */
idg_status idg_profile_enable(idg_plan* plan, int32_t on);

/*
 * idg_profile_read -- accumulated device time and launch counts per kernel
 * since the last read, then reset.  Synchronises the plan's stream.
 *   ms        host double [6]: gridder, fft+adder, splitter+ifft, degridder,
 *             visibility staging, A-term diagonal flags
 *   launches  host int64 [6], same order
 */
idg_status idg_profile_read(idg_plan* plan, double* ms, int64_t* launches);

/*
 * idg_grid_noalloc -- idg_grid without allocating memory.  No counterpart in
 * the paper: it serves callers that cannot call cudaMalloc at the point where
 * they grid -- real-time pipelines that reserve all memory at start-up
 * (cudaMalloc / cudaFree may synchronise the device and take unbounded time)
 * and hosts whose device memory belongs to another allocator.  Same arguments
 * and result as
 * idg_grid, on a device plan; the subgrid images live in one static 32 MiB
 * device buffer compiled into the library (held on every GPU that loads it
 * until the process exits) instead of the plan's scratch, and subgrids are
 * processed in sub-batches that fit it.  Calls no allocating routine.
 *   - the first call on a device looks up the buffer's device address (once
 *     per device, with that device current) and keeps it for the life of the
 *     process: make that call before any capture, and do not reset the device
 *     (cudaDeviceReset) between calls;
 *   - every call shares the buffer: calls that overlap on the GPU (other
 *     streams or threads) race; the buffer keeps the last call's contents;
 *   - IDG_ERR_UNSUPPORTED if one subgrid image would not fit the buffer or
 *     the plan normalises its A-terms (IDG_NORMALIZE_ATERM) or images
 *     Stokes I (IDG_STOKES_I),
 *     IDG_ERR_INVALID_ARG for host-only plans or NULL / misaligned buffers.
 */
idg_status idg_grid_noalloc(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128);

/*
 * idg_invert -- dirty image: Section 2.5 imaging step 3, Eq. 11 with the
 * single w = 0 layer (subgrids here have w0 = 0).  Zeroes `grid`, grids the
 * visibilities into it exactly as idg_grid, then writes
 *   image[pol][q][p] = sum_{X,Y} grid[pol][Y][X] e^{+2 pi i (u_X l_p + v_Y m_q)}
 *                      / (L^2 T(l_p) T(m_q)),
 *   u_X = (X - N/2) / FOV,  l_p = (p - N/2) FOV / N  (likewise v, m),
 * i.e. the adjoint of the measurement equation (Eq. 1) with A-terms on the
 * N x N image, with the gridder's taper and unnormalised L x L transforms
 * divided out.  Pixels where T is small (the outer part of the field) carry
 * amplified errors; the paper images the central part of a padded field.
 *   vis_c64    device complex64 [n_baselines][n_timesteps][n_channels][4], read
 *   aterms_c64 device complex64 [n_intervals][n_stations][nodes][nodes][4], read
 *   grid_c128  device complex128 [n_w_layers][n_pol][N][N]: with one layer at
 *              w0 = 0 it receives the gridded uv plane; with several it is
 *              work space (each layer is transformed in place)
 *   image_c128 device complex128 [n_pol][N][N] (pol, m, l), written
 * With w layers the image is the w-stacked sum of Eq. 11: each layer's
 * transform times e^{+2 pi i w0 n'(l,m)}, n' = sqrt(1 - l^2 - m^2) - 1.
 * The master-grid transform is cuFFT (4 double-complex planes) on the plan's
 * stream; the first call on a plan creates its cuFFT plan (allocates).
 * With IDG_NORMALIZE_ATERM the plan's weights are zeroed first, the
 * gridding is normalised (idg_grid) and the image is then divided by the
 * weighted average of the normalisation factor, W = weights / (sum n_seg) on
 * the subgrid lattice, interpolated bilinearly to image pixel (p, q) at the
 * fractional lattice index ((p - N/2) L/N + L/2, (q - N/2) L/N + L/2) and
 * extended flat beyond the last lattice point.  idg_predict does not
 * normalise (it stays the adjoint of the plain invert).
 * IDG_ERR_UNSUPPORTED with IDG_TAPER_USER (its samples exist only on the
 * subgrid lattice) or an odd grid size; otherwise as idg_grid.
 */
idg_status idg_invert(idg_plan* plan, const void* vis_c64, const void* aterms_c64, void* grid_c128,
                      void* image_c128);

/*
 * idg_predict -- visibilities of an image: Section 2.5 prediction step 2,
 * Eq. 12 with w = 0, in the adjoint reading of idg_invert:
 *   grid[pol][Y][X] = sum_{p,q} image[pol][q][p] e^{-2 pi i (u_X l_p + v_Y m_q)}
 *                     / (L^2 T(l_p) T(m_q)),
 * then idg_degrid(grid) into vis (overwritten).  With the degridder's own
 * taper this predicts Eq. 1 on the image pixels.
 *   image_c128 device complex128 [n_pol][N][N], read;  grid_c128 [n_w_layers][n_pol][N][N]
 *   overwritten (layer w0 from image e^{-2 pi i w0 n'}, Eq. 12);
 *   vis_c64    device complex64 [n_baselines][n_timesteps][n_channels][4], written.
 * Errors as idg_invert.
 */
idg_status idg_predict(idg_plan* plan, const void* image_c128, const void* aterms_c64, void* grid_c128,
                       void* vis_c64);

/*
 * idg_wait_selftest -- exercise the bounded-wait error path.  No counterpart
 * in the paper.  Enqueues on the plan's stream one warp that waits on a
 * shared-memory mbarrier nothing completes; after limit_us microseconds
 * (1 .. 2e6) it gives up and sets the plan's device status word, exactly as
 * a kernel whose bulk copy never landed does.  The next idg_synchronize on
 * the plan returns IDG_ERR_TIMEOUT (and clears the word); the context stays
 * usable.  IDG_ERR_INVALID_ARG for host-only plans or a limit out of range.
 */
idg_status idg_wait_selftest(idg_plan* plan, int32_t limit_us);

/* Message for the last failure (never NULL; "" when none). */
const char* idg_last_error(const idg_plan* plan);

/* Release the plan and its device memory (stream-ordered frees on the plan's
 * stream, which is synchronised; other streams are not). NULL is a no-op. */
idg_status idg_plan_destroy(idg_plan* plan);

/*
 * idg_grid_many / idg_degrid_many -- idg_grid / idg_degrid of n plans whose
 * work items share one launch per wave: wave w runs batch w of every plan
 * that has one (Section 3.4 works through the visibilities in batches that
 * fit memory; here the batches of several observations fill one launch),
 * with the items of all those batches in one gridder (degridder) launch,
 * longest first across plans.  This is the shared work queue a serving loop
 * drains for the requests it has admitted (continuous batching).  Each plan's
 * result is the one idg_grid / idg_degrid gives it.
 *   n            number of plans, >= 1
 *   plans        [n] device plans, distinct, sharing the subgrid size, the
 *                Stokes-I flag, the A-term normalisation flag, grid_chunk,
 *                degrid_channels and mac_unit (IDG_ERR_INVALID_ARG otherwise)
 *   vis_c64, aterms_c64, grid_c128
 *                [n] device buffers, per plan as for idg_grid / idg_degrid
 *   cuda_stream  the stream every launch of the call goes to (the plans' own
 *                streams are not used: work queued on them must be complete
 *                or ordered before the call by the caller)
 * Uses each plan's scratch and staging buffers, so a plan may not run
 * anything else until the call's work on cuda_stream has finished.
 * Allocates two small tables per wave (stream-ordered).  Persistent launch
 * mode is not used here.
 */
idg_status idg_grid_many(int32_t n, idg_plan* const* plans, const void* const* vis_c64,
                         const void* const* aterms_c64, void* const* grid_c128, void* cuda_stream);
idg_status idg_degrid_many(int32_t n, idg_plan* const* plans, const void* const* grid_c128,
                           const void* const* aterms_c64, void* const* vis_c64, void* cuda_stream);

/*
 * idg_peak_rates -- measured throughput of the two units the phasor sums use
 * (Section 5.1: the kernels are bounded by the hardware's measured FP32
 * rate).  Runs, on cuda_stream with every SM of the current device filled,
 * one kernel of independent packed f32x2 FMA chains and one of independent
 * __sincosf evaluations, each timed with CUDA events after a warm-up run.
 *   fma_per_s     receives FP32 fused multiply-adds per second (an f32x2 FMA
 *                 counts as two)
 *   sincos_per_s  receives __sincosf evaluations per second (one sine and one
 *                 cosine each)
 * Allocates a few hundred KB (stream-ordered) and synchronises the stream.
 * IDG_ERR_INVALID_ARG for NULL outputs, IDG_ERR_CUDA / IDG_ERR_OOM otherwise
 * (message in idg_last_error(NULL)).
 */
idg_status idg_peak_rates(void* cuda_stream, double* fma_per_s, double* sincos_per_s);

/* Library version (IDG_ABI_VERSION). */
int32_t idg_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IDG_H */
