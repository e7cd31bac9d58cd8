// Degridder kernel: Section 2.5 prediction step 3c (Eq. 13), read as the
// exact adjoint of the gridder:
//   Z(i,j) = (-1)^(i+j) T_i T_j A_p(i,j) Y(i,j) A_q(i,j)^H
//   V_k    = sum_{ij} Z(i,j) e^{-2 pi i phi_k(i,j)}
// where Y is the uncentred inverse subgrid FFT of the split-out grid
// footprint (the splitter applied (-1)^(x+y)).
//
// Work item = up to kDegridLanes lanes of one or two consecutive segments of
// a subgrid (one A-term each), in groups of 32 (one per warp lane); pairing
// segments fills the lanes that a lone segment would leave idle.  A lane
// holds a channel group: up to C consecutive channels of one timestep row
// (C = 1: one visibility).  The phase is linear in frequency (Eq. 7 with
// u = u_m f / c), so with uniform channel spacing the lane evaluates the
// phasor of its first channel and the phasor of the channel step with
// __sincosf and reaches the others by rotation, one complex multiply per
// pixel each; every Z value it loads serves its C visibilities.  A row's
// nc channels are split into G = ceil(nc / C) groups of balanced size.
// The block walks the subgrid in chunks of pixel blocks (8 consecutive
// pixels of a row each; 512 pixels per chunk, 256 with C = 4).  Within a chunk, warp w sums pixel
// blocks [8w, 8w+8) for every lane group in turn and adds its partial sums
// into a shared-memory accumulator with shared-memory atomics, so all warps
// stay busy whatever the segment size.  Z of the next chunk is built while
// the current chunk is summed: its Y values are loaded into registers before
// the phasor sum and turned into Z (A-term prologue) after it, into the other
// half of a double buffer, one barrier per chunk; with two segments, each
// pixel pair gets one Z per segment and every lane reads the Z of its own
// segment.
// Phases use the same FP64 offset / exact anchor reduction / FP32 increment
// scheme as the gridder, with one anchor per 16 pixels of a row, for the
// first channel and for the channel step alike.
#include "idg_internal.h"

namespace idg {

// the kernels live in degridder_kernels.cuh, instantiated per subgrid size in degridder_lNN.cu
template <int L>
int launch_degridder_l(const DegridArgs& a, int channels, int n_items, int persistent_blocks, void* stream,
                       bool split);
template <int L>
int configure_degridder_l(int nodes, int channels, int* persistent_blocks);
template <int L>
int launch_degridder_multi_l(int channels, bool split, const DegridArgs* args, const int2* items, int n_items,
                             int max_nodes, void* stream);
#define IDG_DEGRID_EXTERN(L)                                                                                     \
  extern template int launch_degridder_l<L>(const DegridArgs&, int, int, int, void*, bool);                     \
  extern template int configure_degridder_l<L>(int, int, int*);                                                 \
  extern template int launch_degridder_multi_l<L>(int, bool, const DegridArgs*, const int2*, int, int, void*);
IDG_DEGRID_EXTERN(32)
IDG_DEGRID_EXTERN(64)
IDG_DEGRID_EXTERN(96)
IDG_DEGRID_EXTERN(128)
#undef IDG_DEGRID_EXTERN

template <int L>
int launch_degridder_tc_l(const DegridArgs& a, int n_items, int persistent_blocks, void* stream);
template <int L>
int configure_degridder_tc_l(int nodes, int* persistent_blocks);
template <int L>
int launch_degridder_tc_multi_l(const DegridArgs* args, const int2* items, int n_items, int max_nodes, void* stream);
#define IDG_DEGRID_TC_EXTERN(L)                                                                                  \
  extern template int launch_degridder_tc_l<L>(const DegridArgs&, int, int, void*);                             \
  extern template int configure_degridder_tc_l<L>(int, int*);                                                   \
  extern template int launch_degridder_tc_multi_l<L>(const DegridArgs*, const int2*, int, int, void*);
IDG_DEGRID_TC_EXTERN(32)
IDG_DEGRID_TC_EXTERN(64)
IDG_DEGRID_TC_EXTERN(96)
IDG_DEGRID_TC_EXTERN(128)
#undef IDG_DEGRID_TC_EXTERN

int launch_degridder_tc(int L, const DegridArgs& a, int n_items, int persistent_blocks, void* stream) {
  switch (L) {
    case 32: return launch_degridder_tc_l<32>(a, n_items, persistent_blocks, stream);
    case 64: return launch_degridder_tc_l<64>(a, n_items, persistent_blocks, stream);
    case 96: return launch_degridder_tc_l<96>(a, n_items, persistent_blocks, stream);
    case 128: return launch_degridder_tc_l<128>(a, n_items, persistent_blocks, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int configure_degridder_tc(int L, int nodes, int* persistent_blocks) {
  switch (L) {
    case 32: return configure_degridder_tc_l<32>(nodes, persistent_blocks);
    case 64: return configure_degridder_tc_l<64>(nodes, persistent_blocks);
    case 96: return configure_degridder_tc_l<96>(nodes, persistent_blocks);
    case 128: return configure_degridder_tc_l<128>(nodes, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}

int launch_degridder_tc_multi(int L, const DegridArgs* args, const int2* items, int n_items, int max_nodes,
                              void* stream) {
  switch (L) {
    case 32: return launch_degridder_tc_multi_l<32>(args, items, n_items, max_nodes, stream);
    case 64: return launch_degridder_tc_multi_l<64>(args, items, n_items, max_nodes, stream);
    case 96: return launch_degridder_tc_multi_l<96>(args, items, n_items, max_nodes, stream);
    case 128: return launch_degridder_tc_multi_l<128>(args, items, n_items, max_nodes, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

bool supported_degrid_channels(int channels) { return channels == 1 || channels == 2 || channels == 4; }

int launch_degridder_multi(int L, int channels, bool split, const DegridArgs* args, const int2* items, int n_items,
                           int max_nodes, void* stream) {
  switch (L) {
    case 32: return launch_degridder_multi_l<32>(channels, split, args, items, n_items, max_nodes, stream);
    case 64: return launch_degridder_multi_l<64>(channels, split, args, items, n_items, max_nodes, stream);
    case 96: return launch_degridder_multi_l<96>(channels, split, args, items, n_items, max_nodes, stream);
    case 128: return launch_degridder_multi_l<128>(channels, split, args, items, n_items, max_nodes, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int launch_degridder(int L, int channels, const DegridArgs& a, int n_items, int persistent_blocks, void* stream,
                     bool split) {
  switch (L) {
    case 32: return launch_degridder_l<32>(a, channels, n_items, persistent_blocks, stream, split);
    case 64: return launch_degridder_l<64>(a, channels, n_items, persistent_blocks, stream, split);
    case 96: return launch_degridder_l<96>(a, channels, n_items, persistent_blocks, stream, split);
    case 128: return launch_degridder_l<128>(a, channels, n_items, persistent_blocks, stream, split);
    default: return int(cudaErrorInvalidValue);
  }
}

int configure_degridder(int L, int nodes, int channels, int* persistent_blocks) {
  switch (L) {
    case 32: return configure_degridder_l<32>(nodes, channels, persistent_blocks);
    case 64: return configure_degridder_l<64>(nodes, channels, persistent_blocks);
    case 96: return configure_degridder_l<96>(nodes, channels, persistent_blocks);
    case 128: return configure_degridder_l<128>(nodes, channels, persistent_blocks);
    default: return int(cudaErrorInvalidValue);
  }
}

}  // namespace idg
