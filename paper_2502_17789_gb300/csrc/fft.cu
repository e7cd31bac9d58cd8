// Subgrid Fourier transforms and the master-grid adder / splitter.
//
// Section 2.5 imaging steps 2b-2c (Eq. 8, Eq. 6) and prediction steps
// 3a-3b.  The centred transform
//   Vhat(x,y) = sum_{ij} X(i,j) e^{-2 pi i [(x-L/2)(i-L/2) + (y-L/2)(j-L/2)]/L}
// equals (-1)^(x+y) FFT[(-1)^(i+j) X](x,y) for even L.  The gridder already
// applied (-1)^(i+j); the adder applies (-1)^(x+y) while it adds into the
// FP64 master grid.  The splitter applies (-1)^(x+y) on the way in and the
// degridder's prologue (-1)^(i+j) after the inverse transform.
//
// One block transforms one polarisation plane of one subgrid (L x L complex
// FP32; 4 correlation planes, or the one Stokes-I plane) in shared memory: row transforms then column transforms, each a
// Stockham autosort sequence of radix-4/2/3 stages.  Every stage reads its
// butterflies into registers, synchronises, and writes them back, so one
// L x L buffer suffices.
#include "kernels_common.cuh"

namespace idg {

constexpr int kFftThreads = 512;
// Blocks per SM the register budget is sized for: two for L <= 96 (a plane of
// at most 74 KB of shared memory, so two blocks fit and one block's global
// loads and atomics overlap the other's transform), one for L = 128 (132 KB).
constexpr int fft_min_blocks(int L) { return L <= 96 ? 2 : 1; }

// radix sequence per supported size
template <int L>
struct Radices;
template <>
struct Radices<32> {
  static constexpr int n = 3;
  static constexpr int r[4] = {4, 4, 2, 1};
};
template <>
struct Radices<64> {
  static constexpr int n = 3;
  static constexpr int r[4] = {4, 4, 4, 1};
};
template <>
struct Radices<96> {
  static constexpr int n = 4;
  static constexpr int r[4] = {4, 4, 2, 3};
};
template <>
struct Radices<128> {
  static constexpr int n = 4;
  static constexpr int r[4] = {4, 4, 4, 2};
};

__device__ __forceinline__ float2 c2mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// R-point DFT in place, DIR = -1 forward (e^{-2 pi i / R}), +1 inverse
template <int R, int DIR>
__device__ __forceinline__ void butterfly(float2* v) {
  if (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
  } else if (R == 4) {
    const float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    const float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    const float2 a2 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    const float2 d = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
    // a3 = d * (DIR * i): forward multiplies by -i, inverse by +i
    const float2 a3 = DIR < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    v[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
    v[1] = make_float2(a1.x + a3.x, a1.y + a3.y);
    v[2] = make_float2(a0.x - a2.x, a0.y - a2.y);
    v[3] = make_float2(a1.x - a3.x, a1.y - a3.y);
  } else if (R == 3) {
    const float s = 0.86602540378443864676f;  // sqrt(3)/2
    const float2 t = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
    const float2 dd = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    // dd * (DIR * i * s)
    const float2 d = DIR < 0 ? make_float2(s * dd.y, -s * dd.x) : make_float2(-s * dd.y, s * dd.x);
    v[0] = make_float2(v[0].x + t.x, v[0].y + t.y);
    v[1] = make_float2(m.x + d.x, m.y + d.y);
    v[2] = make_float2(m.x - d.x, m.y - d.y);
  }
}

// One Stockham stage over all L lines of the plane.
//   COLS = false: lines are rows (element (line, idx) at line*L + idx)
//   COLS = true : lines are columns (element at idx*L + line)
template <int L, int R, int NS, int DIR, bool COLS>
__device__ __forceinline__ void stockham_stage(float2* buf, const float2* tw) {
  constexpr int NB = L / R;
  constexpr int TOT = NB * L;
  constexpr int PER = (TOT + kFftThreads - 1) / kFftThreads;
  constexpr int TWS = L / (NS * R);
  float2 v[PER][R];
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int bi = threadIdx.x + e * kFftThreads;
    if (bi < TOT) {
      const int line = COLS ? bi % L : bi / NB;
      const int jj = COLS ? bi / L : bi % NB;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = jj + r * NB;
        v[e][r] = COLS ? buf[idx * L + line] : buf[line * L + idx];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int bi = threadIdx.x + e * kFftThreads;
    if (bi < TOT) {
      const int line = COLS ? bi % L : bi / NB;
      const int jj = COLS ? bi / L : bi % NB;
      const int k = jj % NS;
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * k * TWS];
          if (DIR > 0) w.y = -w.y;
          v[e][r] = c2mul(v[e][r], w);
        }
      }
      butterfly<R, DIR>(v[e]);
      const int base = (jj / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = base + r * NS;
        if (COLS)
          buf[idx * L + line] = v[e][r];
        else
          buf[line * L + idx] = v[e][r];
      }
    }
  }
  __syncthreads();
}

template <int L, int DIR, bool COLS>
__device__ __forceinline__ void fft_pass(float2* buf, const float2* tw) {
  using RD = Radices<L>;
  constexpr int r0 = RD::r[0], r1 = RD::r[1], r2 = RD::r[2], r3 = RD::r[3];
  stockham_stage<L, r0, 1, DIR, COLS>(buf, tw);
  stockham_stage<L, r1, r0, DIR, COLS>(buf, tw);
  stockham_stage<L, r2, r0 * r1, DIR, COLS>(buf, tw);
  if constexpr (RD::n > 3) stockham_stage<L, r3, r0 * r1 * r2, DIR, COLS>(buf, tw);
}

template <int L, int DIR>
__device__ __forceinline__ void fft2d(float2* buf, const float2* tw) {
  fft_pass<L, DIR, false>(buf, tw);
  fft_pass<L, DIR, true>(buf, tw);
}

// grid-direction: transform the gridder's subgrid image and add it into the
// FP64 master grid (mode 0) or leave the transform in scratch (mode 1)
template <int L, int MODE>
__global__ void __launch_bounds__(kFftThreads, fft_min_blocks(L)) fft_adder_kernel(const FftArgs a) {
  extern __shared__ float2 sbuf[];
  float2* buf = sbuf;
  float2* tw = sbuf + L * L;
  const int sgi = blockIdx.x / a.npol, pol = blockIdx.x % a.npol;
  const SubgridDesc sd = a.sg[sgi];
  float2* plane = a.scratch + (size_t(sgi) * 4 + pol) * L * L;
  for (int e = threadIdx.x; e < L; e += kFftThreads) tw[e] = a.twiddle[e];
  const float4* src = reinterpret_cast<const float4*>(plane);
  float4* b4 = reinterpret_cast<float4*>(buf);
  for (int e = threadIdx.x; e < L * L / 2; e += kFftThreads) b4[e] = src[e];
  __syncthreads();
  fft2d<L, -1>(buf, tw);
  if (MODE == 0) {
    // plane set of the subgrid's w layer, then the polarisation plane
    double* g = reinterpret_cast<double*>(a.grid) + ((size_t(sd.layer) * a.npol + pol) * a.N * a.N) * 2;
    for (int e = threadIdx.x; e < L * L; e += kFftThreads) {
      const int y = e / L, x = e - y * L;
      const float sgn = ((x + y) & 1) ? -1.f : 1.f;
      const float2 v = buf[e];
      double* dst = g + ((size_t(sd.y0 + y) * a.N) + sd.x0 + x) * 2;
      atomicAdd(dst, double(sgn * v.x));
      atomicAdd(dst + 1, double(sgn * v.y));
    }
  } else {
    float4* dst = reinterpret_cast<float4*>(plane);
    for (int e = threadIdx.x; e < L * L / 2; e += kFftThreads) dst[e] = b4[e];
  }
}

// degrid-direction: copy the subgrid's footprint out of the master grid
// (FP64 -> FP32, times (-1)^(x+y)) and inverse-transform it into scratch
template <int L>
__global__ void __launch_bounds__(kFftThreads, fft_min_blocks(L)) splitter_ifft_kernel(const FftArgs a) {
  extern __shared__ float2 sbuf[];
  float2* buf = sbuf;
  float2* tw = sbuf + L * L;
  const int sgi = blockIdx.x / a.npol, pol = blockIdx.x % a.npol;
  const SubgridDesc sd = a.sg[sgi];
  for (int e = threadIdx.x; e < L; e += kFftThreads) tw[e] = a.twiddle[e];
  const double2* g = a.grid + (size_t(sd.layer) * a.npol + pol) * a.N * a.N;  // w layer, then polarisation
  for (int e = threadIdx.x; e < L * L; e += kFftThreads) {
    const int y = e / L, x = e - y * L;
    const double2 v = g[size_t(sd.y0 + y) * a.N + sd.x0 + x];
    const float sgn = ((x + y) & 1) ? -1.f : 1.f;
    buf[e] = make_float2(sgn * float(v.x), sgn * float(v.y));
  }
  __syncthreads();
  fft2d<L, +1>(buf, tw);
  float4* dst = reinterpret_cast<float4*>(a.scratch + (size_t(sgi) * 4 + pol) * L * L);
  const float4* b4 = reinterpret_cast<const float4*>(buf);
  for (int e = threadIdx.x; e < L * L / 2; e += kFftThreads) dst[e] = b4[e];
}

// plan-order export of subgrid images for inspection, undoing (-1)^(x+y)
template <int L>
__global__ void export_kernel(const SubgridDesc* sg, const float2* scratch, float2* out, int npol) {
  const int sgi = blockIdx.x / npol, pol = blockIdx.x % npol;
  const int dst_sg = sg[sgi].plan_index;
  const float2* src = scratch + (size_t(sgi) * 4 + pol) * L * L;
  float2* dst = out + (size_t(dst_sg) * npol + pol) * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int y = e / L, x = e - y * L;
    const float sgn = ((x + y) & 1) ? -1.f : 1.f;
    const float2 v = src[e];
    dst[e] = make_float2(sgn * v.x, sgn * v.y);
  }
}

template <int L>
static size_t fft_smem() {
  return sizeof(float2) * (L * L + L);
}

template <int L>
static int configure_t() {
  const int smem = int(fft_smem<L>());
  cudaError_t e = cudaFuncSetAttribute(fft_adder_kernel<L, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_adder_kernel<L, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(splitter_ifft_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // shared memory is what bounds these kernels' occupancy: ask for the largest carveout
  const void* fns[3] = {reinterpret_cast<const void*>(fft_adder_kernel<L, 0>),
                        reinterpret_cast<const void*>(fft_adder_kernel<L, 1>),
                        reinterpret_cast<const void*>(splitter_ifft_kernel<L>)};
  for (const void* fn : fns)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
  return int(e);
}

int configure_kernels(int L) {
  switch (L) {
    case 32: return configure_t<32>();
    case 64: return configure_t<64>();
    case 96: return configure_t<96>();
    case 128: return configure_t<128>();
    default: return int(cudaErrorInvalidValue);
  }
}

template <int L>
static int fft_adder_t(const FftArgs& a, int n, int mode, void* stream) {
  if (n <= 0) return 0;
  if (mode == 0)
    fft_adder_kernel<L, 0><<<n * a.npol, kFftThreads, fft_smem<L>(), cudaStream_t(stream)>>>(a);
  else
    fft_adder_kernel<L, 1><<<n * a.npol, kFftThreads, fft_smem<L>(), cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

template <int L>
static int splitter_t(const FftArgs& a, int n, void* stream) {
  if (n <= 0) return 0;
  splitter_ifft_kernel<L><<<n * a.npol, kFftThreads, fft_smem<L>(), cudaStream_t(stream)>>>(a);
  return int(cudaGetLastError());
}

template <int L>
static int export_t(const SubgridDesc* sg, const float2* scratch, float2* out, int n, int npol, void* stream) {
  if (n <= 0) return 0;
  export_kernel<L><<<n * npol, 256, 0, cudaStream_t(stream)>>>(sg, scratch, out, npol);
  return int(cudaGetLastError());
}

int launch_fft_adder(int L, const FftArgs& a, int n, int mode, void* stream) {
  switch (L) {
    case 32: return fft_adder_t<32>(a, n, mode, stream);
    case 64: return fft_adder_t<64>(a, n, mode, stream);
    case 96: return fft_adder_t<96>(a, n, mode, stream);
    case 128: return fft_adder_t<128>(a, n, mode, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int launch_splitter_ifft(int L, const FftArgs& a, int n, void* stream) {
  switch (L) {
    case 32: return splitter_t<32>(a, n, stream);
    case 64: return splitter_t<64>(a, n, stream);
    case 96: return splitter_t<96>(a, n, stream);
    case 128: return splitter_t<128>(a, n, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

int launch_export_subgrids(int L, const SubgridDesc* sg, const float2* scratch, float2* out, int n, int npol,
                           void* stream) {
  switch (L) {
    case 32: return export_t<32>(sg, scratch, out, n, npol, stream);
    case 64: return export_t<64>(sg, scratch, out, n, npol, stream);
    case 96: return export_t<96>(sg, scratch, out, n, npol, stream);
    case 128: return export_t<128>(sg, scratch, out, n, npol, stream);
    default: return int(cudaErrorInvalidValue);
  }
}

}  // namespace idg
