// Image-domain wrapper (Section 2.5 imaging step 3, Eq. 11, and prediction
// step 2, Eq. 12, with the single w = 0 layer): the element-wise part around
// the master-grid transform.  With (-1)^(x+y) on both sides, a plain FFT of
// even length N is the centred transform
//   sum_X f(X) e^{-+2 pi i (X - N/2)(p - N/2)/N};
// the taper correction divides by L^2 T(l_p) T(m_q).
#include "kernels_common.cuh"

namespace idg {

// out[k][y][x] = (-1)^(x+y) c w[y] w[x] in[k][y][x]   (w = nullptr: w = 1)
// A memory-bound pass: one 16-byte read and write per element, grid-stride
// over a grid sized in SM multiples.
__global__ void __launch_bounds__(256) sign_scale_kernel(const double2* in, double2* out, const double* w,
                                                         double c, int N, int64_t total) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int x = int(e % N), y = int((e / N) % N);
    double f = ((x + y) & 1) ? -c : c;
    if (w) f *= w[x] * w[y];
    const double2 v = in[e];
    out[e] = make_double2(v.x * f, v.y * f);
  }
}

int launch_sign_scale(const double2* in, double2* out, const double* w, double c, int N, int planes, void* stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return int(e);
  const int64_t total = int64_t(planes) * N * N;
  const int64_t want = (total + 255) / 256;
  const int blocks = int(want < int64_t(sms) * 8 ? want : int64_t(sms) * 8);
  if (blocks <= 0) return 0;
  sign_scale_kernel<<<blocks, 256, 0, cudaStream_t(stream)>>>(in, out, w, c, N, total);
  return int(cudaGetLastError());
}

}  // namespace idg
