// Image-domain wrapper (Section 2.5 imaging step 3, Eq. 11, and prediction
// step 2, Eq. 12): the element-wise passes around the master-grid
// transforms.  With (-1)^(x+y) on both sides, a plain FFT of even length N is
// the centred transform sum_X f(X) e^{-+2 pi i (X - N/2)(p - N/2)/N}; each w
// layer's image is multiplied by e^{+2 pi i w0 n'(l,m)} (w-stacking); the
// taper correction divides by L^2 T(l_p) T(m_q).
#include "kernels_common.cuh"

namespace idg {

// For every pixel (x, y) of N x N and each of the 4 polarisation planes:
//   v = in * c * w[x] w[y] * (kPassSign ? (-1)^(x+y) : 1) * e^{i 2 pi w0 n'(x,y)}
//   out = kPassAccumulate ? out + v : v
// with n' = sqrt(1 - l^2 - m^2) - 1 at l = (x - N/2) FOV/N, m likewise (the
// phase only when w0 != 0; sincospi keeps it accurate for large w0 n').
// One thread per pixel, grid-stride; 16 bytes read (and written) per element.
__global__ void __launch_bounds__(256) image_pass_kernel(const double2* in, double2* out, const double* w, double c,
                                                         double w0, double fov, int N, int flags) {
  const int64_t npix = int64_t(N) * N;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < npix; e += stride) {
    const int x = int(e % N), y = int(e / N);
    double f = c;
    if ((flags & kPassSign) && ((x + y) & 1)) f = -f;
    if (w) f *= w[x] * w[y];
    double pr = f, pi = 0.0;
    if (w0 != 0.0) {
      const double l = double(x - N / 2) * fov / double(N), m = double(y - N / 2) * fov / double(N);
      const double n1 = sqrt(1.0 - l * l - m * m) - 1.0;
      double s, co;
      sincospi(2.0 * w0 * n1, &s, &co);
      pr = f * co;
      pi = f * s;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = int64_t(k) * npix + e;
      const double2 v = in[idx];
      double2 r = make_double2(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
      if (flags & kPassAccumulate) {
        const double2 o = out[idx];
        r.x += o.x;
        r.y += o.y;
      }
      out[idx] = r;
    }
  }
}

int launch_image_pass(const double2* in, double2* out, const double* w, double c, double w0, double fov, int N,
                      int flags, void* stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return int(e);
  const int64_t want = (int64_t(N) * N + 255) / 256;
  const int blocks = int(want < int64_t(sms) * 8 ? want : int64_t(sms) * 8);
  if (blocks <= 0) return 0;
  image_pass_kernel<<<blocks, 256, 0, cudaStream_t(stream)>>>(in, out, w, c, w0, fov, N, flags);
  return int(cudaGetLastError());
}

}  // namespace idg
