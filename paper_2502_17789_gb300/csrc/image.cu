// Image-domain wrapper (Section 2.5 imaging step 3, Eq. 11, and prediction
// step 2, Eq. 12): the element-wise passes around the master-grid
// transforms.  With (-1)^(x+y) on both sides, a plain FFT of even length N is
// the centred transform sum_X f(X) e^{-+2 pi i (X - N/2)(p - N/2)/N}; each w
// layer's image is multiplied by e^{+2 pi i w0 n'(l,m)} (w-stacking); the
// taper correction divides by L^2 T(l_p) T(m_q); with the A-term power
// normalisation of Section 3.3 a last pass divides by the averaged weights.
#include "kernels_common.cuh"

namespace idg {

// For every pixel (x, y) of N x N and each of the npol polarisation planes:
//   v = in * c * w[x] w[y] * (kPassSign ? (-1)^(x+y) : 1) * e^{i 2 pi w0 n'(x,y)}
//   out = kPassAccumulate ? out + v : v
// with n' = sqrt(1 - l^2 - m^2) - 1 at l = (x - N/2) FOV/N, m likewise (the
// phase only when w0 != 0; sincospi keeps it accurate for large w0 n').
// One thread per pixel, grid-stride; 16 bytes read (and written) per element.
__global__ void __launch_bounds__(256) image_pass_kernel(int npol, const double2* in, double2* out, const double* w,
                                                         double c, double w0, double fov, int N, int flags) {
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
#pragma unroll 4
    for (int k = 0; k < npol; ++k) {
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

int launch_image_pass(int npol, const double2* in, double2* out, const double* w, double c, double w0, double fov,
                      int N, int flags, void* stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return int(e);
  const int64_t want = (int64_t(N) * N + 255) / 256;
  const int blocks = int(want < int64_t(sms) * 8 ? want : int64_t(sms) * 8);
  if (blocks <= 0) return 0;
  image_pass_kernel<<<blocks, 256, 0, cudaStream_t(stream)>>>(npol, in, out, w, c, w0, fov, N, flags);
  return int(cudaGetLastError());
}

// A-term power correction (Section 3.3): divide every image pixel by the
// visibility-weighted average of the normalisation factor, W = aw[j L + i] /
// aw[L L] on the subgrid lattice (l_i = (i - L/2) FOV/L), interpolated
// bilinearly at the fractional lattice index (p - N/2) L/N + L/2 (flat beyond
// the last lattice point).  A zero W (no visibilities) leaves the pixel.
__global__ void __launch_bounds__(256) weight_correction_kernel(int npol, double2* img, const double* aw, int N,
                                                                int L) {
  const int64_t npix = int64_t(N) * N;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const double total = aw[int64_t(L) * L];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < npix; e += stride) {
    const int x = int(e % N), y = int(e / N);
    auto lattice = [&](int p, int* i0, double* fr) {
      const double f = double(p - N / 2) * (double(L) / double(N)) + double(L / 2);
      int i = int(floor(f));
      i = i < 0 ? 0 : (i > L - 2 ? L - 2 : i);
      double r = f - double(i);
      *i0 = i;
      *fr = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    };
    int i0, j0;
    double fx, fy;
    lattice(x, &i0, &fx);
    lattice(y, &j0, &fy);
    const double* r0 = aw + int64_t(j0) * L + i0;
    const double* r1 = r0 + L;
    const double wv = ((1.0 - fx) * r0[0] + fx * r0[1]) * (1.0 - fy) + ((1.0 - fx) * r1[0] + fx * r1[1]) * fy;
    if (!(wv > 0.0) || !(total > 0.0)) continue;
    const double c = total / wv;
#pragma unroll 4
    for (int k = 0; k < npol; ++k) {
      double2 v = img[int64_t(k) * npix + e];
      v.x *= c;
      v.y *= c;
      img[int64_t(k) * npix + e] = v;
    }
  }
}

int launch_weight_correction(int npol, double2* image, const double* aweights, int N, int L, void* stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return int(e);
  const int64_t want = (int64_t(N) * N + 255) / 256;
  const int blocks = int(want < int64_t(sms) * 8 ? want : int64_t(sms) * 8);
  if (blocks <= 0) return 0;
  weight_correction_kernel<<<blocks, 256, 0, cudaStream_t(stream)>>>(npol, image, aweights, N, L);
  return int(cudaGetLastError());
}

}  // namespace idg
