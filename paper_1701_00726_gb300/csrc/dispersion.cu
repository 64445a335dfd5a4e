// Free-field quark dispersion relations (Sec. 2, App. A), many momenta at once.
//
// For a spatial momentum p (a = 1) the energy is the zero of the free
// propagator's denominator after p4 -> iE, where cos p4 = cosh E and
// sin^2 p4 = -sinh^2 E:
//   Wilson      K^2 = sum_i sin^2 p_i - sinh^2 E,
//               M = (1/2) p_hat^2 + m = 4 - sum_i cos p_i - cosh E + m;
//   Brillouin   K^2 = (1/729) [sum_i sin^2 p_i prod_{j != i} (c_j + 2)^2 (cosh E + 2)^2
//                               - sinh^2 E prod_i (c_i + 2)^2],
//               M = (1/2) p_check^2 + m = 2 - (1/8) prod_i (c_i + 1) (cosh E + 1) + m;
//   kernel      K^2 + M^2 = 0;
//   overlap     (c^2 + d^2) sqrt(K^2 + M_-^2) + 2 c d M_- = 0 with M_- the kernel's M
//               at m = -rho, c = rho + m/2, d = rho - m/2 (exact sign function).
// One thread per (momentum, mass): the condition is scanned in E from 0 in
// steps of 2e-3 up to E = 8 for its first sign change, which is then refined
// by bisection to the last bit.  No root below E = 8 gives NaN; a condition
// within 1e-12 of zero at E = 0 (massless, p = 0) gives E = 0.
#include "internal.cuh"

#include <cmath>

namespace bri {
namespace {

struct DispArgs {
  int brillouin, overlap;
  double rho;
};

__device__ double condition(const DispArgs& a, const double p[3], double m, double e) {
  const double ch = cosh(e), sh = sinh(e);
  double k2, mass;
  const double mm = a.overlap ? -a.rho : m;
  if (a.brillouin) {
    double c[3], s[3];
    for (int i = 0; i < 3; ++i) {
      c[i] = cos(p[i]);
      s[i] = sin(p[i]);
    }
    double sum = 0.0, prod2 = 1.0, prod1 = 1.0;
    for (int i = 0; i < 3; ++i) {
      double t = s[i] * s[i] * (ch + 2.0) * (ch + 2.0);
      for (int j = 0; j < 3; ++j)
        if (j != i) t *= (c[j] + 2.0) * (c[j] + 2.0);
      sum += t;
      prod2 *= (c[i] + 2.0) * (c[i] + 2.0);
      prod1 *= c[i] + 1.0;
    }
    k2 = (sum - sh * sh * prod2) / 729.0;
    mass = 2.0 - 0.125 * prod1 * (ch + 1.0) + mm;
  } else {
    double s2 = 0.0, csum = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double s = sin(p[i]);
      s2 += s * s;
      csum += cos(p[i]);
    }
    k2 = s2 - sh * sh;
    mass = 4.0 - csum - ch + mm;
  }
  if (!a.overlap) return k2 + mass * mass;
  const double c = a.rho + 0.5 * m, d = a.rho - 0.5 * m;
  const double rad = k2 + mass * mass;
  if (rad < 0.0) return nan("");
  return (c * c + d * d) * sqrt(rad) + 2.0 * c * d * mass;
}

__global__ void k_dispersion(int npts, const double* __restrict__ p, const double* __restrict__ am, DispArgs a,
                             double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double q[3] = {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
  const double m = am[i];
  const int nscan = 4000;
  const double emax = 8.0, h = emax / nscan;
  double prev = condition(a, q, m, 0.0);
  double res = nan("");
  if (fabs(prev) <= 1e-12) {  // the massless quark at rest: zero at E = 0 (up to rounding)
    res = 0.0;
  } else {
    for (int k = 1; k <= nscan; ++k) {
      const double eb = k * h;
      const double cur = condition(a, q, m, eb);
      if (isfinite(prev) && isfinite(cur) && prev * cur <= 0.0) {
        double lo = eb - h, hi = eb, flo = prev;
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          const double fm = condition(a, q, m, mid);
          if (fm == 0.0) {
            lo = hi = mid;
            break;
          }
          if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
          } else {
            hi = mid;
          }
        }
        res = 0.5 * (lo + hi);
        break;
      }
      prev = cur;
    }
  }
  out[i] = res;
}

}  // namespace
}  // namespace bri

using namespace bri;

extern "C" int bri_dispersion(int kernel, int overlap, double rho, int npts, const double* p, const double* am,
                              double* energy, void* stream) {
  if (npts < 1 || !p || !am || !energy || (kernel != BRI_KERNEL_BRILLOUIN && kernel != BRI_KERNEL_WILSON) ||
      (overlap && !(rho > 0.0 && rho < 2.0))) {
    set_error("bri_dispersion: need npts >= 1, non-null arrays, a known kernel and 0 < rho < 2 for the overlap");
    return BRI_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* d = nullptr;
  BRI_CUDA(cudaMallocAsync(&d, sizeof(double) * 5 * (size_t)npts, s));
  note_device_alloc();
  double *dp = d, *dm = d + 3 * (size_t)npts, *de = d + 4 * (size_t)npts;
  cudaError_t e = cudaMemcpyAsync(dp, p, sizeof(double) * 3 * (size_t)npts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, am, sizeof(double) * (size_t)npts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    DispArgs a{kernel == BRI_KERNEL_BRILLOUIN ? 1 : 0, overlap ? 1 : 0, rho};
    k_dispersion<<<blocks_for(npts, 128), 128, 0, s>>>(npts, dp, dm, a, de);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(energy, de, sizeof(double) * (size_t)npts, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "bri_dispersion");
  return BRI_OK;
}
