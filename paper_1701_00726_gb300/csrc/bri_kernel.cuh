// Brillouin stencil kernel (CUDA cores), templated on spinor precision R,
// link storage LS and the number NR of right-hand sides one thread carries.
//
// D_bri x(n) = sum_{d != 0} W_d(n) M_d x(n+d) + (15/8 + m0) x(n) + C(n) x(n)   (Eq. def_bril)
//   M_d = -2^{-k-3} 1 + (4^{2-k}/27) sum_{mu: d_mu != 0} sign(d_mu) gamma_mu,  k = |d|_1
// (the momentum forms of App. A expanded into plane waves).  D^dagger = gamma5 D
// gamma5 only flips the sign of the gamma part.
//
// One thread owns one site and NR right-hand sides.  A runtime loop visits the
// 40 stored offsets d (nu = 1..40 of App. C); each iteration also handles the
// opposite hop -d, whose transporter is the stored link of d at the neighbour
// n-d, daggered (W_{82-nu}(n) = W_nu(n-d)^dagger).  Per hop the source spinor is
// first spin-combined, chi = a_k x + sum_mu c_k s_mu gamma_mu x (in the chiral
// basis gamma_mu only permutes spin components with phases +-1, +-i), then
// colour-transported, acc += W chi.  The per-offset constants come from a
// small table in constant memory; the loop is not unrolled so that the
// compiler does not hoist loads across hops, which keeps the live register set
// (and so the occupancy) bounded.  Links are structure-of-arrays, so a warp of
// consecutive sites reads one contiguous segment per link element.
#pragma once

#include "stencil.cuh"

#include <cstdio>
#include <vector>

namespace bri {

// Stored offsets nu = 1..40 with their identity weight -2^{-k-3} and the
// signed gamma weights c_k s_mu, c_k = 4^{2-k}/27.
template <typename R> struct HopTable {
  int site_d[40][4];
  R a[40];
  R cs[40][4];
};
static __constant__ HopTable<float> c_hops_f;   // one copy per translation unit
static __constant__ HopTable<double> c_hops_d;

template <typename R> __device__ __forceinline__ const HopTable<R>& hops();
template <> __device__ __forceinline__ const HopTable<float>& hops<float>() { return c_hops_f; }
template <> __device__ __forceinline__ const HopTable<double>& hops<double>() { return c_hops_d; }

template <typename R> static void fill_hops(HopTable<R>& h) {
  for (int j = 0; j < 40; ++j) {
    const int d[4] = {j % 3 - 1, (j / 3) % 3 - 1, (j / 9) % 3 - 1, (j / 27) % 3 - 1};
    int k = 0;
    for (int mu = 0; mu < 4; ++mu) k += d[mu] != 0;
    const double c = double(1 << (2 * (4 - k))) / 432.0;
    h.a[j] = (R)(-1.0 / double(1 << (k + 3)));
    for (int mu = 0; mu < 4; ++mu) {
      h.site_d[j][mu] = d[mu];
      h.cs[j][mu] = (R)(c * d[mu]);
    }
  }
}

// Upload this translation unit's tables (once per device).
static int ensure_hops() {
  static int ready_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (ready_dev == dev) return BRI_OK;
  HopTable<float> hf;
  HopTable<double> hd;
  fill_hops(hf);
  fill_hops(hd);
  BRI_CUDA(cudaMemcpyToSymbol(c_hops_f, &hf, sizeof(hf)));
  BRI_CUDA(cudaMemcpyToSymbol(c_hops_d, &hd, sizeof(hd)));
  ready_dev = dev;
  return BRI_OK;
}

// chi = a x + (sum_mu cs_mu gamma_mu) x in the chiral basis:
//   sum_mu s_mu gamma_mu = [[0, B], [B^dagger, 0]],  B = s_4 - i (s_1 sigma_1 + s_2 sigma_2 + s_3 sigma_3).
template <typename R>
__device__ __forceinline__ void spin_combine(Spinor<R>& chi, const Spinor<R>& x, R a, R c1, R c2, R c3, R c4) {
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const C<R> x0 = x.v[0][col], x1 = x.v[1][col], x2 = x.v[2][col], x3 = x.v[3][col];
    R r0 = a * x0.re, i0 = a * x0.im, r1 = a * x1.re, i1 = a * x1.im;
    R r2 = a * x2.re, i2 = a * x2.im, r3 = a * x3.re, i3 = a * x3.im;
    // gamma_1
    r0 = fma(c1, x3.im, r0); i0 = fma(-c1, x3.re, i0); r1 = fma(c1, x2.im, r1); i1 = fma(-c1, x2.re, i1);
    r2 = fma(-c1, x1.im, r2); i2 = fma(c1, x1.re, i2); r3 = fma(-c1, x0.im, r3); i3 = fma(c1, x0.re, i3);
    // gamma_2
    r0 = fma(-c2, x3.re, r0); i0 = fma(-c2, x3.im, i0); r1 = fma(c2, x2.re, r1); i1 = fma(c2, x2.im, i1);
    r2 = fma(c2, x1.re, r2); i2 = fma(c2, x1.im, i2); r3 = fma(-c2, x0.re, r3); i3 = fma(-c2, x0.im, i3);
    // gamma_3
    r0 = fma(c3, x2.im, r0); i0 = fma(-c3, x2.re, i0); r1 = fma(-c3, x3.im, r1); i1 = fma(c3, x3.re, i1);
    r2 = fma(-c3, x0.im, r2); i2 = fma(c3, x0.re, i2); r3 = fma(c3, x1.im, r3); i3 = fma(-c3, x1.re, i3);
    // gamma_4
    r0 = fma(c4, x2.re, r0); i0 = fma(c4, x2.im, i0); r1 = fma(c4, x3.re, r1); i1 = fma(c4, x3.im, i1);
    r2 = fma(c4, x0.re, r2); i2 = fma(c4, x0.im, i2); r3 = fma(c4, x1.re, r3); i3 = fma(c4, x1.im, i3);
    chi.v[0][col] = C<R>{r0, i0};
    chi.v[1][col] = C<R>{r1, i1};
    chi.v[2][col] = C<R>{r2, i2};
    chi.v[3][col] = C<R>{r3, i3};
  }
}

template <typename R, int NR> struct BriOcc { static constexpr int v = NR == 1 ? 4 : 3; };
template <int NR> struct BriOcc<double, NR> { static constexpr int v = 2; };

template <typename R, typename LS, int NR>
__global__ void __launch_bounds__(128, BriOcc<R, NR>::v)
    bri_kernel(Geom g, R* __restrict__ y, const R* __restrict__ x, const LS* __restrict__ W,
               const R* __restrict__ cl, R diag, R sgn, int rhs0) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int V = (int)g.V;
  const int64_t rstride = g.V * 24;
  const int64_t roff = (int64_t)(rhs0 + blockIdx.y * NR) * rstride;
  const R* xin = x + roff;
  int co[4], L[4], str[4];
  {
    int r = n;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      co[mu] = r % g.L[mu];
      r /= g.L[mu];
    }
    co[3] = r;
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    L[mu] = g.L[mu];
    str[mu] = (int)g.str[mu];
  }
  const HopTable<R>& H = hops<R>();
  Spinor<R> acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) zero(acc[r]);
#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    int mp = 0, mm = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int d = H.site_d[j][mu];
      mp += wrap(co[mu] + d, L[mu]) * str[mu];
      mm += wrap(co[mu] - d, L[mu]) * str[mu];
    }
    const R a = H.a[j];
    const R c1 = sgn * H.cs[j][0], c2 = sgn * H.cs[j][1], c3 = sgn * H.cs[j][2], c4 = sgn * H.cs[j][3];
    const LS* wj = W + (int64_t)j * 9 * V;
    {  // +d: W_d(n) M_d x(n+d)
      C<R> w[3][3];
      load_link<R, LS>(w, wj + n, V);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        Spinor<R> xs, chi;
        load_spinor(xs, xin + r * rstride + (int64_t)mp * 24);
        spin_combine(chi, xs, a, c1, c2, c3, c4);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa)
#pragma unroll
            for (int b = 0; b < 3; ++b) cfma(acc[r].v[s][aa], w[aa][b], chi.v[s][b]);
      }
    }
    {  // -d: W_{-d}(n) = W_d(n-d)^dagger, and M_{-d} flips the gamma part
      C<R> w[3][3];
      load_link<R, LS>(w, wj + mm, V);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        Spinor<R> xs, chi;
        load_spinor(xs, xin + r * rstride + (int64_t)mm * 24);
        spin_combine(chi, xs, a, -c1, -c2, -c3, -c4);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa)
#pragma unroll
            for (int b = 0; b < 3; ++b) cfma_cj(acc[r].v[s][aa], w[b][aa], chi.v[s][b]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    Spinor<R> xc;
    load_spinor(xc, xin + r * rstride + (int64_t)n * 24);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        acc[r].v[s][aa].re = fma(diag, xc.v[s][aa].re, acc[r].v[s][aa].re);
        acc[r].v[s][aa].im = fma(diag, xc.v[s][aa].im, acc[r].v[s][aa].im);
      }
    if (cl) add_clover(acc[r], xc, cl, g.V, n);
    store_spinor(y + roff + r * rstride + (int64_t)n * 24, acc[r]);
  }
}

template <typename R, typename LS, int NR>
inline void launch_bri_nr(const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag, R sgn, int rhs0,
                          int groups, int threads, cudaStream_t s) {
  dim3 grid(blocks_for(g.V, threads), groups);
  bri_kernel<R, LS, NR><<<grid, threads, 0, s>>>(g, y, x, W, cl, diag, sgn, rhs0);
  note_launch();
}

// Launch configuration of the stencil: whether pairs of right-hand sides
// share one thread (and so their link loads), and the block size.
struct StencilConfig {
  int pairs = 1;
  int threads = 128;
};

template <typename R, typename LS>
inline void launch_with(const StencilConfig& cf, const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag,
                        R sgn, int nrhs, cudaStream_t s) {
  int done = 0;
  if constexpr (sizeof(R) == 4) {
    if (nrhs >= 2 && cf.pairs) {
      launch_bri_nr<R, LS, 2>(g, y, x, W, cl, diag, sgn, 0, nrhs / 2, cf.threads, s);
      done = (nrhs / 2) * 2;
    }
  }
  if (nrhs > done) launch_bri_nr<R, LS, 1>(g, y, x, W, cl, diag, sgn, done, nrhs - done, cf.threads, s);
}

// Autotuner: on the first launch for a (device, lattice, rhs-count class,
// precision) the candidate configurations are timed (the timing launches
// compute the same y = D x) and the fastest is cached for the process.  No
// tuning happens while the stream is being captured into a graph.
template <typename R, typename LS>
StencilConfig tuned_config(const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag, R sgn, int nrhs,
                           cudaStream_t s) {
  StencilConfig def;
  if (!autotune_enabled()) {
    def.pairs = pair_rhs_enabled();
    return def;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const int cls = nrhs <= 1 ? 1 : (nrhs < 4 ? 2 : 4);
  char key[160];
  snprintf(key, sizeof(key), "%d:%d,%d,%d,%d:%d:%d,%d", dev, g.L[0], g.L[1], g.L[2], g.L[3], cls, (int)sizeof(R),
           (int)sizeof(LS));
  StencilConfig found;
  if (tune_lookup(key, &found)) return found;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone) return def;
  std::vector<StencilConfig> cands;
  for (int pairs = 0; pairs <= ((sizeof(R) == 4 && nrhs >= 2) ? 1 : 0); ++pairs)
    for (int th : {64, 128}) cands.push_back(StencilConfig{pairs, th});
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  StencilConfig bestc = def;
  for (const StencilConfig& cf : cands) {
    launch_with(cf, g, y, x, W, cl, diag, sgn, nrhs, s);  // warm
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3; ++rep) launch_with(cf, g, y, x, W, cl, diag, sgn, nrhs, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestc = cf;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  tune_store(key, bestc);
  return bestc;
}

template <typename R, typename LS>
int launch_bri_t(const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag, int nrhs, int dagger,
                 cudaStream_t s) {
  int rc = ensure_hops();
  if (rc) return rc;
  const R sgn = (R)(dagger ? -1 : 1);
  const StencilConfig cf = tuned_config(g, y, x, W, cl, diag, sgn, nrhs, s);
  launch_with(cf, g, y, x, W, cl, diag, sgn, nrhs, s);
  BRI_LAUNCH_CHECK("bri_kernel");
  return BRI_OK;
}

}  // namespace bri
