// Brillouin and Wilson stencils on CUDA cores (sm_103a).
//
// D_bri x(n) = sum_{d in {-1,0,1}^4, d != 0} W_d(n) M_d x(n+d)
//              + (15/8 + m0) x(n) + C(n) x(n)                        (Eq. def_bril)
// with, for a k-hop offset d (momentum forms of App. A expanded in e^{ip.d}):
//   M_d = -2^{-k-3} 1 + (4^{2-k}/27) sum_{mu: d_mu != 0} sign(d_mu) gamma_mu .
// D^dagger = gamma5 D gamma5 flips the sign of the gamma part only (gamma5
// anticommutes with gamma_mu and commutes with the clover term).
//
// W_d(n) for nu = 1..40 is stored at n; the other 40 are read as
// W_{82-nu}(n+d)^dagger from the neighbour (App. C).  In the chiral basis
//   sum_mu s_mu gamma_mu = [[0, B], [B^dagger, 0]],  B = s_4 - i (s_1 s1 + s_2 s2 + s_3 s3)
// so chi = M_d x needs only additions of +-x and +-i x with a common weight;
// the spin structure is resolved at compile time per offset.  One thread owns
// one site and one right-hand side; links arrive as coalesced structure-of-
// arrays loads, source spinors through L1/L2 (they are reused by 81 sites).
#include "internal.cuh"
#include "cplx.cuh"

#include <cstdlib>
#include <utility>

namespace bri {
namespace {

template <typename R> struct Spinor {
  C<R> v[4][3];
};

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double2; };

// AoS spinor [4][3] complex: 24 reals.
__device__ __forceinline__ void load_spinor(Spinor<float>& s, const float* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float4 v = __ldg(q + i);
    int e0 = 2 * i, e1 = 2 * i + 1;  // complex element index 0..11
    s.v[e0 / 3][e0 % 3] = C<float>{v.x, v.y};
    s.v[e1 / 3][e1 % 3] = C<float>{v.z, v.w};
  }
}
__device__ __forceinline__ void load_spinor(Spinor<double>& s, const double* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    double2 v = __ldg(q + e);
    s.v[e / 3][e % 3] = C<double>{v.x, v.y};
  }
}
__device__ __forceinline__ void store_spinor(float* p, const Spinor<float>& s) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    int e0 = 2 * i, e1 = 2 * i + 1;
    q[i] = make_float4(s.v[e0 / 3][e0 % 3].re, s.v[e0 / 3][e0 % 3].im, s.v[e1 / 3][e1 % 3].re,
                       s.v[e1 / 3][e1 % 3].im);
  }
}
__device__ __forceinline__ void store_spinor(double* p, const Spinor<double>& s) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int e = 0; e < 12; ++e) q[e] = make_double2(s.v[e / 3][e % 3].re, s.v[e / 3][e % 3].im);
}

// r += w * v (w compile-time sign times a runtime-free constant)
template <int S, typename R> __device__ __forceinline__ void acc_term(R& r, R c, R v) {
  if constexpr (S == 1) r = fma(c, v, r);
  else if constexpr (S == -1) r = fma(-c, v, r);
}

// chi = a x + c (sum_mu s_mu gamma_mu) x for constant signs (S1..S4) = d.
template <int S1, int S2, int S3, int S4, typename R>
__device__ __forceinline__ void spin_combine(Spinor<R>& chi, const Spinor<R>& x, R a, R c) {
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const C<R> x0 = x.v[0][col], x1 = x.v[1][col], x2 = x.v[2][col], x3 = x.v[3][col];
    // upper: B x_low, B = [[s4 - i s3, -s2 - i s1], [s2 - i s1, s4 + i s3]]
    R r0 = a * x0.re, i0 = a * x0.im, r1 = a * x1.re, i1 = a * x1.im;
    acc_term<S4>(r0, c, x2.re); acc_term<S4>(i0, c, x2.im);
    acc_term<S3>(r0, c, x2.im); acc_term<-S3>(i0, c, x2.re);
    acc_term<-S2>(r0, c, x3.re); acc_term<-S2>(i0, c, x3.im);
    acc_term<S1>(r0, c, x3.im); acc_term<-S1>(i0, c, x3.re);
    acc_term<S2>(r1, c, x2.re); acc_term<S2>(i1, c, x2.im);
    acc_term<S1>(r1, c, x2.im); acc_term<-S1>(i1, c, x2.re);
    acc_term<S4>(r1, c, x3.re); acc_term<S4>(i1, c, x3.im);
    acc_term<-S3>(r1, c, x3.im); acc_term<S3>(i1, c, x3.re);
    // lower: B^dagger x_up, B^dagger = [[s4 + i s3, s2 + i s1], [-s2 + i s1, s4 - i s3]]
    R r2 = a * x2.re, i2 = a * x2.im, r3 = a * x3.re, i3 = a * x3.im;
    acc_term<S4>(r2, c, x0.re); acc_term<S4>(i2, c, x0.im);
    acc_term<-S3>(r2, c, x0.im); acc_term<S3>(i2, c, x0.re);
    acc_term<S2>(r2, c, x1.re); acc_term<S2>(i2, c, x1.im);
    acc_term<-S1>(r2, c, x1.im); acc_term<S1>(i2, c, x1.re);
    acc_term<-S2>(r3, c, x0.re); acc_term<-S2>(i3, c, x0.im);
    acc_term<-S1>(r3, c, x0.im); acc_term<S1>(i3, c, x0.re);
    acc_term<S4>(r3, c, x1.re); acc_term<S4>(i3, c, x1.im);
    acc_term<S3>(r3, c, x1.im); acc_term<-S3>(i3, c, x1.re);
    chi.v[0][col] = C<R>{r0, i0};
    chi.v[1][col] = C<R>{r1, i1};
    chi.v[2][col] = C<R>{r2, i2};
    chi.v[3][col] = C<R>{r3, i3};
  }
}

template <typename R> struct Nb {
  int64_t o[4][3];  // stride-scaled coordinates of x-1,x,x+1 (etc.), periodic
};

template <typename R> struct HopW {
  R c[5];  // gamma weight of k-hop offsets, sign-flipped for the dagger
};

template <int J, typename R, typename LS>
__device__ __forceinline__ void bri_offset(Spinor<R>& acc, const R* __restrict__ xin, const LS* __restrict__ W,
                                           int64_t V, int64_t n, const Nb<R>& nb, const HopW<R>& hw) {
  constexpr int dx = J % 3 - 1, dy = (J / 3) % 3 - 1, dz = (J / 9) % 3 - 1, dt = (J / 27) % 3 - 1;
  constexpr int k = (dx != 0) + (dy != 0) + (dz != 0) + (dt != 0);
  if constexpr (k == 0) {
    return;
  } else {
    constexpr double a_d = -1.0 / double(1 << (k + 3));
    const int64_t m = nb.o[0][dx + 1] + nb.o[1][dy + 1] + nb.o[2][dz + 1] + nb.o[3][dt + 1];
    Spinor<R> xs, chi;
    load_spinor(xs, xin + m * 24);
    spin_combine<dx, dy, dz, dt, R>(chi, xs, (R)a_d, hw.c[k]);
    C<R> w[3][3];
    if constexpr (J < 40) {
      const LS* wp = W + (int64_t)J * 9 * V + n;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        C<float> t;
        if constexpr (sizeof(R) == 8) {
          w[e / 3][e % 3] = ld2(reinterpret_cast<const double2*>(wp) + (int64_t)e * V);
        } else {
          t = ld2(wp + (int64_t)e * V);
          w[e / 3][e % 3] = C<R>{(R)t.re, (R)t.im};
        }
      }
    } else {  // W_d(n) = W_{-d}(n+d)^dagger
      const LS* wp = W + (int64_t)(80 - J) * 9 * V + m;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        C<R> t;
        if constexpr (sizeof(R) == 8) {
          t = ld2(reinterpret_cast<const double2*>(wp) + (int64_t)e * V);
        } else {
          C<float> f = ld2(wp + (int64_t)e * V);
          t = C<R>{(R)f.re, (R)f.im};
        }
        w[e % 3][e / 3] = conj(t);
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) cfma(acc.v[s][a], w[a][b], chi.v[s][b]);
  }
}

template <typename R, typename LS, int... Js>
__device__ __forceinline__ void bri_all(Spinor<R>& acc, const R* __restrict__ xin, const LS* __restrict__ W,
                                        int64_t V, int64_t n, const Nb<R>& nb, const HopW<R>& hw,
                                        std::integer_sequence<int, Js...>) {
  (bri_offset<Js, R, LS>(acc, xin, W, V, n, nb, hw), ...);
}

template <typename R>
__device__ __forceinline__ void neighbours(const Geom& g, int64_t n, Nb<R>& nb) {
  int64_t r = n;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int L = g.L[mu];
    int c = (mu < 3) ? (int)(r % L) : (int)r;
    if (mu < 3) r /= L;
    int cm = c == 0 ? L - 1 : c - 1;
    int cp = c == L - 1 ? 0 : c + 1;
    nb.o[mu][0] = cm * g.str[mu];
    nb.o[mu][1] = c * g.str[mu];
    nb.o[mu][2] = cp * g.str[mu];
  }
}

// Packed Hermitian 6x6 times a 6-vector: diag reals [0..5], then upper complex.
template <typename R>
__device__ __forceinline__ void clover_block(C<R> out[6], const R* __restrict__ cl, int64_t V, int64_t n,
                                             const C<R> in[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    R d = __ldg(cl + (int64_t)i * V + n);
    out[i] = C<R>{d * in[i].re, d * in[i].im};
  }
  int k = 6;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      C<R> cij{__ldg(cl + (int64_t)k * V + n), __ldg(cl + (int64_t)(k + 1) * V + n)};
      cfma(out[i], cij, in[j]);
      cfma_cj(out[j], cij, in[i]);
      k += 2;
    }
}

template <typename R>
__device__ __forceinline__ void add_clover(Spinor<R>& acc, const Spinor<R>& x, const R* __restrict__ cl,
                                           int64_t V, int64_t n) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    C<R> in[6], out[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) in[i] = x.v[2 * blk + i / 3][i % 3];
    clover_block(out, cl + (int64_t)blk * 36 * V, V, n, in);
#pragma unroll
    for (int i = 0; i < 6; ++i) acc.v[2 * blk + i / 3][i % 3] = acc.v[2 * blk + i / 3][i % 3] + out[i];
  }
}

template <typename R> struct Occ { static constexpr int v = 4; };
template <> struct Occ<double> { static constexpr int v = 2; };

template <typename R, typename LS>
__global__ void __launch_bounds__(128, 2) bri_kernel(Geom g, R* __restrict__ y, const R* __restrict__ x,
                                                  const LS* __restrict__ W, const R* __restrict__ cl, R diag,
                                                  HopW<R> hw) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int64_t rhs_off = (int64_t)blockIdx.y * g.V * 24;
  const R* xin = x + rhs_off;
  Nb<R> nb;
  neighbours(g, n, nb);
  Spinor<R> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.v[s][a] = C<R>{0, 0};
  bri_all<R, LS>(acc, xin, W, g.V, n, nb, hw, std::make_integer_sequence<int, 81>{});
  Spinor<R> xc;
  load_spinor(xc, xin + n * 24);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc.v[s][a].re = fma(diag, xc.v[s][a].re, acc.v[s][a].re);
      acc.v[s][a].im = fma(diag, xc.v[s][a].im, acc.v[s][a].im);
    }
  if (cl) add_clover(acc, xc, cl, g.V, n);
  store_spinor(y + rhs_off + n * 24, acc);
}

// ------------------------------------------------------------- loop variant
// Same operator, written as a runtime loop over the 40 stored offsets d; each
// iteration also handles the opposite offset -d, whose transporter is the
// stored link of d at the neighbour n-d, daggered.  The signs of d enter as
// runtime weights c*s_mu, which costs a few more FMAs than the compile-time
// folding above but keeps the live register set small and the code compact.
struct OffTab {
  int d[40][4];
  float af[40], cf[40];
  double ad[40], cd[40];
};
__constant__ OffTab c_off;

template <typename R> __device__ __forceinline__ R tab_a(int j);
template <> __device__ __forceinline__ float tab_a<float>(int j) { return c_off.af[j]; }
template <> __device__ __forceinline__ double tab_a<double>(int j) { return c_off.ad[j]; }
template <typename R> __device__ __forceinline__ R tab_c(int j);
template <> __device__ __forceinline__ float tab_c<float>(int j) { return c_off.cf[j]; }
template <> __device__ __forceinline__ double tab_c<double>(int j) { return c_off.cd[j]; }

// chi = a x + (sum_mu cs_mu gamma_mu) x, cs_mu = c s_mu (runtime)
template <typename R>
__device__ __forceinline__ void spin_combine_rt(Spinor<R>& chi, const Spinor<R>& x, R a, R c1, R c2, R c3, R c4) {
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const C<R> x0 = x.v[0][col], x1 = x.v[1][col], x2 = x.v[2][col], x3 = x.v[3][col];
    R r0 = a * x0.re, i0 = a * x0.im, r1 = a * x1.re, i1 = a * x1.im;
    R r2 = a * x2.re, i2 = a * x2.im, r3 = a * x3.re, i3 = a * x3.im;
    r0 = fma(c4, x2.re, r0); r0 = fma(c3, x2.im, r0); r0 = fma(-c2, x3.re, r0); r0 = fma(c1, x3.im, r0);
    i0 = fma(c4, x2.im, i0); i0 = fma(-c3, x2.re, i0); i0 = fma(-c2, x3.im, i0); i0 = fma(-c1, x3.re, i0);
    r1 = fma(c2, x2.re, r1); r1 = fma(c1, x2.im, r1); r1 = fma(c4, x3.re, r1); r1 = fma(-c3, x3.im, r1);
    i1 = fma(c2, x2.im, i1); i1 = fma(-c1, x2.re, i1); i1 = fma(c4, x3.im, i1); i1 = fma(c3, x3.re, i1);
    r2 = fma(c4, x0.re, r2); r2 = fma(-c3, x0.im, r2); r2 = fma(c2, x1.re, r2); r2 = fma(-c1, x1.im, r2);
    i2 = fma(c4, x0.im, i2); i2 = fma(c3, x0.re, i2); i2 = fma(c2, x1.im, i2); i2 = fma(c1, x1.re, i2);
    r3 = fma(-c2, x0.re, r3); r3 = fma(-c1, x0.im, r3); r3 = fma(c4, x1.re, r3); r3 = fma(c3, x1.im, r3);
    i3 = fma(-c2, x0.im, i3); i3 = fma(c1, x0.re, i3); i3 = fma(c4, x1.im, i3); i3 = fma(-c3, x1.re, i3);
    chi.v[0][col] = C<R>{r0, i0};
    chi.v[1][col] = C<R>{r1, i1};
    chi.v[2][col] = C<R>{r2, i2};
    chi.v[3][col] = C<R>{r3, i3};
  }
}

template <typename R, typename LS>
__device__ __forceinline__ void load_link(C<R> w[3][3], const LS* __restrict__ p, int V) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    if constexpr (sizeof(R) == 8) {
      w[e / 3][e % 3] = ld2(reinterpret_cast<const double2*>(p) + e * V);
    } else {
      C<float> f = ld2(p + e * V);
      w[e / 3][e % 3] = C<R>{(R)f.re, (R)f.im};
    }
  }
}

__device__ __forceinline__ int wrap(int c, int L) { return c < 0 ? c + L : (c >= L ? c - L : c); }

template <typename R, typename LS>
__global__ void __launch_bounds__(128, Occ<R>::v) bri_kernel_loop(Geom g, R* __restrict__ y, const R* __restrict__ x,
                                                               const LS* __restrict__ W, const R* __restrict__ cl,
                                                               R diag, R sgn) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int V = (int)g.V;
  const int64_t rhs_off = (int64_t)blockIdx.y * g.V * 24;
  const R* xin = x + rhs_off;
  int co[4];
  {
    int r = n;
    co[0] = r % g.L[0]; r /= g.L[0];
    co[1] = r % g.L[1]; r /= g.L[1];
    co[2] = r % g.L[2]; r /= g.L[2];
    co[3] = r;
  }
  const int s1 = (int)g.str[1], s2 = (int)g.str[2], s3 = (int)g.str[3];
  Spinor<R> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.v[s][a] = C<R>{0, 0};
#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    const int dx = c_off.d[j][0], dy = c_off.d[j][1], dz = c_off.d[j][2], dt = c_off.d[j][3];
    const R a = tab_a<R>(j), c = sgn * tab_c<R>(j);
    const R c1 = c * (R)dx, c2 = c * (R)dy, c3 = c * (R)dz, c4 = c * (R)dt;
    const int mp = wrap(co[0] + dx, g.L[0]) + wrap(co[1] + dy, g.L[1]) * s1 + wrap(co[2] + dz, g.L[2]) * s2 +
                   wrap(co[3] + dt, g.L[3]) * s3;
    const int mm = wrap(co[0] - dx, g.L[0]) + wrap(co[1] - dy, g.L[1]) * s1 + wrap(co[2] - dz, g.L[2]) * s2 +
                   wrap(co[3] - dt, g.L[3]) * s3;
    const LS* wj = W + (int64_t)j * 9 * V;
    {  // +d: W_d(n) M_d x(n+d)
      Spinor<R> xs, chi;
      C<R> w[3][3];
      load_spinor(xs, xin + (int64_t)mp * 24);
      load_link<R, LS>(w, wj + n, V);
      spin_combine_rt(chi, xs, a, c1, c2, c3, c4);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
          for (int b = 0; b < 3; ++b) cfma(acc.v[s][aa], w[aa][b], chi.v[s][b]);
    }
    {  // -d: W_d(n-d)^dagger M_{-d} x(n-d)
      Spinor<R> xs, chi;
      C<R> w[3][3];
      load_spinor(xs, xin + (int64_t)mm * 24);
      load_link<R, LS>(w, wj + mm, V);
      spin_combine_rt(chi, xs, a, -c1, -c2, -c3, -c4);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
          for (int b = 0; b < 3; ++b) cfma_cj(acc.v[s][aa], w[b][aa], chi.v[s][b]);
    }
  }
  Spinor<R> xc;
  load_spinor(xc, xin + (int64_t)n * 24);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc.v[s][a].re = fma(diag, xc.v[s][a].re, acc.v[s][a].re);
      acc.v[s][a].im = fma(diag, xc.v[s][a].im, acc.v[s][a].im);
    }
  if (cl) add_clover(acc, xc, cl, g.V, n);
  store_spinor(y + rhs_off + (int64_t)n * 24, acc);
}

// ----------------------------------------------------------------- Wilson
// Spin projection (chiral basis): (1 -+ gamma_mu) x is fixed by its upper half
// h = x_up -+ e_mu x_low (e_k = -i sigma_k, e_4 = 1); its lower half is
// -+ e_mu^dagger h.  U acts on h only (2 spins), then the lower half is rebuilt.
template <typename R> __device__ __forceinline__ C<R> mul_i(C<R> a) { return C<R>{-a.im, a.re}; }
template <typename R> __device__ __forceinline__ C<R> neg(C<R> a) { return C<R>{-a.re, -a.im}; }

// PLUS = true for (1 + gamma_mu), false for (1 - gamma_mu)
template <int MU, bool PLUS, typename R>
__device__ __forceinline__ void project(const Spinor<R>& x, C<R> h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const C<R> x0 = x.v[0][c], x1 = x.v[1][c], x2 = x.v[2][c], x3 = x.v[3][c];
    if constexpr (MU == 0) {
      h[0][c] = PLUS ? x0 - mul_i(x3) : x0 + mul_i(x3);
      h[1][c] = PLUS ? x1 - mul_i(x2) : x1 + mul_i(x2);
    } else if constexpr (MU == 1) {
      h[0][c] = PLUS ? x0 - x3 : x0 + x3;
      h[1][c] = PLUS ? x1 + x2 : x1 - x2;
    } else if constexpr (MU == 2) {
      h[0][c] = PLUS ? x0 - mul_i(x2) : x0 + mul_i(x2);
      h[1][c] = PLUS ? x1 + mul_i(x3) : x1 - mul_i(x3);
    } else {
      h[0][c] = PLUS ? x0 + x2 : x0 - x2;
      h[1][c] = PLUS ? x1 + x3 : x1 - x3;
    }
  }
}

// acc += -1/2 * (projected, transported) spinor reconstructed from uh
template <int MU, bool PLUS, typename R>
__device__ __forceinline__ void reconstruct(Spinor<R>& acc, const C<R> uh[2][3]) {
  const R hf = (R)-0.5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C<R> h0 = uh[0][c], h1 = uh[1][c], v2, v3;
    if constexpr (MU == 0) {
      v2 = PLUS ? mul_i(h1) : neg(mul_i(h1));
      v3 = PLUS ? mul_i(h0) : neg(mul_i(h0));
    } else if constexpr (MU == 1) {
      v2 = PLUS ? h1 : neg(h1);
      v3 = PLUS ? neg(h0) : h0;
    } else if constexpr (MU == 2) {
      v2 = PLUS ? mul_i(h0) : neg(mul_i(h0));
      v3 = PLUS ? neg(mul_i(h1)) : mul_i(h1);
    } else {
      v2 = PLUS ? h0 : neg(h0);
      v3 = PLUS ? h1 : neg(h1);
    }
    acc.v[0][c] = acc.v[0][c] + hf * h0;
    acc.v[1][c] = acc.v[1][c] + hf * h1;
    acc.v[2][c] = acc.v[2][c] + hf * v2;
    acc.v[3][c] = acc.v[3][c] + hf * v3;
  }
}

template <int MU, typename R, typename LS, bool DAG>
__device__ __forceinline__ void wil_dir(Spinor<R>& acc, const R* __restrict__ xin, const LS* __restrict__ U,
                                        int64_t V, int64_t n, const Nb<R>& nb) {
  // forward: -1/2 (1 - gamma_mu) U_mu(n) x(n+mu); backward: -1/2 (1 + gamma_mu) U_mu(n-mu)^+ x(n-mu)
  // (dagger swaps the two projectors).
  int64_t mf = nb.o[0][1] + nb.o[1][1] + nb.o[2][1] + nb.o[3][1] - nb.o[MU][1] + nb.o[MU][2];
  int64_t mb = nb.o[0][1] + nb.o[1][1] + nb.o[2][1] + nb.o[3][1] - nb.o[MU][1] + nb.o[MU][0];
  {
    Spinor<R> xs;
    load_spinor(xs, xin + mf * 24);
    C<R> h[2][3], uh[2][3];
    project<MU, DAG>(xs, h);
    C<R> u[3][3];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      C<float> f;
      if constexpr (sizeof(R) == 8) u[e / 3][e % 3] = ld2(reinterpret_cast<const double2*>(U) + ((int64_t)MU * 9 + e) * V + n);
      else { f = ld2(U + ((int64_t)MU * 9 + e) * V + n); u[e / 3][e % 3] = C<R>{(R)f.re, (R)f.im}; }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        uh[s][a] = C<R>{0, 0};
#pragma unroll
        for (int b = 0; b < 3; ++b) cfma(uh[s][a], u[a][b], h[s][b]);
      }
    reconstruct<MU, DAG>(acc, uh);
  }
  {
    Spinor<R> xs;
    load_spinor(xs, xin + mb * 24);
    C<R> h[2][3], uh[2][3];
    project<MU, !DAG>(xs, h);
    C<R> u[3][3];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      C<float> f;
      if constexpr (sizeof(R) == 8) u[e / 3][e % 3] = ld2(reinterpret_cast<const double2*>(U) + ((int64_t)MU * 9 + e) * V + mb);
      else { f = ld2(U + ((int64_t)MU * 9 + e) * V + mb); u[e / 3][e % 3] = C<R>{(R)f.re, (R)f.im}; }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        uh[s][a] = C<R>{0, 0};
#pragma unroll
        for (int b = 0; b < 3; ++b) cfma_cj(uh[s][a], u[b][a], h[s][b]);
      }
    reconstruct<MU, !DAG>(acc, uh);
  }
}

template <typename R, typename LS, bool DAG, bool CLOV>
__global__ void __launch_bounds__(128) wil_kernel(Geom g, R* __restrict__ y, const R* __restrict__ x,
                                                  const LS* __restrict__ U, const R* __restrict__ cl, R diag) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int64_t rhs_off = (int64_t)blockIdx.y * g.V * 24;
  const R* xin = x + rhs_off;
  Nb<R> nb;
  neighbours(g, n, nb);
  Spinor<R> acc, xc;
  load_spinor(xc, xin + n * 24);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.v[s][a] = diag * xc.v[s][a];
  wil_dir<0, R, LS, DAG>(acc, xin, U, g.V, n, nb);
  wil_dir<1, R, LS, DAG>(acc, xin, U, g.V, n, nb);
  wil_dir<2, R, LS, DAG>(acc, xin, U, g.V, n, nb);
  wil_dir<3, R, LS, DAG>(acc, xin, U, g.V, n, nb);
  if constexpr (CLOV) add_clover(acc, xc, cl, g.V, n);
  store_spinor(y + rhs_off + n * 24, acc);
}

// 0: loop kernel (default), 1: fully unrolled kernel; BRI_STENCIL_VARIANT overrides.
int stencil_variant() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("BRI_STENCIL_VARIANT");
    v = e ? atoi(e) : 0;
  }
  return v;
}

// Stored offsets nu = 1..40 (most significant nonzero component -1), their
// identity weight -2^{-k-3} and gamma weight 4^{2-k}/27 (App. A expanded).
int upload_offset_table() {
  static int done_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (done_dev == dev) return BRI_OK;
  OffTab t;
  for (int j = 0; j < 40; ++j) {
    int d[4] = {j % 3 - 1, (j / 3) % 3 - 1, (j / 9) % 3 - 1, (j / 27) % 3 - 1};
    int k = 0;
    for (int mu = 0; mu < 4; ++mu) {
      t.d[j][mu] = d[mu];
      k += d[mu] != 0;
    }
    t.ad[j] = -1.0 / double(1 << (k + 3));
    t.cd[j] = double(1 << (2 * (4 - k))) / 432.0;
    t.af[j] = (float)t.ad[j];
    t.cf[j] = (float)t.cd[j];
  }
  BRI_CUDA(cudaMemcpyToSymbol(c_off, &t, sizeof(t)));
  done_dev = dev;
  return BRI_OK;
}

template <typename R, typename LS>
int launch_bri(const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag, int nrhs, int dagger,
               cudaStream_t s) {
  const int th = 128;
  dim3 grid(blocks_for(g.V, th), nrhs);
  if (stencil_variant() == 1) {
    HopW<R> hw;
    hw.c[0] = 0;
    for (int k = 1; k <= 4; ++k) hw.c[k] = (R)((dagger ? -1.0 : 1.0) * double(1 << (2 * (4 - k))) / 432.0);
    bri_kernel<R, LS><<<grid, th, 0, s>>>(g, y, x, W, cl, diag, hw);
    note_launch();
  } else {
    int rc = upload_offset_table();
    if (rc) return rc;
    bri_kernel_loop<R, LS><<<grid, th, 0, s>>>(g, y, x, W, cl, diag, (R)(dagger ? -1 : 1));
    note_launch();
  }
  BRI_LAUNCH_CHECK("bri_kernel");
  return BRI_OK;
}

template <typename R, typename LS>
int launch_wil(const Geom& g, R* y, const R* x, const LS* U, const R* cl, R diag, int nrhs, int dagger,
               cudaStream_t s) {
  const int th = 128;
  dim3 grid(blocks_for(g.V, th), nrhs);
  if (dagger) {
    if (cl) wil_kernel<R, LS, true, true><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    else wil_kernel<R, LS, true, false><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    note_launch();
  } else {
    if (cl) wil_kernel<R, LS, false, true><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    else wil_kernel<R, LS, false, false><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    note_launch();
  }
  BRI_LAUNCH_CHECK("wil_kernel");
  return BRI_OK;
}

}  // namespace

int dirac_bri(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec, cudaStream_t s) {
  const double diag = 15.0 / 8.0 + m0;
  cudaEvent_t ev;
  int rc = prof_begin(c, s, &ev);
  if (rc) return rc;
  switch (prec) {
    case BRI_PREC_F64:
      rc = launch_bri<double, double2>(c->g, (double*)y, (const double*)x, c->W64,
                                       c->have_clover ? c->C64 : nullptr, diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32:
      rc = launch_bri<float, float2>(c->g, (float*)y, (const float*)x, c->W32,
                                     c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32_BF16:
      rc = launch_bri<float, __nv_bfloat162>(c->g, (float*)y, (const float*)x, c->W16,
                                             c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, dagger, s);
      break;
    default:
      set_error("bri_apply: unknown precision");
      return BRI_ERR_INVALID;
  }
  if (rc) return rc;
  return prof_end(c, s, ev, 0, prec, (double)c->g.V * nrhs);
}

int dirac_wil(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec, cudaStream_t s) {
  const double diag = 4.0 + m0;
  cudaEvent_t ev;
  int rc = prof_begin(c, s, &ev);
  if (rc) return rc;
  switch (prec) {
    case BRI_PREC_F64:
      rc = launch_wil<double, double2>(c->g, (double*)y, (const double*)x, c->U64,
                                       c->have_clover ? c->C64 : nullptr, diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32:
    case BRI_PREC_F32_BF16:
      rc = launch_wil<float, float2>(c->g, (float*)y, (const float*)x, c->U32,
                                     c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, dagger, s);
      break;
    default:
      set_error("wils_apply: unknown precision");
      return BRI_ERR_INVALID;
  }
  if (rc) return rc;
  return prof_end(c, s, ev, 1, prec, (double)c->g.V * nrhs);
}

}  // namespace bri
