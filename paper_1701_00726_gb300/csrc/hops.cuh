// Per-offset constants of the Brillouin stencil and the spin algebra of its
// hops, shared by the stencil kernel and the adjoint (force) kernel.
#pragma once

#include "stencil.cuh"

namespace bri {

// Stored offsets nu = 1..40 with their identity weight -2^{-k-3} and the
// signed gamma weights c_k s_mu, c_k = 4^{2-k}/27.
template <typename R> struct HopTable {
  int site_d[40][4];
  R a[40];
  R cs[40][4];
};
template <typename R> void fill_hops(HopTable<R>& h) {
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

// The table of one precision, built once per process on the host and passed
// to the kernels by value (a __grid_constant__ parameter, read from the
// constant bank), so no translation unit has device state to upload.
template <typename R> const HopTable<R>& hop_table() {
  static const HopTable<R> t = [] {
    HopTable<R> h;
    fill_hops(h);
    return h;
  }();
  return t;
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

// acc += c gamma_mu v over one colour (four spins), chiral basis (the same
// spin structure as spin_combine): MU = 1..4.
template <int MU, typename R>
__device__ __forceinline__ void gamma_term(C<R> acc[4], const C<R> v[4], R c) {
  if constexpr (MU == 1) {
    acc[0].re = fma(c, v[3].im, acc[0].re); acc[0].im = fma(-c, v[3].re, acc[0].im);
    acc[1].re = fma(c, v[2].im, acc[1].re); acc[1].im = fma(-c, v[2].re, acc[1].im);
    acc[2].re = fma(-c, v[1].im, acc[2].re); acc[2].im = fma(c, v[1].re, acc[2].im);
    acc[3].re = fma(-c, v[0].im, acc[3].re); acc[3].im = fma(c, v[0].re, acc[3].im);
  } else if constexpr (MU == 2) {
    acc[0].re = fma(-c, v[3].re, acc[0].re); acc[0].im = fma(-c, v[3].im, acc[0].im);
    acc[1].re = fma(c, v[2].re, acc[1].re); acc[1].im = fma(c, v[2].im, acc[1].im);
    acc[2].re = fma(c, v[1].re, acc[2].re); acc[2].im = fma(c, v[1].im, acc[2].im);
    acc[3].re = fma(-c, v[0].re, acc[3].re); acc[3].im = fma(-c, v[0].im, acc[3].im);
  } else if constexpr (MU == 3) {
    acc[0].re = fma(c, v[2].im, acc[0].re); acc[0].im = fma(-c, v[2].re, acc[0].im);
    acc[1].re = fma(-c, v[3].im, acc[1].re); acc[1].im = fma(c, v[3].re, acc[1].im);
    acc[2].re = fma(-c, v[0].im, acc[2].re); acc[2].im = fma(c, v[0].re, acc[2].im);
    acc[3].re = fma(c, v[1].im, acc[3].re); acc[3].im = fma(-c, v[1].re, acc[3].im);
  } else {
    acc[0].re = fma(c, v[2].re, acc[0].re); acc[0].im = fma(c, v[2].im, acc[0].im);
    acc[1].re = fma(c, v[3].re, acc[1].re); acc[1].im = fma(c, v[3].im, acc[1].im);
    acc[2].re = fma(c, v[0].re, acc[2].re); acc[2].im = fma(c, v[0].im, acc[2].im);
    acc[3].re = fma(c, v[1].re, acc[3].re); acc[3].im = fma(c, v[1].im, acc[3].im);
  }
}

// One colour of the accumulator (four spins): acc += a u + sum_mu cs_mu gamma_mu v.
template <typename R>
__device__ __forceinline__ void add_pair_terms(C<R> acc[4], const C<R> u[4], const C<R> v[4], R a, R c1, R c2,
                                               R c3, R c4) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    acc[s].re = fma(a, u[s].re, acc[s].re);
    acc[s].im = fma(a, u[s].im, acc[s].im);
  }
  gamma_term<1>(acc, v, c1);
  gamma_term<2>(acc, v, c2);
  gamma_term<3>(acc, v, c3);
  gamma_term<4>(acc, v, c4);
}

}  // namespace bri
