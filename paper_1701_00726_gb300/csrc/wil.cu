// Wilson stencil (Eq. def_wils) with spin projection (App. C, Wilson operator
// flop count): for each of the 8 hops the 4-spinor is projected to 2 spin
// components with (1 -+ gamma_mu), transported, and rebuilt.
#include "stencil.cuh"

namespace bri {
namespace {

template <typename R> struct Nb {
  int64_t o[4][3];  // stride-scaled coordinates of x-1, x, x+1 (etc.), periodic
};

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

}  // namespace

template <typename R, typename LS>
int launch_wil_t(const Geom& g, R* y, const R* x, const LS* U, const R* cl, R diag, int nrhs, int dagger,
                 cudaStream_t s) {
  const int th = 128;
  dim3 grid(blocks_for(g.V, th), nrhs);
  if (dagger) {
    if (cl) wil_kernel<R, LS, true, true><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    else wil_kernel<R, LS, true, false><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
  } else {
    if (cl) wil_kernel<R, LS, false, true><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
    else wil_kernel<R, LS, false, false><<<grid, th, 0, s>>>(g, y, x, U, cl, diag);
  }
  note_launch();
  BRI_LAUNCH_CHECK("wil_kernel");
  return BRI_OK;
}

template int launch_wil_t<double, double2>(const Geom&, double*, const double*, const double2*, const double*,
                                           double, int, int, cudaStream_t);
template int launch_wil_t<float, float2>(const Geom&, float*, const float*, const float2*, const float*, float, int,
                                         int, cudaStream_t);

}  // namespace bri
