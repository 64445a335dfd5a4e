// Brillouin stencil on the paired FP32 pipe (fma.rn.f32x2 through __ffma2_rn)
// with the real and imaginary part of one complex number as the pair: a
// spinor component loads as a native (re, im) register pair, and the complex
// products become
//   w x     = (w_re, w_re) (x_re, x_im) + (w_im, w_im) (-x_im, x_re),
//   w^* x   = (w_re, w_re) (x_re, x_im) + (-w_im, -w_im) (-x_im, x_re),
// so each paired FMA does two of the scalar kernel's FMAs in one issue slot.
//
// The arithmetic is that of the scalar kernel (Eq. def_bril, App. A): per
// stored offset d the hop pair contributes a_k (P + Q) + c_k G (P - Q) with
// P = W_d(n) x(n+d), Q = W_d(n-d)^dagger x(n-d).  Q is accumulated onto P
// (u = P + Q) and the difference is formed as vn = u - 2P = -(P - Q); the
// gamma part is applied to vn with negated weights.
#pragma once

#include "hops.cuh"

namespace bri {

// Per-offset weights as the constant pairs the paired arithmetic needs, for D
// (dagger = 0) or D^dagger (dagger = 1), c_mu = sgn c_k s_mu:
//   k[0] = (a, a),
//   k[1] = (-c1, c1), k[2] = (c1, -c1),   gamma_1 rows on swapped (im, re) pairs
//   k[3] = (c2, c2),  k[4] = (-c2, -c2),  gamma_2
//   k[5] = (-c3, c3), k[6] = (c3, -c3),   gamma_3 rows on swapped pairs
//   k[7] = (-c4, -c4)                     gamma_4
// (signs for the vector vn = -(P - Q)).
struct HopTableC2 {
  int site_d[40][4];
  float2 k[40][8];
};

inline HopTableC2 make_hop_table_c2(int dagger) {
  const HopTable<float>& h = hop_table<float>();
  HopTableC2 t;
  const float sgn = dagger ? -1.f : 1.f;
  for (int j = 0; j < 40; ++j) {
    for (int mu = 0; mu < 4; ++mu) t.site_d[j][mu] = h.site_d[j][mu];
    const float c1 = sgn * h.cs[j][0], c2 = sgn * h.cs[j][1], c3 = sgn * h.cs[j][2], c4 = sgn * h.cs[j][3];
    t.k[j][0] = make_float2(h.a[j], h.a[j]);
    t.k[j][1] = make_float2(-c1, c1);
    t.k[j][2] = make_float2(c1, -c1);
    t.k[j][3] = make_float2(c2, c2);
    t.k[j][4] = make_float2(-c2, -c2);
    t.k[j][5] = make_float2(-c3, c3);
    t.k[j][6] = make_float2(c3, -c3);
    t.k[j][7] = make_float2(-c4, -c4);
  }
  return t;
}

inline const HopTableC2& hop_table_c2(int dagger) {
  static const HopTableC2 t0 = make_hop_table_c2(0);
  static const HopTableC2 t1 = make_hop_table_c2(1);
  return dagger ? t1 : t0;
}

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// Sum of v over the block (FP64, fixed order), valid in thread 0.
__device__ __forceinline__ double block_total_c2(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 swp(float2 v) { return make_float2(v.y, v.x); }
__device__ __forceinline__ float2 rot(float2 v) { return make_float2(-v.y, v.x); }  // i v

// A spinor as (re, im) pairs, loaded with 16-byte loads.
struct SpinorF2 {
  float2 v[4][3];
};
__device__ __forceinline__ void load_spinor_f2(SpinorF2& s, const float* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float4 v = __ldg(q + i);
    const int e0 = 2 * i, e1 = 2 * i + 1;
    s.v[e0 / 3][e0 % 3] = make_float2(v.x, v.y);
    s.v[e1 / 3][e1 % 3] = make_float2(v.z, v.w);
  }
}

// acc += A u + (c G) v over one colour (four spins) with w = vn = -v and the
// constant pairs of HopTableC2 (same spin pattern as gamma_term).
__device__ __forceinline__ void pair_terms_c2(float2 acc[4], const float2 u[4], const float2 w[4], const float2* K) {
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = fma2(K[0], u[s], acc[s]);
  const float2 s0 = swp(w[0]), s1 = swp(w[1]), s2 = swp(w[2]), s3 = swp(w[3]);
  // gamma_1
  acc[0] = fma2(K[1], s3, acc[0]);
  acc[1] = fma2(K[1], s2, acc[1]);
  acc[2] = fma2(K[2], s1, acc[2]);
  acc[3] = fma2(K[2], s0, acc[3]);
  // gamma_2
  acc[0] = fma2(K[3], w[3], acc[0]);
  acc[1] = fma2(K[4], w[2], acc[1]);
  acc[2] = fma2(K[4], w[1], acc[2]);
  acc[3] = fma2(K[3], w[0], acc[3]);
  // gamma_3
  acc[0] = fma2(K[5], s2, acc[0]);
  acc[1] = fma2(K[6], s3, acc[1]);
  acc[2] = fma2(K[6], s0, acc[2]);
  acc[3] = fma2(K[5], s1, acc[3]);
  // gamma_4
  acc[0] = fma2(K[7], w[2], acc[0]);
  acc[1] = fma2(K[7], w[3], acc[1]);
  acc[2] = fma2(K[7], w[0], acc[2]);
  acc[3] = fma2(K[7], w[1], acc[3]);
}

// One hop pair on the paired pipe: acc += a (P + Q) + c G (P - Q) with
// P = W_d(n) x(n+d), Q = W_d(n-d)^dagger x(n-d); w = W_d(n), wm = W_d(n-d)
// already in registers, K the pair constants of this offset.
__device__ __forceinline__ void c2_pair(float2 (&acc)[4][3], const float* __restrict__ xin, int mp, int mm,
                                        const C<float> (&w)[3][3], const C<float> (&wm)[3][3],
                                        const float2* __restrict__ Kp) {
  const float2 m2 = bc2(-2.f);
  // P = W_d(n) x(n+d)
  float2 P[4][3];
  {
    SpinorF2 xs;
    load_spinor_f2(xs, xin + (int64_t)mp * 24);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 ix[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) ix[s] = rot(xs.v[s][b]);
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        const float2 wr = bc2(w[aa][b].re), wi = bc2(w[aa][b].im);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          P[s][aa] = b == 0 ? mul2(wr, xs.v[s][b]) : fma2(wr, xs.v[s][b], P[s][aa]);
          P[s][aa] = fma2(wi, ix[s], P[s][aa]);
        }
      }
    }
  }
  // u = P + W_d(n-d)^dagger x(n-d), vn = u - 2P
  SpinorF2 xs;
  load_spinor_f2(xs, xin + (int64_t)mm * 24);
  float2 U[4][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float2 ix[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) ix[s] = rot(xs.v[s][b]);
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      const float2 wr = bc2(wm[b][aa].re), nwi = bc2(-wm[b][aa].im);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        U[s][aa] = fma2(wr, xs.v[s][b], b == 0 ? P[s][aa] : U[s][aa]);
        U[s][aa] = fma2(nwi, ix[s], U[s][aa]);
      }
    }
  }
  float2 K[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) K[i] = Kp[i];
#pragma unroll
  for (int aa = 0; aa < 3; ++aa) {
    float2 u[4], vn[4], col[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      u[s] = U[s][aa];
      vn[s] = fma2(m2, P[s][aa], U[s][aa]);
      col[s] = acc[s][aa];
    }
    pair_terms_c2(col, u, vn, K);
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s][aa] = col[s];
  }
}

// One thread per site and right-hand side; the grid order of rhs and site
// blocks is that of stencil_grid (gfirst).
template <typename LS, bool EPI>
__global__ void __launch_bounds__(128, 4)
    bri_kernel_c2(Geom g, float* __restrict__ y, const float* __restrict__ x, const LS* __restrict__ W,
                  const float* __restrict__ cl, float diag, int rhs0, int gfirst,
                  const __grid_constant__ HopTableC2 H, ShiftDot<float> sd) {
  const int grp = gfirst ? blockIdx.x : blockIdx.y, blk = gfirst ? blockIdx.y : blockIdx.x;
  const int n0 = blk * blockDim.x + threadIdx.x;
  if (!EPI && n0 >= g.V) return;
  // with the epilogue every thread takes part in the block's reduction
  const bool valid = n0 < g.V;
  const int n = valid ? n0 : 0;
  const int V = (int)g.V;
  const int64_t rstride = g.V * 24;
  const int64_t roff = (int64_t)(rhs0 + grp) * rstride;
  const float* xin = x + roff;
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
  float2 acc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) acc[s][aa] = make_float2(0.f, 0.f);
  auto sites = [&](int j, int& mp, int& mm) {
    mp = 0;
    mm = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int d = H.site_d[j][mu];
      mp += wrap(co[mu] + d, L[mu]) * str[mu];
      mm += wrap(co[mu] - d, L[mu]) * str[mu];
    }
  };
#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    int mp, mm;
    sites(j, mp, mm);
    C<float> w[3][3], wm[3][3];
    load_stored_link<float, LS>(w, W, j, n, V);
    load_stored_link<float, LS>(wm, W, j, mm, V);
    c2_pair(acc, xin, mp, mm, w, wm, H.k[j]);
  }
  Spinor<float> xc, out;
  load_spinor(xc, xin + (int64_t)n * 24);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      out.v[s][aa].re = fmaf(diag, xc.v[s][aa].re, acc[s][aa].x);
      out.v[s][aa].im = fmaf(diag, xc.v[s][aa].im, acc[s][aa].y);
    }
  if (cl) add_clover(out, xc, cl, g.V, n);
  if constexpr (EPI) {
    const int s = rhs0 + grp;
    const float sg = (float)sd.sig[s];
    Spinor<float> pv;
    load_spinor(pv, sd.p + roff + (int64_t)n * 24);
    float dt = 0.f;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        out.v[sp][aa].re = fmaf(sg, pv.v[sp][aa].re, out.v[sp][aa].re);
        out.v[sp][aa].im = fmaf(sg, pv.v[sp][aa].im, out.v[sp][aa].im);
        dt = fmaf(pv.v[sp][aa].re, out.v[sp][aa].re, dt);
        dt = fmaf(pv.v[sp][aa].im, out.v[sp][aa].im, dt);
      }
    if (valid) store_spinor(y + roff + (int64_t)n * 24, out);
    const double t = block_total_c2(valid ? (double)dt : 0.0);
    if (threadIdx.x == 0) sd.part[(int64_t)s * (gfirst ? gridDim.y : gridDim.x) + blk] = t;
  } else {
    store_spinor(y + roff + (int64_t)n * 24, out);
  }
}

// Two right-hand sides per thread on the paired pipe: the links of a hop pair
// (and their broadcast pairs) are loaded once and used for both; the grid's
// groups are rhs pairs (rhs0 + 2 grp, rhs0 + 2 grp + 1).
template <typename LS, bool EPI>
__global__ void __launch_bounds__(128, 3)
    bri_kernel_c2x2(Geom g, float* __restrict__ y, const float* __restrict__ x, const LS* __restrict__ W,
                    const float* __restrict__ cl, float diag, int rhs0, int gfirst,
                    const __grid_constant__ HopTableC2 H, ShiftDot<float> sd) {
  const int grp = gfirst ? blockIdx.x : blockIdx.y, blk = gfirst ? blockIdx.y : blockIdx.x;
  const int n0 = blk * blockDim.x + threadIdx.x;
  if (!EPI && n0 >= g.V) return;
  const bool valid = n0 < g.V;
  const int n = valid ? n0 : 0;
  const int V = (int)g.V;
  const int64_t rstride = g.V * 24;
  const int s0 = rhs0 + 2 * grp;
  const int64_t roff = (int64_t)s0 * rstride;
  const float* xin0 = x + roff;
  const float* xin1 = xin0 + rstride;
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
  float2 acc0[4][3], acc1[4][3];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      acc0[sp][aa] = make_float2(0.f, 0.f);
      acc1[sp][aa] = make_float2(0.f, 0.f);
    }
#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    int mp = 0, mm = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int d = H.site_d[j][mu];
      mp += wrap(co[mu] + d, L[mu]) * str[mu];
      mm += wrap(co[mu] - d, L[mu]) * str[mu];
    }
    C<float> w[3][3], wm[3][3];
    load_stored_link<float, LS>(w, W, j, n, V);
    load_stored_link<float, LS>(wm, W, j, mm, V);
    c2_pair(acc0, xin0, mp, mm, w, wm, H.k[j]);
    c2_pair(acc1, xin1, mp, mm, w, wm, H.k[j]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* xr = r ? xin1 : xin0;
    const float2(&acc)[4][3] = r ? acc1 : acc0;
    const int64_t ro = roff + r * rstride;
    Spinor<float> xc, out;
    load_spinor(xc, xr + (int64_t)n * 24);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        out.v[sp][aa].re = fmaf(diag, xc.v[sp][aa].re, acc[sp][aa].x);
        out.v[sp][aa].im = fmaf(diag, xc.v[sp][aa].im, acc[sp][aa].y);
      }
    if (cl) add_clover(out, xc, cl, g.V, n);
    if constexpr (EPI) {
      const int s = s0 + r;
      const float sg = (float)sd.sig[s];
      Spinor<float> pv;
      load_spinor(pv, sd.p + ro + (int64_t)n * 24);
      float dt = 0.f;
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          out.v[sp][aa].re = fmaf(sg, pv.v[sp][aa].re, out.v[sp][aa].re);
          out.v[sp][aa].im = fmaf(sg, pv.v[sp][aa].im, out.v[sp][aa].im);
          dt = fmaf(pv.v[sp][aa].re, out.v[sp][aa].re, dt);
          dt = fmaf(pv.v[sp][aa].im, out.v[sp][aa].im, dt);
        }
      if (valid) store_spinor(y + ro + (int64_t)n * 24, out);
      const double t = block_total_c2(valid ? (double)dt : 0.0);
      if (threadIdx.x == 0) sd.part[(int64_t)s * (gfirst ? gridDim.y : gridDim.x) + blk] = t;
    } else {
      store_spinor(y + ro + (int64_t)n * 24, out);
    }
  }
}

template <typename LS>
inline void launch_bri_c2x2(const Geom& g, float* y, const float* x, const LS* W, const float* cl, float diag,
                            int dagger, int rhs0, int npairs, int threads, cudaStream_t s,
                            const ShiftDot<float>* sd = nullptr) {
  const StencilGrid sg = stencil_grid(blocks_for(g.V, threads), npairs);
  if (sd)
    bri_kernel_c2x2<LS, true><<<sg.grid, threads, 0, s>>>(g, y, x, W, cl, diag, rhs0, sg.gfirst,
                                                          hop_table_c2(dagger), *sd);
  else
    bri_kernel_c2x2<LS, false><<<sg.grid, threads, 0, s>>>(g, y, x, W, cl, diag, rhs0, sg.gfirst,
                                                           hop_table_c2(dagger),
                                                           ShiftDot<float>{nullptr, nullptr, nullptr});
  note_launch();
}

template <typename LS>
inline void launch_bri_c2(const Geom& g, float* y, const float* x, const LS* W, const float* cl, float diag,
                          int dagger, int rhs0, int nrhs, int threads, cudaStream_t s,
                          const ShiftDot<float>* sd = nullptr) {
  const StencilGrid sg = stencil_grid(blocks_for(g.V, threads), nrhs);
  if (sd)
    bri_kernel_c2<LS, true><<<sg.grid, threads, 0, s>>>(g, y, x, W, cl, diag, rhs0, sg.gfirst, hop_table_c2(dagger),
                                                        *sd);
  else
    bri_kernel_c2<LS, false><<<sg.grid, threads, 0, s>>>(g, y, x, W, cl, diag, rhs0, sg.gfirst, hop_table_c2(dagger),
                                                         ShiftDot<float>{nullptr, nullptr, nullptr});
  note_launch();
}

}  // namespace bri
