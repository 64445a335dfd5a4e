// Device helpers shared by the Brillouin and Wilson stencil kernels.
#pragma once

#include "internal.cuh"
#include "cplx.cuh"

#include <mutex>

namespace bri {

template <typename R> struct Spinor {
  C<R> v[4][3];
};

// AoS spinor [4][3] complex: 24 reals, 16-byte vector loads.
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

template <typename R> __device__ __forceinline__ void zero(Spinor<R>& s) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.v[a][b] = C<R>{0, 0};
}

// One 3x3 link in structure-of-arrays storage: element e of the link at site
// n sits at p[e*V] (p already offset by n).
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

// Stored link of offset j at site m.  FP64 and BF16 links are [40][9][V]
// (element e at (j*9 + e)*V + m); FP32 links pair consecutive elements in one
// 16-byte word, [40][5][V] float4 (elements 2k, 2k+1; the tenth slot is
// padding), so a link takes five 16-byte loads instead of nine 8-byte ones.
template <typename R, typename LS>
__device__ __forceinline__ void load_stored_link(C<R> w[3][3], const LS* __restrict__ W, int j, int m, int V) {
  if constexpr (sizeof(R) == 4 && sizeof(LS) == 8) {
    const float4* q = reinterpret_cast<const float4*>(W) + (int64_t)j * 5 * V + m;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float4 v = __ldg(q + (int64_t)k * V);
      const int e0 = 2 * k, e1 = 2 * k + 1;
      w[e0 / 3][e0 % 3] = C<R>{v.x, v.y};
      if (e1 < 9) w[e1 / 3][e1 % 3] = C<R>{v.z, v.w};
    }
  } else {
    load_link<R, LS>(w, W + (int64_t)j * 9 * V + m, V);
  }
}

__device__ __forceinline__ int wrap(int c, int L) { return c < 0 ? c + L : (c >= L ? c - L : c); }

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

// acc += C(n) x, C the two chiral 6x6 clover blocks.
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

// Whether FP32 stencils carry two right-hand sides per thread (shared link
// loads); BRI_PAIR_RHS=0 turns it off.
int pair_rhs_enabled();
// Stencil autotuning (BRI_AUTOTUNE=0 disables it) and its process-wide cache.
int autotune_enabled();
// Launch configuration of the FP32 stencil: pairs = 0 one right-hand side per
// thread, 1 two per thread (shared link loads), 2 the paired-FP32 kernel
// (bri_c2.cuh, one per thread); and the block size.
struct StencilConfig {
  int pairs = 1;
  int threads = 128;
  int rg = 1;  // right-hand sides on consecutive lanes (shared link loads), instead of pairs
};
bool tune_lookup(const char* key, StencilConfig* out);
void tune_store(const char* key, const StencilConfig& cf);
std::mutex& tune_mutex();

// Fused solver epilogue of a stencil launch: q = D x + sigma_s p_s at every
// site, and per block the partial sums of Re<p_s, q> in FP64 (the inner
// product of the multi-shift CG), written to part[s * blocks + site block] for
// the launch's right-hand side s.  p has the spinors' layout.
template <typename R> struct ShiftDot {
  const R* p;          // base search directions p_s (nullptr: no epilogue)
  const double* sig;   // per-system shift sigma_s
  double* part;        // [nsys][site blocks]
};

// Grid of a stencil launch: the right-hand-side groups in x (fastest, so the
// groups of one site block run together and reuse its links from L2) and the
// site blocks in y, unless there are more site blocks than a grid's y extent
// allows; gfirst tells the kernel which order was chosen.
struct StencilGrid {
  dim3 grid;
  int gfirst;
};
inline StencilGrid stencil_grid(int64_t site_blocks, int groups) {
  if (site_blocks <= 65535) return StencilGrid{dim3((unsigned)groups, (unsigned)site_blocks), 1};
  return StencilGrid{dim3((unsigned)site_blocks, (unsigned)groups), 0};
}

// Host-side launchers (one translation unit per precision).
template <typename R, typename LS>
int launch_bri_t(const Geom& g, R* y, const R* x, const LS* W, const R* cl, R diag, int nrhs, int dagger,
                 cudaStream_t s, const ShiftDot<R>* sd = nullptr, int* sd_blocks = nullptr);
template <typename R, typename LS>
int launch_wil_t(const Geom& g, R* y, const R* x, const LS* U, const R* cl, R diag, int nrhs, int dagger,
                 cudaStream_t s);

}  // namespace bri
