// Multi-shift CG on A = D^dagger D and the Kenney-Laub sign function / overlap.
//
// Sec. 3.3 and App. B: f_nn(H) b = H r(H^2) b, r(s) = c0 + sum_i w_i/(s + sigma_i),
// so with H = gamma5 D (gamma5-hermitian kernel at m0 = -rho, Eq. def_over)
//   gamma5 f(H) b = D (c0 b + sum_i w_i x_i),   x_i = (D^dagger D + sigma_i)^{-1} b.
// All x_i come out of one Krylov space (multi-shift CG, Jegerlehner form):
// the base system is the smallest shift, the others follow from the collinear
// residual recurrences
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                [alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + delta alpha_k)]
//   alpha^i_k = alpha_k zeta_{k+1}/zeta_k,  beta^i_k = beta_k (zeta_{k+1}/zeta_k)^2.
//
// Device-resident scalars: the CG coefficients of every system live in device
// memory and are advanced by one-block "scalar" kernels, so the host only
// polls a done flag every few iterations.  Global inner products are FP64
// block partials summed in a fixed order (deterministic).
//
// Mixed precision (prec = F32 or F32/BF16 links): the multi-shift solve runs
// with FP32 vectors and operator (FP64 scalars and reductions) to 1e-7 (BF16
// links: 1e-6, and only this phase uses them).  Then every shift is refined by defect
// correction: its FP64 residual r_i = b - (A + sigma_i) X_i is computed once
// with the FP64 operator, an FP32 CG correction (A + sigma_i) e_i = r_i is
// added to X_i in FP64, and r_i is updated with the FP32 operator applied to
// e_i.  The update's rounding error (~eps32 kappa_i ||r_i||, kappa_i estimated
// from the Lanczos coefficients of the first phase) is accumulated per shift;
// where it could matter the residual is recomputed in FP64 before the shift is
// declared converged.  All corrections of a round run as one batched CG with a
// per-system shift, hardest systems first, and converged systems drop out.
#include "internal.cuh"
#include "cplx.cuh"
#include "bri_kernel.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace bri {

static thread_local ScratchArena* t_arena = nullptr;
void set_current_arena(ScratchArena* a) { t_arena = a; }
ScratchArena* current_arena() { return t_arena; }

namespace {

constexpr int NS = BRI_MAX_SHIFTS;
constexpr int RED_THREADS = 256;

struct MsState {
  double rr, bnorm2, pq, alpha, alpha_prev, beta_prev, tol2;
  double lam_max;  // largest diagonal entry of the CG Lanczos matrix (estimate of lambda_max(A + sigma_base))
  double sig_base;
  double delta[NS];
  double zeta[NS], zeta_prev[NS], zeta_next[NS];
  double a_s[NS], b_s[NS];
  int active[NS];
  int nshift, done, iters, maxiter, error;
};

// Deferred shifted updates (FP32 solves): the coefficients of up to DW
// iterations, recorded by k_scalar_alpha, and applied in one pass over the
// shifted vectors by k_flush_shifts (residuals of those iterations kept in a
// ring of DW vectors).  Step m of the window is iteration first_iter + m.
constexpr int DW = 4;
struct ShiftHist {
  int n;         // recorded steps not yet applied
  int first[DW]; // the step is the solve's first iteration (p_i = b, no direction update)
  float z[DW][NS], b[DW][NS];
  double a[DW][NS];
  unsigned char act[DW][NS];
};

template <typename R> struct P2;
template <> struct P2<float> { using T = float2; };
template <> struct P2<double> { using T = double2; };

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    r = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// ----------------------------------------------------------------- vector kernels
// Vectors are flat arrays of n2 pairs (re, im) per system; system s at s*n2.

// r = b, p_i = b (all shifts), x_i = 0, partial ||b||^2
template <typename R, typename XT = typename P2<R>::T>
__global__ void k_init(int64_t n2, int nsys, int nshift, const typename P2<R>::T* __restrict__ b,
                       typename P2<R>::T* r, typename P2<R>::T* p, XT* x, double* part) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    T v = b[s * n2 + i];
    r[s * n2 + i] = v;
    for (int k = 0; k < nshift; ++k) {
      p[((int64_t)k * nsys + s) * n2 + i] = v;
      x[((int64_t)k * nsys + s) * n2 + i] = XT{0, 0};
    }
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// q += sigma_base p_0 ; partial Re <p_0, q>
template <typename R>
__global__ void k_shift_dot(int64_t n2, const MsState* __restrict__ st, const typename P2<R>::T* __restrict__ p0,
                            typename P2<R>::T* q, double* part) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  if (st[s].done) return;
  const R sb = (R)st[s].sig_base;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    T pv = p0[s * n2 + i];
    T qv = q[s * n2 + i];
    qv.x = fma(sb, pv.x, qv.x);
    qv.y = fma(sb, pv.y, qv.y);
    q[s * n2 + i] = qv;
    acc += (double)pv.x * qv.x + (double)pv.y * qv.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// One pass over the shifted vectors per iteration.  For every active shift
// i > 0 the direction update left over from the previous iteration,
// p_i = zeta_i r + beta_i p_i, is applied first (r is still the previous
// residual here), then x_i += alpha_i p_i; finally r -= alpha q and the
// partial ||r||^2.  The base direction p_0 is updated separately (k_update_p0)
// because the next matrix-vector product needs it.
// The per-shift coefficients are staged in shared memory once per block (the
// active shifts compacted to a list), so the element loop reads no scalars
// from global memory.
template <typename R, typename XT = typename P2<R>::T>
__global__ void k_update_fused(int64_t n2, int nsys, const MsState* __restrict__ st,
                               const typename P2<R>::T* __restrict__ q, typename P2<R>::T* r, typename P2<R>::T* p,
                               XT* x, double* part, int first) {
  using T = typename P2<R>::T;
  using XR = decltype(XT::x);
  const int s = blockIdx.y;
  if (st[s].done) return;
  __shared__ R sz[NS], sb[NS];
  __shared__ XR sa[NS];
  __shared__ int sk[NS], snact;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int k = 0; k < st[s].nshift; ++k)
      if (st[s].active[k]) {
        sk[m] = k;
        sz[m] = (R)st[s].zeta[k];
        sb[m] = (R)st[s].b_s[k];
        sa[m] = (XR)st[s].a_s[k];
        ++m;
      }
    snact = m;
  }
  __syncthreads();
  const int nact = snact;
  const R alpha = (R)st[s].alpha;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    T rv = r[s * n2 + i];
    for (int m = 0; m < nact; ++m) {
      const int k = sk[m];
      const int64_t o = ((int64_t)k * nsys + s) * n2 + i;
      T pv = p[o];
      if (k > 0 && !first) {
        const R z = sz[m], bt = sb[m];
        pv.x = fma(bt, pv.x, z * rv.x);
        pv.y = fma(bt, pv.y, z * rv.y);
        p[o] = pv;
      }
      const XR a = sa[m];
      XT xv = x[o];
      xv.x = fma(a, (XR)pv.x, xv.x);
      xv.y = fma(a, (XR)pv.y, xv.y);
      x[o] = xv;
    }
    const T qv = q[s * n2 + i];
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    r[s * n2 + i] = rv;
    acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// Per-iteration part of the deferred scheme (FP32 solves): r_j goes to the
// ring slot of this step, x_0 += alpha_0 p_0 (FP64), r -= alpha q and the
// partial ||r||^2.  The shifted directions and solutions wait for
// k_flush_shifts.
__global__ void k_update_base(int64_t n2, int nsys, const MsState* __restrict__ st,
                              const ShiftHist* __restrict__ hist, const float2* __restrict__ q, float2* r,
                              const float2* __restrict__ p, double2* x, float2* ring, double* part) {
  const int s = blockIdx.y;
  if (st[s].done) return;
  const float alpha = (float)st[s].alpha;
  const double a0 = st[s].a_s[0];
  const int m = hist[s].n - 1;
  float2* rs = ring + ((int64_t)m * nsys + s) * n2;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    float2 rv = r[s * n2 + i];
    rs[i] = rv;
    const float2 pv = p[s * n2 + i];
    double2 xv = x[s * n2 + i];
    xv.x = fma(a0, (double)pv.x, xv.x);
    xv.y = fma(a0, (double)pv.y, xv.y);
    x[s * n2 + i] = xv;
    const float2 qv = q[s * n2 + i];
    rv.x = fmaf(-alpha, qv.x, rv.x);
    rv.y = fmaf(-alpha, qv.y, rv.y);
    r[s * n2 + i] = rv;
    acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// The recorded steps of every shift i > 0 in one pass: for each step m (in
// order) p_i = zeta_i r_m + beta_i p_i (not on the first iteration), then
// x_i += alpha_i p_i -- the arithmetic of k_update_fused, step by step, with
// p_i and x_i read and written once per window instead of once per step.
// Called while the system may already be done (its last steps still pending).
__global__ void k_flush_shifts(int64_t n2, int nsys, ShiftHist* hist, const float2* __restrict__ ring, float2* p,
                               double2* x) {
  const int s = blockIdx.y;
  __shared__ float sz[DW][NS], sb[DW][NS];
  __shared__ double sa[DW][NS];
  __shared__ unsigned char sact[DW][NS];
  __shared__ int sk[NS], snk, sn, sfirst[DW];
  if (threadIdx.x == 0) {
    const ShiftHist& h = hist[s];
    const int nst = h.n;
    int mk = 0;
    for (int k = 1; k < NS; ++k) {
      int any = 0;
      for (int m = 0; m < nst; ++m) any |= h.act[m][k];
      if (any) sk[mk++] = k;
    }
    for (int m = 0; m < nst; ++m) {
      sfirst[m] = h.first[m];
      for (int j = 0; j < mk; ++j) {
        const int k = sk[j];
        sz[m][j] = h.z[m][k];
        sb[m][j] = h.b[m][k];
        sa[m][j] = h.a[m][k];
        sact[m][j] = h.act[m][k];
      }
    }
    snk = mk;
    sn = nst;
  }
  __syncthreads();
  const int nk = snk, nst = sn;
  if (nst > 0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
      float2 rv[DW];
#pragma unroll
      for (int m = 0; m < DW; ++m)
        if (m < nst) rv[m] = ring[((int64_t)m * nsys + s) * n2 + i];
      for (int j = 0; j < nk; ++j) {
        const int64_t o = ((int64_t)sk[j] * nsys + s) * n2 + i;
        float2 pv = p[o];
        double2 xv = x[o];
#pragma unroll
        for (int m = 0; m < DW; ++m) {
          if (m >= nst || !sact[m][j]) continue;
          if (!sfirst[m]) {
            const float z = sz[m][j], bt = sb[m][j];
            pv.x = fmaf(bt, pv.x, z * rv[m].x);
            pv.y = fmaf(bt, pv.y, z * rv[m].y);
          }
          const double a = sa[m][j];
          xv.x = fma(a, (double)pv.x, xv.x);
          xv.y = fma(a, (double)pv.y, xv.y);
        }
        p[o] = pv;
        x[o] = xv;
      }
    }
  }
}

// The window is applied: start the next one (a kernel of its own, after every
// block of k_flush_shifts has read the history).
__global__ void k_hist_reset(ShiftHist* hist, int nsys) {
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) hist[s].n = 0;
}

// p_0 = r + beta p_0 (base direction, zeta_0 = 1)
template <typename R>
__global__ void k_update_p0(int64_t n2, const MsState* __restrict__ st, const typename P2<R>::T* __restrict__ r,
                            typename P2<R>::T* p) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  if (st[s].done) return;
  const R bt = (R)st[s].b_s[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[s * n2 + i];
    T pv = p[s * n2 + i];
    pv.x = fma(bt, pv.x, rv.x);
    pv.y = fma(bt, pv.y, rv.y);
    p[s * n2 + i] = pv;
  }
}

// ----------------------------------------------------------------- scalar kernels (one block per system)
__global__ void k_scalar_init(MsState* st, const double* part, int nblk) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[s * nblk + i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) {
    MsState& S = st[s];
    S.rr = t;
    S.lam_max = 0.0;
    S.bnorm2 = t;
    S.alpha_prev = 1.0;
    S.beta_prev = 0.0;
    S.iters = 0;
    S.error = 0;
    for (int k = 0; k < S.nshift; ++k) {
      S.zeta[k] = 1.0;
      S.zeta_prev[k] = 1.0;
      S.active[k] = 1;
    }
    S.done = (t == 0.0) ? 1 : 0;
    if (t == 0.0)
      for (int k = 0; k < S.nshift; ++k) S.active[k] = 0;
  }
}

__global__ void k_scalar_alpha(MsState* st, const double* part, int nblk, ShiftHist* hist = nullptr) {
  const int s = blockIdx.x;
  if (st[s].done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[s * nblk + i];
  double pq = block_sum(acc);
  if (threadIdx.x == 0) {
    MsState& S = st[s];
    if (!(pq > 0.0) || !isfinite(pq)) {
      S.error = 1;
      S.done = 1;
      for (int k = 0; k < S.nshift; ++k) S.active[k] = 0;
      return;
    }
    const double alpha = S.rr / pq;
    S.pq = pq;
    S.alpha = alpha;
    // Lanczos diagonal T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}
    const double tkk = 1.0 / alpha + (S.iters > 0 ? S.beta_prev / S.alpha_prev : 0.0);
    S.lam_max = fmax(S.lam_max, tkk);
    for (int k = 0; k < S.nshift; ++k) {
      if (!S.active[k]) continue;  // frozen shifts keep their last coefficients
      const double den = alpha * S.beta_prev * (S.zeta_prev[k] - S.zeta[k]) +
                         S.zeta_prev[k] * S.alpha_prev * (1.0 + S.delta[k] * alpha);
      const double zn = S.zeta[k] * S.zeta_prev[k] * S.alpha_prev / den;
      S.zeta_next[k] = zn;
      S.a_s[k] = alpha * zn / S.zeta[k];
    }
    if (hist) {  // the coefficients this iteration's shifted update (i > 0) uses
      ShiftHist& h = hist[s];
      const int m = h.n++;
      h.first[m] = S.iters == 0;
      for (int k = 0; k < S.nshift; ++k) {
        h.act[m][k] = (k > 0 && S.active[k]) ? 1 : 0;
        h.z[m][k] = (float)S.zeta[k];
        h.b[m][k] = (float)S.b_s[k];
        h.a[m][k] = S.a_s[k];
      }
    }
  }
}

__global__ void k_scalar_beta(MsState* st, const double* part, int nblk) {
  const int s = blockIdx.x;
  if (st[s].done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[s * nblk + i];
  double rr = block_sum(acc);
  if (threadIdx.x == 0) {
    MsState& S = st[s];
    if (!isfinite(rr)) {
      S.error = 1;
      S.done = 1;
      for (int k = 0; k < S.nshift; ++k) S.active[k] = 0;
      return;
    }
    const double beta = rr / S.rr;
    for (int k = 0; k < S.nshift; ++k) {
      if (!S.active[k]) continue;
      const double ratio = S.zeta_next[k] / S.zeta[k];
      S.b_s[k] = beta * ratio * ratio;
      S.zeta_prev[k] = S.zeta[k];
      S.zeta[k] = S.zeta_next[k];
    }
    S.alpha_prev = S.alpha;
    S.beta_prev = beta;
    S.rr = rr;
    S.iters += 1;
    for (int k = 0; k < S.nshift; ++k)
      if (S.active[k] && S.zeta[k] * S.zeta[k] * rr <= S.tol2 * S.bnorm2) S.active[k] = 0;
    if (!S.active[0] || S.iters >= S.maxiter) {
      // p updates of the still-active (larger) shifts are skipped once the base stops
      S.done = 1;
    }
  }
}

// rhs32[j] = (float) res[slot[j]]
__global__ void k_gather_f32(int64_t n, const double* __restrict__ res, const long long* __restrict__ slot,
                             float* out) {
  const int j = blockIdx.y;
  const double* src = res + slot[j] * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[j * n + i] = (float)src[i];
}

// X[slot] += e ; res[slot] -= (A e + sigma e) ; partial ||res||^2
__global__ void k_correct(int64_t n, const long long* __restrict__ slot, const double* __restrict__ sig,
                          const float* __restrict__ e, const float* __restrict__ ae, double* X, double* res,
                          double* part) {
  const int j = blockIdx.y;
  const double sg = sig[j];
  double* xs = X + slot[j] * n;
  double* rs = res + slot[j] * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ev = (double)e[j * n + i];
    xs[i] += ev;
    const double rv = rs[i] - ((double)ae[j * n + i] + sg * ev);
    rs[i] = rv;
    acc += rv * rv;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = t;
}

__global__ void k_gather_done(const MsState* __restrict__ st, int nsys, int* out) {
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) out[s] = st[s].done;
}

// ----------------------------------------------------------------- precision / algebra helpers
template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* __restrict__ in, B* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

// res = b - q - sigma X ; partial ||res||^2 ; q is (A X)
__global__ void k_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                           const double* __restrict__ X, double sigma, double* res, double* part) {
  const int s = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = s * n + i;
    double v = b[o] - q[o] - sigma * X[o];
    if (res) res[o] = v;
    acc += v * v;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// partials of Re<a_s, b_s> (FP64)
__global__ void k_dot_re(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* part) {
  const int s = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[s * n + i] * b[s * n + i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

__global__ void k_sum_partials(const double* part, int nblk, double* out) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[s * nblk + i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) out[s] = t;
}

// acc = c0 b + sum_i w_i X_i   (FP64, X = [nshift][nsys][n])
__global__ void k_rational(int64_t n, int nsys, int nshift, double c0, const double* __restrict__ w,
                           const double* __restrict__ b, const double* __restrict__ X, double* out) {
  const int s = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = c0 * b[s * n + i];
    for (int k = 0; k < nshift; ++k) v += w[k] * X[((int64_t)k * nsys + s) * n + i];
    out[s * n + i] = v;
  }
}

// y = cb b + cz z
__global__ void k_axpby(int64_t n, double cb, const double* __restrict__ b, double cz, const double* __restrict__ z,
                        double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cb * b[i] + cz * z[i];
}

// Reduction grids: blocks per system, at most kMaxPartials partial sums in all
// (for nsys <= kMaxPartials: blocks * nsys <= kMaxPartials).
constexpr int kMaxPartials = 2048;
int grid_for(int64_t n, int nsys) {
  int64_t b = (n + RED_THREADS - 1) / RED_THREADS;
  int64_t cap = std::max<int64_t>(1, kMaxPartials / std::max(1, nsys));
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

// ----------------------------------------------------------------- batched lattices (device work list)
// Several lattices of uneven volume solved as one system table: system s
// belongs to lattice sd[s].lat, has n2 complex entries and its vectors sit at
// complex offset off (r, t, q) and offn + k n2 (shift k of p and x).  The
// stencil walks a work list of (system, 128-site block) items, so one launch
// covers every lattice and every right-hand side; items of converged systems
// return at once.  Per-system scalars are the MsState of the single-lattice
// solver.
constexpr int kMaxBatch = 32;
struct BatchLat {
  Geom g;
  const void* W;
  const void* C;
  double diag;
};
struct BatchTab {
  int nlat;
  BatchLat lat[kMaxBatch];
};
struct SysDesc {
  int lat, pad;
  int64_t n2, off, offn;
};

// NR = 2: the item's system s and s + 1 (same lattice, adjacent in the table)
// share the link loads, as in the lattice-wide kernel with two right-hand
// sides per thread; the pair is skipped only when both have converged.
template <typename R, typename LS, int NR, int MINB>
__global__ void __launch_bounds__(128, MINB)
    kb_stencil(const __grid_constant__ BatchTab T, const SysDesc* __restrict__ sd, const int2* __restrict__ items,
               const MsState* __restrict__ st, typename P2<R>::T* y, const typename P2<R>::T* x, int x_from_p,
               int nshift, R sgn, const __grid_constant__ HopTable<R> H) {
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const bool live = !st[s].done || (NR == 2 && !st[s + 1].done);
  if (!live) return;
  const SysDesc d = sd[s];
  const BatchLat& L = T.lat[d.lat];
  const int n = it.y * 128 + threadIdx.x;
  if (n >= L.g.V) return;
  const R* xin = reinterpret_cast<const R*>(x + (x_from_p ? d.offn : d.off));
  R* yout = reinterpret_cast<R*>(y + d.off);
  const int64_t xstride = 2 * (x_from_p ? (int64_t)nshift * d.n2 : d.n2), ystride = 2 * d.n2;
  bri_site<R, LS, NR>(L.g, n, yout, xin, xstride, ystride, (const LS*)L.W, (const R*)L.C, (R)L.diag, sgn, H);
}

// r = b, p_k = b, x_k = 0, partial ||b||^2
template <typename R>
__global__ void kb_init(const SysDesc* __restrict__ sd, int nshift, const typename P2<R>::T* __restrict__ b,
                        typename P2<R>::T* r, typename P2<R>::T* p, double2* x, double* part) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  const SysDesc d = sd[s];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = b[d.off + i];
    r[d.off + i] = v;
    for (int k = 0; k < nshift; ++k) {
      p[d.offn + k * d.n2 + i] = v;
      x[d.offn + k * d.n2 + i] = make_double2(0.0, 0.0);
    }
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// q += sigma_base p_0 ; partial Re <p_0, q>
template <typename R>
__global__ void kb_shift_dot(const SysDesc* __restrict__ sd, const MsState* __restrict__ st,
                             const typename P2<R>::T* __restrict__ p, typename P2<R>::T* q, double* part) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  if (st[s].done) return;
  const SysDesc d = sd[s];
  const R sb = (R)st[s].sig_base;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x) {
    const T pv = p[d.offn + i];
    T qv = q[d.off + i];
    qv.x = fma(sb, pv.x, qv.x);
    qv.y = fma(sb, pv.y, qv.y);
    q[d.off + i] = qv;
    acc += (double)pv.x * qv.x + (double)pv.y * qv.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// the fused shift pass of k_update_fused on the system table (solutions in FP64)
template <typename R>
__global__ void kb_update(const SysDesc* __restrict__ sd, const MsState* __restrict__ st,
                          const typename P2<R>::T* __restrict__ q, typename P2<R>::T* r, typename P2<R>::T* p,
                          double2* x, double* part, int first) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  if (st[s].done) return;
  __shared__ R sz[NS], sb[NS];
  __shared__ double sa[NS];
  __shared__ int sk[NS], snact;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int k = 0; k < st[s].nshift; ++k)
      if (st[s].active[k]) {
        sk[m] = k;
        sz[m] = (R)st[s].zeta[k];
        sb[m] = (R)st[s].b_s[k];
        sa[m] = st[s].a_s[k];
        ++m;
      }
    snact = m;
  }
  __syncthreads();
  const SysDesc d = sd[s];
  const int nact = snact;
  const R alpha = (R)st[s].alpha;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x) {
    T rv = r[d.off + i];
    for (int m = 0; m < nact; ++m) {
      const int k = sk[m];
      const int64_t o = d.offn + k * d.n2 + i;
      T pv = p[o];
      if (k > 0 && !first) {
        pv.x = fma(sb[m], pv.x, sz[m] * rv.x);
        pv.y = fma(sb[m], pv.y, sz[m] * rv.y);
        p[o] = pv;
      }
      double2 xv = x[o];
      xv.x = fma(sa[m], (double)pv.x, xv.x);
      xv.y = fma(sa[m], (double)pv.y, xv.y);
      x[o] = xv;
    }
    const T qv = q[d.off + i];
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    r[d.off + i] = rv;
    acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
}

// p_0 = r + beta p_0
template <typename R>
__global__ void kb_update_p0(const SysDesc* __restrict__ sd, const MsState* __restrict__ st,
                             const typename P2<R>::T* __restrict__ r, typename P2<R>::T* p) {
  using T = typename P2<R>::T;
  const int s = blockIdx.y;
  if (st[s].done) return;
  const SysDesc d = sd[s];
  const R bt = (R)st[s].b_s[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[d.off + i];
    T pv = p[d.offn + i];
    pv.x = fma(bt, pv.x, rv.x);
    pv.y = fma(bt, pv.y, rv.y);
    p[d.offn + i] = pv;
  }
}

// Loop condition of the graph's WHILE node: another iteration while any
// system is still running (k_scalar_beta marks a system done at its iteration
// cap, so the loop ends after at most maxiter passes).
__global__ void kb_while(cudaGraphConditionalHandle h, const MsState* __restrict__ st, int nsys) {
  int any = 0;
  for (int s = 0; s < nsys; ++s) any |= !st[s].done;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

// X_l[k][r][i] (one lattice's layout) = x[offn(s) + k n2 + i] of system s = s0 + r
__global__ void kb_gather_x(const SysDesc* __restrict__ sd, int s0, int nrhs, int nshift,
                            const double2* __restrict__ x, double2* X) {
  const int r = blockIdx.y, k = blockIdx.z;
  const SysDesc d = sd[s0 + r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x)
    X[((int64_t)k * nrhs + r) * d.n2 + i] = x[d.offn + k * d.n2 + i];
}

// b of one lattice (FP64, [nrhs][n2]) into the system table's vector
template <typename R>
__global__ void kb_scatter_b(const SysDesc* __restrict__ sd, int s0, const double2* __restrict__ b,
                             typename P2<R>::T* out) {
  const int r = blockIdx.y;
  const SysDesc d = sd[s0 + r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n2; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = b[(int64_t)r * d.n2 + i];
    out[d.off + i] = typename P2<R>::T{(R)v.x, (R)v.y};
  }
}

// ----------------------------------------------------------------- device memory from the stream-ordered pool
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ScratchArena* arena = nullptr;  // set when carved from a caller-provided arena
  size_t arena_mark = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (!p) return;
    if (arena) {
      // stack discipline: give the space back when this is the newest block
      if (arena->used == arena_mark + ((arena_bytes + 255) & ~size_t(255))) arena->used = arena_mark;
      arena = nullptr;
    } else {
      cudaFreeAsync(p, s);
    }
    p = nullptr;
  }
  size_t arena_bytes = 0;
  int alloc(size_t bytes, cudaStream_t st) {
    s = st;
    release();
    if (bytes == 0) bytes = 16;
    if (ScratchArena* a = current_arena()) {
      const size_t need = (bytes + 255) & ~size_t(255);
      if (a->used + need > a->cap) {
        set_error("no-allocation scratch exhausted: the problem is larger than the static scratch array");
        return BRI_ERR_INVALID;
      }
      arena = a;
      arena_mark = a->used;
      arena_bytes = bytes;
      p = a->base + a->used;
      a->used += need;
      return BRI_OK;
    }
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error(std::string("cudaMallocAsync failed: ") + cudaGetErrorString(e));
      return BRI_ERR_OOM;
    }
    note_device_alloc();
    return BRI_OK;
  }
  void reset() { release(); }
  template <typename T> T* as() const { return (T*)p; }
};

void configure_pool_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

// Operator application for the solver: out = D in (dagger 0) / D^dagger in.
template <typename R> int op_prec(int prec);
template <> int op_prec<double>(int) { return BRI_PREC_F64; }
template <> int op_prec<float>(int prec) { return prec == BRI_PREC_F32_BF16 ? BRI_PREC_F32_BF16 : BRI_PREC_F32; }


// Solve (A + sig[s][k]) x[k][s] = b[s] for nsys systems with nshift shifts each.
// sig: host [nsys][nshift], increasing within a system.  x64 (R = float only):
// the solutions are accumulated in FP64 there instead of in x (x unused).
template <typename R>
int multishift_solve(bri_ctx* c, int prec, double m0, int nsys, int nshift, const double* sig, const R* b, R* x,
                     double tol, int maxiter, int* iters_out, Counters* cnt, const double* tols,
                     double* lam_out = nullptr, const KernelOp* op = nullptr, double* x64 = nullptr) {
  using T = typename P2<R>::T;
  cudaStream_t st = c->stream;
  const int64_t n2 = c->g.V * 12;  // complex pairs per system
  const int nblk = grid_for(n2, nsys);
  const int oprec = op_prec<R>(prec);
  DevBuf br, bp, bt, bq, bst, bpart;
  int rc;
  if ((rc = br.alloc(sizeof(T) * n2 * nsys, st))) return rc;
  if ((rc = bp.alloc(sizeof(T) * n2 * nsys * nshift, st))) return rc;
  if ((rc = bt.alloc(sizeof(T) * n2 * nsys, st))) return rc;
  if ((rc = bq.alloc(sizeof(T) * n2 * nsys, st))) return rc;
  if ((rc = bst.alloc(sizeof(MsState) * nsys, st))) return rc;
  if ((rc = bpart.alloc(sizeof(double) * nblk * nsys, st))) return rc;
  T* r = br.as<T>();
  T* p = bp.as<T>();
  T* t = bt.as<T>();
  T* q_vec = bq.as<T>();
  MsState* S = bst.as<MsState>();
  double* part = bpart.as<double>();

  std::vector<MsState> hs(nsys);
  for (int s = 0; s < nsys; ++s) {
    MsState& h = hs[s];
    memset(&h, 0, sizeof(h));
    h.nshift = nshift;
    h.sig_base = sig[s * nshift];
    for (int k = 0; k < nshift; ++k) h.delta[k] = sig[s * nshift + k] - h.sig_base;
    const double ts = tols ? tols[s] : tol;
    h.tol2 = ts * ts;
    h.maxiter = maxiter;
  }
  BRI_CUDA(cudaMemcpyAsync(S, hs.data(), sizeof(MsState) * nsys, cudaMemcpyHostToDevice, st));
  // Fused D^dagger application (Brillouin kernel): q = D^dagger t + sigma_base p_0
  // and the partials of Re<p_0, q> come out of the stencil's epilogue, so
  // k_shift_dot's pass over q and p_0 is not needed.
  const bool fused = op == nullptr && c->kernel == BRI_KERNEL_BRILLOUIN;
  // Deferred shifted updates (FP32 solve with FP64 solutions): the shifted
  // directions and solutions are advanced every DW iterations from a ring of
  // the residuals of those iterations (same arithmetic, fewer passes).
  const bool defer = sizeof(R) == 4 && x64 != nullptr;
  DevBuf bring, bhist;
  if (defer) {
    if ((rc = bring.alloc(sizeof(T) * n2 * nsys * DW, st))) return rc;
    if ((rc = bhist.alloc(sizeof(ShiftHist) * nsys, st))) return rc;
    BRI_CUDA(cudaMemsetAsync(bhist.p, 0, sizeof(ShiftHist) * nsys, st));
  }
  ShiftHist* hist = defer ? bhist.as<ShiftHist>() : nullptr;
  DevBuf bsig, bpart_sd;
  std::vector<double> hsig(nsys);
  for (int s = 0; s < nsys; ++s) hsig[s] = hs[s].sig_base;
  if (fused) {
    if ((rc = bsig.alloc(sizeof(double) * nsys, st))) return rc;
    if ((rc = bpart_sd.alloc(sizeof(double) * nsys * (size_t)blocks_for(c->g.V, 64), st))) return rc;
    BRI_CUDA(cudaMemcpyAsync(bsig.p, hsig.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
  }
  dim3 vg(nblk, nsys);
  if (x64)
    k_init<R, double2><<<vg, RED_THREADS, 0, st>>>(n2, nsys, nshift, (const T*)b, r, p, (double2*)x64, part);
  else
    k_init<R><<<vg, RED_THREADS, 0, st>>>(n2, nsys, nshift, (const T*)b, r, p, (T*)x, part);
  note_launch();
  k_scalar_init<<<nsys, RED_THREADS, 0, st>>>(S, part, nblk); note_launch();
  BRI_LAUNCH_CHECK("multishift init");

  int* hdone = (int*)c->host_pinned;  // pinned scratch, >= 4 KB
  const int check_every = 8;
  int it = 0;
  // Systems [nact, nsys) have all converged: the stencil and the vector
  // kernels only run over the prefix [0, nact) (callers put the hardest
  // systems first).  Converged systems inside the prefix are skipped by the
  // vector kernels through their done flags.
  int nact = nsys;
  DevBuf bflags;
  if ((rc = bflags.alloc(sizeof(int) * nsys, st))) return rc;
  // One block of iterations over the active prefix of systems.
  auto enqueue_block = [&](int na, int it0, int count) -> int {
    dim3 vga(nblk, na);
    for (int j = 0; j < count; ++j) {
      int q;
      if (op) {  // an FP64 operator given by the caller (R = double)
        if ((q = op->apply((double2*)t, (const double2*)p, na, 0))) return q;
        if ((q = op->apply((double2*)q_vec, (const double2*)t, na, 1))) return q;
      } else if (fused) {
        if ((q = dirac_kernel(c, t, p, na, m0, 0, oprec, st))) return q;
        int nb = 0;
        if ((q = dirac_bri_shiftdot(c, q_vec, t, na, m0, oprec, st, p, bsig.as<double>(), bpart_sd.as<double>(), &nb)))
          return q;
        k_scalar_alpha<<<na, RED_THREADS, 0, st>>>(S, bpart_sd.as<double>(), nb, hist); note_launch();
      } else {
        if ((q = dirac_kernel(c, t, p, na, m0, 0, oprec, st))) return q;
        if ((q = dirac_kernel(c, q_vec, t, na, m0, 1, oprec, st))) return q;
      }
      if (!fused || op) {
        k_shift_dot<R><<<vga, RED_THREADS, 0, st>>>(n2, S, p, q_vec, part); note_launch();
        k_scalar_alpha<<<na, RED_THREADS, 0, st>>>(S, part, nblk, hist); note_launch();
      }
      if (defer)
        k_update_base<<<vga, RED_THREADS, 0, st>>>(n2, nsys, S, hist, (const float2*)q_vec, (float2*)r,
                                                   (const float2*)p, (double2*)x64, (float2*)bring.p, part);
      else if (x64)
        k_update_fused<R, double2><<<vga, RED_THREADS, 0, st>>>(n2, nsys, S, q_vec, r, p, (double2*)x64, part,
                                                                it0 + j == 0 ? 1 : 0);
      else
        k_update_fused<R><<<vga, RED_THREADS, 0, st>>>(n2, nsys, S, q_vec, r, p, (T*)x, part, it0 + j == 0 ? 1 : 0);
      note_launch();
      k_scalar_beta<<<na, RED_THREADS, 0, st>>>(S, part, nblk); note_launch();
      k_update_p0<R><<<vga, RED_THREADS, 0, st>>>(n2, S, r, p); note_launch();
      if (defer && ((j + 1) % DW == 0 || j == count - 1)) {
        k_flush_shifts<<<vga, RED_THREADS, 0, st>>>(n2, nsys, hist, (const float2*)bring.p, (float2*)p,
                                                    (double2*)x64);
        note_launch();
        k_hist_reset<<<1, 64, 0, st>>>(hist, na); note_launch();
      }
    }
    return BRI_OK;
  };
  // Blocks after the first are captured once per active-prefix size into a CUDA
  // graph and replayed (fewer launch gaps on small lattices).  Not while the
  // stencils are being profiled, and not on the legacy default stream.
  const bool graphs = graphs_enabled() && !c->prof_on && st != nullptr && op == nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_nact = -1;
  long long g_launches = 0;
  while (nact > 0 && it < maxiter) {
    const int count = std::min(check_every, maxiter - it);
    if (graphs && it > 0 && count == check_every) {
      if (g_nact != nact) {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        cudaGraph_t graph = nullptr;
        const long long l0 = bri_kernel_launches();
        BRI_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const int erc = enqueue_block(nact, it, count);
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        g_launches = bri_kernel_launches() - l0;
        if (erc) {
          if (graph) cudaGraphDestroy(graph);
          return erc;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "multishift: graph capture");
        const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ie, "multishift: graph instantiate");
        g_nact = nact;
      } else {
        note_launches(g_launches);
      }
      BRI_CUDA(cudaGraphLaunch(gexec, st));
    } else {
      if ((rc = enqueue_block(nact, it, count))) return rc;
    }
    cnt->matvecs += 2 * count;
    if (sizeof(R) == 8) cnt->matvecs64 += 2 * count;
    it += count;
    BRI_LAUNCH_CHECK("multishift iteration");
    // poll the done flags
    k_gather_done<<<1, 256, 0, st>>>(S, nsys, bflags.as<int>()); note_launch();
    BRI_CUDA(cudaMemcpyAsync(hdone, bflags.as<int>(), sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    BRI_CUDA(cudaStreamSynchronize(st));
    while (nact > 0 && hdone[nact - 1]) --nact;
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  BRI_CUDA(cudaMemcpyAsync(hs.data(), S, sizeof(MsState) * nsys, cudaMemcpyDeviceToHost, st));
  BRI_CUDA(cudaStreamSynchronize(st));
  int maxit = 0, err = 0, notconv = 0;
  for (int s = 0; s < nsys; ++s) {
    maxit = std::max(maxit, hs[s].iters);
    err |= hs[s].error;
    if (hs[s].active[0] && !hs[s].error) notconv = 1;
  }
  *iters_out = maxit;
  if (lam_out) {
    double lm = 0.0;
    for (int s = 0; s < nsys; ++s) lm = std::max(lm, hs[s].lam_max - hs[s].sig_base);
    *lam_out = lm;
  }
  if (err) {
    set_error("multi-shift CG: non-finite or non-positive curvature in a reduction");
    return BRI_ERR_NONFINITE;
  }
  return notconv ? BRI_NOT_CONVERGED : BRI_OK;
}

// ||b - (A + sigma) X||^2 per system for one shift (FP64 operator); res may be null.
int residual64(bri_ctx* c, double m0, int nsys, const double* b, const double* X, double sigma, double* res,
               double* tmp1, double* tmp2, double* part, double* dsum, double* hsum, Counters* cnt,
               const KernelOp* op = nullptr) {
  cudaStream_t st = c->stream;
  const int64_t n = c->g.V * 24;
  int rc;
  if (op) {
    if ((rc = op->apply((double2*)tmp1, (const double2*)X, nsys, 0))) return rc;
    if ((rc = op->apply((double2*)tmp2, (const double2*)tmp1, nsys, 1))) return rc;
  } else {
    if ((rc = dirac_kernel(c, tmp1, X, nsys, m0, 0, BRI_PREC_F64, st))) return rc;
    if ((rc = dirac_kernel(c, tmp2, tmp1, nsys, m0, 1, BRI_PREC_F64, st))) return rc;
  }
  cnt->matvecs += 2;
  cnt->matvecs64 += 2;
  const int nblk = grid_for(n / 2, nsys);
  k_residual<<<dim3(nblk, nsys), RED_THREADS, 0, st>>>(n, b, tmp2, X, sigma, res, part); note_launch();
  k_sum_partials<<<nsys, RED_THREADS, 0, st>>>(part, nblk, dsum); note_launch();
  BRI_LAUNCH_CHECK("residual64");
  BRI_CUDA(cudaMemcpyAsync(hsum, dsum, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  BRI_CUDA(cudaStreamSynchronize(st));
  return BRI_OK;
}

// The same residual with A = D^dagger D applied in double-word FP32 arithmetic
// (Brillouin kernel, bri_dw.cu): FP64-class accuracy on the FP32 pipe.
int residual_dw(bri_ctx* c, double m0, int nsys, const double* b, const double* X, double sigma, double* res,
                double* tmp1, double* tmp2, double* part, double* dsum, double* hsum, Counters* cnt) {
  cudaStream_t st = c->stream;
  const int64_t n = c->g.V * 24;
  int rc = normal_op_dw(c, tmp2, X, nsys, m0, tmp1, tmp2, st);
  if (rc) return rc;
  cnt->matvecs += 2;
  const int nblk = grid_for(n / 2, nsys);
  k_residual<<<dim3(nblk, nsys), RED_THREADS, 0, st>>>(n, b, tmp2, X, sigma, res, part); note_launch();
  k_sum_partials<<<nsys, RED_THREADS, 0, st>>>(part, nblk, dsum); note_launch();
  BRI_LAUNCH_CHECK("residual_dw");
  BRI_CUDA(cudaMemcpyAsync(hsum, dsum, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  BRI_CUDA(cudaStreamSynchronize(st));
  return BRI_OK;
}

// ||X_s||^2 per system (FP64)
int norms64(bri_ctx* c, int nsys, const double* X, double* part, double* dsum, double* hsum) {
  cudaStream_t st = c->stream;
  const int64_t n = c->g.V * 24;
  const int nblk = grid_for(n / 2, nsys);
  k_residual<<<dim3(nblk, nsys), RED_THREADS, 0, st>>>(n, X, X, X, -1.0, nullptr, part); note_launch();
  k_sum_partials<<<nsys, RED_THREADS, 0, st>>>(part, nblk, dsum); note_launch();
  BRI_LAUNCH_CHECK("norms64");
  BRI_CUDA(cudaMemcpyAsync(hsum, dsum, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  BRI_CUDA(cudaStreamSynchronize(st));
  return BRI_OK;
}

// Bound on the error of the double-word normal operator relative to the norm
// of its argument, ||A_dw x - A x|| <= kDwRelErr ||x||.  The inputs are split
// to ~2^-49 of each component, the products and sums are error-free up to the
// second word (~2^-48 of the terms, which cancel in D x), and the intermediate
// D x is stored as a double-word pair.  Measured against the FP64 operator on
// the 24^3 x 48 stout-smeared field: 2.5e-14 ||x|| for Gaussian x, 3.7e-14
// ||x|| for a smooth x (the low-mode shape of the small shifts' solutions);
// the bound takes 1e-13.
constexpr double kDwRelErr = 1e-13;

// The double-word residual serves a shift when its error bound stays below 5 %
// of the target for every right-hand side: kDwRelErr ||X_s|| <= 0.05 tol ||b_s||.
bool dw_residual_ok(const bri_ctx* c, const double* xn2, const double* bn2, int nsys, double tol) {
  if (c->kernel != BRI_KERNEL_BRILLOUIN) return false;
  for (int s = 0; s < nsys; ++s)
    if (kDwRelErr * std::sqrt(xn2[s]) > 0.05 * tol * std::sqrt(bn2[s])) return false;
  return true;
}

// Phases 2 and 3 of the mixed scheme for X = the FP32 multi-shift solution
// (converted to FP64): one FP64 residual per (shift, rhs), then batched FP32
// CG corrections of every shift still above tol, with the FP32-tracked
// residuals checked in FP64 where their rounding error could matter.
int refine_mixed(bri_ctx* c, const double* b, int nrhs, int n, const double* sig, double m0, double tol, int maxiter,
                 double* X, double lam_est, SolveInfo& info, const std::function<void(int)>& lap) {
  cudaStream_t st = c->stream;
  const int64_t nreal = c->g.V * 24;
  int rc = BRI_OK;
  int solve_rc = BRI_OK;
  Counters& cnt = info.cnt;
  int& refinements = info.refinements;
  // phase 2: one FP64 residual per (shift, rhs), r_i = b - (A + sigma_i) X_i
  DevBuf btmp1, btmp2, bpart, bdsum, bres;
  if ((rc = btmp1.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
  if ((rc = btmp2.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
  // The partials buffer serves three grids: the nrhs-wide residuals below,
  // the correction update (up to 32 systems) and the single-system FP64
  // verification residuals; grid_for caps every one of them at kMaxPartials.
  const int nblk_r = grid_for(nreal / 2, nrhs);
  if ((rc = bpart.alloc(sizeof(double) * std::max<int64_t>((int64_t)nblk_r * nrhs, kMaxPartials), st))) return rc;
  if ((rc = bdsum.alloc(sizeof(double) * std::max(nrhs, 32), st))) return rc;
  if ((rc = bres.alloc(sizeof(double) * nreal * nrhs * n, st))) return rc;
  std::vector<double> bn2(nrhs), rn2((size_t)n * nrhs), tmp(std::max(nrhs, 32));
  std::vector<double> err_acc((size_t)n * nrhs, 0.0);  // accumulated FP32 tracking error bound per slot
  k_residual<<<dim3(nblk_r, nrhs), RED_THREADS, 0, st>>>(nreal, b, b, b, -1.0, nullptr, bpart.as<double>());
  note_launch();
  k_sum_partials<<<nrhs, RED_THREADS, 0, st>>>(bpart.as<double>(), nblk_r, bdsum.as<double>()); note_launch();
  BRI_CUDA(cudaMemcpyAsync(bn2.data(), bdsum.as<double>(), sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  BRI_CUDA(cudaStreamSynchronize(st));
  // Each shift's residual in double-word arithmetic where its error bound
  // allows (||X_k|| small enough against tol ||b||), else in FP64.
  std::vector<double> xn2((size_t)n * nrhs);
  std::vector<char> dw_slot((size_t)n * nrhs, 0);
  for (int k = 0; k < n; ++k) {
    const double* Xk = X + (int64_t)k * nrhs * nreal;
    if ((rc = norms64(c, nrhs, Xk, bpart.as<double>(), bdsum.as<double>(), tmp.data()))) return rc;
    for (int s = 0; s < nrhs; ++s) xn2[(size_t)k * nrhs + s] = tmp[s];
    const bool dw = dw_residual_ok(c, tmp.data(), bn2.data(), nrhs, tol);
    for (int s = 0; s < nrhs; ++s) dw_slot[(size_t)k * nrhs + s] = dw;
    if (dw)
      rc = residual_dw(c, m0, nrhs, b, Xk, sig[k], bres.as<double>() + (int64_t)k * nrhs * nreal, btmp1.as<double>(),
                       btmp2.as<double>(), bpart.as<double>(), bdsum.as<double>(), tmp.data(), &cnt);
    else
      rc = residual64(c, m0, nrhs, b, Xk, sig[k], bres.as<double>() + (int64_t)k * nrhs * nreal, btmp1.as<double>(),
                      btmp2.as<double>(), bpart.as<double>(), bdsum.as<double>(), tmp.data(), &cnt);
    if (rc) return rc;
    for (int s = 0; s < nrhs; ++s) rn2[(size_t)k * nrhs + s] = tmp[s];
  }
  const bool rlog = getenv("BRI_REFINE_LOG") != nullptr;
  if (rlog)
    for (int k = 0; k < n; ++k) {
      double worst = 0.0, xmax = 0.0;
      for (int s = 0; s < nrhs; ++s) {
        worst = std::max(worst, std::sqrt(rn2[(size_t)k * nrhs + s] / std::max(bn2[s], 1e-300)));
        xmax = std::max(xmax, std::sqrt(xn2[(size_t)k * nrhs + s] / std::max(bn2[s], 1e-300)));
      }
      // alignment of this shift's residual with the base shift's (per rhs, worst)
      const int nblk_c = grid_for(nreal / 2, nrhs);
      k_dot_re<<<dim3(nblk_c, nrhs), RED_THREADS, 0, st>>>(nreal, bres.as<double>(),
                                                           bres.as<double>() + (int64_t)k * nrhs * nreal,
                                                           bpart.as<double>());
      k_sum_partials<<<nrhs, RED_THREADS, 0, st>>>(bpart.as<double>(), nblk_c, bdsum.as<double>());
      cudaMemcpyAsync(tmp.data(), bdsum.as<double>(), sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      double cmin = 1.0;
      for (int s = 0; s < nrhs; ++s)
        cmin = std::min(cmin, tmp[s] / std::sqrt(std::max(rn2[s] * rn2[(size_t)k * nrhs + s], 1e-300)));
      fprintf(stderr,
              "bri refine: shift %d sigma %.4e  relres after phase 1 %.3e  |X|/|b| %.3e  cos(r_k, r_0) %.4f  (%s "
              "residual)\n",
              k, sig[k], worst, xmax, cmin, dw_slot[(size_t)k * nrhs] ? "double-word" : "FP64");
    }
  btmp1.reset();
  btmp2.reset();
  lap(1);
  // phase 3: FP32 defect correction of every shift still above tol; the
  // residual is then updated with the FP32 operator applied to the small
  // correction (its rounding error is ~1e-7 of the old residual).
  const int max_rounds = 6;
  for (int round = 0; round < max_rounds; ++round) {
    std::vector<int> todo;  // slot = k * nrhs + s, hardest (smallest shift) first
    for (int k = 0; k < n; ++k)
      for (int sidx = 0; sidx < nrhs; ++sidx) {
        const size_t slot = (size_t)k * nrhs + sidx;
        if (std::sqrt(rn2[slot] / std::max(bn2[sidx], 1e-300)) > tol) todo.push_back((int)slot);
      }
    if (todo.empty()) break;
    if (round == max_rounds - 1) {
      solve_rc = BRI_NOT_CONVERGED;
      break;
    }
    refinements++;
    const int chunk = 32;
    for (size_t c0i = 0; c0i < todo.size(); c0i += chunk) {
      const int m = (int)std::min<size_t>(chunk, todo.size() - c0i);
      std::vector<double> msig(m), mtol(m);
      std::vector<long long> slots(m);
      for (int j = 0; j < m; ++j) {
        const int slot = todo[c0i + j], k = slot / nrhs, sidx = slot % nrhs;
        msig[j] = sig[k];
        slots[j] = slot;
        const double ratio = tol * std::sqrt(bn2[sidx] / std::max(rn2[slot], 1e-300));
        mtol[j] = std::min(0.5, std::max(1e-6, 0.3 * ratio));
      }
      DevBuf brhs, bsol, bt1, bt2, bslot, bsig;
      if ((rc = brhs.alloc(sizeof(float) * nreal * m, st))) return rc;
      if ((rc = bsol.alloc(sizeof(float) * nreal * m, st))) return rc;
      if ((rc = bslot.alloc(sizeof(long long) * m, st))) return rc;
      if ((rc = bsig.alloc(sizeof(double) * m, st))) return rc;
      BRI_CUDA(cudaMemcpyAsync(bslot.as<long long>(), slots.data(), sizeof(long long) * m,
                               cudaMemcpyHostToDevice, st));
      BRI_CUDA(cudaMemcpyAsync(bsig.as<double>(), msig.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
      k_gather_f32<<<dim3(512, m), 256, 0, st>>>(nreal, bres.as<double>(), bslot.as<long long>(),
                                                 brhs.as<float>()); note_launch();
      int itc = 0;
      // Corrections always use FP32 links: with BF16 links the operator error
      // (~4e-3 relative) times the condition number of the small shifts
      // exceeds one, so a BF16 correction would not reduce the residual.
      auto tc0 = std::chrono::steady_clock::now();
      rc = multishift_solve<float>(c, BRI_PREC_F32, m0, m, 1, msig.data(), brhs.as<float>(), bsol.as<float>(),
                                   1e-5, maxiter, &itc, &cnt, mtol.data());
      if (rc < 0) return rc;
      if (rlog) {
        cudaStreamSynchronize(st);
        fprintf(stderr, "bri refine: round %d chunk of %d systems (slots %lld..%lld, tol %.2e..%.2e): %d iterations, %.3f s\n",
                round, m, slots[0], slots[m - 1], *std::min_element(mtol.begin(), mtol.end()),
                *std::max_element(mtol.begin(), mtol.end()), itc,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - tc0).count());
      }
      // X += e (FP64); r -= (A + sigma) e with the FP32 operator
      if ((rc = bt1.alloc(sizeof(float) * nreal * m, st))) return rc;
      if ((rc = bt2.alloc(sizeof(float) * nreal * m, st))) return rc;
      // (FP32 links even when the solve used BF16 ones: the update must be
      // accurate to ~1e-7 of the old residual)
      if ((rc = dirac_kernel(c, bt1.as<float>(), bsol.as<float>(), m, m0, 0, BRI_PREC_F32, st))) return rc;
      if ((rc = dirac_kernel(c, bt2.as<float>(), bt1.as<float>(), m, m0, 1, BRI_PREC_F32, st))) return rc;
      cnt.matvecs += 2;
      const int nblk_u = grid_for(nreal / 2, m);
      k_correct<<<dim3(nblk_u, m), RED_THREADS, 0, st>>>(nreal, bslot.as<long long>(), bsig.as<double>(),
                                                        bsol.as<float>(), bt2.as<float>(), X, bres.as<double>(),
                                                        bpart.as<double>()); note_launch();
      k_sum_partials<<<m, RED_THREADS, 0, st>>>(bpart.as<double>(), nblk_u, bdsum.as<double>()); note_launch();
      BRI_LAUNCH_CHECK("refinement update");
      BRI_CUDA(cudaMemcpyAsync(tmp.data(), bdsum.as<double>(), sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      BRI_CUDA(cudaStreamSynchronize(st));
      // The FP32-tracked residual is trusted only where its rounding error,
      // ~eps32 kappa_i ||r_old|| with kappa_i = (lambda_max + sigma_i)/sigma_i,
      // is well below tol; otherwise the residual is recomputed in FP64.
      std::vector<int> verify;
      for (int j = 0; j < m; ++j) {
        const int slot = (int)slots[j], k = slot / nrhs, sidx = slot % nrhs;
        const double kappa = (lam_est + sig[k]) / sig[k];
        err_acc[slot] += 2e-7 * kappa * std::sqrt(rn2[slot]);
        const double goal = tol * std::sqrt(bn2[sidx]);
        rn2[slot] = tmp[j];
        if (err_acc[slot] > 0.25 * goal && std::sqrt(rn2[slot]) <= goal) verify.push_back(slot);
      }
      if (rlog) fprintf(stderr, "bri refine: round %d: %zu verification residuals\n", round, verify.size());
      if (!verify.empty()) {
        DevBuf v1, v2;
        if ((rc = v1.alloc(sizeof(double) * nreal, st))) return rc;
        if ((rc = v2.alloc(sizeof(double) * nreal, st))) return rc;
        for (int slot : verify) {
          const int k = slot / nrhs, sidx = slot % nrhs;
          // the solution has changed by a correction of ~1e-7 of its norm, so
          // the phase-2 norm still decides the residual's arithmetic
          if (dw_slot[slot])
            rc = residual_dw(c, m0, 1, b + (int64_t)sidx * nreal, X + (int64_t)slot * nreal, sig[k],
                             bres.as<double>() + (int64_t)slot * nreal, v1.as<double>(), v2.as<double>(),
                             bpart.as<double>(), bdsum.as<double>(), tmp.data(), &cnt);
          else
            rc = residual64(c, m0, 1, b + (int64_t)sidx * nreal, X + (int64_t)slot * nreal, sig[k],
                            bres.as<double>() + (int64_t)slot * nreal, v1.as<double>(), v2.as<double>(),
                            bpart.as<double>(), bdsum.as<double>(), tmp.data(), &cnt);
          if (rc) return rc;
          rn2[slot] = tmp[0];
          err_acc[slot] = 0.0;
        }
      }
    }
  }
  return solve_rc;
}

// Phase 1 on the system table: multi-shift CG of every system of every
// lattice at once.  The first iteration is launched directly; the rest run
// inside one CUDA graph whose WHILE node repeats the iteration body until
// every system is done (the condition is set on the device by kb_while), so
// the host neither polls nor relaunches.  x = [system][shift][n2].
template <typename R, typename LS>
int batch_multishift(cudaStream_t st, const BatchTab& tab, const std::vector<SysDesc>& sdh, int nshift,
                     const double* sig, const typename P2<R>::T* b, double2* x, double tol, int maxiter,
                     int* iters_out, Counters* cnt, double* lam_out) {
  using T = typename P2<R>::T;
  const int S = (int)sdh.size();
  int64_t tot = 0, maxn2 = 0;
  // work items: (first system of a same-lattice pair, block) and (single system, block)
  std::vector<int2> items2, items1;
  for (int s = 0; s < S; ++s) {
    tot += sdh[s].n2;
    maxn2 = std::max(maxn2, sdh[s].n2);
  }
  for (int s = 0; s < S;) {
    const int64_t nb = (tab.lat[sdh[s].lat].g.V + 127) / 128;
    const bool pair = s + 1 < S && sdh[s + 1].lat == sdh[s].lat;
    for (int64_t k = 0; k < nb; ++k) (pair ? items2 : items1).push_back(make_int2(s, (int)k));
    s += pair ? 2 : 1;
  }
  const int n2items = (int)items2.size(), n1items = (int)items1.size();
  const int nitems = n2items + n1items;
  const int nblk = grid_for(maxn2, S);
  DevBuf bsd, bit, br, bt, bq, bp, bst, bpart;
  int rc;
  if ((rc = bsd.alloc(sizeof(SysDesc) * S, st))) return rc;
  if ((rc = bit.alloc(sizeof(int2) * nitems, st))) return rc;
  if ((rc = br.alloc(sizeof(T) * tot, st))) return rc;
  if ((rc = bt.alloc(sizeof(T) * tot, st))) return rc;
  if ((rc = bq.alloc(sizeof(T) * tot, st))) return rc;
  if ((rc = bp.alloc(sizeof(T) * tot * nshift, st))) return rc;
  if ((rc = bst.alloc(sizeof(MsState) * S, st))) return rc;
  if ((rc = bpart.alloc(sizeof(double) * std::max<int64_t>((int64_t)nblk * S, kMaxPartials), st))) return rc;
  const SysDesc* sd = bsd.as<SysDesc>();
  MsState* S_ = bst.as<MsState>();
  double* part = bpart.as<double>();
  T *r = br.as<T>(), *t = bt.as<T>(), *q = bq.as<T>(), *p = bp.as<T>();
  std::vector<MsState> hs(S);
  for (int s = 0; s < S; ++s) {
    MsState& h = hs[s];
    memset(&h, 0, sizeof(h));
    h.nshift = nshift;
    h.sig_base = sig[0];
    for (int k = 0; k < nshift; ++k) h.delta[k] = sig[k] - sig[0];
    h.tol2 = tol * tol;
    h.maxiter = maxiter;
  }
  BRI_CUDA(cudaMemcpyAsync(bsd.p, sdh.data(), sizeof(SysDesc) * S, cudaMemcpyHostToDevice, st));
  if (n2items)
    BRI_CUDA(cudaMemcpyAsync(bit.p, items2.data(), sizeof(int2) * n2items, cudaMemcpyHostToDevice, st));
  if (n1items)
    BRI_CUDA(cudaMemcpyAsync(bit.as<int2>() + n2items, items1.data(), sizeof(int2) * n1items, cudaMemcpyHostToDevice,
                             st));
  BRI_CUDA(cudaMemcpyAsync(S_, hs.data(), sizeof(MsState) * S, cudaMemcpyHostToDevice, st));
  // the host copies above read pageable vectors: complete them before they go out of scope
  BRI_CUDA(cudaStreamSynchronize(st));
  const dim3 vg(nblk, S);
  constexpr int MINB1 = sizeof(R) == 8 ? 2 : 4, MINB2 = sizeof(R) == 8 ? 2 : 3;
  const HopTable<R>& H = hop_table<R>();
  const int2* it2 = bit.as<int2>();
  const int2* it1 = bit.as<int2>() + n2items;
  auto stencil = [&](typename P2<R>::T* out, const typename P2<R>::T* in, int from_p, R sgn) {
    if (n2items)
      kb_stencil<R, LS, 2, MINB2><<<n2items, 128, 0, st>>>(tab, sd, it2, S_, out, in, from_p, nshift, sgn, H);
    if (n1items)
      kb_stencil<R, LS, 1, MINB1><<<n1items, 128, 0, st>>>(tab, sd, it1, S_, out, in, from_p, nshift, sgn, H);
  };
  const int nst = (n2items ? 1 : 0) + (n1items ? 1 : 0);  // stencil launches per application
  kb_init<R><<<vg, RED_THREADS, 0, st>>>(sd, nshift, b, r, p, x, part); note_launch();
  k_scalar_init<<<S, RED_THREADS, 0, st>>>(S_, part, nblk); note_launch();
  auto iteration = [&](int first) {
    stencil(t, p, 1, (R)1);
    stencil(q, t, 0, (R)-1);
    kb_shift_dot<R><<<vg, RED_THREADS, 0, st>>>(sd, S_, p, q, part);
    k_scalar_alpha<<<S, RED_THREADS, 0, st>>>(S_, part, nblk);
    kb_update<R><<<vg, RED_THREADS, 0, st>>>(sd, S_, q, r, p, x, part, first);
    k_scalar_beta<<<S, RED_THREADS, 0, st>>>(S_, part, nblk);
    kb_update_p0<R><<<vg, RED_THREADS, 0, st>>>(sd, S_, r, p);
  };
  iteration(1);
  note_launches(5 + 2 * nst);
  BRI_LAUNCH_CHECK("batched multi-shift: first iteration");
  // graph: WHILE (any system running) { iteration }
  cudaGraph_t graph = nullptr;
  BRI_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphExec_t gexec = nullptr;
  auto fail = [&](cudaError_t e, const char* where) {
    if (gexec) cudaGraphExecDestroy(gexec);
    cudaGraphDestroy(graph);
    return cuda_fail(e, where);
  };
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: conditional handle");
  // (the parameter union has no default constructor: zeroed storage instead)
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: conditional node");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: capture");
  iteration(0);
  kb_while<<<1, 1, 0, st>>>(handle, S_, S);
  e = cudaStreamEndCapture(st, &body);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: end capture");
  e = cudaGraphInstantiate(&gexec, graph, 0);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: instantiate");
  e = cudaGraphLaunch(gexec, st);
  if (e != cudaSuccess) return fail(e, "batched multi-shift: graph launch");
  e = cudaMemcpyAsync(hs.data(), S_, sizeof(MsState) * S, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(gexec);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "batched multi-shift: graph run");
  int maxit = 0, err = 0, notconv = 0;
  double lm = 0.0;
  for (int s = 0; s < S; ++s) {
    maxit = std::max(maxit, hs[s].iters);
    err |= hs[s].error;
    if (hs[s].active[0] && !hs[s].error) notconv = 1;
    lm = std::max(lm, hs[s].lam_max - hs[s].sig_base);
  }
  note_launches((long long)(6 + 2 * nst) * std::max(0, maxit - 1));
  *iters_out = maxit;
  cnt->matvecs += 2 * maxit;
  if (sizeof(R) == 8) cnt->matvecs64 += 2 * maxit;
  if (lam_out) *lam_out = lm;
  if (err) {
    set_error("batched multi-shift CG: non-finite or non-positive curvature in a reduction");
    return BRI_ERR_NONFINITE;
  }
  return notconv ? BRI_NOT_CONVERGED : BRI_OK;
}

}  // namespace

// Solve (A + sigma_k) X_k = b_s for every shift k < n and system s < nsys,
// X = [n][nsys][V*24] FP64; FP64 multi-shift CG or the mixed scheme above.

int solve_shifts(bri_ctx* c, const double* b, int nrhs, int n, const double* sig, double m0, double tol,
                 int prec, int maxiter, double* X, SolveInfo& info, const KernelOp* op) {
  cudaStream_t st = c->stream;
  const int64_t nreal = c->g.V * 24;
  int rc = BRI_OK;
  Counters& cnt = info.cnt;
  int& iters = info.iters;
  int& refinements = info.refinements;
  std::vector<double> sig_all((size_t)nrhs * n);
  for (int s = 0; s < nrhs; ++s)
    for (int k = 0; k < n; ++k) sig_all[(size_t)s * n + k] = sig[k];

  auto tnow = [&]() {
    cudaStreamSynchronize(st);
    return std::chrono::steady_clock::now();
  };
  auto tmark = tnow();
  auto lap = [&](int ph) {
    auto t1 = tnow();
    info.tph[ph] += std::chrono::duration<double>(t1 - tmark).count();
    tmark = t1;
  };
  int solve_rc = BRI_OK;
  if (op && prec != BRI_PREC_F64) {
    set_error("multi-shift solve: an operator given by the caller needs FP64");
    return BRI_ERR_INVALID;
  }
  if (prec == BRI_PREC_F64) {
    solve_rc = multishift_solve<double>(c, prec, m0, nrhs, n, sig_all.data(), b, X, tol, maxiter, &iters, &cnt,
                                        nullptr, nullptr, op);
    if (solve_rc < 0) return solve_rc;
    lap(0);
  } else if (prec == BRI_PREC_F32 || prec == BRI_PREC_F32_BF16) {
    // phase 1: FP32 multi-shift (FP64 scalars and reductions).  The shifted
    // solutions accumulate in FP64, straight into X: rounded to FP32 they would
    // carry an error that, times the condition number of the small shifts,
    // dominates their true residual (2e-5 of ||b|| for the smallest shift of
    // the 24^3 x 48 workload, against 8e-7 with FP64 accumulation).
    DevBuf bb32;
    if ((rc = bb32.alloc(sizeof(float) * nreal * nrhs, st))) return rc;
    k_convert<double, float><<<1024, 256, 0, st>>>(nreal * nrhs, b, bb32.as<float>()); note_launch();
    // The FP32 solve is run to 1e-7 (FP32 links) where the gap between its
    // recursive and true residuals (the FP32 operator's rounding, 3e-8 to
    // 8e-7 of ||b|| from the largest to the smallest shift) stops further
    // progress from helping the corrections; with BF16 links to 1e-6.
    const double tol1 = std::max(tol, prec == BRI_PREC_F32 ? 1e-7 : 1e-6);
    int it1 = 0;
    double lam_est = 0.0;
    rc = multishift_solve<float>(c, prec, m0, nrhs, n, sig_all.data(), bb32.as<float>(), nullptr, tol1, maxiter,
                                 &it1, &cnt, nullptr, &lam_est, nullptr, X);
    lam_est = 1.1 * lam_est + 1e-3;
    if (rc < 0) return rc;
    iters = it1;
    BRI_LAUNCH_CHECK("phase 1");
    bb32.reset();
    lap(0);
    solve_rc = refine_mixed(c, b, nrhs, n, sig, m0, tol, maxiter, X, lam_est, info, lap);
    if (solve_rc < 0) return solve_rc;
    lap(2);
  } else {
    set_error("sign_apply_multishift: unknown precision");
    return BRI_ERR_INVALID;
  }

  return solve_rc;
}

// y = b_coeff b + out_scale D (c0 b + sum_i w_i X_i) for X = [n][nrhs][V*24] FP64
int finish_sign(bri_ctx* c, double* y, const double* b, int nrhs, int n, double c0, const double* w, const double* X,
                double m0, double out_scale, double b_coeff, Counters& cnt, const KernelOp* op) {
  cudaStream_t st = c->stream;
  const int64_t nreal = c->g.V * 24;
  int rc = BRI_OK;
  // y = b_coeff b + out_scale D (c0 b + sum_i w_i X_i)
  DevBuf bacc, bz, bw;
  if ((rc = bacc.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
  if ((rc = bz.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
  if ((rc = bw.alloc(sizeof(double) * NS, st))) return rc;
  BRI_CUDA(cudaMemcpyAsync(bw.as<double>(), w, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  k_rational<<<dim3(grid_for(nreal, nrhs), nrhs), RED_THREADS, 0, st>>>(nreal, nrhs, n, c0, bw.as<double>(), b, X,
                                                                       bacc.as<double>()); note_launch();
  BRI_LAUNCH_CHECK("k_rational");
  if (op) {
    if ((rc = op->apply(bz.as<double2>(), bacc.as<double2>(), nrhs, 0))) return rc;
  } else if ((rc = dirac_kernel(c, bz.as<double>(), bacc.as<double>(), nrhs, m0, 0, BRI_PREC_F64, st))) {
    return rc;
  }
  cnt.matvecs += 1;
  cnt.matvecs64 += 1;
  k_axpby<<<2048, 256, 0, st>>>(nreal * nrhs, b_coeff, b, out_scale, bz.as<double>(), y); note_launch();
  BRI_LAUNCH_CHECK("k_axpby");
  return BRI_OK;
}

// Runs the enclosed solver work on the context's own non-blocking stream
// (fenced after the caller's stream on entry and before it on exit), so that
// iterations can be graph-captured and contexts driven from different host
// threads overlap on the GPU.  Nested scopes and allocation-free calls keep
// the current stream.
struct StreamScope {
  bri_ctx* c;
  cudaStream_t user;
  bool active = false;
  explicit StreamScope(bri_ctx* cx) : c(cx), user(cx->stream) {
    if (!graphs_enabled() || (c->own_stream && c->stream == c->own_stream)) return;
    if (!c->own_stream) {
      if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
    }
    cudaEventRecord(c->ev_in, user);
    cudaStreamWaitEvent(c->own_stream, c->ev_in, 0);
    c->stream = c->own_stream;
    active = true;
  }
  ~StreamScope() {
    if (!active) return;
    cudaEventRecord(c->ev_out, c->own_stream);
    cudaStreamWaitEvent(user, c->ev_out, 0);
    c->stream = user;
  }
};

int sign_apply(bri_ctx* c, double2* y, const double2* x, int nrhs, int n, int kind, double rho, double scale,
               double tol, int prec, double out_scale, double b_coeff, bri_stats* stats, const KernelOp* op) {
  StreamScope scope(c);
  auto t0 = std::chrono::steady_clock::now();
  configure_pool_once();
  cudaStream_t st = c->stream;
  const int64_t nreal = c->g.V * 24;
  const double m0 = -rho;
  double c0, w[NS], sig[NS];
  int rc = kl_host(n, kind, scale, &c0, w, sig);
  if (rc) return rc;
  const int maxiter = (stats && stats->maxiter > 0) ? stats->maxiter : 20000;
  const double* b = (const double*)x;

  double tph[4] = {0, 0, 0, 0};
  DevBuf bX;
  if ((rc = bX.alloc(sizeof(double) * nreal * nrhs * n, st))) return rc;
  double* X = bX.as<double>();
  SolveInfo info;
  int solve_rc = solve_shifts(c, b, nrhs, n, sig, m0, tol, prec, maxiter, X, info, op);
  if (solve_rc < 0) return solve_rc;
  Counters& cnt = info.cnt;
  const int iters = info.iters, refinements = info.refinements;
  for (int ph = 0; ph < 3; ++ph) tph[ph] = info.tph[ph];
  auto tmark = std::chrono::steady_clock::now();
  // optional FP64 true residuals for the statistics
  if (stats && stats->want_true_residual) {
    DevBuf btmp1, btmp2, bpart, bdsum;
    const int nblk_r = grid_for(nreal / 2, nrhs);
    if ((rc = btmp1.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
    if ((rc = btmp2.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
    if ((rc = bpart.alloc(sizeof(double) * nblk_r * nrhs, st))) return rc;
    if ((rc = bdsum.alloc(sizeof(double) * nrhs, st))) return rc;
    std::vector<double> bn2(nrhs), rn2(nrhs);
    k_residual<<<dim3(nblk_r, nrhs), RED_THREADS, 0, st>>>(nreal, b, b, b, -1.0, nullptr, bpart.as<double>()); note_launch();
    k_sum_partials<<<nrhs, RED_THREADS, 0, st>>>(bpart.as<double>(), nblk_r, bdsum.as<double>()); note_launch();
    BRI_CUDA(cudaMemcpyAsync(bn2.data(), bdsum.as<double>(), sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    BRI_CUDA(cudaStreamSynchronize(st));
    Counters dummy;
    stats->max_true_residual = 0.0;
    for (int k = 0; k < n; ++k) {
      rc = residual64(c, m0, nrhs, b, X + (int64_t)k * nrhs * nreal, sig[k], nullptr, btmp1.as<double>(),
                      btmp2.as<double>(), bpart.as<double>(), bdsum.as<double>(), rn2.data(), &dummy, op);
      if (rc) return rc;
      double worst = 0.0;
      for (int s = 0; s < nrhs; ++s) worst = std::max(worst, std::sqrt(rn2[s] / std::max(bn2[s], 1e-300)));
      if (k < NS) stats->shift_residual[k] = worst;
      stats->max_true_residual = std::max(stats->max_true_residual, worst);
    }
  }

  if ((rc = finish_sign(c, (double*)y, b, nrhs, n, c0, w, X, m0, out_scale, b_coeff, cnt, op))) return rc;
  BRI_CUDA(cudaStreamSynchronize(st));
  tph[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tmark).count();
  if (stats) {
    stats->iterations = iters;
    stats->matvecs = cnt.matvecs;
    stats->matvecs_f64 = cnt.matvecs64;
    stats->refinements = refinements;
    stats->n_shifts = n;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int ph = 0; ph < 4; ++ph) stats->phase_seconds[ph] = tph[ph];
  }
  return solve_rc;
}

// Batched sign function / overlap over several lattices (row a8): phase 1 of
// every lattice and right-hand side in one system table (work-list stencil,
// device-resident scalars, WHILE-node graph); then, for the mixed scheme, the
// FP64 residuals and FP32 corrections of each lattice, and the final
// y = b_coeff b + out_scale D (c0 b + sum_i w_i X_i), the lattices concurrently
// on their own streams (one host thread each).
int batch_sign_apply(bri_ctx* const* cs, int nctx, void* const* ys, const void* const* xs, const int* nrhs, int n,
                     int kind, double rho, double scale, double tol, int prec, double out_scale, double b_coeff,
                     bri_stats* stats) {
  if (nctx > kMaxBatch) {
    set_error("overlap_apply_batch: at most 32 lattices per batch");
    return BRI_ERR_INVALID;
  }
  for (int i = 0; i < nctx; ++i)
    if (cs[i]->kernel != BRI_KERNEL_BRILLOUIN) {
      set_error("overlap_apply_batch: the batched work-list stencil is the Brillouin kernel's");
      return BRI_ERR_INVALID;
    }
  auto t0 = std::chrono::steady_clock::now();
  configure_pool_once();
  double c0, w[NS], sig[NS];
  int rc = kl_host(n, kind, scale, &c0, w, sig);
  if (rc) return rc;
  const double m0 = -rho;
  const int maxiter = (stats && stats->maxiter > 0) ? stats->maxiter : 20000;
  for (int i = 0; i < nctx; ++i) BRI_CUDA(cudaStreamSynchronize(cs[i]->stream));
  cudaStream_t bs = nullptr;
  BRI_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } guard{bs};
  // system table
  BatchTab tab;
  memset(&tab, 0, sizeof(tab));
  tab.nlat = nctx;
  std::vector<SysDesc> sd;
  std::vector<int> first_sys(nctx);
  int64_t off = 0;
  for (int i = 0; i < nctx; ++i) {
    bri_ctx* c = cs[i];
    tab.lat[i].g = c->g;
    tab.lat[i].diag = 15.0 / 8.0 + m0;
    if (prec == BRI_PREC_F64) {
      tab.lat[i].W = c->W64;
      tab.lat[i].C = c->have_clover ? (const void*)c->C64 : nullptr;
    } else {
      tab.lat[i].W = prec == BRI_PREC_F32_BF16 ? (const void*)c->W16 : (const void*)c->W32;
      tab.lat[i].C = c->have_clover ? (const void*)c->C32 : nullptr;
    }
    first_sys[i] = (int)sd.size();
    for (int r = 0; r < nrhs[i]; ++r) {
      SysDesc d;
      d.lat = i;
      d.pad = 0;
      d.n2 = c->g.V * 12;
      d.off = off;
      d.offn = off * n;
      off += d.n2;
      sd.push_back(d);
    }
  }
  const int S = (int)sd.size();
  DevBuf bsd;
  if ((rc = bsd.alloc(sizeof(SysDesc) * S, bs))) return rc;
  BRI_CUDA(cudaMemcpyAsync(bsd.p, sd.data(), sizeof(SysDesc) * S, cudaMemcpyHostToDevice, bs));
  std::vector<DevBuf> Xs(nctx);
  SolveInfo info1;
  int solve_rc = BRI_OK;
  double lam_est = 0.0;
  auto phase1 = [&](auto tag, auto ltag) -> int {
    using R = decltype(tag);
    using LS = decltype(ltag);
    using T = typename P2<R>::T;
    DevBuf bb, bx;
    int q;
    if ((q = bb.alloc(sizeof(T) * off, bs))) return q;
    if ((q = bx.alloc(sizeof(double2) * off * n, bs))) return q;
    for (int i = 0; i < nctx; ++i) {
      kb_scatter_b<R><<<dim3(grid_for(cs[i]->g.V * 12, nrhs[i]), nrhs[i]), RED_THREADS, 0, bs>>>(
          bsd.as<SysDesc>(), first_sys[i], (const double2*)xs[i], bb.as<T>());
      note_launch();
    }
    const double tol1 = sizeof(R) == 8 ? tol : std::max(tol, prec == BRI_PREC_F32 ? 1e-7 : 1e-6);
    q = batch_multishift<R, LS>(bs, tab, sd, n, sig, bb.as<T>(), bx.as<double2>(), tol1, maxiter, &info1.iters, &info1.cnt,
                                &lam_est);
    if (q < 0) return q;
    solve_rc = std::max(solve_rc, q);
    for (int i = 0; i < nctx; ++i) {
      const int64_t nreal = cs[i]->g.V * 24;
      int qq;
      if ((qq = Xs[i].alloc(sizeof(double) * nreal * nrhs[i] * n, bs))) return qq;
      kb_gather_x<<<dim3(grid_for(cs[i]->g.V * 12, nrhs[i] * n), nrhs[i], n), RED_THREADS, 0, bs>>>(
          bsd.as<SysDesc>(), first_sys[i], nrhs[i], n, bx.as<double2>(), Xs[i].as<double2>());
      note_launch();
    }
    BRI_LAUNCH_CHECK("batched phase 1");
    BRI_CUDA(cudaStreamSynchronize(bs));
    return BRI_OK;
  };
  if (prec == BRI_PREC_F64) rc = phase1(double(), double2());
  else if (prec == BRI_PREC_F32) rc = phase1(float(), float2());
  else rc = phase1(float(), __nv_bfloat162());
  if (rc < 0) return rc;
  lam_est = 1.1 * lam_est + 1e-3;
  const double t_phase1 = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // per lattice: refinement (mixed) and the final application, concurrently
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> rcs(nctx, BRI_OK);
  std::vector<std::string> errs(nctx);
  std::vector<SolveInfo> infos(nctx);
  std::vector<std::thread> pool;
  for (int i = 0; i < nctx; ++i) {
    pool.emplace_back([&, i]() {
      cudaSetDevice(dev);
      bri_ctx* c = cs[i];
      StreamScope scope(c);
      SolveInfo& inf = infos[i];
      auto tm = std::chrono::steady_clock::now();
      auto lap = [&](int ph) {
        cudaStreamSynchronize(c->stream);
        auto t1 = std::chrono::steady_clock::now();
        inf.tph[ph] += std::chrono::duration<double>(t1 - tm).count();
        tm = t1;
      };
      int q = BRI_OK;
      if (prec != BRI_PREC_F64)
        q = refine_mixed(c, (const double*)xs[i], nrhs[i], n, sig, m0, tol, maxiter, Xs[i].as<double>(), lam_est, inf,
                         lap);
      if (q >= 0) {
        if (prec != BRI_PREC_F64) lap(2);
        const int q2 = finish_sign(c, (double*)ys[i], (const double*)xs[i], nrhs[i], n, c0, w, Xs[i].as<double>(), m0,
                                   out_scale, b_coeff, inf.cnt, nullptr);
        if (q2) q = q2;
        cudaStreamSynchronize(c->stream);
        lap(3);
      }
      rcs[i] = q;
      if (q < 0) errs[i] = bri_last_error();
    });
  }
  for (auto& th : pool) th.join();
  int worst = solve_rc;
  for (int i = 0; i < nctx; ++i) {
    if (rcs[i] < 0) {
      set_error("overlap_apply_batch: lattice " + std::to_string(i) + ": " + errs[i]);
      return rcs[i];
    }
    worst = std::max(worst, rcs[i]);
  }
  const double total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < nctx; ++i) {
      bri_stats& s = stats[i];
      const int want = s.want_true_residual, mi = s.maxiter;
      memset(&s, 0, sizeof(s));
      s.want_true_residual = want;
      s.maxiter = mi;
      s.iterations = info1.iters;
      s.matvecs = info1.cnt.matvecs + infos[i].cnt.matvecs;
      s.matvecs_f64 = info1.cnt.matvecs64 + infos[i].cnt.matvecs64;
      s.refinements = infos[i].refinements;
      s.n_shifts = n;
      s.seconds = total;
      s.phase_seconds[0] = t_phase1;
      for (int ph = 1; ph < 4; ++ph) s.phase_seconds[ph] = infos[i].tph[ph];
    }
  return worst;
}

}  // namespace bri
