// Quality diagnostics of the overlap operator (Sec. 5) and the nested
// Kenney-Laub iterates of shifted kernels (Sec. 4.1).
//
// Sec. 5 verifies three properties of D = D_ov (a fixed-order rational):
//   normality      ||(D D^dagger - D^dagger D) eta||            (Sec. 5.1)
//   GW defect      ||(D gamma5 + gamma5 D - (1/rho) D gamma5 D) eta||   (Sec. 5.2,
//                  Eq. ginswils_one)
//   locality       |zeta(x)|, zeta = D eta with eta supported on one site,
//                  against the Euclidean distance |x| (Sec. 5.3).
// With D^dagger = gamma5 D gamma5 two applications of D to two vectors per
// source give all of them:
//   A0 = D eta, A1 = D gamma5 eta, B0 = D gamma5 A0, B1 = D gamma5 A1,
//   D D^dagger eta = B1, D^dagger D eta = gamma5 B0,
//   GW vector = A1 + gamma5 A0 - B0 / rho.
//
// Sec. 4.1 nests the mappings: with X = D_{-rho} (the kernel), Y_1 =
// X r_{n1}(X^dagger X) (the sign-function approximation of order n1),
// Y_j = Y_{j-1} r_{nj}(Y_{j-1}^dagger Y_{j-1}), and D^(k) = rho (1 + Y_k).  Each
// level is the multi-shift solve of sign_apply on the operator of the level
// below, which stays gamma5-hermitian, so its adjoint is gamma5 Y gamma5.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace bri {
namespace {

constexpr int TH = 256;

// out = gamma5 in (spins 2 and 3 negated) for n_sites_rhs site-spinors
__global__ void k_g5(int64_t nsr, const double2* __restrict__ in, double2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsr * 12; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = in[i];
    if (((i % 12) / 3) >= 2) {
      v.x = -v.x;
      v.y = -v.y;
    }
    out[i] = v;
  }
}

__device__ __forceinline__ double2 g5c(double2 v, int64_t i) {
  return ((i % 12) / 3) >= 2 ? make_double2(-v.x, -v.y) : v;
}

// Per rhs r: partial sums of ||B1 - g5 B0||^2 and ||A1 + g5 A0 - B0/rho||^2.
__global__ void k_defects(int64_t n, const double2* __restrict__ A0, const double2* __restrict__ A1,
                          const double2* __restrict__ B0, const double2* __restrict__ B1, double inv_rho,
                          double* part) {
  const int r = blockIdx.y;
  const int64_t off = (int64_t)r * n;
  double sn = 0.0, sg = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a0 = g5c(A0[off + i], i), a1 = A1[off + i], b0 = B0[off + i], b1 = B1[off + i];
    const double2 g5b0 = g5c(b0, i);
    const double nx = b1.x - g5b0.x, ny = b1.y - g5b0.y;
    const double gx = a1.x + a0.x - inv_rho * b0.x, gy = a1.y + a0.y - inv_rho * b0.y;
    sn += nx * nx + ny * ny;
    sg += gx * gx + gy * gy;
  }
  __shared__ double s1[TH / 32], s2[TH / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
    sg += __shfl_xor_sync(0xffffffffu, sg, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = sn;
    s2[threadIdx.x >> 5] = sg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < TH / 32; ++w) {
      a += s1[w];
      b += s2[w];
    }
    part[((int64_t)r * gridDim.x + blockIdx.x) * 2 + 0] = a;
    part[((int64_t)r * gridDim.x + blockIdx.x) * 2 + 1] = b;
  }
}

// profile[r][bin] += ||zeta_r(x)||, counts[bin] += 1 (rhs 0 only), bin = |x - src|^2
// with the minimal periodic image in each direction (bins >= nbins dropped).
__global__ void k_locality(Geom g, int nrhs, const double2* __restrict__ z, int src, int nbins, double* profile,
                           int* counts) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  int64_t rn = n, rs = src;
  int r2 = 0;
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int cn = (int)(mu < 3 ? rn % L : rn), cs = (int)(mu < 3 ? rs % L : rs);
    if (mu < 3) {
      rn /= L;
      rs /= L;
    }
    int d = cn - cs;
    if (d < 0) d = -d;
    d = d < L - d ? d : L - d;
    r2 += d * d;
  }
  if (r2 >= nbins) return;
  atomicAdd(counts + r2, 1);
  for (int r = 0; r < nrhs; ++r) {
    const double2* zz = z + ((int64_t)r * g.V + n) * 12;
    double s = 0.0;
    for (int e = 0; e < 12; ++e) s += zz[e].x * zz[e].x + zz[e].y * zz[e].y;
    atomicAdd(profile + (int64_t)r * nbins + r2, sqrt(s));
  }
}

struct Buf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~Buf() {
    if (p) cudaFreeAsync(p, s);
  }
  int alloc(size_t bytes, cudaStream_t st) {
    s = st;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error(std::string("cudaMallocAsync failed: ") + cudaGetErrorString(e));
      return BRI_ERR_OOM;
    }
    note_device_alloc();
    return BRI_OK;
  }
  template <typename T> T* as() const { return (T*)p; }
};

// y = D_ov x = rho (x + gamma5 f(H) x) (massless), nsys systems
int dov(bri_ctx* c, double2* y, const double2* x, int nsys, int n, int kind, double rho, double tol, int prec,
        bri_stats* acc) {
  bri_stats s;
  memset(&s, 0, sizeof(s));
  int rc = sign_apply(c, y, x, nsys, n, kind, rho, 1.0, tol, prec, rho, rho, &s);
  if (acc) {
    acc->iterations = std::max(acc->iterations, s.iterations);
    acc->matvecs += s.matvecs;
    acc->matvecs_f64 += s.matvecs_f64;
    acc->refinements += s.refinements;
  }
  return rc;
}

}  // namespace
}  // namespace bri

using namespace bri;

static int check_diag(bri_ctx* c, const void* eta, int nrhs, int n, double rho, double tol, int prec, const char* who) {
  if (!c || !eta || nrhs < 1 || nrhs > 4096 || n < 1 || n > BRI_MAX_SHIFTS || !(rho > 0.0 && rho < 2.0) ||
      !(tol > 0.0 && tol < 1.0) || ((uintptr_t)eta & 15) ||
      (prec != BRI_PREC_F64 && prec != BRI_PREC_F32 && prec != BRI_PREC_F32_BF16)) {
    set_error(std::string(who) + ": invalid argument");
    return BRI_ERR_INVALID;
  }
  if (!c->have_links) {
    set_error(std::string(who) + ": call bri_build_links first");
    return BRI_ERR_NOLINKS;
  }
  return BRI_OK;
}

extern "C" int overlap_quality(bri_ctx* c, const void* eta, int nrhs, int n, int kind, double rho, double tol,
                               int prec, double* normality, double* gw, bri_stats* st) {
  int rc = check_diag(c, eta, nrhs, n, rho, tol, prec, "overlap_quality");
  if (rc) return rc;
  if (!normality || !gw) {
    set_error("overlap_quality: null output");
    return BRI_ERR_INVALID;
  }
  cudaStream_t s = c->stream;
  const int64_t nc = c->g.V * 12;  // complex entries per vector
  Buf bin, bA, bB, bpart;
  if ((rc = bin.alloc(sizeof(double2) * nc * 2 * nrhs, s))) return rc;
  if ((rc = bA.alloc(sizeof(double2) * nc * 2 * nrhs, s))) return rc;
  if ((rc = bB.alloc(sizeof(double2) * nc * 2 * nrhs, s))) return rc;
  const int nblk = 256;
  if ((rc = bpart.alloc(sizeof(double) * 2 * nblk * nrhs, s))) return rc;
  double2* in = bin.as<double2>();
  double2* A = bA.as<double2>();
  double2* B = bB.as<double2>();
  BRI_CUDA(cudaMemcpyAsync(in, eta, sizeof(double2) * nc * nrhs, cudaMemcpyDeviceToDevice, s));
  k_g5<<<1024, TH, 0, s>>>(c->g.V * nrhs, (const double2*)eta, in + nc * nrhs); note_launch();
  bri_stats acc;
  memset(&acc, 0, sizeof(acc));
  int solve_rc = dov(c, A, in, 2 * nrhs, n, kind, rho, tol, prec, &acc);  // [D eta ; D g5 eta]
  if (solve_rc < 0) return solve_rc;
  k_g5<<<1024, TH, 0, s>>>(c->g.V * 2 * nrhs, A, in); note_launch();
  rc = dov(c, B, in, 2 * nrhs, n, kind, rho, tol, prec, &acc);  // [D g5 D eta ; D g5 D g5 eta]
  if (rc < 0) return rc;
  solve_rc = std::max(solve_rc, rc);
  k_defects<<<dim3(nblk, nrhs), TH, 0, s>>>(nc, A, A + nc * nrhs, B, B + nc * nrhs, 1.0 / rho, bpart.as<double>());
  note_launch();
  BRI_LAUNCH_CHECK("overlap_quality");
  std::vector<double> h((size_t)2 * nblk * nrhs);
  BRI_CUDA(cudaMemcpyAsync(h.data(), bpart.as<double>(), sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  BRI_CUDA(cudaStreamSynchronize(s));
  for (int r = 0; r < nrhs; ++r) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblk; ++k) {
      a += h[((size_t)r * nblk + k) * 2 + 0];
      b += h[((size_t)r * nblk + k) * 2 + 1];
    }
    normality[r] = std::sqrt(a);
    gw[r] = std::sqrt(b);
  }
  if (st) {
    const int want = st->want_true_residual, mi = st->maxiter;
    *st = acc;
    st->n_shifts = n;
    st->want_true_residual = want;
    st->maxiter = mi;
  }
  return solve_rc;
}

extern "C" int overlap_locality(bri_ctx* c, const void* eta, int nrhs, int src, int n, int kind, double rho,
                                double tol, int prec, int nbins, double* profile, int* counts, bri_stats* st) {
  int rc = check_diag(c, eta, nrhs, n, rho, tol, prec, "overlap_locality");
  if (rc) return rc;
  if (!profile || !counts || nbins < 1 || nbins > (1 << 20) || src < 0 || src >= c->g.V) {
    set_error("overlap_locality: need 1 <= nbins <= 2^20, 0 <= src < V and non-null outputs");
    return BRI_ERR_INVALID;
  }
  cudaStream_t s = c->stream;
  const int64_t nc = c->g.V * 12;
  Buf bz, bprof, bcnt;
  if ((rc = bz.alloc(sizeof(double2) * nc * nrhs, s))) return rc;
  if ((rc = bprof.alloc(sizeof(double) * (size_t)nbins * nrhs, s))) return rc;
  if ((rc = bcnt.alloc(sizeof(int) * (size_t)nbins, s))) return rc;
  bri_stats acc;
  memset(&acc, 0, sizeof(acc));
  int solve_rc = dov(c, bz.as<double2>(), (const double2*)eta, nrhs, n, kind, rho, tol, prec, &acc);
  if (solve_rc < 0) return solve_rc;
  BRI_CUDA(cudaMemsetAsync(bprof.as<double>(), 0, sizeof(double) * (size_t)nbins * nrhs, s));
  BRI_CUDA(cudaMemsetAsync(bcnt.as<int>(), 0, sizeof(int) * (size_t)nbins, s));
  k_locality<<<blocks_for(c->g.V, TH), TH, 0, s>>>(c->g, nrhs, bz.as<double2>(), src, nbins, bprof.as<double>(),
                                                  bcnt.as<int>());
  note_launch();
  BRI_LAUNCH_CHECK("overlap_locality");
  BRI_CUDA(cudaMemcpyAsync(profile, bprof.as<double>(), sizeof(double) * (size_t)nbins * nrhs,
                           cudaMemcpyDeviceToHost, s));
  BRI_CUDA(cudaMemcpyAsync(counts, bcnt.as<int>(), sizeof(int) * (size_t)nbins, cudaMemcpyDeviceToHost, s));
  BRI_CUDA(cudaStreamSynchronize(s));
  if (st) {
    const int want = st->want_true_residual, mi = st->maxiter;
    *st = acc;
    st->n_shifts = n;
    st->want_true_residual = want;
    st->maxiter = mi;
  }
  return solve_rc;
}

extern "C" int overlap_nested_apply(bri_ctx* c, void* y, const void* x, int nrhs, int levels, const int* orders,
                                    double rho, double tol, bri_stats* st) {
  int rc = check_diag(c, x, nrhs, 1, rho, tol, BRI_PREC_F64, "overlap_nested_apply");
  if (rc) return rc;
  if (!y || y == x || ((uintptr_t)y & 15) || !orders || levels < 1 || levels > 4) {
    set_error("overlap_nested_apply: need 1 <= levels <= 4, an orders array and distinct aligned x, y");
    return BRI_ERR_INVALID;
  }
  for (int j = 0; j < levels; ++j)
    if (orders[j] < 1 || orders[j] > BRI_MAX_SHIFTS) {
      set_error("overlap_nested_apply: every order must be in [1, 32]");
      return BRI_ERR_INVALID;
    }
  cudaStream_t s = c->stream;
  const int64_t nc = c->g.V * 12;
  const double m0 = -rho;
  bri_stats acc;
  memset(&acc, 0, sizeof(acc));
  int worst = BRI_OK;
  // ops[j] applies Y_j (j >= 1) or X = D_{-rho} (j = 0); the adjoint is
  // gamma5 Y_j gamma5 (every level is gamma5-hermitian)
  std::vector<KernelOp> ops(levels);
  ops[0].apply = [=](double2* out, const double2* in, int nsys, int dagger) -> int {
    return dirac_kernel(c, out, in, nsys, m0, dagger, BRI_PREC_F64, c->stream);
  };
  for (int j = 1; j < levels; ++j) {
    const KernelOp* below = &ops[j - 1];
    const int nj = orders[j - 1];
    ops[j].apply = [=, &acc, &worst](double2* out, const double2* in, int nsys, int dagger) -> int {
      cudaStream_t ss = c->stream;
      Buf tmp;
      int q;
      const double2* src = in;
      if (dagger) {
        if ((q = tmp.alloc(sizeof(double2) * nc * nsys, ss))) return q;
        k_g5<<<1024, TH, 0, ss>>>(c->g.V * nsys, in, tmp.as<double2>()); note_launch();
        src = tmp.as<double2>();
      }
      bri_stats sl;
      memset(&sl, 0, sizeof(sl));
      q = sign_apply(c, out, src, nsys, nj, BRI_KL_DIAGONAL, rho, 1.0, tol, BRI_PREC_F64, 1.0, 0.0, &sl, below);
      if (q < 0) return q;
      worst = std::max(worst, q);
      acc.matvecs += sl.matvecs;
      acc.matvecs_f64 += sl.matvecs_f64;
      if (dagger) {
        k_g5<<<1024, TH, 0, ss>>>(c->g.V * nsys, out, out); note_launch();
      }
      return BRI_OK;
    };
  }
  // D^(k) x = rho x + rho Y_k x, Y_k = Y_{k-1} r_{n_k}(Y_{k-1}^dagger Y_{k-1})
  bri_stats top;
  memset(&top, 0, sizeof(top));
  rc = sign_apply(c, (double2*)y, (const double2*)x, nrhs, orders[levels - 1], BRI_KL_DIAGONAL, rho, 1.0, tol,
                  BRI_PREC_F64, rho, rho, &top, &ops[levels - 1]);
  if (rc < 0) return rc;
  worst = std::max(worst, rc);
  BRI_CUDA(cudaStreamSynchronize(s));
  if (st) {
    const int want = st->want_true_residual, mi = st->maxiter;
    *st = acc;
    st->iterations = top.iterations;
    st->matvecs += top.matvecs;
    st->matvecs_f64 += top.matvecs_f64;
    st->n_shifts = orders[levels - 1];
    st->want_true_residual = want;
    st->maxiter = mi;
  }
  return worst;
}
