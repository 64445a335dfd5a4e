// Massive overlap solve with cascaded preconditioning (Secs. 4.2-4.4, Sec. 8).
//
// The massive Dirac equation D_m x = b becomes (D_ov + mt) x = bt with
// mt = am / (1 - am/(2 rho)) and, for the traditional form (Eq.
// upshot_traditional) bt = b / (1 - am/(2 rho)), for the complete form (Eq.
// upshot_complete) bt = [1 + am/(2 rho) (1 - D_ov/(2 rho))] b / (1 - am/(2 rho)).
// Divided by rho, every operator of the cascade has the form
//   K_j = D_{-rho} r_j(D^dagger D) + (1 + mt/rho),
// with r_j the Kenney-Laub rational of order j (K_0 uses r = 1: the kernel
// itself plus the constant, Eq. cascaded_one) and D the context's kernel
// operator.  Without a cascade (n_inner = 0) K_n is solved by BiCGstab, the
// paper's outer method.  With the cascade the preconditioner of K_n is an
// inexact solve with K_{n_inner} (relative 1e-2), itself preconditioned by an
// inexact solve with K_0 (Eqs. cascaded_one, cascaded_two).  An inexact inner
// solve is a different operator at every application, so the two outer levels
// use flexible GMRES (Saad, SIAM J. Sci. Comput. 14 (1993) 461), which keeps
// the preconditioned directions z_j and stays exact for a varying
// preconditioner; x = solution of K_n x = bt / rho.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <vector>

namespace bri {
namespace {

using cplx = std::complex<double>;
constexpr int TH = 256;

__global__ void k_cdot(int64_t n, const double2* __restrict__ a, const double2* __restrict__ b, double2* part) {
  double re = 0.0, im = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    re += x.x * y.x + x.y * y.y;  // conj(a) b
    im += x.x * y.y - x.y * y.x;
  }
  __shared__ double sr[TH / 32], si[TH / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, q = 0.0;
    for (int w = 0; w < TH / 32; ++w) {
      r += sr[w];
      q += si[w];
    }
    part[blockIdx.x] = make_double2(r, q);
  }
}

// y = a x + b y  (complex scalars)
__global__ void k_caxpby(int64_t n, double2 a, const double2* __restrict__ x, double2 b, double2* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 xv = x[i], yv = y[i];
    y[i] = make_double2(a.x * xv.x - a.y * xv.y + b.x * yv.x - b.y * yv.y,
                        a.x * xv.y + a.y * xv.x + b.x * yv.y + b.y * yv.x);
  }
}

// y = a x (real a)
__global__ void k_scale(int64_t n, double a, const double2* __restrict__ x, double2* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i] = make_double2(a * v.x, a * v.y);
  }
}

constexpr int NBLK = 1024;

struct Vec {
  double2* p = nullptr;
  cudaStream_t s = nullptr;
  ~Vec() {
    if (p) cudaFreeAsync(p, s);
  }
  int alloc(int64_t n, cudaStream_t st) {
    s = st;
    cudaError_t e = cudaMallocAsync(&p, sizeof(double2) * n, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("overlap_solve: cudaMallocAsync failed");
      return BRI_ERR_OOM;
    }
    note_device_alloc();
    return BRI_OK;
  }
};

struct Ctx {
  bri_ctx* c;
  int64_t n;  // complex entries of one vector
  double2* part;
  std::vector<double2> hpart;
  int rc = BRI_OK;

  cplx dot(const double2* a, const double2* b) {
    k_cdot<<<NBLK, TH, 0, c->stream>>>(n, a, b, part);
    note_launch();
    if (cudaMemcpyAsync(hpart.data(), part, sizeof(double2) * NBLK, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "overlap_solve: reduction");
      return 0.0;
    }
    double re = 0.0, im = 0.0;
    for (int i = 0; i < NBLK; ++i) {
      re += hpart[i].x;
      im += hpart[i].y;
    }
    return cplx(re, im);
  }
  void axpby(cplx a, const double2* x, cplx b, double2* y) {
    k_caxpby<<<NBLK, TH, 0, c->stream>>>(n, make_double2(a.real(), a.imag()), x, make_double2(b.real(), b.imag()), y);
    note_launch();
  }
  void copy(double2* dst, const double2* src) {
    cudaMemcpyAsync(dst, src, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c->stream);
  }
};

using Op = std::function<int(double2* y, const double2* x)>;

// Right-preconditioned BiCGstab for K x = b to relative residual tol; the
// preconditioner may be an inexact inner solve.  x holds the initial guess.
int bicgstab(Ctx& cx, const Op& K, const Op* M, double2* x, const double2* b, double tol, int maxit, int* iters,
             double* relres) {
  cudaStream_t st = cx.c->stream;
  Vec r, rh, p, v, s, t, ph, sh;
  int rc;
  for (Vec* w : {&r, &rh, &p, &v, &s, &t, &ph, &sh})
    if ((rc = w->alloc(cx.n, st))) return rc;
  if ((rc = K(r.p, x))) return rc;
  cx.axpby(1.0, b, -1.0, r.p);  // r = b - K x
  cx.copy(rh.p, r.p);
  cudaMemsetAsync(p.p, 0, sizeof(double2) * cx.n, st);
  cudaMemsetAsync(v.p, 0, sizeof(double2) * cx.n, st);
  const double bn = std::sqrt(cx.dot(b, b).real());
  cplx rho_old = 1.0, alpha = 1.0, omega = 1.0;
  double rn = std::sqrt(cx.dot(r.p, r.p).real());
  int it = 0;
  while (it < maxit && rn > tol * bn && cx.rc == BRI_OK) {
    ++it;
    const cplx rho_new = cx.dot(rh.p, r.p);
    const cplx beta = (rho_new / rho_old) * (alpha / omega);
    cx.axpby(-omega, v.p, 1.0, p.p);  // p = p - omega v
    cx.axpby(1.0, r.p, beta, p.p);    // p = r + beta p
    if (M) {
      cudaMemsetAsync(ph.p, 0, sizeof(double2) * cx.n, st);
      if ((rc = (*M)(ph.p, p.p))) return rc;
    } else {
      cx.copy(ph.p, p.p);
    }
    if ((rc = K(v.p, ph.p))) return rc;
    alpha = rho_new / cx.dot(rh.p, v.p);
    cx.copy(s.p, r.p);
    cx.axpby(-alpha, v.p, 1.0, s.p);  // s = r - alpha v
    if (M) {
      cudaMemsetAsync(sh.p, 0, sizeof(double2) * cx.n, st);
      if ((rc = (*M)(sh.p, s.p))) return rc;
    } else {
      cx.copy(sh.p, s.p);
    }
    if ((rc = K(t.p, sh.p))) return rc;
    const cplx tt = cx.dot(t.p, t.p);
    omega = tt.real() > 0.0 ? cx.dot(t.p, s.p) / tt : 0.0;
    cx.axpby(alpha, ph.p, 1.0, x);  // x += alpha ph + omega sh
    cx.axpby(omega, sh.p, 1.0, x);
    cx.copy(r.p, s.p);
    cx.axpby(-omega, t.p, 1.0, r.p);  // r = s - omega t
    rn = std::sqrt(cx.dot(r.p, r.p).real());
    rho_old = rho_new;
    if (!std::isfinite(rn)) {
      set_error("overlap_solve: BiCGstab broke down (non-finite residual)");
      return BRI_ERR_NONFINITE;
    }
  }
  if (cx.rc) return cx.rc;
  *iters = it;
  *relres = rn / bn;
  return rn <= tol * bn ? BRI_OK : BRI_NOT_CONVERGED;
}

// Gram-Schmidt helpers of FGMRES: the Krylov basis is one contiguous block
// V = [j][n] complex.  part[i][blk] = partial <V_i, w> (conj(V_i) w).
constexpr int MD_BLK = 256;
__global__ void k_multidot(int64_t n, const double2* __restrict__ V, const double2* __restrict__ w, double2* part) {
  const double2* v = V + (int64_t)blockIdx.y * n;
  double re = 0.0, im = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[i], b = w[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double sr[TH / 32], si[TH / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, q = 0.0;
    for (int k = 0; k < TH / 32; ++k) {
      r += sr[k];
      q += si[k];
    }
    part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(r, q);
  }
}

constexpr int MAXM = 64;
struct Coefs {
  double2 c[MAXM];
};
// w += sum_{k<j} c_k V_k
__global__ void k_multi_axpy(int64_t n, int j, const __grid_constant__ Coefs cf, const double2* __restrict__ V,
                             double2* w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[i];
    for (int k = 0; k < j; ++k) {
      const double2 v = V[(int64_t)k * n + i], c = cf.c[k];
      acc.x += c.x * v.x - c.y * v.y;
      acc.y += c.x * v.y + c.y * v.x;
    }
    w[i] = acc;
  }
}

// h[k] = <V_k, w> for k < j (one launch, host sum in a fixed order)
int multidot(Ctx& cx, const double2* V, int j, const double2* w, std::vector<cplx>& h) {
  k_multidot<<<dim3(MD_BLK, j), TH, 0, cx.c->stream>>>(cx.n, V, w, cx.part);
  note_launch();
  BRI_CUDA(cudaMemcpyAsync(cx.hpart.data(), cx.part, sizeof(double2) * MD_BLK * j, cudaMemcpyDeviceToHost,
                           cx.c->stream));
  BRI_CUDA(cudaStreamSynchronize(cx.c->stream));
  h.assign(j, cplx(0.0, 0.0));
  for (int k = 0; k < j; ++k) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < MD_BLK; ++b) {
      re += cx.hpart[(size_t)k * MD_BLK + b].x;
      im += cx.hpart[(size_t)k * MD_BLK + b].y;
    }
    h[k] = cplx(re, im);
  }
  return BRI_OK;
}

void multi_axpy(Ctx& cx, const double2* V, int j, const std::vector<cplx>& c, double sign, double2* w) {
  Coefs cf;
  for (int k = 0; k < j; ++k) cf.c[k] = make_double2(sign * c[k].real(), sign * c[k].imag());
  k_multi_axpy<<<NBLK, TH, 0, cx.c->stream>>>(cx.n, j, cf, V, w);
  note_launch();
}

// Flexible GMRES(m) for K x = b with a right preconditioner M that may change
// from one application to the next (an inexact inner solve): the Arnoldi
// relation K Z_m = V_{m+1} Hbar_m holds with the preconditioned directions
// z_j = M(v_j) kept, and x = x0 + Z_m y with y minimising
// ||beta e_1 - Hbar_m y|| (complex Givens rotations).  Orthogonalisation is
// classical Gram-Schmidt applied twice.  x holds the initial guess.  A cycle
// ends when the Arnoldi residual estimate reaches tol ||b||; with check_true
// the true residual b - K x then decides, and the next cycle restarts from x.
int fgmres(Ctx& cx, const Op& K, const Op* M, double2* x, const double2* b, double tol, int m, int maxit,
           bool check_true, int* iters, double* relres) {
  cudaStream_t st = cx.c->stream;
  m = std::max(1, std::min(m, MAXM - 1));
  Vec V, Z, w;
  int rc;
  if ((rc = V.alloc(cx.n * (m + 1), st))) return rc;
  if ((rc = Z.alloc(cx.n * m, st))) return rc;
  if ((rc = w.alloc(cx.n, st))) return rc;
  const double bn = std::sqrt(cx.dot(b, b).real());
  if (cx.rc) return cx.rc;
  *iters = 0;
  *relres = 0.0;
  if (bn == 0.0) {
    cudaMemsetAsync(x, 0, sizeof(double2) * cx.n, st);
    return BRI_OK;
  }
  int it = 0;
  double rn = 0.0;
  std::vector<cplx> h, h2, g(m + 1), cs(m), sn(m), y(m);
  std::vector<std::vector<cplx>> H(m, std::vector<cplx>(m + 1));
  while (true) {
    // r0 = b - K x, v_0 = r0 / ||r0||
    if ((rc = K(w.p, x))) return rc;
    cx.axpby(1.0, b, -1.0, w.p);
    rn = std::sqrt(cx.dot(w.p, w.p).real());
    if (cx.rc) return cx.rc;
    if (!std::isfinite(rn)) {
      set_error("overlap_solve: FGMRES met a non-finite residual");
      return BRI_ERR_NONFINITE;
    }
    if (rn <= tol * bn || it >= maxit) break;
    cx.axpby(1.0 / rn, w.p, 0.0, V.p);
    std::fill(g.begin(), g.end(), cplx(0.0, 0.0));
    g[0] = rn;
    int j = 0;
    double est = rn;
    while (j < m && it < maxit) {
      ++it;
      double2* vj = V.p + (int64_t)j * cx.n;
      double2* zj = Z.p + (int64_t)j * cx.n;
      if (M) {
        cudaMemsetAsync(zj, 0, sizeof(double2) * cx.n, st);
        if ((rc = (*M)(zj, vj))) return rc;
      } else {
        cx.copy(zj, vj);
      }
      if ((rc = K(w.p, zj))) return rc;
      // two passes of classical Gram-Schmidt against v_0..v_j
      if ((rc = multidot(cx, V.p, j + 1, w.p, h))) return rc;
      multi_axpy(cx, V.p, j + 1, h, -1.0, w.p);
      if ((rc = multidot(cx, V.p, j + 1, w.p, h2))) return rc;
      multi_axpy(cx, V.p, j + 1, h2, -1.0, w.p);
      for (int i = 0; i <= j; ++i) h[i] += h2[i];
      const double hn = std::sqrt(cx.dot(w.p, w.p).real());
      if (cx.rc) return cx.rc;
      if (!std::isfinite(hn)) {
        set_error("overlap_solve: FGMRES met a non-finite basis vector");
        return BRI_ERR_NONFINITE;
      }
      for (int i = 0; i <= j; ++i) H[j][i] = h[i];
      H[j][j + 1] = hn;
      if (hn > 0.0) cx.axpby(1.0 / hn, w.p, 0.0, V.p + (int64_t)(j + 1) * cx.n);
      // the previous rotations on the new column, then the one that zeroes H[j][j+1]
      for (int i = 0; i < j; ++i) {
        const cplx a = H[j][i], bb = H[j][i + 1];
        H[j][i] = cs[i] * a + sn[i] * bb;
        H[j][i + 1] = -std::conj(sn[i]) * a + cs[i] * bb;
      }
      const cplx a = H[j][j];
      const double r = std::hypot(std::abs(a), hn);
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = std::abs(a) / r;
        sn[j] = (a / std::abs(a)) * hn / r;
      }
      H[j][j] = cs[j] * a + sn[j] * hn;
      H[j][j + 1] = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      est = std::abs(g[j + 1]);
      ++j;
      if (est <= tol * bn || hn == 0.0) break;
    }
    // y = R^{-1} g, x += Z y
    for (int i = j - 1; i >= 0; --i) {
      cplx v = g[i];
      for (int k = i + 1; k < j; ++k) v -= H[k][i] * y[k];
      y[i] = v / H[i][i];
    }
    multi_axpy(cx, Z.p, j, y, 1.0, x);
    if (!check_true && (est <= tol * bn || it >= maxit)) {
      rn = est;
      break;
    }
  }
  if (cx.rc) return cx.rc;
  *iters = it;
  *relres = rn / bn;
  return rn <= tol * bn ? BRI_OK : BRI_NOT_CONVERGED;
}

}  // namespace

int overlap_solve_impl(bri_ctx* c, double2* x, const double2* b, int n_outer, int n_inner, int kind, double rho,
                       double am, int complete, double tol, int prec, int maxiter, bri_stats* st_out) {
  cudaStream_t st = c->stream;
  const int64_t n = c->g.V * 12;
  const double m0 = -rho;
  const double k = 1.0 - am / (2.0 * rho);
  const double mt = am / k;
  const double shift = 1.0 + mt / rho;
  // Accuracy of the outer operator's sign function: the solution can be ~rho/mt
  // times larger than the right-hand side, so the rational is applied to
  // 0.1 tol mt/rho (at most 1e-10, at least 1e-14) for the outer residual to
  // be meaningful at tol.
  const double inner_tol_sign = std::max(1e-14, std::min(1e-10, 0.1 * tol * std::min(1.0, mt / rho)));
  Vec part, bt, tmp;
  int rc;
  if ((rc = part.alloc(std::max(NBLK, MD_BLK * MAXM), st))) return rc;
  if ((rc = bt.alloc(n, st))) return rc;
  if ((rc = tmp.alloc(n, st))) return rc;
  Ctx cx{c, n, part.p, std::vector<double2>(std::max(NBLK, MD_BLK * MAXM))};
  int matvecs = 0, sign_iters = 0;

  // K_j y = D r_j(A) x + shift x  (j = 0: the kernel)
  auto make_K = [&](int order, double sign_tol) -> Op {
    return [=, &matvecs, &sign_iters](double2* y, const double2* xin) -> int {
      if (order == 0) {
        int r = dirac_kernel(c, y, xin, 1, m0, 0, BRI_PREC_F64, st);
        if (r) return r;
        k_caxpby<<<NBLK, TH, 0, st>>>(n, make_double2(shift, 0.0), xin, make_double2(1.0, 0.0), y);
        note_launch();
        matvecs += 1;
        return BRI_OK;
      }
      bri_stats s;
      memset(&s, 0, sizeof(s));
      int r = sign_apply(c, y, xin, 1, order, kind, rho, 1.0, sign_tol, prec, 1.0, shift, &s);
      matvecs += s.matvecs;
      sign_iters += s.iterations;
      return r < 0 ? r : BRI_OK;
    };
  };

  // bt / rho (traditional or complete right-hand side)
  if (complete) {
    // bt = [1 + am/(2 rho)] b / k - am/(4 rho^2) D_ov b / k, D_ov b = rho (b + D r(A) b)
    bri_stats s;
    memset(&s, 0, sizeof(s));
    rc = sign_apply(c, tmp.p, b, 1, n_outer, kind, rho, 1.0, inner_tol_sign, prec, rho, rho, &s);
    if (rc < 0) return rc;
    matvecs += s.matvecs;
    cx.copy(bt.p, b);
    k_caxpby<<<NBLK, TH, 0, st>>>(n, make_double2(-am / (4.0 * rho * rho * k * rho), 0.0), tmp.p,
                                  make_double2((1.0 + am / (2.0 * rho)) / (k * rho), 0.0), bt.p);
    note_launch();
  } else {
    k_scale<<<NBLK, TH, 0, st>>>(n, 1.0 / (k * rho), b, bt.p);
    note_launch();
  }

  const Op K_outer = make_K(n_outer, inner_tol_sign);
  int outer_it = 0, inner_it_total = 0;
  double relres = 0.0;
  cudaMemsetAsync(x, 0, sizeof(double2) * n, st);
  if (n_inner > 0) {
    const Op K_inner = make_K(n_inner, 1e-6);
    const Op K_kernel = make_K(0, 0.0);
    // level 0: inexact solve with the kernel operator (a fixed operator, BiCGstab)
    const Op M0 = [&](double2* y, const double2* r) -> int {
      int it = 0;
      double rr = 0.0;
      int q = bicgstab(cx, K_kernel, nullptr, y, r, 1e-2, 200, &it, &rr);
      inner_it_total += it;
      return q < 0 ? q : BRI_OK;
    };
    // level 1: inexact solve with K_{n_inner}, flexibly preconditioned by level 0
    const Op M1 = [&](double2* y, const double2* r) -> int {
      int it = 0;
      double rr = 0.0;
      int q = fgmres(cx, K_inner, &M0, y, r, 1e-2, 32, 32, false, &it, &rr);
      inner_it_total += it;
      return q < 0 ? q : BRI_OK;
    };
    rc = fgmres(cx, K_outer, &M1, x, bt.p, tol, 24, maxiter, true, &outer_it, &relres);
  } else {
    rc = bicgstab(cx, K_outer, nullptr, x, bt.p, tol, maxiter, &outer_it, &relres);
  }
  if (rc < 0) return rc;
  // FP64 true residual ||bt/rho - K x|| / ||bt/rho||
  {
    const int q = K_outer(tmp.p, x);
    if (q < 0) return q;
    cx.axpby(1.0, bt.p, -1.0, tmp.p);
    relres = std::sqrt(cx.dot(tmp.p, tmp.p).real() / cx.dot(bt.p, bt.p).real());
    if (cx.rc) return cx.rc;
    if (rc == BRI_OK && relres > tol) rc = BRI_NOT_CONVERGED;
  }
  cudaStreamSynchronize(st);
  if (st_out) {
    st_out->iterations = outer_it;
    st_out->refinements = inner_it_total;
    st_out->matvecs = matvecs;
    st_out->max_true_residual = relres;
    st_out->n_shifts = n_outer;
  }
  return rc;
}

}  // namespace bri
