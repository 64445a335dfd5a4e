// C ABI entry points, context management and the host-side Kenney-Laub
// coefficients.
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace bri {

static thread_local std::string g_err = "no error";
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_dev_allocs{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_device_alloc() { g_dev_allocs.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int graphs_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("BRI_GRAPHS");
    v = e ? (atoi(e) != 0) : 1;
  }
  return v && current_arena() == nullptr;
}

static cudaEvent_t pool_event(bri_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_begin(bri_ctx* c, cudaStream_t s, cudaEvent_t* a) {
  *a = nullptr;
  if (!c->prof_on) return BRI_OK;
  *a = pool_event(c);
  BRI_CUDA(cudaEventRecord(*a, s));
  return BRI_OK;
}

int prof_end(bri_ctx* c, cudaStream_t s, cudaEvent_t a, int op, int prec, double units) {
  if (!c->prof_on || !a) return BRI_OK;
  cudaEvent_t b = pool_event(c);
  BRI_CUDA(cudaEventRecord(b, s));
  c->prof_pending.push_back(ProfRec{a, b, op, prec, units});
  return BRI_OK;
}

static int prof_collect(bri_ctx* c) {
  for (auto& r : c->prof_pending) {
    BRI_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    BRI_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    c->prof_launches[r.op][r.prec] += 1;
    c->prof_ms[r.op][r.prec] += ms;
    c->prof_units[r.op][r.prec] += r.units;
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_pending.clear();
  return BRI_OK;
}

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? BRI_ERR_OOM : BRI_ERR_CUDA;
}

// Eq. KLnn_parfrac: g_{2n+1}(x) = x/(2n+1) sum_{i=0}^{n} (2 - delta_{in}) / (sin^2 t_i + cos^2 t_i x^2),
// t_i = (2i+1) pi/(4n+2); the i = n term is the constant.  Upper diagonal (Sec. 3.3):
// g_{2n}(x) = (x/n) sum_{i<n} 1/(sin^2 t_i + cos^2 t_i x^2), t_i = (2i+1) pi/(4n).
// With a scale s, f(x/s) = x [c0/s + sum (w_i s)/(x^2 + sigma_i s^2)].
int kl_host(int n, int kind, double scale, double* c0, double* w, double* sigma) {
  if (n < 1 || n > BRI_MAX_SHIFTS) {
    set_error("kl_coeffs: order n must be in [1, 32]");
    return BRI_ERR_INVALID;
  }
  if (!(scale > 0.0) || !std::isfinite(scale)) {
    set_error("kl_coeffs: scale must be positive");
    return BRI_ERR_INVALID;
  }
  if (!c0 || !w || !sigma) {
    set_error("kl_coeffs: null output pointer");
    return BRI_ERR_INVALID;
  }
  const double pi = 3.14159265358979323846;
  if (kind == BRI_KL_DIAGONAL) {
    for (int i = 0; i < n; ++i) {
      const double th = (2 * i + 1) * pi / (4.0 * n + 2.0);
      const double cs = std::cos(th), sn = std::sin(th);
      sigma[i] = (sn / cs) * (sn / cs) * scale * scale;
      w[i] = 2.0 / ((2.0 * n + 1.0) * cs * cs) * scale;
    }
    *c0 = 1.0 / ((2.0 * n + 1.0) * scale);
  } else if (kind == BRI_KL_UPPER) {
    for (int i = 0; i < n; ++i) {
      const double th = (2 * i + 1) * pi / (4.0 * n);
      const double cs = std::cos(th), sn = std::sin(th);
      sigma[i] = (sn / cs) * (sn / cs) * scale * scale;
      w[i] = 1.0 / (n * cs * cs) * scale;
    }
    *c0 = 0.0;
  } else {
    set_error("kl_coeffs: kind must be BRI_KL_DIAGONAL or BRI_KL_UPPER");
    return BRI_ERR_INVALID;
  }
  return BRI_OK;
}

}  // namespace bri

using namespace bri;

extern "C" {

const char* bri_last_error(void) { return g_err.c_str(); }

int bri_create(bri_ctx** out, const int dims[4], int flags, void* stream) {
  if (!out || !dims) {
    set_error("bri_create: null argument");
    return BRI_ERR_INVALID;
  }
  *out = nullptr;
  int64_t V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || dims[mu] > 4096) {
      set_error("bri_create: every extent must be in [2, 4096]");
      return BRI_ERR_INVALID;
    }
    V *= dims[mu];
  }
  if (V > (int64_t(1) << 31) / 40) {
    set_error("bri_create: lattice volume too large for one device");
    return BRI_ERR_INVALID;
  }
  if (flags & ~BRI_ANTIPERIODIC_T) {
    set_error("bri_create: unknown flag");
    return BRI_ERR_INVALID;
  }
  bri_ctx* c = new bri_ctx();
  for (int mu = 0; mu < 4; ++mu) c->g.L[mu] = dims[mu];
  c->g.V = V;
  c->g.str[0] = 1;
  c->g.str[1] = dims[0];
  c->g.str[2] = (int64_t)dims[0] * dims[1];
  c->g.str[3] = (int64_t)dims[0] * dims[1] * dims[2];
  c->flags = flags;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaMallocHost(&c->host_pinned, 1 << 16);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "bri_create: cudaMallocHost");
  }
  *out = c;
  return BRI_OK;
}

void bri_destroy(bri_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  cudaFree(c->W64);
  cudaFree(c->W32);
  cudaFree(c->W16);
  cudaFree(c->U64);
  cudaFree(c->U32);
  cudaFree(c->C64);
  cudaFree(c->C32);
  cudaFree(c->Wdw);
  cudaFree(c->Cdw);
  for (auto& r : c->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  cudaFree(c->ws.ptr);
  cudaFree(c->ws_small.ptr);
  cudaFreeHost(c->host_pinned);
  cudaGetLastError();
  delete c;
}

int bri_set_stream(bri_ctx* c, void* stream) {
  if (!c) {
    set_error("bri_set_stream: null context");
    return BRI_ERR_INVALID;
  }
  c->stream = (cudaStream_t)stream;
  return BRI_OK;
}

int bri_set_kernel(bri_ctx* c, int kernel) {
  if (!c || (kernel != BRI_KERNEL_BRILLOUIN && kernel != BRI_KERNEL_WILSON)) {
    set_error("bri_set_kernel: null context or unknown kernel");
    return BRI_ERR_INVALID;
  }
  c->kernel = kernel;
  return BRI_OK;
}

int bri_build_links(bri_ctx* c, const double* U, double c_sw) {
  if (!c || !U) {
    set_error("bri_build_links: null argument");
    return BRI_ERR_INVALID;
  }
  if (!std::isfinite(c_sw)) {
    set_error("bri_build_links: c_sw must be finite");
    return BRI_ERR_INVALID;
  }
  int rc = launch_build_links(c, U, c_sw);
  if (rc) return rc;
  // set-up of the allocation-free entry point on this device
  return noalloc_prepare_current_device();
}

int bri_get_links(bri_ctx* c, double* W) {
  if (!c || !W) {
    set_error("bri_get_links: null argument");
    return BRI_ERR_INVALID;
  }
  if (!c->have_links) {
    set_error("bri_get_links: call bri_build_links first");
    return BRI_ERR_NOLINKS;
  }
  return launch_export_links(c, W);
}

static int check_apply(bri_ctx* c, void* y, const void* x, int nrhs, int prec, const char* who,
                       bool allow_dw = false) {
  if (!c || !y || !x) {
    set_error(std::string(who) + ": null argument");
    return BRI_ERR_INVALID;
  }
  if (!c->have_links) {
    set_error(std::string(who) + ": call bri_build_links first");
    return BRI_ERR_NOLINKS;
  }
  if (nrhs < 1 || nrhs > 65535) {
    set_error(std::string(who) + ": nrhs must be in [1, 65535]");
    return BRI_ERR_INVALID;
  }
  if (prec != BRI_PREC_F64 && prec != BRI_PREC_F32 && prec != BRI_PREC_F32_BF16 &&
      !(allow_dw && prec == BRI_PREC_DW)) {
    set_error(std::string(who) + ": unknown precision");
    return BRI_ERR_INVALID;
  }
  if (y == x) {
    set_error(std::string(who) + ": x and y must not alias");
    return BRI_ERR_INVALID;
  }
  if (((uintptr_t)x | (uintptr_t)y) & 15) {
    set_error(std::string(who) + ": spinor pointers must be 16-byte aligned");
    return BRI_ERR_INVALID;
  }
  return BRI_OK;
}

int bri_apply(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec) {
  int rc = check_apply(c, y, x, nrhs, prec, "bri_apply", true);
  if (rc) return rc;
  if (prec != BRI_PREC_DW) return dirac_bri(c, y, x, nrhs, m0, dagger ? 1 : 0, prec, c->stream);
  void* tmp = nullptr;
  const size_t bytes = sizeof(float4) * 2 * (size_t)c->g.V * 12 * nrhs;
  cudaError_t e = cudaMallocAsync(&tmp, bytes, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("bri_apply: cudaMallocAsync failed: ") + cudaGetErrorString(e));
    return BRI_ERR_OOM;
  }
  note_device_alloc();
  rc = dirac_bri_dw64(c, (double*)y, (const double*)x, nrhs, m0, dagger ? 1 : 0, tmp, c->stream);
  cudaFreeAsync(tmp, c->stream);
  return rc;
}

int wils_apply(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec) {
  int rc = check_apply(c, y, x, nrhs, prec, "wils_apply");
  if (rc) return rc;
  return dirac_wil(c, y, x, nrhs, m0, dagger ? 1 : 0, prec, c->stream);
}

int kl_coeffs(int n, int kind, double scale, double* c0, double* w, double* sigma) {
  return kl_host(n, kind, scale, c0, w, sigma);
}

static int check_solver(bri_ctx* c, void* y, const void* x, int nrhs, int n, double rho, double tol, int prec,
                        const char* who) {
  int rc = check_apply(c, y, x, nrhs, prec, who);
  if (rc) return rc;
  if (n < 1 || n > BRI_MAX_SHIFTS) {
    set_error(std::string(who) + ": KL order n must be in [1, 32]");
    return BRI_ERR_INVALID;
  }
  if (!(rho > 0.0 && rho < 2.0)) {
    set_error(std::string(who) + ": rho must be in (0, 2)");
    return BRI_ERR_INVALID;
  }
  if (!(tol > 0.0 && tol < 1.0)) {
    set_error(std::string(who) + ": tol must be in (0, 1)");
    return BRI_ERR_INVALID;
  }
  return BRI_OK;
}

int sign_apply_multishift(bri_ctx* c, void* y, const void* x, int nrhs, int n, int kind, double rho, double scale,
                          double tol, int prec, bri_stats* st) {
  int rc = check_solver(c, y, x, nrhs, n, rho, tol, prec, "sign_apply_multishift");
  if (rc) return rc;
  return sign_apply(c, (double2*)y, (const double2*)x, nrhs, n, kind, rho, scale, tol, prec, 1.0, 0.0, st);
}

int overlap_apply(bri_ctx* c, void* y, const void* x, int nrhs, int n, int kind, double rho, double am,
                  double scale, double tol, int prec, bri_stats* st) {
  int rc = check_solver(c, y, x, nrhs, n, rho, tol, prec, "overlap_apply");
  if (rc) return rc;
  if (!std::isfinite(am) || am >= 2.0 * rho) {
    set_error("overlap_apply: the traditional massive form needs am < 2 rho");
    return BRI_ERR_INVALID;
  }
  // (1 - am/(2 rho)) rho (x + s) + am x
  const double k = (1.0 - am / (2.0 * rho)) * rho;
  return sign_apply(c, (double2*)y, (const double2*)x, nrhs, n, kind, rho, scale, tol, prec, k, k + am, st);
}

int overlap_grad(bri_ctx* c, void* g_psi, void* g_U, const void* eta, const void* psi, int nrhs, int n, int kind,
                 double rho, double am, double scale, double tol, int prec, bri_stats* st) {
  int rc = check_solver(c, g_psi, psi, nrhs, n, rho, tol, prec, "overlap_grad");
  if (rc) return rc;
  if (!g_U || !eta || eta == g_psi || ((uintptr_t)eta & 15) || ((uintptr_t)g_U & 15)) {
    set_error("overlap_grad: null, aliased or misaligned eta / g_U");
    return BRI_ERR_INVALID;
  }
  if (!std::isfinite(am) || am >= 2.0 * rho) {
    set_error("overlap_grad: the traditional massive form needs am < 2 rho");
    return BRI_ERR_INVALID;
  }
  return overlap_grad_impl(c, (double*)g_psi, (double*)g_U, (const double*)eta, (const double*)psi, nrhs, n, kind,
                           rho, am, scale, tol, prec, st);
}

int overlap_solve(bri_ctx* c, void* x, const void* b, int nrhs, int n_outer, int n_inner, int kind, double rho,
                  double am, int complete, double tol, int prec, bri_stats* st) {
  int rc = check_solver(c, x, b, nrhs, n_outer, rho, tol, prec, "overlap_solve");
  if (rc) return rc;
  if (n_inner < 0 || n_inner > BRI_MAX_SHIFTS || !std::isfinite(am) || am < 0.0 || am >= 2.0 * rho) {
    set_error("overlap_solve: need 0 <= n_inner <= 32 and 0 <= am < 2 rho");
    return BRI_ERR_INVALID;
  }
  const int64_t nc = c->g.V * 12;
  const int maxiter = (st && st->maxiter > 0) ? st->maxiter : 1000;
  int worst = BRI_OK;
  bri_stats acc;
  memset(&acc, 0, sizeof(acc));
  for (int r = 0; r < nrhs; ++r) {
    bri_stats one;
    memset(&one, 0, sizeof(one));
    rc = overlap_solve_impl(c, (double2*)x + r * nc, (const double2*)b + r * nc, n_outer, n_inner, kind, rho, am,
                            complete, tol, prec, maxiter, &one);
    if (rc < 0) return rc;
    worst = std::max(worst, rc);
    acc.iterations = std::max(acc.iterations, one.iterations);
    acc.refinements += one.refinements;
    acc.matvecs += one.matvecs;
    acc.max_true_residual = std::max(acc.max_true_residual, one.max_true_residual);
  }
  if (st) {
    const int want = st->want_true_residual, mi = st->maxiter;
    *st = acc;
    st->n_shifts = n_outer;
    st->want_true_residual = want;
    st->maxiter = mi;
  }
  return worst;
}

int overlap_apply_batch(bri_ctx* const* ctxs, int nctx, void* const* ys, const void* const* xs, const int* nrhs,
                        int n, int kind, double rho, double am, double scale, double tol, int prec, bri_stats* st) {
  if (!ctxs || !ys || !xs || !nrhs || nctx < 1 || nctx > 256) {
    set_error("overlap_apply_batch: need 1 <= nctx <= 256 and non-null arrays");
    return BRI_ERR_INVALID;
  }
  for (int i = 0; i < nctx; ++i) {
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) {
        set_error("overlap_apply_batch: a context appears twice");
        return BRI_ERR_INVALID;
      }
    int rc = check_solver(ctxs[i], ys[i], xs[i], nrhs[i], n, rho, tol, prec, "overlap_apply_batch");
    if (rc) return rc;
  }
  if (!std::isfinite(am) || am >= 2.0 * rho) {
    set_error("overlap_apply_batch: the traditional massive form needs am < 2 rho");
    return BRI_ERR_INVALID;
  }
  // autotune every lattice's stencil launches (used by the per-lattice
  // refinement) first, one lattice at a time
  for (int i = 0; i < nctx; ++i) {
    int rc = pretune_stencils(ctxs[i], prec);
    if (rc) return rc;
  }
  const double k = (1.0 - am / (2.0 * rho)) * rho;
  return batch_sign_apply(ctxs, nctx, ys, xs, nrhs, n, kind, rho, scale, tol, prec, k, k + am, st);
}

int bri_profile_enable(bri_ctx* c, int enable) {
  if (!c) {
    set_error("bri_profile_enable: null context");
    return BRI_ERR_INVALID;
  }
  c->prof_on = enable != 0;
  return BRI_OK;
}

int bri_profile_read(bri_ctx* c, int op, int prec, long long* launches, double* ms, double* site_rhs) {
  if (!c || op < 0 || op > 1 || prec < 0 || prec > 2 || !launches || !ms || !site_rhs) {
    set_error("bri_profile_read: bad argument");
    return BRI_ERR_INVALID;
  }
  int rc = prof_collect(c);
  if (rc) return rc;
  *launches = c->prof_launches[op][prec];
  *ms = c->prof_ms[op][prec];
  *site_rhs = c->prof_units[op][prec];
  c->prof_launches[op][prec] = 0;
  c->prof_ms[op][prec] = 0.0;
  c->prof_units[op][prec] = 0.0;
  return BRI_OK;
}

long long bri_kernel_launches(void) { return g_launches.load(); }

long long bri_device_allocations(void) { return g_dev_allocs.load(); }

}  // extern "C"
