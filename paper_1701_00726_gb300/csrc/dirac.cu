// Stencil dispatch by precision, with optional event brackets (profiling).
#include "stencil.cuh"

#include <map>
#include <mutex>
#include <string>

#include <cstdlib>

namespace bri {

int autotune_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("BRI_AUTOTUNE");
    v = e ? (atoi(e) != 0) : 1;
  }
  return v;
}

static std::mutex g_tune_mu;
static std::map<std::string, StencilConfig> g_tune;

bool tune_lookup(const char* key, StencilConfig* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const char* key, const StencilConfig& cf) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = cf;
}

// D^dagger x + sigma_s p with the per-block partials of Re<p_s, .> (the fused
// solver epilogue, Brillouin kernel): sd_blocks receives the number of
// partials per system.
int dirac_bri_shiftdot(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int prec, cudaStream_t s,
                       const void* p, const double* sig, double* part, int* sd_blocks) {
  const double diag = 15.0 / 8.0 + m0;
  cudaEvent_t ev;
  int rc = prof_begin(c, s, &ev);
  if (rc) return rc;
  switch (prec) {
    case BRI_PREC_F64: {
      const ShiftDot<double> sd{(const double*)p, sig, part};
      rc = launch_bri_t<double, double2>(c->g, (double*)y, (const double*)x, c->W64,
                                       c->have_clover ? c->C64 : nullptr, diag, nrhs, 1, s, &sd, sd_blocks);
      break;
    }
    case BRI_PREC_F32: {
      const ShiftDot<float> sd{(const float*)p, sig, part};
      rc = launch_bri_t<float, float2>(c->g, (float*)y, (const float*)x, c->W32,
                                     c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, 1, s, &sd, sd_blocks);
      break;
    }
    case BRI_PREC_F32_BF16: {
      const ShiftDot<float> sd{(const float*)p, sig, part};
      rc = launch_bri_t<float, __nv_bfloat162>(c->g, (float*)y, (const float*)x, c->W16,
                                             c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, 1, s, &sd,
                                             sd_blocks);
      break;
    }
    default:
      set_error("bri_apply: unknown precision");
      return BRI_ERR_INVALID;
  }
  if (rc) return rc;
  return prof_end(c, s, ev, 0, prec, (double)c->g.V * nrhs);
}

int dirac_kernel(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec, cudaStream_t s) {
  if (c->kernel == BRI_KERNEL_WILSON) return dirac_wil(c, y, x, nrhs, m0, dagger, prec, s);
  return dirac_bri(c, y, x, nrhs, m0, dagger, prec, s);
}

std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}

// Runs the stencil once for every right-hand-side class (1, 2-3, >= 4) and
// precision a solve of precision prec uses, so that the autotuner's choices
// for this lattice are made now, with nothing else on the GPU.
int pretune_stencils(bri_ctx* c, int prec) {
  if (!autotune_enabled() || !c->have_links) return BRI_OK;
  cudaStream_t s = c->stream;
  const int64_t nreal = c->g.V * 24;
  void* buf = nullptr;
  const size_t bytes = sizeof(double) * nreal * 4 * 2;
  cudaError_t e = cudaMallocAsync(&buf, bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "pretune: cudaMallocAsync");
  note_device_alloc();
  int rc = BRI_OK;
  if ((e = cudaMemsetAsync(buf, 0, bytes, s)) != cudaSuccess) rc = cuda_fail(e, "pretune: cudaMemsetAsync");
  int precs[3] = {BRI_PREC_F64, -1, -1};
  if (prec != BRI_PREC_F64) {
    precs[1] = BRI_PREC_F32;
    if (prec == BRI_PREC_F32_BF16) precs[2] = BRI_PREC_F32_BF16;
  }
  for (int pi = 0; pi < 3 && rc == BRI_OK; ++pi) {
    if (precs[pi] < 0) continue;
    const size_t half = precs[pi] == BRI_PREC_F64 ? sizeof(double) * nreal * 4 : sizeof(float) * nreal * 4;
    for (int nr : {1, 2, 4}) {
      rc = dirac_bri(c, (char*)buf + half, buf, nr, -1.0, 0, precs[pi], s);
      if (rc) break;
    }
  }
  cudaFreeAsync(buf, s);
  cudaGetLastError();
  return rc;
}

int pair_rhs_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("BRI_PAIR_RHS");
    v = e ? (atoi(e) != 0) : 1;
  }
  return v;
}

int dirac_bri(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec, cudaStream_t s) {
  const double diag = 15.0 / 8.0 + m0;
  cudaEvent_t ev;
  int rc = prof_begin(c, s, &ev);
  if (rc) return rc;
  switch (prec) {
    case BRI_PREC_F64:
      rc = launch_bri_t<double, double2>(c->g, (double*)y, (const double*)x, c->W64,
                                       c->have_clover ? c->C64 : nullptr, diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32:
      rc = launch_bri_t<float, float2>(c->g, (float*)y, (const float*)x, c->W32,
                                     c->have_clover ? c->C32 : nullptr, (float)diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32_BF16:
      rc = launch_bri_t<float, __nv_bfloat162>(c->g, (float*)y, (const float*)x, c->W16,
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
      rc = launch_wil_t<double, double2>(c->g, (double*)y, (const double*)x, c->U64,
                                       c->have_clover ? c->C64 : nullptr, diag, nrhs, dagger, s);
      break;
    case BRI_PREC_F32:
    case BRI_PREC_F32_BF16:
      rc = launch_wil_t<float, float2>(c->g, (float*)y, (const float*)x, c->U32,
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
