// Entry point that allocates no device memory: the FP64 sign-function solve
// with all of its solver workspace carved out of one file-scope device array.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating
// routine) at the point where they apply the operator -- for example an
// application whose device memory is entirely reserved up front by its own
// pool, or a latency-critical loop in which an implicitly synchronising
// allocation is not acceptable.  Those callers build the context (links) at
// set-up time and afterwards use this call, which only launches kernels and
// copies a few scalars.
//
// The array is a static __device__ object of this translation unit: every
// device on which the library is loaded holds it (32 MiB) until the process
// exits.  Host code must not use its name as a device address; the address is
// obtained with cudaGetSymbolAddress once per device, with that device
// current, when bri_build_links runs there (set-up time).  Under CUDA's lazy
// module loading that lookup is also the moment the array's memory is
// committed, so a caller whose memory is reserved by its own pool pays for it
// at set-up, not inside the allocation-free call.
#include "internal.cuh"

#include <mutex>
#include <string>

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Bytes the FP64 solve needs: the n solution vectors, the n shifted search
// directions and three work vectors per right-hand side (192 B per site each),
// plus per-system solver state, reduction partials (those of the stencil's
// fused epilogue: one per 64 sites) and alignment slack.
size_t noalloc_need(int64_t V, int nrhs, int n) {
  return size_t(192) * size_t(V) * size_t(nrhs) * size_t(2 * n + 3) + size_t(64) * 1024 + size_t(4096) * nrhs +
         size_t(8) * size_t(nrhs) * size_t((V + 63) / 64) + 512;
}

}  // namespace

namespace bri {

// Looks up (once per device, with that device current) the device address of
// the static scratch array.  Called from bri_build_links.
int noalloc_prepare_current_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc set-up: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("noalloc set-up: device ordinal out of range");
    return BRI_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_addr[dev]) return BRI_OK;
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc set-up: cudaGetSymbolAddress");
  g_scratch_addr[dev] = (char*)ptr;
  return BRI_OK;
}

}  // namespace bri

using namespace bri;

extern "C" int sign_apply_multishift_noalloc(bri_ctx* c, void* y, const void* x, int nrhs, int n, int kind,
                                             double rho, double scale, double tol, bri_stats* st) {
  if (!c || !y || !x) {
    set_error("sign_apply_multishift_noalloc: null argument");
    return BRI_ERR_INVALID;
  }
  if (!c->have_links) {
    set_error("sign_apply_multishift_noalloc: call bri_build_links first");
    return BRI_ERR_NOLINKS;
  }
  if (nrhs < 1 || n < 1 || n > BRI_MAX_SHIFTS || !(rho > 0.0 && rho < 2.0) || !(tol > 0.0 && tol < 1.0) || x == y ||
      (((uintptr_t)x | (uintptr_t)y) & 15)) {
    set_error("sign_apply_multishift_noalloc: invalid argument (nrhs >= 1, 1 <= n <= 32, 0 < rho < 2, "
              "0 < tol < 1, distinct 16-byte aligned x and y)");
    return BRI_ERR_INVALID;
  }
  const size_t need = noalloc_need(c->g.V, nrhs, n);
  if (need > kNoallocScratchBytes) {
    set_error("sign_apply_multishift_noalloc: V * nrhs * (2n + 3) * 192 bytes (" + std::to_string(need) +
              " with state) exceeds the 32 MiB static scratch; use sign_apply_multishift");
    return BRI_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "sign_apply_multishift_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sign_apply_multishift_noalloc: device ordinal out of range");
    return BRI_ERR_INVALID;
  }
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    base = g_scratch_addr[dev];
  }
  if (!base) {  // links built with another device current: set up this one now
    const int prc = noalloc_prepare_current_device();
    if (prc) return prc;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    base = g_scratch_addr[dev];
  }
  ScratchArena arena{base, kNoallocScratchBytes, 0};
  bri_stats local;
  if (st) local = *st;
  else memset(&local, 0, sizeof(local));
  local.want_true_residual = 0;  // the FP64 check would need extra vectors
  set_current_arena(&arena);
  int rc = sign_apply(c, (double2*)y, (const double2*)x, nrhs, n, kind, rho, scale, tol, BRI_PREC_F64, 1.0, 0.0,
                      &local);
  set_current_arena(nullptr);
  if (st) {
    const int want = st->want_true_residual;
    *st = local;
    st->want_true_residual = want;
  }
  return rc;
}
