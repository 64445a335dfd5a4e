// Internal declarations shared by the CUDA translation units of libbri.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <cstring>
#include <functional>
#include <string>

#include "../../include/bri.h"

namespace bri {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define BRI_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::bri::cuda_fail(e_, #call); \
  } while (0)

#define BRI_LAUNCH_CHECK(where)                          \
  do {                                                   \
    cudaError_t e_ = cudaGetLastError();                 \
    if (e_ != cudaSuccess) return ::bri::cuda_fail(e_, where); \
  } while (0)

// ---------------------------------------------------------------- geometry
struct Geom {
  int L[4];      // Lx, Ly, Lz, Lt
  int64_t V;     // volume
  int64_t str[4];// site strides 1, Lx, Lx*Ly, Lx*Ly*Lz
};

// ---------------------------------------------------------------- context
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Event-bracketed stencil launches (profiling), per operator x precision.
struct ProfRec {
  cudaEvent_t a, b;
  int op, prec;
  double units;
};

void note_launch();
void note_launches(long long n);
// CUDA-graph replay of solver iterations (BRI_GRAPHS=0 disables it).
int graphs_enabled();

}  // namespace bri

#include <vector>

struct bri_ctx {
  bri::Geom g;
  int flags = 0;
  cudaStream_t stream = nullptr;
  bool have_links = false;
  bool have_clover = false;
  double c_sw = 0.0;
  // kernel operator of the overlap solvers: BRI_KERNEL_BRILLOUIN or BRI_KERNEL_WILSON
  int kernel = BRI_KERNEL_BRILLOUIN;
  // Stored off-axis links, structure-of-arrays: FP64 and BF16 [40][9][V]
  // complex, element (nu, e, n) at (nu*9 + e)*V + n; FP32 [40][5][V] pairs of
  // complex (elements 2k, 2k+1 in one 16-byte word, tenth slot padding).  A
  // warp of consecutive sites reads one contiguous segment per load.
  double2* W64 = nullptr;
  float2* W32 = nullptr;
  __nv_bfloat162* W16 = nullptr;
  // Thin links with the time boundary applied, [4][9][V] (Wilson kernel).
  double2* U64 = nullptr;
  float2* U32 = nullptr;
  // Clover: two Hermitian 6x6 chiral blocks per site, packed as 72 reals:
  // [block][36][V]: 6 diagonal reals, then 15 upper off-diagonal complex.
  double* C64 = nullptr;
  float* C32 = nullptr;
  // Double-word FP32 copies (h, l) of W64 and C64 for the FP64-class stencil
  // on the FP32 pipe: [40][9][V] float4 and [2][36][V] float2, made on first
  // use after each bri_build_links (dw_valid).
  void* Wdw = nullptr;
  void* Cdw = nullptr;
  bool dw_valid = false;
  // solver workspace (grown on demand)
  bri::Workspace ws;
  bri::Workspace ws_small;
  void* host_pinned = nullptr;
  // library-owned stream the solvers run on (capture-capable, concurrent
  // across contexts), fenced against the caller's stream with two events
  cudaStream_t own_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // profiling of stencil launches
  bool prof_on = false;
  std::vector<bri::ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  long long prof_launches[2][3] = {{0, 0, 0}, {0, 0, 0}};
  double prof_ms[2][3] = {{0, 0, 0}, {0, 0, 0}};
  double prof_units[2][3] = {{0, 0, 0}, {0, 0, 0}};
};

namespace bri {

// ---------------------------------------------------------------- kernels (host launchers)
// Offsets (nu - 1) with exactly k nonzero components.
struct LevelList {
  int count;
  int nu[32];
};
LevelList level_list(int k);
int launch_build_links(bri_ctx* c, const double* U, double c_sw);
// All 81 path-averaged transporters [81][9][V] (FP64) from the thin links of the context.
int build_transporters(bri_ctx* c, double2* T);
int launch_export_links(bri_ctx* c, double* W);

// spinor precision dispatch for the stencils
int dirac_bri(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec,
              cudaStream_t s);
int dirac_wil(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec,
              cudaStream_t s);
// The solver's fused D^dagger application: y = D^dagger x + sigma_s p_s and the
// Double-word FP32 Brillouin stencil (bri_dw.cu): y = D x or D^dagger x on
// double-word vectors ([nrhs][V][12] float4), FP64 in and out through the
// split/join kernels (tmp: two double-word vectors of nrhs right-hand sides),
// and the normal operator D^dagger D on FP64 vectors (t1, t2 double-word
// scratch; t2 may be out).
int ensure_dw_links(bri_ctx* c);
int dirac_bri_dw(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, cudaStream_t s);
int dirac_bri_dw64(bri_ctx* c, double* y, const double* x, int nrhs, double m0, int dagger, void* tmp,
                   cudaStream_t s);
int normal_op_dw(bri_ctx* c, double* out, const double* x, int nrhs, double m0, void* t1, void* t2, cudaStream_t s);
// per-site-block partials of Re<p_s, y> (Brillouin kernel only); sd_blocks
// receives the number of partials per system (part: [nrhs][sd_blocks]).
int dirac_bri_shiftdot(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int prec, cudaStream_t s,
                       const void* p, const double* sig, double* part, int* sd_blocks);
// The overlap's kernel operator selected on the context (bri_set_kernel):
// the Brillouin stencil (Eq. def_bril) or the Wilson stencil (Eq. def_wils).
int dirac_kernel(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, int prec,
                 cudaStream_t s);
// Makes the stencil autotuner's choices for this lattice (every rhs class and
// precision a solve of precision prec uses) before concurrent work starts.
int pretune_stencils(bri_ctx* c, int prec);

// Device scratch from a caller-provided block (used by the entry point that
// allocates nothing); when no arena is set the solvers allocate from the
// stream-ordered pool.  Thread-local, so concurrent host threads do not mix.
struct ScratchArena {
  char* base;
  size_t cap;
  size_t used;
};
void set_current_arena(ScratchArena* a);
ScratchArena* current_arena();
// Device address of the allocation-free entry point's static scratch array,
// looked up once per device (with that device current) at set-up time.
int noalloc_prepare_current_device();
// Process-wide count of device allocations the library has made (solver
// workspaces, link and clover storage).
void note_device_alloc();

// host-side KL coefficients
int kl_host(int n, int kind, double scale, double* c0, double* w, double* sigma);

// A gamma5-hermitian operator in place of the context's kernel for the FP64
// solvers (the nested Kenney-Laub iterates of Sec. 4.1 solve on Y^dagger Y with
// Y itself an overlap-type operator): y = K x (dagger = 0) or K^dagger x for
// nsys systems of V*12 complex128 each, on the context stream.
struct KernelOp {
  std::function<int(double2* y, const double2* x, int nsys, int dagger)> apply;
};

// solvers
struct Counters {
  int matvecs = 0, matvecs64 = 0;
};
struct SolveInfo {
  Counters cnt;
  int iters = 0, refinements = 0;
  double tph[4] = {0, 0, 0, 0};
};
// (A + sigma_k) X_k = b_s for all shifts k < n, systems s < nsys: X = [n][nsys][V*24] FP64.
int solve_shifts(bri_ctx* c, const double* b, int nsys, int n, const double* sig, double m0, double tol, int prec,
                 int maxiter, double* X, SolveInfo& info, const KernelOp* op = nullptr);
int overlap_grad_impl(bri_ctx* c, double* g_psi, double* g_U, const double* eta, const double* psi, int nrhs, int n,
                      int kind, double rho, double am, double scale, double tol, int prec, bri_stats* stats);
int overlap_solve_impl(bri_ctx* c, double2* x, const double2* b, int n_outer, int n_inner, int kind, double rho,
                       double am, int complete, double tol, int prec, int maxiter, bri_stats* st_out);
// Batched lattices (overlap_apply_batch): phase 1 on one system table with a
// work-list stencil and a WHILE-node graph, then per-lattice refinement.
int batch_sign_apply(bri_ctx* const* cs, int nctx, void* const* ys, const void* const* xs, const int* nrhs, int n,
                     int kind, double rho, double scale, double tol, int prec, double out_scale, double b_coeff,
                     bri_stats* stats);
int sign_apply(bri_ctx* c, double2* y, const double2* x, int nrhs, int n, int kind, double rho,
               double scale, double tol, int prec, double out_scale, double b_coeff,
               bri_stats* st, const KernelOp* op = nullptr);

// profiling brackets (no-ops unless enabled on the context)
int prof_begin(bri_ctx* c, cudaStream_t s, cudaEvent_t* a);
int prof_end(bri_ctx* c, cudaStream_t s, cudaEvent_t a, int op, int prec, double units);

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace bri
