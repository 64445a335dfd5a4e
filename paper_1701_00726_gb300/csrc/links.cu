// Link preparation (once per gauge configuration):
//  * thin links with the time boundary applied, structure-of-arrays;
//  * the 80 path-averaged off-axis transporters W_d(n) (App. C: average over
//    the k! shortest paths, no SU(3) back-projection), built level by level
//    with the last-step recursion
//        W_d(n) = (1/k) sum_{mu: d_mu != 0} W_{d - s_mu e_mu}(n) U_step(n + d - s_mu e_mu, mu, s_mu)
//    which groups the k! paths by their final hop; 40 of them are kept
//    (nu = 1..40; W_{82-nu}(n) = W_nu(n + d)^dagger) in FP64, FP32 and BF16;
//  * the clover term -(c_SW/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu} (Eq. def_bril)
//    in the chiral basis, two Hermitian 6x6 blocks per site.
#include "internal.cuh"
#include "cplx.cuh"

namespace bri {
namespace {

struct SiteCoord {
  int c[4];
};

__device__ __forceinline__ SiteCoord coords(const Geom& g, int64_t n) {
  SiteCoord s;
  int64_t r = n;
  s.c[0] = (int)(r % g.L[0]); r /= g.L[0];
  s.c[1] = (int)(r % g.L[1]); r /= g.L[1];
  s.c[2] = (int)(r % g.L[2]); r /= g.L[2];
  s.c[3] = (int)r;
  return s;
}

__device__ __forceinline__ int64_t site_of(const Geom& g, const int c[4]) {
  int64_t n = 0;
#pragma unroll
  for (int mu = 3; mu >= 0; --mu) {
    int v = c[mu] % g.L[mu];
    if (v < 0) v += g.L[mu];
    n = n * g.L[mu] + v;
  }
  return n;
}

__device__ __forceinline__ int64_t displaced(const Geom& g, const SiteCoord& s, int dx, int dy, int dz, int dt) {
  int c[4] = {s.c[0] + dx, s.c[1] + dy, s.c[2] + dz, s.c[3] + dt};
  return site_of(g, c);
}

__device__ __forceinline__ M3<double> load_soa(const double2* base, int64_t V, int64_t n) {
  M3<double> m;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.m[e / 3][e % 3] = ld2(base + (int64_t)e * V + n);
  return m;
}

__device__ __forceinline__ void store_soa(double2* base, int64_t V, int64_t n, const M3<double>& m) {
#pragma unroll
  for (int e = 0; e < 9; ++e) base[(int64_t)e * V + n] = make_double2(m.m[e / 3][e % 3].re, m.m[e / 3][e % 3].im);
}

// AoS caller layout [V][4][3][3] complex128 -> SoA [4][9][V] FP64 and FP32,
// with the antiperiodic sign on U_t of the last time slice.
__global__ void thin_links_kernel(Geom g, const double2* __restrict__ U, double2* U64, float2* U32, int anti) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  int t = (int)(n / g.str[3]);
  for (int mu = 0; mu < 4; ++mu) {
    double sgn = (anti && mu == 3 && t == g.L[3] - 1) ? -1.0 : 1.0;
    for (int e = 0; e < 9; ++e) {
      double2 v = U[(n * 4 + mu) * 9 + e];
      v.x *= sgn;
      v.y *= sgn;
      U64[((int64_t)mu * 9 + e) * g.V + n] = v;
      U32[((int64_t)mu * 9 + e) * g.V + n] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__device__ __forceinline__ int nu_of(int dx, int dy, int dz, int dt) {
  return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1) + 27 * (dt + 1);
}

// One-hop transporters: W_{+mu}(n) = U_mu(n), W_{-mu}(n) = U_mu(n - mu)^dagger.
__global__ void level1_kernel(Geom g, const double2* __restrict__ U64, double2* T) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  SiteCoord s = coords(g, n);
  for (int mu = 0; mu < 4; ++mu) {
    int e[4] = {0, 0, 0, 0};
    e[mu] = 1;
    M3<double> fwd = load_soa(U64 + (int64_t)mu * 9 * g.V, g.V, n);
    int64_t nb = displaced(g, s, -e[0], -e[1], -e[2], -e[3]);
    M3<double> bwd = adj(load_soa(U64 + (int64_t)mu * 9 * g.V, g.V, nb));
    store_soa(T + (int64_t)nu_of(e[0], e[1], e[2], e[3]) * 9 * g.V, g.V, n, fwd);
    store_soa(T + (int64_t)nu_of(-e[0], -e[1], -e[2], -e[3]) * 9 * g.V, g.V, n, bwd);
  }
}

}  // namespace

LevelList level_list(int k) {
  LevelList lst;
  lst.count = 0;
  for (int nu = 0; nu < 81; ++nu) {
    int d[4] = {nu % 3 - 1, (nu / 3) % 3 - 1, (nu / 9) % 3 - 1, (nu / 27) % 3 - 1};
    int h = (d[0] != 0) + (d[1] != 0) + (d[2] != 0) + (d[3] != 0);
    if (h == k) lst.nu[lst.count++] = nu;
  }
  return lst;
}

namespace {

// k-hop transporters from (k-1)-hop ones at the same site (last-step recursion).
__global__ void levelk_kernel(Geom g, const double2* __restrict__ U64, double2* T, LevelList lst, int k) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int which = blockIdx.y;
  if (n >= g.V || which >= lst.count) return;
  int nu = lst.nu[which];
  int d[4] = {nu % 3 - 1, (nu / 3) % 3 - 1, (nu / 9) % 3 - 1, (nu / 27) % 3 - 1};
  SiteCoord s = coords(g, n);
  M3<double> acc;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc.m[i][j] = C<double>{0.0, 0.0};
  for (int mu = 0; mu < 4; ++mu) {
    if (d[mu] == 0) continue;
    int sg = d[mu];
    int dp[4] = {d[0], d[1], d[2], d[3]};
    dp[mu] -= sg;  // d' = d - s e_mu
    M3<double> wprev = load_soa(T + (int64_t)nu_of(dp[0], dp[1], dp[2], dp[3]) * 9 * g.V, g.V, n);
    M3<double> step;
    if (sg > 0) {  // U_mu(n + d')
      int64_t m = displaced(g, s, dp[0], dp[1], dp[2], dp[3]);
      step = load_soa(U64 + (int64_t)mu * 9 * g.V, g.V, m);
    } else {       // U_mu(n + d' - mu)^dagger
      int q[4] = {dp[0], dp[1], dp[2], dp[3]};
      q[mu] -= 1;
      int64_t m = displaced(g, s, q[0], q[1], q[2], q[3]);
      step = adj(load_soa(U64 + (int64_t)mu * 9 * g.V, g.V, m));
    }
    madd(acc, mmul(wprev, step));
  }
  double inv = 1.0 / k;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc.m[i][j] = inv * acc.m[i][j];
  store_soa(T + (int64_t)nu * 9 * g.V, g.V, n, acc);
}

// FP32 copy in the paired layout [40][5][V] float4 (elements 2k, 2k+1 of one
// site in one 16-byte word); BF16 copy in the FP64 layout [40][9][V].
__global__ void narrow_links_kernel(int64_t count, const double2* __restrict__ W64, float2* W32,
                                    __nv_bfloat162* W16, int64_t V) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 v = W64[i];
  const int64_t nu9e = i / V, n = i - nu9e * V, nu = nu9e / 9, e = nu9e - nu * 9;
  W32[((nu * 5 + e / 2) * V + n) * 2 + (e & 1)] = make_float2((float)v.x, (float)v.y);
  W16[i] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

// ------------------------------------------------------------------ clover
__device__ __forceinline__ M3<double> linkU(const Geom& g, const double2* U64, const SiteCoord& s, int mu,
                                            int dx, int dy, int dz, int dt) {
  int64_t m = displaced(g, s, dx, dy, dz, dt);
  return load_soa(U64 + (int64_t)mu * 9 * g.V, g.V, m);
}

// F_{mu nu}(n): traceless part of (Q - Q^dagger)/(8i), Q the sum of the four
// counter-clockwise plaquette leaves around n in the (mu, nu) plane.
__device__ M3<double> field_strength(const Geom& g, const double2* U64, const SiteCoord& s, int mu, int nu) {
  int em[4] = {0, 0, 0, 0}, en[4] = {0, 0, 0, 0};
  em[mu] = 1;
  en[nu] = 1;
#define SH(a, b) (a * em[0] + b * en[0]), (a * em[1] + b * en[1]), (a * em[2] + b * en[2]), (a * em[3] + b * en[3])
  M3<double> q;
  // l1 = U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
  q = mmul(mmul(linkU(g, U64, s, mu, SH(0, 0)), linkU(g, U64, s, nu, SH(1, 0))),
           mmul(adj(linkU(g, U64, s, mu, SH(0, 1))), adj(linkU(g, U64, s, nu, SH(0, 0)))));
  // l2 = U_nu(n) U_mu(n+nu-mu)^+ U_nu(n-mu)^+ U_mu(n-mu)
  madd(q, mmul(mmul(linkU(g, U64, s, nu, SH(0, 0)), adj(linkU(g, U64, s, mu, SH(-1, 1)))),
               mmul(adj(linkU(g, U64, s, nu, SH(-1, 0))), linkU(g, U64, s, mu, SH(-1, 0)))));
  // l3 = U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu) U_nu(n-nu)
  madd(q, mmul(mmul(adj(linkU(g, U64, s, mu, SH(-1, 0))), adj(linkU(g, U64, s, nu, SH(-1, -1)))),
               mmul(linkU(g, U64, s, mu, SH(-1, -1)), linkU(g, U64, s, nu, SH(0, -1)))));
  // l4 = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu) U_mu(n)^+
  madd(q, mmul(mmul(adj(linkU(g, U64, s, nu, SH(0, -1))), linkU(g, U64, s, mu, SH(0, -1))),
               mmul(linkU(g, U64, s, nu, SH(1, -1)), adj(linkU(g, U64, s, mu, SH(0, 0))))));
#undef SH
  M3<double> f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // (Q - Q^+)_{ij} / (8i) = -i (Q_ij - conj(Q_ji)) / 8
      C<double> a = q.m[i][j] - conj(q.m[j][i]);
      f.m[i][j] = C<double>{a.im / 8.0, -a.re / 8.0};
    }
  C<double> tr = f.m[0][0] + f.m[1][1] + f.m[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) f.m[i][i] = f.m[i][i] - (1.0 / 3.0) * tr;
  return f;
}

// Chiral basis: sigma_{jk} = -eps_{jkl} diag(s_l, s_l), sigma_{j4} = diag(s_j, -s_j)
// (s = Pauli, sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]).  Hence the upper
// (lower) 6x6 block of sum_{mu<nu} sigma_{mu nu} F_{mu nu} is sum_l s_l (x) X_l with
//   X_1 = -F_23 +- F_14,  X_2 = F_13 +- F_24,  X_3 = -F_12 +- F_34.
__global__ void clover_kernel(Geom g, const double2* __restrict__ U64, double c_sw, double* C64, float* C32) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  SiteCoord s = coords(g, n);
  M3<double> F12 = field_strength(g, U64, s, 0, 1), F13 = field_strength(g, U64, s, 0, 2);
  M3<double> F14 = field_strength(g, U64, s, 0, 3), F23 = field_strength(g, U64, s, 1, 2);
  M3<double> F24 = field_strength(g, U64, s, 1, 3), F34 = field_strength(g, U64, s, 2, 3);
  const double pre = -0.5 * c_sw;
  for (int blk = 0; blk < 2; ++blk) {
    const double sg = blk == 0 ? 1.0 : -1.0;
    C<double> full[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        C<double> x1, x2, x3;
        x1 = C<double>{-F23.m[a][b].re + sg * F14.m[a][b].re, -F23.m[a][b].im + sg * F14.m[a][b].im};
        x2 = C<double>{F13.m[a][b].re + sg * F24.m[a][b].re, F13.m[a][b].im + sg * F24.m[a][b].im};
        x3 = C<double>{-F12.m[a][b].re + sg * F34.m[a][b].re, -F12.m[a][b].im + sg * F34.m[a][b].im};
        // s_1 X_1 + s_2 X_2 + s_3 X_3 = [[X3, X1 - i X2], [X1 + i X2, -X3]]
        C<double> m01 = C<double>{x1.re + x2.im, x1.im - x2.re};
        C<double> m10 = C<double>{x1.re - x2.im, x1.im + x2.re};
        full[0 * 3 + a][0 * 3 + b] = pre * x3;
        full[1 * 3 + a][1 * 3 + b] = (-pre) * x3;
        full[0 * 3 + a][1 * 3 + b] = pre * m01;
        full[1 * 3 + a][0 * 3 + b] = pre * m10;
      }
    int64_t base = (int64_t)blk * 36;
    for (int i = 0; i < 6; ++i) {
      C64[(base + i) * g.V + n] = full[i][i].re;
      C32[(base + i) * g.V + n] = (float)full[i][i].re;
    }
    int k = 6;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        C64[(base + k) * g.V + n] = full[i][j].re;
        C64[(base + k + 1) * g.V + n] = full[i][j].im;
        C32[(base + k) * g.V + n] = (float)full[i][j].re;
        C32[(base + k + 1) * g.V + n] = (float)full[i][j].im;
        k += 2;
      }
  }
}

__global__ void export_links_kernel(Geom g, const double2* __restrict__ W64, double2* out) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  for (int nu = 0; nu < 40; ++nu)
    for (int e = 0; e < 9; ++e) out[(n * 40 + nu) * 9 + e] = W64[((int64_t)nu * 9 + e) * g.V + n];
}

}  // namespace

int build_transporters(bri_ctx* c, double2* T) {
  const Geom& g = c->g;
  const int64_t V = g.V;
  cudaStream_t st = c->stream;
  const int th = 128;
  level1_kernel<<<blocks_for(V, th), th, 0, st>>>(g, c->U64, T); note_launch();
  for (int k = 2; k <= 4; ++k) {
    LevelList lst = level_list(k);
    dim3 grid(blocks_for(V, th), lst.count);
    levelk_kernel<<<grid, th, 0, st>>>(g, c->U64, T, lst, k); note_launch();
  }
  BRI_LAUNCH_CHECK("link construction kernels");
  return BRI_OK;
}

int launch_build_links(bri_ctx* c, const double* U, double c_sw) {
  const Geom& g = c->g;
  const int64_t V = g.V;
  cudaStream_t st = c->stream;
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (*p) return BRI_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
      return BRI_ERR_OOM;
    }
    note_device_alloc();
    return BRI_OK;
  };
  int rc;
  if ((rc = alloc((void**)&c->W64, sizeof(double2) * 360 * V))) return rc;
  if ((rc = alloc((void**)&c->W32, sizeof(float2) * 400 * V))) return rc;
  if ((rc = alloc((void**)&c->W16, sizeof(__nv_bfloat162) * 360 * V))) return rc;
  if ((rc = alloc((void**)&c->U64, sizeof(double2) * 36 * V))) return rc;
  if ((rc = alloc((void**)&c->U32, sizeof(float2) * 36 * V))) return rc;
  double2* T = nullptr;
  if ((rc = alloc((void**)&T, sizeof(double2) * 81 * 9 * V))) return rc;

  const int th = 128;
  thin_links_kernel<<<blocks_for(V, th), th, 0, st>>>(g, (const double2*)U, c->U64, c->U32,
                                                       (c->flags & BRI_ANTIPERIODIC_T) ? 1 : 0); note_launch();
  if ((rc = build_transporters(c, T))) return rc;
  BRI_CUDA(cudaMemcpyAsync(c->W64, T, sizeof(double2) * 360 * V, cudaMemcpyDeviceToDevice, st));
  narrow_links_kernel<<<blocks_for(360 * V, 256), 256, 0, st>>>(360 * V, c->W64, c->W32, c->W16, V); note_launch();
  BRI_LAUNCH_CHECK("narrow_links_kernel");
  c->have_clover = false;
  c->dw_valid = false;
  c->c_sw = c_sw;
  if (c_sw != 0.0) {
    if ((rc = alloc((void**)&c->C64, sizeof(double) * 72 * V))) return rc;
    if ((rc = alloc((void**)&c->C32, sizeof(float) * 72 * V))) return rc;
    clover_kernel<<<blocks_for(V, 64), 64, 0, st>>>(g, c->U64, c_sw, c->C64, c->C32); note_launch();
    BRI_LAUNCH_CHECK("clover_kernel");
    c->have_clover = true;
  }
  BRI_CUDA(cudaStreamSynchronize(st));
  BRI_CUDA(cudaFree(T));
  c->have_links = true;
  return BRI_OK;
}

int launch_export_links(bri_ctx* c, double* W) {
  export_links_kernel<<<blocks_for(c->g.V, 128), 128, 0, c->stream>>>(c->g, c->W64, (double2*)W); note_launch();
  BRI_LAUNCH_CHECK("export_links_kernel");
  return BRI_OK;
}

}  // namespace bri
