// Adjoint of the overlap application: gradients of
//   L = sum_r Re <eta_r, D_m psi_r>,  D_m = (1 - am/(2 rho)) D_ov + am,
//   D_ov = rho (1 + D r(D^dagger D)),  r(s) = c0 + sum_i w_i/(s + sigma_i)
// with respect to the sources psi and the thin links U given to
// bri_build_links (real-gradient convention dL = Re<g, dpsi> and
// dL = Re sum tr(G^dagger dU)).  With k = (1 - am/(2 rho)) rho,
// x_i = (A + sigma_i)^{-1} psi, z_i = (A + sigma_i)^{-1} D^dagger eta and
// y = c0 psi + sum_i w_i x_i (both multi-shift solves share the shifts):
//   g_psi = D_m^dagger eta = k (eta + r(A) D^dagger eta) + am eta
//         = k (eta + c0 D^dagger eta + sum_i w_i z_i) + am eta   (z_i reused),
//   dL = k Re<eta, dD y> - k sum_i w_i (Re<D x_i, dD z_i> + Re<D z_i, dD x_i>).
// Each term Re<u, dD v> gives every transporter W_d(n) the gradient
// G_W = u(n) (M_d v(n+d))^dagger (kernel k_force); the gradients are then
// pushed back through the path average (App. C) by reversing the last-step
// recursion W_d = (1/k) sum_mu W_{d - s e_mu} U_step level by level, as
// gathers (no atomics).  With the Wilson kernel (Eq. def_wils) the transporters
// are the thin links themselves, so only the one-hop terms exist and the
// gradients go straight to the links.  The clover term adds, per site and
// plane, the gradient of its leaf sum (kernels k_clover_force, k_clover_links).
#include "hops.cuh"

#include <chrono>

namespace bri {
namespace {

struct PairList {
  const double* u[512];
  const double* v[512];
  double w[512];
};

// Stored offsets (0..39) a force launch covers: all 40 for the Brillouin
// kernel, the four one-hop ones for the Wilson kernel.
struct OffsetList {
  int count;
  int j[40];
};

// G_W[idx](n) += sum_p w_p u_p(n) (M_d v_p(n+d))^dagger for the hops d.
// blockIdx.y = entry of the offset list, blockIdx.z = 0 for +d, 1 for -d.
__global__ void __launch_bounds__(128) k_force(Geom g, const PairList* __restrict__ pl, int npair, double2* GW,
                                              const __grid_constant__ HopTable<double> H, OffsetList ol) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int j = ol.j[blockIdx.y], opp = blockIdx.z;
  int m = 0;
  {
    int r = n;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int L = g.L[mu];
      const int cmu = (mu < 3) ? r % L : r;
      if (mu < 3) r /= L;
      const int d = opp ? -H.site_d[j][mu] : H.site_d[j][mu];
      m += wrap(cmu + d, L) * (int)g.str[mu];
    }
  }
  const double a = H.a[j];
  const double sg = opp ? -1.0 : 1.0;
  const double c1 = sg * H.cs[j][0], c2 = sg * H.cs[j][1], c3 = sg * H.cs[j][2], c4 = sg * H.cs[j][3];
  C<double> G[3][3];
#pragma unroll
  for (int aa = 0; aa < 3; ++aa)
#pragma unroll
    for (int b = 0; b < 3; ++b) G[aa][b] = C<double>{0, 0};
  for (int p = 0; p < npair; ++p) {
    Spinor<double> us, vs, chi;
    load_spinor(us, pl->u[p] + (int64_t)n * 24);
    load_spinor(vs, pl->v[p] + (int64_t)m * 24);
    spin_combine(chi, vs, a, c1, c2, c3, c4);
    const double wp = pl->w[p];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        const C<double> ua{wp * us.v[s][aa].re, wp * us.v[s][aa].im};
#pragma unroll
        for (int b = 0; b < 3; ++b) cfma_cj(G[aa][b], chi.v[s][b], ua);  // u_a conj(chi_b)
      }
  }
  const int idx = opp ? 80 - j : j;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    double2* q = GW + ((int64_t)idx * 9 + e) * g.V + n;
    double2 v = *q;
    v.x += G[e / 3][e % 3].re;
    v.y += G[e / 3][e % 3].im;
    *q = v;
  }
}

__device__ __forceinline__ int site_shift(const Geom& g, int n, const int d[4]) {
  int r = n, m = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int cmu = (mu < 3) ? r % L : r;
    if (mu < 3) r /= L;
    int v = (cmu + d[mu]) % L;
    if (v < 0) v += L;
    m += v * (int)g.str[mu];
  }
  return m;
}

__device__ __forceinline__ M3<double> ldm(const double2* base, int64_t V, int64_t n) {
  M3<double> m;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double2 v = base[(int64_t)e * V + n];
    m.m[e / 3][e % 3] = C<double>{v.x, v.y};
  }
  return m;
}

__device__ __forceinline__ void addm(double2* base, int64_t V, int64_t n, const M3<double>& a, double s) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    double2* q = base + (int64_t)e * V + n;
    double2 v = *q;
    v.x += s * a.m[e / 3][e % 3].re;
    v.y += s * a.m[e / 3][e % 3].im;
    *q = v;
  }
}

__device__ __forceinline__ int nu_idx(const int d[4]) {
  return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) + 27 * (d[3] + 1);
}

// Level-k link gradients (gather over the transporters whose last hop is U_mu(m)):
//   forward hop  W_d(n) = ... W_{d'}(n) U_mu(n + d'):        G_U_mu(m) += (1/k) W_{d'}(n)^dagger G_W[d](n), n = m - d'
//   backward hop W_d(n) = ... W_{d'}(n) U_mu(n + d' - mu)^+: G_U_mu(m) += (1/k) G_W[d](n)^dagger W_{d'}(n), n = m - d' + mu
__global__ void k_rev_links(Geom g, LevelList lst, int k, const double2* __restrict__ T,
                            const double2* __restrict__ GW, double2* GU) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (m >= g.V) return;
  M3<double> acc;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) acc.m[a][b] = C<double>{0, 0};
  for (int i = 0; i < lst.count; ++i) {
    const int nu = lst.nu[i];
    int d[4] = {nu % 3 - 1, (nu / 3) % 3 - 1, (nu / 9) % 3 - 1, (nu / 27) % 3 - 1};
    const int s = d[mu];
    if (s == 0) continue;
    int dp[4] = {d[0], d[1], d[2], d[3]};
    dp[mu] -= s;
    int back[4] = {-dp[0], -dp[1], -dp[2], -dp[3]};
    if (s < 0) back[mu] += 1;
    const int n = site_shift(g, m, back);
    const M3<double> gw = ldm(GW + (int64_t)nu * 9 * g.V, g.V, n);
    const M3<double> wp = ldm(T + (int64_t)nu_idx(dp) * 9 * g.V, g.V, n);
    madd(acc, s > 0 ? mmul(adj(wp), gw) : mmul(adj(gw), wp));
  }
  addm(GU + (int64_t)mu * 9 * g.V, g.V, m, acc, 1.0 / k);
}

// Level-k transporter gradients passed down to level k-1 (same site):
//   G_W[d'](n) += (1/k) sum_{mu: d'_mu = 0, s = +-1} G_W[d' + s e_mu](n) S^dagger,
//   S = U_mu(n + d') (s = +1) or U_mu(n + d' - mu)^dagger (s = -1).
__global__ void k_rev_transporters(Geom g, LevelList lower, int k, const double2* __restrict__ U64, double2* GW) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int which = blockIdx.y;
  if (n >= g.V || which >= lower.count) return;
  const int nup = lower.nu[which];
  const int dp[4] = {nup % 3 - 1, (nup / 3) % 3 - 1, (nup / 9) % 3 - 1, (nup / 27) % 3 - 1};
  M3<double> acc;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) acc.m[a][b] = C<double>{0, 0};
  for (int mu = 0; mu < 4; ++mu) {
    if (dp[mu] != 0) continue;
    for (int s = -1; s <= 1; s += 2) {
      int d[4] = {dp[0], dp[1], dp[2], dp[3]};
      d[mu] = s;
      const M3<double> gw = ldm(GW + (int64_t)nu_idx(d) * 9 * g.V, g.V, n);
      int at[4] = {dp[0], dp[1], dp[2], dp[3]};
      if (s < 0) at[mu] -= 1;
      const int ms = site_shift(g, n, at);
      const M3<double> u = ldm(U64 + (int64_t)mu * 9 * g.V, g.V, ms);
      madd(acc, s > 0 ? mmul(gw, adj(u)) : mmul(gw, u));
    }
  }
  addm(GW + (int64_t)nup * 9 * g.V, g.V, n, acc, 1.0 / k);
}

// One-hop transporters: W_{+mu}(m) = U_mu(m), W_{-mu}(m + mu) = U_mu(m)^dagger.
__global__ void k_rev_level1(Geom g, const double2* __restrict__ GW, double2* GU) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (m >= g.V) return;
  int e[4] = {0, 0, 0, 0};
  e[mu] = 1;
  const int fwd = nu_idx(e);
  int ne[4] = {-e[0], -e[1], -e[2], -e[3]};
  const int bwd = nu_idx(ne);
  const int mp = site_shift(g, m, e);
  M3<double> acc = ldm(GW + (int64_t)fwd * 9 * g.V, g.V, m);
  madd(acc, adj(ldm(GW + (int64_t)bwd * 9 * g.V, g.V, mp)));
  addm(GU + (int64_t)mu * 9 * g.V, g.V, m, acc, 1.0);
}

// SoA [4][9][V] -> caller layout [V][4][3][3], with the antiperiodic sign of
// U_t on the last time slice carried back to the original links.
__global__ void k_links_out(Geom g, const double2* __restrict__ GU, double2* out, int anti) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int t = (int)(n / g.str[3]);
  for (int mu = 0; mu < 4; ++mu) {
    const double sg = (anti && mu == 3 && t == g.L[3] - 1) ? -1.0 : 1.0;
    for (int e = 0; e < 9; ++e) {
      double2 v = GU[((int64_t)mu * 9 + e) * g.V + n];
      out[((int64_t)n * 4 + mu) * 9 + e] = make_double2(sg * v.x, sg * v.y);
    }
  }
}

__global__ void k_zero(int64_t n, double2* p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------ clover term
// C(n) = -(c_SW/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(n), F = P[(Q - Q^+)/(8i)].
// Re<u, dC v> has the gradient G_F = -(c_SW/2) sum_{t,s} sigma_{ts} O_{st} with
// the colour outer products O_{st} = u_s(n) v_t(n)^dagger, and
// G_Q = (i/8) (P G_F + (P G_F)^dagger) with respect to the leaf sum Q.  In the
// chiral basis sigma_{mu nu} is block diagonal: sigma_12 = -diag(s3, s3),
// sigma_13 = diag(s2, s2), sigma_23 = -diag(s1, s1), sigma_j4 = diag(s_j, -s_j),
// so only the four outer products within one chirality block enter, through
//   B_1 = O_{10} + O_{01},  B_2 = i (O_{01} - O_{10}),  B_3 = O_{00} - O_{11}
// (spins of the block renumbered 0, 1); the upper block enters every plane with
// the sign +1, the lower block with -1 in the (j, 4) planes.  One launch per
// chirality block (blk), each adding its part of G_Q into GQ = [6][9][V], the
// planes ordered (01, 02, 03, 12, 13, 23).
__global__ void __launch_bounds__(128) k_clover_force(Geom g, const PairList* __restrict__ pl, int npair, int blk,
                                                     double c_sw, double2* GQ) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  C<double> O[2][2][3][3];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) O[s][t][a][b] = C<double>{0, 0};
  for (int p = 0; p < npair; ++p) {
    const double2* up = reinterpret_cast<const double2*>(pl->u[p]) + (int64_t)n * 12 + 6 * blk;
    const double2* vp = reinterpret_cast<const double2*>(pl->v[p]) + (int64_t)n * 12 + 6 * blk;
    const double wp = pl->w[p];
    C<double> u[2][3], v[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double2 x = up[s * 3 + a], y = vp[s * 3 + a];
        u[s][a] = C<double>{wp * x.x, wp * x.y};
        v[s][a] = C<double>{y.x, y.y};
      }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) cfma_cj(O[s][t][a][b], v[t][b], u[s][a]);  // u_sa conj(v_tb)
  }
  const double pre = -0.5 * c_sw;
  const double lo = blk == 0 ? 1.0 : -1.0;  // sign of this block in the (j, 4) planes
  // plane -> (Pauli index l, sign): 01: (3, -1), 02: (2, +1), 03: (1, lo), 12: (1, -1), 13: (2, lo), 23: (3, lo)
  const int lidx[6] = {3, 2, 1, 1, 2, 3};
  const double sgn[6] = {-1.0, 1.0, lo, -1.0, lo, lo};
#pragma unroll 1
  for (int pi = 0; pi < 6; ++pi) {
    C<double> F[3][3];
    const int l = lidx[pi];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        C<double> v;
        if (l == 1) {
          v = O[1][0][a][b] + O[0][1][a][b];
        } else if (l == 2) {
          const C<double> d = O[0][1][a][b] - O[1][0][a][b];
          v = C<double>{-d.im, d.re};
        } else {
          v = O[0][0][a][b] - O[1][1][a][b];
        }
        F[a][b] = (pre * sgn[pi]) * v;
      }
    const C<double> tr = F[0][0] + F[1][1] + F[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a][a] = F[a][a] - (1.0 / 3.0) * tr;
    // G_Q = (i/8) (F + F^dagger)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const C<double> h = F[a][b] + conj(F[b][a]);
        double2* q = GQ + ((int64_t)pi * 9 + a * 3 + b) * g.V + n;
        double2 cur = *q;
        cur.x += -h.im / 8.0;
        cur.y += h.re / 8.0;
        *q = cur;
      }
  }
}

// The four leaves of a plane (mu, nu) at n, each as four factors in product
// order: {role (0: U_mu, 1: U_nu), daggered, a, b} for the link at n + a e_mu + b e_nu
// (the leaves of the clover construction); passed to the kernel by value.
struct LeafTable {
  int f[4][4][4];
};
constexpr LeafTable kLeaves = {{
    {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {1, 1, 0, 0}},
    {{1, 0, 0, 0}, {0, 1, -1, 1}, {1, 1, -1, 0}, {0, 0, -1, 0}},
    {{0, 1, -1, 0}, {1, 1, -1, -1}, {0, 0, -1, -1}, {1, 0, 0, -1}},
    {{1, 1, 0, -1}, {0, 0, 0, -1}, {1, 0, 1, -1}, {0, 1, 0, 0}},
}};

__device__ __forceinline__ M3<double> leaf_factor(const Geom& g, const double2* __restrict__ U64, int n, int mu,
                                                  int nu, const int f[4]) {
  int d[4] = {0, 0, 0, 0};
  d[mu] += f[2];
  d[nu] += f[3];
  const int dir = f[0] == 0 ? mu : nu;
  const M3<double> m = ldm(U64 + (int64_t)dir * 9 * g.V, g.V, site_shift(g, n, d));
  return f[1] ? adj(m) : m;
}

// G_U_rho(m) += sum over the clover leaves containing U_rho(m): a forward
// factor of the leaf A U B receives A^dagger G_Q B^dagger, a daggered one
// (A U^dagger B) receives B G_Q^dagger A (G_Q at the leaf's base site n).
__global__ void k_clover_links(Geom g, const double2* __restrict__ U64, const double2* __restrict__ GQ, double2* GU,
                               const __grid_constant__ LeafTable kLeaf) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int rho = blockIdx.y;
  if (m >= g.V) return;
  M3<double> acc;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) acc.m[a][b] = C<double>{0, 0};
  int pi = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++pi) {
      if (mu != rho && nu != rho) continue;
      for (int lf = 0; lf < 4; ++lf)
        for (int j = 0; j < 4; ++j) {
          const int* fj = kLeaf.f[lf][j];
          if ((fj[0] == 0 ? mu : nu) != rho) continue;
          int back[4] = {0, 0, 0, 0};
          back[mu] -= fj[2];
          back[nu] -= fj[3];
          const int n = site_shift(g, m, back);  // base site of the leaf
          M3<double> A, B;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              A.m[a][b] = C<double>{a == b ? 1.0 : 0.0, 0};
              B.m[a][b] = A.m[a][b];
            }
          for (int k = 0; k < j; ++k) A = mmul(A, leaf_factor(g, U64, n, mu, nu, kLeaf.f[lf][k]));
          for (int k = j + 1; k < 4; ++k) B = mmul(B, leaf_factor(g, U64, n, mu, nu, kLeaf.f[lf][k]));
          const M3<double> gq = ldm(GQ + (int64_t)pi * 9 * g.V, g.V, n);
          madd(acc, fj[1] ? mmul(mmul(B, adj(gq)), A) : mmul(mmul(adj(A), gq), adj(B)));
        }
    }
  addm(GU + (int64_t)rho * 9 * g.V, g.V, m, acc, 1.0);
}

// Hop table of the Wilson kernel in the Brillouin table's form: the one-hop
// offsets carry M_{+-mu} = -1/2 (1 -+ gamma_mu), every other offset zero.
const HopTable<double>& wilson_hop_table() {
  static const HopTable<double> t = [] {
    HopTable<double> h;
    fill_hops(h);
    for (int j = 0; j < 40; ++j) {
      int k = 0;
      for (int mu = 0; mu < 4; ++mu) k += h.site_d[j][mu] != 0;
      h.a[j] = k == 1 ? -0.5 : 0.0;
      for (int mu = 0; mu < 4; ++mu) h.cs[j][mu] = k == 1 ? 0.5 * h.site_d[j][mu] : 0.0;
    }
    return h;
  }();
  return t;
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

// y = a x + b y (real coefficients, FP64)
__global__ void k_axpby_real(int64_t n, double a, const double* __restrict__ x, double b, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// acc = c0 b + sum_i w_i X_i for systems s < nout of an X with nsys systems per shift
__global__ void k_rational_sub(int64_t nreal, int nsys, int nshift, double c0, const double* __restrict__ w,
                               const double* __restrict__ b, const double* __restrict__ X, double* out) {
  const int s = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nreal; i += (int64_t)gridDim.x * blockDim.x) {
    double v = c0 * b[s * nreal + i];
    for (int k = 0; k < nshift; ++k) v += w[k] * X[((int64_t)k * nsys + s) * nreal + i];
    out[s * nreal + i] = v;
  }
}

}  // namespace

int overlap_grad_impl(bri_ctx* c, double* g_psi, double* g_U, const double* eta, const double* psi, int nrhs, int n,
                      int kind, double rho, double am, double scale, double tol, int prec, bri_stats* stats) {
  cudaStream_t st = c->stream;
  const Geom& g = c->g;
  const int64_t V = g.V, nreal = V * 24;
  const double m0 = -rho;
  double c0, w[BRI_MAX_SHIFTS], sig[BRI_MAX_SHIFTS];
  int rc = kl_host(n, kind, scale, &c0, w, sig);
  if (rc) return rc;
  const double kfac = (1.0 - am / (2.0 * rho)) * rho;

  int solve_rc = BRI_OK;
  // shifted solves for psi and D^dagger eta (2 nrhs systems, same shifts)
  const int nsys = 2 * nrhs;
  Buf bb, bX, bDX, by;
  if ((rc = bb.alloc(sizeof(double) * nreal * nsys, st))) return rc;
  BRI_CUDA(cudaMemcpyAsync(bb.as<double>(), psi, sizeof(double) * nreal * nrhs, cudaMemcpyDeviceToDevice, st));
  if ((rc = dirac_kernel(c, bb.as<double>() + nreal * nrhs, eta, nrhs, m0, 1, BRI_PREC_F64, st))) return rc;
  std::vector<double> sig_all((size_t)nsys * n);
  for (int s = 0; s < nsys; ++s)
    for (int k = 0; k < n; ++k) sig_all[(size_t)s * n + k] = sig[k];
  if ((rc = bX.alloc(sizeof(double) * nreal * nsys * n, st))) return rc;
  SolveInfo info;
  // phase times (stream-synchronised): solves, D X and rationals, forces, link back-propagation
  double tph[4] = {0, 0, 0, 0};
  auto tmark = std::chrono::steady_clock::now();
  auto lap = [&](int ph) {
    cudaStreamSynchronize(st);
    const auto t1 = std::chrono::steady_clock::now();
    tph[ph] += std::chrono::duration<double>(t1 - tmark).count();
    tmark = t1;
  };
  const int maxiter = (stats && stats->maxiter > 0) ? stats->maxiter : 20000;
  rc = solve_shifts(c, bb.as<double>(), nsys, n, sig_all.data(), m0, tol, prec, maxiter, bX.as<double>(), info);
  if (rc < 0) return rc;
  if (rc > solve_rc) solve_rc = rc;
  double* X = bX.as<double>();
  lap(0);

  // y = c0 psi + sum w_i x_i ; D X for every shift and system
  Buf bw;
  if ((rc = bw.alloc(sizeof(double) * BRI_MAX_SHIFTS, st))) return rc;
  BRI_CUDA(cudaMemcpyAsync(bw.as<double>(), w, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if ((rc = by.alloc(sizeof(double) * nreal * nrhs, st))) return rc;
  k_rational_sub<<<dim3(256, nrhs), 256, 0, st>>>(nreal, nsys, n, c0, bw.as<double>(), psi, X, by.as<double>());
  note_launch();
  // g_psi = k eta + am eta + k (c0 D^dagger eta + sum_i w_i z_i): the rational of the
  // second half of the systems (right-hand sides D^dagger eta), then the axpy
  k_rational_sub<<<dim3(256, nrhs), 256, 0, st>>>(nreal, nsys, n, c0, bw.as<double>(), bb.as<double>() + nreal * nrhs,
                                                  X + nreal * nrhs, g_psi);
  note_launch();
  k_axpby_real<<<1024, 256, 0, st>>>(nreal * nrhs, kfac + am, eta, kfac, g_psi);
  note_launch();
  if ((rc = bDX.alloc(sizeof(double) * nreal * nsys * n, st))) return rc;
  if ((rc = dirac_kernel(c, bDX.as<double>(), X, nsys * n, m0, 0, BRI_PREC_F64, st))) return rc;
  BRI_LAUNCH_CHECK("overlap_grad solves");

  lap(1);
  // transporter gradients from all (u, v, weight) pairs
  const bool wilson = c->kernel == BRI_KERNEL_WILSON;
  const HopTable<double>& htab = wilson ? wilson_hop_table() : hop_table<double>();
  OffsetList ol;
  ol.count = 0;
  for (int j = 0; j < 40; ++j) {
    int k = 0;
    for (int mu = 0; mu < 4; ++mu) k += htab.site_d[j][mu] != 0;
    if (!wilson || k == 1) ol.j[ol.count++] = j;
  }
  Buf bGW, bpl, bGQ;
  if ((rc = bGW.alloc(sizeof(double2) * 81 * 9 * V, st))) return rc;
  k_zero<<<2048, 256, 0, st>>>(81 * 9 * V, bGW.as<double2>()); note_launch();
  if (c->have_clover) {
    if ((rc = bGQ.alloc(sizeof(double2) * 6 * 9 * V, st))) return rc;
    k_zero<<<512, 256, 0, st>>>(6 * 9 * V, bGQ.as<double2>()); note_launch();
  }
  if ((rc = bpl.alloc(sizeof(PairList), st))) return rc;
  const int per_rhs = 1 + 2 * n;
  const int rhs_per_chunk = std::max(1, 512 / per_rhs);
  std::vector<PairList> hpl((nrhs + rhs_per_chunk - 1) / rhs_per_chunk);
  for (int r0 = 0, ci = 0; r0 < nrhs; r0 += rhs_per_chunk, ++ci) {
    PairList& pl = hpl[ci];
    int np = 0;
    for (int r = r0; r < std::min(nrhs, r0 + rhs_per_chunk); ++r) {
      pl.u[np] = eta + r * nreal;
      pl.v[np] = by.as<double>() + r * nreal;
      pl.w[np++] = kfac;
      for (int i = 0; i < n; ++i) {
        const double* xi = X + ((int64_t)i * nsys + r) * nreal;
        const double* zi = X + ((int64_t)i * nsys + nrhs + r) * nreal;
        const double* dxi = bDX.as<double>() + ((int64_t)i * nsys + r) * nreal;
        const double* dzi = bDX.as<double>() + ((int64_t)i * nsys + nrhs + r) * nreal;
        pl.u[np] = dxi;
        pl.v[np] = zi;
        pl.w[np++] = -kfac * w[i];
        pl.u[np] = dzi;
        pl.v[np] = xi;
        pl.w[np++] = -kfac * w[i];
      }
    }
    BRI_CUDA(cudaMemcpyAsync(bpl.as<PairList>(), &pl, sizeof(PairList), cudaMemcpyHostToDevice, st));
    dim3 grid(blocks_for(V, 128), ol.count, 2);
    k_force<<<grid, 128, 0, st>>>(g, bpl.as<PairList>(), np, bGW.as<double2>(), htab, ol); note_launch();
    if (c->have_clover)
      for (int blk = 0; blk < 2; ++blk) {
        k_clover_force<<<blocks_for(V, 128), 128, 0, st>>>(g, bpl.as<PairList>(), np, blk, c->c_sw,
                                                           bGQ.as<double2>());
        note_launch();
      }
    BRI_CUDA(cudaStreamSynchronize(st));  // the pair list buffer is reused
  }

  lap(2);
  // back through the path average to the thin links (the Wilson kernel's
  // transporters are the links: one-hop level only)
  Buf bT, bGU;
  if (!wilson) {
    if ((rc = bT.alloc(sizeof(double2) * 81 * 9 * V, st))) return rc;
    if ((rc = build_transporters(c, bT.as<double2>()))) return rc;
  }
  if ((rc = bGU.alloc(sizeof(double2) * 36 * V, st))) return rc;
  k_zero<<<512, 256, 0, st>>>(36 * V, bGU.as<double2>()); note_launch();
  for (int k = 4; k >= 2 && !wilson; --k) {
    const LevelList lst = level_list(k), lower = level_list(k - 1);
    k_rev_links<<<dim3(blocks_for(V, 128), 4), 128, 0, st>>>(g, lst, k, bT.as<double2>(), bGW.as<double2>(),
                                                            bGU.as<double2>()); note_launch();
    k_rev_transporters<<<dim3(blocks_for(V, 128), lower.count), 128, 0, st>>>(g, lower, k, c->U64,
                                                                             bGW.as<double2>()); note_launch();
  }
  k_rev_level1<<<dim3(blocks_for(V, 128), 4), 128, 0, st>>>(g, bGW.as<double2>(), bGU.as<double2>()); note_launch();
  if (c->have_clover) {
    k_clover_links<<<dim3(blocks_for(V, 128), 4), 128, 0, st>>>(g, c->U64, bGQ.as<double2>(), bGU.as<double2>(),
                                                               kLeaves);
    note_launch();
  }
  k_links_out<<<blocks_for(V, 128), 128, 0, st>>>(g, bGU.as<double2>(), (double2*)g_U,
                                                  (c->flags & BRI_ANTIPERIODIC_T) ? 1 : 0); note_launch();
  BRI_LAUNCH_CHECK("overlap_grad backward");
  BRI_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats->iterations = info.iters;
    stats->matvecs = info.cnt.matvecs + 1 + nsys * n;
    stats->matvecs_f64 = info.cnt.matvecs64 + 1 + nsys * n;
    stats->refinements = info.refinements;
    stats->n_shifts = n;
    lap(3);
    for (int ph = 0; ph < 4; ++ph) stats->phase_seconds[ph] = tph[ph];
  }
  return solve_rc;
}

}  // namespace bri
