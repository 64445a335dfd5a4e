// Brillouin stencil in double-word FP32 arithmetic (a value is the unevaluated
// sum h + l of two floats, about 48 significant bits), for FP64-class operator
// applications on the FP32 pipe.  GB300 runs FP64 at 1/64 of its FP32 rate,
// so the FP64 residuals of the mixed-precision scheme are cheaper this way.
//
// Arithmetic, from published error-free transformations:
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Moller 1965): s + e = a + b exactly,
//    six operations, no ordering condition;
//  * Fast2Sum (Dekker 1971): s + e = a + b exactly when |a| >= |b|;
//  * TwoProduct with a fused multiply-add (Ogita, Rump and Oishi, "Accurate
//    sum and dot product", SIAM J. Sci. Comput. 26 (2005)): p + e = a b exactly;
//  * their Dot2 accumulation: the leading parts of the products are summed by
//    TwoSum, and every rounding error (of the sums and of the products) is
//    collected in a second FP32 word.  With double-word operands the two cross
//    products u_h v_l + u_l v_h join that word too (their own rounding is
//    ~2^-48 of the product).  The accumulators are renormalised by Fast2Sum
//    once per hop pair.
// The products and sums of the transformations are written with the _rn
// intrinsics, which the compiler never contracts into fused operations.
//
// The stencil is that of the FP32/FP64 kernels (Eq. def_bril, App. C), but the
// spin matrix of each hop is applied before the colour transport:
//   W_d(n) M_d x(n+d) = W_d(n) (M_d x(n+d)),   M_{+-d} = a_k 1 +- c_k S_d,
//   S_d = sum_mu d_mu gamma_mu,
// so that every colour product accumulates straight into the site's
// double-word accumulators.  a_k = -2^{-k-3} is a power of two (exact
// scaling); c_k = 4^{2-k}/27 is carried as a double-word constant.
//
// Storage: spinors as [rhs][V][12] float4 (re_h, re_l, im_h, im_l), links
// [40][9][V] float4 and clover [2][36][V] float2 (h, l): the byte layout of the
// FP64 arrays, so an FP64 vector and its double-word copy have the same size.
#include "stencil.cuh"
#include "hops.cuh"

#include <string>

namespace bri {

namespace {

struct DW {
  float h, l;
};
// accumulator: h + l, l not normalised against h between renormalisations
struct Acc {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc += u v (one Dot2 step with double-word operands)
__device__ __forceinline__ void mac(Acc& acc, float uh, float ul, float vh, float vl) {
  const float p = __fmul_rn(uh, vh);
  const float pe = __fmaf_rn(uh, vh, -p);
  float s, e;
  two_sum(acc.h, p, s, e);
  acc.h = s;
  float t = __fadd_rn(e, pe);
  t = __fmaf_rn(uh, vl, t);
  t = __fmaf_rn(ul, vh, t);
  acc.l = __fadd_rn(acc.l, t);
}
__device__ __forceinline__ void mac(Acc& acc, DW u, DW v) { mac(acc, u.h, u.l, v.h, v.l); }
// acc += t (double-word addend)
__device__ __forceinline__ void add(Acc& acc, float th, float tl) {
  float s, e;
  two_sum(acc.h, th, s, e);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, tl));
}
__device__ __forceinline__ DW renorm(const Acc& a) {
  DW r;
  fast_two_sum(a.h, a.l, r.h, r.l);
  return r;
}
__device__ __forceinline__ DW finish(const Acc& a) {
  DW r;
  two_sum(a.h, a.l, r.h, r.l);
  return r;
}

struct CDW {
  DW re, im;
};
struct CAcc {
  Acc re, im;
};

// acc += w v and acc += conj(w) v (complex, double-word)
__device__ __forceinline__ void cmac(CAcc& acc, const float4& w, const CDW& v) {
  mac(acc.re, w.x, w.y, v.re.h, v.re.l);
  mac(acc.re, -w.z, -w.w, v.im.h, v.im.l);
  mac(acc.im, w.x, w.y, v.im.h, v.im.l);
  mac(acc.im, w.z, w.w, v.re.h, v.re.l);
}
__device__ __forceinline__ void cmac_cj(CAcc& acc, const float4& w, const CDW& v) {
  mac(acc.re, w.x, w.y, v.re.h, v.re.l);
  mac(acc.re, w.z, w.w, v.im.h, v.im.l);
  mac(acc.im, w.x, w.y, v.im.h, v.im.l);
  mac(acc.im, -w.z, -w.w, v.re.h, v.re.l);
}

// Per-offset constants: a_k (exact in FP32), c_k as a double-word pair.
struct HopTableDW {
  int site_d[40][4];
  float a[40];
  float ch[40], cl[40];
};

HopTableDW make_hop_table_dw() {
  const HopTable<double>& h = hop_table<double>();
  HopTableDW t;
  for (int j = 0; j < 40; ++j) {
    double c = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
      t.site_d[j][mu] = h.site_d[j][mu];
      if (h.cs[j][mu] != 0.0) c = h.cs[j][mu] > 0 ? h.cs[j][mu] : -h.cs[j][mu];
    }
    t.a[j] = (float)h.a[j];
    t.ch[j] = (float)c;
    t.cl[j] = (float)(c - (double)t.ch[j]);
  }
  return t;
}

const HopTableDW& hop_table_dw() {
  static const HopTableDW t = make_hop_table_dw();
  return t;
}

__device__ __forceinline__ CDW ld_cdw(const float4* p) {
  const float4 v = __ldg(p);
  return CDW{DW{v.x, v.y}, DW{v.z, v.w}};
}

// phase * z for phase = 1, i, -1, -i (q = 0..3), times sign sg = +-1
__device__ __forceinline__ void phased(const CDW& z, int q, float sg, float& rh, float& rl, float& ih, float& il) {
  // i z = (-z_im, z_re)
  float ar = z.re.h, arl = z.re.l, ai = z.im.h, ail = z.im.l;
  if (q == 1) {
    ar = -z.im.h; arl = -z.im.l; ai = z.re.h; ail = z.re.l;
  } else if (q == 2) {
    ar = -ar; arl = -arl; ai = -ai; ail = -ail;
  } else if (q == 3) {
    ar = z.im.h; arl = z.im.l; ai = -z.re.h; ail = -z.re.l;
  }
  rh = sg * ar; rl = sg * arl; ih = sg * ai; il = sg * ail;
}

// y = a x + c S_d x over one colour (four spins), S_d = sum_mu d_mu gamma_mu in
// the chiral basis (the spin structure of gamma_term):
//   gamma_1 x = (-i x3, -i x2, i x1, i x0), gamma_2 x = (-x3, x2, x1, -x0),
//   gamma_3 x = (-i x2, i x3, i x0, -i x1), gamma_4 x = (x2, x3, x0, x1).
__device__ __forceinline__ void spin_apply(CDW y[4], const CDW x[4], float a, DW c, const int d[4]) {
  // source spin and phase (1, i, -1, -i as 0..3) of gamma_mu x at spin s
  constexpr int src[4][4] = {{3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}, {2, 3, 0, 1}};
  constexpr int ph[4][4] = {{3, 3, 1, 1}, {2, 0, 0, 2}, {3, 1, 1, 3}, {0, 0, 0, 0}};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    CAcc S{{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      if (d[mu] == 0) continue;
      float rh, rl, ih, il;
      phased(x[src[mu][s]], ph[mu][s], (float)d[mu], rh, rl, ih, il);
      add(S.re, rh, rl);
      add(S.im, ih, il);
    }
    // y_s = a x_s + c S (a x_s exact: a is a power of two)
    CAcc Y{{0.f, 0.f}, {0.f, 0.f}};
    Y.re.h = a * x[s].re.h;
    Y.re.l = a * x[s].re.l;
    Y.im.h = a * x[s].im.h;
    Y.im.l = a * x[s].im.l;
    mac(Y.re, c.h, c.l, S.re.h, S.re.l);
    mac(Y.im, c.h, c.l, S.im.h, S.im.l);
    y[s].re = renorm(Y.re);
    y[s].im = renorm(Y.im);
  }
}

// One thread per site and right-hand side (grid groups = right-hand sides, in
// the order of stencil_grid).  One source colour at a time keeps 128
// registers (16 warps per SM) without spills.
__global__ void __launch_bounds__(128, 4)
    bri_kernel_dw(Geom g, float4* __restrict__ y, const float4* __restrict__ x, const float4* __restrict__ W,
                  const float2* __restrict__ cl, DW diag, float sgn, int gfirst, const __grid_constant__ HopTableDW H) {
  const int grp = gfirst ? blockIdx.x : blockIdx.y, blk = gfirst ? blockIdx.y : blockIdx.x;
  const int n = blk * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int64_t V = g.V;
  const int64_t roff = (int64_t)grp * V * 12;
  const float4* xin = x + roff;
  int co[4], L[4], str[4];
  {
    int r = n;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      co[mu] = r % g.L[mu];
      r /= g.L[mu];
    }
    co[3] = r;
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    L[mu] = g.L[mu];
    str[mu] = (int)g.str[mu];
  }
  CAcc acc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) acc[s][aa] = CAcc{{0.f, 0.f}, {0.f, 0.f}};

#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    int d[4], mp = 0, mm = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      d[mu] = H.site_d[j][mu];
      mp += wrap(co[mu] + d[mu], L[mu]) * str[mu];
      mm += wrap(co[mu] - d[mu], L[mu]) * str[mu];
    }
    const float a = H.a[j];
    const DW c{sgn * H.ch[j], sgn * H.cl[j]};
    const DW cm{-c.h, -c.l};
    // The two hops of the pair, one source colour b at a time (the spin matrix
    // mixes spins only), as rolled loops so that the body fits the instruction
    // cache:
    //   forward  (h = 0): acc[.][aa] += W_d(n)[aa][b] (M_d x(n+d))[.][b]
    //   backward (h = 1): acc[.][aa] += conj(W_d(n-d)[b][aa]) (M_{-d} x(n-d))[.][b]
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int m = h ? mm : mp;
      const float4* wp = W + (int64_t)j * 9 * V + (h ? mm : n);
      const DW ch = h ? cm : c;
      const float cs = h ? -1.f : 1.f;  // conj(w) = (w_re, -w_im)
#pragma unroll 1
      for (int b = 0; b < 3; ++b) {
        CDW xs[4], ys[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) xs[s] = ld_cdw(xin + (int64_t)m * 12 + s * 3 + b);
        spin_apply(ys, xs, a, ch, d);
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          float4 w = __ldg(wp + (int64_t)(h ? b * 3 + aa : aa * 3 + b) * V);
          w.z *= cs;
          w.w *= cs;
#pragma unroll
          for (int s = 0; s < 4; ++s) cmac(acc[s][aa], w, ys[s]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        const DW r = renorm(acc[s][aa].re), i = renorm(acc[s][aa].im);
        acc[s][aa] = CAcc{{r.h, r.l}, {i.h, i.l}};
      }
  }
  // diagonal and clover terms at the site itself
  CDW xc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      xc[s][b] = ld_cdw(xin + (int64_t)n * 12 + s * 3 + b);
      mac(acc[s][b].re, diag, xc[s][b].re);
      mac(acc[s][b].im, diag, xc[s][b].im);
    }
  if (cl) {
    // two Hermitian 6x6 chiral blocks: 6 diagonal reals, then the 15 upper
    // off-diagonal complex entries row by row (the FP64 packing)
#pragma unroll
    for (int blk6 = 0; blk6 < 2; ++blk6) {
      const float2* cb = cl + (int64_t)blk6 * 36 * V + n;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float2 dd = __ldg(cb + (int64_t)i * V);
        const CDW& in = xc[2 * blk6 + i / 3][i % 3];
        CAcc& o = acc[2 * blk6 + i / 3][i % 3];
        mac(o.re, dd.x, dd.y, in.re.h, in.re.l);
        mac(o.im, dd.x, dd.y, in.im.h, in.im.l);
      }
      int k = 6;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int jj = i + 1; jj < 6; ++jj) {
          const float2 cr = __ldg(cb + (int64_t)k * V), ci = __ldg(cb + (int64_t)(k + 1) * V);
          const float4 cij = make_float4(cr.x, cr.y, ci.x, ci.y);
          cmac(acc[2 * blk6 + i / 3][i % 3], cij, xc[2 * blk6 + jj / 3][jj % 3]);
          cmac_cj(acc[2 * blk6 + jj / 3][jj % 3], cij, xc[2 * blk6 + i / 3][i % 3]);
          k += 2;
        }
    }
  }
  float4* yo = y + roff + (int64_t)n * 12;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      const DW r = finish(acc[s][aa].re), i = finish(acc[s][aa].im);
      yo[s * 3 + aa] = make_float4(r.h, r.l, i.h, i.l);
    }
}

// FP64 (re, im) -> double-word (re_h, re_l, im_h, im_l), element by element
__global__ void k_split_dw(int64_t n, const double2* __restrict__ in, float4* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    out[i] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
}
__global__ void k_split_dw_real(int64_t n, const double* __restrict__ in, float2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
}
__global__ void k_join_dw(int64_t n, const float4* __restrict__ in, double2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

}  // namespace

// Double-word copies of the FP64 links and clover, made on first use after
// each bri_build_links.
int ensure_dw_links(bri_ctx* c) {
  if (c->dw_valid) return BRI_OK;
  const int64_t V = c->g.V;
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
  if ((rc = alloc(&c->Wdw, sizeof(float4) * 360 * V))) return rc;
  k_split_dw<<<1024, 256, 0, st>>>(360 * V, c->W64, (float4*)c->Wdw); note_launch();
  if (c->have_clover) {
    if ((rc = alloc(&c->Cdw, sizeof(float2) * 72 * V))) return rc;
    k_split_dw_real<<<1024, 256, 0, st>>>(72 * V, c->C64, (float2*)c->Cdw); note_launch();
  }
  BRI_LAUNCH_CHECK("double-word links");
  c->dw_valid = true;
  return BRI_OK;
}

// y = D x or D^dagger x on double-word vectors (Brillouin kernel).
int dirac_bri_dw(bri_ctx* c, void* y, const void* x, int nrhs, double m0, int dagger, cudaStream_t s) {
  int rc = ensure_dw_links(c);
  if (rc) return rc;
  const double dg = 15.0 / 8.0 + m0;
  DW diag;
  diag.h = (float)dg;
  diag.l = (float)(dg - (double)diag.h);
  const int threads = 128;
  const StencilGrid sg = stencil_grid(blocks_for(c->g.V, threads), nrhs);
  bri_kernel_dw<<<sg.grid, threads, 0, s>>>(c->g, (float4*)y, (const float4*)x, (const float4*)c->Wdw,
                                             c->have_clover ? (const float2*)c->Cdw : nullptr, diag,
                                             dagger ? -1.f : 1.f, sg.gfirst, hop_table_dw());
  note_launch();
  BRI_LAUNCH_CHECK("bri_kernel_dw");
  return BRI_OK;
}

// FP64 in, FP64 out: split, stencil, join (tmp: two double-word vectors of
// nrhs right-hand sides, 16 bytes per complex element each).
int dirac_bri_dw64(bri_ctx* c, double* y, const double* x, int nrhs, double m0, int dagger, void* tmp,
                   cudaStream_t s) {
  const int64_t ne = c->g.V * 12 * nrhs;
  float4* xa = (float4*)tmp;
  float4* ya = xa + ne;
  k_split_dw<<<1024, 256, 0, s>>>(ne, (const double2*)x, xa); note_launch();
  int rc = dirac_bri_dw(c, ya, xa, nrhs, m0, dagger, s);
  if (rc) return rc;
  k_join_dw<<<1024, 256, 0, s>>>(ne, ya, (double2*)y); note_launch();
  BRI_LAUNCH_CHECK("double-word apply");
  return BRI_OK;
}

// A x = D^dagger D x on FP64 vectors through double-word stencils; out = A x
// (FP64).  t1, t2: double-word scratch of nrhs vectors each.
int normal_op_dw(bri_ctx* c, double* out, const double* x, int nrhs, double m0, void* t1, void* t2, cudaStream_t s) {
  const int64_t ne = c->g.V * 12 * nrhs;
  k_split_dw<<<1024, 256, 0, s>>>(ne, (const double2*)x, (float4*)t1); note_launch();
  int rc = dirac_bri_dw(c, t2, t1, nrhs, m0, 0, s);
  if (rc) return rc;
  rc = dirac_bri_dw(c, t1, t2, nrhs, m0, 1, s);
  if (rc) return rc;
  k_join_dw<<<1024, 256, 0, s>>>(ne, (const float4*)t1, (double2*)out); note_launch();
  BRI_LAUNCH_CHECK("double-word normal operator");
  return BRI_OK;
}

}  // namespace bri
