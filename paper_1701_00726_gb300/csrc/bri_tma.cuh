// Brillouin stencil with the streamed links staged in shared memory by bulk
// asynchronous copies (warp-specialised; FP32 spinors, FP32 links in the
// paired layout).
//
// Each block owns 128 consecutive sites and NR right-hand sides (grid order as
// in stencil_grid: with the groups fastest, the groups of one site block run
// together and their link tiles come from L2 after the first).  Warp 4 is the producer: lane 0
// copies, for every stored offset d in turn, the tile W_d(n0 .. n0+127) (five
// 2 KB planes of 16-byte element pairs) from global memory into a ring of three
// shared-memory stages with cp.async.bulk, completing the stage's "full"
// mbarrier by transaction count, and refills a stage once the four consumer
// warps have arrived on its "empty" mbarrier.  Warps 0-3 are the consumers:
// one site (and NR right-hand sides) per thread, the arithmetic of bri_pair
// with W_d(n) read from the stage and the neighbour's link W_d(n-d) loaded
// from global memory (mostly an L2 hit, it was streamed by another block).  No
// block barrier is taken inside the offset loop, so the producer runs two
// offsets ahead of the slowest consumer warp and the link stream's memory
// latency hides behind the arithmetic.
//
// Every mbarrier wait is bounded.  A consumer whose wait runs out stops
// computing but keeps waiting (bounded) on the remaining stages, so that no
// copy is still in flight when the block exits, and writes NaN into its
// outputs; the solvers' reductions then report a non-finite value.
#pragma once

#include "stencil.cuh"

namespace bri {

constexpr int kStageSites = 128;
constexpr int kStages = 3;
constexpr unsigned kStageBytes = 5u * kStageSites * 16u;  // five planes of 128 16-byte words
constexpr unsigned kStagedSmem = kStages * kStageBytes + 2 * kStages * 8;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the completion of the phase with the given parity; false after
// 2^16 unsuccessful polls (each poll itself blocks for a bounded time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < (1 << 16); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_copy_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int NR>
__global__ void __launch_bounds__(160, NR == 1 ? 3 : 2)
    bri_kernel_staged(Geom g, float* __restrict__ y, const float* __restrict__ x, const float2* __restrict__ W,
                      const float* __restrict__ cl, float diag, float sgn, int rhs0, int gfirst,
                      const __grid_constant__ HopTable<float> H) {
  const int grp = gfirst ? blockIdx.x : blockIdx.y, blk = gfirst ? blockIdx.y : blockIdx.x;
  extern __shared__ __align__(128) unsigned char smem[];
  float4* tiles = reinterpret_cast<float4*>(smem);  // [stage][plane][site]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  const int V = (int)g.V;
  const int n0 = blk * kStageSites;
  const int nsites = min(kStageSites, V - n0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 4) {  // producer
    if (lane == 0) {
      const float4* W4 = reinterpret_cast<const float4*>(W);
      const uint32_t bytes = 5u * (uint32_t)nsites * 16u;
      for (int j = 0; j < 40; ++j) {
        const int s = j % kStages;
        const uint32_t round = j / kStages;
        // the consumers' arrivals after round - 1 complete phase round - 1 of empty[s];
        // if they never come (a consumer gave up) the refill is skipped
        if (j >= kStages && !mbar_wait(&empty[s], (round - 1) & 1)) continue;
        mbar_arrive_expect_tx(&full[s], bytes);
        for (int k = 0; k < 5; ++k)
          bulk_copy_to_smem(tiles + (s * 5 + k) * kStageSites, W4 + ((int64_t)j * 5 + k) * V + n0,
                            (uint32_t)nsites * 16u, &full[s]);
      }
    }
    return;
  }

  // consumers: one site per thread
  const int t = threadIdx.x;
  const int n = n0 + t;
  const bool site = t < nsites;
  const int64_t rstride = g.V * 24;
  const int rb = rhs0 + grp * NR;  // first right-hand side of this block
  const float* xin = x + (int64_t)rb * rstride;
  int co[4], L[4], str[4];
  {
    int r = site ? n : n0;
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
  Spinor<float> acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) zero(acc[r]);
  bool ok = true;
#pragma unroll 1
  for (int j = 0; j < 40; ++j) {
    const int s = j % kStages;
    if (!mbar_wait(&full[s], (j / kStages) & 1)) ok = false;
    if (ok && site) {
      int mp = 0, mm = 0;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const int d = H.site_d[j][mu];
        mp += wrap(co[mu] + d, L[mu]) * str[mu];
        mm += wrap(co[mu] - d, L[mu]) * str[mu];
      }
      C<float> w[3][3], wm[3][3];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const float4 v = tiles[(s * 5 + k) * kStageSites + t];
        const int e0 = 2 * k, e1 = 2 * k + 1;
        w[e0 / 3][e0 % 3] = C<float>{v.x, v.y};
        if (e1 < 9) w[e1 / 3][e1 % 3] = C<float>{v.z, v.w};
      }
      load_stored_link<float, float2>(wm, W, j, mm, V);
      bri_pair<float, NR>(acc, xin, rstride, mp, mm, w, wm, H.a[j], sgn * H.cs[j][0], sgn * H.cs[j][1],
                          sgn * H.cs[j][2], sgn * H.cs[j][3]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (!site) return;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    Spinor<float> xc;
    load_spinor(xc, xin + r * rstride + (int64_t)n * 24);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        acc[r].v[s][aa].re = fmaf(diag, xc.v[s][aa].re, acc[r].v[s][aa].re);
        acc[r].v[s][aa].im = fmaf(diag, xc.v[s][aa].im, acc[r].v[s][aa].im);
      }
    if (cl) add_clover(acc[r], xc, cl, g.V, n);
    if (!ok) {
      const float nan = __int_as_float(0x7fc00000);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) acc[r].v[s][aa] = C<float>{nan, nan};
    }
    store_spinor(y + (int64_t)rb * rstride + r * rstride + (int64_t)n * 24, acc[r]);
  }
}

}  // namespace bri
