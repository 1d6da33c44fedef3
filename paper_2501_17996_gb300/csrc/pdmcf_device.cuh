// pdmcf_device.cuh — sm_103a kernels of one PDMCF iteration (Zhang & Boyd, Algorithm 2.1).
//
// Layout in HBM (edge-major, so every per-edge or per-node vector is one coalesced
// stream of 16-byte words):
//   Ft[e][i]  = F_{i,l(e)}      m x ld, S (float | double | bf16), e = internal edge id
//                               (edges sorted by head), ld = n rounded up to 8
//   Yt[j][i]  = Y_{i,j}         n x ld, P (float | double)   — ping-pong pair
//   Pt[j][i]  = (F A^T)_{i,j}   n x ld, P  — kept for the relaxation identity below
//   Wt[j][i]  = w_{i,j}         n x ld, P
// Pad entries i in [n, ld) are zero in every array and stay zero.
//
// One iteration k (Eq. e-pdhg-step, Algorithm 2.1 step 2) is three launches:
//   edge_kernel   per edge l: q = f + alpha (Y_{:,head} - Y_{:,tail}), formed relative to the
//                 previous multiplier; mu by Newton on phi(mu) = sum (q - mu)_+ - c (the
//                 capped-simplex projection of Sec. 2.3), f^ = (q - mu)_+,
//                 f_new = rho f^ + (1 - rho) f; ||dF||^2 (FP32 per thread, FP64 across).
//                 Variants: edge_insum_kernel (in-sums of F^{k+1/2} per head, so the node
//                 phase gathers out-edges only) and edge_tma_kernel (bulk-copy pipeline).
//   node_kernel   per node j: p = sum_{in(j)} f_new - sum_{out(j)} f_new = (F^{k+1/2}A^T)_{:,j},
//                 F^ A^T = (p - (1-rho) P_old)/rho, F^{k+1} A^T = 2 F^ A^T - P_old,
//                 v = Y_{:,j} - beta F^{k+1}A^T, Y^ = prox(v) (0 at i = j),
//                 Y_new = rho Y^ + (1 - rho) Y (head FP32 + tail BF16 for FP32 iterates);
//                 ||dY||^2 and, in the check variant, the objective/conjugate/consistency
//                 partials.
//   scalar_kernel one block: fixed-order FP64 reductions, the primal weight rule of
//                 Eq. (e-primal_weight), alpha/beta for the next iteration and, on check
//                 iterations, r (Eq. e-res), the duality gap and the relative KKT measure.
// plus check_kernel (per edge, check iterations only) for ||G||^2, <G, F^-Q>, ||F^-Q||^2
// and the linear part of the dual bound.
//
// The F^{k+1} A^T identity: F^{k+1/2} = rho F^ + (1-rho) F^{k-1/2}, so
// F^ A^T = (F^{k+1/2} A^T - (1-rho) F^{k-1/2} A^T) / rho and F^{k+1} = 2 F^ - F^{k-1/2};
// the node phase therefore needs only the freshly written F^{k+1/2} rows and the n x n
// state P = F^{k-1/2} A^T, never a stored F^{k+1}.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#include <type_traits>

#include "pdmcf_types.h"

namespace pdmcf {

// ------------------------------------------------------------------ element helpers

template <typename S> struct StoreTraits;
template <> struct StoreTraits<float>  { static constexpr int VW = 4; };
template <> struct StoreTraits<double> { static constexpr int VW = 2; };
template <> struct StoreTraits<__nv_bfloat16> { static constexpr int VW = 8; };

template <typename P> __device__ __forceinline__ P to_p(float x) { return (P)x; }
template <typename P> __device__ __forceinline__ P to_p(double x) { return (P)x; }
template <typename P> __device__ __forceinline__ P to_p(__nv_bfloat16 x) { return (P)__bfloat162float(x); }

template <typename S, typename P> __device__ __forceinline__ S from_p(P x);
template <> __device__ __forceinline__ float from_p<float, float>(float x) { return x; }
template <> __device__ __forceinline__ double from_p<double, double>(double x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_p<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}

// 16-byte (or, for 8-byte chunks, 8-byte) vector loads/stores. "stream" = touched once per
// pass (evict-first), "keep" = read-only data that other CTAs re-read soon (default caching).
template <typename T, int N>
__device__ __forceinline__ void ld_keep(const T* p, T (&v)[N]) {
  static_assert((N * sizeof(T)) % 16 == 0 || N * sizeof(T) == 8, "8- or 16-byte words");
  if constexpr (N * sizeof(T) == 8) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    memcpy(&v[0], &u, 8);
  } else {
    constexpr int W = N * (int)sizeof(T) / 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + k);
      memcpy(&v[k * 16 / sizeof(T)], &u, 16);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void ld_stream(const T* p, T (&v)[N]) {
  if constexpr (N * sizeof(T) == 8) {
    uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    memcpy(&v[0], &u, 8);
  } else {
    constexpr int W = N * (int)sizeof(T) / 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint4 u = __ldcs(reinterpret_cast<const uint4*>(p) + k);
      memcpy(&v[k * 16 / sizeof(T)], &u, 16);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void ld_plain(const T* p, T (&v)[N]) {
  if constexpr (N * sizeof(T) == 8) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    memcpy(&v[0], &u, 8);
  } else {
    constexpr int W = N * (int)sizeof(T) / 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint4 u = *(reinterpret_cast<const uint4*>(p) + k);
      memcpy(&v[k * 16 / sizeof(T)], &u, 16);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void st_stream(T* p, const T (&v)[N]) {
  if constexpr (N * sizeof(T) == 8) {
    uint2 u;
    memcpy(&u, &v[0], 8);
    __stcs(reinterpret_cast<uint2*>(p), u);
  } else {
    constexpr int W = N * (int)sizeof(T) / 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint4 u;
      memcpy(&u, &v[k * 16 / sizeof(T)], 16);
      __stcs(reinterpret_cast<uint4*>(p) + k, u);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void st_plain(T* p, const T (&v)[N]) {
  if constexpr (N * sizeof(T) == 8) {
    uint2 u;
    memcpy(&u, &v[0], 8);
    *reinterpret_cast<uint2*>(p) = u;
  } else {
    constexpr int W = N * (int)sizeof(T) / 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint4 u;
      memcpy(&u, &v[k * 16 / sizeof(T)], 16);
      *(reinterpret_cast<uint4*>(p) + k) = u;
    }
  }
}

// Chunk width of the head-aligned kinds (bulk-copy and in-sum edge phases and their node
// phase): 4 entries whatever the storage type of F, so a BF16 row has as many chunks as an
// FP32 one (its F words are 8 bytes, its Y words 16) and the 512-thread groups stay as full.
template <typename S> struct RowTraits { static constexpr int VW = 4; };


// ------------------------------------------------------------------ TMA bulk copies + mbarrier
// 1-D bulk copies global -> shared (cp.async.bulk) completing on an mbarrier; sizes and
// addresses are multiples of 16 bytes. Every wait is bounded.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Returns false if the phase did not complete within 2^22 polls or 2 s, whichever comes first
// (a poll may suspend for a system-dependent time, so the deadline bounds the wall clock).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned source) into L2: a hint with
// no completion to wait for and no destination in this CTA.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ group reductions
// A "group" is GROUP consecutive threads that own one edge (or node): a warp when
// GROUP == 32, the whole block when GROUP == blockDim.x > 32. All threads of a group get
// the same result (butterfly sums are commutative pairwise, so every lane sees the same
// rounding; block sums read the per-warp partials in one fixed order).

template <int GROUP> struct GroupScratch {
  static constexpr int NW = GROUP > 32 ? GROUP / 32 : 1;
  double s[2][NW];
  int c[2][NW];
  double x[2][NW];
  float sf[2][NW];   // FP32 partials stay FP32: a double round trip would run on the FP64 pipe
  float xf[2][NW];
  float mnf[2][NW];  // per-warp minima / maxima of the projection's certificates
  float mxf[2][NW];
  double mnd[2][NW];
  double mxd[2][NW];
};

// Cross-warp stage of a block-wide group reduction: lane l < NW of every warp loads warp
// l's partial and a butterfly over NW lanes finishes it. Every warp evaluates the same
// tree on the same values, so all threads agree bit for bit. NW is a power of two.
template <int NW, typename T, typename Op>
__device__ __forceinline__ T cross_warp(T mine_if_lane_lt_nw, T ident, Op op) {
  T v = mine_if_lane_lt_nw;
#pragma unroll
  for (int o = NW / 2; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  (void)ident;
  return __shfl_sync(0xffffffffu, v, 0);
}

template <int GROUP, typename P>
__device__ __forceinline__ void group_sum_count(P& s, int& c, GroupScratch<GROUP>& sh, int& phase) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if constexpr (GROUP > 32) {
    constexpr int NW = GROUP / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P ps;
    if constexpr (std::is_same<P, float>::value) {
      if (lane == 0) { sh.sf[phase][warp] = s; sh.c[phase][warp] = c; }
      __syncthreads();
      ps = lane < NW ? sh.sf[phase][lane] : 0.f;
    } else {
      if (lane == 0) { sh.s[phase][warp] = (double)s; sh.c[phase][warp] = c; }
      __syncthreads();
      ps = lane < NW ? (P)sh.s[phase][lane] : P(0);
    }
    int pc = lane < NW ? sh.c[phase][lane] : 0;
    s = cross_warp<NW>(ps, P(0), [](P a, P b) { return a + b; });
    c = cross_warp<NW>(pc, 0, [](int a, int b) { return a + b; });
    phase ^= 1;
  }
}

// Warp-wide minimum / maximum, the same value in every lane: one redux instruction for
// FP32, a butterfly for FP64.
__device__ __forceinline__ float warp_min(float v) {
  float r;
  asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float warp_max(float v) {
  float r;
  asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Group-wide statistics of one projection pass: the sum and count of the active entries
// (the same butterfly as group_sum_count, so the sum is bitwise the same), the smallest
// active entry and, with IMAX, the largest inactive one.
template <int GROUP, bool IMAX, typename P>
__device__ __forceinline__ void group_stats(P& s, int& c, P& amin, P& imax,
                                            GroupScratch<GROUP>& sh, int& phase) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  c = __reduce_add_sync(0xffffffffu, c);
  amin = warp_min(amin);
  if constexpr (IMAX) imax = warp_max(imax);
  if constexpr (GROUP > 32) {
    constexpr int NW = GROUP / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P ps, pmn, pmx = P(0);
    if constexpr (std::is_same<P, float>::value) {
      if (lane == 0) {
        sh.sf[phase][warp] = s;
        sh.c[phase][warp] = c;
        sh.mnf[phase][warp] = amin;
        if constexpr (IMAX) sh.mxf[phase][warp] = imax;
      }
      __syncthreads();
      ps = lane < NW ? sh.sf[phase][lane] : 0.f;
      pmn = lane < NW ? sh.mnf[phase][lane] : INFINITY;
      if constexpr (IMAX) pmx = lane < NW ? sh.mxf[phase][lane] : -INFINITY;
    } else {
      if (lane == 0) {
        sh.s[phase][warp] = (double)s;
        sh.c[phase][warp] = c;
        sh.mnd[phase][warp] = (double)amin;
        if constexpr (IMAX) sh.mxd[phase][warp] = (double)imax;
      }
      __syncthreads();
      ps = lane < NW ? (P)sh.s[phase][lane] : P(0);
      pmn = lane < NW ? (P)sh.mnd[phase][lane] : (P)INFINITY;
      if constexpr (IMAX) pmx = lane < NW ? (P)sh.mxd[phase][lane] : (P)(-INFINITY);
    }
    const int pc = lane < NW ? sh.c[phase][lane] : 0;
    s = cross_warp<NW>(ps, P(0), [](P a, P b) { return a + b; });
    c = __reduce_add_sync(0xffffffffu, pc);
    amin = warp_min(pmn);
    if constexpr (IMAX) imax = warp_max(pmx);
    phase ^= 1;
  }
}

template <int GROUP, typename P>
__device__ __forceinline__ P group_max(P v, GroupScratch<GROUP>& sh, int& phase) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if constexpr (GROUP > 32) {
    constexpr int NW = GROUP / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P pv;
    if constexpr (std::is_same<P, float>::value) {
      if (lane == 0) sh.xf[phase][warp] = v;
      __syncthreads();
      pv = lane < NW ? sh.xf[phase][lane] : -INFINITY;
    } else {
      if (lane == 0) sh.x[phase][warp] = (double)v;
      __syncthreads();
      pv = lane < NW ? (P)sh.x[phase][lane] : (P)(-INFINITY);
    }
    v = cross_warp<NW>(pv, (P)(-INFINITY), [](P a, P b) { return fmax(a, b); });
    phase ^= 1;
  }
  return v;
}

// Group-wide sum of one double (same value in every thread of the group).
template <int GROUP>
__device__ __forceinline__ double group_sum_double(double v, GroupScratch<GROUP>& sh, int& phase) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if constexpr (GROUP > 32) {
    constexpr int NW = GROUP / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh.x[phase][warp] = v;
    __syncthreads();
    double pv = lane < NW ? sh.x[phase][lane] : 0.0;
    v = cross_warp<NW>(pv, 0.0, [](double a, double b) { return a + b; });
    phase ^= 1;
  }
  return v;
}

// Block-wide sum of K doubles per thread, written by thread 0 to out[0..K).
template <int BLOCK, int K>
__device__ __forceinline__ void block_sum_write(double (&v)[K], double* out) {
  __shared__ double red[K][BLOCK / 32];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int w = 0; w < BLOCK / 32; ++w) t += red[k][w];
      out[k] = t;
    }
  }
}

// ------------------------------------------------------------------ utilities (Sec. 1.1, 2.3)

// prox_{beta (-u)^*}(y) for u = w log s: (y - sqrt(y^2 + 4 beta w))/2 (Sec. 2.3), evaluated
// as -2 beta w / (y + sqrt(...)) when y > 0 to avoid cancellation (same value).
template <typename P>
__device__ __forceinline__ P prox_log(P y, P beta, P w) {
  const P bw = beta * w;
  const P s = sqrt(fma(y, y, P(4) * bw));
  return y <= P(0) ? P(0.5) * (y - s) : (P(-2) * bw) / (y + s);
}

// prox_{beta (-u)^*}(y) for u = w s^gamma: z = -t, t the root of
// h(t) = t^(c1+1) (t + y) - K (Sec. 2.3), c1 = gamma/(1-gamma), K = c1 c2,
// c2 = beta (1/gamma - 1)(w gamma)^(1/(1-gamma)). h is increasing and convex on
// t >= t_lo = max(0, -y), so Newton from any point right of the root decreases
// monotonically to it. The start is the smaller of two upper bounds of the root (derived):
//   y >= 0: t^(c1+2) < K and t^(c1+1) y < K, so t < min(K^(1/(c1+2)), (K/y)^(1/(c1+1)));
//   y < 0:  t = -y + d with t > |y| and t >= d, so d < min(K^(1/(c1+2)), K/|y|^(c1+1)).
// In each regime the bound that applies is within a factor 4 of the root (the other term
// of h is at most the dominant one there), so a handful of Newton steps reach FP
// precision; the plain start t_lo + K^(1/(c1+2)) can be orders of magnitude too far right,
// where each step only shrinks t by a constant factor. gamma = 1/2 (c1 = 1) is a cubic and
// needs no transcendental calls beyond one cube root and one square root.
template <typename P>
__device__ __forceinline__ P newton_quot(P h, P dh) { return h / dh; }
template <>
__device__ __forceinline__ float newton_quot<float>(float h, float dh) {
  return __fdividef(h, dh);   // a Newton correction: its last-bit rounding does not matter
}

template <typename P>
__device__ __forceinline__ P prox_pow(P y, P beta, P w, P gamma) {
  const P tlo = y < P(0) ? -y : P(0);
  P t, k;
  if (gamma == P(0.5)) {
    k = beta * P(0.25) * w * w;                       // c1 c2 with c1 = 1
    const P b1 = cbrt(k);
    if (y >= P(0)) t = y > P(0) ? fmin(b1, sqrt(k / y)) : b1;
    else t = tlo + fmin(b1, k / (y * y));
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
      const P h = t * t * (t + y) - k;
      const P dh = t * (P(3) * t + P(2) * y);
      P tn = t - newton_quot<P>(h, dh);
      tn = tn < tlo ? tlo : tn;
      if (!(tn < t)) break;
      t = tn;
    }
  } else {
    const P c1 = gamma / (P(1) - gamma);
    k = c1 * beta * (P(1) / gamma - P(1)) * pow(w * gamma, P(1) / (P(1) - gamma));
    const P b1 = pow(k, P(1) / (c1 + P(2)));
    if (y >= P(0)) t = y > P(0) ? fmin(b1, pow(k / y, P(1) / (c1 + P(1)))) : b1;
    else t = tlo + fmin(b1, k / pow(tlo, c1 + P(1)));
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
      const P p = pow(t, c1);
      const P h = p * t * (t + y) - k;
      const P dh = p * ((c1 + P(2)) * t + (c1 + P(1)) * y);
      P tn = t - newton_quot<P>(h, dh);
      tn = tn < tlo ? tlo : tn;
      if (!(tn < t)) break;
      t = tn;
    }
  }
  return -t;
}

template <typename P>
__device__ __forceinline__ P util_value(int kind, P t, P w, P g) {      // u(t)
  if (kind == 0) return w * log(t);
  return g == P(0.5) ? w * sqrt(t) : w * pow(t, g);
}
template <typename P>
__device__ __forceinline__ P util_grad(int kind, P t, P w, P g) {       // u'(t)
  if (kind == 0) return w / t;
  return g == P(0.5) ? P(0.5) * w / sqrt(t) : w * g * pow(t, g - P(1));
}
// (-u)^*(y), y < 0: log: w log(w/(-y)) - w ; power: (1/g - 1)(w g)^(1/(1-g)) (-y)^(-g/(1-g))
template <typename P>
__device__ __forceinline__ P util_conj_neg(int kind, P y, P w, P g) {
  if (kind == 0) return w * log(w / (-y)) - w;
  if (g == P(0.5)) return P(0.25) * w * w / (-y);
  return (P(1) / g - P(1)) * pow(w * g, P(1) / (P(1) - g)) * pow(-y, -g / (P(1) - g));
}
// (u')^{-1}(-y): the traffic whose marginal utility is -y
template <typename P>
__device__ __forceinline__ P util_traffic(int kind, P y, P w, P g) {
  if (kind == 0) return w / (-y);
  if (g == P(0.5)) { const P x = w / (P(-2) * y); return x * x; }   // (w gamma/(-y))^2
  return pow(w * g / (-y), P(1) / (P(1) - g));
}


// ------------------------------------------------------------------ compensated duals
// Y is stored as an FP32 head plus a BF16 tail (Y = hi + lo), which holds the rounding error
// of the head: edge differences Y_{:,h} - Y_{:,t} are formed as (hi_h - hi_t) + (lo_h - lo_t)
// and the dual update is applied in increment form, so FP32 iterates are not limited by the
// FP32 spacing of the (large) dual values.

template <int N>
__device__ __forceinline__ void ld_lo(const __nv_bfloat16* p, float (&v)[N]) {
  static_assert(N == 2 || N == 4 || N == 8, "lo chunk");
  if constexpr (N == 8) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __bfloat162float(b[k]);
  } else if constexpr (N == 4) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __bfloat162float(b[k]);
  } else {
    unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
    v[0] = __bfloat162float(b[0]);
    v[1] = __bfloat162float(b[1]);
  }
}

template <int N>
__device__ __forceinline__ void st_lo(__nv_bfloat16* p, const float (&v)[N]) {
  __nv_bfloat16 b[N];
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = __float2bfloat16_rn(v[k]);
  if constexpr (N == 8) *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(b);
  else if constexpr (N == 4) *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(b);
  else *reinterpret_cast<unsigned*>(p) = *reinterpret_cast<const unsigned*>(b);
}

// hi + lo + x as a new (hi, lo): Fast2Sum (|hi| >= |lo + x| holds for the tails used here;
// when hi = 0 the sum is exact anyway).
template <typename P>
__device__ __forceinline__ void add_split(P& hi, P& lo, P x) {
  const P t = lo + x;
  const P s = hi + t;
  lo = (hi - s) + t;
  hi = s;
}

// t = T(Y^), the traffic of the prox output Y^ = prox_{beta(-u)^*}(v) = v - beta t
// (Moreau's identity): for log utility t = (v + sqrt(v^2 + 4 beta w)) / (2 beta), evaluated
// as 2w / (sqrt(v^2 + 4 beta w) - v) when v <= 0; for power utility t = (u')^{-1}(-Y^) from
// the dual root. Both are small traffic-scale numbers with relative accuracy ~ulp.
template <typename P>
__device__ __forceinline__ P prox_traffic(int kind, P v, P beta, P w, P g) {
  if (kind == 0) {
    const P s = sqrt(fma(v, v, P(4) * beta * w));
    return v <= P(0) ? (P(2) * w) / (s - v) : (v + s) / (P(2) * beta);
  }
  const P z = prox_pow<P>(v, beta, w, g);
  return util_traffic<P>(kind, z, w, g);
}

// ------------------------------------------------------------------ scalar tail

// Deterministic sum of base[b*stride + field] over b < nb by 256 threads: contiguous
// per-thread segments, then a fixed binary tree.
static __device__ __forceinline__ double det_sum(const double* base, int nb, int stride, int field, double* sh) {
  const int per = (nb + 255) / 256;
  const int b0 = threadIdx.x * per;
  const int b1 = min(nb, b0 + per);
  double s = 0.0;
  for (int b = b0; b < b1; ++b) s += base[(size_t)b * stride + field];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Scalar tail of one iteration (thread 0 of the reducing block): Delta_F, Delta_Y, on check
// iterations r (Eq. e-res), the dual bound and the relative KKT parts, then the primal weight
// rule (Eq. e-primal_weight) and alpha/beta for the next iteration.
static __device__ __forceinline__ void scalar_update(DevScalars* s, double dF2, double dY2,
                                                     const double* nodep, const double* chk,
                                                     bool check) {
  const double inf = INFINITY;
  const double dF = sqrt(dF2), dY = sqrt(dY2);
  s->dF = dF;
  s->dY = dY;
  if (!isfinite(dF) || !isfinite(dY)) s->numeric_error = 1;
  const long long k = s->k;
  if (check) {
    const double nonpos = nodep[1], Psum = nodep[2], conj = nodep[3], cons2 = nodep[4];
    const double t2 = nodep[5], ybad = nodep[6];
    const double g2 = chk[0], gd = chk[1], d2 = chk[2], lin = chk[3];
    const bool feasible = nonpos == 0.0;
    // Eq. (e-res): r = ||G||^2 - <G,D>^2/||D||^2 if D != 0 and <G,D> >= 0, else ||G||^2
    double r = inf;
    if (feasible) {
      r = (d2 == 0.0 || gd < 0.0) ? g2 : g2 - gd * gd / d2;
      if (r < 0.0) r = 0.0;
    }
    const double P = feasible ? Psum : -inf;
    const double D = ybad > 0.0 ? inf : conj + lin;
    s->feasible = feasible ? 1 : 0;
    s->r = r;
    s->P = P;
    s->D = D;
    s->g_norm = sqrt(g2);
    s->rel_gap = (feasible && isfinite(D)) ? (D - P) / (1.0 + fabs(P) + fabs(D)) : inf;
    s->rel_cons = ybad > 0.0 ? inf : sqrt(cons2) / (1.0 + sqrt(t2));
    s->rel_stat = feasible ? sqrt(r) / (1.0 + sqrt(g2)) : inf;
    s->rel_kkt = fmax(s->rel_gap, fmax(s->rel_cons, s->rel_stat));
    s->nonpos_frac = nonpos / ((double)s->n * (double)(s->n - 1));
    s->check_k = k + 1;
    if (!isfinite(Psum) && feasible) s->numeric_error = 1;
  }
  // Algorithm 2.1, step 3 (Eq. e-primal_weight)
  s->alpha_last = s->alpha;
  s->beta_last = s->beta;
  if (k % s->k_adapt == 0 && dF > s->tau && dY > s->tau && (s->freeze < 0 || k < s->freeze)) {
    s->omega = pow(dY / dF, s->theta) * pow(s->omega, 1.0 - s->theta);
  }
  // Sec. 2.4: omega may stop adapting after some iterations (a constant omega keeps the
  // convergence proof). omega_ref records omega at the first check with a finite measure,
  // omega_arm at the first one with a measure below guard_below (the final phase). At every
  // later check, omega stops adapting from the next iteration once it leaves a factor
  // guard^2 of omega_ref, or, in the final phase, once it leaves a factor guard of
  // omega_arm or a finite measure exceeds guard x its best.
  if (check && s->guard > 0.0) {
    const bool fin = isfinite(s->rel_kkt);
    const double g2 = s->guard * s->guard;
    const bool drift_ref = s->omega_ref > 0.0 &&
                           (s->omega > g2 * s->omega_ref || s->omega * g2 < s->omega_ref);
    const bool final_phase = s->omega_arm > 0.0 &&
                             ((fin && s->rel_kkt > s->guard * s->best_kkt) ||
                              s->omega > s->guard * s->omega_arm ||
                              s->omega * s->guard < s->omega_arm);
    if ((drift_ref || final_phase) && (s->freeze < 0 || s->freeze > k + 1)) s->freeze = k + 1;
    if (fin) {
      if (s->rel_kkt < s->best_kkt) s->best_kkt = s->rel_kkt;
      if (s->omega_ref == 0.0) s->omega_ref = s->omega;
      if (s->omega_arm == 0.0 && s->best_kkt < s->guard_below) s->omega_arm = s->omega;
    }
  }
  s->alpha = s->eta / s->omega;
  s->beta = s->eta * s->omega;
  s->k = k + 1;
}

// ------------------------------------------------------------------ kernel arguments

template <typename P, typename S>
struct IterArgs {
  int n, m, ld;
  const int32_t* e_tail;
  const int32_t* e_head;
  const int32_t* in_ptr;
  const int32_t* out_ptr;
  const int32_t* out_idx;
  const P* cap;
  S* F[2];
  P* Y[2];
  __nv_bfloat16* Ylo[2];  // tails of the compensated duals (nullptr: plain Y)
  P* Pm;
  const P* W;
  const P* Gm;        // per-pair gamma (n x ld) or nullptr
  P gamma;            // scalar gamma when Gm == nullptr
  int kind;           // 0 log, 1 power
  P* mu;          // projection multipliers: mu + mu_lo (hi/lo pair), one per edge
  P* mu_lo;
  P* That;
  P* Uprime;
  P* Yhat;
  double* part_edge;  // [grid_edge]
  double* part_node;  // [grid_node * NODE_PARTS]
  double* part_check; // [grid_edge * CHECK_PARTS]
  P* Pin;             // n x ld: sum_{in(j)} F^{k+1/2} per head j (pipelined edge phase only)
  const int32_t* cta_ptr;  // [grid + 1] head-aligned edge ranges of the pipelined edge phase
  DevScalars* sc;
  P rho;
  int parity;         // F[parity], Y[parity] hold F^{k-1/2}, Y^k; the other slot receives k+1
  int check;          // 1 on check iterations
  int withhold;       // testing aid (bulk-copy edge phase): block 0 arms its first stage for
                      // copies it never issues, so that stage's bounded wait runs out
};

// ------------------------------------------------------------------ projection

// Entries of q in the frame shifted by the previous multiplier mu0 = m0 + m0l (a hi/lo pair).
// On the active set q = f + alpha (y_h - y_t) and mu are both about alpha times the edge's
// price, far above f^ = (q - mu)_+; subtracting mu0 before the projection (y_h - y_t taken
// exactly by TwoSum, alpha (y_h - y_t) - m0 rounded once by an FMA) keeps the rounding of f^
// at the scale of f^ and f rather than of alpha * price. The capped-simplex projection is
// shift-invariant; its floor mu >= 0 becomes nu >= -m0 for nu = mu - mu0.
template <typename P>
__device__ __forceinline__ P shifted_q(P f, P yh, P yt, P dl, P alpha, P m0, P m0l) {
  const P s = yh - yt;
  const P bb = s - yh;
  const P err = (yh - (s - bb)) - (yt + bb);
  return f + (fma(alpha, s, -m0) + fma(alpha, err + dl, -m0l));
}

// The floor of nu: -(m0 + m0l) rounded, the value shifted_q gives a zero entry (f = 0,
// y_h = y_t = 0, e.g. the row padding), which therefore never enters the active set.
template <typename P>
__device__ __forceinline__ P shifted_floor(P m0, P m0l) { return -m0 - m0l; }

// mu = mu0 + nu as a hi/lo pair (TwoSum, then renormalised); nu at the floor gives mu = 0.
template <typename P>
__device__ __forceinline__ void shifted_mu(P m0, P m0l, P nu, P& hi, P& lo) {
  if (nu <= shifted_floor<P>(m0, m0l)) { hi = P(0); lo = P(0); return; }
  const P s = m0 + nu;
  const P bb = s - m0;
  const P l = ((m0 - (s - bb)) + (nu - bb)) + m0l;
  hi = s + l;
  lo = l - (hi - s);
}

// ------------------------------------------------------------------ packed FP32 pairs
// sm_100-class SMs issue two FP32 adds, multiplies or FMAs as one instruction
// (add/sub/mul/fma.rn.f32x2); each lane is rounded exactly like the scalar operation, so the
// packed code gives bitwise the scalar results with half the instructions.
__device__ __forceinline__ float2 p2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 p2(float x) { return make_float2(x, x); }

// shifted_q on a pair of entries (the same operations in the same order, packed).
__device__ __forceinline__ float2 shifted_q2(float2 f, float2 yh, float2 yt, float2 dl,
                                             float2 alpha, float2 nm0, float2 nm0l) {
  const float2 s = p2_sub(yh, yt);
  const float2 bb = p2_sub(s, yh);
  const float2 err = p2_sub(p2_sub(yh, p2_sub(s, bb)), p2_add(yt, bb));
  return p2_add(f, p2_add(p2_fma(alpha, s, nm0), p2_fma(alpha, p2_add(err, dl), nm0l)));
}

// Capped-simplex projection of one column (Sec. 2.3): mu = 0 if sum (q)_+ <= c, else the
// root of phi(mu) = sum_i (q_i - mu)_+ - c. phi is convex, decreasing and piecewise
// linear, so Newton from a point left of the root, mu' = (sum_{q>mu} q - c)/#{q > mu},
// rises monotonically and stops exactly when the active set {q > mu} no longer changes
// (then mu = (sum_active q - c)/|active|, the value the sorted scan of Sec. 2.6 finds).
// The previous iteration's mu is the starting point; if it lies right of the root, one
// Newton step from there lands at or left of the root (tangents of a convex function lie
// below it). `lo` is the floor of mu: 0 for q itself, -mu0 in the shifted frame above.
//
// Each pass also returns the smallest active entry (and, on the first pass, the largest
// inactive one). A Newton step mu -> mu' keeps the active set exactly when no entry lies
// between them: mu' < min{q > mu} going right, mu' >= max{q <= mu} going left. Then
// phi(mu') = 0 and mu' is returned without a confirming pass; the value is bitwise the one
// the confirming pass would have accepted (same active set, same fixed-order sum).
// The entries are this thread's N values get(0..N-1), in a fixed order (the order of the
// thread's partial sums, so every layout of the same values gives the same multiplier).
template <int GROUP, int N, typename P, typename Get>
__device__ __forceinline__ P project_mu_n(Get get, P c, P mu0, P lo, GroupScratch<GROUP>& sh,
                                          int& phase) {
  auto eval = [&](P mu, P& s, int& cnt, P& amin, P& imax, auto want_imax) {
    constexpr bool IM = decltype(want_imax)::value;
    P ls = 0, am = (P)INFINITY, im = (P)(-INFINITY);
    int lc = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const P x = get(i);
      if (x > mu) { ls += x; ++lc; am = fmin(am, x); }
      else if constexpr (IM) { im = fmax(im, x); }
    }
    group_stats<GROUP, IM, P>(ls, lc, am, im, sh, phase);
    s = ls; cnt = lc; amin = am;
    if constexpr (IM) imax = im;
  };
  using with_imax = std::true_type;
  using without_imax = std::false_type;
  P mu = mu0 > lo ? mu0 : lo;
  P s, amin, imax;
  int cnt;
  eval(mu, s, cnt, amin, imax, with_imax{});
  P phi = s - (P)cnt * mu - c;
  if (phi <= P(0)) {
    if (mu == lo || phi == P(0)) return mu;            // at the floor, or exactly at the root
    P mn = cnt > 0 ? (s - c) / (P)cnt : lo;            // Newton step from the right
    if (mn <= lo) {
      mu = lo;
      eval(mu, s, cnt, amin, imax, without_imax{});
      if (s - (P)cnt * lo - c <= P(0)) return lo;
    } else {
      if (cnt > 0 && mn >= imax) return mn;            // no inactive entry joins: the root
      mu = mn;
      eval(mu, s, cnt, amin, imax, without_imax{});
    }
  }
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    if (cnt == 0) break;
    const P mn = (s - c) / (P)cnt;
    if (!(mn > mu)) break;
    if (mn < amin) return mn;                          // no active entry leaves: the root
    mu = mn;
    eval(mu, s, cnt, amin, imax, without_imax{});
  }
  return mu;
}

template <int GROUP, int VPT, int VW, typename P>
__device__ __forceinline__ P project_mu(const P (&q)[VPT][VW], P c, P mu0, P lo,
                                        GroupScratch<GROUP>& sh, int& phase) {
  return project_mu_n<GROUP, VPT * VW, P>([&](int i) { return q[i / VW][i % VW]; }, c, mu0, lo,
                                          sh, phase);
}

// The same on entries held as FP32 pairs (q[v][p] = entries 2p and 2p+1 of chunk v).
template <int GROUP, int VPT, int H>
__device__ __forceinline__ float project_mu2(const float2 (&q)[VPT][H], float c, float mu0,
                                             float lo, GroupScratch<GROUP>& sh, int& phase) {
  return project_mu_n<GROUP, VPT * H * 2, float>(
      [&](int i) { const float2 z = q[i / (2 * H)][(i % (2 * H)) / 2]; return (i & 1) ? z.y : z.x; },
      c, mu0, lo, sh, phase);
}

// ------------------------------------------------------------------ edge phase

template <typename P, typename S, int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
edge_kernel(IterArgs<P, S> a) {
  constexpr int VW = StoreTraits<S>::VW;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int nchunks = a.ld / VW;
  const P alpha = (P)a.sc->alpha;
  const P rho = a.rho;
  const S* __restrict__ Fo = a.F[a.parity];
  S* __restrict__ Fn = a.F[a.parity ^ 1];
  const P* __restrict__ Y = a.Y[a.parity];
  const __nv_bfloat16* __restrict__ ylo = a.Ylo[a.parity];
  P dsum = P(0);   // this thread's ||dF||^2 over its edges (FP64 across threads)

  int nh = 0, nt = 0;
  P nc = P(0), nmu = P(0), nmul = P(0);
  if (gid < a.m) {
    nh = a.e_head[gid]; nt = a.e_tail[gid]; nc = a.cap[gid]; nmu = a.mu[gid]; nmul = a.mu_lo[gid];
  }
  for (int e = gid; e < a.m; e += ngroups) {
    const int h = nh, t = nt;
    const P c = nc;
    const P mu0 = nmu, mu0l = nmul;
    if (e + ngroups < a.m) {   // next edge's indices and scalars, one edge ahead
      nh = a.e_head[e + ngroups];
      nt = a.e_tail[e + ngroups];
      nc = a.cap[e + ngroups];
      nmu = a.mu[e + ngroups];
      nmul = a.mu_lo[e + ngroups];
      // and its rows into L2 while this edge is projected (rows are 16-byte aligned and
      // ld * element size is a multiple of 16)
      if (lane == 0) {
        prefetch_l2(Fo + (size_t)(e + ngroups) * a.ld, (uint32_t)(a.ld * sizeof(S)));
        prefetch_l2(Y + (size_t)nt * a.ld, (uint32_t)(a.ld * sizeof(P)));
        prefetch_l2(Y + (size_t)nh * a.ld, (uint32_t)(a.ld * sizeof(P)));
        if (ylo) {
          prefetch_l2(ylo + (size_t)nt * a.ld, (uint32_t)(a.ld * 2));
          prefetch_l2(ylo + (size_t)nh * a.ld, (uint32_t)(a.ld * 2));
        }
      }
    }
    const S* fo = Fo + (size_t)e * a.ld;
    const P* yh = Y + (size_t)h * a.ld;
    const P* yt = Y + (size_t)t * a.ld;
    P q[VPT][VW], f[VPT][VW];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        S fs[VW]; P a1[VW], a2[VW];
        ld_stream<S, VW>(fo + ci * VW, fs);
        ld_keep<P, VW>(yh + ci * VW, a1);
        ld_keep<P, VW>(yt + ci * VW, a2);
        P dl[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) dl[u] = P(0);
        if constexpr (std::is_same<P, float>::value) {
          if (ylo) {
            float l1[VW], l2[VW];
            ld_lo<VW>(ylo + (size_t)h * a.ld + ci * VW, l1);
            ld_lo<VW>(ylo + (size_t)t * a.ld + ci * VW, l2);
#pragma unroll
            for (int u = 0; u < VW; ++u) dl[u] = l1[u] - l2[u];
          }
        }
        if constexpr (std::is_same<P, float>::value) {   // packed pairs, same rounding
#pragma unroll
          for (int u = 0; u < VW; u += 2) {
            const float2 ff = make_float2(to_p<P>(fs[u]), to_p<P>(fs[u + 1]));
            const float2 qq = shifted_q2(ff, make_float2(a1[u], a1[u + 1]),
                                         make_float2(a2[u], a2[u + 1]),
                                         make_float2(dl[u], dl[u + 1]), p2(alpha), p2(-mu0),
                                         p2(-mu0l));
            f[v][u] = ff.x; f[v][u + 1] = ff.y;
            q[v][u] = qq.x; q[v][u + 1] = qq.y;
          }
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) {
            f[v][u] = to_p<P>(fs[u]);
            q[v][u] = shifted_q<P>(f[v][u], a1[u], a2[u], dl[u], alpha, mu0, mu0l);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < VW; ++u) { f[v][u] = P(0); q[v][u] = shifted_floor<P>(mu0, mu0l); }
      }
    }
    const P mu = project_mu<GROUP, VPT, VW, P>(q, c, P(0), shifted_floor<P>(mu0, mu0l), sh, phase);
    P dloc = P(0);   // this thread's part of ||dF||^2 for this edge; FP64 across edges
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        S out[VW];
        if constexpr (std::is_same<P, float>::value) {
          // f_new = f + rho (f^ - f) and (f^ - f)^2 on packed pairs; rho^2 is applied per edge
          float2 sq = p2(0.f);
#pragma unroll
          for (int u = 0; u < VW; u += 2) {
            const float2 ff = make_float2(f[v][u], f[v][u + 1]);
            const float2 t2 = p2_add(make_float2(q[v][u], q[v][u + 1]), p2(-mu));
            const float2 fh = make_float2(fmaxf(t2.x, 0.f), fmaxf(t2.y, 0.f));
            const float2 st = p2_sub(fh, ff);
            const float2 fnew = p2_fma(p2(rho), st, ff);
            sq = p2_fma(st, st, sq);
            out[u] = from_p<S, P>(fnew.x);
            out[u + 1] = from_p<S, P>(fnew.y);
          }
          dloc += rho * rho * (sq.x + sq.y);
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) {
            const P fh = q[v][u] > mu ? q[v][u] - mu : P(0);
            const P fnew = rho * fh + (P(1) - rho) * f[v][u];
            out[u] = from_p<S, P>(fnew);
            // Delta_F uses the step rho (f^ - f) itself: the rounding of the stored iterate
            // (about one ulp per entry) would otherwise swamp Delta_F near convergence and
            // drive the primal weight rule
            const P d = rho * (fh - f[v][u]);
            dloc = fma(d, d, dloc);
          }
        }
        st_stream<S, VW>(Fn + (size_t)e * a.ld + ci * VW, out);
      }
    }
    dsum += dloc;
    if (lane == 0) {
      P hi, lo;
      shifted_mu<P>(mu0, mu0l, mu, hi, lo);
      a.mu[e] = hi;
      a.mu_lo[e] = lo;
    }
  }
  double v1[1] = {(double)dsum};
  block_sum_write<BLOCK, 1>(v1, a.part_edge + blockIdx.x);
}

// ------------------------------------------------------------------ node phase

// CHECK: the variant for check iterations, which also evaluates U(T^), (-u)^*(Y^), the
// consistency and domain counts and writes T^, U'(T^) and Y^ (the other variant keeps only
// what every iteration needs, and fewer registers).
template <typename P, typename S, int VPT, int GROUP, int BLOCK, int MINB, bool PIN, bool CHECK>
__global__ void __launch_bounds__(BLOCK, MINB)
node_kernel(IterArgs<P, S> a) {
  // the in-sum (PIN) variant pairs with the head-aligned edge phases and their chunk width
  constexpr int VW = PIN ? RowTraits<S>::VW : StoreTraits<S>::VW;
  constexpr int GPB = BLOCK / GROUP;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int nchunks = a.ld / VW;
  const P beta = (P)a.sc->beta;
  const P rho = a.rho;
  const P inv_rho = P(1) / rho;
  const S* __restrict__ Fn = a.F[a.parity ^ 1];
  const P* __restrict__ Yo = a.Y[a.parity];
  P* __restrict__ Yn = a.Y[a.parity ^ 1];
  // partials: 0 ||dY||^2, 1 #nonpositive T, 2 sum u(T), 3 sum (-u)^*(Y^), 4 ||T(Y^)-T||^2,
  //           5 ||T||^2, 6 #(Y^ >= 0 off-diagonal)
  double acc[NODE_PARTS];
#pragma unroll
  for (int k = 0; k < NODE_PARTS; ++k) acc[k] = 0.0;

  for (int j = gid; j < a.n; j += ngroups) {
    // p_j = sum_{in(j)} f_new - sum_{out(j)} f_new. With PIN the edge phase already summed
    // the in-edges into Pin[j]. One 16-byte chunk at a time: its sum over the node's rows
    // (four rows in flight, added as consecutive pairs), then the dual update of that chunk,
    // so only one chunk's accumulator is live.
    const int ib = a.in_ptr[j], nin = PIN ? 0 : a.in_ptr[j + 1] - ib;
    const int ob = a.out_ptr[j], deg = nin + (a.out_ptr[j + 1] - ob);
    const bool pin_rows = PIN && a.in_ptr[j + 1] > ib;   // only heads of some edge were written
    auto row = [&](int k) -> const S* {
      return Fn + (size_t)(k < nin ? ib + k : a.out_idx[ob + k - nin]) * a.ld;
    };
    P loc[NODE_PARTS];
#pragma unroll
    for (int k = 0; k < NODE_PARTS; ++k) loc[k] = P(0);
    P* prow = a.Pm + (size_t)j * a.ld;
    const P* yrow = Yo + (size_t)j * a.ld;
    const P* wrow = a.W + (size_t)j * a.ld;
    const P* grow = a.Gm ? a.Gm + (size_t)j * a.ld : nullptr;
#pragma unroll 1
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci >= nchunks) break;
      P s[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) s[u] = P(0);
      if (pin_rows) ld_plain<P, VW>(a.Pin + (size_t)j * a.ld + ci * VW, s);
      int k = 0;
      if constexpr (sizeof(S) == 2 && VW == 4) {
        // 8-byte BF16 words: eight rows in flight keep as many bytes in flight as four FP32
        // rows; the rows are added in the same pairs and order as below
        for (; k + 7 < deg; k += 8) {
          S fr[8][VW];
#pragma unroll
          for (int r = 0; r < 8; ++r) ld_plain<S, VW>(row(k + r) + ci * VW, fr[r]);
#pragma unroll
          for (int r = 0; r < 8; r += 2) {
            const P sa = k + r < nin ? P(1) : P(-1), sb = k + r + 1 < nin ? P(1) : P(-1);
#pragma unroll
            for (int u = 0; u < VW; ++u) s[u] += sa * to_p<P>(fr[r][u]) + sb * to_p<P>(fr[r + 1][u]);
          }
        }
      }
      for (; k + 3 < deg; k += 4) {
        const S* r0 = row(k);
        const S* r1 = row(k + 1);
        const S* r2 = row(k + 2);
        const S* r3 = row(k + 3);
        S f0[VW], f1[VW], f2[VW], f3[VW];
        ld_plain<S, VW>(r0 + ci * VW, f0);
        ld_plain<S, VW>(r1 + ci * VW, f1);
        ld_plain<S, VW>(r2 + ci * VW, f2);
        ld_plain<S, VW>(r3 + ci * VW, f3);
        const P s0 = k < nin ? P(1) : P(-1), s1 = k + 1 < nin ? P(1) : P(-1);
        const P s2 = k + 2 < nin ? P(1) : P(-1), s3 = k + 3 < nin ? P(1) : P(-1);
#pragma unroll
        for (int u = 0; u < VW; ++u) s[u] += s0 * to_p<P>(f0[u]) + s1 * to_p<P>(f1[u]);
#pragma unroll
        for (int u = 0; u < VW; ++u) s[u] += s2 * to_p<P>(f2[u]) + s3 * to_p<P>(f3[u]);
      }
      if (k + 1 < deg) {
        const S* r0 = row(k);
        const S* r1 = row(k + 1);
        S f0[VW], f1[VW];
        ld_plain<S, VW>(r0 + ci * VW, f0);
        ld_plain<S, VW>(r1 + ci * VW, f1);
        const P s0 = k < nin ? P(1) : P(-1), s1 = k + 1 < nin ? P(1) : P(-1);
#pragma unroll
        for (int u = 0; u < VW; ++u) s[u] += s0 * to_p<P>(f0[u]) + s1 * to_p<P>(f1[u]);
        k += 2;
      }
      if (k < deg) {
        S f0[VW];
        ld_plain<S, VW>(row(k) + ci * VW, f0);
        const P s0 = k < nin ? P(1) : P(-1);
#pragma unroll
        for (int u = 0; u < VW; ++u) s[u] += s0 * to_p<P>(f0[u]);
      }
      P po[VW], yo[VW], wv[VW], gv[VW], yn[VW];
      ld_plain<P, VW>(prow + ci * VW, po);
      ld_plain<P, VW>(yrow + ci * VW, yo);
      ld_keep<P, VW>(wrow + ci * VW, wv);
      if (grow) ld_keep<P, VW>(grow + ci * VW, gv);
      else {
#pragma unroll
        for (int u = 0; u < VW; ++u) gv[u] = a.gamma;
      }
      P that_v[VW], up_v[VW], yh_v[VW];
      P yl[VW];                    // tail of the compensated dual (0 when plain)
#pragma unroll
      for (int u = 0; u < VW; ++u) yl[u] = P(0);
      if constexpr (std::is_same<P, float>::value) {
        if (a.Ylo[a.parity]) ld_lo<VW>(a.Ylo[a.parity] + (size_t)j * a.ld + ci * VW, yl);
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const int i = ci * VW + u;
        const P fhat_at = (s[u] - (P(1) - rho) * po[u]) * inv_rho;   // (F^ A^T)_{ij}
        const P fplus_at = P(2) * fhat_at - po[u];                       // (F^{k+1} A^T)_{ij}
        const bool live = (i < a.n) && (i != j);
        // Y^ - Y = -beta (F^{k+1}A^T + t), t = T(Y^) (Moreau): the increment is formed from
        // traffic-scale quantities; Y^ = 0 on the diagonal and in the pads.
        P delta, tr = P(0);
        if (live) {
          const P vv = yo[u] + (yl[u] - beta * fplus_at);
          tr = prox_traffic<P>(a.kind, vv, beta, wv[u], gv[u]);
          delta = -beta * (fplus_at + tr);
        } else {
          delta = -(yo[u] + yl[u]);
        }
        const P yhat = live ? (yo[u] + (yl[u] + delta)) : P(0);
        P hi = yo[u], lo = yl[u];
        add_split(hi, lo, rho * delta);                                  // Y + rho (Y^ - Y)
        yn[u] = hi;
        yl[u] = lo;
        const P dy = rho * delta;
        loc[0] = fma(dy, dy, loc[0]);
        const P th = -fhat_at;
        that_v[u] = i < a.n ? th : P(0);
        yh_v[u] = yhat;
        up_v[u] = P(0);
        if (CHECK && live) {
          if (!(th > P(0))) loc[1] += P(1);
          else {
            loc[2] += util_value<P>(a.kind, th, wv[u], gv[u]);
            up_v[u] = util_grad<P>(a.kind, th, wv[u], gv[u]);
          }
          if (yhat < P(0)) {
            loc[3] += util_conj_neg<P>(a.kind, yhat, wv[u], gv[u]);
            const P dt = tr - th;
            loc[4] = fma(dt, dt, loc[4]);
          } else {
            loc[6] += P(1);
          }
          loc[5] = fma(th, th, loc[5]);
        }
      }
      if constexpr (std::is_same<P, float>::value) {
        if (a.Ylo[a.parity ^ 1]) st_lo<VW>(a.Ylo[a.parity ^ 1] + (size_t)j * a.ld + ci * VW, yl);
      }
      st_plain<P, VW>(Yn + (size_t)j * a.ld + ci * VW, yn);
      st_plain<P, VW>(prow + ci * VW, s);
      if constexpr (CHECK) {
        st_plain<P, VW>(a.That + (size_t)j * a.ld + ci * VW, that_v);
        st_plain<P, VW>(a.Uprime + (size_t)j * a.ld + ci * VW, up_v);
        st_plain<P, VW>(a.Yhat + (size_t)j * a.ld + ci * VW, yh_v);
      }
    }
#pragma unroll
    for (int k = 0; k < NODE_PARTS; ++k) acc[k] += (double)loc[k];
  }
  block_sum_write<BLOCK, NODE_PARTS>(acc, a.part_node + (size_t)blockIdx.x * NODE_PARTS);
}


// ------------------------------------------------------------------ pipelined edge phase
// Large n: one CTA of 512 threads per SM walks a contiguous, head-aligned range of edges.
// The F^{k-1/2} row and the Y_{:,tail} row of each edge arrive in shared memory by 1-D bulk
// copies into two stages; as soon as edge i has been read into registers its stage is
// refilled with edge i+2, so the copies overlap edge i's projection and edge i+1 is ready
// when edge i is stored. Y_{:,head} stays in registers for the whole head group, and the
// group's in-sum of F^{k+1/2} is written to Pin[head] so the node phase only gathers
// out-edges.
template <typename S, int VPT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
edge_tma_kernel(IterArgs<float, S> a) {
  using P = float;
  constexpr int VW = RowTraits<S>::VW;
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ GroupScratch<BLOCK> sh;
  __shared__ int ok_flag;
  int phase = 0;
  const int tid = threadIdx.x;
  const int nchunks = a.ld / VW;
  const uint32_t frow = (uint32_t)a.ld * (uint32_t)sizeof(S);
  const uint32_t yrow = (uint32_t)a.ld * (uint32_t)sizeof(P);
  S* sF[2] = {(S*)dyn, (S*)(dyn + frow + yrow)};
  P* sY[2] = {(P*)(dyn + frow), (P*)(dyn + 2 * frow + yrow)};
  const int e0 = a.cta_ptr[blockIdx.x];
  const int cnt = a.cta_ptr[blockIdx.x + 1] - e0;
  const P alpha = (P)a.sc->alpha;
  const P rho = a.rho;
  const S* __restrict__ Fo = a.F[a.parity];
  S* __restrict__ Fn = a.F[a.parity ^ 1];
  const P* __restrict__ Y = a.Y[a.parity];
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    ok_flag = 1;
    fence_proxy_async();
  }
  __syncthreads();
  auto issue = [&](int i) {   // thread 0: bring edge e0+i into stage i&1
    const int e = e0 + i, st = i & 1;
    mbar_arrive_expect_tx(&full[st], frow + yrow);
    if (a.withhold && blockIdx.x == 0 && i == 0) return;   // the copies never come
    tma_load_1d(sF[st], Fo + (size_t)e * a.ld, frow, &full[st]);
    tma_load_1d(sY[st], Y + (size_t)a.e_tail[e] * a.ld, yrow, &full[st]);
  };
  if (tid == 0) {
    if (cnt > 0) issue(0);
    if (cnt > 1) issue(1);
  }
  P dsum = P(0);   // this thread's ||dF||^2 over its edges (FP64 across threads)
  int cur_h = -1;
  const __nv_bfloat16* __restrict__ ylo = a.Ylo[a.parity];
  P yh[VPT][VW], yhl[VPT][VW], sin_[VPT][VW];   // head's Y (hi, tail) and the in-sum
#pragma unroll
  for (int v = 0; v < VPT; ++v)
#pragma unroll
    for (int u = 0; u < VW; ++u) { yh[v][u] = P(0); yhl[v][u] = P(0); sin_[v][u] = P(0); }
  // per-edge scalars of the next edge are fetched one edge ahead (off the critical path)
  int nx_h = cnt > 0 ? a.e_head[e0] : 0;
  P nx_c = cnt > 0 ? a.cap[e0] : P(0), nx_mu = cnt > 0 ? a.mu[e0] : P(0);
  P nx_mul = cnt > 0 ? a.mu_lo[e0] : P(0);

  for (int i = 0; i < cnt; ++i) {
    const int e = e0 + i, st = i & 1;
    const int h = nx_h;
    const P c_e = nx_c, mu_e = nx_mu, mu_el = nx_mul;
    if (i + 1 < cnt) {
      nx_h = a.e_head[e + 1];
      nx_c = a.cap[e + 1];
      nx_mu = a.mu[e + 1];
      nx_mul = a.mu_lo[e + 1];
    }
    if (h != cur_h) {   // new head group: flush the in-sum, fetch Y_{:,h} while we wait
      if (cur_h >= 0) {
        P* pr = a.Pin + (size_t)cur_h * a.ld;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int ci = v * BLOCK + tid;
          if (ci < nchunks) st_plain<P, VW>(pr + ci * VW, sin_[v]);
        }
      }
      const P* yr = Y + (size_t)h * a.ld;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int ci = v * BLOCK + tid;
        if (ci < nchunks) {
          ld_keep<P, VW>(yr + ci * VW, yh[v]);
          if (ylo) ld_lo<VW>(ylo + (size_t)h * a.ld + ci * VW, yhl[v]);
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) sin_[v][u] = P(0);
      }
      cur_h = h;
    }
    if (tid == 0 && !mbar_wait_bounded(&full[st], (uint32_t)((i >> 1) & 1))) ok_flag = 0;
    __syncthreads();
    if (!ok_flag) {   // a copy never completed: report, drain what is in flight, leave
      if (tid == 0) {
        a.sc->wait_timeout = 1;
        mbar_wait_bounded(&full[st], (uint32_t)((i >> 1) & 1));
        if (i + 1 < cnt) mbar_wait_bounded(&full[st ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
      }
      return;
    }
    P f[VPT][VW], q[VPT][VW];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) {
        S fs[VW];
        P yt[VW], dl[VW];
        ld_plain<S, VW>(sF[st] + ci * VW, fs);
        ld_plain<P, VW>(sY[st] + ci * VW, yt);
#pragma unroll
        for (int u = 0; u < VW; ++u) dl[u] = P(0);
        if (ylo) {
          float l[VW];
          ld_lo<VW>(ylo + (size_t)a.e_tail[e] * a.ld + ci * VW, l);
#pragma unroll
          for (int u = 0; u < VW; ++u) dl[u] = yhl[v][u] - l[u];
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          f[v][u] = to_p<P>(fs[u]);
          q[v][u] = shifted_q<P>(f[v][u], yh[v][u], yt[u], dl[u], alpha, mu_e, mu_el);
        }
      } else {
#pragma unroll
        for (int u = 0; u < VW; ++u) { f[v][u] = P(0); q[v][u] = shifted_floor<P>(mu_e, mu_el); }
      }
    }
    __syncthreads();   // every thread is done with stage st: refill it with edge i+2
    if (tid == 0 && i + 2 < cnt) {
      fence_proxy_async();
      issue(i + 2);
    }
    const P mu = project_mu<BLOCK, VPT, VW, P>(q, c_e, P(0), shifted_floor<P>(mu_e, mu_el), sh, phase);
    P dloc = P(0);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) {
        S out[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          const P fh = q[v][u] > mu ? q[v][u] - mu : P(0);
          out[u] = from_p<S, P>(rho * fh + (P(1) - rho) * f[v][u]);
          const P fnew = to_p<P>(out[u]);
          sin_[v][u] += fnew;
          const P d = rho * (fh - f[v][u]);   // the step itself (see edge_kernel)
          dloc = fma(d, d, dloc);
        }
        st_stream<S, VW>(Fn + (size_t)e * a.ld + ci * VW, out);
      }
    }
    dsum += dloc;
    if (tid == 0) {
      P hi, lo;
      shifted_mu<P>(mu_e, mu_el, mu, hi, lo);
      a.mu[e] = hi;
      a.mu_lo[e] = lo;
    }
  }
  if (cur_h >= 0) {
    P* pr = a.Pin + (size_t)cur_h * a.ld;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) st_plain<P, VW>(pr + ci * VW, sin_[v]);
    }
  }
  double v1[1] = {(double)dsum};
  block_sum_write<BLOCK, 1>(v1, a.part_edge + blockIdx.x);
}


// ------------------------------------------------------------------ edge phase with in-sums
// The register edge phase over head-aligned contiguous edge ranges (one range per CTA, two
// CTAs per SM): Y_{:,head} and the running in-sum of F^{k+1/2} live in this thread's slices
// of shared memory (each thread touches only its own chunk positions, so no barriers are
// added), and the in-sum is written to Pin[head] when the head changes, so the node phase
// gathers only out-edges. One thread prefetches the next edge's F row and Y_{:,tail} row
// into L2 while this edge is projected, and the per-entry arithmetic runs on packed FP32
// pairs (FP32 iterates only).
template <typename P, typename S, int VPT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 2)
edge_insum_kernel(IterArgs<P, S> a) {
  static_assert(std::is_same<P, float>::value, "in-sum edge phase: FP32 iterates");
  constexpr int VW = RowTraits<S>::VW;
  extern __shared__ __align__(16) unsigned char dyn_is[];
  P* yh_s = reinterpret_cast<P*>(dyn_is);
  P* sin_s = yh_s + a.ld;
  __shared__ GroupScratch<BLOCK> sh;
  int phase = 0;
  const int tid = threadIdx.x;
  const int nchunks = a.ld / VW;
  const float alpha_s = (float)a.sc->alpha;
  const float2 alpha = p2(alpha_s);
  const float2 rho = p2(a.rho);
  const S* __restrict__ Fo = a.F[a.parity];
  S* __restrict__ Fn = a.F[a.parity ^ 1];
  const P* __restrict__ Y = a.Y[a.parity];
  const __nv_bfloat16* __restrict__ ylo = a.Ylo[a.parity];
  const int e0 = a.cta_ptr[blockIdx.x], e1 = a.cta_ptr[blockIdx.x + 1];
  const uint32_t frow = (uint32_t)a.ld * (uint32_t)sizeof(S);   // multiples of 16 bytes
  const uint32_t yrow = (uint32_t)a.ld * 4u;
  float2 dsum = p2(0.f);   // this thread's sum of (f^ - f)^2 over its edges (x rho^2 at the end)
  int cur_h = -1;
  auto flush = [&](int hh) {
    P* pr = a.Pin + (size_t)hh * a.ld;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) {
        P x[VW];
        ld_plain<P, VW>(sin_s + ci * VW, x);
        st_plain<P, VW>(pr + ci * VW, x);
      }
    }
  };
  int nh = 0, nt = 0;
  P nc = P(0), nmu = P(0), nmul = P(0);
  if (e0 < e1) {
    nh = a.e_head[e0]; nt = a.e_tail[e0]; nc = a.cap[e0]; nmu = a.mu[e0]; nmul = a.mu_lo[e0];
  }
  for (int e = e0; e < e1; ++e) {
    const int h = nh, t = nt;
    const P c = nc, mu0 = nmu, mu0l = nmul;
    if (e + 1 < e1) {
      nh = a.e_head[e + 1];
      nt = a.e_tail[e + 1];
      nc = a.cap[e + 1];
      nmu = a.mu[e + 1];
      nmul = a.mu_lo[e + 1];
      if (tid == 0) {   // the next edge's streamed rows, into L2 during this edge's projection
        prefetch_l2(Fo + (size_t)(e + 1) * a.ld, frow);
        prefetch_l2(Y + (size_t)nt * a.ld, yrow);
        if (ylo) prefetch_l2(ylo + (size_t)nt * a.ld, yrow / 2);
      }
    }
    if (h != cur_h) {   // new head group: flush, then stage Y_{:,h} (its tail stays in L1/L2)
      if (cur_h >= 0) flush(cur_h);
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int ci = v * BLOCK + tid;
        if (ci < nchunks) {
          P y[VW], z[VW];
          ld_keep<P, VW>(Y + (size_t)h * a.ld + ci * VW, y);
#pragma unroll
          for (int u = 0; u < VW; ++u) z[u] = P(0);
          st_plain<P, VW>(yh_s + ci * VW, y);
          st_plain<P, VW>(sin_s + ci * VW, z);
        }
      }
      cur_h = h;
    }
    const S* fo = Fo + (size_t)e * a.ld;
    const P* yt = Y + (size_t)t * a.ld;
    const float2 nm0 = p2(-mu0), nm0l = p2(-mu0l);
    constexpr int H = VW / 2;
    float2 q[VPT][H], f[VPT][H];   // entry pairs: whole 64-bit registers for the packed ops
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) {
        S fs[VW];
        P a1[VW], a2[VW], l1[VW], l2[VW];
        ld_stream<S, VW>(fo + ci * VW, fs);
        ld_plain<P, VW>(yh_s + ci * VW, a1);
        ld_stream<P, VW>(yt + ci * VW, a2);   // read once per edge: streamed, not kept in L1
        if (ylo) {
          ld_lo<VW>(ylo + (size_t)h * a.ld + ci * VW, l1);
          ld_lo<VW>(ylo + (size_t)t * a.ld + ci * VW, l2);
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) { l1[u] = 0.f; l2[u] = 0.f; }
        }
#pragma unroll
        for (int u = 0; u < VW; u += 2) {
          const float2 ff = make_float2(to_p<P>(fs[u]), to_p<P>(fs[u + 1]));
          const float2 dl = p2_sub(make_float2(l1[u], l1[u + 1]), make_float2(l2[u], l2[u + 1]));
          f[v][u / 2] = ff;
          q[v][u / 2] = shifted_q2(ff, make_float2(a1[u], a1[u + 1]),
                                   make_float2(a2[u], a2[u + 1]), dl, alpha, nm0, nm0l);
        }
      } else {
#pragma unroll
        for (int h = 0; h < H; ++h) { f[v][h] = p2(0.f); q[v][h] = p2(shifted_floor<P>(mu0, mu0l)); }
      }
    }
    const P mu = project_mu2<BLOCK, VPT, H>(q, c, P(0), shifted_floor<P>(mu0, mu0l), sh, phase);
    const float2 nmu2 = p2(-mu);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * BLOCK + tid;
      if (ci < nchunks) {
        S out[VW];
        P acc[VW];
        ld_plain<P, VW>(sin_s + ci * VW, acc);
#pragma unroll
        for (int u = 0; u < VW; u += 2) {
          const float2 ff = f[v][u / 2];
          const float2 t2 = p2_add(q[v][u / 2], nmu2);
          const float2 fh = make_float2(fmaxf(t2.x, 0.f), fmaxf(t2.y, 0.f));   // (q - mu)_+
          const float2 st = p2_sub(fh, ff);                                      // f^ - f
          const float2 fnew = p2_fma(rho, st, ff);        // rho f^ + (1 - rho) f
          dsum = p2_fma(st, st, dsum);
          out[u] = from_p<S, P>(fnew.x);
          out[u + 1] = from_p<S, P>(fnew.y);
          const float2 sum = p2_add(make_float2(acc[u], acc[u + 1]),
                                    make_float2(to_p<P>(out[u]), to_p<P>(out[u + 1])));
          acc[u] = sum.x; acc[u + 1] = sum.y;
        }
        st_stream<S, VW>(Fn + (size_t)e * a.ld + ci * VW, out);
        st_plain<P, VW>(sin_s + ci * VW, acc);
      }
    }
    if (tid == 0) {
      P hi, lo;
      shifted_mu<P>(mu0, mu0l, mu, hi, lo);
      a.mu[e] = hi;
      a.mu_lo[e] = lo;
    }
  }
  if (cur_h >= 0) flush(cur_h);
  // Delta_F uses the step rho (f^ - f) itself, not the rounded stored iterate (see edge_kernel)
  const float r2 = a.rho * a.rho;
  double v1[1] = {(double)(r2 * (dsum.x + dsum.y))};
  block_sum_write<BLOCK, 1>(v1, a.part_edge + blockIdx.x);
}

// ------------------------------------------------------------------ check (residual) phase
// Per edge: Q column from F^{k-1/2} and Y^k, F^ = (q - mu)_+ with the mu just computed,
// D = F^ - Q, G = U'_{:,head} - U'_{:,tail}; partial sums of ||G||^2, <G,D>, ||D||^2
// (Eq. e-res) and c_l max(0, max_i (Y^ A)_il) for the dual bound.
template <typename P, typename S, int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
check_kernel(IterArgs<P, S> a) {
  constexpr int VW = StoreTraits<S>::VW;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int nchunks = a.ld / VW;
  const P alpha = (P)a.sc->alpha;
  const S* __restrict__ Fo = a.F[a.parity];
  const P* __restrict__ Y = a.Y[a.parity];
  double acc[CHECK_PARTS] = {0.0, 0.0, 0.0, 0.0};
  for (int e = gid; e < a.m; e += ngroups) {
    const int h = a.e_head[e], t = a.e_tail[e];
    const P mu = a.mu[e];
    const size_t fo = (size_t)e * a.ld, ho = (size_t)h * a.ld, to = (size_t)t * a.ld;
    P ymax = -INFINITY;
    P lg2 = P(0), lgd = P(0), ld2 = P(0);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci >= nchunks) continue;
      S fs[VW];
      P y1[VW], y2[VW], g1[VW], g2[VW], z1[VW], z2[VW];
      ld_plain<S, VW>(Fo + fo + ci * VW, fs);
      ld_keep<P, VW>(Y + ho + ci * VW, y1);
      ld_keep<P, VW>(Y + to + ci * VW, y2);
      ld_keep<P, VW>(a.Uprime + ho + ci * VW, g1);
      ld_keep<P, VW>(a.Uprime + to + ci * VW, g2);
      ld_keep<P, VW>(a.Yhat + ho + ci * VW, z1);
      ld_keep<P, VW>(a.Yhat + to + ci * VW, z2);
      P dl[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) dl[u] = P(0);
      if constexpr (std::is_same<P, float>::value) {
        if (a.Ylo[a.parity]) {
          float l1[VW], l2[VW];
          ld_lo<VW>(a.Ylo[a.parity] + ho + ci * VW, l1);
          ld_lo<VW>(a.Ylo[a.parity] + to + ci * VW, l2);
#pragma unroll
          for (int u = 0; u < VW; ++u) dl[u] = l1[u] - l2[u];
        }
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const int i = ci * VW + u;
        if (i >= a.n) continue;
        const P q = to_p<P>(fs[u]) + alpha * ((y1[u] - y2[u]) + dl[u]);
        const P fh = q > mu ? q - mu : P(0);
        const P d = fh - q;
        const P g = g1[u] - g2[u];
        lg2 = fma(g, g, lg2);
        lgd = fma(g, d, lgd);
        ld2 = fma(d, d, ld2);
        ymax = fmax(ymax, z1[u] - z2[u]);
      }
    }
    acc[0] += (double)lg2;
    acc[1] += (double)lgd;
    acc[2] += (double)ld2;
    ymax = group_max<GROUP, P>(ymax, sh, phase);
    if (lane == 0 && ymax > P(0)) acc[3] += (double)a.cap[e] * (double)ymax;
  }
  block_sum_write<BLOCK, CHECK_PARTS>(acc, a.part_check + (size_t)blockIdx.x * CHECK_PARTS);
}

// ------------------------------------------------------------------ standalone projection
// Pi of Sec. 2.3 applied to m columns given as rows of Qt (edge-major, ld >= n floats per
// row): Ft row l = (q_l - mu_l)_+, mu in/out (warm start in, multipliers out), and the
// per-column FP64 squared distance ||Pi(q_l) - q_l||^2 into col_d2[l]. Entries n..ld-1 of
// Qt are ignored; those of Ft are written as zero.
struct ProjArgs {
  int n, m, ld;
  const float* Qt;
  const float* cap;
  float* Ft;
  float* mu;
  double* col_d2;
};

template <int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
project_kernel(ProjArgs a) {
  constexpr int VW = 4;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int nchunks = a.ld / VW;
  for (int e = gid; e < a.m; e += ngroups) {
    const float* qr = a.Qt + (size_t)e * a.ld;
    float q[VPT][VW];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        ld_stream<float, VW>(qr + ci * VW, q[v]);
#pragma unroll
        for (int u = 0; u < VW; ++u)
          if (ci * VW + u >= a.n) q[v][u] = 0.f;       // pads never enter the active set
      } else {
#pragma unroll
        for (int u = 0; u < VW; ++u) q[v][u] = 0.f;
      }
    }
    const float mu0 = a.mu[e];
    const float mu = project_mu<GROUP, VPT, VW, float>(q, a.cap[e], mu0 > 0.f ? mu0 : 0.f, 0.f, sh, phase);
    float dloc = 0.f;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        float out[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          out[u] = q[v][u] > mu ? q[v][u] - mu : 0.f;
          const float d = out[u] - q[v][u];
          dloc = fmaf(d, d, dloc);
        }
        st_stream<float, VW>(a.Ft + (size_t)e * a.ld + ci * VW, out);
      }
    }
    const double d2 = group_sum_double<GROUP>((double)dloc, sh, phase);
    if (lane == 0) {
      a.mu[e] = mu;
      a.col_d2[e] = d2;
    }
  }
}

}  // namespace pdmcf
