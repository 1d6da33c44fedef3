// pdmcf_batch.cuh — batched PDMCF iteration: many independent instances of different sizes
// advanced by one launch per phase (Algorithm 2.1, step 2, for every resident instance).
//
// Instances are grouped into classes by launch shape. A class launch walks a global work
// list (all edges, or all nodes, of the class's instances) with a grid-stride loop; the
// owning instance of a work item is found by binary search in the class's prefix sums.
// Each instance keeps its scalars (k, parity, alpha, beta, omega, stop state) on the device,
// so kernels decide on their own whether an iteration is a check iteration and whether the
// instance is still active; a captured iteration therefore replays for any mix.
// Reductions are per work item (one FP64 value per edge and per node, summed in a fixed
// order by the instance's own scalar block), so an instance's iterates are bit-identical
// whether it runs alone or with others.
#pragma once

#include "pdmcf_device.cuh"

namespace pdmcf {

struct BatchScalars {
  DevScalars s;            // shared fields (step sizes, k, check results, ...)
  int parity;              // F[parity], Y[parity] hold F^{k-1/2}, Y^k
  int active;              // 1 while the instance iterates
  int done;                // set by the scalar kernel when the stop rule holds
  int stop_mode;           // MCF_STOP_*
  long long max_iters;
  long long k_check;
  double eps;
  int stall_checks;        // stall rule (see mcf_options.stall_checks)
  int stall_count;
  int stalled;
  double stall_best;
  int stall_frozen;        // omega had stopped adapting when the count last restarted
};

struct BatchInst {
  int n, m, ld, kind;
  float gamma, rho;
  const int32_t* e_tail;
  const int32_t* e_head;
  const int32_t* in_ptr;
  const int32_t* out_ptr;
  const int32_t* out_idx;
  const float* cap;
  const float* W;
  const float* Gm;
  float* F[2];
  float* Y[2];
  __nv_bfloat16* Ylo[2];   // compensated-dual tails (nullptr: plain Y)
  float* Pm;
  float* mu;               // projection multipliers, hi/lo pair
  float* mu_lo;
  float* That;
  float* Uprime;
  float* Yhat;
  double* pe;              // [m] per-edge ||dF||^2 parts
  double* pn;              // [n * NODE_PARTS] per-node parts
  double* pc;              // [m * CHECK_PARTS] per-edge check parts
  BatchScalars* sc;
};

struct BatchClassDev {
  const int* count;        // number of instances in the class (device, so graphs replay)
  const int* inst;         // [count] indices into the instance table
  const long long* eoff;   // [count + 1] edge prefix sums
  const long long* noff;   // [count + 1] node prefix sums
};

__device__ __forceinline__ int batch_find(const long long* off, int count, long long g) {
  int lo = 0, hi = count - 1;            // largest b with off[b] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool batch_is_check(const BatchScalars* sc) {
  const long long k1 = sc->s.k + 1;
  return (k1 % sc->k_check) == 0 || k1 >= sc->max_iters;
}

// ------------------------------------------------------------------ edge phase

template <int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
batch_edge_kernel(const BatchInst* __restrict__ insts, BatchClassDev cls) {
  using P = float;
  constexpr int VW = 4;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int count = *cls.count;
  if (count == 0) return;
  const long long total = cls.eoff[count];
  for (long long g = gid; g < total; g += ngroups) {
    const int b = batch_find(cls.eoff, count, g);
    const BatchInst& I = insts[cls.inst[b]];
    const BatchScalars* sc = I.sc;
    if (!sc->active) continue;
    const int e = (int)(g - cls.eoff[b]);
    const int par = sc->parity;
    const P alpha = (P)sc->s.alpha;
    const P rho = I.rho;
    const int nchunks = I.ld / VW;
    const int h = I.e_head[e], t = I.e_tail[e];
    const P mu0 = I.mu[e], mu0l = I.mu_lo[e];
    const float* fo = I.F[par] + (size_t)e * I.ld;
    const float* yh = I.Y[par] + (size_t)h * I.ld;
    const float* yt = I.Y[par] + (size_t)t * I.ld;
    P q[VPT][VW], f[VPT][VW];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        P a1[VW], a2[VW], dl[VW];
        ld_plain<P, VW>(fo + ci * VW, f[v]);
        ld_plain<P, VW>(yh + ci * VW, a1);
        ld_plain<P, VW>(yt + ci * VW, a2);
#pragma unroll
        for (int u = 0; u < VW; ++u) dl[u] = P(0);
        if (I.Ylo[par]) {
          float l1[VW], l2[VW];
          ld_lo<VW>(I.Ylo[par] + (size_t)h * I.ld + ci * VW, l1);
          ld_lo<VW>(I.Ylo[par] + (size_t)t * I.ld + ci * VW, l2);
#pragma unroll
          for (int u = 0; u < VW; ++u) dl[u] = l1[u] - l2[u];
        }
#pragma unroll
        for (int u = 0; u < VW; u += 2) {   // packed pairs, the same rounding as shifted_q
          const float2 qq = shifted_q2(make_float2(f[v][u], f[v][u + 1]),
                                       make_float2(a1[u], a1[u + 1]), make_float2(a2[u], a2[u + 1]),
                                       make_float2(dl[u], dl[u + 1]), p2(alpha), p2(-mu0), p2(-mu0l));
          q[v][u] = qq.x;
          q[v][u + 1] = qq.y;
        }
      } else {
#pragma unroll
        for (int u = 0; u < VW; ++u) { f[v][u] = P(0); q[v][u] = shifted_floor<P>(mu0, mu0l); }
      }
    }
    const P mu = project_mu<GROUP, VPT, VW, P>(q, I.cap[e], P(0), shifted_floor<P>(mu0, mu0l), sh, phase);
    P dloc = P(0);
    float* fn = I.F[par ^ 1] + (size_t)e * I.ld;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci < nchunks) {
        P out[VW];
        float2 sq = p2(0.f);   // (f^ - f)^2, the step itself (not the rounded difference)
#pragma unroll
        for (int u = 0; u < VW; u += 2) {
          const float2 ff = make_float2(f[v][u], f[v][u + 1]);
          const float2 t2 = p2_add(make_float2(q[v][u], q[v][u + 1]), p2(-mu));
          const float2 st = p2_sub(make_float2(fmaxf(t2.x, 0.f), fmaxf(t2.y, 0.f)), ff);
          const float2 fnew = p2_fma(p2(rho), st, ff);   // rho f^ + (1 - rho) f
          sq = p2_fma(st, st, sq);
          out[u] = fnew.x;
          out[u + 1] = fnew.y;
        }
        dloc += rho * rho * (sq.x + sq.y);
        st_plain<P, VW>(fn + ci * VW, out);
      }
    }
    const double d2 = group_sum_double<GROUP>((double)dloc, sh, phase);
    if (lane == 0) {
      P hi, lo;
      shifted_mu<P>(mu0, mu0l, mu, hi, lo);
      I.mu[e] = hi;
      I.mu_lo[e] = lo;
      I.pe[e] = d2;
    }
  }
}

// ------------------------------------------------------------------ node phase

template <int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
batch_node_kernel(const BatchInst* __restrict__ insts, BatchClassDev cls) {
  using P = float;
  constexpr int VW = 4;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int count = *cls.count;
  if (count == 0) return;
  const long long total = cls.noff[count];
  for (long long g = gid; g < total; g += ngroups) {
    const int b = batch_find(cls.noff, count, g);
    const BatchInst& I = insts[cls.inst[b]];
    const BatchScalars* sc = I.sc;
    if (!sc->active) continue;
    const int j = (int)(g - cls.noff[b]);
    const int par = sc->parity;
    const bool check = batch_is_check(sc);
    const P beta = (P)sc->s.beta;
    const P rho = I.rho;
    const P inv_rho = P(1) / rho;
    const int nchunks = I.ld / VW;
    const float* Fn = I.F[par ^ 1];
    const int ib = I.in_ptr[j], nin = I.in_ptr[j + 1] - ib;
    const int ob = I.out_ptr[j], deg = nin + (I.out_ptr[j + 1] - ob);
    auto row = [&](int k) {
      return Fn + (size_t)(k < nin ? ib + k : I.out_idx[ob + k - nin]) * I.ld;
    };
    P loc[NODE_PARTS];
#pragma unroll
    for (int kk = 0; kk < NODE_PARTS; ++kk) loc[kk] = P(0);
    float* prow = I.Pm + (size_t)j * I.ld;
    const float* yrow = I.Y[par] + (size_t)j * I.ld;
    const float* wrow = I.W + (size_t)j * I.ld;
    const float* grow = I.Gm ? I.Gm + (size_t)j * I.ld : nullptr;
    // one 4-entry chunk at a time (only its accumulator is live): the chunk's sum over the
    // node's edge rows, four rows in flight and added in edge order, then its dual update
#pragma unroll 1
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci >= nchunks) continue;
      P sv[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) sv[u] = P(0);
      int k = 0;
      for (; k + 4 <= deg; k += 4) {
        P fr[4][VW];
#pragma unroll
        for (int q = 0; q < 4; ++q) ld_plain<P, VW>(row(k + q) + ci * VW, fr[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const P sg = k + q < nin ? P(1) : P(-1);
#pragma unroll
          for (int u = 0; u < VW; ++u) sv[u] += sg * fr[q][u];
        }
      }
      for (; k < deg; ++k) {
        P fr[VW];
        ld_plain<P, VW>(row(k) + ci * VW, fr);
        const P sg = k < nin ? P(1) : P(-1);
#pragma unroll
        for (int u = 0; u < VW; ++u) sv[u] += sg * fr[u];
      }
      P po[VW], yo[VW], wv[VW], gv[VW], yn[VW], that_v[VW], up_v[VW], yh_v[VW], yl[VW];
      ld_plain<P, VW>(prow + ci * VW, po);
      ld_plain<P, VW>(yrow + ci * VW, yo);
      ld_plain<P, VW>(wrow + ci * VW, wv);
      if (grow) ld_plain<P, VW>(grow + ci * VW, gv);
      else {
#pragma unroll
        for (int u = 0; u < VW; ++u) gv[u] = I.gamma;
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) yl[u] = P(0);
      if (I.Ylo[par]) ld_lo<VW>(I.Ylo[par] + (size_t)j * I.ld + ci * VW, yl);
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const int i = ci * VW + u;
        const P fhat_at = (sv[u] - (P(1) - rho) * po[u]) * inv_rho;
        const P fplus_at = P(2) * fhat_at - po[u];
        const bool live = (i < I.n) && (i != j);
        P delta, tr = P(0);
        if (live) {
          const P vv = yo[u] + (yl[u] - beta * fplus_at);
          tr = prox_traffic<P>(I.kind, vv, beta, wv[u], gv[u]);
          delta = -beta * (fplus_at + tr);
        } else {
          delta = -(yo[u] + yl[u]);
        }
        const P yhat = live ? (yo[u] + (yl[u] + delta)) : P(0);
        P hi = yo[u], lo = yl[u];
        add_split(hi, lo, rho * delta);
        yn[u] = hi;
        yl[u] = lo;
        const P dy = rho * delta;
        loc[0] = fma(dy, dy, loc[0]);
        const P th = -fhat_at;
        that_v[u] = i < I.n ? th : P(0);
        yh_v[u] = yhat;
        up_v[u] = P(0);
        if (check && live) {
          if (!(th > P(0))) loc[1] += P(1);
          else {
            loc[2] += util_value<P>(I.kind, th, wv[u], gv[u]);
            up_v[u] = util_grad<P>(I.kind, th, wv[u], gv[u]);
          }
          if (yhat < P(0)) {
            loc[3] += util_conj_neg<P>(I.kind, yhat, wv[u], gv[u]);
            const P dt = tr - th;
            loc[4] = fma(dt, dt, loc[4]);
          } else {
            loc[6] += P(1);
          }
          loc[5] = fma(th, th, loc[5]);
        }
      }
      if (I.Ylo[par ^ 1]) st_lo<VW>(I.Ylo[par ^ 1] + (size_t)j * I.ld + ci * VW, yl);
      st_plain<P, VW>(I.Y[par ^ 1] + (size_t)j * I.ld + ci * VW, yn);
      st_plain<P, VW>(prow + ci * VW, sv);
      if (check) {
        st_plain<P, VW>(I.That + (size_t)j * I.ld + ci * VW, that_v);
        st_plain<P, VW>(I.Uprime + (size_t)j * I.ld + ci * VW, up_v);
        st_plain<P, VW>(I.Yhat + (size_t)j * I.ld + ci * VW, yh_v);
      }
    }
    const int nparts = check ? NODE_PARTS : 1;
    for (int kk = 0; kk < nparts; ++kk) {
      const double tot = group_sum_double<GROUP>((double)loc[kk], sh, phase);
      if (lane == 0) I.pn[(size_t)j * NODE_PARTS + kk] = tot;
    }
  }
}

// ------------------------------------------------------------------ check phase

template <int VPT, int GROUP, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
batch_check_kernel(const BatchInst* __restrict__ insts, BatchClassDev cls) {
  using P = float;
  constexpr int VW = 4;
  constexpr int GPB = BLOCK / GROUP;
  __shared__ GroupScratch<GROUP> sh_all[GPB];
  GroupScratch<GROUP>& sh = sh_all[threadIdx.x / GROUP];
  int phase = 0;
  const int lane = threadIdx.x % GROUP;
  const int gid = blockIdx.x * GPB + threadIdx.x / GROUP;
  const int ngroups = gridDim.x * GPB;
  const int count = *cls.count;
  if (count == 0) return;
  const long long total = cls.eoff[count];
  for (long long g = gid; g < total; g += ngroups) {
    const int b = batch_find(cls.eoff, count, g);
    const BatchInst& I = insts[cls.inst[b]];
    const BatchScalars* sc = I.sc;
    if (!sc->active || !batch_is_check(sc)) continue;
    const int e = (int)(g - cls.eoff[b]);
    const int par = sc->parity;
    const P alpha = (P)sc->s.alpha;
    const int nchunks = I.ld / VW;
    const int h = I.e_head[e], t = I.e_tail[e];
    const P mu = I.mu[e];
    const size_t fo = (size_t)e * I.ld, ho = (size_t)h * I.ld, to = (size_t)t * I.ld;
    P ymax = -INFINITY;
    P lg2 = P(0), lgd = P(0), ld2 = P(0);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int ci = v * GROUP + lane;
      if (ci >= nchunks) continue;
      P fs[VW], y1[VW], y2[VW], g1[VW], g2[VW], z1[VW], z2[VW];
      ld_plain<P, VW>(I.F[par] + fo + ci * VW, fs);
      ld_plain<P, VW>(I.Y[par] + ho + ci * VW, y1);
      ld_plain<P, VW>(I.Y[par] + to + ci * VW, y2);
      ld_plain<P, VW>(I.Uprime + ho + ci * VW, g1);
      ld_plain<P, VW>(I.Uprime + to + ci * VW, g2);
      ld_plain<P, VW>(I.Yhat + ho + ci * VW, z1);
      ld_plain<P, VW>(I.Yhat + to + ci * VW, z2);
      P dl[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) dl[u] = P(0);
      if (I.Ylo[par]) {
        float l1[VW], l2[VW];
        ld_lo<VW>(I.Ylo[par] + ho + ci * VW, l1);
        ld_lo<VW>(I.Ylo[par] + to + ci * VW, l2);
#pragma unroll
        for (int u = 0; u < VW; ++u) dl[u] = l1[u] - l2[u];
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const int i = ci * VW + u;
        if (i >= I.n) continue;
        const P q = fs[u] + alpha * ((y1[u] - y2[u]) + dl[u]);
        const P fh = q > mu ? q - mu : P(0);
        const P d = fh - q;
        const P gg = g1[u] - g2[u];
        lg2 = fma(gg, gg, lg2);
        lgd = fma(gg, d, lgd);
        ld2 = fma(d, d, ld2);
        ymax = fmax(ymax, z1[u] - z2[u]);
      }
    }
    const double t0 = group_sum_double<GROUP>((double)lg2, sh, phase);
    const double t1 = group_sum_double<GROUP>((double)lgd, sh, phase);
    const double t2 = group_sum_double<GROUP>((double)ld2, sh, phase);
    ymax = group_max<GROUP, P>(ymax, sh, phase);
    if (lane == 0) {
      double* pc = I.pc + (size_t)e * CHECK_PARTS;
      pc[0] = t0;
      pc[1] = t1;
      pc[2] = t2;
      pc[3] = ymax > P(0) ? (double)I.cap[e] * (double)ymax : 0.0;
    }
  }
}

}  // namespace pdmcf
