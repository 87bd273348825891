// Restricted Wilson stencil on batches of domain instances (paper Sec. 3, D_X).
//
// The even-odd split of a domain X gives D_X = [[1, -k H_eo], [-k H_oe, 1]];
// k_hop computes, for one output parity p and every (instance, rhs) system of
// a batch,
//     out_p = a1 * s1_p + a2 * s2_p + b * (H_{p,1-p} in_{1-p})
// where hops that leave X are dropped (Dirichlet boundary), and can fuse the
// per-system inner products the Krylov solver needs into its epilogue.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

constexpr int HOP_THREADS = 128;

template <class S>
__device__ __forceinline__ const S* links_of(const DomInst& d);
template <>
__device__ __forceinline__ const double2* links_of<double2>(const DomInst& d) { return d.link64; }
template <>
__device__ __forceinline__ const float2* links_of<float2>(const DomInst& d) { return d.link32; }
template <>
__device__ __forceinline__ const __nv_bfloat162* links_of<__nv_bfloat162>(const DomInst& d) {
  return d.link16;
}
template <>
__device__ __forceinline__ const df2s* links_of<df2s>(const DomInst& d) { return d.linkdf; }

// A^{-1} of the clover term on the hop sum of output site g: FP64 from the full
// table, FP32 and double-float from the hermitian-packed tables
__device__ __forceinline__ void clover_epilogue(const void* t, long long g, double2 (&acc)[12]) {
  clover_mul((const double2*)t + 72LL * g, acc);
}
__device__ __forceinline__ void clover_epilogue(const void* t, long long g, float2 (&acc)[12]) {
  clover_mul_h((const float4*)t + (CLOV_H32_FLOATS / 4) * g, acc);
}
__device__ __forceinline__ void clover_epilogue(const void* t, long long g, dfc (&acc)[12]) {
  clover_mul_h((const float4*)t + CLOV_HDF_F4 * g, acc);
}

// ROWS: the link is read one row (U) or column (U^+) at a time after the spin
// projection, so 3 of its entries are live instead of 9 (the double-float form,
// whose 12-number accumulator and neighbour spinor fill the register budget)
template <int DIR, class S, class C, bool ROWS = false>
__device__ __forceinline__ void hop_one(C (&acc)[12], int n0, int p, int i, int n_out,
                                        int n_in, int j, const S* __restrict__ in_sys,
                                        const S* __restrict__ lk) {
  constexpr int MU = DIR & 3;
  constexpr bool FWD = DIR < 4;
  if (j < 0) return;
  C psi[12];
  ld_site<12>(in_sys, n_in, j, psi);
  if constexpr (ROWS) {
    C h[2][3];
    hop_project<MU, FWD>(psi, h);
    const S* blk = FWD ? lk + link_block(p, MU, n0, n_out) : lk + link_block(1 - p, MU, n0, n_in);
    const long long nn = FWD ? n_out : n_in, site = FWD ? i : j;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C u0 = cmk<C>(0.0, 0.0), u1 = cmk<C>(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const C e = ldc(blk + cidx(FWD ? a * 3 + b : b * 3 + a, nn, site));
        if (FWD) {
          cfma(u0, e, h[0][b]);
          cfma(u1, e, h[1][b]);
        } else {
          cfmac(u0, e, h[0][b]);
          cfmac(u1, e, h[1][b]);
        }
      }
      hop_accum_row<MU, FWD>(acc, a, u0, u1);
    }
    return;
  }
  C U[9];
  if (FWD) ld_link(lk + link_block(p, MU, n0, n_out), n_out, i, U);
  else ld_link(lk + link_block(1 - p, MU, n0, n_in), n_in, j, U);
  hop_dir<MU, FWD>(acc, psi, U);
}

// grid: nitems[p] * nrhs CTAs, rhs fastest (the CTAs that share a site chunk,
// and so its links, run together and hit L2); one output site per thread.
// One CTA work unit t = item * nrhs + rhs of the hop launch.
template <class S, bool CLOV, bool ROWS = false>
__device__ __forceinline__ void hop_unit(const BatchDev& bd, const HopArgs& a, long long t,
                                         double* red) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  const int p = a.p_out;
  const int item = (int)(t / bd.nrhs);
  const int r = (int)(t - (long long)item * bd.nrhs);
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  const int sys = it.x * bd.nrhs + r;
  if (a.active && !a.active[(long long)sys * a.active_stride]) return;
  if (a.work_bytes && threadIdx.x == 0) atomicAdd(a.work_bytes, a.site_bytes * it.z);
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const int i = it.y + threadIdx.x;
  const bool live = threadIdx.x < it.z;
  const S* in_sys = (const S*)a.in + (p ? bd.off[0] : bd.off[1])[sys];
  S* out_sys = (S*)a.out + (p ? bd.off[1] : bd.off[0])[sys];
  C out[12];
  if (live) {
    C acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = cmk<C>(0.0, 0.0);
    const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
    const S* lk = links_of<S>(*dp);
    int jn[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) jn[d] = __ldg(nbr + d * n_out + i);
    hop_one<0, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[0], in_sys, lk);
    hop_one<1, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[1], in_sys, lk);
    hop_one<2, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[2], in_sys, lk);
    hop_one<3, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[3], in_sys, lk);
    hop_one<4, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[4], in_sys, lk);
    hop_one<5, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[5], in_sys, lk);
    hop_one<6, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[6], in_sys, lk);
    hop_one<7, S, C, ROWS>(acc, n0, p, i, n_out, n_in, jn[7], in_sys, lk);
    // clover term: the hop sum times A^{-1} of the output site (compiled into
    // the FP64 forms and the clover instantiations only)
    if constexpr (CLOV) {
      if (a.clov_inv) clover_epilogue(a.clov_inv, dp->glob[(p ? n0 : 0) + i], acc);
    }
    const auto b = mkscal<C>(a.b);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = scale(acc[k], b);
    if (a.s1) {
      const S* s1 = (const S*)a.s1 + (p ? bd.off[1] : bd.off[0])[sys];
      const auto a1 = mkscal<C>(a.a1);
      C v[12];
      ld_site<12>(s1, n_out, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) axpy(out[k], a1, v[k]);
    }
    if (a.s2) {
      const S* s2 = (const S*)a.s2 + (p ? bd.off[1] : bd.off[0])[sys];
      const auto a2 = mkscal<C>(a.a2);
      C v[12];
      ld_site<12>(s2, n_out, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) axpy(out[k], a2, v[k]);
    }
    st_site<12>(out_sys, n_out, i, out);
  }
  if constexpr (std::is_same<C, dfc>::value) {
    // the double-float residual kernel: optionally |out|^2 (high parts, FP32 per
    // thread, FP64 across threads) per (item, rhs) into partial slot 0
    if (a.norm_out) {
      float t[1] = {0.f};
      double v[1] = {0.0};
      if (live)
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          dfc o = out[k];
          df_renorm(o);                 // the stored (nearest) high part
          t[0] += nrm2f(o);
        }
      block_reduce_t<float, 1>(t, v, red);
      if (threadIdx.x == 0) {
        const long long my = (long long)item * bd.nrhs + r;
        a.partial[2 * my] = v[0];
        a.partial[2 * my + 1] = 0.0;
      }
    }
    return;
  } else {
  const long long slot_stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
  const long long my = (long long)item * bd.nrhs + r;
  // per-thread sums in the storage's compute type (12 terms), FP64 across threads
  if (a.dotq) {
    double v[2] = {0.0, 0.0};
    T t[2] = {0, 0};
    if (live) {
      const S* q = (const S*)a.dotq + (p ? bd.off[1] : bd.off[0])[sys];
      C wv[12];
      ld_rhat(a.rhat_seed, sys, q, n_out, i, wv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const C w = wv[k];
        t[0] = fma(w.x, out[k].x, fma(w.y, out[k].y, t[0]));
        t[1] = fma(w.x, out[k].y, fma(-w.y, out[k].x, t[1]));
      }
    }
    block_reduce_t<T, 2>(t, v, red);
    if (threadIdx.x == 0) {
      a.partial[2 * my] = v[0];
      a.partial[2 * my + 1] = v[1];
    }
  }
  if (a.dots) {
    double v[3] = {0.0, 0.0, 0.0};
    T t[3] = {0, 0, 0};
    if (live) {
      const S* q = (const S*)a.dots + (p ? bd.off[1] : bd.off[0])[sys];
      C wv[12];
      ld_site<12>(q, n_out, i, wv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const C w = wv[k];
        // (out, s) = sum conj(out) s ; (out, out)
        t[0] = fma(out[k].x, w.x, fma(out[k].y, w.y, t[0]));
        t[1] = fma(out[k].x, w.y, fma(-out[k].y, w.x, t[1]));
        t[2] = fma(out[k].x, out[k].x, fma(out[k].y, out[k].y, t[2]));
      }
    }
    block_reduce_t<T, 3>(t, v, red);
    if (threadIdx.x == 0) {
      double* P = a.partial + (a.dotq ? 2 * slot_stride : 0);
      P[2 * my] = v[0];
      P[2 * my + 1] = v[1];
      P[2 * (slot_stride + my)] = v[2];
      P[2 * (slot_stride + my) + 1] = 0.0;
    }
  }
  if (a.dotqs) {
    // (dotq, s1): the self term is re-read here (it was loaded moments ago)
    double v[2] = {0.0, 0.0};
    T t[2] = {0, 0};
    if (live) {
      const long long oq = (p ? bd.off[1] : bd.off[0])[sys];
      C wv[12], sv[12];
      ld_rhat(a.rhat_seed, sys, (const S*)a.dotq + oq, n_out, i, wv);
      ld_site<12>((const S*)a.s1 + oq, n_out, i, sv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        t[0] = fma(wv[k].x, sv[k].x, fma(wv[k].y, sv[k].y, t[0]));
        t[1] = fma(wv[k].x, sv[k].y, fma(-wv[k].y, sv[k].x, t[1]));
      }
    }
    block_reduce_t<T, 2>(t, v, red);
    if (threadIdx.x == 0) {
      a.partial[2 * (3 * slot_stride + my)] = v[0];
      a.partial[2 * (3 * slot_stride + my) + 1] = v[1];
    }
  }
  }
}

// Register-blocked variant: one thread computes R rhs of the same output site,
// loading each link once for the R systems (work unit t = item * ceil(nrhs/R) + group).
template <int DIR, class S, class C, int R>
__device__ __forceinline__ void hop_one_r(C (&acc)[R][12], int n0, int p, int i, int n_out, int n_in,
                                          int j, const S* const (&in_sys)[R], const bool (&act)[R],
                                          const S* __restrict__ lk) {
  constexpr int MU = DIR & 3;
  constexpr bool FWD = DIR < 4;
  if (j < 0) return;
  C U[9];
  if (FWD) ld_link(lk + link_block(p, MU, n0, n_out), n_out, i, U);
  else ld_link(lk + link_block(1 - p, MU, n0, n_in), n_in, j, U);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (!act[q]) continue;
    C psi[12];
    ld_site<12>(in_sys[q], n_in, j, psi);
    hop_dir<MU, FWD>(acc[q], psi, U);
  }
}

template <class S, int R>
__device__ __forceinline__ void hop_unit_r(const BatchDev& bd, const HopArgs& a, long long t,
                                           double* red) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  const int p = a.p_out;
  const int ng = (bd.nrhs + R - 1) / R;
  const int item = (int)(t / ng);
  const int g = (int)(t - (long long)item * ng);
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  bool act[R];
  int nact = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = g * R + q;
    act[q] = r < bd.nrhs &&
             (!a.active || a.active[(long long)(it.x * bd.nrhs + r) * a.active_stride]);
    nact += act[q] ? 1 : 0;
  }
  if (nact == 0) return;
  if (a.work_bytes && threadIdx.x == 0) atomicAdd(a.work_bytes, a.site_bytes * it.z * nact);
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const int i = it.y + threadIdx.x;
  const bool live = threadIdx.x < it.z;
  const long long* off_in = p ? bd.off[0] : bd.off[1];
  const long long* off_out = p ? bd.off[1] : bd.off[0];
  const S* in_sys[R];
  long long oo[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = min(g * R + q, bd.nrhs - 1);
    const int sys = it.x * bd.nrhs + r;
    in_sys[q] = (const S*)a.in + off_in[sys];
    oo[q] = off_out[sys];
  }
  C out[R][12];
  if (live) {
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int k = 0; k < 12; ++k) out[q][k] = cmk<C>(0.0, 0.0);
    const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
    const S* lk = links_of<S>(*dp);
    int jn[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) jn[d] = __ldg(nbr + d * n_out + i);
    hop_one_r<0, S, C, R>(out, n0, p, i, n_out, n_in, jn[0], in_sys, act, lk);
    hop_one_r<1, S, C, R>(out, n0, p, i, n_out, n_in, jn[1], in_sys, act, lk);
    hop_one_r<2, S, C, R>(out, n0, p, i, n_out, n_in, jn[2], in_sys, act, lk);
    hop_one_r<3, S, C, R>(out, n0, p, i, n_out, n_in, jn[3], in_sys, act, lk);
    hop_one_r<4, S, C, R>(out, n0, p, i, n_out, n_in, jn[4], in_sys, act, lk);
    hop_one_r<5, S, C, R>(out, n0, p, i, n_out, n_in, jn[5], in_sys, act, lk);
    hop_one_r<6, S, C, R>(out, n0, p, i, n_out, n_in, jn[6], in_sys, act, lk);
    hop_one_r<7, S, C, R>(out, n0, p, i, n_out, n_in, jn[7], in_sys, act, lk);
    const T b = (T)a.b, a1 = (T)a.a1, a2 = (T)a.a2;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!act[q]) continue;
#pragma unroll
      for (int k = 0; k < 12; ++k) out[q][k] = cscale(out[q][k], b);
      if (a.s1) {
        C v[12];
        ld_site<12>((const S*)a.s1 + oo[q], n_out, i, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          out[q][k].x = fma(a1, v[k].x, out[q][k].x);
          out[q][k].y = fma(a1, v[k].y, out[q][k].y);
        }
      }
      if (a.s2) {
        C v[12];
        ld_site<12>((const S*)a.s2 + oo[q], n_out, i, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          out[q][k].x = fma(a2, v[k].x, out[q][k].x);
          out[q][k].y = fma(a2, v[k].y, out[q][k].y);
        }
      }
      st_site<12>((S*)a.out + oo[q], n_out, i, out[q]);
    }
  }
  if (!a.dotq && !a.dots && !a.dotqs) return;
  const long long slot_stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (!act[q]) continue;                       // uniform over the CTA
    const long long my = (long long)item * bd.nrhs + g * R + q;
    if (a.dotq) {
      double v[2] = {0.0, 0.0};
      T tt[2] = {0, 0};
      if (live) {
        C wv[12];
        ld_rhat(a.rhat_seed, it.x * bd.nrhs + g * R + q, (const S*)a.dotq + oo[q], n_out, i, wv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const C w = wv[k];
          tt[0] = fma(w.x, out[q][k].x, fma(w.y, out[q][k].y, tt[0]));
          tt[1] = fma(w.x, out[q][k].y, fma(-w.y, out[q][k].x, tt[1]));
        }
      }
      block_reduce_t<T, 2>(tt, v, red);
      if (threadIdx.x == 0) {
        a.partial[2 * my] = v[0];
        a.partial[2 * my + 1] = v[1];
      }
    }
    if (a.dots) {
      double v[3] = {0.0, 0.0, 0.0};
      T tt[3] = {0, 0, 0};
      if (live) {
        C wv[12];
        ld_site<12>((const S*)a.dots + oo[q], n_out, i, wv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const C w = wv[k];
          tt[0] = fma(out[q][k].x, w.x, fma(out[q][k].y, w.y, tt[0]));
          tt[1] = fma(out[q][k].x, w.y, fma(-out[q][k].y, w.x, tt[1]));
          tt[2] = fma(out[q][k].x, out[q][k].x, fma(out[q][k].y, out[q][k].y, tt[2]));
        }
      }
      block_reduce_t<T, 3>(tt, v, red);
      if (threadIdx.x == 0) {
        double* P = a.partial + (a.dotq ? 2 * slot_stride : 0);
        P[2 * my] = v[0];
        P[2 * my + 1] = v[1];
        P[2 * (slot_stride + my)] = v[2];
        P[2 * (slot_stride + my) + 1] = 0.0;
      }
    }
    if (a.dotqs) {
      double v[2] = {0.0, 0.0};
      T tt[2] = {0, 0};
      if (live) {
        C wv[12], sv[12];
        ld_rhat(a.rhat_seed, it.x * bd.nrhs + g * R + q, (const S*)a.dotq + oo[q], n_out, i, wv);
        ld_site<12>((const S*)a.s1 + oo[q], n_out, i, sv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          tt[0] = fma(wv[k].x, sv[k].x, fma(wv[k].y, sv[k].y, tt[0]));
          tt[1] = fma(wv[k].x, sv[k].y, fma(-wv[k].y, sv[k].x, tt[1]));
        }
      }
      block_reduce_t<T, 2>(tt, v, red);
      if (threadIdx.x == 0) {
        a.partial[2 * (3 * slot_stride + my)] = v[0];
        a.partial[2 * (3 * slot_stride + my) + 1] = v[1];
      }
    }
  }
}

// Direction-split variant: 256 threads per 128-site work item; thread t works
// on site t % 128 and on the forward (t < 128) or backward hops, so the eight
// dependent load-compute phases of a site run as two parallel chains of four.
// The two halves are summed through shared memory and the epilogue (self
// terms, store, inner products) is shared: each half writes 6 components.
template <class S>
__device__ __forceinline__ void hop_unit_split(const BatchDev& bd, const HopArgs& a, long long t,
                                               double* red, typename StoreTraits<S>::T* xs) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  const int p = a.p_out;
  const int item = (int)(t / bd.nrhs);
  const int r = (int)(t - (long long)item * bd.nrhs);
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  const int sys = it.x * bd.nrhs + r;
  if (a.active && !a.active[(long long)sys * a.active_stride]) return;
  if (a.work_bytes && threadIdx.x == 0) atomicAdd(a.work_bytes, a.site_bytes * it.z);
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const int s = threadIdx.x & (HOP_THREADS - 1);
  const int half = threadIdx.x >> 7;
  const int i = it.y + s;
  const bool live = s < it.z;
  const S* in_sys = (const S*)a.in + (p ? bd.off[0] : bd.off[1])[sys];
  S* out_sys = (S*)a.out + (p ? bd.off[1] : bd.off[0])[sys];
  C acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cmk<C>(0.0, 0.0);
  if (live) {
    const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
    const S* lk = links_of<S>(*dp);
    if (half == 0) {
      int jn[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) jn[d] = __ldg(nbr + d * n_out + i);
      hop_one<0, S>(acc, n0, p, i, n_out, n_in, jn[0], in_sys, lk);
      hop_one<1, S>(acc, n0, p, i, n_out, n_in, jn[1], in_sys, lk);
      hop_one<2, S>(acc, n0, p, i, n_out, n_in, jn[2], in_sys, lk);
      hop_one<3, S>(acc, n0, p, i, n_out, n_in, jn[3], in_sys, lk);
    } else {
      int jn[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) jn[d] = __ldg(nbr + (4 + d) * n_out + i);
      hop_one<4, S>(acc, n0, p, i, n_out, n_in, jn[0], in_sys, lk);
      hop_one<5, S>(acc, n0, p, i, n_out, n_in, jn[1], in_sys, lk);
      hop_one<6, S>(acc, n0, p, i, n_out, n_in, jn[2], in_sys, lk);
      hop_one<7, S>(acc, n0, p, i, n_out, n_in, jn[3], in_sys, lk);
    }
  }
  // exchange: half h keeps components 6h..6h+5 and receives them from the other half
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int kk = half ? k : 6 + k;           // components the other half keeps
    xs[(k * 2 + 0) * 2 * HOP_THREADS + half * HOP_THREADS + s] = acc[kk].x;
    xs[(k * 2 + 1) * 2 * HOP_THREADS + half * HOP_THREADS + s] = acc[kk].y;
  }
  __syncthreads();
  C out[6];
  const int other = 1 - half;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int kk = half ? 6 + k : k;
    C o = acc[kk];
    o.x += xs[(k * 2 + 0) * 2 * HOP_THREADS + other * HOP_THREADS + s];
    o.y += xs[(k * 2 + 1) * 2 * HOP_THREADS + other * HOP_THREADS + s];
    out[k] = o;
  }
  const int q0 = 3 * half;                     // first pair of this half's components
  if (live) {
    const T b = (T)a.b;
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = cscale(out[k], b);
    if (a.s1) {
      const S* s1 = (const S*)a.s1 + (p ? bd.off[1] : bd.off[0])[sys];
      const T a1 = (T)a.a1;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        C v0, v1;
        ld_pair(s1 + ((long long)(q0 + q) * n_out + i) * 2, v0, v1);
        out[2 * q].x = fma(a1, v0.x, out[2 * q].x);
        out[2 * q].y = fma(a1, v0.y, out[2 * q].y);
        out[2 * q + 1].x = fma(a1, v1.x, out[2 * q + 1].x);
        out[2 * q + 1].y = fma(a1, v1.y, out[2 * q + 1].y);
      }
    }
    if (a.s2) {
      const S* s2 = (const S*)a.s2 + (p ? bd.off[1] : bd.off[0])[sys];
      const T a2 = (T)a.a2;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        C v0, v1;
        ld_pair(s2 + ((long long)(q0 + q) * n_out + i) * 2, v0, v1);
        out[2 * q].x = fma(a2, v0.x, out[2 * q].x);
        out[2 * q].y = fma(a2, v0.y, out[2 * q].y);
        out[2 * q + 1].x = fma(a2, v1.x, out[2 * q + 1].x);
        out[2 * q + 1].y = fma(a2, v1.y, out[2 * q + 1].y);
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      st_pair(out_sys + ((long long)(q0 + q) * n_out + i) * 2, out[2 * q], out[2 * q + 1]);
  }
  const long long slot_stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
  const long long my = (long long)item * bd.nrhs + r;
  if (a.dotq) {
    double v[2] = {0.0, 0.0};
    T tt[2] = {0, 0};
    if (live) {
      const S* qv = (const S*)a.dotq + (p ? bd.off[1] : bd.off[0])[sys];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        C w0, w1;
        ld_rhat_pair(a.rhat_seed, sys, qv, n_out, i, q0 + q, w0, w1);
        const C w[2] = {w0, w1};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const C o = out[2 * q + e];
          tt[0] = fma(w[e].x, o.x, fma(w[e].y, o.y, tt[0]));
          tt[1] = fma(w[e].x, o.y, fma(-w[e].y, o.x, tt[1]));
        }
      }
    }
    block_reduce_t<T, 2>(tt, v, red);
    if (threadIdx.x == 0) {
      a.partial[2 * my] = v[0];
      a.partial[2 * my + 1] = v[1];
    }
  }
  if (a.dots) {
    double v[3] = {0.0, 0.0, 0.0};
    T tt[3] = {0, 0, 0};
    if (live) {
      const S* qv = (const S*)a.dots + (p ? bd.off[1] : bd.off[0])[sys];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        C w0, w1;
        ld_pair(qv + ((long long)(q0 + q) * n_out + i) * 2, w0, w1);
        const C w[2] = {w0, w1};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const C o = out[2 * q + e];
          tt[0] = fma(o.x, w[e].x, fma(o.y, w[e].y, tt[0]));
          tt[1] = fma(o.x, w[e].y, fma(-o.y, w[e].x, tt[1]));
          tt[2] = fma(o.x, o.x, fma(o.y, o.y, tt[2]));
        }
      }
    }
    block_reduce_t<T, 3>(tt, v, red);
    if (threadIdx.x == 0) {
      double* P = a.partial + (a.dotq ? 2 * slot_stride : 0);
      P[2 * my] = v[0];
      P[2 * my + 1] = v[1];
      P[2 * (slot_stride + my)] = v[2];
      P[2 * (slot_stride + my) + 1] = 0.0;
    }
  }
  if (a.dotqs) {
    double v[2] = {0.0, 0.0};
    T tt[2] = {0, 0};
    if (live) {
      const long long oq = (p ? bd.off[1] : bd.off[0])[sys];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        C w0, w1, s0, s1v;
        ld_rhat_pair(a.rhat_seed, sys, (const S*)a.dotq + oq, n_out, i, q0 + q, w0, w1);
        ld_pair((const S*)a.s1 + oq + ((long long)(q0 + q) * n_out + i) * 2, s0, s1v);
        tt[0] = fma(w0.x, s0.x, fma(w0.y, s0.y, tt[0]));
        tt[1] = fma(w0.x, s0.y, fma(-w0.y, s0.x, tt[1]));
        tt[0] = fma(w1.x, s1v.x, fma(w1.y, s1v.y, tt[0]));
        tt[1] = fma(w1.x, s1v.y, fma(-w1.y, s1v.x, tt[1]));
      }
    }
    block_reduce_t<T, 2>(tt, v, red);
    if (threadIdx.x == 0) {
      a.partial[2 * (3 * slot_stride + my)] = v[0];
      a.partial[2 * (3 * slot_stride + my) + 1] = v[1];
    }
  }
}

template <class S, int MINB, bool PERSIST>
__global__ void __launch_bounds__(2 * HOP_THREADS, MINB) k_hop_split(BatchDev bd, HopArgs a,
                                                                      long long nunits) {
  __shared__ double red[32 * 4];
  __shared__ typename StoreTraits<S>::T xs[12 * 2 * HOP_THREADS];
  if (PERSIST) {
    for (long long t = blockIdx.x; t < nunits; t += gridDim.x) {
      hop_unit_split<S>(bd, a, t, red, xs);
      __syncthreads();
    }
  } else {
    hop_unit_split<S>(bd, a, blockIdx.x, red, xs);
  }
}

// Launch variants chosen by the autotuner: MINB = resident CTAs per SM asked
// of the register allocator; PERSIST = a grid of (SMs x MINB) CTAs that walks
// the work units with a stride (one launch of persistent CTAs over blocks of
// any size) instead of one CTA per unit.
template <class S, int MINB, bool PERSIST, int R, bool CLOV = std::is_same<S, double2>::value,
          bool ROWS = false>
__global__ void __launch_bounds__(HOP_THREADS, MINB) k_hop(BatchDev bd, HopArgs a, long long nunits) {
  __shared__ double red[32 * 4];
  if (PERSIST) {
    for (long long t = blockIdx.x; t < nunits; t += gridDim.x) {
      if constexpr (R == 1) hop_unit<S, CLOV, ROWS>(bd, a, t, red);
      else hop_unit_r<S, R>(bd, a, t, red);
    }
  } else {
    if constexpr (R == 1) hop_unit<S, CLOV, ROWS>(bd, a, blockIdx.x, red);
    else hop_unit_r<S, R>(bd, a, blockIdx.x, red);
  }
}

// ---- bundle form: links and neighbour indices by bulk copy ----------------------
// One CTA per (128-site chunk, group of up to LB_MAX_RHS rhs), one warp per rhs,
// each lane one site of each of the chunk's four 32-site quarters.  Thread 0
// starts four bulk copies (cp.async.bulk, completion counted in bytes on one
// mbarrier per quarter) of the quarters' link bundles into shared memory; the
// warps then read links and neighbour indices from shared memory, so all rhs
// of the chunk share one copy and the only per-thread global loads left are
// the neighbour spinors.  Waits are bounded: a wait that gives up sets *a.err
// and the quarter is skipped (the host turns the flag into DD_ETIMEOUT).
constexpr int LB_MAX_RHS = 12;
constexpr unsigned LB_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// the same test with a suspend-time hint (ns): each unsuccessful poll returns
// after at most about that long
__device__ __forceinline__ bool mbar_try_wait_hint(unsigned long long* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// test-hook limit: 64 polls of at most ~1 us
constexpr unsigned LB_FAULT_POLLS = 64;
constexpr unsigned LB_FAULT_POLL_NS = 1000;
// bounded wait for the phase of parity `par` (short: the test hook's CTA)
__device__ __forceinline__ bool mbar_waitp(unsigned long long* bar, unsigned par, bool short_wait) {
  if (short_wait) {
    for (unsigned k = 0; k < LB_FAULT_POLLS; ++k)
      if (mbar_try_wait_hint(bar, par, LB_FAULT_POLL_NS)) return true;
    return false;
  }
  for (unsigned k = 0; k < LB_WAIT_LIMIT; ++k)
    if (mbar_try_wait(bar, par)) return true;
  return false;
}

// plain loads of a link from a shared-memory bundle (lane's column)
__device__ __forceinline__ void lds_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void lds_pair(const __nv_bfloat162* p, float2& a, float2& b) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 x, y;
  memcpy(&x, &v.x, 4);
  memcpy(&y, &v.y, 4);
  a = __bfloat1622float2(x);
  b = __bfloat1622float2(y);
}
__device__ __forceinline__ float2 lds_c(const float2* p) { return *p; }
__device__ __forceinline__ float2 lds_c(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }

template <class S, class C>
__device__ __forceinline__ void lds_link(const S* dirblk, int lane, C (&U)[9]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) lds_pair(dirblk + (e * LB_LANES + lane) * 2, U[2 * e], U[2 * e + 1]);
  U[8] = lds_c(dirblk + 4 * LB_LANES * 2 + lane);
}

// one direction of the hop for the RR rhs of a thread: the link is read from
// the shared-memory bundle once and applied to each rhs's neighbour spinor
template <int DIR, class S, class C, int RR>
__device__ __forceinline__ void hop_lb_dir(C (&acc)[RR][12], const int* qi, const S* ql, int lane,
                                           int n_in, const void* in, const long long* off_in,
                                           const int (&sysk)[RR], const bool (&actk)[RR]) {
  constexpr int MU = DIR & 3;
  constexpr bool FWD = DIR < 4;
  const int j = qi[DIR * LB_LANES + lane];
  if (j < 0) return;
  C U[9];
  lds_link(ql + DIR * LB_DIR_S, lane, U);
#pragma unroll
  for (int k = 0; k < RR; ++k) {
    if (!actk[k]) continue;
    C psi[12];
    ld_site<12>((const S*)in + off_in[sysk[k]], n_in, j, psi);
    hop_dir<MU, FWD>(acc[k], psi, U);
  }
}

template <class S>
__device__ __forceinline__ const unsigned char* bundle_of(const DomInst& d);
template <>
__device__ __forceinline__ const unsigned char* bundle_of<float2>(const DomInst& d) { return d.lb32; }
template <>
__device__ __forceinline__ const unsigned char* bundle_of<__nv_bfloat162>(const DomInst& d) {
  return d.lb16;
}

template <class S>
constexpr int lb_smem_bytes() { return LB_QUARTERS * lb_quarter_bytes<S>() + 64; }

// grid: nitems[p] * ngroups CTAs (group fastest), 32 * ceil(rb / RR) threads;
// thread (warp w, lane) computes rhs g * rb + w * RR + k, k < RR, of one site,
// reading each link from shared memory once for its RR rhs
// QPC: quarters of the item per CTA (4: the whole item; 2: half of it, so two
// CTAs share an item and add their inner-product partials atomically onto
// zeroed slots); MAXR: most rhs per CTA.
// One work unit (item, rhs group, part of the item) of the bundle form; the
// barriers of the QPC quarter slots are initialised by the caller, and slot q
// waits for the phase parity (ph >> q) & 1.  Returns the number of slots it used
// (0 when the unit had nothing to do); every CTA-wide barrier inside is reached
// by all threads or by none.
template <class S, int RR, int QPC, int MAXR, bool CLOV>
__device__ __forceinline__ int lb_unit(const BatchDev& bd, const HopArgs& a, int ngroups, int rb, long long unit,
                                       unsigned ph, bool fault) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  constexpr int QB = lb_quarter_bytes<S>();
  constexpr int NH = LB_QUARTERS / QPC;
  extern __shared__ __align__(128) unsigned char lb_smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(lb_smem + QPC * QB);
  const int p = a.p_out;
  const int item = (int)(unit / (ngroups * NH));
  const int rem = (int)(unit - (long long)item * ngroups * NH);
  const int hh = NH == 1 ? 0 : rem / ngroups;
  const int g = rem - hh * ngroups;
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  const int q0 = hh * QPC;
  const int nq = min(QPC, (it.z + LB_LANES - 1) / LB_LANES - q0);   // quarters of this CTA
  if (nq <= 0) return 0;                       // the item is shorter than this part (uniform)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool actk[RR];
  int sysk[RR];
  bool act = false;
#pragma unroll
  for (int k = 0; k < RR; ++k) {
    const int rr = w * RR + k;
    const int r = g * rb + rr;
    sysk[k] = it.x * bd.nrhs + r;
    actk[k] = rr < rb && r < bd.nrhs &&
              (!a.active || a.active[(long long)sysk[k] * a.active_stride]);
    act = act || actk[k];
  }
  // active rhs of the CTA: each warp contributes its count as that many lanes
  int nact_rhs = 0;
#pragma unroll
  for (int k = 0; k < RR; ++k) nact_rhs += actk[k] ? 1 : 0;
  const int cta_rhs = __syncthreads_count(lane < nact_rhs);   // lanes 0 .. nact_rhs-1 of each warp
  if (cta_rhs == 0) return 0;                  // every rhs of the group has converged
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  // test hook: the first unit of CTA 0 arms the barrier of its last quarter
  // without issuing the copy, so that wait gives up (nothing is in flight for it)
  // after a short limit
  const int fq = fault ? nq - 1 : -1;
  if (threadIdx.x == 0) {
    // one atomic per unit for the algorithmic-byte accounting (timing only)
    if (a.work_bytes)
      atomicAdd(a.work_bytes, a.site_bytes * min(it.z - q0 * LB_LANES, nq * LB_LANES) * cta_rhs);
    // the bulk copies below overwrite shared memory an earlier unit of this CTA read
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned char* src = bundle_of<S>(*dp) +
        (lb_quarter_base(p, n0) + (long long)LB_QUARTERS * (it.y / LB_CHUNK) + q0) * QB;
    for (int q = 0; q < nq; ++q) {
      mbar_expect_tx(&bar[q], QB);
      if (q != fq) bulk_copy_g2s(lb_smem + q * QB, src + (long long)q * QB, QB, &bar[q]);
    }
  }
  // Thread 0 waits on every quarter on each path.  If a wait on an issued copy
  // gives up, thread 0 at once waits for that copy once more (bounded), so the
  // CTA's shared memory outlives every copy it started.
  if (!act) {
    // idle warp of a busy CTA: thread 0 still sees its copies land before leaving
    if (threadIdx.x == 0)
      for (int q = 0; q < nq; ++q)
        if (!mbar_waitp(&bar[q], (ph >> q) & 1u, fault)) {
          atomicExch(a.err, 1);
          if (q != fq) mbar_waitp(&bar[q], (ph >> q) & 1u, false);
        }
    return nq;
  }
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const long long* off_in = p ? bd.off[0] : bd.off[1];
  const long long* off_out = p ? bd.off[1] : bd.off[0];
  const auto bsc = mkscal<C>(a.b);
  const auto a1 = mkscal<C>(a.a1);
  const auto a2 = mkscal<C>(a.a2);
  // fused (out, dots) and |out|^2 in the self-term pass when the dot vector is
  // the only self term (t = s - k^2 H tmp with (t, s)): s is read once
  const bool dots_in_s1 = a.dots && a.dots == a.s1 && !a.s2;
  // the end-of-iteration launch of BiCGstab (see end_mode below)
  const bool end_mode = dots_in_s1 && a.dotq && a.dotqs;
  T tq[RR][2], ts[RR][3], tqs[RR][2];
#pragma unroll
  for (int k = 0; k < RR; ++k) {
    tq[k][0] = tq[k][1] = 0;
    ts[k][0] = ts[k][1] = ts[k][2] = 0;
    tqs[k][0] = tqs[k][1] = 0;
  }
  for (int q = 0; q < nq; ++q) {
    if (!mbar_waitp(&bar[q], (ph >> q) & 1u, fault)) {
      if (lane == 0) atomicExch(a.err, 1);
      if (threadIdx.x == 0 && q != fq) mbar_waitp(&bar[q], (ph >> q) & 1u, false);
      continue;
    }
    const int li = (q0 + q) * LB_LANES + lane;
    if (li >= it.z) continue;
    const int i = it.y + li;
    if constexpr (CLOV) {
      // the site's A^{-1} rows (288 B) into L1 while the eight directions run;
      // the CTA's other rhs warps then read them from L1 in the epilogue
      if (w == 0) {
        const char* t = (const char*)((const float4*)a.clov_inv + (CLOV_H32_FLOATS / 4) * dp->glob[(p ? n0 : 0) + i]);
#pragma unroll
        for (int o = 0; o < 288; o += 96) asm volatile("prefetch.global.L1 [%0];" ::"l"(t + o));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(t + 287));
      }
    }
    const unsigned char* qb = lb_smem + q * QB;
    const S* ql = reinterpret_cast<const S*>(qb);
    const int* qi = reinterpret_cast<const int*>(qb + lb_link_bytes<S>());
    C acc[RR][12];
#pragma unroll
    for (int k = 0; k < RR; ++k)
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[k][c] = cmk<C>(0.0, 0.0);
    // forward and backward hop of a direction back to back: along x3 and x2
    // the two neighbour sets of a warp's 32 sites nearly coincide, so the
    // second load finds the first one's lines in L1
    hop_lb_dir<3, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<7, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<2, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<6, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<1, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<5, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<0, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    hop_lb_dir<4, S, C, RR>(acc, qi, ql, lane, n_in, a.in, off_in, sysk, actk);
    if constexpr (CLOV) {
      // clover term: the hop sums times A^{-1} of the output site
      const long long gs = dp->glob[(p ? n0 : 0) + i];
#pragma unroll
      for (int k = 0; k < RR; ++k)
        if (actk[k]) clover_epilogue(a.clov_inv, gs, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      if (!actk[k]) continue;
      const long long oo = off_out[sysk[k]];
      if (end_mode) {
        // t = s - k^2 H tmp with (r^, t), (t, s), |t|^2 and (r^, s): one pass over
        // the component pairs reads s and r^ once each
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const long long e = oo + ((long long)q * n_out + i) * 2;
          C sv[2], rv[2], ov[2];
          ld_pair((const S*)a.s1 + e, sv[0], sv[1]);
          ld_rhat_pair(a.rhat_seed, sysk[k], (const S*)a.dotq + oo, n_out, i, q, rv[0], rv[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            ov[h] = scale(acc[k][2 * q + h], bsc);
            axpy(ov[h], a1, sv[h]);
            const C o = ov[h], w = rv[h], z = sv[h];
            ts[k][0] = fma(o.x, z.x, fma(o.y, z.y, ts[k][0]));
            ts[k][1] = fma(o.x, z.y, fma(-o.y, z.x, ts[k][1]));
            ts[k][2] = fma(o.x, o.x, fma(o.y, o.y, ts[k][2]));
            tq[k][0] = fma(w.x, o.x, fma(w.y, o.y, tq[k][0]));
            tq[k][1] = fma(w.x, o.y, fma(-w.y, o.x, tq[k][1]));
            tqs[k][0] = fma(w.x, z.x, fma(w.y, z.y, tqs[k][0]));
            tqs[k][1] = fma(w.x, z.y, fma(-w.y, z.x, tqs[k][1]));
          }
          st_pair((S*)a.out + e, ov[0], ov[1]);
        }
        continue;
      }
      C out[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) out[c] = scale(acc[k][c], bsc);
      if (a.s1) {
        C v[12];
        ld_site<12>((const S*)a.s1 + oo, n_out, i, v);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          axpy(out[c], a1, v[c]);
          if (dots_in_s1) {
            ts[k][0] = fma(out[c].x, v[c].x, fma(out[c].y, v[c].y, ts[k][0]));
            ts[k][1] = fma(out[c].x, v[c].y, fma(-out[c].y, v[c].x, ts[k][1]));
            ts[k][2] = fma(out[c].x, out[c].x, fma(out[c].y, out[c].y, ts[k][2]));
          }
        }
      }
      if (a.s2) {
        C v[12];
        ld_site<12>((const S*)a.s2 + oo, n_out, i, v);
#pragma unroll
        for (int c = 0; c < 12; ++c) axpy(out[c], a2, v[c]);
      }
      st_site<12>((S*)a.out + oo, n_out, i, out);
      if (a.dotq) {
        C wv[12];
        ld_rhat(a.rhat_seed, sysk[k], (const S*)a.dotq + oo, n_out, i, wv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          tq[k][0] = fma(wv[c].x, out[c].x, fma(wv[c].y, out[c].y, tq[k][0]));
          tq[k][1] = fma(wv[c].x, out[c].y, fma(-wv[c].y, out[c].x, tq[k][1]));
        }
        if (a.dotqs) {
          // (dotq, s1): the self term is re-read (it was loaded moments ago)
          C sv[12];
          ld_site<12>((const S*)a.s1 + oo, n_out, i, sv);
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            tqs[k][0] = fma(wv[c].x, sv[c].x, fma(wv[c].y, sv[c].y, tqs[k][0]));
            tqs[k][1] = fma(wv[c].x, sv[c].y, fma(-wv[c].y, sv[c].x, tqs[k][1]));
          }
        }
      }
      if (a.dots && !dots_in_s1) {
        C wv[12];
        ld_site<12>((const S*)a.dots + oo, n_out, i, wv);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          ts[k][0] = fma(out[c].x, wv[c].x, fma(out[c].y, wv[c].y, ts[k][0]));
          ts[k][1] = fma(out[c].x, wv[c].y, fma(-out[c].y, wv[c].x, ts[k][1]));
          ts[k][2] = fma(out[c].x, out[c].x, fma(out[c].y, out[c].y, ts[k][2]));
        }
      }
    }
  }
  // per-(warp, k) = per-system partial sums of the chunk
  const long long slot_stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
#pragma unroll
  for (int k = 0; k < RR; ++k) {
    // actk[k] is uniform over the warp, so the shuffles below see full warps
    if (!actk[k]) continue;
    const long long my = (long long)item * bd.nrhs + (sysk[k] - (long long)it.x * bd.nrhs);
    // one CTA per item stores its partials; with parts (NH > 1) each part adds
    // its own onto the zeroed slot (two addends onto zero: order-independent)
    auto put = [&](double* dst, double v) {
      if (NH == 1) *dst = v;
      else atomicAdd(dst, v);
    };
    if (a.dotq) {
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tq[k][e] += __shfl_down_sync(0xffffffffu, tq[k][e], o);
      if (lane == 0) {
        put(&a.partial[2 * my], (double)tq[k][0]);
        put(&a.partial[2 * my + 1], (double)tq[k][1]);
      }
    }
    if (a.dots) {
#pragma unroll
      for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ts[k][e] += __shfl_down_sync(0xffffffffu, ts[k][e], o);
      if (lane == 0) {
        double* P = a.partial + (a.dotq ? 2 * slot_stride : 0);
        put(&P[2 * my], (double)ts[k][0]);
        put(&P[2 * my + 1], (double)ts[k][1]);
        put(&P[2 * (slot_stride + my)], (double)ts[k][2]);
        if (NH == 1) P[2 * (slot_stride + my) + 1] = 0.0;
      }
    }
    if (a.dotqs) {
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tqs[k][e] += __shfl_down_sync(0xffffffffu, tqs[k][e], o);
      if (lane == 0) {
        put(&a.partial[2 * (3 * slot_stride + my)], (double)tqs[k][0]);
        put(&a.partial[2 * (3 * slot_stride + my) + 1], (double)tqs[k][1]);
      }
    }
  }
  return nq;
}

template <class S, int MINB, int RR, int QPC, int MAXR, bool CLOV = false>
__global__ void __launch_bounds__(32 * MAXR / RR, MINB)
    k_hop_lb(BatchDev bd, HopArgs a, int ngroups, int rb) {
  extern __shared__ __align__(128) unsigned char lb_smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(lb_smem + QPC * lb_quarter_bytes<S>());
  if (threadIdx.x == 0) {
    for (int q = 0; q < QPC; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  __syncthreads();
  lb_unit<S, RR, QPC, MAXR, CLOV>(bd, a, ngroups, rb, blockIdx.x, 0u, a.lb_fault && blockIdx.x == 0);
}

// Persistent form with a work queue: a grid of (SMs x resident CTAs) CTAs pulls
// units (item, rhs group, part) from a device counter (a.queue, zeroed before
// the launch), so blocks of uneven sizes and converged systems are balanced at
// run time; the quarter barriers are initialised once and reused phase by phase.
template <class S, int MINB, int RR, int QPC, int MAXR>
__global__ void __launch_bounds__(32 * MAXR / RR, MINB)
    k_hop_lbq(BatchDev bd, HopArgs a, int ngroups, int rb, int nunits) {
  extern __shared__ __align__(128) unsigned char lb_smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(lb_smem + QPC * lb_quarter_bytes<S>());
  __shared__ int next_unit;
  if (threadIdx.x == 0) {
    for (int q = 0; q < QPC; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  unsigned ph = 0;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) next_unit = atomicAdd(a.queue, 1);
    __syncthreads();                       // also: every thread is done with the previous unit
    const int u = next_unit;
    // a wait that gave up (here or in another CTA) stops the queue: a barrier
    // whose phase did not complete cannot serve another unit
    const bool stop = *(volatile const int*)a.err != 0;
    __syncthreads();                       // next_unit is rewritten only after all have read it
    if (u >= nunits || stop) break;
    const int used = lb_unit<S, RR, QPC, MAXR, false>(bd, a, ngroups, rb, u, ph, a.lb_fault && blockIdx.x == 0 && first);
    ph ^= (1u << used) - 1u;
    first = false;
  }
}

template <class S, int MINB, int RR, int QPC = LB_QUARTERS, int MAXR = LB_MAX_RHS, bool CLOV = false>
static void launch_lb(const BatchDev& bd, const HopArgs& a, long long nitems_p, cudaStream_t s) {
  const int ngroups = (bd.nrhs + MAXR - 1) / MAXR;
  const int rb = (bd.nrhs + ngroups - 1) / ngroups;
  const int nthreads = 32 * ((rb + RR - 1) / RR);
  constexpr int NH = LB_QUARTERS / QPC;
  if (NH > 1 && a.partial) {
    // the slots this launch writes start at zero (its parts add onto them)
    const long long stride = nitems_p * bd.nrhs;
    auto zero = [&](int slot) { cudaMemsetAsync(a.partial + 2 * slot * stride, 0, 16 * stride, s); };
    if (a.dotq) zero(0);
    if (a.dots) {
      zero(a.dotq ? 1 : 0);
      zero(a.dotq ? 2 : 1);
    }
    if (a.dotqs) zero(3);
  }
  DD_COUNT_LAUNCH(), k_hop_lb<S, MINB, RR, QPC, MAXR, CLOV>
      <<<(unsigned)(nitems_p * ngroups * NH), nthreads, QPC * lb_quarter_bytes<S>() + 64, s>>>(bd, a, ngroups, rb);
}

// the work-queue form: (SMs x MINB) CTAs pull the units from a zeroed counter
template <class S, int MINB, int RR, int QPC = LB_QUARTERS, int MAXR = LB_MAX_RHS>
static void launch_lbq(const BatchDev& bd, const HopArgs& a, long long nitems_p, int nsm, cudaStream_t s) {
  const int ngroups = (bd.nrhs + MAXR - 1) / MAXR;
  const int rb = (bd.nrhs + ngroups - 1) / ngroups;
  const int nthreads = 32 * ((rb + RR - 1) / RR);
  constexpr int NH = LB_QUARTERS / QPC;
  if (NH > 1 && a.partial) {
    const long long stride = nitems_p * bd.nrhs;
    auto zero = [&](int slot) { cudaMemsetAsync(a.partial + 2 * slot * stride, 0, 16 * stride, s); };
    if (a.dotq) zero(0);
    if (a.dots) {
      zero(a.dotq ? 1 : 0);
      zero(a.dotq ? 2 : 1);
    }
    if (a.dotqs) zero(3);
  }
  const long long nunits = nitems_p * ngroups * NH;
  cudaMemsetAsync(a.queue, 0, sizeof(int), s);
  const long long grid = std::min<long long>(nunits, (long long)nsm * MINB);
  DD_COUNT_LAUNCH(), k_hop_lbq<S, MINB, RR, QPC, MAXR>
      <<<(unsigned)grid, nthreads, QPC * lb_quarter_bytes<S>() + 64, s>>>(bd, a, ngroups, rb, (int)nunits);
}

void hop_bundle_prepare() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  const int b32 = lb_smem_bytes<float2>(), b16 = lb_smem_bytes<__nv_bfloat162>();
  const int h32 = 2 * lb_quarter_bytes<float2>() + 64, h16 = 2 * lb_quarter_bytes<__nv_bfloat162>() + 64;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(k_hop_lb<float2, 2, 1, 4, 12>, at, b32);
  cudaFuncSetAttribute(k_hop_lb<float2, 2, 1, 4, 12, true>, at, b32);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 2, 1, 4, 12, true>, at, b16);
  cudaFuncSetAttribute(k_hop_lb<float2, 1, 1, 4, 12>, at, b32);
  cudaFuncSetAttribute(k_hop_lb<float2, 2, 2, 4, 12>, at, b32);
  cudaFuncSetAttribute(k_hop_lb<float2, 2, 3, 4, 12>, at, b32);
  cudaFuncSetAttribute(k_hop_lb<float2, 2, 1, 2, 12>, at, h32);
  cudaFuncSetAttribute(k_hop_lb<float2, 5, 1, 2, 6>, at, h32);
  cudaFuncSetAttribute(k_hop_lb<float2, 4, 1, 2, 6>, at, h32);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 2, 1, 4, 12>, at, b16);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 1, 1, 4, 12>, at, b16);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 3, 2, 4, 12>, at, b16);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 4, 3, 4, 12>, at, b16);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 2, 1, 2, 12>, at, h16);
  cudaFuncSetAttribute(k_hop_lb<__nv_bfloat162, 5, 1, 2, 6>, at, h16);
  cudaFuncSetAttribute(k_hop_lbq<float2, 2, 1, 4, 12>, at, b32);
  cudaFuncSetAttribute(k_hop_lbq<float2, 4, 1, 2, 6>, at, h32);
  cudaFuncSetAttribute(k_hop_lbq<__nv_bfloat162, 2, 1, 4, 12>, at, b16);
  done[dev] = true;
}

struct HopVariant {
  int minb;
  bool persist;
  int r;          // rhs per thread (0: direction-split, 256 threads per item; -k: bundle form
                  // with k rhs per thread)
  int qpc = 4;    // bundle form: link quarters of the 128-site item per CTA
  int maxr = 12;  // bundle form: most rhs per CTA
};
// per storage precision; index 0 is the default before tuning
static const HopVariant kVariants64[] = {{3, false, 1}, {2, false, 1}, {3, true, 1}, {2, false, 2},
                                         {2, false, 0}};
static const HopVariant kVariants32[] = {{6, false, 1}, {4, false, 1}, {8, false, 1}, {6, true, 1},
                                         {4, true, 1}, {4, false, 2}, {5, false, 2}, {4, true, 2},
                                         {3, false, 3}, {3, false, 4}, {3, false, 0}, {4, false, 0},
                                         {3, true, 0}, {2, false, -1}, {1, false, -1}, {2, false, -2},
                                         {2, false, -3}, {2, false, -1, 2, 12}, {5, false, -1, 2, 6},
                                         {4, false, -1, 2, 6}, {2, true, -1}, {4, true, -1, 2, 6}};
static const HopVariant kVariants16[] = {{5, false, 1}, {4, false, 1}, {8, false, 1}, {5, true, 1},
                                         {4, false, 2}, {3, false, 3}, {3, false, 0}, {4, false, 0},
                                         {2, false, -1}, {1, false, -1}, {3, false, -2}, {4, false, -3},
                                         {2, false, -1, 2, 12}, {5, false, -1, 2, 6}, {2, true, -1}};

int hop_variant_count(dd_prec prec) { return prec == DD_F64 ? 5 : (prec == DD_F32 ? 22 : 15); }

static const HopVariant& variant_of(dd_prec prec, int v) {
  const HopVariant* t = prec == DD_F64 ? kVariants64 : (prec == DD_F32 ? kVariants32 : kVariants16);
  if (v < 0 || v >= hop_variant_count(prec)) v = 0;
  return t[v];
}

template <class S, int MINB, bool PERSIST, int R, bool CLOV = std::is_same<S, double2>::value,
          bool ROWS = false>
static void launch_variant(const BatchDev& bd, const HopArgs& a, long long nitems_p, int nsm,
                           cudaStream_t s) {
  const long long nunits = nitems_p * ((bd.nrhs + R - 1) / R);
  long long grid = nunits;
  if (PERSIST) grid = std::min<long long>(nunits, (long long)nsm * MINB);
  DD_COUNT_LAUNCH(), k_hop<S, MINB, PERSIST, R, CLOV, ROWS><<<(unsigned)grid, HOP_THREADS, 0, s>>>(bd, a, nunits);
}

template <class S, int MINB, bool PERSIST>
static void launch_split(const BatchDev& bd, const HopArgs& a, long long nitems_p, int nsm,
                         cudaStream_t s) {
  const long long nunits = nitems_p * bd.nrhs;
  long long grid = nunits;
  if (PERSIST) grid = std::min<long long>(nunits, (long long)nsm * MINB);
  DD_COUNT_LAUNCH(), k_hop_split<S, MINB, PERSIST><<<(unsigned)grid, 2 * HOP_THREADS, 0, s>>>(bd, a, nunits);
}

static void dispatch_hop(dd_prec prec, int v, const BatchDev& bd, const HopArgs& a, long long ni,
                         int nsm, cudaStream_t s) {
  if (prec == DD_DF64) {
    if (a.clov_inv) launch_variant<df2s, 4, false, 1, true>(bd, a, ni, nsm, s);
    else launch_variant<df2s, 4, false, 1, false, true>(bd, a, ni, nsm, s);
    return;
  }
  if (prec == DD_F64 && a.clov_inv) {      // the clover epilogue lives in the plain form
    launch_variant<double2, 3, false, 1>(bd, a, ni, nsm, s);
    return;
  }
  if (a.clov_inv) {
    // FP32 / BF16 storage with the clover term: the bundle form with the
    // epilogue compiled in (no launch-form tuning)
    if (prec == DD_F32) launch_lb<float2, 2, 1, LB_QUARTERS, LB_MAX_RHS, true>(bd, a, ni, s);
    else launch_lb<__nv_bfloat162, 2, 1, LB_QUARTERS, LB_MAX_RHS, true>(bd, a, ni, s);
    return;
  }
  const HopVariant& hv = variant_of(prec, v);
  if (hv.r < 0) {
    const int rr = -hv.r;
    if (hv.persist) {
      if (prec == DD_F32 && hv.qpc == 2) launch_lbq<float2, 4, 1, 2, 6>(bd, a, ni, nsm, s);
      else if (prec == DD_F32) launch_lbq<float2, 2, 1>(bd, a, ni, nsm, s);
      else launch_lbq<__nv_bfloat162, 2, 1>(bd, a, ni, nsm, s);
      return;
    }
    if (prec == DD_F32) {
      if (hv.qpc == 2 && hv.maxr == 6 && hv.minb == 5) launch_lb<float2, 5, 1, 2, 6>(bd, a, ni, s);
      else if (hv.qpc == 2 && hv.maxr == 6) launch_lb<float2, 4, 1, 2, 6>(bd, a, ni, s);
      else if (hv.qpc == 2) launch_lb<float2, 2, 1, 2, 12>(bd, a, ni, s);
      else if (rr == 3) launch_lb<float2, 2, 3>(bd, a, ni, s);
      else if (rr == 2) launch_lb<float2, 2, 2>(bd, a, ni, s);
      else if (hv.minb == 1) launch_lb<float2, 1, 1>(bd, a, ni, s);
      else launch_lb<float2, 2, 1>(bd, a, ni, s);
    } else {
      if (hv.qpc == 2 && hv.maxr == 6) launch_lb<__nv_bfloat162, 5, 1, 2, 6>(bd, a, ni, s);
      else if (hv.qpc == 2) launch_lb<__nv_bfloat162, 2, 1, 2, 12>(bd, a, ni, s);
      else if (rr == 3) launch_lb<__nv_bfloat162, 4, 3>(bd, a, ni, s);
      else if (rr == 2) launch_lb<__nv_bfloat162, 3, 2>(bd, a, ni, s);
      else if (hv.minb == 1) launch_lb<__nv_bfloat162, 1, 1>(bd, a, ni, s);
      else launch_lb<__nv_bfloat162, 2, 1>(bd, a, ni, s);
    }
    return;
  }
  if (hv.r == 0) {
    if (prec == DD_F64) launch_split<double2, 2, false>(bd, a, ni, nsm, s);
    else if (prec == DD_F32 && hv.persist) launch_split<float2, 3, true>(bd, a, ni, nsm, s);
    else if (prec == DD_F32 && hv.minb == 4) launch_split<float2, 4, false>(bd, a, ni, nsm, s);
    else if (prec == DD_F32) launch_split<float2, 3, false>(bd, a, ni, nsm, s);
    else if (hv.minb == 4) launch_split<__nv_bfloat162, 4, false>(bd, a, ni, nsm, s);
    else launch_split<__nv_bfloat162, 3, false>(bd, a, ni, nsm, s);
    return;
  }
  if (prec == DD_F64) {
    if (hv.r == 2) launch_variant<double2, 2, false, 2>(bd, a, ni, nsm, s);
    else if (hv.persist) launch_variant<double2, 3, true, 1>(bd, a, ni, nsm, s);
    else if (hv.minb == 2) launch_variant<double2, 2, false, 1>(bd, a, ni, nsm, s);
    else launch_variant<double2, 3, false, 1>(bd, a, ni, nsm, s);
  } else if (prec == DD_F32) {
    if (hv.r == 4) launch_variant<float2, 3, false, 4>(bd, a, ni, nsm, s);
    else if (hv.r == 3) launch_variant<float2, 3, false, 3>(bd, a, ni, nsm, s);
    else if (hv.r == 2 && hv.persist) launch_variant<float2, 4, true, 2>(bd, a, ni, nsm, s);
    else if (hv.r == 2 && hv.minb == 5) launch_variant<float2, 5, false, 2>(bd, a, ni, nsm, s);
    else if (hv.r == 2) launch_variant<float2, 4, false, 2>(bd, a, ni, nsm, s);
    else if (hv.persist && hv.minb == 4) launch_variant<float2, 4, true, 1>(bd, a, ni, nsm, s);
    else if (hv.persist) launch_variant<float2, 6, true, 1>(bd, a, ni, nsm, s);
    else if (hv.minb == 4) launch_variant<float2, 4, false, 1>(bd, a, ni, nsm, s);
    else if (hv.minb == 8) launch_variant<float2, 8, false, 1>(bd, a, ni, nsm, s);
    else launch_variant<float2, 6, false, 1>(bd, a, ni, nsm, s);
  } else {
    if (hv.r == 3) launch_variant<__nv_bfloat162, 3, false, 3>(bd, a, ni, nsm, s);
    else if (hv.r == 2) launch_variant<__nv_bfloat162, 4, false, 2>(bd, a, ni, nsm, s);
    else if (hv.persist) launch_variant<__nv_bfloat162, 5, true, 1>(bd, a, ni, nsm, s);
    else if (hv.minb == 4) launch_variant<__nv_bfloat162, 4, false, 1>(bd, a, ni, nsm, s);
    else if (hv.minb == 8) launch_variant<__nv_bfloat162, 8, false, 1>(bd, a, ni, nsm, s);
    else launch_variant<__nv_bfloat162, 5, false, 1>(bd, a, ni, nsm, s);
  }
}

// Algorithmic bytes per output (site, rhs) of one hop launch: the neighbour
// input read once, the output written once, each self term read once, and
// the 8 links of the site read once and shared by the batch's nrhs systems.
// The kernel adds it for the CTAs that actually run (converged systems skip).
static double hop_site_bytes(const Batch& b, size_t cb, int nself) {
  return 12.0 * cb * (2 + nself) + 8.0 * 9.0 * cb / b.nrhs;
}

dd_status launch_hop(dd_ctx* c, const Batch& b, dd_prec prec, const HopArgs& a0, cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  BatchDev bd = batch_view(c, b);
  HopArgs a = a0;
  a.err = c->d_err;
  a.clov_inv = nullptr;
  if (c->clover_active)
    a.clov_inv = prec == DD_F64 ? (const void*)c->d_clovi
                                : (prec == DD_DF64 ? (const void*)c->d_clovi_df : (const void*)c->d_clovi32);
  a.lb_fault = c->debug_wait_fault ? 1 : 0;
  a.queue = c->d_err + 1;
  int p = a.p_out;
  if (b.nitems[p] == 0) return DD_OK;
  const long long nblk = (long long)b.nitems[p] * b.nrhs;
  if (nblk > 0x7fffffffLL) return fail(c, DD_EINVAL, "batch too large for one launch");
  dd::TimingRec rec;
  bool tm = c->timing;
  if (tm) {
    if (!c->d_tbytes) {
      if ((st = dalloc(c, (void**)&c->d_tbytes, 3 * sizeof(double))) != DD_OK) return st;
      DD_CUDA(c, cudaMemset(c->d_tbytes, 0, 3 * sizeof(double)));
    }
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    rec.which = (prec == DD_F64 || prec == DD_DF64) ? 0 : (prec == DD_F32 ? 1 : 2);
    rec.bytes = 0.0;
    a.work_bytes = c->d_tbytes + rec.which;
    a.site_bytes = hop_site_bytes(b, prec_bytes(prec), (a.s1 ? 1 : 0) + (a.s2 ? 1 : 0));
    cudaEventRecord(rec.a, s);
  }
  if (!c->nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (c->nsm <= 0) c->nsm = 1;
  }
  const int pi = (prec == DD_F64 || prec == DD_DF64) ? 0 : (prec == DD_F32 ? 1 : 2);
  const int v = c->forced_variant[pi] >= 0 ? c->forced_variant[pi] : b.hop_variant[pi];
  dispatch_hop(prec, v, bd, a, b.nitems[p], c->nsm, s);
  if (tm) {
    cudaEventRecord(rec.b, s);
    c->trec.push_back(rec);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// ---- caller layout <-> internal SoA --------------------------------------------
// caller: [j][r][field-order site][12] complex128; internal: per parity, per
// system 12 x n_p complex at the storage precision.  grid: (nfitems, nrhs), one
// thread per field position, so a warp reads or writes one contiguous 6 KB run
// of the caller layout; each parity's share of it is a contiguous run too.
struct FieldSite {
  int p, i, np, f;
  bool live;
};
__device__ __forceinline__ FieldSite field_site(const BatchDev& bd, const DomInst* d, int4 it) {
  FieldSite fs;
  fs.live = threadIdx.x < it.z;
  fs.f = it.y + (fs.live ? threadIdx.x : 0);
  const int v = d->ifm[fs.f];
  fs.p = v >> 30;
  fs.i = v & ((1 << 30) - 1);
  fs.np = fs.p ? d->n[1] : d->n[0];
  return fs;
}

template <class S>
__global__ void k_pack(BatchDev bd, const double2* __restrict__ user, S* __restrict__ ve, S* __restrict__ vo) {
  typedef typename StoreTraits<S>::C C;
  const int4 it = bd.fitems[blockIdx.x];
  const int r = blockIdx.y;
  if (threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* d = bd.inst_tab + bd.inst[it.x];
  const FieldSite fs = field_site(bd, d, it);
  const double2* src = user + bd.uoff[sys] + 12LL * fs.f;
  S* dst = (fs.p ? vo + bd.off[1][sys] : ve + bd.off[0][sys]);
  C w[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) w[k] = cmk<C>(src[k].x, src[k].y);
  st_site<12>(dst, fs.np, fs.i, w);
}

template <class S>
__global__ void k_unpack(BatchDev bd, const S* __restrict__ ve, const S* __restrict__ vo,
                         double2* __restrict__ user) {
  const int4 it = bd.fitems[blockIdx.x];
  const int r = blockIdx.y;
  if (threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* d = bd.inst_tab + bd.inst[it.x];
  const FieldSite fs = field_site(bd, d, it);
  double2* dst = user + bd.uoff[sys] + 12LL * fs.f;
  const S* src = (fs.p ? vo + bd.off[1][sys] : ve + bd.off[0][sys]);
  typename StoreTraits<S>::C w[12];
  ld_site<12>(src, fs.np, fs.i, w);
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = to_d2(w[k]);
}

// start of a solve in one pass: b (caller layout) -> b and r = b at the outer
// precision (FP64 or double-float), x = 0
template <class S>
__global__ void k_pack_init(BatchDev bd, const double2* __restrict__ user, S* be, S* bo, S* re, S* ro, S* xe,
                            S* xo) {
  typedef typename StoreTraits<S>::C C;
  const int4 it = bd.fitems[blockIdx.x];
  const int r = blockIdx.y;
  if (threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* d = bd.inst_tab + bd.inst[it.x];
  const FieldSite fs = field_site(bd, d, it);
  const double2* src = user + bd.uoff[sys] + 12LL * fs.f;
  const long long o = fs.p ? bd.off[1][sys] : bd.off[0][sys];
  C w[12], z[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    w[k] = cmk<C>(src[k].x, src[k].y);
    z[k] = cmk<C>(0.0, 0.0);
  }
  st_site<12>((fs.p ? bo : be) + o, fs.np, fs.i, w);
  st_site<12>((fs.p ? ro : re) + o, fs.np, fs.i, w);
  st_site<12>((fs.p ? xo : xe) + o, fs.np, fs.i, z);
}

dd_status launch_pack_init(dd_ctx* c, const Batch& b, const double* user, void* be, void* bo, void* re,
                           void* ro, void* xe, void* xo, dd_prec prec, cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  if (prec != DD_F64 && prec != DD_DF64) return fail(c, DD_EINVAL, "internal: outer precision");
  if (b.nfitems == 0) return DD_OK;
  BatchDev bd = batch_view(c, b);
  dim3 grid(b.nfitems, b.nrhs);
  const double2* u = (const double2*)user;
  if (prec == DD_DF64)
    DD_COUNT_LAUNCH(), k_pack_init<df2s><<<grid, 128, 0, s>>>(bd, u, (df2s*)be, (df2s*)bo, (df2s*)re, (df2s*)ro,
                                                              (df2s*)xe, (df2s*)xo);
  else
    DD_COUNT_LAUNCH(), k_pack_init<double2><<<grid, 128, 0, s>>>(bd, u, (double2*)be, (double2*)bo, (double2*)re,
                                                                 (double2*)ro, (double2*)xe, (double2*)xo);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

dd_status launch_pack(dd_ctx* c, const Batch& b, const double* user, void* ve, void* vo,
                      dd_prec prec, cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  if (b.nfitems == 0) return DD_OK;
  BatchDev bd = batch_view(c, b);
  dim3 grid(b.nfitems, b.nrhs);
  const double2* u = (const double2*)user;
  if (prec == DD_DF64) DD_COUNT_LAUNCH(), k_pack<df2s><<<grid, 128, 0, s>>>(bd, u, (df2s*)ve, (df2s*)vo);
  else if (prec == DD_F64) DD_COUNT_LAUNCH(), k_pack<double2><<<grid, 128, 0, s>>>(bd, u, (double2*)ve, (double2*)vo);
  else if (prec == DD_F32) DD_COUNT_LAUNCH(), k_pack<float2><<<grid, 128, 0, s>>>(bd, u, (float2*)ve, (float2*)vo);
  else
    DD_COUNT_LAUNCH(), k_pack<__nv_bfloat162><<<grid, 128, 0, s>>>(bd, u, (__nv_bfloat162*)ve, (__nv_bfloat162*)vo);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

dd_status launch_unpack(dd_ctx* c, const Batch& b, const void* ve, const void* vo, double* user, dd_prec prec,
                        cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  if (b.nfitems == 0) return DD_OK;
  BatchDev bd = batch_view(c, b);
  dim3 grid(b.nfitems, b.nrhs);
  double2* u = (double2*)user;
  if (prec == DD_DF64)
    DD_COUNT_LAUNCH(), k_unpack<df2s><<<grid, 128, 0, s>>>(bd, (const df2s*)ve, (const df2s*)vo, u);
  else if (prec == DD_F64)
    DD_COUNT_LAUNCH(), k_unpack<double2><<<grid, 128, 0, s>>>(bd, (const double2*)ve, (const double2*)vo, u);
  else if (prec == DD_F32)
    DD_COUNT_LAUNCH(), k_unpack<float2><<<grid, 128, 0, s>>>(bd, (const float2*)ve, (const float2*)vo, u);
  else
    DD_COUNT_LAUNCH(), k_unpack<__nv_bfloat162><<<grid, 128, 0, s>>>(bd, (const __nv_bfloat162*)ve,
                                                                     (const __nv_bfloat162*)vo, u);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

}  // namespace dd

extern "C" {

int dd_hop_variants(dd_prec prec) { return dd::hop_variant_count(prec); }

const char* dd_hop_variant_name(dd_prec prec, int v) {
  if (prec != DD_F64 && prec != DD_F32 && prec != DD_BF16) return nullptr;
  if (v < 0 || v >= dd::hop_variant_count(prec) || v >= 32) return nullptr;
  static char names[3][32][112];
  static bool made = false;
  if (!made) {
    const dd_prec ps[3] = {DD_F64, DD_F32, DD_BF16};
    const char* ty[3] = {"double2", "float2", "bfloat162"};
    for (int k = 0; k < 3; ++k)
      for (int u = 0; u < dd::hop_variant_count(ps[k]) && u < 32; ++u) {
        const dd::HopVariant& h = dd::variant_of(ps[k], u);
        if (h.r < 0 && h.qpc == 4 && h.maxr == 12 && !h.persist)
          snprintf(names[k][u], sizeof names[k][u],
                   "k_hop_lb<%s,%d,%d>: links by bulk copy into shared memory, up to 12 rhs per CTA, %d per thread",
                   ty[k], h.minb, -h.r, -h.r);
        else if (h.r < 0 && h.persist)
          snprintf(names[k][u], sizeof names[k][u],
                   "k_hop_lbq<%s,%d,%d,%d,%d>: work-queue persistent bundle form, %d sites and up to %d rhs per unit",
                   ty[k], h.minb, -h.r, h.qpc, h.maxr, 32 * h.qpc, h.maxr);
        else if (h.r < 0)
          snprintf(names[k][u], sizeof names[k][u],
                   "k_hop_lb<%s,%d,%d,%d,%d>: bulk-copied links, %d sites and up to %d rhs per CTA",
                   ty[k], h.minb, -h.r, h.qpc, h.maxr, 32 * h.qpc, h.maxr);
        else if (h.r == 0)
          snprintf(names[k][u], sizeof names[k][u], "k_hop_split<%s,%d,%s>: forward/backward split",
                   ty[k], h.minb, h.persist ? "persistent" : "grid");
        else
          snprintf(names[k][u], sizeof names[k][u], "k_hop<%s,%d,%s,%d>: %d rhs per thread", ty[k], h.minb,
                   h.persist ? "persistent" : "grid", h.r, h.r);
      }
    made = true;
  }
  return names[prec == DD_F64 ? 0 : (prec == DD_F32 ? 1 : 2)][v];
}

dd_status dd_set_hop_variant(dd_ctx* c, dd_prec prec, int v) {
  if (!c || (prec != DD_F64 && prec != DD_F32 && prec != DD_BF16)) return DD_EINVAL;
  if (v < -1 || v >= dd::hop_variant_count(prec)) return dd::fail(c, DD_EINVAL, "variant out of range");
  c->forced_variant[prec == DD_F64 ? 0 : (prec == DD_F32 ? 1 : 2)] = v;
  return DD_OK;
}

dd_status dd_debug_wait_fault(dd_ctx* c, int on) {
  if (!c) return DD_EINVAL;
  c->debug_wait_fault = on != 0;
  return DD_OK;
}

}  // extern "C"
