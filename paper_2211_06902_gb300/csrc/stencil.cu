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

template <int DIR, class S, class C>
__device__ __forceinline__ void hop_one(C (&acc)[12], int n0, int p, int i, int n_out,
                                        int n_in, int j, const S* __restrict__ in_sys,
                                        const S* __restrict__ lk) {
  constexpr int MU = DIR & 3;
  constexpr bool FWD = DIR < 4;
  if (j < 0) return;
  C psi[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) psi[k] = ldc(in_sys + (long long)k * n_in + j);
  C U[9];
  if (FWD) {
    const S* l = lk + (p ? 36LL * n0 : 0) + (long long)MU * 9 * n_out + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) U[c] = ldc(l + (long long)c * n_out);
  } else {
    const int q = 1 - p;
    const S* l = lk + (q ? 36LL * n0 : 0) + (long long)MU * 9 * n_in + j;
#pragma unroll
    for (int c = 0; c < 9; ++c) U[c] = ldc(l + (long long)c * n_in);
  }
  hop_dir<MU, FWD>(acc, psi, U);
}

// grid: nitems[p] * nrhs CTAs, rhs fastest (the CTAs that share a site chunk,
// and so its links, run together and hit L2); one output site per thread.
// One CTA work unit t = item * nrhs + rhs of the hop launch.
template <class S>
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
    hop_one<0, S>(acc, n0, p, i, n_out, n_in, jn[0], in_sys, lk);
    hop_one<1, S>(acc, n0, p, i, n_out, n_in, jn[1], in_sys, lk);
    hop_one<2, S>(acc, n0, p, i, n_out, n_in, jn[2], in_sys, lk);
    hop_one<3, S>(acc, n0, p, i, n_out, n_in, jn[3], in_sys, lk);
    hop_one<4, S>(acc, n0, p, i, n_out, n_in, jn[4], in_sys, lk);
    hop_one<5, S>(acc, n0, p, i, n_out, n_in, jn[5], in_sys, lk);
    hop_one<6, S>(acc, n0, p, i, n_out, n_in, jn[6], in_sys, lk);
    hop_one<7, S>(acc, n0, p, i, n_out, n_in, jn[7], in_sys, lk);
    const T b = (T)a.b;
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = cscale(acc[k], b);
    if (a.s1) {
      const S* s1 = (const S*)a.s1 + (p ? bd.off[1] : bd.off[0])[sys];
      const T a1 = (T)a.a1;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        C v = ldc(s1 + (long long)k * n_out + i);
        out[k].x = fma(a1, v.x, out[k].x);
        out[k].y = fma(a1, v.y, out[k].y);
      }
    }
    if (a.s2) {
      const S* s2 = (const S*)a.s2 + (p ? bd.off[1] : bd.off[0])[sys];
      const T a2 = (T)a.a2;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        C v = ldc(s2 + (long long)k * n_out + i);
        out[k].x = fma(a2, v.x, out[k].x);
        out[k].y = fma(a2, v.y, out[k].y);
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) stc(out_sys + (long long)k * n_out + i, out[k]);
  }
  const long long slot_stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
  const long long my = (long long)item * bd.nrhs + r;
  // per-thread sums in the storage's compute type (12 terms), FP64 across threads
  if (a.dotq) {
    double v[2] = {0.0, 0.0};
    T t[2] = {0, 0};
    if (live) {
      const S* q = (const S*)a.dotq + (p ? bd.off[1] : bd.off[0])[sys];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        C w = ldc(q + (long long)k * n_out + i);
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
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        C w = ldc(q + (long long)k * n_out + i);
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
}

// Launch variants chosen by the autotuner: MINB = resident CTAs per SM asked
// of the register allocator; PERSIST = a grid of (SMs x MINB) CTAs that walks
// the work units with a stride (one launch of persistent CTAs over blocks of
// any size) instead of one CTA per unit.
template <class S, int MINB, bool PERSIST>
__global__ void __launch_bounds__(HOP_THREADS, MINB) k_hop(BatchDev bd, HopArgs a, long long nunits) {
  __shared__ double red[32 * 4];
  if (PERSIST) {
    for (long long t = blockIdx.x; t < nunits; t += gridDim.x) hop_unit<S>(bd, a, t, red);
  } else {
    hop_unit<S>(bd, a, blockIdx.x, red);
  }
}

struct HopVariant {
  int minb;
  bool persist;
};
// per storage precision; index 0 is the default before tuning
static const HopVariant kVariants64[] = {{3, false}, {2, false}, {3, true}};
static const HopVariant kVariants32[] = {{6, false}, {4, false}, {8, false}, {6, true}, {4, true}};
static const HopVariant kVariants16[] = {{5, false}, {4, false}, {8, false}, {5, true}};

int hop_variant_count(dd_prec prec) { return prec == DD_F64 ? 3 : (prec == DD_F32 ? 5 : 4); }

static const HopVariant& variant_of(dd_prec prec, int v) {
  const HopVariant* t = prec == DD_F64 ? kVariants64 : (prec == DD_F32 ? kVariants32 : kVariants16);
  if (v < 0 || v >= hop_variant_count(prec)) v = 0;
  return t[v];
}

template <class S, int MINB, bool PERSIST>
static void launch_variant(const BatchDev& bd, const HopArgs& a, long long nunits, int nsm,
                           cudaStream_t s) {
  long long grid = nunits;
  if (PERSIST) grid = std::min<long long>(nunits, (long long)nsm * MINB);
  DD_COUNT_LAUNCH(), k_hop<S, MINB, PERSIST><<<(unsigned)grid, HOP_THREADS, 0, s>>>(bd, a, nunits);
}

static void dispatch_hop(dd_prec prec, int v, const BatchDev& bd, const HopArgs& a, long long n,
                         int nsm, cudaStream_t s) {
  const HopVariant& hv = variant_of(prec, v);
  if (prec == DD_F64) {
    if (hv.persist) launch_variant<double2, 3, true>(bd, a, n, nsm, s);
    else if (hv.minb == 2) launch_variant<double2, 2, false>(bd, a, n, nsm, s);
    else launch_variant<double2, 3, false>(bd, a, n, nsm, s);
  } else if (prec == DD_F32) {
    if (hv.persist && hv.minb == 4) launch_variant<float2, 4, true>(bd, a, n, nsm, s);
    else if (hv.persist) launch_variant<float2, 6, true>(bd, a, n, nsm, s);
    else if (hv.minb == 4) launch_variant<float2, 4, false>(bd, a, n, nsm, s);
    else if (hv.minb == 8) launch_variant<float2, 8, false>(bd, a, n, nsm, s);
    else launch_variant<float2, 6, false>(bd, a, n, nsm, s);
  } else {
    if (hv.persist) launch_variant<__nv_bfloat162, 5, true>(bd, a, n, nsm, s);
    else if (hv.minb == 4) launch_variant<__nv_bfloat162, 4, false>(bd, a, n, nsm, s);
    else if (hv.minb == 8) launch_variant<__nv_bfloat162, 8, false>(bd, a, n, nsm, s);
    else launch_variant<__nv_bfloat162, 5, false>(bd, a, n, nsm, s);
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
    rec.which = prec == DD_F64 ? 0 : (prec == DD_F32 ? 1 : 2);
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
  const int pi = prec == DD_F64 ? 0 : (prec == DD_F32 ? 1 : 2);
  dispatch_hop(prec, b.hop_variant[pi], bd, a, nblk, c->nsm, s);
  if (tm) {
    cudaEventRecord(rec.b, s);
    c->trec.push_back(rec);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// ---- caller layout <-> internal SoA --------------------------------------------
// caller: [j][r][field-order site][12] complex128; internal: per parity, per
// system 12 x n_p complex at the storage precision.  grid: (nitems[p], nrhs).
template <class S>
__global__ void k_pack(BatchDev bd, int p, const double2* __restrict__ user, S* __restrict__ v) {
  typedef typename StoreTraits<S>::C C;
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  if (threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst d = bd.inst_tab[bd.inst[it.x]];
  const int i = it.y + threadIdx.x;
  const int np = p ? d.n[1] : d.n[0];
  const int f = d.fmap[(p ? d.n[0] : 0) + i];
  const double2* src = user + bd.uoff[sys] + 12LL * f;
  S* dst = v + (p ? bd.off[1] : bd.off[0])[sys] + i;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 x = src[k];
    stc(dst + (long long)k * np, cmk<C>(x.x, x.y));
  }
}

template <class S>
__global__ void k_unpack(BatchDev bd, int p, const S* __restrict__ v, double2* __restrict__ user) {
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  if (threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst d = bd.inst_tab[bd.inst[it.x]];
  const int i = it.y + threadIdx.x;
  const int np = p ? d.n[1] : d.n[0];
  const int f = d.fmap[(p ? d.n[0] : 0) + i];
  double2* dst = user + bd.uoff[sys] + 12LL * f;
  const S* src = v + (p ? bd.off[1] : bd.off[0])[sys] + i;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    auto x = ldc(src + (long long)k * np);
    dst[k] = make_double2((double)x.x, (double)x.y);
  }
}

dd_status launch_pack(dd_ctx* c, const Batch& b, const double* user, void* ve, void* vo,
                      dd_prec prec, cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  BatchDev bd = batch_view(c, b);
  for (int p = 0; p < 2; ++p) {
    if (b.nitems[p] == 0) continue;
    dim3 grid(b.nitems[p], b.nrhs);
    void* v = p ? vo : ve;
    if (prec == DD_F64) DD_COUNT_LAUNCH(), k_pack<double2><<<grid, 128, 0, s>>>(bd, p, (const double2*)user, (double2*)v);
    else if (prec == DD_F32) DD_COUNT_LAUNCH(), k_pack<float2><<<grid, 128, 0, s>>>(bd, p, (const double2*)user, (float2*)v);
    else DD_COUNT_LAUNCH(), k_pack<__nv_bfloat162><<<grid, 128, 0, s>>>(bd, p, (const double2*)user, (__nv_bfloat162*)v);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

dd_status launch_unpack(dd_ctx* c, const Batch& b, const void* ve, const void* vo, double* user,
                        dd_prec prec, cudaStream_t s) {
  dd_status st = sync_instances(c);
  if (st != DD_OK) return st;
  BatchDev bd = batch_view(c, b);
  for (int p = 0; p < 2; ++p) {
    if (b.nitems[p] == 0) continue;
    dim3 grid(b.nitems[p], b.nrhs);
    const void* v = p ? vo : ve;
    if (prec == DD_F64) DD_COUNT_LAUNCH(), k_unpack<double2><<<grid, 128, 0, s>>>(bd, p, (const double2*)v, (double2*)user);
    else if (prec == DD_F32) DD_COUNT_LAUNCH(), k_unpack<float2><<<grid, 128, 0, s>>>(bd, p, (const float2*)v, (double2*)user);
    else DD_COUNT_LAUNCH(), k_unpack<__nv_bfloat162><<<grid, 128, 0, s>>>(bd, p, (const __nv_bfloat162*)v, (double2*)user);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

}  // namespace dd
