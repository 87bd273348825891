// Batched block solves x = D_X^{-1} b (paper Sec. 3: D_{Omega0^a}^{-1},
// D_{Phi1^a}^{-1}, D_{Lambda1}^{-1}) for many (domain instance, rhs) systems.
//
// Each system is even-odd preconditioned:
//   (1 - k^2 H_eo H_oe) x_e = b_e + k H_eo b_o,   x_o = b_o + k H_oe x_e,
// and the even system is solved by BiCGstab (van der Vorst 1992) inside an
// FP64 defect-correction loop: the outer residual r = b^_e - M x_e is always
// formed in FP64; the inner BiCGstab runs at FP64 (plain form) or at
// FP32 / BF16 storage with FP32 arithmetic (mixed forms) and FP64 inner
// products.  All per-system scalars live on the device; the host only polls
// the number of unconverged systems every `check_every` iterations.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

struct SysState {
  double2 rho, alpha, omega, beta;
  double rr;        // current |r|^2 of the inner recursion (or outer residual)
  double target2;   // inner stopping threshold on |r|^2
  double bnorm2;    // |b|^2 of the full (both-parity) right-hand side
  double outer2;    // outer threshold (tol |b|)^2
  int active;       // inner recursion running
  int outer_active; // outer loop still running
  int iters;        // inner iterations, summed over cycles
  int status;       // 0 ok, 1 converged, 2 breakdown
};

namespace {

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// sum of one partial slot for system (j, r) over the items of instance j
__device__ __forceinline__ double2 sum_slot(const double* partial, int slot, long long stride,
                                            int ib0, int ib1, int nrhs, int r) {
  double2 s = make_double2(0.0, 0.0);
  const double* P = partial + 2 * slot * stride;
  for (int it = ib0; it < ib1; ++it) {
    long long k = (long long)it * nrhs + r;
    s.x += P[2 * k];
    s.y += P[2 * k + 1];
  }
  return s;
}

// ---- elementwise kernels over the even parity, grid (nitems[0], nrhs) -----------
#define ELEM_PROLOGUE                                            \
  const int4 it = bd.items[0][blockIdx.x];                       \
  const int rh = blockIdx.y;                                     \
  const int sys = it.x * bd.nrhs + rh;                           \
  const DomInst d = bd.inst_tab[bd.inst[it.x]];                  \
  const int n = d.n[0];                                          \
  const int i = it.y + threadIdx.x;                              \
  const bool live = threadIdx.x < it.z;                          \
  const long long o = bd.off[0][sys] + i;

template <class S>
__global__ void k_inner_init(BatchDev bd, const SysState* st, const S* __restrict__ rhs, S* r,
                             S* rhat, S* p, S* v, S* x, double* partial) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[64];
  ELEM_PROLOGUE
  double acc[1] = {0.0};
  if (live) {
    const C z = cmk<C>(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      long long q = o + (long long)k * n;
      C b = ldc(rhs + q);
      stc(r + q, b);
      stc(rhat + q, b);
      stc(p + q, z);
      stc(v + q, z);
      stc(x + q, z);
      acc[0] += (double)b.x * b.x + (double)b.y * b.y;
    }
  }
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) {
    long long stride = (long long)bd.nitems[0] * bd.nrhs;
    long long m = (long long)blockIdx.x * bd.nrhs + rh;
    partial[2 * m] = acc[0];
    partial[2 * m + 1] = 0.0;
    partial[2 * (stride + m)] = acc[0];
    partial[2 * (stride + m) + 1] = 0.0;
  }
  (void)st;
}

template <class S>
__global__ void k_p_update(BatchDev bd, const SysState* st, const S* __restrict__ r, S* p,
                           const S* __restrict__ v) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  ELEM_PROLOGUE
  if (!live || !st[sys].active) return;
  const C beta = cmk<C>(st[sys].beta.x, st[sys].beta.y);
  const C om = cmk<C>(st[sys].omega.x, st[sys].omega.y);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    long long q = o + (long long)k * n;
    C pp = ldc(p + q), vv = ldc(v + q), rr = ldc(r + q);
    C t = csub(pp, cmul(om, vv));
    C res = cadd(rr, cmul(beta, t));
    stc(p + q, res);
  }
  (void)sizeof(T);
}

template <class S>
__global__ void k_s_update(BatchDev bd, const SysState* st, const S* __restrict__ r,
                           const S* __restrict__ v, S* s) {
  typedef typename StoreTraits<S>::C C;
  ELEM_PROLOGUE
  if (!live || !st[sys].active) return;
  const C al = cmk<C>(st[sys].alpha.x, st[sys].alpha.y);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    long long q = o + (long long)k * n;
    stc(s + q, csub(ldc(r + q), cmul(al, ldc(v + q))));
  }
}

// x += alpha p + omega s ; r = s - omega t ; partials (rhat, r) and |r|^2
template <class S>
__global__ void k_xr_update(BatchDev bd, const SysState* st, S* x, S* r, const S* __restrict__ p,
                            const S* __restrict__ s, const S* __restrict__ t,
                            const S* __restrict__ rhat, double* partial) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[96];
  ELEM_PROLOGUE
  if (!st[sys].active) return;
  double acc[3] = {0.0, 0.0, 0.0};
  if (live) {
    const C al = cmk<C>(st[sys].alpha.x, st[sys].alpha.y);
    const C om = cmk<C>(st[sys].omega.x, st[sys].omega.y);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      long long q = o + (long long)k * n;
      C ss = ldc(s + q);
      C xx = cadd(ldc(x + q), cadd(cmul(al, ldc(p + q)), cmul(om, ss)));
      stc(x + q, xx);
      C rr = csub(ss, cmul(om, ldc(t + q)));
      stc(r + q, rr);
      C rh = ldc(rhat + q);
      acc[0] += (double)rh.x * rr.x + (double)rh.y * rr.y;
      acc[1] += (double)rh.x * rr.y - (double)rh.y * rr.x;
      acc[2] += (double)rr.x * rr.x + (double)rr.y * rr.y;
    }
  }
  block_reduce<3>(acc, red);
  if (threadIdx.x == 0) {
    long long stride = (long long)bd.nitems[0] * bd.nrhs;
    long long m = (long long)blockIdx.x * bd.nrhs + rh;
    partial[2 * m] = acc[0];
    partial[2 * m + 1] = acc[1];
    partial[2 * (stride + m)] = acc[2];
    partial[2 * (stride + m) + 1] = 0.0;
  }
}

// |v|^2 per system over parity p into slot `slot`
template <class S>
__global__ void k_norm2(BatchDev bd, int p, const S* __restrict__ v, double* partial, int slot) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[64];
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  const int sys = it.x * bd.nrhs + r;
  const DomInst d = bd.inst_tab[bd.inst[it.x]];
  const int n = p ? d.n[1] : d.n[0];
  const int i = it.y + threadIdx.x;
  double acc[1] = {0.0};
  if (threadIdx.x < it.z) {
    const long long o = (p ? bd.off[1] : bd.off[0])[sys] + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      C w = ldc(v + o + (long long)k * n);
      acc[0] += (double)w.x * w.x + (double)w.y * w.y;
    }
  }
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) {
    long long stride = (long long)(p ? bd.nitems[1] : bd.nitems[0]) * bd.nrhs;
    long long m = (long long)blockIdx.x * bd.nrhs + r;
    partial[2 * (slot * stride + m)] = acc[0];
    partial[2 * (slot * stride + m) + 1] = 0.0;
  }
}

// y (type D) = x (type S), even parity, every system
template <class SD, class SS>
__global__ void k_convert(BatchDev bd, SD* y, const SS* __restrict__ x, const SysState* st,
                          int only_outer_active) {
  typedef typename StoreTraits<SD>::C CD;
  ELEM_PROLOGUE
  if (!live) return;
  if (only_outer_active && !st[sys].outer_active) return;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    long long q = o + (long long)k * n;
    auto v = ldc(x + q);
    stc(y + q, cmk<CD>((double)v.x, (double)v.y));
  }
}

// x64 += e (type S) for systems still in the outer loop
template <class S>
__global__ void k_accumulate(BatchDev bd, double2* x, const S* __restrict__ e, const SysState* st) {
  ELEM_PROLOGUE
  if (!live || !st[sys].outer_active) return;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    long long q = o + (long long)k * n;
    auto v = ldc(e + q);
    double2 a = x[q];
    x[q] = make_double2(a.x + (double)v.x, a.y + (double)v.y);
  }
}

__global__ void k_zero64(double2* x, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) x[k] = make_double2(0.0, 0.0);
}

// ---- per-system scalar kernels (one thread per system) ----------------------------
struct ScalarArgs {
  SysState* st;
  const double* partial;
  const int* item_begin;
  long long stride;
  int nsys, nrhs;
};

__global__ void k_sc_bnorm(ScalarArgs a, const double* partial_o, const int* ib_o, long long stride_o,
                           double tol2) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double be = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  double bo = sum_slot(partial_o, 0, stride_o, ib_o[j], ib_o[j + 1], a.nrhs, r).x;
  SysState& s = a.st[sys];
  memset(&s, 0, sizeof(SysState));
  s.bnorm2 = be + bo;
  s.outer2 = tol2 * (be + bo);
  s.outer_active = 1;
}

// outer residual |r|^2 (slot 0) -> outer_active
__global__ void k_sc_outer(ScalarArgs a, int* count) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  SysState& s = a.st[sys];
  double rr = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.rr = rr;
  s.outer_active = (rr > s.outer2) && !(rr != rr) ? 1 : 0;
  if (rr != rr) s.status = 3;
  if (s.outer_active) atomicAdd(count, 1);
}

// inner init: rho = |r|^2, alpha = omega = 1, threshold, active
__global__ void k_sc_inner_init(ScalarArgs a, double inner_tol2, double floor_frac) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  SysState& s = a.st[sys];
  double rr = sum_slot(a.partial, 1, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.rr = rr;
  s.rho = make_double2(rr, 0.0);
  s.alpha = s.omega = make_double2(1.0, 0.0);
  s.beta = make_double2(0.0, 0.0);
  s.target2 = fmax(inner_tol2 * rr, floor_frac * s.outer2);
  s.active = s.outer_active && rr > s.target2;
}

__global__ void k_sc_beta(ScalarArgs a, int* count) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  SysState& s = a.st[sys];
  if (!s.active) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double2 rho_new = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r);
  double rr = sum_slot(a.partial, 1, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.rr = rr;
  if (!(rr > s.target2)) {            // converged (or NaN: caught by the outer check)
    s.active = 0;
    return;
  }
  if (rho_new.x == 0.0 && rho_new.y == 0.0) {
    s.active = 0;
    s.status = 2;
    return;
  }
  s.beta = zmul(zdiv(rho_new, s.rho), zdiv(s.alpha, s.omega));
  s.rho = rho_new;
  s.iters += 1;
  if (count) atomicAdd(count, 1);
}

__global__ void k_sc_alpha(ScalarArgs a) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  SysState& s = a.st[sys];
  if (!s.active) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double2 den = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r);
  if (den.x == 0.0 && den.y == 0.0) {
    s.active = 0;
    s.status = 2;
    return;
  }
  s.alpha = zdiv(s.rho, den);
}

__global__ void k_sc_omega(ScalarArgs a) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  SysState& s = a.st[sys];
  if (!s.active) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double2 ts = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r);
  double tt = sum_slot(a.partial, 1, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.omega = tt > 0.0 ? make_double2(ts.x / tt, ts.y / tt) : make_double2(0.0, 0.0);
}

__global__ void k_sc_residual(ScalarArgs a, const double* partial_o, const int* ib_o,
                              long long stride_o, double* relres) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double re = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  double ro = sum_slot(partial_o, 0, stride_o, ib_o[j], ib_o[j + 1], a.nrhs, r).x;
  double b2 = a.st[sys].bnorm2;
  relres[sys] = b2 > 0 ? sqrt((re + ro) / b2) : sqrt(re + ro);
}

}  // namespace

// ---------------------------------------------------------------------------
// workspace

struct Workspace {
  std::vector<void*> bufs;
  std::vector<size_t> sizes;
};

static dd_status ws_get(dd_ctx* c, int slot, size_t bytes, void** out) {
  static thread_local int dummy = 0;
  (void)dummy;
  // the context keeps a flat list of growable buffers in its scratch vector
  auto* ws = reinterpret_cast<Workspace*>(c->scratch);
  if (!ws) {
    ws = new Workspace();
    c->scratch = ws;
  }
  if ((int)ws->bufs.size() <= slot) {
    ws->bufs.resize(slot + 1, nullptr);
    ws->sizes.resize(slot + 1, 0);
  }
  if (ws->sizes[slot] < bytes) {
    dfree(ws->bufs[slot]);
    ws->bufs[slot] = nullptr;
    ws->sizes[slot] = 0;
    dd_status st = dalloc(c, &ws->bufs[slot], bytes);
    if (st != DD_OK) return st;
    ws->sizes[slot] = bytes;
  }
  *out = ws->bufs[slot];
  return DD_OK;
}

void free_workspace(dd_ctx* c) {
  auto* ws = reinterpret_cast<Workspace*>(c->scratch);
  if (!ws) return;
  for (void* p : ws->bufs) dfree(p);
  delete ws;
  c->scratch = nullptr;
}

dd_status workspace(dd_ctx* c, int slot, size_t bytes, void** out) { return ws_get(c, slot, bytes, out); }

// ---------------------------------------------------------------------------
// the solver

namespace {

struct InnerVecs {
  void *r, *rhat, *p, *v, *s, *t, *x, *tmp;
};

template <class S>
dd_status run_bicgstab(dd_ctx* c, const Batch& b, dd_prec prec, const InnerVecs& w, SysState* st,
                       double* partial, int* d_count, int* h_count, const void* rhs,
                       double inner_tol2, double floor_frac, int maxiter, int check_every,
                       cudaStream_t s, int* iters_run) {
  BatchDev bd = batch_view(c, b);
  const int nsys = b.nb * b.nrhs;
  const long long stride = (long long)b.nitems[0] * b.nrhs;
  ScalarArgs sa{st, partial, b.d_item_begin[0], stride, nsys, b.nrhs};
  const int sth = 128, sbl = (nsys + sth - 1) / sth;
  dim3 eg(b.nitems[0], b.nrhs);
  const double k2 = c->kappa * c->kappa;
  k_inner_init<S><<<eg, 128, 0, s>>>(bd, st, (const S*)rhs, (S*)w.r, (S*)w.rhat, (S*)w.p, (S*)w.v,
                                     (S*)w.x, partial);
  k_sc_inner_init<<<sbl, sth, 0, s>>>(sa, inner_tol2, floor_frac);
  DD_CUDA(c, cudaGetLastError());
  int it = 0;
  for (; it < maxiter; ++it) {
    bool check = ((it + 1) % check_every) == 0;
    if (check) DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
    k_sc_beta<<<sbl, sth, 0, s>>>(sa, check ? d_count : nullptr);
    k_p_update<S><<<eg, 128, 0, s>>>(bd, st, (const S*)w.r, (S*)w.p, (const S*)w.v);
    // v = M p = p - k^2 H_eo H_oe p ; partial (rhat, v)
    HopArgs h1{};
    h1.p_out = 1; h1.in = w.p; h1.out = w.tmp; h1.b = 1.0;
    h1.active = (const int*)((const char*)st + offsetof(SysState, active));
    h1.active_stride = (int)(sizeof(SysState) / sizeof(int));
    dd_status e = launch_hop(c, b, prec, h1, s);
    if (e != DD_OK) return e;
    HopArgs h2{};
    h2.p_out = 0; h2.in = w.tmp; h2.out = w.v; h2.s1 = w.p; h2.a1 = 1.0; h2.b = -k2;
    h2.dotq = w.rhat; h2.partial = partial;
    h2.active = h1.active; h2.active_stride = h1.active_stride;
    if ((e = launch_hop(c, b, prec, h2, s)) != DD_OK) return e;
    k_sc_alpha<<<sbl, sth, 0, s>>>(sa);
    k_s_update<S><<<eg, 128, 0, s>>>(bd, st, (const S*)w.r, (const S*)w.v, (S*)w.s);
    HopArgs h3{};
    h3.p_out = 1; h3.in = w.s; h3.out = w.tmp; h3.b = 1.0;
    h3.active = h1.active; h3.active_stride = h1.active_stride;
    if ((e = launch_hop(c, b, prec, h3, s)) != DD_OK) return e;
    HopArgs h4{};
    h4.p_out = 0; h4.in = w.tmp; h4.out = w.t; h4.s1 = w.s; h4.a1 = 1.0; h4.b = -k2;
    h4.dots = w.s; h4.partial = partial;
    h4.active = h1.active; h4.active_stride = h1.active_stride;
    if ((e = launch_hop(c, b, prec, h4, s)) != DD_OK) return e;
    k_sc_omega<<<sbl, sth, 0, s>>>(sa);
    k_xr_update<S><<<eg, 128, 0, s>>>(bd, st, (S*)w.x, (S*)w.r, (const S*)w.p, (const S*)w.s,
                                      (const S*)w.t, (const S*)w.rhat, partial);
    DD_CUDA(c, cudaGetLastError());
    if (check) {
      DD_CUDA(c, cudaMemcpyAsync(h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
      DD_CUDA(c, cudaStreamSynchronize(s));
      if (*h_count == 0) {
        ++it;
        break;
      }
    }
  }
  // final beta pass marks converged systems (updates rr) without a p update
  k_sc_beta<<<sbl, sth, 0, s>>>(sa, nullptr);
  *iters_run = it;
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

}  // namespace

dd_status solve_batch(dd_ctx* c, const Batch& b, const double* b_user, double* x_user,
                      const dd_solve_params* prm, dd_solve_stats* stats, cudaStream_t s,
                      bool /*user_layout*/) {
  dd_status e;
  const int nsys = b.nb * b.nrhs;
  const dd_prec ip = prm->inner_prec;
  const size_t c64 = 16, cin = prec_bytes(ip);
  const long long ne = b.tot[0], no = b.tot[1];
  // workspace slots: 0..6 FP64 outer, 7..14 inner, 15 partial, 16 states, 17 counters, 18 relres, 19 partial_o
  void *be, *bo, *bh, *xe, *xo, *r64, *t64;
  if ((e = ws_get(c, 0, ne * c64, &be)) || (e = ws_get(c, 1, no * c64, &bo)) ||
      (e = ws_get(c, 2, ne * c64, &bh)) || (e = ws_get(c, 3, ne * c64, &xe)) ||
      (e = ws_get(c, 4, no * c64, &xo)) || (e = ws_get(c, 5, ne * c64, &r64)) ||
      (e = ws_get(c, 6, no * c64, &t64)))
    return e;
  InnerVecs w;
  if ((e = ws_get(c, 7, ne * cin, &w.r)) || (e = ws_get(c, 8, ne * cin, &w.rhat)) ||
      (e = ws_get(c, 9, ne * cin, &w.p)) || (e = ws_get(c, 10, ne * cin, &w.v)) ||
      (e = ws_get(c, 11, ne * cin, &w.s)) || (e = ws_get(c, 12, ne * cin, &w.t)) ||
      (e = ws_get(c, 13, ne * cin, &w.x)) || (e = ws_get(c, 14, no * cin, &w.tmp)))
    return e;
  void *vpart, *vst, *vcnt, *vrel, *vpart_o;
  const long long stride = (long long)b.nitems[0] * b.nrhs;
  const long long stride_o = (long long)b.nitems[1] * b.nrhs;
  if ((e = ws_get(c, 15, sizeof(double) * 2 * 3 * std::max<long long>(1, stride), &vpart)) ||
      (e = ws_get(c, 16, sizeof(SysState) * nsys, &vst)) || (e = ws_get(c, 17, 64, &vcnt)) ||
      (e = ws_get(c, 18, sizeof(double) * nsys, &vrel)) ||
      (e = ws_get(c, 19, sizeof(double) * 2 * std::max<long long>(1, stride_o), &vpart_o)))
    return e;
  double* partial = (double*)vpart;
  double* partial_o = (double*)vpart_o;
  SysState* st = (SysState*)vst;
  int* d_count = (int*)vcnt;
  int h_count = 0;
  for (int j = 0; j < b.nb; ++j) {
    if ((e = ensure_links(c, b.inst[j], DD_F64)) != DD_OK) return e;
    if (ip != DD_F64 && (e = ensure_links(c, b.inst[j], ip)) != DD_OK) return e;
  }
  if ((e = sync_instances(c)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  ScalarArgs sa{st, partial, b.d_item_begin[0], stride, nsys, b.nrhs};
  const int sth = 128, sbl = (nsys + sth - 1) / sth;
  dim3 eg(b.nitems[0], b.nrhs), og(b.nitems[1], b.nrhs);
  const double kap = c->kappa, k2 = kap * kap;

  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, s);

  if ((e = launch_pack(c, b, b_user, be, bo, DD_F64, s)) != DD_OK) return e;
  // |b|^2 over both parities
  k_norm2<double2><<<eg, 128, 0, s>>>(bd, 0, (const double2*)be, partial, 0);
  if (b.nitems[1]) k_norm2<double2><<<og, 128, 0, s>>>(bd, 1, (const double2*)bo, partial_o, 0);
  k_sc_bnorm<<<sbl, sth, 0, s>>>(sa, partial_o, b.d_item_begin[1], stride_o, prm->tol * prm->tol);
  // b^_e = b_e + k H_eo b_o
  {
    HopArgs h{};
    h.p_out = 0; h.in = bo; h.out = bh; h.s1 = be; h.a1 = 1.0; h.b = kap;
    if ((e = launch_hop(c, b, DD_F64, h, s)) != DD_OK) return e;
  }
  k_zero64<<<(ne + 255) / 256, 256, 0, s>>>((double2*)xe, ne);
  DD_CUDA(c, cudaMemcpyAsync(r64, bh, ne * c64, cudaMemcpyDeviceToDevice, s));
  DD_CUDA(c, cudaGetLastError());

  const int check_every = std::max(1, prm->check_every);
  const int max_outer = ip == DD_F64 ? std::max(1, prm->max_outer) : std::max(1, prm->max_outer);
  const double inner_tol2 = ip == DD_F64 ? 0.0 : prm->inner_tol * prm->inner_tol;
  const double floor_frac = ip == DD_F64 ? 0.25 : 0.0;
  int cycles = 0, total_iters = 0;
  for (int cyc = 0; cyc < max_outer; ++cyc) {
    // outer residual norm and convergence
    k_norm2<double2><<<eg, 128, 0, s>>>(bd, 0, (const double2*)r64, partial, 0);
    DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
    k_sc_outer<<<sbl, sth, 0, s>>>(sa, d_count);
    DD_CUDA(c, cudaMemcpyAsync(&h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    if (h_count == 0) break;
    ++cycles;
    const void* rhs = r64;
    if (ip != DD_F64) {
      if (ip == DD_F32)
        k_convert<float2, double2><<<eg, 128, 0, s>>>(bd, (float2*)w.s, (const double2*)r64, st, 0);
      else
        k_convert<__nv_bfloat162, double2><<<eg, 128, 0, s>>>(bd, (__nv_bfloat162*)w.s,
                                                              (const double2*)r64, st, 0);
      rhs = w.s;   // k_inner_init copies rhs into r and rhat before s is reused
    }
    int its = 0;
    if (ip == DD_F64)
      e = run_bicgstab<double2>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                                floor_frac, prm->maxiter, check_every, s, &its);
    else if (ip == DD_F32)
      e = run_bicgstab<float2>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                               floor_frac, prm->maxiter, check_every, s, &its);
    else
      e = run_bicgstab<__nv_bfloat162>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                                       floor_frac, prm->maxiter, check_every, s, &its);
    if (e != DD_OK) return e;
    total_iters += its;
    // x_e += e ; r = b^_e - M x_e (FP64)
    if (ip == DD_F64) k_accumulate<double2><<<eg, 128, 0, s>>>(bd, (double2*)xe, (const double2*)w.x, st);
    else if (ip == DD_F32) k_accumulate<float2><<<eg, 128, 0, s>>>(bd, (double2*)xe, (const float2*)w.x, st);
    else k_accumulate<__nv_bfloat162><<<eg, 128, 0, s>>>(bd, (double2*)xe, (const __nv_bfloat162*)w.x, st);
    HopArgs h1{};
    h1.p_out = 1; h1.in = xe; h1.out = t64; h1.b = 1.0;
    if ((e = launch_hop(c, b, DD_F64, h1, s)) != DD_OK) return e;
    HopArgs h2{};
    h2.p_out = 0; h2.in = t64; h2.out = r64; h2.s1 = bh; h2.a1 = 1.0; h2.s2 = xe; h2.a2 = -1.0;
    h2.b = k2;
    if ((e = launch_hop(c, b, DD_F64, h2, s)) != DD_OK) return e;
  }
  // x_o = b_o + k H_oe x_e
  {
    HopArgs h{};
    h.p_out = 1; h.in = xe; h.out = xo; h.s1 = bo; h.a1 = 1.0; h.b = kap;
    if ((e = launch_hop(c, b, DD_F64, h, s)) != DD_OK) return e;
  }
  // true residual of the full system: res = b - D x, both parities (FP64)
  {
    HopArgs h{};
    h.p_out = 0; h.in = xo; h.out = r64; h.s1 = be; h.a1 = 1.0; h.s2 = xe; h.a2 = -1.0; h.b = kap;
    if ((e = launch_hop(c, b, DD_F64, h, s)) != DD_OK) return e;
    HopArgs g{};
    g.p_out = 1; g.in = xe; g.out = t64; g.s1 = bo; g.a1 = 1.0; g.s2 = xo; g.a2 = -1.0; g.b = kap;
    if ((e = launch_hop(c, b, DD_F64, g, s)) != DD_OK) return e;
    k_norm2<double2><<<eg, 128, 0, s>>>(bd, 0, (const double2*)r64, partial, 0);
    if (b.nitems[1]) k_norm2<double2><<<og, 128, 0, s>>>(bd, 1, (const double2*)t64, partial_o, 0);
    k_sc_residual<<<sbl, sth, 0, s>>>(sa, partial_o, b.d_item_begin[1], stride_o, (double*)vrel);
  }
  if ((e = launch_unpack(c, b, xe, xo, x_user, DD_F64, s)) != DD_OK) return e;
  cudaEventRecord(ev1, s);
  DD_CUDA(c, cudaGetLastError());
  std::vector<double> rel(nsys);
  std::vector<SysState> hst(nsys);
  DD_CUDA(c, cudaMemcpyAsync(rel.data(), vrel, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaMemcpyAsync(hst.data(), st, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  dd_solve_stats out{};
  out.systems = nsys;
  out.outer_cycles = cycles;
  out.seconds = ms * 1e-3;
  bool nan = false;
  for (int k = 0; k < nsys; ++k) {
    if (!(rel[k] == rel[k])) nan = true;
    out.max_relres = std::max(out.max_relres, rel[k]);
    out.max_iters = std::max(out.max_iters, hst[k].iters);
    if (rel[k] <= prm->tol) out.converged++;
  }
  (void)total_iters;
  if (stats) *stats = out;
  if (nan) return fail(c, DD_ENAN, "NaN in a solve residual");
  if (out.converged < nsys) {
    char buf[160];
    snprintf(buf, sizeof buf, "%d of %d systems above tolerance (max relres %.3e)",
             nsys - out.converged, nsys, out.max_relres);
    return fail(c, DD_ENOCONV, buf);
  }
  return DD_OK;
}

}  // namespace dd
