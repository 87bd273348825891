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
#include <functional>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

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
  const long long o = bd.off[0][sys];

// (the elementwise kernels touch the 12 components of site i of every vector
// at the same pair-layout positions o + cidx(k, n, i))

// r = p = rhs, x = 0; partials (r^, r) into slot 0 and |r|^2 into slot 1, with
// the generated shadow vector r^ of seed `seed` (nothing is stored for r^)
template <class S>
__global__ void k_inner_init(BatchDev bd, const S* __restrict__ rhs, S* r, S* p, S* x,
                             unsigned seed, double* partial) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  __shared__ double red[64];
  ELEM_PROLOGUE
  double acc[3] = {0.0, 0.0, 0.0};
  T t[3] = {0, 0, 0};
  if (live) {
    C b[12], z[12];
    ld_site<12>(rhs + o, n, i, b);
    const unsigned h = rhat_bits(seed, sys, i);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      z[k] = cmk<C>(0.0, 0.0);
      const C w = rhat_comp<C>(h, k);
      t[0] = fma(w.x, b[k].x, fma(w.y, b[k].y, t[0]));
      t[1] = fma(w.x, b[k].y, fma(-w.y, b[k].x, t[1]));
      t[2] = fma(b[k].x, b[k].x, fma(b[k].y, b[k].y, t[2]));
    }
    st_site<12>(r + o, n, i, b);
    st_site<12>(p + o, n, i, b);
    st_site<12>(x + o, n, i, z);
  }
  block_reduce_t<T, 3>(t, acc, red);
  if (threadIdx.x == 0) {
    long long stride = (long long)bd.nitems[0] * bd.nrhs;
    long long m = (long long)blockIdx.x * bd.nrhs + rh;
    partial[2 * m] = acc[0];
    partial[2 * m + 1] = acc[1];
    partial[2 * (stride + m)] = acc[2];
    partial[2 * (stride + m) + 1] = 0.0;
  }
}

template <class S>
__global__ void k_s_update(BatchDev bd, const SysState* st, const S* __restrict__ r,
                           const S* __restrict__ v, S* s) {
  typedef typename StoreTraits<S>::C C;
  ELEM_PROLOGUE
  if (!live || !st[sys].active) return;
  const C al = cmk<C>(st[sys].alpha.x, st[sys].alpha.y);
  C rr[12], vv[12];
  ld_site<12>(r + o, n, i, rr);
  ld_site<12>(v + o, n, i, vv);
#pragma unroll
  for (int k = 0; k < 12; ++k) rr[k] = csub(rr[k], cmul(al, vv[k]));
  st_site<12>(s + o, n, i, rr);
}

// End of a BiCGstab iteration with the next search direction fused in:
//   x += alpha p + omega s ;  r = s - omega t ;  p = r + beta (p - omega v)
// (beta of the next iteration is already known: rho_new = (r^, s) - omega (r^, t)
// comes from the inner products fused into the t = M s hop); partial |r|^2 into
// slot 1 for the convergence check
template <class S>
__global__ void k_xrp_update(BatchDev bd, const SysState* st, S* x, S* r, S* p,
                             const S* __restrict__ s, const S* __restrict__ t,
                             const S* __restrict__ v, double* partial) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[64];
  ELEM_PROLOGUE
  if (!st[sys].active) return;
  typedef typename StoreTraits<S>::T T;
  double acc[1] = {0.0};
  T tt[1] = {0};
  if (live) {
    const C al = cmk<C>(st[sys].alpha.x, st[sys].alpha.y);
    const C om = cmk<C>(st[sys].omega.x, st[sys].omega.y);
    const C be = cmk<C>(st[sys].beta.x, st[sys].beta.y);
    // two components at a time (one pair-layout word per vector): few live registers
#pragma unroll 2
    for (int q = 0; q < 6; ++q) {
      const long long e = o + ((long long)q * n + i) * 2;
      C xv[2], pv[2], sv[2], tv[2], vv[2];
      ld_pair(x + e, xv[0], xv[1]);
      ld_pair(p + e, pv[0], pv[1]);
      ld_pair(s + e, sv[0], sv[1]);
      ld_pair(t + e, tv[0], tv[1]);
      ld_pair(v + e, vv[0], vv[1]);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        xv[k] = cadd(xv[k], cadd(cmul(al, pv[k]), cmul(om, sv[k])));
        const C rr = csub(sv[k], cmul(om, tv[k]));
        tt[0] = fma(rr.x, rr.x, fma(rr.y, rr.y, tt[0]));
        pv[k] = cadd(rr, cmul(be, csub(pv[k], cmul(om, vv[k]))));
        sv[k] = rr;
      }
      st_pair(x + e, xv[0], xv[1]);
      st_pair(r + e, sv[0], sv[1]);
      st_pair(p + e, pv[0], pv[1]);
    }
  }
  block_reduce_t<T, 1>(tt, acc, red);
  if (threadIdx.x == 0) {
    long long stride = (long long)bd.nitems[0] * bd.nrhs;
    long long m = (long long)blockIdx.x * bd.nrhs + rh;
    partial[2 * (stride + m)] = acc[0];
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
    C w[12];
    ld_site<12>(v + (p ? bd.off[1] : bd.off[0])[sys], n, i, w);
    if constexpr (std::is_same<C, dfc>::value) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) t += nrm2f(w[k]);
      acc[0] = t;
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[0] += (double)w[k].x * w[k].x + (double)w[k].y * w[k].y;
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

#define ELEM_PROLOGUE_P                                              \
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];        \
  const int rh = blockIdx.y;                                          \
  const int sys = it.x * bd.nrhs + rh;                                \
  const DomInst* dp_ = bd.inst_tab + bd.inst[it.x];                   \
  const int n = p ? dp_->n[1] : dp_->n[0];                            \
  const int i = it.y + threadIdx.x;                                   \
  const bool live = threadIdx.x < it.z;                               \
  const long long o = (p ? bd.off[1] : bd.off[0])[sys];

// y (type SD) = x (type SS) on parity p, for systems still in the outer loop
template <class SD, class SS>
__global__ void k_convert(BatchDev bd, int p, SD* y, const SS* __restrict__ x, const SysState* st) {
  typedef typename StoreTraits<SD>::C CD;
  typedef typename StoreTraits<SS>::C CS;
  ELEM_PROLOGUE_P
  if (!live || !st[sys].outer_active) return;
  CS v[12];
  CD w[12];
  ld_site<12>(x + o, n, i, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    if constexpr (std::is_same<CS, dfc>::value) w[k] = v[k].h;      // nearest FP32 value
    else w[k] = cmk<CD>((double)v[k].x, (double)v[k].y);
  }
  st_site<12>(y + o, n, i, w);
}

// outer x += sign * e (e of type S) on parity p, for systems still in the
// outer loop; the outer vector is FP64 (double2) or double-float (df2s)
// (with partial: |x|^2 per (item, rhs) into slot 0 afterwards, for every
// system, updated or not, so the outer check needs no separate norm pass)
template <class O, class S>
__global__ void k_axpy64(BatchDev bd, int p, O* x, const S* __restrict__ e, double sign,
                         const SysState* st, double* partial) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<O>::C CO;
  __shared__ double red[64];
  ELEM_PROLOGUE_P
  const bool upd = live && st[sys].outer_active;
  if (!partial && !upd) return;
  double acc[1] = {0.0};
  if (live) {
    CO a[12];
    ld_site<12>(x + o, n, i, a);
    if (upd) {
      C v[12];
      ld_site<12>(e + o, n, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        if constexpr (std::is_same<CO, dfc>::value) {
          df_add(a[k].h.x, a[k].l.x, (float)sign * (float)v[k].x, 0.f);
          df_add(a[k].h.y, a[k].l.y, (float)sign * (float)v[k].y, 0.f);
        } else {
          a[k] = make_double2(fma(sign, (double)v[k].x, a[k].x), fma(sign, (double)v[k].y, a[k].y));
        }
      }
      st_site<12>(x + o, n, i, a);
    }
    if (partial) {
      if constexpr (std::is_same<CO, dfc>::value) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) t += nrm2f(a[k]);
        acc[0] = t;
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[0] += a[k].x * a[k].x + a[k].y * a[k].y;
      }
    }
  }
  if (!partial) return;
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) {
    const long long m = (long long)blockIdx.x * bd.nrhs + rh;
    partial[2 * m] = acc[0];
    partial[2 * m + 1] = 0.0;
  }
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

// outer residual |r|^2 over both parities -> outer_active, relres, count,
// largest relative residual (as ordered bits of a non-negative double)
__global__ void k_sc_outer(ScalarArgs a, const double* partial_o, const int* ib_o,
                           long long stride_o, double margin2, int* count,
                           unsigned long long* maxrel, double* relres, const int* last_true = nullptr) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  // inside the whole-solve graph the margin follows the device-side flag
  if (last_true) margin2 = *last_true ? 1.0 : 0.25;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  SysState& s = a.st[sys];
  double re = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  double ro = sum_slot(partial_o, 0, stride_o, ib_o[j], ib_o[j + 1], a.nrhs, r).x;
  double rr = re + ro;
  s.rr = rr;
  if (rr != rr) s.status = 3;
  s.outer_active = (rr > margin2 * s.outer2) && (rr == rr) ? 1 : 0;
  double rel = s.bnorm2 > 0 ? sqrt(rr / s.bnorm2) : sqrt(rr);
  relres[sys] = rel;
  if (s.outer_active) atomicAdd(count, 1);
  atomicMax(maxrel, (unsigned long long)__double_as_longlong(rel == rel ? rel : 1e300));
}

// inner init: rho = (r^, r), alpha = omega = 1, threshold, active
__global__ void k_sc_inner_init(ScalarArgs a, double inner_tol2, double floor_frac) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  SysState& s = a.st[sys];
  double rr = sum_slot(a.partial, 1, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.rr = rr;
  s.rho = sum_slot(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r);
  s.alpha = s.omega = make_double2(1.0, 0.0);
  s.beta = make_double2(0.0, 0.0);
  s.target2 = fmax(inner_tol2 * rr, floor_frac * s.outer2);
  if (s.status == 2) s.status = 0;      // a breakdown ends one inner solve, not the outer loop
  s.active = s.outer_active && rr > s.target2;
}

// start of an iteration: |r|^2 (slot 1) against the inner target; systems
// that converged or broke down stop; the others count as running
__global__ void k_sc_check(ScalarArgs a, int* count) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  SysState& s = a.st[sys];
  if (!s.active) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  double rr = sum_slot(a.partial, 1, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  s.rr = rr;
  if (!(rr > s.target2) || s.status == 2) {   // converged (or NaN: caught by the outer check)
    s.active = 0;
    return;
  }
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

// omega = (t, s) / (t, t); rho_new = (r^, r_new) = (r^, s) - omega (r^, t) from
// fresh inner products of this iteration; beta = (rho_new / rho) (alpha / omega).
// Slots: 0 (r^, t), 1 (t, s), 2 |t|^2, 3 (r^, s).  rho_new = 0 is a breakdown:
// the iteration finishes its update and the system stops at the next check.
__global__ void k_sc_omega(ScalarArgs a) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  SysState& s = a.st[sys];
  if (!s.active) return;
  int j = sys / a.nrhs, r = sys % a.nrhs;
  const int ib0 = a.item_begin[j], ib1 = a.item_begin[j + 1];
  double2 rt = sum_slot(a.partial, 0, a.stride, ib0, ib1, a.nrhs, r);
  double2 ts = sum_slot(a.partial, 1, a.stride, ib0, ib1, a.nrhs, r);
  double tt = sum_slot(a.partial, 2, a.stride, ib0, ib1, a.nrhs, r).x;
  double2 rs = sum_slot(a.partial, 3, a.stride, ib0, ib1, a.nrhs, r);
  s.omega = tt > 0.0 ? make_double2(ts.x / tt, ts.y / tt) : make_double2(0.0, 0.0);
  const double2 rho_new = make_double2(rs.x - (s.omega.x * rt.x - s.omega.y * rt.y),
                                       rs.y - (s.omega.x * rt.y + s.omega.y * rt.x));
  const bool rho0 = s.rho.x == 0.0 && s.rho.y == 0.0;
  if ((rho_new.x == 0.0 && rho_new.y == 0.0) || (s.omega.x == 0.0 && s.omega.y == 0.0) || rho0) {
    s.beta = make_double2(0.0, 0.0);
    if ((rho_new.x == 0.0 && rho_new.y == 0.0) || rho0) s.status = 2;
  } else {
    s.beta = zmul(zdiv(rho_new, s.rho), zdiv(s.alpha, s.omega));
  }
  s.rho = rho_new;
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

// condition of the device-side inner loop (DD_SOLVE_GRAPH_LOOP): one more
// iteration while some system runs and the cap is not reached
__global__ void k_loop_cond(const int* count, int* iter, int maxiter, cudaGraphConditionalHandle h) {
  const int it = *iter + 1;
  *iter = it;
  cudaGraphSetConditional(h, (*count > 0 && it < maxiter) ? 1u : 0u);
}

// The launches of the inner BiCGstab on one batch (van der Vorst 1992), shared
// by the host-driven loop and the captured graphs.
// Device-side state of the outer defect-correction loop of the whole-solve graph
struct OuterState {
  int cyc;         // correction cycles run
  int last_true;   // the current residual is a true one (b - D x)
  int tr;          // this cycle ends with a true residual
  int osteps;      // outer-loop passes (bounded)
  int iters;       // inner iterations started, all cycles
  int n_verify;    // verification passes
  int n_tr;        // cycles that ended with a true residual
  int pad;
};

__global__ void k_outer_init(OuterState* o) {
  o->cyc = 0;
  o->last_true = 1;
  o->tr = 1;
  o->osteps = 0;
  o->iters = 0;
  o->n_verify = 0;
  o->n_tr = 0;
}

// After the outer check (k_sc_outer): verify (all stopped on an updated
// residual), run a cycle (systems left and cycles left), or stop; the loop
// also stops after max_outer + 3 passes whatever the flags say.
__global__ void k_outer_decide(OuterState* o, const int* count, const unsigned long long* maxrel_bits,
                               int max_outer, int f32, double theta, double inner_tol, double tol,
                               cudaGraphConditionalHandle h_verify, cudaGraphConditionalHandle h_cycle,
                               cudaGraphConditionalHandle h_outer) {
  const int n = count[0];
  const double maxrel = __longlong_as_double((long long)maxrel_bits[0]);
  const int verify = (n == 0 && !o->last_true) ? 1 : 0;
  const int cycle = (n > 0 && o->cyc < max_outer) ? 1 : 0;
  o->tr = (!f32 || o->cyc == 0 || maxrel > theta || inner_tol * maxrel <= 0.25 * tol) ? 1 : 0;
  o->osteps += 1;
  cudaGraphSetConditional(h_verify, verify);
  cudaGraphSetConditional(h_cycle, cycle);
  cudaGraphSetConditional(h_outer, ((verify || cycle) && o->osteps < max_outer + 3) ? 1u : 0u);
}

__global__ void k_outer_verified(OuterState* o) {
  o->last_true = 1;
  o->n_verify += 1;
}

__global__ void k_outer_cycle_end(OuterState* o, const int* d_iter) {
  o->last_true = o->tr;
  o->n_tr += o->tr;
  o->cyc += 1;
  o->iters += *d_iter;
}

__global__ void k_cond_set(const int* flag, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, (!flag || *flag) ? 1u : 0u);
}

template <class S>
struct BicgOps {
  dd_ctx* c;
  const Batch& b;
  dd_prec prec;
  InnerVecs w;
  SysState* st;
  double* partial;
  BatchDev bd;
  int nsys;
  ScalarArgs sa;
  int sth = 128, sbl;
  dim3 eg;
  double k2;
  // seed of the generated shadow vector r^ (any nonzero constant)
  static constexpr unsigned rseed = 0x2211u;
  const int* act;
  int act_stride;
  BicgOps(dd_ctx* cc, const Batch& bb, dd_prec pp, const InnerVecs& ww, SysState* ss, double* part)
      : c(cc), b(bb), prec(pp), w(ww), st(ss), partial(part), bd(batch_view(cc, bb)), nsys(bb.nb * bb.nrhs),
        sa{ss, part, bb.d_item_begin[0], (long long)bb.nitems[0] * bb.nrhs, bb.nb * bb.nrhs, bb.nrhs},
        sbl((bb.nb * bb.nrhs + 127) / 128), eg(bb.nitems[0], bb.nrhs), k2(cc->kappa * cc->kappa),
        act((const int*)((const char*)ss + offsetof(SysState, active))),
        act_stride((int)(sizeof(SysState) / sizeof(int))) {}
  // r = p = rhs, x = 0, rho = (r^, r), the per-system inner targets
  dd_status init(const void* rhs, double inner_tol2, double floor_frac, cudaStream_t s) {
    DD_COUNT_LAUNCH(), k_inner_init<S><<<eg, 128, 0, s>>>(bd, (const S*)rhs, (S*)w.r, (S*)w.p, (S*)w.x, rseed,
                                                          partial);
    DD_COUNT_LAUNCH(), k_sc_inner_init<<<sbl, sth, 0, s>>>(sa, inner_tol2, floor_frac);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  }
  // one BiCGstab iteration for every active system, enqueued on stream s
  // (captured into a graph when s is capturing).  p enters the iteration
  // already updated (by the previous k_xrp_update, or p = r at the start), so
  // an iteration is: check, v = M p with (r^, v), alpha, s, t = M s with
  // (r^, t), (t, s), |t|^2, (r^, s), omega and beta, and the fused x, r, p update.
  dd_status iteration(int* d_count, bool check, cudaStream_t s) {
    if (check) DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
    DD_COUNT_LAUNCH(), k_sc_check<<<sbl, sth, 0, s>>>(sa, check ? d_count : nullptr);
    // v = M p = p - k^2 H_eo H_oe p ; partial (rhat, v)
    HopArgs h1{};
    h1.p_out = 1; h1.in = w.p; h1.out = w.tmp; h1.b = 1.0;
    h1.active = act; h1.active_stride = act_stride;
    dd_status e = launch_hop(c, b, prec, h1, s);
    if (e != DD_OK) return e;
    HopArgs h2{};
    h2.p_out = 0; h2.in = w.tmp; h2.out = w.v; h2.s1 = w.p; h2.a1 = 1.0; h2.b = -k2;
    h2.dotq = w.rhat; h2.rhat_seed = rseed; h2.partial = partial;
    h2.active = act; h2.active_stride = act_stride;
    if ((e = launch_hop(c, b, prec, h2, s)) != DD_OK) return e;
    DD_COUNT_LAUNCH(), k_sc_alpha<<<sbl, sth, 0, s>>>(sa);
    DD_COUNT_LAUNCH(), k_s_update<S><<<eg, 128, 0, s>>>(bd, st, (const S*)w.r, (const S*)w.v, (S*)w.s);
    HopArgs h3{};
    h3.p_out = 1; h3.in = w.s; h3.out = w.tmp; h3.b = 1.0;
    h3.active = act; h3.active_stride = act_stride;
    if ((e = launch_hop(c, b, prec, h3, s)) != DD_OK) return e;
    HopArgs h4{};
    h4.p_out = 0; h4.in = w.tmp; h4.out = w.t; h4.s1 = w.s; h4.a1 = 1.0; h4.b = -k2;
    h4.dots = w.s; h4.dotq = w.rhat; h4.dotqs = true; h4.rhat_seed = rseed; h4.partial = partial;
    h4.active = act; h4.active_stride = act_stride;
    if ((e = launch_hop(c, b, prec, h4, s)) != DD_OK) return e;
    DD_COUNT_LAUNCH(), k_sc_omega<<<sbl, sth, 0, s>>>(sa);
    DD_COUNT_LAUNCH(), k_xrp_update<S><<<eg, 128, 0, s>>>(bd, st, (S*)w.x, (S*)w.r, (S*)w.p, (const S*)w.s,
                                                          (const S*)w.t, (const S*)w.v, partial);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  }
  // marks the systems that converged in the last iteration
  void final_check(cudaStream_t s) { DD_COUNT_LAUNCH(), k_sc_check<<<sbl, sth, 0, s>>>(sa, nullptr); }
};

template <class S>
dd_status run_bicgstab(dd_ctx* c, const Batch& b, dd_prec prec, const InnerVecs& w, SysState* st,
                       double* partial, int* d_count, int* h_count, const void* rhs,
                       double inner_tol2, double floor_frac, int maxiter, int check_every,
                       bool use_graph, cudaStream_t s, int* iters_run, bool device_loop = false) {
  BicgOps<S> ops(c, b, prec, w, st, partial);
  dd_status e0 = ops.init(rhs, inner_tol2, floor_frac, s);
  if (e0 != DD_OK) return e0;
  auto iteration = [&](bool check, cudaStream_t s) -> dd_status { return ops.iteration(d_count, check, s); };
  auto poll = [&]() -> dd_status {
    DD_CUDA(c, cudaMemcpyAsync(h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    return DD_OK;
  };
  int it = 0;
  bool done = false;
  if (device_loop) {
    // the whole inner solve as one graph: a memset node zeroes the iteration
    // counter, then a conditional WHILE node repeats {iteration, condition}
    // until no system runs or maxiter iterations have started
    int* d_iter = d_count + 1;
    char key[256];
    // (the instance table's address is part of the key: a reallocation of it
    // must not leave a replay reading the old one)
    snprintf(key, sizeof key, "loop:%d:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%d:%a:%d%d%d:%p", (int)prec, w.r, w.rhat,
             w.p, w.v, w.s, w.t, w.x, w.tmp, (void*)st, (void*)partial, (void*)d_count, maxiter, c->kappa,
             b.hop_variant[0], b.hop_variant[1], b.hop_variant[2], (void*)c->d_inst);
    cudaGraphExec_t exec = nullptr;
    for (auto& g : b.graphs)
      if (g.first == key) exec = g.second;
    if (!exec) {
      if (!c->capture_stream)
        DD_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
      cudaStream_t cs = c->capture_stream;
      cudaGraph_t graph = nullptr;
      DD_CUDA(c, cudaGraphCreate(&graph, 0));
      struct GraphGuard {
        cudaGraph_t g;
        ~GraphGuard() { if (g) cudaGraphDestroy(g); }
      } guard{graph};
      cudaMemsetParams mp{};
      mp.dst = d_iter;
      mp.value = 0;
      mp.elementSize = sizeof(int);
      mp.width = 1;
      mp.height = 1;
      cudaGraphNode_t n0 = nullptr, n1 = nullptr;
      DD_CUDA(c, cudaGraphAddMemsetNode(&n0, graph, nullptr, 0, &mp));
      cudaGraphConditionalHandle h;
      DD_CUDA(c, cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      DD_CUDA(c, cudaGraphAddNode(&n1, graph, &n0, nullptr, 1, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      DD_CUDA(c, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      const long long l0 = g_launches.load();
      dd_status e = iteration(true, cs);
      if (e == DD_OK) DD_COUNT_LAUNCH(), k_loop_cond<<<1, 1, 0, cs>>>(d_count, d_iter, maxiter, h);
      // captured launches are not executions: the replays count them
      const long long nk = g_launches.load() - l0;
      g_launches.fetch_sub(nk);
      b.graph_kernels[key] = nk;
      cudaGraph_t body_out = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cs, &body_out);
      if (e != DD_OK) return e;
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture (inner loop body)");
      ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaGraphInstantiate (inner loop)");
      if (b.graphs.size() >= 8) {
        cudaGraphExecDestroy(b.graphs.front().second);
        b.graphs.erase(b.graphs.begin());
      }
      b.graphs.push_back({std::string(key), exec});
    }
    DD_CUDA(c, cudaGraphLaunch(exec, s));
    int hv[2] = {0, 0};
    DD_CUDA(c, cudaMemcpyAsync(hv, d_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    *h_count = hv[0];
    it = hv[1];
    g_launches.fetch_add(b.graph_kernels[key] * it);
    done = true;
  }
  if (!done && use_graph && check_every <= maxiter) {
    // the check_every iterations between two polls, captured once per batch,
    // precision, buffers and launch variant, then replayed
    char key[256];
    snprintf(key, sizeof key, "%d:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%d:%a:%d%d%d:%p", (int)prec, w.r,
             w.rhat, w.p, w.v, w.s, w.t, w.x, w.tmp, (void*)st, (void*)partial, (void*)d_count,
             check_every, c->kappa, b.hop_variant[0], b.hop_variant[1], b.hop_variant[2], (void*)c->d_inst);
    cudaGraphExec_t exec = nullptr;
    for (auto& g : b.graphs)
      if (g.first == key) exec = g.second;
    if (!exec) {
      // captured on the context's own stream (the caller's may be the legacy
      // default stream, which cannot be captured), replayed on the caller's
      if (!c->capture_stream)
        DD_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
      cudaStream_t cs = c->capture_stream;
      DD_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      const long long l0 = g_launches.load();
      dd_status e = DD_OK;
      for (int i = 0; i < check_every && e == DD_OK; ++i) e = iteration(i == check_every - 1, cs);
      const long long nk = g_launches.load() - l0;
      g_launches.fetch_sub(nk);
      b.graph_kernels[key] = nk;
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      if (e != DD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return e;
      }
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaGraphInstantiate");
      if (b.graphs.size() >= 8) {
        cudaGraphExecDestroy(b.graphs.front().second);
        b.graphs.erase(b.graphs.begin());
      }
      b.graphs.push_back({std::string(key), exec});
    }
    const long long nk = b.graph_kernels[key];
    while (it + check_every <= maxiter) {
      DD_CUDA(c, cudaGraphLaunch(exec, s));
      g_launches.fetch_add(nk);
      it += check_every;
      dd_status e = poll();
      if (e != DD_OK) return e;
      if (*h_count == 0) {
        done = true;
        break;
      }
    }
  }
  for (; !done && it < maxiter; ++it) {
    bool check = ((it + 1) % check_every) == 0;
    dd_status e = iteration(check, s);
    if (e != DD_OK) return e;
    if (check) {
      if ((e = poll()) != DD_OK) return e;
      if (*h_count == 0) {
        ++it;
        break;
      }
    }
  }
  // a final check marks the systems that converged in the last iteration
  ops.final_check(s);
  *iters_run = it;
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// Measures every compiled variant of the hop launch on this batch (the
// H_oe half-apply of an initialised even vector `in` into `out`) and keeps
// the fastest for the precision.
dd_status tune_hop(dd_ctx* c, const Batch& b, dd_prec prec, const void* in, void* out,
                   cudaStream_t s) {
  const int pi = prec == DD_F64 ? 0 : (prec == DD_F32 ? 1 : 2);
  const bool timing = c->timing;
  c->timing = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_v = 0;
  dd_status st = DD_OK;
  // per variant: two warm-up launches, then the best of three rounds of three
  // (single short timings let near-equal variants trade places by noise)
  for (int v = 0; v < hop_variant_count(prec) && st == DD_OK; ++v) {
    b.hop_variant[pi] = v;
    HopArgs h{};
    h.p_out = 1; h.in = in; h.out = out; h.b = 1.0;
    for (int k = 0; k < 2 && st == DD_OK; ++k) st = launch_hop(c, b, prec, h, s);
    float vbest = 1e30f;
    for (int round = 0; round < 3 && st == DD_OK; ++round) {
      cudaEventRecord(e0, s);
      for (int k = 0; k < 3 && st == DD_OK; ++k) st = launch_hop(c, b, prec, h, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      vbest = std::min(vbest, ms);
    }
    if (st == DD_OK && vbest < best) {
      best = vbest;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = timing;
  b.hop_variant[pi] = best_v;
  b.tuned[pi] = true;
  return st;
}

// outer-vector launches: the outer vectors are FP64 (plain FP64 solve) or
// double-float (mixed solve); `sp` is the precision of the added vector
template <class O>
void axpy_outer_t(const BatchDev& bd, dim3 g, int p, void* x, const void* v, dd_prec sp, double sign,
                  const SysState* st, double* partial, cudaStream_t s) {
  if (sp == DD_F64)
    DD_COUNT_LAUNCH(), k_axpy64<O, double2><<<g, 128, 0, s>>>(bd, p, (O*)x, (const double2*)v, sign, st, partial);
  else if (sp == DD_F32)
    DD_COUNT_LAUNCH(), k_axpy64<O, float2><<<g, 128, 0, s>>>(bd, p, (O*)x, (const float2*)v, sign, st, partial);
  else
    DD_COUNT_LAUNCH(), k_axpy64<O, __nv_bfloat162><<<g, 128, 0, s>>>(bd, p, (O*)x, (const __nv_bfloat162*)v, sign,
                                                                     st, partial);
}
// x += sign v on parity p; with partial, also |x|^2 per (item, rhs) into slot 0
void axpy_outer(bool dfo, const BatchDev& bd, dim3 g, int p, void* x, const void* v, dd_prec sp,
                double sign, const SysState* st, cudaStream_t s, double* partial = nullptr) {
  if (dfo) axpy_outer_t<df2s>(bd, g, p, x, v, sp, sign, st, partial, s);
  else axpy_outer_t<double2>(bd, g, p, x, v, sp, sign, st, partial, s);
}
void norm2_outer(bool dfo, const BatchDev& bd, dim3 g, int p, const void* v, double* partial,
                 cudaStream_t s) {
  if (dfo) DD_COUNT_LAUNCH(), k_norm2<df2s><<<g, 128, 0, s>>>(bd, p, (const df2s*)v, partial, 0);
  else DD_COUNT_LAUNCH(), k_norm2<double2><<<g, 128, 0, s>>>(bd, p, (const double2*)v, partial, 0);
}
// outer residual -> inner precision ip (F32 or BF16)
void convert_outer(bool dfo, dd_prec ip, const BatchDev& bd, dim3 g, int p, void* y, const void* x,
                   const SysState* st, cudaStream_t s) {
  if (ip == DD_F32) {
    if (dfo) DD_COUNT_LAUNCH(), k_convert<float2, df2s><<<g, 128, 0, s>>>(bd, p, (float2*)y, (const df2s*)x, st);
    else DD_COUNT_LAUNCH(), k_convert<float2, double2><<<g, 128, 0, s>>>(bd, p, (float2*)y, (const double2*)x, st);
  } else {
    if (dfo) DD_COUNT_LAUNCH(), k_convert<__nv_bfloat162, df2s><<<g, 128, 0, s>>>(bd, p, (__nv_bfloat162*)y, (const df2s*)x, st);
    else DD_COUNT_LAUNCH(), k_convert<__nv_bfloat162, double2><<<g, 128, 0, s>>>(bd, p, (__nv_bfloat162*)y, (const double2*)x, st);
  }
}

// r = b - D x at the outer precision (both parities); the double-float
// residual also writes the |r|^2 partials of the next outer check
dd_status true_residual_pass(dd_ctx* c, const Batch& b, dd_prec op, bool dfo, const void* xe, const void* xo,
                             const void* be, const void* bo, void* re, void* ro, double* partial,
                             double* partial_o, cudaStream_t s) {
  const double kap = c->kappa;
  HopArgs h{};
  h.p_out = 0; h.in = xo; h.out = re; h.s1 = be; h.a1 = 1.0; h.s2 = xe; h.a2 = -1.0; h.b = kap;
  HopArgs g{};
  g.p_out = 1; g.in = xe; g.out = ro; g.s1 = bo; g.a1 = 1.0; g.s2 = xo; g.a2 = -1.0; g.b = kap;
  if (dfo) {
    h.norm_out = g.norm_out = true;
    h.partial = partial;
    g.partial = partial_o;
  }
  dd_status e;
  if ((e = launch_hop(c, b, op, h, s)) != DD_OK) return e;
  return launch_hop(c, b, op, g, s);
}

// Sequential construction of a CUDA graph from captured segments and
// conditional nodes: each segment is captured onto the current leaves, each
// conditional node depends on them and becomes the only leaf.
struct GraphSeq {
  dd_ctx* c;
  cudaGraph_t g;
  cudaStream_t cs;
  std::vector<cudaGraphNode_t> deps;
  long long kernels = 0;   // kernel launches captured by the last segment
  dd_status capture(const std::function<dd_status(cudaStream_t)>& fn) {
    DD_CUDA(c, cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                             cudaStreamCaptureModeThreadLocal));
    const long long l0 = g_launches.load();
    dd_status e = fn(cs);
    // captured launches are not executions: the replays count them
    kernels = g_launches.load() - l0;
    g_launches.fetch_sub(kernels);
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t ci = cudaStreamGetCaptureInfo(cs, &stt, nullptr, nullptr, &d, nullptr, &nd);
    std::vector<cudaGraphNode_t> leaves(d, d + (ci == cudaSuccess ? nd : 0));
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &out);
    if (e != DD_OK) return e;
    if (ci != cudaSuccess) return cuda_fail(c, ci, "cudaStreamGetCaptureInfo");
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture (solve graph)");
    deps = leaves;
    return DD_OK;
  }
  dd_status cond(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned size,
                 cudaGraph_t* bodies) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = size;
    cudaGraphNode_t n = nullptr;
    DD_CUDA(c, cudaGraphAddNode(&n, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
    for (unsigned k = 0; k < size; ++k) bodies[k] = cp.conditional.phGraph_out[k];
    deps.assign(1, n);
    return DD_OK;
  }
};

// The whole mixed-precision solve after the right-hand side is packed, as one
// graph launch:
//   OuterState init; WHILE (outer) {
//     outer check (k_sc_outer) and decision (k_outer_decide);
//     IF (verify) { r = b - D x };
//     IF (cycle)  { residual to the inner precision; Schur right-hand side;
//                   inner BiCGstab: init, WHILE (inner) { iteration }, final check;
//                   x += e; IF (true residual) { r = b - D x } ELSE { r -= D e };
//                   cycle bookkeeping } }
// Every decision of the host-driven loop is taken by a one-thread kernel from
// the same device-side counts; the outer loop is capped at max_outer + 3
// passes and the inner one at maxiter iterations.
template <class S>
dd_status whole_solve(dd_ctx* c, const Batch& b, dd_prec ip, const InnerVecs& w, SysState* st, double* partial,
                      double* partial_o, int* d_count, unsigned long long* d_maxrel, double* vrel, const void* rhs,
                      double inner_tol2, double floor_frac, double theta, const dd_solve_params* prm,
                      int max_outer, const std::function<dd_status(cudaStream_t)>& to_inner,
                      const std::function<dd_status(cudaStream_t)>& schur_rhs,
                      const std::function<dd_status(cudaStream_t)>& correct_x,
                      const std::function<dd_status(cudaStream_t)>& true_res,
                      const std::function<dd_status(cudaStream_t)>& update_res, const std::string& keyx,
                      cudaStream_t s, int* cycles_out) {
  dd_status e;
  void* vos;
  if ((e = ws_get(c, 39, sizeof(OuterState), &vos)) != DD_OK) return e;
  OuterState* os = (OuterState*)vos;
  int* d_iter = d_count + 1;
  const int nsys = b.nb * b.nrhs;
  const long long stride = (long long)b.nitems[0] * b.nrhs;
  const long long stride_o = (long long)b.nitems[1] * b.nrhs;
  ScalarArgs sa{st, partial, b.d_item_begin[0], stride, nsys, b.nrhs};
  const int sth = 128, sbl = (nsys + sth - 1) / sth;
  BicgOps<S> ops(c, b, ip, w, st, partial);
  char kb[512];
  snprintf(kb, sizeof kb,
           "solve:%d:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p:%a:%a:%a:%a:%d:%d:%d%d%d:%d:%p:%p:%p:%p",
           (int)ip, w.r, w.rhat, w.p, w.v, w.s, w.t, w.x, w.tmp, (void*)st, (void*)partial, (void*)partial_o,
           (void*)d_count, (void*)vrel, rhs, c->kappa, prm->tol, prm->inner_tol, floor_frac, max_outer,
           prm->maxiter, b.hop_variant[0], b.hop_variant[1], b.hop_variant[2], c->clover_active ? 1 : 0,
           (void*)c->d_clovi32, (void*)c->d_clovi_df, (void*)c->d_inst, vos);
  const std::string key = std::string(kb) + keyx;
  // kernels per pass of each part (for the launch count), kept with the batch's
  // graphs under the graph's key and a suffix per part
  struct Counts {
    long long init, check, verify, pre, inner, post, tres, upd, end;
  };
  static const char* const parts[9] = {":init", ":check", ":verify", ":pre", ":inner", ":post", ":tres", ":upd",
                                       ":end"};
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b.graphs)
    if (g.first == key) exec = g.second;
  if (!exec) {
    if (!c->capture_stream) DD_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    DD_CUDA(c, cudaGraphCreate(&graph, 0));
    struct GraphGuard {
      cudaGraph_t g;
      ~GraphGuard() { if (g) cudaGraphDestroy(g); }
    } guard{graph};
    Counts n{};
    const int f32 = ip == DD_F32 ? 1 : 0;
    GraphSeq top{c, graph, c->capture_stream, {}};
    cudaGraphConditionalHandle h_outer;
    DD_CUDA(c, cudaGraphConditionalHandleCreate(&h_outer, graph, 1, cudaGraphCondAssignDefault));
    if ((e = top.capture([&](cudaStream_t q) {
           DD_COUNT_LAUNCH(), k_outer_init<<<1, 1, 0, q>>>(os);
           return DD_OK;
         })) != DD_OK)
      return e;
    n.init = top.kernels;
    cudaGraph_t body_outer;
    if ((e = top.cond(h_outer, cudaGraphCondTypeWhile, 1, &body_outer)) != DD_OK) return e;
    GraphSeq ob{c, body_outer, c->capture_stream, {}};
    cudaGraphConditionalHandle h_verify, h_cycle;
    DD_CUDA(c, cudaGraphConditionalHandleCreate(&h_verify, body_outer, 0, 0));
    DD_CUDA(c, cudaGraphConditionalHandleCreate(&h_cycle, body_outer, 0, 0));
    if ((e = ob.capture([&](cudaStream_t q) {
           DD_CUDA(c, cudaMemsetAsync(d_count, 0, 64, q));
           DD_COUNT_LAUNCH(), k_sc_outer<<<sbl, sth, 0, q>>>(sa, partial_o, b.d_item_begin[1], stride_o, 1.0,
                                                            d_count, d_maxrel, vrel, &os->last_true);
           DD_COUNT_LAUNCH(), k_outer_decide<<<1, 1, 0, q>>>(os, d_count, d_maxrel, max_outer, f32, theta,
                                                            prm->inner_tol, prm->tol, h_verify, h_cycle, h_outer);
           DD_CUDA(c, cudaGetLastError());
           return DD_OK;
         })) != DD_OK)
      return e;
    n.check = ob.kernels;
    cudaGraph_t body_verify;
    if ((e = ob.cond(h_verify, cudaGraphCondTypeIf, 1, &body_verify)) != DD_OK) return e;
    GraphSeq vb{c, body_verify, c->capture_stream, {}};
    if ((e = vb.capture([&](cudaStream_t q) {
           dd_status r = true_res(q);
           DD_COUNT_LAUNCH(), k_outer_verified<<<1, 1, 0, q>>>(os);
           return r;
         })) != DD_OK)
      return e;
    n.verify = vb.kernels;
    cudaGraph_t body_cycle;
    if ((e = ob.cond(h_cycle, cudaGraphCondTypeIf, 1, &body_cycle)) != DD_OK) return e;
    GraphSeq cb{c, body_cycle, c->capture_stream, {}};
    cudaGraphConditionalHandle h_inner, h_true;
    DD_CUDA(c, cudaGraphConditionalHandleCreate(&h_inner, body_cycle, 1, 0));
    DD_CUDA(c, cudaGraphConditionalHandleCreate(&h_true, body_cycle, 1, 0));
    if ((e = cb.capture([&](cudaStream_t q) {
           dd_status r;
           if ((r = to_inner(q)) != DD_OK || (r = schur_rhs(q)) != DD_OK ||
               (r = ops.init(rhs, inner_tol2, floor_frac, q)) != DD_OK)
             return r;
           DD_CUDA(c, cudaMemsetAsync(d_iter, 0, sizeof(int), q));
           // the inner loop's condition starts at 1 on every pass of the outer loop
           DD_COUNT_LAUNCH(), k_cond_set<<<1, 1, 0, q>>>(nullptr, h_inner);
           DD_CUDA(c, cudaGetLastError());
           return DD_OK;
         })) != DD_OK)
      return e;
    n.pre = cb.kernels;
    cudaGraph_t body_inner;
    if ((e = cb.cond(h_inner, cudaGraphCondTypeWhile, 1, &body_inner)) != DD_OK) return e;
    GraphSeq ib{c, body_inner, c->capture_stream, {}};
    if ((e = ib.capture([&](cudaStream_t q) {
           dd_status r = ops.iteration(d_count, true, q);
           if (r != DD_OK) return r;
           DD_COUNT_LAUNCH(), k_loop_cond<<<1, 1, 0, q>>>(d_count, d_iter, prm->maxiter, h_inner);
           DD_CUDA(c, cudaGetLastError());
           return DD_OK;
         })) != DD_OK)
      return e;
    n.inner = ib.kernels;
    if ((e = cb.capture([&](cudaStream_t q) {
           ops.final_check(q);
           dd_status r = correct_x(q);
           DD_COUNT_LAUNCH(), k_cond_set<<<1, 1, 0, q>>>(&os->tr, h_true);
           DD_CUDA(c, cudaGetLastError());
           return r;
         })) != DD_OK)
      return e;
    n.post = cb.kernels;
    cudaGraph_t body_tr[2];
    if ((e = cb.cond(h_true, cudaGraphCondTypeIf, 2, body_tr)) != DD_OK) return e;
    GraphSeq tb{c, body_tr[0], c->capture_stream, {}};
    if ((e = tb.capture(true_res)) != DD_OK) return e;
    n.tres = tb.kernels;
    GraphSeq ub{c, body_tr[1], c->capture_stream, {}};
    if ((e = ub.capture(update_res)) != DD_OK) return e;
    n.upd = ub.kernels;
    if ((e = cb.capture([&](cudaStream_t q) {
           DD_COUNT_LAUNCH(), k_outer_cycle_end<<<1, 1, 0, q>>>(os, d_iter);
           DD_CUDA(c, cudaGetLastError());
           return DD_OK;
         })) != DD_OK)
      return e;
    n.end = cb.kernels;
    cudaError_t ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaGraphInstantiate (solve graph)");
    if (b.graphs.size() >= 8) {
      cudaGraphExecDestroy(b.graphs.front().second);
      b.graphs.erase(b.graphs.begin());
    }
    b.graphs.push_back({key, exec});
    const long long nv[9] = {n.init, n.check, n.verify, n.pre, n.inner, n.post, n.tres, n.upd, n.end};
    for (int k = 0; k < 9; ++k) b.graph_kernels[key + parts[k]] = nv[k];
  }
  DD_CUDA(c, cudaGraphLaunch(exec, s));
  OuterState ho{};
  DD_CUDA(c, cudaMemcpyAsync(&ho, os, sizeof ho, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  long long nv[9];
  for (int k = 0; k < 9; ++k) nv[k] = b.graph_kernels[key + parts[k]];
  const Counts n{nv[0], nv[1], nv[2], nv[3], nv[4], nv[5], nv[6], nv[7], nv[8]};
  g_launches.fetch_add(n.init + n.check * ho.osteps + n.verify * ho.n_verify + (n.pre + n.post + n.end) * ho.cyc +
                       n.inner * ho.iters + n.tres * ho.n_tr + n.upd * (ho.cyc - ho.n_tr));
  *cycles_out = ho.cyc;
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
  // clover term: left preconditioning by A^{-1} (clover.cu); every hop of the
  // solve applies A^{-1} of its output site, at the hop's own precision
  const bool clov = c->csw != 0.0;
  if (clov) {
    if (prm->flags & (DD_SOLVE_NET_GUESS | DD_SOLVE_NET_PRECOND))
      return fail(c, DD_EINVAL, "the learned network does not include the clover term");
    if (!c->clover_ready && (e = clover_build(c)) != DD_OK) return e;
    if (ip != DD_F64 && (e = clover_mixed_tables(c)) != DD_OK) return e;
  }
  // The solve stops on the preconditioned residual A^{-1}(b - D x) relative to
  // A^{-1} b; running it to tol / c_A with c_A >= |A| |A^{-1}| keeps the true
  // residual |b - D x| <= tol |b|.
  dd_solve_params prm_clov;
  if (clov) {
    prm_clov = *prm;
    prm_clov.tol = prm->tol / c->clover_cond;
    prm = &prm_clov;
  }
  struct ActiveGuard {
    dd_ctx* c;
    ActiveGuard(dd_ctx* cc, bool on) : c(cc) { c->clover_active = on; }
    ~ActiveGuard() { c->clover_active = false; }
  } guard(c, clov);
  const long long ne = b.tot[0], no = b.tot[1];
  // Outer vectors b, x, r (both parities), 16 bytes per complex number: FP64
  // for the plain FP64 solve; double-float for the mixed solves, whose true
  // residual r = b - D x then runs on the FP32 pipes (GB300 issues FP64 at a
  // small fraction of its FP32 rate) with about 44 significant bits.
  const bool dfo = ip != DD_F64;
  const dd_prec op = dfo ? DD_DF64 : DD_F64;
  void *be, *bo, *xe, *xo, *re, *ro;
  if ((e = ws_get(c, 0, ne * c64, &be)) || (e = ws_get(c, 1, no * c64, &bo)) ||
      (e = ws_get(c, 2, ne * c64, &xe)) || (e = ws_get(c, 3, no * c64, &xo)) ||
      (e = ws_get(c, 4, ne * c64, &re)) || (e = ws_get(c, 5, no * c64, &ro)))
    return e;
  // inner vectors at the inner precision
  InnerVecs w;
  void *rso, *rhs, *eo;
  if ((e = ws_get(c, 7, ne * cin, &w.r)) || (e = ws_get(c, 8, ne * cin, &w.rhat)) ||
      (e = ws_get(c, 9, ne * cin, &w.p)) || (e = ws_get(c, 10, ne * cin, &w.v)) ||
      (e = ws_get(c, 11, ne * cin, &w.s)) || (e = ws_get(c, 12, ne * cin, &w.t)) ||
      (e = ws_get(c, 13, ne * cin, &w.x)) || (e = ws_get(c, 14, no * cin, &w.tmp)) ||
      (e = ws_get(c, 24, no * cin, &rso)) || (e = ws_get(c, 25, ne * cin, &rhs)) ||
      (e = ws_get(c, 26, no * cin, &eo)))
    return e;
  void *vpart, *vst, *vcnt, *vrel, *vpart_o;
  const long long stride = (long long)b.nitems[0] * b.nrhs;
  const long long stride_o = (long long)b.nitems[1] * b.nrhs;
  if ((e = ws_get(c, 15, sizeof(double) * 2 * 4 * std::max<long long>(1, stride), &vpart)) ||
      (e = ws_get(c, 16, sizeof(SysState) * nsys, &vst)) || (e = ws_get(c, 17, 64, &vcnt)) ||
      (e = ws_get(c, 18, sizeof(double) * nsys, &vrel)) ||
      (e = ws_get(c, 19, sizeof(double) * 2 * std::max<long long>(1, stride_o), &vpart_o)))
    return e;
  double* partial = (double*)vpart;
  double* partial_o = (double*)vpart_o;
  SysState* st = (SysState*)vst;
  int* d_count = (int*)vcnt;
  unsigned long long* d_maxrel = (unsigned long long*)((char*)vcnt + 16);
  for (int j = 0; j < b.nb; ++j) {
    if ((e = ensure_links(c, b.inst[j], op)) != DD_OK) return e;
    if (ip != DD_F64 && (e = ensure_links(c, b.inst[j], ip)) != DD_OK) return e;
  }
  if ((e = sync_instances(c)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  ScalarArgs sa{st, partial, b.d_item_begin[0], stride, nsys, b.nrhs};
  const int sth = 128, sbl = (nsys + sth - 1) / sth;
  dim3 eg(b.nitems[0], b.nrhs), og(b.nitems[1], b.nrhs);
  const double kap = c->kappa;
  const bool has_odd = b.nitems[1] > 0;

  EventPair evs;
  cudaEvent_t ev0 = evs.a, ev1 = evs.b;
  cudaEventRecord(ev0, s);

  // b, r = b and x = 0 in one pass over the caller layout; |b|^2 (= |r|^2)
  // partials by a coalesced pass over the parity vectors
  if ((e = launch_pack_init(c, b, b_user, be, bo, re, ro, xe, xo, op, s)) != DD_OK) return e;
  if (clov) {
    // solve (1 - kappa A^{-1} H) x = A^{-1} b: b and r = b preconditioned once
    // (in FP64 arithmetic also for the double-float vectors of the mixed forms)
    if ((e = dfo ? clover_apply_inv_df(c, b, be, bo, s) : clover_apply(c, b, be, bo, true, s)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(re, be, ne * c64, cudaMemcpyDeviceToDevice, s));
    if (no > 0) DD_CUDA(c, cudaMemcpyAsync(ro, bo, no * c64, cudaMemcpyDeviceToDevice, s));
  }
  norm2_outer(dfo, bd, eg, 0, be, partial, s);
  if (has_odd) norm2_outer(dfo, bd, og, 1, bo, partial_o, s);
  DD_COUNT_LAUNCH(), k_sc_bnorm<<<sbl, sth, 0, s>>>(sa, partial_o, b.d_item_begin[1], stride_o, prm->tol * prm->tol);
  // the |r|^2 partials of the next outer check are already written
  bool norms_ready = true;
  // learned initial guess: x = N(b), r = b - D x with D x in FP32 (the first
  // correction cycle is followed by an FP64 residual, which absorbs its rounding)
  bool all_omega = true;
  for (int j = 0; j < b.nb; ++j)
    if (c->inst[b.inst[j]].d.kind != DD_DOMAIN_OMEGA) all_omega = false;
  if ((prm->flags & DD_SOLVE_NET_GUESS) && c->net && all_omega) {
    void *ge, *go, *te, *to;
    if ((e = ws_get(c, 28, ne * 8, &ge)) || (e = ws_get(c, 29, no * 8 + 16, &go)) ||
        (e = ws_get(c, 80, ne * 8, &te)) || (e = ws_get(c, 81, no * 8 + 16, &to)))
      return e;
    if ((e = net_guess(c, c->net, b, be, bo, dfo, (float2*)ge, (float2*)go, s)) != DD_OK) return e;
    if ((e = ensure_links(c, b.inst[0], DD_F32)) != DD_OK) return e;
    for (int j = 0; j < b.nb; ++j)
      if ((e = ensure_links(c, b.inst[j], DD_F32)) != DD_OK) return e;
    if ((e = sync_instances(c)) != DD_OK) return e;
    bd = batch_view(c, b);
    axpy_outer(dfo, bd, eg, 0, xe, ge, DD_F32, 1.0, st, s);
    if (has_odd) axpy_outer(dfo, bd, og, 1, xo, go, DD_F32, 1.0, st, s);
    HopArgs h{};
    h.p_out = 0; h.in = go; h.out = te; h.s1 = ge; h.a1 = 1.0; h.b = -kap;
    if ((e = launch_hop(c, b, DD_F32, h, s)) != DD_OK) return e;
    HopArgs g{};
    g.p_out = 1; g.in = ge; g.out = to; g.s1 = go; g.a1 = 1.0; g.b = -kap;
    if ((e = launch_hop(c, b, DD_F32, g, s)) != DD_OK) return e;
    axpy_outer(dfo, bd, eg, 0, re, te, DD_F32, -1.0, st, s, partial);
    if (has_odd) axpy_outer(dfo, bd, og, 1, ro, to, DD_F32, -1.0, st, s, partial_o);
    DD_CUDA(c, cudaGetLastError());
  }

  const int check_every = std::max(1, prm->check_every);
  const int max_outer = std::max(1, prm->max_outer);
  // CUDA graphs replay the inner iterations between polls (not while the
  // per-launch kernel timing is on: its events are host-side records)
  const bool use_graph = (prm->flags & DD_SOLVE_GRAPH) && !c->timing;
  // each inner solve as one graph launch with its loop on the device
  const bool device_loop = (prm->flags & DD_SOLVE_GRAPH_LOOP) && !c->timing;
  void* tune64 = nullptr;
  if ((prm->flags & DD_SOLVE_AUTOTUNE) &&
      (e = ws_get(c, 27, std::max(ne, no) * c64, &tune64)) != DD_OK)
    return e;
  const double inner_tol2 = ip == DD_F64 ? 0.0 : prm->inner_tol * prm->inner_tol;
  // inner solves stop at inner_tol |r| but never below (tol/2)^2 |b|^2 (plain
  // FP64) or (tol/4)^2 |b|^2 (mixed, whose last cycle must clear tol/2)
  const double floor_frac = ip == DD_F64 ? 0.25 : 0.0625;
  // The residual after a correction is recomputed in FP64 (r = b - D x) until
  // it is below theta |b|; from there on, with an FP32 inner solve, it is
  // updated as r -= D e with D e in FP32, whose rounding error
  // (~ u32 cond(D) |r|) stays far below tol |b|.  Systems then stop at tol / 2
  // to keep a margin.  BF16 links round at 2^-9, so BF16 inner solves always
  // recompute the residual in FP64.
  const double theta = prm->tol * 1e5;
  // the launches of one correction cycle, shared by the host-driven loop and
  // the whole-solve graph
  const void* rin_e = ip != DD_F64 ? w.s : re;   // residual at the inner precision
  const void* rin_o = ip != DD_F64 ? rso : ro;
  auto to_inner = [&](cudaStream_t q) -> dd_status {
    if (ip != DD_F64) {
      convert_outer(dfo, ip, bd, eg, 0, w.s, re, st, q);
      if (has_odd) convert_outer(dfo, ip, bd, og, 1, rso, ro, st, q);
    }
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  };
  // Schur right-hand side r^_e = r_e + k H_eo r_o
  auto schur_rhs = [&](cudaStream_t q) -> dd_status {
    HopArgs h{};
    h.p_out = 0; h.in = rin_o; h.out = rhs; h.s1 = rin_e; h.a1 = 1.0; h.b = kap;
    return launch_hop(c, b, ip, h, q);
  };
  // e_o = r_o + k H_oe e_e, then x += e
  auto correct_x = [&](cudaStream_t q) -> dd_status {
    HopArgs h{};
    h.p_out = 1; h.in = w.x; h.out = eo; h.s1 = rin_o; h.a1 = 1.0; h.b = kap;
    dd_status r = launch_hop(c, b, ip, h, q);
    if (r != DD_OK) return r;
    axpy_outer(dfo, bd, eg, 0, xe, w.x, ip, 1.0, st, q);
    if (has_odd) axpy_outer(dfo, bd, og, 1, xo, eo, ip, 1.0, st, q);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  };
  auto true_res = [&](cudaStream_t q) -> dd_status {
    return true_residual_pass(c, b, op, dfo, xe, xo, be, bo, re, ro, partial, partial_o, q);
  };
  // r -= D e with D e at the inner precision (and the |r|^2 partials)
  auto update_res = [&](cudaStream_t q) -> dd_status {
    HopArgs h{};
    h.p_out = 0; h.in = eo; h.out = w.t; h.s1 = w.x; h.a1 = 1.0; h.b = -kap;
    dd_status r = launch_hop(c, b, ip, h, q);
    if (r != DD_OK) return r;
    HopArgs g{};
    g.p_out = 1; g.in = w.x; g.out = w.tmp; g.s1 = eo; g.a1 = 1.0; g.b = -kap;
    if ((r = launch_hop(c, b, ip, g, q)) != DD_OK) return r;
    axpy_outer(dfo, bd, eg, 0, re, w.t, ip, -1.0, st, q, partial);
    if (has_odd) axpy_outer(dfo, bd, og, 1, ro, w.tmp, ip, -1.0, st, q, partial_o);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  };
  int cycles = 0;
  // The whole solve as one graph launch (mixed forms with BiCGstab inner
  // solves, once the launch form is tuned): the outer checks and their
  // decisions run on the device (whole_solve below).
  const int pi_in = ip == DD_F32 ? 1 : 2;
  const bool graph_solve = (prm->flags & DD_SOLVE_GRAPH_SOLVE) && !c->timing && dfo &&
                           !(prm->flags & (DD_SOLVE_FGMRES | DD_SOLVE_NET_PRECOND)) &&
                           (!(prm->flags & DD_SOLVE_AUTOTUNE) || b.tuned[pi_in]);
  if (graph_solve) {
    auto run = [&](auto tag) -> dd_status {
      using S = decltype(tag);
      char kx[256];
      snprintf(kx, sizeof kx, ":%p:%p:%p:%p:%p:%p:%p:%p", be, bo, xe, xo, re, ro, rso, eo);
      return whole_solve<S>(c, b, ip, w, st, partial, partial_o, (int*)vcnt, d_maxrel, (double*)vrel, rhs,
                            inner_tol2, floor_frac, theta, prm, max_outer, to_inner, schur_rhs, correct_x,
                            true_res, update_res, std::string(kx), s, &cycles);
    };
    if ((e = ip == DD_F32 ? run(float2{}) : run(__nv_bfloat162{})) != DD_OK) return e;
  }
  bool last_true = true;
  double maxrel = 1.0;
  for (int cyc = 0; !graph_solve; ++cyc) {
    // |r|^2 of both parities -> convergence
    if (!norms_ready) {
      norm2_outer(dfo, bd, eg, 0, re, partial, s);
      if (has_odd) norm2_outer(dfo, bd, og, 1, ro, partial_o, s);
    }
    norms_ready = false;
    DD_CUDA(c, cudaMemsetAsync(vcnt, 0, 64, s));
    DD_COUNT_LAUNCH(), k_sc_outer<<<sbl, sth, 0, s>>>(sa, partial_o, b.d_item_begin[1], stride_o,
                                                     last_true ? 1.0 : 0.25, d_count, d_maxrel,
                                                     (double*)vrel);
    int h_count = 0;
    unsigned long long h_max = 0;
    DD_CUDA(c, cudaMemcpyAsync(&h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaMemcpyAsync(&h_max, d_maxrel, sizeof(h_max), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    memcpy(&maxrel, &h_max, sizeof(double));
    // A decision to stop that rests on an updated (recursive) residual is
    // verified: r = b - D x once more at the outer precision, and the check
    // repeats on it, so the residuals a solve reports are true residuals.
    if (h_count == 0 && !last_true) {
      if ((e = true_res(s)) != DD_OK) return e;
      last_true = true;
      norms_ready = dfo;
      continue;
    }
    if (h_count == 0 || cyc >= max_outer) break;
    ++cycles;
    // the cycle whose inner target is the floor for every system (inner_tol
    // times the largest residual already below tol/4) is expected to end the
    // solve: its residual is computed as b - D x straight away
    const bool last_cycle = prm->inner_tol * maxrel <= 0.25 * prm->tol;
    const bool true_residual = (ip != DD_F32) || cyc == 0 || maxrel > theta || last_cycle;
    if ((e = to_inner(s)) != DD_OK) return e;
    if ((prm->flags & DD_SOLVE_AUTOTUNE) && cyc == 0) {
      const int pi = ip == DD_F64 ? 0 : (ip == DD_F32 ? 1 : 2);
      if (!b.tuned[pi] && (e = tune_hop(c, b, ip, rin_e, ip == DD_F64 ? tune64 : w.tmp, s)) != DD_OK)
        return e;
    }
    if ((e = schur_rhs(s)) != DD_OK) return e;
    int its = 0;
    if (prm->flags & DD_SOLVE_FGMRES) {
      dd_net* pn = ((prm->flags & DD_SOLVE_NET_PRECOND) && c->net && all_omega) ? c->net : nullptr;
      e = run_fgmres(c, b, ip, st, rhs, w.x, prm->restart, inner_tol2, floor_frac, prm->maxiter, pn, s, &its);
    } else if (ip == DD_F64)
      e = run_bicgstab<double2>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                                floor_frac, prm->maxiter, check_every, use_graph, s, &its, device_loop);
    else if (ip == DD_F32)
      e = run_bicgstab<float2>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                               floor_frac, prm->maxiter, check_every, use_graph, s, &its, device_loop);
    else
      e = run_bicgstab<__nv_bfloat162>(c, b, ip, w, st, partial, d_count, &h_count, rhs, inner_tol2,
                                       floor_frac, prm->maxiter, check_every, use_graph, s, &its, device_loop);
    if (e != DD_OK) return e;
    if ((e = correct_x(s)) != DD_OK) return e;
    if (true_residual) {
      if ((e = true_res(s)) != DD_OK) return e;
      norms_ready = dfo;
    } else {
      if ((e = update_res(s)) != DD_OK) return e;
      norms_ready = true;
    }
    last_true = true_residual;
    DD_CUDA(c, cudaGetLastError());
  }
  if ((e = launch_unpack(c, b, xe, xo, x_user, op, s)) != DD_OK) return e;
  cudaEventRecord(ev1, s);
  DD_CUDA(c, cudaGetLastError());
  std::vector<double> rel(nsys);
  std::vector<SysState> hst(nsys);
  DD_CUDA(c, cudaMemcpyAsync(rel.data(), vrel, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaMemcpyAsync(hst.data(), st, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  if ((e = check_device_error(c, s)) != DD_OK) return e;
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  dd_solve_stats out{};
  out.systems = nsys;
  out.outer_cycles = cycles;
  out.seconds = ms * 1e-3;
  {
    const int pi = ip == DD_F64 ? 0 : (ip == DD_F32 ? 1 : 2);
    out.hop_variant = c->forced_variant[pi] >= 0 ? c->forced_variant[pi] : b.hop_variant[pi];
  }
  bool nan = false;
  for (int k = 0; k < nsys; ++k) {
    if (!(rel[k] == rel[k])) nan = true;
    out.max_relres = std::max(out.max_relres, rel[k]);
    out.max_iters = std::max(out.max_iters, hst[k].iters);
    if (rel[k] <= prm->tol) out.converged++;
  }
  if (stats) *stats = out;
  c->last_stats = out;
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
