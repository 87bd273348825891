// Flexible GMRES(m) (Saad 1993) for the batched even-odd Schur systems
//   M x_e = rhs_e,  M = 1 - k^2 H_eo H_oe
// of the framed blocks, frame pieces and the frame (the inner solve of the
// defect-correction loop in krylov.cu, beside BiCGstab).  One Arnoldi process
// per (instance, rhs) system, all systems in step: for j = 0 .. m-1
//   z_j = P(v_j)              (P = 1, or the learned network: variable in j)
//   w = M z_j ;  h_ij = (v_i, w), w -= sum_i h_ij v_i  (classical Gram-Schmidt)
//   h_{j+1,j} = |w| ;  v_{j+1} = w / h_{j+1,j}
// with the Hessenberg column reduced by complex Givens rotations on the device,
// so |g_{j+1}| is the residual norm of the least-squares solution after j+1
// steps; at the end of a cycle x += sum_j y_j z_j with R y = g, and the next
// cycle restarts from r = rhs - M x.  Vectors at the inner precision (FP32 or
// FP64), inner products and every scalar in FP64.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "spinor.cuh"

namespace dd {
namespace {

constexpr int FG_MAX = 16;

struct FgState {
  double2 H[(FG_MAX + 1) * FG_MAX];   // H[i + (FG_MAX + 1) j], rotated in place
  double2 g[FG_MAX + 1];              // rotated right-hand side of the least squares
  double2 sn[FG_MAX];
  double cs[FG_MAX];
  double2 y[FG_MAX];
  double target2;                     // stop when |r|^2 <= target2
  double beta;                        // |r| at the start of the cycle
  double hnext;                       // h_{j+1,j} before rotation (the scale of v_{j+1})
  int k;                              // Arnoldi steps of the current cycle
  int active;                         // the current cycle runs for this system
  int run;                            // the system is not solved yet
  int pad;
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zdivr(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double2 slot_sum(const double* partial, int slot, long long stride, int ib0, int ib1,
                                            int nrhs, int r) {
  double2 s = make_double2(0.0, 0.0);
  const double* P = partial + 2 * slot * stride;
  for (int it = ib0; it < ib1; ++it) {
    const long long k = (long long)it * nrhs + r;
    s.x += P[2 * k];
    s.y += P[2 * k + 1];
  }
  return s;
}

#define FG_PROLOGUE                                           \
  const int4 it = bd.items[0][blockIdx.x];                    \
  const int rh = blockIdx.y;                                  \
  const int sys = it.x * bd.nrhs + rh;                        \
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];            \
  const int n = dp->n[0];                                     \
  const int i = it.y + threadIdx.x;                           \
  const bool live = threadIdx.x < it.z;                       \
  const long long o = bd.off[0][sys];                         \
  const long long m_ = (long long)blockIdx.x * bd.nrhs + rh;  \
  const long long stride = (long long)bd.nitems[0] * bd.nrhs;

// r = rhs - mx (mx null: r = rhs), |r|^2 into slot 0; with zero_x also x = 0
template <class S>
__global__ void k_fg_resid(BatchDev bd, const S* __restrict__ rhs, const S* __restrict__ mx, S* r, S* x,
                           const FgState* fg, bool zero_x, double* partial) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[64];
  FG_PROLOGUE
  if (!zero_x && !fg[sys].run) return;
  double acc[1] = {0.0};
  if (live) {
    C b[12];
    ld_site<12>(rhs + o, n, i, b);
    if (mx) {
      C v[12];
      ld_site<12>(mx + o, n, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) b[k] = csub(b[k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0] += (double)b[k].x * b[k].x + (double)b[k].y * b[k].y;
    st_site<12>(r + o, n, i, b);
    if (zero_x) {
      C z[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) z[k] = cmk<C>(0.0, 0.0);
      st_site<12>(x + o, n, i, z);
    }
  }
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) {
    partial[2 * m_] = acc[0];
    partial[2 * m_ + 1] = 0.0;
  }
  (void)stride;
}

// dst = src / scale (v_0 = r / beta, v_{j+1} = w / h_{j+1,j}) for active systems
template <class S>
__global__ void k_fg_scale(BatchDev bd, const FgState* fg, const S* __restrict__ src, S* dst, bool first) {
  typedef typename StoreTraits<S>::C C;
  FG_PROLOGUE
  if (!live || !fg[sys].active) return;
  const double sc = 1.0 / (first ? fg[sys].beta : fg[sys].hnext);
  C v[12];
  ld_site<12>(src + o, n, i, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = cmk<C>((double)v[k].x * sc, (double)v[k].y * sc);
  st_site<12>(dst + o, n, i, v);
  (void)stride;
  (void)m_;
}

// partials of (v_i, w) = sum conj(v_i) w, i < nv, into slots 0 .. nv-1
template <class S>
__global__ void k_fg_dots(BatchDev bd, const FgState* fg, const S* __restrict__ V, long long vstride, int nv,
                          const S* __restrict__ w, double* partial) {
  typedef typename StoreTraits<S>::C C;
  typedef typename StoreTraits<S>::T T;
  __shared__ double red[64];
  FG_PROLOGUE
  if (!fg[sys].active) return;
  C wv[12];
  if (live) ld_site<12>(w + o, n, i, wv);
  for (int q = 0; q < nv; ++q) {
    T t[2] = {0, 0};
    if (live) {
      C v[12];
      ld_site<12>(V + q * vstride + o, n, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        t[0] = fma(v[k].x, wv[k].x, fma(v[k].y, wv[k].y, t[0]));
        t[1] = fma(v[k].x, wv[k].y, fma(-v[k].y, wv[k].x, t[1]));
      }
    }
    double acc[2];
    block_reduce_t<T, 2>(t, acc, red);
    if (threadIdx.x == 0) {
      partial[2 * (q * stride + m_)] = acc[0];
      partial[2 * (q * stride + m_) + 1] = acc[1];
    }
  }
}

// w -= sum_{i < nv} h_ij v_i, |w|^2 into slot 0
template <class S>
__global__ void k_fg_orth(BatchDev bd, const FgState* fg, const S* __restrict__ V, long long vstride, int nv,
                          int j, S* w, double* partial) {
  typedef typename StoreTraits<S>::C C;
  __shared__ double red[64];
  FG_PROLOGUE
  if (!fg[sys].active) return;
  double acc[1] = {0.0};
  if (live) {
    C wv[12];
    ld_site<12>(w + o, n, i, wv);
    for (int q = 0; q < nv; ++q) {
      const double2 h = fg[sys].H[q + (FG_MAX + 1) * j];
      const C hc = cmk<C>(h.x, h.y);
      C v[12];
      ld_site<12>(V + q * vstride + o, n, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) wv[k] = csub(wv[k], cmul(hc, v[k]));
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0] += (double)wv[k].x * wv[k].x + (double)wv[k].y * wv[k].y;
    st_site<12>(w + o, n, i, wv);
  }
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) {
    partial[2 * m_] = acc[0];
    partial[2 * m_ + 1] = 0.0;
  }
  (void)stride;
}

// x += sum_{i < k} y_i z_i for the systems that ran steps in this cycle
template <class S>
__global__ void k_fg_update(BatchDev bd, const FgState* fg, S* x, const S* __restrict__ Z, long long vstride) {
  typedef typename StoreTraits<S>::C C;
  FG_PROLOGUE
  const int kk = fg[sys].k;
  if (!live || kk == 0) return;
  C xv[12];
  ld_site<12>(x + o, n, i, xv);
  for (int q = 0; q < kk; ++q) {
    const double2 yq = fg[sys].y[q];
    const C yc = cmk<C>(yq.x, yq.y);
    C z[12];
    ld_site<12>(Z + q * vstride + o, n, i, z);
#pragma unroll
    for (int k = 0; k < 12; ++k) xv[k] = cadd(xv[k], cmul(yc, z[k]));
  }
  st_site<12>(x + o, n, i, xv);
  (void)stride;
  (void)m_;
}

// ---- per-system scalar kernels (one thread per system) ------------------------------
struct FgArgs {
  FgState* fg;
  SysState* st;
  const double* partial;
  const int* item_begin;
  long long stride;
  int nsys, nrhs;
};

// start of a cycle: beta = |r|; the first cycle also sets the target
// max(inner_tol2 |rhs|^2, floor_frac outer2) and takes the systems still in
// the outer loop; systems at or below the target stop
__global__ void k_fg_start(FgArgs a, bool first, double inner_tol2, double floor_frac, int* count) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  const int j = sys / a.nrhs, r = sys % a.nrhs;
  FgState& f = a.fg[sys];
  SysState& s = a.st[sys];
  const double rr = slot_sum(a.partial, 0, a.stride, a.item_begin[j], a.item_begin[j + 1], a.nrhs, r).x;
  if (first) {
    f.target2 = fmax(inner_tol2 * rr, floor_frac * s.outer2);
    f.run = s.outer_active;
  }
  if (!(rr == rr)) f.run = 0;
  if (f.run && rr <= f.target2) f.run = 0;
  f.beta = sqrt(rr);
  f.k = 0;
  f.active = f.run;
  for (int q = 0; q <= FG_MAX; ++q) f.g[q] = make_double2(0.0, 0.0);
  f.g[0] = make_double2(f.beta, 0.0);
  if (f.active) atomicAdd(count, 1);
}

// column j of H from the slot partials (i <= j)
__global__ void k_fg_hcol(FgArgs a, int j) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  FgState& f = a.fg[sys];
  if (!f.active) return;
  const int jj = sys / a.nrhs, r = sys % a.nrhs;
  for (int q = 0; q <= j; ++q)
    f.H[q + (FG_MAX + 1) * j] = slot_sum(a.partial, q, a.stride, a.item_begin[jj], a.item_begin[jj + 1], a.nrhs, r);
}

// h_{j+1,j} = |w|; the earlier rotations and a new one applied to column j;
// |g_{j+1}| is the residual norm after j+1 steps
__global__ void k_fg_givens(FgArgs a, int j, int m, int* count) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  FgState& f = a.fg[sys];
  if (!f.active) return;
  const int jj = sys / a.nrhs, r = sys % a.nrhs;
  const double hn = sqrt(slot_sum(a.partial, 0, a.stride, a.item_begin[jj], a.item_begin[jj + 1], a.nrhs, r).x);
  f.hnext = hn;
  double2* col = f.H + (FG_MAX + 1) * j;
  for (int q = 0; q < j; ++q) {
    const double2 x0 = col[q], x1 = col[q + 1];
    col[q] = zadd(make_double2(f.cs[q] * x0.x, f.cs[q] * x0.y), zmul(f.sn[q], x1));
    col[q + 1] = zsub(make_double2(f.cs[q] * x1.x, f.cs[q] * x1.y), zmul(zconj(f.sn[q]), x0));
  }
  const double2 aa = col[j];
  const double na = sqrt(aa.x * aa.x + aa.y * aa.y);
  const double rho = sqrt(na * na + hn * hn);
  double c;
  double2 sn, rj;
  if (na == 0.0) {
    c = 0.0;
    sn = make_double2(1.0, 0.0);
    rj = make_double2(hn, 0.0);
  } else {
    const double2 ph = make_double2(aa.x / na, aa.y / na);
    c = na / rho;
    sn = make_double2(ph.x * hn / rho, ph.y * hn / rho);
    rj = make_double2(ph.x * rho, ph.y * rho);
  }
  f.cs[j] = c;
  f.sn[j] = sn;
  col[j] = rj;
  col[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = f.g[j];
  f.g[j + 1] = zmul(make_double2(-sn.x, sn.y), gj);          // -conj(sn) g_j
  f.g[j] = make_double2(c * gj.x, c * gj.y);
  f.k = j + 1;
  a.st[sys].iters += 1;
  const double res2 = f.g[j + 1].x * f.g[j + 1].x + f.g[j + 1].y * f.g[j + 1].y;
  if (!(res2 == res2)) {
    f.active = 0;
    f.run = 0;
    a.st[sys].status = 3;
  } else if (res2 <= f.target2) {
    f.active = 0;
    f.run = 0;
  } else if (f.k == m || hn == 0.0 || rho == 0.0) {
    f.active = 0;                                // end of the cycle (or an exact breakdown)
  } else {
    atomicAdd(count, 1);
  }
}

// R y = g by back-substitution over the k steps of the cycle
__global__ void k_fg_solve(FgArgs a) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys) return;
  FgState& f = a.fg[sys];
  for (int q = f.k - 1; q >= 0; --q) {
    double2 v = f.g[q];
    for (int l = q + 1; l < f.k; ++l) v = zsub(v, zmul(f.H[q + (FG_MAX + 1) * l], f.y[l]));
    const double2 d = f.H[q + (FG_MAX + 1) * q];
    f.y[q] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : zdivr(v, d);
  }
}

}  // namespace

template <class S>
static dd_status fgmres_t(dd_ctx* c, const Batch& b, dd_prec prec, SysState* st, const void* rhs, void* x,
                          int m, double inner_tol2, double floor_frac, int maxiter, dd_net* net, cudaStream_t s,
                          int* iters_run) {
  const int nsys = b.nb * b.nrhs;
  const long long ne = b.tot[0], no = b.tot[1];
  const long long stride = (long long)b.nitems[0] * b.nrhs;
  const size_t vb = sizeof(S) * (size_t)ne;
  dd_status e;
  void *vV, *vZ, *vfg, *vpart, *vw, *vt, *vr, *vcnt;
  if ((e = workspace(c, 150, vb * (m + 1), &vV)) || (e = workspace(c, 152, sizeof(FgState) * nsys, &vfg)) ||
      (e = workspace(c, 153, sizeof(double) * 2 * (FG_MAX + 1) * std::max<long long>(1, stride), &vpart)) ||
      (e = workspace(c, 154, vb, &vw)) || (e = workspace(c, 155, sizeof(S) * (size_t)no + 16, &vt)) ||
      (e = workspace(c, 156, vb, &vr)) || (e = workspace(c, 157, 64, &vcnt)))
    return e;
  if (net) {
    if ((e = workspace(c, 151, vb * m, &vZ)) != DD_OK) return e;
  } else {
    vZ = vV;                                      // unpreconditioned: z_j = v_j
  }
  S* V = (S*)vV;
  S* Z = (S*)vZ;
  FgState* fg = (FgState*)vfg;
  double* partial = (double*)vpart;
  int* d_count = (int*)vcnt;
  BatchDev bd = batch_view(c, b);
  FgArgs fa{fg, st, partial, b.d_item_begin[0], stride, nsys, b.nrhs};
  const int sth = 128, sbl = (nsys + sth - 1) / sth;
  dim3 eg(b.nitems[0], b.nrhs);
  const double k2 = c->kappa * c->kappa;
  const int* act = (const int*)((const char*)fg + offsetof(FgState, active));
  const int* runf = (const int*)((const char*)fg + offsetof(FgState, run));
  const int fstride = (int)(sizeof(FgState) / sizeof(int));
  auto count = [&](int* h) -> dd_status {
    DD_CUDA(c, cudaMemcpyAsync(h, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    return DD_OK;
  };
  // w = M z (two hops), for the systems whose flag is set
  auto matvec = [&](const void* z, void* w, const int* flags) -> dd_status {
    HopArgs h1{};
    h1.p_out = 1; h1.in = z; h1.out = vt; h1.b = 1.0;
    h1.active = flags; h1.active_stride = fstride;
    dd_status q = launch_hop(c, b, prec, h1, s);
    if (q != DD_OK) return q;
    HopArgs h2{};
    h2.p_out = 0; h2.in = vt; h2.out = w; h2.s1 = z; h2.a1 = 1.0; h2.b = -k2;
    h2.active = flags; h2.active_stride = fstride;
    return launch_hop(c, b, prec, h2, s);
  };
  DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
  DD_COUNT_LAUNCH(), k_fg_resid<S><<<eg, 128, 0, s>>>(bd, (const S*)rhs, nullptr, (S*)vr, (S*)x, fg, true, partial);
  DD_COUNT_LAUNCH(), k_fg_start<<<sbl, sth, 0, s>>>(fa, true, inner_tol2, floor_frac, d_count);
  DD_CUDA(c, cudaGetLastError());
  int h = 0, steps = 0;
  if ((e = count(&h)) != DD_OK) return e;
  while (h > 0 && steps < maxiter) {
    DD_COUNT_LAUNCH(), k_fg_scale<S><<<eg, 128, 0, s>>>(bd, fg, (const S*)vr, V, true);
    int j = 0;
    for (; j < m && steps < maxiter; ++j, ++steps) {
      S* vj = V + (size_t)j * ne;
      S* zj = Z + (size_t)j * ne;
      if (net && (e = net_precondition(c, net, b, (const float2*)vj, (float2*)zj, s)) != DD_OK) return e;
      if ((e = matvec(zj, vw, act)) != DD_OK) return e;
      DD_COUNT_LAUNCH(), k_fg_dots<S><<<eg, 128, 0, s>>>(bd, fg, V, ne, j + 1, (const S*)vw, partial);
      DD_COUNT_LAUNCH(), k_fg_hcol<<<sbl, sth, 0, s>>>(fa, j);
      DD_COUNT_LAUNCH(), k_fg_orth<S><<<eg, 128, 0, s>>>(bd, fg, V, ne, j + 1, j, (S*)vw, partial);
      DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
      DD_COUNT_LAUNCH(), k_fg_givens<<<sbl, sth, 0, s>>>(fa, j, m, d_count);
      if (j + 1 < m)
        DD_COUNT_LAUNCH(), k_fg_scale<S><<<eg, 128, 0, s>>>(bd, fg, (const S*)vw, V + (size_t)(j + 1) * ne, false);
      DD_CUDA(c, cudaGetLastError());
      if ((e = count(&h)) != DD_OK) return e;
      if (h == 0) {
        ++j;
        ++steps;
        break;
      }
    }
    DD_COUNT_LAUNCH(), k_fg_solve<<<sbl, sth, 0, s>>>(fa);
    DD_COUNT_LAUNCH(), k_fg_update<S><<<eg, 128, 0, s>>>(bd, fg, (S*)x, Z, ne);
    // restart from r = rhs - M x for the systems not yet solved
    if ((e = matvec(x, vw, runf)) != DD_OK) return e;
    DD_CUDA(c, cudaMemsetAsync(d_count, 0, sizeof(int), s));
    DD_COUNT_LAUNCH(), k_fg_resid<S><<<eg, 128, 0, s>>>(bd, (const S*)rhs, (const S*)vw, (S*)vr, nullptr, fg, false,
                                                        partial);
    DD_COUNT_LAUNCH(), k_fg_start<<<sbl, sth, 0, s>>>(fa, false, inner_tol2, floor_frac, d_count);
    DD_CUDA(c, cudaGetLastError());
    if ((e = count(&h)) != DD_OK) return e;
  }
  *iters_run = steps;
  return DD_OK;
}

dd_status run_fgmres(dd_ctx* c, const Batch& b, dd_prec prec, SysState* st, const void* rhs, void* x, int restart,
                     double inner_tol2, double floor_frac, int maxiter, dd_net* net, cudaStream_t s,
                     int* iters_run) {
  const int m = std::min(std::max(restart, 1), FG_MAX);
  if (prec == DD_F32)
    return fgmres_t<float2>(c, b, prec, st, rhs, x, m, inner_tol2, floor_frac, maxiter, net, s, iters_run);
  if (net) return fail(c, DD_EINVAL, "the network preconditions FP32 inner solves only");
  if (prec == DD_F64)
    return fgmres_t<double2>(c, b, prec, st, rhs, x, m, inner_tol2, floor_frac, maxiter, nullptr, s, iters_run);
  return fail(c, DD_EINVAL, "FGMRES runs FP32 or FP64 inner solves");
}

}  // namespace dd
