// The clover (Sheikholeslami-Wohlert) term: the site-local 12x12 term that the
// paper admits in D (Sec. 1), in kappa normalisation
//
//   A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu F_mu_nu(x),
//   sigma_mu_nu = (i/2)[gamma_mu, gamma_nu],  F_mu_nu = (Q_mu_nu - Q_mu_nu^+) / 8,
//
// Q_mu_nu(x) the four plaquettes of the mu-nu plane that start and end at x,
// each traversed mu first.  sigma_mu_nu commutes with gamma_5, so in the chiral
// basis A(x) is two Hermitian 6x6 blocks: components 0..5 (spins 0, 1) and 6..11
// (spins 2, 3), colour fastest.  Tables A and A^{-1}: [V][2][6][6] complex FP64,
// site-major (72 complex numbers per site).
//
// Solves use A as a left preconditioner: D_X x = b is solved as
// (1 - kappa A^{-1} H) x = A^{-1} b, i.e. every hop launch of the solver applies
// A^{-1} of its output site to the hop sum (epilogue in the FP64 stencil), and
// the right-hand side is multiplied by A^{-1} once.  The even-odd Schur form of
// that operator is 1 - kappa^2 A_ee^{-1} H_eo A_oo^{-1} H_oe.
#include <cmath>
#include <cstring>
#include <complex>
#include <vector>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

namespace {

struct SigmaBlocks {
  double2 s[6][2][2][2];   // plane (01, 02, 03, 12, 13, 23), chirality, row, column
};

// sigma_mu_nu in the chiral basis of the stencil: gamma_0 = [[0, -1], [-1, 0]],
// gamma_k = [[0, -i s_k], [i s_k, 0]] (2x2 blocks, s_k Pauli); the chiral blocks
// of (i/2)[gamma_mu, gamma_nu] (its off-diagonal blocks vanish)
bool sigma_blocks(SigmaBlocks& out) {
  typedef std::complex<double> cd;
  const cd I(0, 1);
  cd pauli[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  cd g[4][4][4] = {};
  for (int r = 0; r < 2; ++r) {
    g[0][r][2 + r] = -1.0;
    g[0][2 + r][r] = -1.0;
  }
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) {
        g[k + 1][r][2 + c] = -I * pauli[k][r][c];
        g[k + 1][2 + r][c] = I * pauli[k][r][c];
      }
  int plane = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
      cd sg[4][4];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          cd v = 0;
          for (int k = 0; k < 4; ++k) v += g[mu][r][k] * g[nu][k][c] - g[nu][r][k] * g[mu][k][c];
          sg[r][c] = 0.5 * I * v;
        }
      for (int ch = 0; ch < 2; ++ch)
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) {
            if (std::abs(sg[2 * ch + r][2 * (1 - ch) + c]) > 1e-14) return false;
            const cd v = sg[2 * ch + r][2 * ch + c];
            out.s[plane][ch][r][c] = make_double2(v.real(), v.imag());
          }
    }
  return true;
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cjg(double2 a) { return make_double2(a.x, -a.y); }

// C = op(A) op(B), op = identity or conjugate transpose
__device__ void mul3(const double2* A, bool da, const double2* B, bool db, double2* C) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double2 v = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const double2 a = da ? cjg(A[k * 3 + r]) : A[r * 3 + k];
        const double2 b = db ? cjg(B[c * 3 + k]) : B[k * 3 + c];
        const double2 t = cm(a, b);
        v.x += t.x;
        v.y += t.y;
      }
      C[r * 3 + c] = v;
    }
}

struct Lat {
  int L[4];
  int time_bc;
  const double2* U;   // [V][4][9], time sign folded into U_0(x0 = L0 - 1)
};

__device__ int site_of(const Lat& g, const int* x) {
  return ((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// U_mu at x + a e_m + b e_n (periodic), with the time sign unfolded (the clover
// uses the links themselves; the sign belongs to the fermion hops)
__device__ void link_at(const Lat& g, const int* x, int m, int a, int n, int b, int mu, double2* out) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[m] = ((y[m] + a) % g.L[m] + g.L[m]) % g.L[m];
  y[n] = ((y[n] + b) % g.L[n] + g.L[n]) % g.L[n];
  const double2* p = g.U + (long long)site_of(g, y) * 36 + mu * 9;
  const double sg = (mu == 0 && y[0] == g.L[0] - 1) ? (double)g.time_bc : 1.0;
  for (int k = 0; k < 9; ++k) out[k] = make_double2(sg * p[k].x, sg * p[k].y);
}

// one thread per site: A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu (x) F_mu_nu
__global__ void k_clover_build(Lat g, SigmaBlocks sig, double kc, double2* __restrict__ A) {
  const long long V = (long long)g.L[0] * g.L[1] * g.L[2] * g.L[3];
  const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= V) return;
  int x[4];
  long long r = site;
  for (int m = 3; m >= 0; --m) {
    x[m] = (int)(r % g.L[m]);
    r /= g.L[m];
  }
  double2* a = A + site * 72;
  for (int k = 0; k < 72; ++k) a[k] = make_double2(((k % 36) % 7 == 0) ? 1.0 : 0.0, 0.0);
  int plane = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
      double2 Q[9], P[9], T1[9], T2[9], l1[9], l2[9], l3[9], l4[9];
      for (int k = 0; k < 9; ++k) Q[k] = make_double2(0.0, 0.0);
      // x -> x+mu -> x+mu+nu -> x+nu -> x
      link_at(g, x, mu, 0, nu, 0, mu, l1);
      link_at(g, x, mu, 1, nu, 0, nu, l2);
      link_at(g, x, mu, 0, nu, 1, mu, l3);
      link_at(g, x, mu, 0, nu, 0, nu, l4);
      mul3(l1, false, l2, false, T1);
      mul3(T1, false, l3, true, T2);
      mul3(T2, false, l4, true, P);
      for (int k = 0; k < 9; ++k) { Q[k].x += P[k].x; Q[k].y += P[k].y; }
      // x -> x+nu -> x+nu-mu -> x-mu -> x
      link_at(g, x, mu, 0, nu, 0, nu, l1);
      link_at(g, x, mu, -1, nu, 1, mu, l2);
      link_at(g, x, mu, -1, nu, 0, nu, l3);
      link_at(g, x, mu, -1, nu, 0, mu, l4);
      mul3(l1, false, l2, true, T1);
      mul3(T1, false, l3, true, T2);
      mul3(T2, false, l4, false, P);
      for (int k = 0; k < 9; ++k) { Q[k].x += P[k].x; Q[k].y += P[k].y; }
      // x -> x-mu -> x-mu-nu -> x-nu -> x
      link_at(g, x, mu, -1, nu, 0, mu, l1);
      link_at(g, x, mu, -1, nu, -1, nu, l2);
      link_at(g, x, mu, -1, nu, -1, mu, l3);
      link_at(g, x, mu, 0, nu, -1, nu, l4);
      mul3(l1, true, l2, true, T1);
      mul3(T1, false, l3, false, T2);
      mul3(T2, false, l4, false, P);
      for (int k = 0; k < 9; ++k) { Q[k].x += P[k].x; Q[k].y += P[k].y; }
      // x -> x-nu -> x-nu+mu -> x+mu -> x
      link_at(g, x, mu, 0, nu, -1, nu, l1);
      link_at(g, x, mu, 0, nu, -1, mu, l2);
      link_at(g, x, mu, 1, nu, -1, nu, l3);
      link_at(g, x, mu, 0, nu, 0, mu, l4);
      mul3(l1, true, l2, false, T1);
      mul3(T1, false, l3, false, T2);
      mul3(T2, false, l4, true, P);
      for (int k = 0; k < 9; ++k) { Q[k].x += P[k].x; Q[k].y += P[k].y; }
      // F = (Q - Q^+) / 8; block ch gains i kc sigma^ch[s][t] F[a][b] at (3s+a, 3t+b)
      double2 F[9];
      for (int ra = 0; ra < 3; ++ra)
        for (int cb = 0; cb < 3; ++cb) {
          const double2 q = Q[ra * 3 + cb], qt = cjg(Q[cb * 3 + ra]);
          F[ra * 3 + cb] = make_double2((q.x - qt.x) * 0.125, (q.y - qt.y) * 0.125);
        }
      for (int ch = 0; ch < 2; ++ch)
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) {
            const double2 sv = sig.s[plane][ch][s][t];
            const double2 coef = make_double2(-kc * sv.y, kc * sv.x);     // i kc sigma
            if (coef.x == 0.0 && coef.y == 0.0) continue;
            for (int ra = 0; ra < 3; ++ra)
              for (int cb = 0; cb < 3; ++cb) {
                const double2 t2 = cm(coef, F[ra * 3 + cb]);
                double2& e = a[ch * 36 + (3 * s + ra) * 6 + (3 * t + cb)];
                e.x += t2.x;
                e.y += t2.y;
              }
          }
    }
}

// one thread per (site, chirality): Gauss-Jordan inverse with partial pivoting
__global__ void k_clover_invert(const double2* __restrict__ A, double2* __restrict__ Ai, long long V) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * V) return;
  const double2* a = A + k * 36;
  double2 M[36], R[36];
  for (int e = 0; e < 36; ++e) {
    M[e] = a[e];
    R[e] = make_double2(e % 7 == 0 ? 1.0 : 0.0, 0.0);
  }
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = M[col * 6 + col].x * M[col * 6 + col].x + M[col * 6 + col].y * M[col * 6 + col].y;
    for (int row = col + 1; row < 6; ++row) {
      const double2 v = M[row * 6 + col];
      const double m2 = v.x * v.x + v.y * v.y;
      if (m2 > best) {
        best = m2;
        piv = row;
      }
    }
    if (piv != col)
      for (int c = 0; c < 6; ++c) {
        double2 t = M[col * 6 + c]; M[col * 6 + c] = M[piv * 6 + c]; M[piv * 6 + c] = t;
        t = R[col * 6 + c]; R[col * 6 + c] = R[piv * 6 + c]; R[piv * 6 + c] = t;
      }
    // 1 / pivot (a singular block gives Inf/NaN, which the solver reports)
    const double2 p = M[col * 6 + col];
    const double d = p.x * p.x + p.y * p.y;
    const double2 inv = make_double2(p.x / d, -p.y / d);
    for (int c = 0; c < 6; ++c) {
      M[col * 6 + c] = cm(M[col * 6 + c], inv);
      R[col * 6 + c] = cm(R[col * 6 + c], inv);
    }
    for (int row = 0; row < 6; ++row) {
      if (row == col) continue;
      const double2 f = M[row * 6 + col];
      if (f.x == 0.0 && f.y == 0.0) continue;
      for (int c = 0; c < 6; ++c) {
        const double2 tm = cm(f, M[col * 6 + c]), tr = cm(f, R[col * 6 + c]);
        M[row * 6 + c].x -= tm.x; M[row * 6 + c].y -= tm.y;
        R[row * 6 + c].x -= tr.x; R[row * 6 + c].y -= tr.y;
      }
    }
  }
  double2* o = Ai + k * 36;
  for (int e = 0; e < 36; ++e) o[e] = R[e];
}

// v <- M(x) v on one parity of a batch (M = A or A^{-1}, site-major tables)
__global__ void k_clover_apply(BatchDev bd, int p, double2* v, const double2* __restrict__ M) {
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* d = bd.inst_tab + bd.inst[it.x];
  const int n0 = d->n[0];
  const int n = p ? d->n[1] : n0;
  if ((int)threadIdx.x >= it.z) return;
  const int i = it.y + threadIdx.x;
  double2* base = v + (p ? bd.off[1] : bd.off[0])[sys];
  double2 w[12];
  ld_site<12>(base, n, i, w);
  clover_mul(M + 72LL * d->glob[(p ? n0 : 0) + i], w);
  st_site<12>(base, n, i, w);
}

// one thread per (site, chirality block): the largest absolute row sum of the
// 6x6 block of A (m = 0) and of A^{-1} (m = 1), folded into out[m] by an atomic
// max on the bit pattern (non-negative doubles order like their bits).  For a
// hermitian matrix the row-sum norm bounds the spectral norm.
__global__ void k_clover_rownorm(const double2* __restrict__ A, const double2* __restrict__ Ai, long long V,
                                 unsigned long long* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * V) return;
  for (int m = 0; m < 2; ++m) {
    const double2* a = (m ? Ai : A) + k * 36;
    double best = 0.0;
    for (int r = 0; r < 6; ++r) {
      double sum = 0.0;
      for (int c = 0; c < 6; ++c) sum += hypot(a[r * 6 + c].x, a[r * 6 + c].y);
      best = fmax(best, sum);
    }
    atomicMax(out + m, (unsigned long long)__double_as_longlong(best));
  }
}

// one thread per (site, chirality block): the hermitian-packed FP32 and
// double-float copies of A^{-1} (diagonal real parts, then the entries above
// the diagonal row by row)
__global__ void k_clover_pack(const double2* __restrict__ Ai, float4* __restrict__ t32,
                              float4* __restrict__ tdf, long long V) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * V) return;
  const double2* a = Ai + k * 36;
  float f[36];
  float4* o = tdf + k * 18;
  for (int q = 0; q < 3; ++q) {
    const float2 d0 = split_d(a[(2 * q) * 7].x), d1 = split_d(a[(2 * q + 1) * 7].x);
    o[q] = make_float4(d0.x, d0.y, d1.x, d1.y);
  }
  for (int r = 0; r < 6; ++r) f[r] = (float)a[r * 7].x;
  int z = 6, zq = 3;
  for (int r = 0; r < 6; ++r)
    for (int c = r + 1; c < 6; ++c, z += 2, ++zq) {
      const double2 m = a[r * 6 + c];
      f[z] = (float)m.x;
      f[z + 1] = (float)m.y;
      const float2 re = split_d(m.x), im = split_d(m.y);
      o[zq] = make_float4(re.x, im.x, re.y, im.y);
    }
  float4* o32 = t32 + k * 9;
  for (int q = 0; q < 9; ++q) o32[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

// v <- A^{-1}(x) v on one parity of a batch of double-float vectors, in FP64
// from the full table (once per solve: the preconditioned right-hand side)
__global__ void k_clover_apply_df(BatchDev bd, int p, df2s* v, const double2* __restrict__ M) {
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* d = bd.inst_tab + bd.inst[it.x];
  const int n0 = d->n[0];
  const int n = p ? d->n[1] : n0;
  if ((int)threadIdx.x >= it.z) return;
  const int i = it.y + threadIdx.x;
  df2s* base = v + (p ? bd.off[1] : bd.off[0])[sys];
  dfc u[12];
  ld_site<12>(base, n, i, u);
  double2 w[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) w[k] = to_d2(u[k]);
  clover_mul(M + 72LL * d->glob[(p ? n0 : 0) + i], w);
#pragma unroll
  for (int k = 0; k < 12; ++k) u[k] = cmk<dfc>(w[k].x, w[k].y);
  st_site<12>(base, n, i, u);
}

}  // namespace

dd_status clover_mixed_tables(dd_ctx* c) {
  if (!c->clover_ready) return fail(c, DD_EINVAL, "clover term not built");
  if (c->clover_mixed_ready) return DD_OK;
  dd_status e;
  if (!c->d_clovi32 && (e = dalloc(c, (void**)&c->d_clovi32, sizeof(float4) * 18ULL * c->V)) != DD_OK) return e;
  if (!c->d_clovi_df && (e = dalloc(c, (void**)&c->d_clovi_df, sizeof(float4) * 36ULL * c->V)) != DD_OK)
    return e;
  DD_COUNT_LAUNCH(), k_clover_pack<<<(unsigned)((2LL * c->V + 127) / 128), 128>>>(c->d_clovi, c->d_clovi32,
                                                                                  c->d_clovi_df, (long long)c->V);
  DD_CUDA(c, cudaGetLastError());
  DD_CUDA(c, cudaDeviceSynchronize());
  c->clover_mixed_ready = true;
  return DD_OK;
}

dd_status clover_apply_inv_df(dd_ctx* c, const Batch& b, void* ve, void* vo, cudaStream_t s) {
  if (!c->clover_ready) return fail(c, DD_EINVAL, "clover term not built");
  dd_status e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  if (b.nitems[0] > 0)
    DD_COUNT_LAUNCH(), k_clover_apply_df<<<dim3(b.nitems[0], b.nrhs), 128, 0, s>>>(bd, 0, (df2s*)ve, c->d_clovi);
  if (b.nitems[1] > 0)
    DD_COUNT_LAUNCH(), k_clover_apply_df<<<dim3(b.nitems[1], b.nrhs), 128, 0, s>>>(bd, 1, (df2s*)vo, c->d_clovi);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

dd_status clover_build(dd_ctx* c) {
  c->clover_ready = false;
  c->clover_mixed_ready = false;
  if (c->csw == 0.0 || !c->gauge_ready) return DD_OK;
  SigmaBlocks sig;
  if (!sigma_blocks(sig)) return fail(c, DD_EINVAL, "sigma_mu_nu is not chirally block-diagonal");
  const size_t bytes = sizeof(double2) * 72ULL * c->V;
  dd_status e;
  if (!c->d_clov && (e = dalloc(c, (void**)&c->d_clov, bytes)) != DD_OK) return e;
  if (!c->d_clovi && (e = dalloc(c, (void**)&c->d_clovi, bytes)) != DD_OK) return e;
  Lat g;
  for (int m = 0; m < 4; ++m) g.L[m] = c->L[m];
  g.time_bc = c->time_bc;
  g.U = c->d_U;
  DD_COUNT_LAUNCH(), k_clover_build<<<(c->V + 127) / 128, 128>>>(g, sig, c->kappa * c->csw, c->d_clov);
  DD_CUDA(c, cudaGetLastError());
  DD_COUNT_LAUNCH(), k_clover_invert<<<(unsigned)((2LL * c->V + 127) / 128), 128>>>(c->d_clov, c->d_clovi,
                                                                                    (long long)c->V);
  DD_CUDA(c, cudaGetLastError());
  // cond_2(A) <= max_x |A_x|_inf * max_x |A_x^{-1}|_inf (hermitian chiral blocks)
  unsigned long long* dn = nullptr;
  if ((e = dalloc(c, (void**)&dn, 2 * sizeof(unsigned long long))) != DD_OK) return e;
  DD_CUDA(c, cudaMemset(dn, 0, 2 * sizeof(unsigned long long)));
  DD_COUNT_LAUNCH(), k_clover_rownorm<<<(unsigned)((2LL * c->V + 127) / 128), 128>>>(c->d_clov, c->d_clovi,
                                                                                     (long long)c->V, dn);
  DD_CUDA(c, cudaGetLastError());
  unsigned long long hn[2] = {0, 0};
  DD_CUDA(c, cudaMemcpy(hn, dn, sizeof hn, cudaMemcpyDeviceToHost));
  dfree(dn);
  double na, ni;
  memcpy(&na, &hn[0], sizeof na);
  memcpy(&ni, &hn[1], sizeof ni);
  c->clover_cond = na * ni;
  if (!(c->clover_cond >= 1.0) || std::isinf(c->clover_cond))
    return fail(c, DD_EINVAL, "the clover term A is singular or ill-conditioned");
  c->clover_ready = true;
  return DD_OK;
}

dd_status clover_apply(dd_ctx* c, const Batch& b, void* ve, void* vo, bool inverse, cudaStream_t s) {
  if (!c->clover_ready) return fail(c, DD_EINVAL, "clover term not built");
  dd_status e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  const double2* M = inverse ? c->d_clovi : c->d_clov;
  if (b.nitems[0] > 0)
    DD_COUNT_LAUNCH(), k_clover_apply<<<dim3(b.nitems[0], b.nrhs), 128, 0, s>>>(bd, 0, (double2*)ve, M);
  if (b.nitems[1] > 0)
    DD_COUNT_LAUNCH(), k_clover_apply<<<dim3(b.nitems[1], b.nrhs), 128, 0, s>>>(bd, 1, (double2*)vo, M);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_clover_cond(dd_ctx* c, double* c_A) {
  if (!c || !c_A) return DD_EINVAL;
  if (c->csw != 0.0 && !c->clover_ready) {
    dd_status e = clover_build(c);
    if (e != DD_OK) return e;
  }
  *c_A = c->csw != 0.0 ? c->clover_cond : 1.0;
  return DD_OK;
}

dd_status dd_set_clover(dd_ctx* c, double csw) {
  if (!c) return DD_EINVAL;
  if (!(csw == csw) || std::isinf(csw)) return fail(c, DD_EINVAL, "c_sw must be finite");
  c->csw = csw;
  if (csw == 0.0) {
    c->clover_ready = false;
    return DD_OK;
  }
  return clover_build(c);
}

}  // extern "C"
