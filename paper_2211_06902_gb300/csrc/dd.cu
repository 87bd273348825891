// The operator w (paper Sec. 3, Eqs. Wz and offdiagW1) and the multi-boson
// action (paper Sec. 4, Eqs. MBaction, localMB, globalMB).
//
// W_1 = diag(D^d, D^_{dPi1})^{-1} M is the matrix of the second Schur
// decomposition as the paper prints it (the hopping block D^h in its
// symmetrised form over the frame pieces Phi1^a and Phi1^b).  It factors as
// W_1 = E (1 - Q): Q maps chi on dLambda0 to dPi1,
//   (Q chi)(x) = sum_{b : x in Phi1^b} [D_{Phi1^b}^{-1} D_{Phi1^b, dLambda0^b} chi](x),
// and E is the Dirichlet extension of chi into the framed blocks and the frame,
//   (E chi)_{dLambda0^a} = chi + P D_{Omega0^a}^{-1} D_{Omega0^a, ext} chi,
//   (E chi)_{dPi1}       = chi + P D_{Lambda1}^{-1} D_{Lambda1, dLambda0} chi.
// (Both sides are linear in the printed blocks: the rows of D^h unfold, by the
// block inverses of D_{Omega0^a} and D_{Lambda1}, into the Phi-solve of Q followed
// by the Omega-solve of E.)  So one application of w = 1 - W_1 is
//   stage A: the frame pieces Y_b = D_{Phi_b}^{-1} D_{Phi_b, dL0b} chi of every block
//            and the frame y = D_{Lambda1}^{-1} D_{Lambda1, dL0} chi, one batch;
//            chi' = chi - Q chi on dPi1, (w chi)_{dPi1} = Q chi - y;
//   stage B: the framed blocks x_a = D_{Omega_a}^{-1} D_{Omega_a, ext} chi', one batch;
//            (w chi)_{dLambda0^a} = -x_a.
// Without dPi1 (one decomposed direction) Q = 0 and stage A is skipped.
//
//   S = sum_k |(u_k - w) chi_k|^2 = sum_a S^a + S^r
//
// Boundary injection (D_{X, ext} chi: the hops from the sites just outside X
// into X) is a gather from chi on dPi with the global FP64 links; the block,
// frame-piece and frame solves go through the batched solver; extraction and the
// FP64 reductions follow in fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

namespace {

struct InjectArgs {
  const double2* U;        // global links [V][4][9], time sign folded
  const double2* chi;      // [f][n_dpi][12]
  const int* dpi_pos;      // [V] -> dPi index or -1
  double2* src;            // caller-layout sources of the batch
  int L[4];
  int n_dpi, n_f;
  double kappa;
};

__device__ __forceinline__ void site_coords(long long s, const int* dims, int* x) {
  x[3] = (int)(s % dims[3]);
  x[2] = (int)((s / dims[3]) % dims[2]);
  x[1] = (int)((s / ((long long)dims[3] * dims[2])) % dims[1]);
  x[0] = (int)(s / ((long long)dims[3] * dims[2] * dims[1]));
}

__device__ __forceinline__ int glob_index(const int* x, const int* L) {
  return ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3];
}

// Adds the hop from global site y (direction dir seen from x) into acc.
__device__ void add_exterior_hop(double2 (&acc)[12], int dir, int gx, int gy, const InjectArgs& a,
                                 int f) {
  const int mu = dir & 3;
  const bool fwd = dir < 4;
  const int q = a.dpi_pos[gy];
  if (q < 0) return;     // cannot happen for a valid geometry (exterior sites lie on dPi)
  double2 psi[12];
  const double2* c = a.chi + ((long long)f * a.n_dpi + q) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) psi[k] = c[k];
  double2 U[9];
  const double2* l = a.U + (long long)(fwd ? gx : gy) * 36 + mu * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) U[k] = l[k];
  switch (dir) {
    case 0: hop_dir<0, true>(acc, psi, U); break;
    case 1: hop_dir<1, true>(acc, psi, U); break;
    case 2: hop_dir<2, true>(acc, psi, U); break;
    case 3: hop_dir<3, true>(acc, psi, U); break;
    case 4: hop_dir<0, false>(acc, psi, U); break;
    case 5: hop_dir<1, false>(acc, psi, U); break;
    case 6: hop_dir<2, false>(acc, psi, U); break;
    default: hop_dir<3, false>(acc, psi, U); break;
  }
}

// Sources for the Omega blocks: s(x) = D_{Omega, ext} chi, x in the box.
// grid: (ceil(max_sites/128), n_f, nblk)
__global__ void k_inject_omega(BatchDev bd, InjectArgs a) {
  const int f = blockIdx.y, j = blockIdx.z;
  const int sys = j * a.n_f + f;
  const DomInst* d = bd.inst_tab + bd.inst[j];
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d->nsites) return;
  int dims[4] = {d->dims[0], d->dims[1], d->dims[2], d->dims[3]};
  int x[4];
  site_coords(l, dims, x);
  int g[4];
  for (int m = 0; m < 4; ++m) g[m] = (d->origin[m] + x[m]) % a.L[m];
  const int gx = glob_index(g, a.L);
  double2 acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = make_double2(0.0, 0.0);
  for (int dir = 0; dir < 8; ++dir) {
    const int mu = dir & 3, step = dir < 4 ? 1 : -1;
    const int y = x[mu] + step;
    if (y >= 0 && y < dims[mu]) continue;           // hop stays inside the box
    if (dims[mu] == a.L[mu]) continue;              // box wraps (direction not decomposed)
    int gy[4] = {g[0], g[1], g[2], g[3]};
    gy[mu] = (g[mu] + step + a.L[mu]) % a.L[mu];
    add_exterior_hop(acc, dir, gx, glob_index(gy, a.L), a, f);
  }
  double2* out = a.src + bd.uoff[sys] + 12 * l;
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = make_double2(-a.kappa * acc[k].x, -a.kappa * acc[k].y);
}

// Sources for the frame: t(x) = D_{Lambda1, dLambda0} chi, x in Lambda1 (field order).
__global__ void k_inject_frame(const int* __restrict__ l1_glob, int n_l1,
                               const unsigned char* __restrict__ in_l1, InjectArgs a) {
  const int f = blockIdx.y;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_l1) return;
  const int gx = l1_glob[k];
  int g[4];
  site_coords(gx, a.L, g);
  double2 acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = make_double2(0.0, 0.0);
  for (int dir = 0; dir < 8; ++dir) {
    const int mu = dir & 3, step = dir < 4 ? 1 : -1;
    int gy[4] = {g[0], g[1], g[2], g[3]};
    gy[mu] = (g[mu] + step + a.L[mu]) % a.L[mu];
    const int y = glob_index(gy, a.L);
    if (in_l1[y]) continue;                           // neighbour inside the frame
    add_exterior_hop(acc, dir, gx, y, a, f);
  }
  double2* out = a.src + ((long long)f * n_l1 + k) * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) out[c] = make_double2(-a.kappa * acc[c].x, -a.kappa * acc[c].y);
}

// Sources of the frame pieces: t(x) = D_{Phi1^b, dLambda0^b} chi for x in
// Phi1^b, the hops into x from the boundary sites of its own core b (batch
// position j holds Phi1^b, b = blk_of_pos[j], or b = j without the map).
// grid: (ceil(max_sites/128), n_f, nb)
__global__ void k_inject_phi(BatchDev bd, InjectArgs a, const int* __restrict__ dpi_kind,
                             const int* __restrict__ blk_of_pos) {
  const int f = blockIdx.y, j = blockIdx.z;
  const int sys = j * a.n_f + f;
  const int blk = blk_of_pos ? blk_of_pos[j] : j;
  const DomInst* d = bd.inst_tab + bd.inst[j];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d->nsites) return;
  const int gx = d->glob[k];
  int g[4];
  site_coords(gx, a.L, g);
  double2 acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = make_double2(0.0, 0.0);
  for (int dir = 0; dir < 8; ++dir) {
    const int mu = dir & 3, step = dir < 4 ? 1 : -1;
    int gy[4] = {g[0], g[1], g[2], g[3]};
    gy[mu] = (g[mu] + step + a.L[mu]) % a.L[mu];
    const int y = glob_index(gy, a.L);
    const int q = a.dpi_pos[y];
    if (q < 0 || dpi_kind[q] != blk) continue;        // not a boundary site of this core
    add_exterior_hop(acc, dir, gx, y, a, f);
  }
  double2* out = a.src + bd.uoff[sys] + 12LL * d->fmap[k];
#pragma unroll
  for (int c = 0; c < 12; ++c) out[c] = make_double2(-a.kappa * acc[c].x, -a.kappa * acc[c].y);
}

// On every dPi1 site x and field f: q = (Q chi)(x), the sum of the frame-piece
// solutions Y_b(x) over the pieces that hold x (in block order), then
// chi'(x) = chi(x) - q and, with the frame solved in the same batch (position
// frame_pos), (w chi)(x) = q - y(x).
__global__ void k_frame_q(const int* __restrict__ q_beg, const int* __restrict__ q_blk,
                          const long long* __restrict__ q_loc, const long long* __restrict__ c_loc,
                          const int* __restrict__ c_dpi, int nC, int n_f, int n_dpi, int frame_pos,
                          const long long* __restrict__ uoff, const double2* __restrict__ sol,
                          const double2* __restrict__ chi, double2* __restrict__ chi_p,
                          double2* __restrict__ w, const int* __restrict__ pos_of_blk,
                          double2* __restrict__ q_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= nC) return;
  double2 q[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) q[c] = make_double2(0.0, 0.0);
  for (int e = q_beg[k]; e < q_beg[k + 1]; ++e) {
    const int pos = pos_of_blk ? pos_of_blk[q_blk[e]] : q_blk[e];
    if (pos < 0) continue;                     // a frame piece outside this batch
    const double2* s = sol + uoff[(long long)pos * n_f + f] + q_loc[e];
#pragma unroll
    for (int c = 0; c < 12; ++c) q[c] = make_double2(q[c].x + s[c].x, q[c].y + s[c].y);
  }
  const long long o = ((long long)f * n_dpi + c_dpi[k]) * 12;
  if (q_out) {                                 // Q chi of the batch's frame pieces only
#pragma unroll
    for (int c = 0; c < 12; ++c) q_out[o + c] = q[c];
    return;
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) chi_p[o + c] = make_double2(chi[o + c].x - q[c].x, chi[o + c].y - q[c].y);
  if (w) {
    const double2* y = sol + uoff[(long long)frame_pos * n_f + f] + c_loc[k];
#pragma unroll
    for (int c = 0; c < 12; ++c) w[o + c] = make_double2(q[c].x - y[c].x, q[c].y - y[c].y);
  }
}

// (w chi) on dLambda0: -x at the block-boundary sites; on dPi1: -y.  For
// every listed site: its system's instance in the batch (a block, or the
// frame at position nblocks), its offset
// inside the system's caller-layout solution and its dPi index.
__global__ void k_extract(const int* __restrict__ sys_blk, int blk_fixed, const long long* __restrict__ loc,
                          const int* __restrict__ dpi_idx, int n, int n_f, int n_dpi,
                          const long long* __restrict__ uoff, const double2* __restrict__ sol,
                          double2* __restrict__ w, const int* __restrict__ pos_of_blk) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= n) return;
  int blk = sys_blk ? sys_blk[k] : blk_fixed;
  if (sys_blk && pos_of_blk) {
    blk = pos_of_blk[blk];
    if (blk < 0) return;                       // a block outside this batch
  }
  const double2* s = sol + uoff[(long long)blk * n_f + f] + loc[k];
  double2* o = w + ((long long)f * n_dpi + dpi_idx[k]) * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) o[c] = make_double2(-s[c].x, -s[c].y);
}

// S^a (one CTA per block) and partial S^r over the dPi1 sites.
__global__ void k_action_blocks(const int* __restrict__ grp_begin, const int* __restrict__ dpi_idx,
                                int n_f, int n_dpi, const double2* __restrict__ u,
                                const double2* __restrict__ chi, const double2* __restrict__ w,
                                double* out) {
  __shared__ double red[32];
  const int a = blockIdx.x;
  double acc[1] = {0.0};
  for (int f = 0; f < n_f; ++f) {
    const double2 uk = u[f];
    for (int k = grp_begin[a] + threadIdx.x; k < grp_begin[a + 1]; k += blockDim.x) {
      const long long base = ((long long)f * n_dpi + dpi_idx[k]) * 12;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const double2 x = chi[base + c], y = w[base + c];
        const double re = uk.x * x.x - uk.y * x.y - y.x;
        const double im = uk.x * x.y + uk.y * x.x - y.y;
        acc[0] += re * re + im * im;
      }
    }
  }
  block_reduce<1>(acc, red);
  if (threadIdx.x == 0) out[a] = acc[0];
}

// ---- heat-bath of the multi-boson fields: BLAS-1 on dPi vectors [f][n] ---------
// y_f = u_f x_f - wx_f (the operator W_u = u - w applied through w)
__global__ void k_hb_wu(int n_f, long long n, const double2* __restrict__ u, const double2* __restrict__ x,
                        const double2* __restrict__ wx, double2* __restrict__ y) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= n) return;
  const long long o = (long long)f * n + k;
  const double2 a = x[o], b = wx[o], uf = u[f];
  y[o] = make_double2(uf.x * a.x - uf.y * a.y - b.x, uf.x * a.y + uf.y * a.x - b.y);
}
// y_f = c1_f x1_f + c2_f x2_f + c3_f x3_f (any x may be null), for fields with active[f]
__global__ void k_hb_lin(int n_f, long long n, const int* __restrict__ active, const double2* __restrict__ c,
                         const double2* x1, const double2* x2, const double2* x3, double2* y) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= n || (active && !active[f])) return;
  const long long o = (long long)f * n + k;
  double2 acc = make_double2(0.0, 0.0);
  const double2* xs[3] = {x1, x2, x3};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    if (!xs[m]) continue;
    const double2 cf = c[3 * f + m], v = xs[m][o];
    acc.x += cf.x * v.x - cf.y * v.y;
    acc.y += cf.x * v.y + cf.y * v.x;
  }
  y[o] = acc;
}
// per-field partial sums of conj(a) . b over fixed chunks (grid (nchunk, n_f), 256 threads)
__global__ void k_hb_dot(long long n, const double2* __restrict__ a, const double2* __restrict__ b,
                         double* __restrict__ partial) {
  __shared__ double red[64];
  const int f = blockIdx.y;
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long k0 = blockIdx.x * chunk, k1 = min(n, k0 + chunk);
  double acc[2] = {0.0, 0.0};
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double2 x = a[(long long)f * n + k], y = b[(long long)f * n + k];
    acc[0] += x.x * y.x + x.y * y.y;
    acc[1] += x.x * y.y - x.y * y.x;
  }
  block_reduce<2>(acc, red);
  if (threadIdx.x == 0) {
    partial[2 * ((long long)f * gridDim.x + blockIdx.x)] = acc[0];
    partial[2 * ((long long)f * gridDim.x + blockIdx.x) + 1] = acc[1];
  }
}

}  // namespace

// ---------------------------------------------------------------------------

// ---- force of the factorized multi-boson action on the active links ----------
// rhs of the adjoint solves: gamma_5 P_{dLambda0^a}(u_f chi_f + y_f) at the B sites
// of every block (the buffer is zero elsewhere); D_Omega^dag = gamma_5 D_Omega gamma_5
__global__ void k_force_rhs(const int* __restrict__ b_blk, const long long* __restrict__ b_loc,
                            const int* __restrict__ b_dpi, int nB, int n_f, int n_dpi,
                            const long long* __restrict__ uoff, const double2* __restrict__ u,
                            const double2* __restrict__ chi, const double2* __restrict__ y,
                            double2* __restrict__ rhs) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (k >= nB) return;
  const long long o = uoff[(long long)b_blk[k] * n_f + f] + b_loc[k];
  const double2* c = chi + ((long long)f * n_dpi + b_dpi[k]) * 12;
  const double2 uf = u[f];
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    const double2 x = c[e], yv = y[o + e];
    double2 r = make_double2(uf.x * x.x - uf.y * x.y + yv.x, uf.x * x.y + uf.y * x.x + yv.y);
    if (e >= 6) r = make_double2(-r.x, -r.y);
    rhs[o + e] = r;
  }
}

// half spinors: with P = 1 -/+ gamma_mu (P^2 = 2P, the lower two spins of P psi a
// unitary recombination of the upper two), a^dag P b = sum_{s=0,1} h_s(a)^dag h_s(b)
// for h = the upper half of P psi (hop_project).  So
//   z(x)^dag [P_fwd (x) T U] y(x+mu)   = sum_s h_s(z(x))^dag T U h_s(y(x+mu))
//   z(x+mu)^dag [P_bwd (x) U^dag T] y(x) = sum_s (U h_s(z(x+mu)))^dag T h_s(y(x))
template <int MU>
__device__ __forceinline__ void force_link(const double2 (&U)[9], const double2* __restrict__ yx,
                                           const double2* __restrict__ yxp, const double2* __restrict__ zx,
                                           const double2* __restrict__ zxp, double2 (&N)[9]) {
  double2 v[12], hy[2][3], hz[2][3];
  // N -= sum_s conj(h_s(z(x)))_a (U h_s(y(x+mu)))_b
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = yxp[c];
  hop_project<MU, true>(v, hy);
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = c >= 6 ? make_double2(-zx[c].x, -zx[c].y) : zx[c];
  hop_project<MU, true>(v, hz);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    double2 uh[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      uh[a] = make_double2(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) cfma(uh[a], U[a * 3 + b], hy[sp][b]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double2 zc = hz[sp][a], qb = uh[b];
        N[a * 3 + b].x -= zc.x * qb.x + zc.y * qb.y;
        N[a * 3 + b].y -= zc.x * qb.y - zc.y * qb.x;
      }
  }
  // N += sum_s conj(U h_s(z(x+mu)))_a h_s(y(x))_b
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = yx[c];
  hop_project<MU, false>(v, hy);
#pragma unroll
  for (int c = 0; c < 12; ++c) v[c] = c >= 6 ? make_double2(-zxp[c].x, -zxp[c].y) : zxp[c];
  hop_project<MU, false>(v, hz);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    double2 uz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      uz[a] = make_double2(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) cfma(uz[a], U[a * 3 + b], hz[sp][b]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double2 pc = uz[a], rb = hy[sp][b];
        N[a * 3 + b].x += pc.x * rb.x + pc.y * rb.y;
        N[a * 3 + b].y += pc.x * rb.y - pc.y * rb.x;
      }
  }
}

// one thread per active link: F_t = 2 kappa Im sum_ab (T_t)_ab N_ab summed over the
// fields, N = sum_f [ conj(U h(z(x+mu))) (x) h(y(x)) - conj(h(z(x))) (x) U h(y(x+mu)) ]
// (half spinors of the backward / forward projectors, see force_link), T_t = lambda_t/2,
// z = gamma_5 times the solution of the gamma_5-rotated adjoint system
__global__ void __launch_bounds__(128) k_mb_force(const int4* __restrict__ al, const long long* __restrict__ al_loc, long long n_al,
                           int n_f, const long long* __restrict__ uoff, const double2* __restrict__ gU,
                           const double2* __restrict__ y, const double2* __restrict__ zg, double kappa,
                           double* __restrict__ F, int accumulate) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_al) return;
  const int4 e = al[k];
  const int blk = e.x, xg = e.y, mu = e.z;
  double2 U[9];
  const double2* lp = gU + (long long)xg * 36 + mu * 9;
#pragma unroll
  for (int m = 0; m < 9; ++m) U[m] = lp[m];
  double2 N[9];
#pragma unroll
  for (int m = 0; m < 9; ++m) N[m] = make_double2(0.0, 0.0);
  for (int f = 0; f < n_f; ++f) {
    const long long base = uoff[(long long)blk * n_f + f];
    const long long ox = base + al_loc[2 * k], oxp = base + al_loc[2 * k + 1];
    switch (mu) {
      case 0: force_link<0>(U, y + ox, y + oxp, zg + ox, zg + oxp, N); break;
      case 1: force_link<1>(U, y + ox, y + oxp, zg + ox, zg + oxp, N); break;
      case 2: force_link<2>(U, y + ox, y + oxp, zg + ox, zg + oxp, N); break;
      default: force_link<3>(U, y + ox, y + oxp, zg + ox, zg + oxp, N); break;
    }
  }
  double* o = F + ((long long)xg * 4 + mu) * 8;
  const double h = kappa;            // 2 kappa * (1/2 of lambda)
  double f[8];
  f[0] = h * (N[1].y + N[3].y);
  f[1] = h * (N[3].x - N[1].x);
  f[2] = h * (N[0].y - N[4].y);
  f[3] = h * (N[2].y + N[6].y);
  f[4] = h * (N[6].x - N[2].x);
  f[5] = h * (N[5].y + N[7].y);
  f[6] = h * (N[7].x - N[5].x);
  f[7] = h * (N[0].y + N[4].y - 2.0 * N[8].y) / sqrt(3.0);
  // each active link has one thread, so adding onto F needs no atomics
#pragma unroll
  for (int t = 0; t < 8; ++t) o[t] = accumulate ? o[t] + f[t] : f[t];
}

// v -> gamma_5 v on caller-layout spinors (components 6..11 of a site change sign)
__global__ void k_gamma5(long long n, const double2* __restrict__ in, double2* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double2 v = in[k];
  out[k] = (k % 12) >= 6 ? make_double2(-v.x, -v.y) : v;
}

__global__ void k_scale(long long n, double a, double* __restrict__ v) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[k] *= a;
}

struct WPlan {           // host-built gather lists, one per context
  int n_l1 = 0;
  int* d_l1_glob = nullptr;          // [n_l1] global site of Lambda1 field index
  unsigned char* d_in_l1 = nullptr;  // [V]
  int* d_b_blk = nullptr;            // [n_B] block of the B site (grouped by block)
  long long* d_b_loc = nullptr;      // [n_B] 12 * field position inside Omega0^b
  int* d_b_dpi = nullptr;            // [n_B] dPi index
  int* d_b_grp = nullptr;            // [nblocks + 1] group boundaries
  long long* d_c_loc = nullptr;      // [n_C] 12 * field position inside Lambda1
  int* d_c_dpi = nullptr;            // [n_C]
  int* d_c_grp = nullptr;            // C sites split into chunks for the S^r partials
  int n_cgrp = 0;
  // Q chi on dPi1 (built with the frame pieces on first use): for every dPi1
  // site (C order) the frame pieces Phi1^b holding it and its field position there
  bool q_ready = false;
  int* d_q_beg = nullptr;            // [n_C + 1]
  int* d_q_blk = nullptr;            // [n_q] block b
  long long* d_q_loc = nullptr;      // [n_q] 12 * field position inside Phi1^b
  int max_phi = 0;
  // active links (both end points in one core), built on the first force call
  bool force_ready = false;
  long long n_al = 0;
  int4* d_al = nullptr;              // [n_al] (block, global site x, mu, unused)
  long long* d_al_loc = nullptr;     // [n_al][2] 12 * field position of x, x + mu in Omega0^b
};

void free_plan(dd_ctx* c) {
  WPlan* P = (WPlan*)c->wplan;
  if (!P) return;
  dfree(P->d_l1_glob); dfree(P->d_in_l1); dfree(P->d_b_blk); dfree(P->d_b_loc);
  dfree(P->d_b_dpi); dfree(P->d_b_grp); dfree(P->d_c_loc); dfree(P->d_c_dpi); dfree(P->d_c_grp);
  dfree(P->d_al); dfree(P->d_al_loc);
  dfree(P->d_q_beg); dfree(P->d_q_blk); dfree(P->d_q_loc);
  delete P;
  c->wplan = nullptr;
}

static dd_status build_plan(dd_ctx* c, WPlan** out) {
  if (c->wplan) {
    *out = (WPlan*)c->wplan;
    return DD_OK;
  }
  WPlan* P = new WPlan();
  c->wplan = P;
  const int V = c->V, nb = (int)c->blocks.size();
  dd_status e;
  const Instance& l1 = c->inst[c->lambda1];
  std::vector<int> l1_glob(l1.d.nsites);
  for (int k = 0; k < l1.d.nsites; ++k) l1_glob[l1.h_fmap[k]] = l1.h_glob[k];
  std::vector<unsigned char> in_l1(V, 0);
  std::vector<int> l1_pos(V, -1);
  for (int k = 0; k < (int)l1_glob.size(); ++k) {
    in_l1[l1_glob[k]] = 1;
    l1_pos[l1_glob[k]] = k;
  }
  std::vector<int> b_blk, b_dpi, b_grp(1, 0);
  std::vector<long long> b_loc;
  std::vector<int> fpos(V, -1);
  for (int b = 0; b < nb; ++b) {
    const Instance& om = c->inst[c->omega0 + b];
    for (int k = 0; k < om.d.nsites; ++k) fpos[om.h_glob[k]] = om.h_fmap[k];
    for (int s : c->B_of_block[b]) {
      b_blk.push_back(b);
      b_loc.push_back(12LL * fpos[s]);
      b_dpi.push_back(c->dpi_pos[s]);
    }
    for (int k = 0; k < om.d.nsites; ++k) fpos[om.h_glob[k]] = -1;
    b_grp.push_back((int)b_loc.size());
  }
  std::vector<long long> c_loc;
  std::vector<int> c_dpi, c_grp(1, 0);
  for (int s : c->C_sites) {
    c_loc.push_back(12LL * l1_pos[s]);
    c_dpi.push_back(c->dpi_pos[s]);
  }
  const int CG = 4096;
  for (int k = CG; k < (int)c_loc.size(); k += CG) c_grp.push_back(k);
  c_grp.push_back((int)c_loc.size());
  auto up = [&](auto& vec, auto** dst) -> dd_status {
    size_t bytes = sizeof(vec[0]) * std::max<size_t>(1, vec.size());
    dd_status st = dalloc(c, (void**)dst, bytes);
    if (st != DD_OK) return st;
    if (!vec.empty())
      cudaMemcpy(*dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice);
    return DD_OK;
  };
  if ((e = up(l1_glob, &P->d_l1_glob)) || (e = up(in_l1, &P->d_in_l1)) ||
      (e = up(b_blk, &P->d_b_blk)) || (e = up(b_loc, &P->d_b_loc)) || (e = up(b_dpi, &P->d_b_dpi)) ||
      (e = up(b_grp, &P->d_b_grp)) || (e = up(c_loc, &P->d_c_loc)) || (e = up(c_dpi, &P->d_c_dpi)) ||
      (e = up(c_grp, &P->d_c_grp))) {
    free_plan(c);
    return e;
  }
  P->n_l1 = (int)l1_glob.size();
  P->n_cgrp = (int)c_grp.size() - 1;
  *out = P;
  return DD_OK;
}

// gather lists of Q: the frame pieces holding each dPi1 site
static dd_status build_q_plan(dd_ctx* c, WPlan& P) {
  if (P.q_ready) return DD_OK;
  dd_status e;
  if ((e = ensure_phi(c)) != DD_OK) return e;
  const int nb = (int)c->blocks.size(), nC = (int)c->C_sites.size();
  std::vector<int> c_index(c->V, -1);
  for (int k = 0; k < nC; ++k) c_index[c->C_sites[k]] = k;
  std::vector<std::vector<std::pair<int, long long>>> per(nC);
  int max_phi = 0;
  for (int b = 0; b < nb; ++b) {
    const Instance& ph = c->inst[c->phi0 + b];
    max_phi = std::max(max_phi, ph.d.nsites);
    for (int k = 0; k < ph.d.nsites; ++k) {
      const int ci = c_index[ph.h_glob[k]];
      if (ci >= 0) per[ci].push_back({b, 12LL * ph.h_fmap[k]});
    }
  }
  std::vector<int> beg(1, 0), blk;
  std::vector<long long> loc;
  for (int k = 0; k < nC; ++k) {
    for (auto& pr : per[k]) {          // blocks in increasing order: fixed summation order
      blk.push_back(pr.first);
      loc.push_back(pr.second);
    }
    beg.push_back((int)blk.size());
  }
  auto up = [&](auto& vec, auto** dst) -> dd_status {
    size_t bytes = sizeof(vec[0]) * std::max<size_t>(1, vec.size());
    dd_status st = dalloc(c, (void**)dst, bytes);
    if (st != DD_OK) return st;
    if (!vec.empty()) cudaMemcpy(*dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice);
    return DD_OK;
  };
  if ((e = up(beg, &P.d_q_beg)) || (e = up(blk, &P.d_q_blk)) || (e = up(loc, &P.d_q_loc))) return e;
  P.max_phi = max_phi;
  P.q_ready = true;
  return DD_OK;
}

// merged statistics of two batched solves of one call
static void merge_stats(dd_solve_stats& a, const dd_solve_stats& b) {
  a.systems += b.systems;
  a.converged += b.converged;
  a.max_iters = std::max(a.max_iters, b.max_iters);
  a.outer_cycles = std::max(a.outer_cycles, b.outer_cycles);
  a.max_relres = std::max(a.max_relres, b.max_relres);
  a.seconds += b.seconds;
}

// Stage A of w (see the top of the file): the frame pieces of every block (and
// with with_frame the frame Lambda1) in one batch, then chi' = chi - Q chi on dPi1
// (chi' = chi elsewhere) and, with the frame, (w chi)_{dPi1} = Q chi - y.
static dd_status frame_stage(dd_ctx* c, WPlan& P, int n_f, const double* chi, double* chi_p, double* wchi,
                             bool with_frame, const dd_solve_params* prm, dd_solve_stats* st,
                             cudaStream_t s) {
  dd_status e;
  if ((e = build_q_plan(c, P)) != DD_OK) return e;
  const int nb = (int)c->blocks.size();
  std::vector<int> insts(nb + (with_frame ? 1 : 0));
  for (int b = 0; b < nb; ++b) insts[b] = c->phi0 + b;
  if (with_frame) insts[nb] = c->lambda1;
  Batch* ab;
  if ((e = get_batch_insts(c, insts, n_f, &ab)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  void *src_a, *sol_a;
  if ((e = workspace(c, 36, 16ULL * ab->user_tot, &src_a)) || (e = workspace(c, 37, 16ULL * ab->user_tot, &sol_a)))
    return e;
  InjectArgs a;
  a.U = c->d_U;
  a.chi = (const double2*)chi;
  a.dpi_pos = c->d_dpi_pos;
  for (int m = 0; m < 4; ++m) a.L[m] = c->L[m];
  a.n_dpi = c->info.n_dpi;
  a.n_f = n_f;
  a.kappa = c->kappa;
  a.src = (double2*)src_a;
  BatchDev bd = batch_view(c, *ab);
  dim3 g1((P.max_phi + 127) / 128, n_f, nb);
  DD_COUNT_LAUNCH(), k_inject_phi<<<g1, 128, 0, s>>>(bd, a, c->d_dpi_kind, nullptr);
  if (with_frame) {
    long long phi_user = 0;
    for (int b = 0; b < nb; ++b) phi_user += 12LL * c->inst[c->phi0 + b].d.nsites * n_f;
    a.src = (double2*)src_a + phi_user;
    dim3 g2((P.n_l1 + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_inject_frame<<<g2, 128, 0, s>>>(P.d_l1_glob, P.n_l1, P.d_in_l1, a);
  }
  DD_CUDA(c, cudaGetLastError());
  dd_status r = solve_batch(c, *ab, (const double*)src_a, (double*)sol_a, prm, st, s, true);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  const size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  DD_CUDA(c, cudaMemcpyAsync(chi_p, chi, bytes, cudaMemcpyDeviceToDevice, s));
  const int nC = c->info.n_C;
  if (nC) {
    dim3 g((nC + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_frame_q<<<g, 128, 0, s>>>(P.d_q_beg, P.d_q_blk, P.d_q_loc, P.d_c_loc, P.d_c_dpi, nC, n_f,
                                                   c->info.n_dpi, nb, ab->d_uoff, (const double2*)sol_a,
                                                   (const double2*)chi, (double2*)chi_p,
                                                   with_frame ? (double2*)wchi : nullptr, nullptr, nullptr);
    DD_CUDA(c, cudaGetLastError());
  }
  return r;
}

// active links of every block: (x, mu) with x and x + mu both in the core
// Lambda0^b (cores are intervals that do not wrap, except an undecomposed
// direction's virtual core spanning the whole periodic extent)
static dd_status build_force_plan(dd_ctx* c, WPlan& P) {
  if (P.force_ready) return DD_OK;
  const int* L = c->L;
  const int nb = (int)c->blocks.size();
  std::vector<int4> al;
  std::vector<long long> loc;
  std::vector<int> fpos(c->V, -1);
  for (int b = 0; b < nb; ++b) {
    const Instance& om = c->inst[c->omega0 + b];
    for (int k = 0; k < om.d.nsites; ++k) fpos[om.h_glob[k]] = om.h_fmap[k];
    const BlockDesc& bd = c->blocks[b];
    auto in_core = [&](int m, int v) { return v >= bd.core_lo[m] && v <= bd.core_hi[m]; };
    int x[4];
    for (x[0] = bd.core_lo[0]; x[0] <= bd.core_hi[0]; ++x[0])
      for (x[1] = bd.core_lo[1]; x[1] <= bd.core_hi[1]; ++x[1])
        for (x[2] = bd.core_lo[2]; x[2] <= bd.core_hi[2]; ++x[2])
          for (x[3] = bd.core_lo[3]; x[3] <= bd.core_hi[3]; ++x[3]) {
            const int gx = ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3];
            for (int mu = 0; mu < 4; ++mu) {
              int y[4] = {x[0], x[1], x[2], x[3]};
              y[mu] = (y[mu] + 1) % L[mu];
              if (!in_core(mu, y[mu])) continue;
              const int gy = ((y[0] * L[1] + y[1]) * L[2] + y[2]) * L[3] + y[3];
              if (fpos[gx] < 0 || fpos[gy] < 0) return fail(c, DD_EINVAL, "core site outside its block");
              al.push_back(make_int4(b, gx, mu, 0));
              loc.push_back(12LL * fpos[gx]);
              loc.push_back(12LL * fpos[gy]);
            }
          }
    for (int k = 0; k < om.d.nsites; ++k) fpos[om.h_glob[k]] = -1;
  }
  dd_status e;
  if ((e = dalloc(c, (void**)&P.d_al, sizeof(int4) * std::max<size_t>(1, al.size()))) ||
      (e = dalloc(c, (void**)&P.d_al_loc, sizeof(long long) * std::max<size_t>(1, loc.size()))))
    return e;
  if (!al.empty()) {
    DD_CUDA(c, cudaMemcpy(P.d_al, al.data(), sizeof(int4) * al.size(), cudaMemcpyHostToDevice));
    DD_CUDA(c, cudaMemcpy(P.d_al_loc, loc.data(), sizeof(long long) * loc.size(), cudaMemcpyHostToDevice));
  }
  P.n_al = (long long)al.size();
  P.force_ready = true;
  return DD_OK;
}

// w chi for n_f fields (device pointers, caller layout on dPi): stage A (frame
// pieces and frame, skipped without dPi1), stage B (framed blocks on chi').
static dd_status apply_w_dev(dd_ctx* c, int n_f, const double* chi, double* wchi,
                             const dd_solve_params* prm, cudaStream_t s) {
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  const int nb = (int)c->blocks.size();
  dd_status e;
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  bool noconv = false;
  dd_solve_stats tot{};
  const double* chi_b = chi;
  if (c->info.n_C > 0) {
    void* cp;
    if ((e = workspace(c, 42, 16ULL * n_f * c->info.n_dpi * 12, &cp)) != DD_OK) return e;
    dd_solve_stats sa{};
    dd_status ra = frame_stage(c, P, n_f, chi, (double*)cp, wchi, true, prm, &sa, s);
    if (ra == DD_ENOCONV) noconv = true;
    else if (ra != DD_OK) return ra;
    merge_stats(tot, sa);
    chi_b = (const double*)cp;
  }
  // stage B: every framed block Omega0^a, n_f fields each, sources from chi'
  std::vector<int> insts(nb);
  for (int b = 0; b < nb; ++b) insts[b] = c->omega0 + b;
  Batch* ob;
  if ((e = get_batch_insts(c, insts, n_f, &ob)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  void *src_o, *sol_o;
  if ((e = workspace(c, 40, 16ULL * ob->user_tot, &src_o)) ||
      (e = workspace(c, 41, 16ULL * ob->user_tot, &sol_o)))
    return e;
  InjectArgs a;
  a.U = c->d_U;
  a.chi = (const double2*)chi_b;
  a.dpi_pos = c->d_dpi_pos;
  for (int m = 0; m < 4; ++m) a.L[m] = c->L[m];
  a.n_dpi = c->info.n_dpi;
  a.n_f = n_f;
  a.kappa = c->kappa;
  a.src = (double2*)src_o;
  BatchDev bd = batch_view(c, *ob);
  dim3 g1((c->info.max_omega + 127) / 128, n_f, nb);
  DD_COUNT_LAUNCH(), k_inject_omega<<<g1, 128, 0, s>>>(bd, a);
  DD_CUDA(c, cudaGetLastError());
  dd_solve_stats sb{};
  dd_status rb = solve_batch(c, *ob, (const double*)src_o, (double*)sol_o, prm, &sb, s, true);
  if (rb == DD_ENOCONV) noconv = true;
  else if (rb != DD_OK) return rb;
  merge_stats(tot, sb);
  c->last_stats = tot;
  // extraction into w chi on dLambda0 (dPi1 was written by stage A)
  const int nB = c->info.n_B;
  if (nB) {
    dim3 g((nB + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_extract<<<g, 128, 0, s>>>(P.d_b_blk, 0, P.d_b_loc, P.d_b_dpi, nB, n_f,
                                                   c->info.n_dpi, ob->d_uoff, (const double2*)sol_o,
                                                   (double2*)wchi, nullptr);
  }
  DD_CUDA(c, cudaGetLastError());
  if (noconv) return fail(c, DD_ENOCONV, "a block, frame-piece or frame solve missed its tolerance");
  return DD_OK;
}

// One stage of w for a subset of blocks (dd_apply_w_part): the pieces a rank
// that owns some of the blocks computes.  Writes only the entries of its stage.
static dd_status apply_w_part_dev(dd_ctx* c, int part, int n_f, const int* ids, int nblk, const double* in,
                                  double* out, const dd_solve_params* prm, cudaStream_t s) {
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  const int nb = (int)c->blocks.size();
  dd_status e;
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  std::vector<int> pos(nb, -1), blk;
  if (part != DD_W_FRAME) {
    if (!ids || nblk < 1 || nblk > nb) return fail(c, DD_EINVAL, "block list required");
    for (int k = 0; k < nblk; ++k) {
      if (ids[k] < 0 || ids[k] >= nb || pos[ids[k]] >= 0) return fail(c, DD_EINVAL, "bad or repeated block id");
      pos[ids[k]] = k;
      blk.push_back(ids[k]);
    }
  }
  InjectArgs a;
  a.U = c->d_U;
  a.chi = (const double2*)in;
  a.dpi_pos = c->d_dpi_pos;
  for (int m = 0; m < 4; ++m) a.L[m] = c->L[m];
  a.n_dpi = c->info.n_dpi;
  a.n_f = n_f;
  a.kappa = c->kappa;
  std::vector<int> insts;
  if (part == DD_W_FRAME_Q) {
    if ((e = build_q_plan(c, P)) != DD_OK) return e;
    for (int b : blk) insts.push_back(c->phi0 + b);
  } else if (part == DD_W_BLOCKS) {
    for (int b : blk) insts.push_back(c->omega0 + b);
  } else if (part == DD_W_FRAME) {
    insts.push_back(c->lambda1);
  } else {
    return fail(c, DD_EINVAL, "unknown stage of w");
  }
  Batch* bt;
  if ((e = get_batch_insts(c, insts, n_f, &bt)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  void *src, *sol, *dmap;
  if ((e = workspace(c, 36, 16ULL * bt->user_tot, &src)) || (e = workspace(c, 37, 16ULL * bt->user_tot, &sol)) ||
      (e = workspace(c, 43, sizeof(int) * (2 * nb + 2), &dmap)))
    return e;
  int* d_pos = (int*)dmap;
  int* d_blk = d_pos + nb + 1;
  if (part != DD_W_FRAME) {
    DD_CUDA(c, cudaMemcpyAsync(d_pos, pos.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    DD_CUDA(c, cudaMemcpyAsync(d_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice, s));
  }
  a.src = (double2*)src;
  BatchDev bd = batch_view(c, *bt);
  if (part == DD_W_FRAME_Q) {
    dim3 g1((P.max_phi + 127) / 128, n_f, nblk);
    DD_COUNT_LAUNCH(), k_inject_phi<<<g1, 128, 0, s>>>(bd, a, c->d_dpi_kind, d_blk);
  } else if (part == DD_W_BLOCKS) {
    dim3 g1((c->info.max_omega + 127) / 128, n_f, nblk);
    DD_COUNT_LAUNCH(), k_inject_omega<<<g1, 128, 0, s>>>(bd, a);
  } else {
    dim3 g2((P.n_l1 + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_inject_frame<<<g2, 128, 0, s>>>(P.d_l1_glob, P.n_l1, P.d_in_l1, a);
  }
  DD_CUDA(c, cudaGetLastError());
  dd_solve_stats st{};
  dd_status r = solve_batch(c, *bt, (const double*)src, (double*)sol, prm, &st, s, true);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  const int nB = c->info.n_B, nC = c->info.n_C;
  if (part == DD_W_FRAME_Q && nC) {
    dim3 g((nC + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_frame_q<<<g, 128, 0, s>>>(P.d_q_beg, P.d_q_blk, P.d_q_loc, P.d_c_loc, P.d_c_dpi, nC, n_f,
                                                   c->info.n_dpi, -1, bt->d_uoff, (const double2*)sol, nullptr,
                                                   nullptr, nullptr, d_pos, (double2*)out);
  } else if (part == DD_W_BLOCKS && nB) {
    dim3 g((nB + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_extract<<<g, 128, 0, s>>>(P.d_b_blk, 0, P.d_b_loc, P.d_b_dpi, nB, n_f, c->info.n_dpi,
                                                   bt->d_uoff, (const double2*)sol, (double2*)out, d_pos);
  } else if (part == DD_W_FRAME && nC) {
    dim3 g((nC + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_extract<<<g, 128, 0, s>>>(nullptr, 0, P.d_c_loc, P.d_c_dpi, nC, n_f, c->info.n_dpi,
                                                   bt->d_uoff, (const double2*)sol, (double2*)out, nullptr);
  }
  DD_CUDA(c, cudaGetLastError());
  if (r == DD_ENOCONV) return fail(c, DD_ENOCONV, "a solve of this stage missed its tolerance");
  return DD_OK;
}

// Heat-bath of the multi-boson fields (paper Sec. 4): chi_f = W_{u_f}^{-1} eta_f on
// dPi for every field f, by BiCGstab (van der Vorst 1992) over all fields at
// once; each matvec is one dd_apply_w batch (every block and frame solve of all
// fields) followed by u chi - w chi.  The start chi = eta / u is already close
// (w is small where the frame is thick).  Per-field scalars live on the host
// (the matvecs dominate); inner products are summed in a fixed order.
static constexpr int HB_CHUNKS = 64;

static dd_status hb_dot(dd_ctx* c, int n_f, long long n, const double2* a, const double2* b, double* dpart,
                        std::vector<double2>& out, cudaStream_t s) {
  DD_COUNT_LAUNCH(), k_hb_dot<<<dim3(HB_CHUNKS, n_f), 256, 0, s>>>(n, a, b, dpart);
  DD_CUDA(c, cudaGetLastError());
  std::vector<double> h(2 * (size_t)n_f * HB_CHUNKS);
  DD_CUDA(c, cudaMemcpyAsync(h.data(), dpart, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  out.assign(n_f, make_double2(0.0, 0.0));
  for (int f = 0; f < n_f; ++f)
    for (int k = 0; k < HB_CHUNKS; ++k) {
      out[f].x += h[2 * ((size_t)f * HB_CHUNKS + k)];
      out[f].y += h[2 * ((size_t)f * HB_CHUNKS + k) + 1];
    }
  return DD_OK;
}

static double2 zdiv_h(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
static double2 zmul_h(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

static dd_status heatbath_dev(dd_ctx* c, int n_f, const double2* u_h, const double2* eta, double2* x,
                              double tol, int maxiter, const dd_solve_params* prm, dd_heatbath_stats* out,
                              cudaStream_t s) {
  const long long n = 12LL * c->info.n_dpi;
  const size_t vb = sizeof(double2) * (size_t)n_f * n;
  void *vr, *vrh, *vp, *vv, *vs, *vt, *vw, *vu, *vc, *va, *vpart;
  dd_status e;
  if ((e = workspace(c, 200, vb, &vr)) || (e = workspace(c, 201, vb, &vrh)) || (e = workspace(c, 202, vb, &vp)) ||
      (e = workspace(c, 203, vb, &vv)) || (e = workspace(c, 204, vb, &vs)) || (e = workspace(c, 205, vb, &vt)) ||
      (e = workspace(c, 206, vb, &vw)) || (e = workspace(c, 207, sizeof(double2) * n_f, &vu)) ||
      (e = workspace(c, 208, sizeof(double2) * 3 * n_f, &vc)) || (e = workspace(c, 209, sizeof(int) * n_f, &va)) ||
      (e = workspace(c, 210, sizeof(double) * 2 * n_f * HB_CHUNKS, &vpart)))
    return e;
  double2 *r = (double2*)vr, *rh = (double2*)vrh, *p = (double2*)vp, *v = (double2*)vv, *sv = (double2*)vs,
          *t = (double2*)vt, *wx = (double2*)vw, *du = (double2*)vu, *dc = (double2*)vc;
  int* dact = (int*)va;
  double* dpart = (double*)vpart;
  const dim3 grid((unsigned)((n + 255) / 256), n_f);
  EventPair evs;
  cudaEvent_t e0 = evs.a, e1 = evs.b;
  cudaEventRecord(e0, s);
  DD_CUDA(c, cudaMemcpyAsync(du, u_h, sizeof(double2) * n_f, cudaMemcpyHostToDevice, s));
  std::vector<double2> cf(3 * n_f);
  std::vector<int> act(n_f, 1);
  auto set_coef = [&](const std::vector<double2>& c3) -> dd_status {
    DD_CUDA(c, cudaMemcpyAsync(dc, c3.data(), sizeof(double2) * 3 * n_f, cudaMemcpyHostToDevice, s));
    DD_CUDA(c, cudaMemcpyAsync(dact, act.data(), sizeof(int) * n_f, cudaMemcpyHostToDevice, s));
    return DD_OK;
  };
  int matvecs = 0;
  // y = W_u z
  auto matvec = [&](const double2* z, double2* y) -> dd_status {
    dd_status r0 = apply_w_dev(c, n_f, (const double*)z, (double*)wx, prm, s);
    if (r0 != DD_OK) return r0;
    DD_COUNT_LAUNCH(), k_hb_wu<<<grid, 256, 0, s>>>(n_f, n, du, z, wx, y);
    DD_CUDA(c, cudaGetLastError());
    ++matvecs;
    return DD_OK;
  };
  auto lin = [&](double2* y, const double2* x1, const double2* x2, const double2* x3) -> dd_status {
    if ((e = set_coef(cf)) != DD_OK) return e;
    DD_COUNT_LAUNCH(), k_hb_lin<<<grid, 256, 0, s>>>(n_f, n, dact, dc, x1, x2, x3, y);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  };
  // x = eta / u ; r = eta - W_u x ; rhat = p = r
  for (int f = 0; f < n_f; ++f) {
    cf[3 * f] = zdiv_h(make_double2(1.0, 0.0), u_h[f]);
    cf[3 * f + 1] = cf[3 * f + 2] = make_double2(0.0, 0.0);
  }
  if ((e = lin(x, eta, nullptr, nullptr)) != DD_OK) return e;
  if ((e = matvec(x, t)) != DD_OK) return e;
  for (int f = 0; f < n_f; ++f) {
    cf[3 * f] = make_double2(1.0, 0.0);
    cf[3 * f + 1] = make_double2(-1.0, 0.0);
  }
  if ((e = lin(r, eta, t, nullptr)) != DD_OK) return e;
  DD_CUDA(c, cudaMemcpyAsync(rh, r, vb, cudaMemcpyDeviceToDevice, s));
  DD_CUDA(c, cudaMemcpyAsync(p, r, vb, cudaMemcpyDeviceToDevice, s));
  std::vector<double2> eta2, rho, rr, tmp, ts, tt;
  if ((e = hb_dot(c, n_f, n, eta, eta, dpart, eta2, s)) != DD_OK) return e;
  if ((e = hb_dot(c, n_f, n, rh, r, dpart, rho, s)) != DD_OK) return e;
  if ((e = hb_dot(c, n_f, n, r, r, dpart, rr, s)) != DD_OK) return e;
  std::vector<double2> alpha(n_f), omega(n_f);
  int it = 0;
  auto relres = [&](int f) { return eta2[f].x > 0 ? sqrt(rr[f].x / eta2[f].x) : sqrt(rr[f].x); };
  for (; it < maxiter; ++it) {
    int live = 0;
    for (int f = 0; f < n_f; ++f) {
      act[f] = act[f] && relres(f) > tol && (rho[f].x != 0.0 || rho[f].y != 0.0);
      live += act[f];
    }
    if (!live) break;
    if ((e = matvec(p, v)) != DD_OK) return e;
    if ((e = hb_dot(c, n_f, n, rh, v, dpart, tmp, s)) != DD_OK) return e;
    for (int f = 0; f < n_f; ++f) {
      alpha[f] = (tmp[f].x != 0.0 || tmp[f].y != 0.0) ? zdiv_h(rho[f], tmp[f]) : make_double2(0.0, 0.0);
      cf[3 * f] = make_double2(1.0, 0.0);
      cf[3 * f + 1] = make_double2(-alpha[f].x, -alpha[f].y);
    }
    if ((e = lin(sv, r, v, nullptr)) != DD_OK) return e;     // s = r - alpha v
    if ((e = matvec(sv, t)) != DD_OK) return e;
    if ((e = hb_dot(c, n_f, n, t, sv, dpart, ts, s)) != DD_OK) return e;
    if ((e = hb_dot(c, n_f, n, t, t, dpart, tt, s)) != DD_OK) return e;
    for (int f = 0; f < n_f; ++f) {
      omega[f] = tt[f].x > 0 ? make_double2(ts[f].x / tt[f].x, ts[f].y / tt[f].x) : make_double2(0.0, 0.0);
      cf[3 * f] = make_double2(1.0, 0.0);
      cf[3 * f + 1] = alpha[f];
      cf[3 * f + 2] = omega[f];
    }
    if ((e = lin(x, x, p, sv)) != DD_OK) return e;           // x += alpha p + omega s
    for (int f = 0; f < n_f; ++f) {
      cf[3 * f] = make_double2(1.0, 0.0);
      cf[3 * f + 1] = make_double2(-omega[f].x, -omega[f].y);
      cf[3 * f + 2] = make_double2(0.0, 0.0);
    }
    if ((e = lin(r, sv, t, nullptr)) != DD_OK) return e;     // r = s - omega t
    std::vector<double2> rho_new;
    if ((e = hb_dot(c, n_f, n, rh, r, dpart, rho_new, s)) != DD_OK) return e;
    if ((e = hb_dot(c, n_f, n, r, r, dpart, rr, s)) != DD_OK) return e;
    for (int f = 0; f < n_f; ++f) {
      const bool ok = (omega[f].x != 0.0 || omega[f].y != 0.0) && (rho[f].x != 0.0 || rho[f].y != 0.0);
      const double2 beta = ok ? zmul_h(zdiv_h(rho_new[f], rho[f]), zdiv_h(alpha[f], omega[f])) : make_double2(0.0, 0.0);
      rho[f] = rho_new[f];
      cf[3 * f] = make_double2(1.0, 0.0);                    // p = r + beta p - beta omega v
      cf[3 * f + 1] = beta;
      cf[3 * f + 2] = zmul_h(make_double2(-beta.x, -beta.y), omega[f]);
    }
    if ((e = lin(p, r, p, v)) != DD_OK) return e;
  }
  cudaEventRecord(e1, s);
  DD_CUDA(c, cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  dd_heatbath_stats st{};
  st.iterations = it;
  st.matvecs = matvecs;
  st.seconds = ms * 1e-3;
  int conv = 0;
  for (int f = 0; f < n_f; ++f) {
    const double rel = relres(f);
    if (!(rel == rel)) return fail(c, DD_ENAN, "NaN in the heat-bath residual");
    st.max_relres = std::max(st.max_relres, rel);
    conv += rel <= tol;
  }
  st.converged = conv;
  if (out) *out = st;
  if (conv < n_f) return fail(c, DD_ENOCONV, "heat-bath: some field above tolerance");
  return DD_OK;
}

// ---- reweighting factor of Eq. (rw): samples s = |eta|^2 - |M eta|^2 ------------
// M = 1 - R_{N+1}(W_1) and 1 - W_1 = w, so R_{N+1}(W_1) = T_{N+1}(w/c) / T_{N+1}(1/c)
// (w^{N+1} at c = 0).  R eta by the three-term recurrence in w, normalised so that
// every iterate stays O(|eta|): t_j = T_j(w/c) eta / T_j(1/c), t_0 = eta, t_1 = w eta,
// t_{j+1} = a_j w t_j - b_j t_{j-1} with a_j = (2/c) T_j/T_{j+1}, b_j = T_{j-1}/T_{j+1}
// (a = 1, b = 0 at c = 0).  N + 1 dd_apply_w batches over all sources.  The sample is
// formed as 2 Re(eta, R eta) - |R eta|^2, which equals |eta|^2 - |eta - R eta|^2
// without the cancellation of two nearly equal norms.
static dd_status reweight_dev(dd_ctx* c, int N, double cpar, int n_src, const double2* eta, double* s_out,
                              double2** r_eta_dev, const dd_solve_params* prm, cudaStream_t s) {
  const long long n = 12LL * c->info.n_dpi;
  const size_t vb = sizeof(double2) * (size_t)n_src * n;
  void *va, *vb2, *vw, *vc, *vpart;
  dd_status e;
  if ((e = workspace(c, 213, vb, &va)) || (e = workspace(c, 214, vb, &vb2)) || (e = workspace(c, 215, vb, &vw)) ||
      (e = workspace(c, 216, sizeof(double2) * 3 * n_src, &vc)) ||
      (e = workspace(c, 217, sizeof(double) * 2 * n_src * HB_CHUNKS, &vpart)))
    return e;
  double2 *A = (double2*)va, *B = (double2*)vb2, *wt = (double2*)vw, *dc = (double2*)vc;
  double* dpart = (double*)vpart;
  const dim3 grid((unsigned)((n + 255) / 256), n_src);
  // T_j(1/c), j = 0..N+1 (host scalars; the recurrence is exact in exact arithmetic)
  std::vector<double> T(N + 2, 1.0);
  if (cpar > 0.0) {
    T[1] = 1.0 / cpar;
    for (int j = 1; j <= N; ++j) T[j + 1] = 2.0 / cpar * T[j] - T[j - 1];
  }
  bool noconv = false;
  auto w_of = [&](const double2* x, double2* y) -> dd_status {
    dd_status r0 = apply_w_dev(c, n_src, (const double*)x, (double*)y, prm, s);
    if (r0 == DD_ENOCONV) noconv = true;
    else if (r0 != DD_OK) return r0;
    return DD_OK;
  };
  std::vector<double2> cf(3 * n_src);
  // t_1 = w eta
  if ((e = w_of(eta, A)) != DD_OK) return e;
  const double2* prev = eta;
  double2* cur = A;
  for (int j = 1; j <= N; ++j) {
    double2* next = (prev == eta) ? B : const_cast<double2*>(prev);
    if (cpar > 0.0) {
      if ((e = w_of(cur, wt)) != DD_OK) return e;
      const double a = 2.0 / cpar * T[j] / T[j + 1], b = T[j - 1] / T[j + 1];
      for (int f = 0; f < n_src; ++f) {
        cf[3 * f] = make_double2(a, 0.0);
        cf[3 * f + 1] = make_double2(-b, 0.0);
        cf[3 * f + 2] = make_double2(0.0, 0.0);
      }
      DD_CUDA(c, cudaMemcpyAsync(dc, cf.data(), sizeof(double2) * 3 * n_src, cudaMemcpyHostToDevice, s));
      DD_COUNT_LAUNCH(), k_hb_lin<<<grid, 256, 0, s>>>(n_src, n, nullptr, dc, wt, prev, nullptr, next);
      DD_CUDA(c, cudaGetLastError());
    } else {
      if ((e = w_of(cur, next)) != DD_OK) return e;
    }
    prev = cur;
    cur = next;
  }
  std::vector<double2> er, rr;
  if ((e = hb_dot(c, n_src, n, eta, cur, dpart, er, s)) != DD_OK) return e;
  if ((e = hb_dot(c, n_src, n, cur, cur, dpart, rr, s)) != DD_OK) return e;
  for (int f = 0; f < n_src; ++f) {
    s_out[f] = 2.0 * er[f].x - rr[f].x;
    if (!(s_out[f] == s_out[f])) return fail(c, DD_ENAN, "NaN in a reweighting sample");
  }
  if (r_eta_dev) *r_eta_dev = cur;
  if (noconv) return fail(c, DD_ENOCONV, "a block or frame solve missed its tolerance");
  return DD_OK;
}

// ---- block-local molecular dynamics of the active links (Sec. 4, Eq. SFeffN) ----
// Momenta P[x][mu][t] (8 per link, generators T_t = lambda_t / 2) live on the
// active links; the kernels walk the active-link list of the force plan, in
// which every active link appears once.

// U <- exp(i H) U for hermitian traceless H = sum_t h_t T_t, FP64: scaling and
// squaring with a degree-12 Taylor polynomial (Moler & Van Loan, "Nineteen
// dubious ways to compute the exponential of a matrix", 2003): A = iH / 2^s
// with |A|_F <= 1/4, exp(A) by Horner's rule, then s squarings.
__device__ void su3_expi_mul(const double (&h)[8], double2 (&U)[9]) {
  const double r3 = 0.57735026918962576451;         // 1 / sqrt(3)
  double2 H[9];
  H[0] = make_double2(0.5 * (h[2] + r3 * h[7]), 0.0);
  H[4] = make_double2(0.5 * (-h[2] + r3 * h[7]), 0.0);
  H[8] = make_double2(-r3 * h[7], 0.0);
  H[1] = make_double2(0.5 * h[0], -0.5 * h[1]);
  H[3] = make_double2(0.5 * h[0], 0.5 * h[1]);
  H[2] = make_double2(0.5 * h[3], -0.5 * h[4]);
  H[6] = make_double2(0.5 * h[3], 0.5 * h[4]);
  H[5] = make_double2(0.5 * h[5], -0.5 * h[6]);
  H[7] = make_double2(0.5 * h[5], 0.5 * h[6]);
  double nrm = 0.0;
  for (int k = 0; k < 9; ++k) nrm += H[k].x * H[k].x + H[k].y * H[k].y;
  nrm = sqrt(nrm);
  int sq = 0;
  while (nrm > 0.25 && sq < 60) {
    nrm *= 0.5;
    ++sq;
  }
  const double sc = ldexp(1.0, -sq);
  double2 A[9];
  for (int k = 0; k < 9; ++k) A[k] = make_double2(-sc * H[k].y, sc * H[k].x);     // i H / 2^s
  double2 E[9];
  for (int k = 0; k < 9; ++k) E[k] = make_double2(k % 4 == 0 ? 1.0 : 0.0, 0.0);
  for (int n = 12; n >= 1; --n) {
    double2 T[9];
    const double inv = 1.0 / n;
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < 3; ++k) {
          const double2 a = A[r * 3 + k], e = E[k * 3 + q];
          acc.x += a.x * e.x - a.y * e.y;
          acc.y += a.x * e.y + a.y * e.x;
        }
        T[r * 3 + q] = make_double2(acc.x * inv + (r == q ? 1.0 : 0.0), acc.y * inv);
      }
    for (int k = 0; k < 9; ++k) E[k] = T[k];
  }
  for (int q = 0; q < sq; ++q) {
    double2 T[9];
    for (int r = 0; r < 3; ++r)
      for (int p = 0; p < 3; ++p) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < 3; ++k) {
          const double2 a = E[r * 3 + k], e = E[k * 3 + p];
          acc.x += a.x * e.x - a.y * e.y;
          acc.y += a.x * e.y + a.y * e.x;
        }
        T[r * 3 + p] = acc;
      }
    for (int k = 0; k < 9; ++k) E[k] = T[k];
  }
  double2 W[9];
  for (int r = 0; r < 3; ++r)
    for (int p = 0; p < 3; ++p) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const double2 a = E[r * 3 + k], u = U[k * 3 + p];
        acc.x += a.x * u.x - a.y * u.y;
        acc.y += a.x * u.y + a.y * u.x;
      }
      W[r * 3 + p] = acc;
    }
  for (int k = 0; k < 9; ++k) U[k] = W[k];
}

// Pm[active link] = P[active link] (Pm zeroed before)
__global__ void k_md_gather(const int4* __restrict__ al, long long n_al, const double* __restrict__ P,
                            double* __restrict__ Pm) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_al) return;
  const long long o = ((long long)al[k].y * 4 + al[k].z) * 8;
#pragma unroll
  for (int t = 0; t < 8; ++t) Pm[o + t] = P[o + t];
}

// P -= c F on the active links
__global__ void k_md_momenta(const int4* __restrict__ al, long long n_al, double* __restrict__ P,
                             const double* __restrict__ F, double c) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_al) return;
  const long long o = ((long long)al[k].y * 4 + al[k].z) * 8;
#pragma unroll
  for (int t = 0; t < 8; ++t) P[o + t] -= c * F[o + t];
}

// U_mu(x) <- exp(i dt sum_t P_t T_t) U_mu(x) on the active links (the stored
// links carry the time-boundary sign, a factor that commutes with the update)
__global__ void k_md_links(const int4* __restrict__ al, long long n_al, const double* __restrict__ P, double dt,
                           double2* __restrict__ U) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_al) return;
  const long long l = (long long)al[k].y * 4 + al[k].z;
  double h[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) h[t] = dt * P[l * 8 + t];
  double2 u[9];
  double2* p = U + l * 9;
#pragma unroll
  for (int m = 0; m < 9; ++m) u[m] = p[m];
  su3_expi_mul(h, u);
#pragma unroll
  for (int m = 0; m < 9; ++m) p[m] = u[m];
}

// S, the per-block S^a (host array or null) and S^r of device fields chi
// (dd_multiboson_action); DD_ENOCONV (values filled) if a solve missed its tolerance
static dd_status mb_action_dev(dd_ctx* c, int n_f, const double* u, const double* din, double* S,
                               double* S_block, double* S_r, const dd_solve_params* prm, cudaStream_t s) {
  const int nb = (int)c->blocks.size();
  const size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  dd_status e;
  void *wv, *du, *dS;
  if ((e = workspace(c, 46, bytes, &wv)) || (e = workspace(c, 47, 16ULL * n_f, &du)) ||
      (e = workspace(c, 48, sizeof(double) * (nb + 1 + 4096), &dS)))
    return e;
  dd_status r = apply_w_dev(c, n_f, din, (double*)wv, prm, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  DD_CUDA(c, cudaMemcpyAsync(du, u, 16ULL * n_f, cudaMemcpyHostToDevice, s));
  WPlan& P = *(WPlan*)c->wplan;
  DD_COUNT_LAUNCH(), k_action_blocks<<<nb, 256, 0, s>>>(P.d_b_grp, P.d_b_dpi, n_f, c->info.n_dpi,
                                     (const double2*)du, (const double2*)din,
                                     (const double2*)wv, (double*)dS);
  if (P.n_cgrp > 0)
    DD_COUNT_LAUNCH(), k_action_blocks<<<P.n_cgrp, 256, 0, s>>>(P.d_c_grp, P.d_c_dpi, n_f, c->info.n_dpi,
                                             (const double2*)du, (const double2*)din,
                                             (const double2*)wv, (double*)dS + nb);
  DD_CUDA(c, cudaGetLastError());
  std::vector<double> h(nb + P.n_cgrp);
  DD_CUDA(c, cudaMemcpyAsync(h.data(), dS, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  double sb = 0.0, sr = 0.0;
  for (int b = 0; b < nb; ++b) {
    sb += h[b];
    if (S_block) S_block[b] = h[b];
  }
  for (int k = 0; k < P.n_cgrp; ++k) sr += h[nb + k];
  *S_r = sr;
  *S = sb + sr;
  return r;
}

// The multi-boson force on the active links (dd_mb_force) from device fields
// chi into the device array dF (added onto it with `accumulate`); a block or
// frame-piece solve that missed its tolerance sets *noconv.
static dd_status mb_force_dev(dd_ctx* c, int n_f, const double* u, const double* din, double* dF,
                              bool accumulate, const dd_solve_params* prm, bool* noconv, cudaStream_t s) {
  const int nb = (int)c->blocks.size();
  const size_t vbytes = 16ULL * n_f * c->info.n_dpi * 12;
  const size_t fbytes = sizeof(double) * 32ULL * c->V;
  dd_status e;
  std::vector<int> insts(nb);
  for (int b = 0; b < nb; ++b) insts[b] = c->omega0 + b;
  Batch* ob;
  if ((e = get_batch_insts(c, insts, n_f, &ob)) != DD_OK) return e;
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  if ((e = build_force_plan(c, P)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  void *vsrc, *vy, *vrhs, *vz, *vu;
  if ((e = workspace(c, 231, 16ULL * ob->user_tot, &vsrc)) || (e = workspace(c, 232, 16ULL * ob->user_tot, &vy)) ||
      (e = workspace(c, 233, 16ULL * ob->user_tot, &vrhs)) || (e = workspace(c, 234, 16ULL * ob->user_tot, &vz)) ||
      (e = workspace(c, 235, 16ULL * n_f, &vu)))
    return e;
  DD_CUDA(c, cudaMemcpyAsync(vu, u, 16ULL * n_f, cudaMemcpyHostToDevice, s));
  dd_solve_stats st1{};
  // chi' = chi - Q chi (stage A without the frame; S^a holds the frame pieces only
  // through it), then y = D_Omega^{-1} D_{Omega,ext} chi' for every block and field
  const double* chi_b = din;
  if (c->info.n_C > 0) {
    void* cp;
    if ((e = workspace(c, 237, vbytes, &cp)) != DD_OK) return e;
    dd_status r0 = frame_stage(c, P, n_f, din, (double*)cp, nullptr, false, prm, &st1, s);
    if (r0 == DD_ENOCONV) *noconv = true;
    else if (r0 != DD_OK) return r0;
    chi_b = (const double*)cp;
  }
  InjectArgs a;
  a.U = c->d_U;
  a.chi = (const double2*)chi_b;
  a.dpi_pos = c->d_dpi_pos;
  for (int m = 0; m < 4; ++m) a.L[m] = c->L[m];
  a.n_dpi = c->info.n_dpi;
  a.n_f = n_f;
  a.kappa = c->kappa;
  a.src = (double2*)vsrc;
  BatchDev bd = batch_view(c, *ob);
  dim3 g1((c->info.max_omega + 127) / 128, n_f, nb);
  DD_COUNT_LAUNCH(), k_inject_omega<<<g1, 128, 0, s>>>(bd, a);
  DD_CUDA(c, cudaGetLastError());
  dd_status r1 = solve_batch(c, *ob, (const double*)vsrc, (double*)vy, prm, &st1, s, true);
  if (r1 == DD_ENOCONV) *noconv = true;
  else if (r1 != DD_OK) return r1;
  // z = (D_Omega^dag)^{-1} P_B (u chi + y) = gamma_5 D_Omega^{-1} gamma_5 P_B (u chi + y)
  DD_CUDA(c, cudaMemsetAsync(vrhs, 0, 16ULL * ob->user_tot, s));
  const int nB = c->info.n_B;
  if (nB) {
    dim3 g((nB + 127) / 128, n_f);
    DD_COUNT_LAUNCH(), k_force_rhs<<<g, 128, 0, s>>>(P.d_b_blk, P.d_b_loc, P.d_b_dpi, nB, n_f, c->info.n_dpi,
                                                     ob->d_uoff, (const double2*)vu, (const double2*)din,
                                                     (const double2*)vy, (double2*)vrhs);
    DD_CUDA(c, cudaGetLastError());
  }
  dd_status r2 = solve_batch(c, *ob, (const double*)vrhs, (double*)vz, prm, &st1, s, true);
  if (r2 == DD_ENOCONV) *noconv = true;
  else if (r2 != DD_OK) return r2;
  if (!accumulate) DD_CUDA(c, cudaMemsetAsync(dF, 0, fbytes, s));
  if (P.n_al > 0) {
    TimingRec rec{};
    if (c->timing) {
      cudaEventCreate(&rec.a);
      cudaEventCreate(&rec.b);
      rec.which = 3;
      rec.bytes = 576.0 * (double)P.n_al * n_f;     // algorithmic FP64 flops
      cudaEventRecord(rec.a, s);
    }
    DD_COUNT_LAUNCH(), k_mb_force<<<(unsigned)((P.n_al + 127) / 128), 128, 0, s>>>(
        P.d_al, P.d_al_loc, P.n_al, n_f, ob->d_uoff, (const double2*)c->d_U, (const double2*)vy,
        (const double2*)vz, c->kappa, dF, accumulate ? 1 : 0);
    if (c->timing) {
      cudaEventRecord(rec.b, s);
      c->trec.push_back(rec);
    }
    DD_CUDA(c, cudaGetLastError());
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// The pseudofermion force of S_pf = sum_a |(D_Omega^dag)^{-1} phi_a|^2 added onto
// dF, and S_pf: zg = D_Omega^{-1} gamma_5 phi, Y = gamma_5 zg = (D^dag)^{-1} phi,
// X = D_Omega^{-1} Y; dS_pf = -2 Re <Y, dD X> is the link kernel with (y, z) = (X, zg).
static dd_status pf_force_dev(dd_ctx* c, const double* dphi, double* dF, const dd_solve_params* prm,
                              bool* noconv, double* s_pf, cudaStream_t s) {
  const int nb = (int)c->blocks.size();
  std::vector<int> insts(nb);
  for (int b = 0; b < nb; ++b) insts[b] = c->omega0 + b;
  Batch* ob;
  dd_status e;
  if ((e = get_batch_insts(c, insts, 1, &ob)) != DD_OK) return e;
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  if ((e = build_force_plan(c, P)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  const long long ntot = ob->user_tot;
  void *vg, *vzg, *vY, *vX, *vpart;
  if ((e = workspace(c, 260, 16ULL * ntot, &vg)) || (e = workspace(c, 261, 16ULL * ntot, &vzg)) ||
      (e = workspace(c, 262, 16ULL * ntot, &vY)) || (e = workspace(c, 263, 16ULL * ntot, &vX)) ||
      (e = workspace(c, 264, sizeof(double) * 2 * HB_CHUNKS, &vpart)))
    return e;
  const unsigned g5 = (unsigned)((ntot + 255) / 256);
  DD_COUNT_LAUNCH(), k_gamma5<<<g5, 256, 0, s>>>(ntot, (const double2*)dphi, (double2*)vg);
  DD_CUDA(c, cudaGetLastError());
  dd_solve_stats st1{};
  dd_status r = solve_batch(c, *ob, (const double*)vg, (double*)vzg, prm, &st1, s, true);
  if (r == DD_ENOCONV) *noconv = true;
  else if (r != DD_OK) return r;
  DD_COUNT_LAUNCH(), k_gamma5<<<g5, 256, 0, s>>>(ntot, (const double2*)vzg, (double2*)vY);
  DD_CUDA(c, cudaGetLastError());
  r = solve_batch(c, *ob, (const double*)vY, (double*)vX, prm, &st1, s, true);
  if (r == DD_ENOCONV) *noconv = true;
  else if (r != DD_OK) return r;
  if (P.n_al > 0)
    DD_COUNT_LAUNCH(), k_mb_force<<<(unsigned)((P.n_al + 127) / 128), 128, 0, s>>>(
        P.d_al, P.d_al_loc, P.n_al, 1, ob->d_uoff, (const double2*)c->d_U, (const double2*)vX,
        (const double2*)vzg, c->kappa, dF, 1);
  DD_CUDA(c, cudaGetLastError());
  std::vector<double2> n2;
  if ((e = hb_dot(c, 1, ntot, (const double2*)vzg, (const double2*)vzg, (double*)vpart, n2, s)) != DD_OK) return e;
  *s_pf = n2[0].x;
  return DD_OK;
}

// one leapfrog trajectory of the active links; dP: device momenta, zero off the
// active links; dchi / dphi: device fields or null
static dd_status md_dev(dd_ctx* c, int n_f, const double* u, const double* dchi, const double* dphi, double* dP,
                        double tau, int nsteps, const dd_solve_params* prm, dd_md_stats* st, cudaStream_t s) {
  WPlan* PP;
  dd_status e;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  if ((e = build_force_plan(c, P)) != DD_OK) return e;
  const long long nlink = 4LL * c->V;
  void *vF, *vpart;
  if ((e = workspace(c, 265, sizeof(double) * 8 * nlink, &vF)) ||
      (e = workspace(c, 266, sizeof(double) * 2 * HB_CHUNKS, &vpart)))
    return e;
  double* dF = (double*)vF;
  bool noconv = false;
  double s_pf = 0.0;
  auto kinetic = [&](double* out) -> dd_status {
    std::vector<double2> k2;
    dd_status r = hb_dot(c, 1, 4 * nlink, (const double2*)dP, (const double2*)dP, (double*)vpart, k2, s);
    *out = 0.5 * k2[0].x;
    return r;
  };
  auto action = [&](double* out) -> dd_status {
    *out = 0.0;
    if (n_f == 0) return DD_OK;
    double Sr = 0.0;
    dd_status r = mb_action_dev(c, n_f, u, dchi, out, nullptr, &Sr, prm, s);
    if (r == DD_ENOCONV) {
      noconv = true;
      r = DD_OK;
    }
    return r;
  };
  auto force = [&]() -> dd_status {
    DD_CUDA(c, cudaMemsetAsync(dF, 0, sizeof(double) * 8 * nlink, s));
    dd_status r;
    if (n_f > 0 && (r = mb_force_dev(c, n_f, u, dchi, dF, true, prm, &noconv, s)) != DD_OK) return r;
    if (dphi && (r = pf_force_dev(c, dphi, dF, prm, &noconv, &s_pf, s)) != DD_OK) return r;
    ++st->force_evals;
    return DD_OK;
  };
  const unsigned gl = (unsigned)std::max<long long>(1, (P.n_al + 127) / 128);
  auto kick = [&](double cfac) -> dd_status {
    if (P.n_al > 0) DD_COUNT_LAUNCH(), k_md_momenta<<<gl, 128, 0, s>>>(P.d_al, P.n_al, dP, dF, cfac);
    DD_CUDA(c, cudaGetLastError());
    return DD_OK;
  };
  EventPair evs;
  cudaEventRecord(evs.a, s);
  const double dt = tau / nsteps;
  if ((e = kinetic(&st->kinetic0)) || (e = action(&st->s_mb0)) || (e = force())) return e;
  st->s_pf0 = dphi ? s_pf : 0.0;
  if ((e = kick(0.5 * dt)) != DD_OK) return e;
  for (int i = 0; i < nsteps; ++i) {
    if (P.n_al > 0) DD_COUNT_LAUNCH(), k_md_links<<<gl, 128, 0, s>>>(P.d_al, P.n_al, dP, dt, (double2*)c->d_U);
    DD_CUDA(c, cudaGetLastError());
    gauge_touched(c);
    if ((e = force()) != DD_OK) return e;
    if ((e = kick(i + 1 < nsteps ? dt : 0.5 * dt)) != DD_OK) return e;
  }
  st->s_pf1 = dphi ? s_pf : 0.0;
  if ((e = kinetic(&st->kinetic1)) || (e = action(&st->s_mb1))) return e;
  cudaEventRecord(evs.b, s);
  DD_CUDA(c, cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, evs.a, evs.b);
  st->seconds = ms * 1e-3;
  st->H0 = st->kinetic0 + st->s_mb0 + st->s_pf0;
  st->H1 = st->kinetic1 + st->s_mb1 + st->s_pf1;
  st->steps = nsteps;
  if (noconv) return fail(c, DD_ENOCONV, "a solve of the trajectory missed its tolerance");
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_apply_w(dd_ctx* c, int n_f, const double* chi, double* w_chi,
                     const dd_solve_params* prm, void* stream) {
  if (!c || !chi || !w_chi || !prm || n_f < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_f > 65535) return fail(c, DD_EINVAL, "n_f must be <= 65535");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  cudaStream_t s = (cudaStream_t)stream;
  size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  const double* din = chi;
  double* dout = w_chi;
  bool hin = !is_device_ptr(chi), hout = !is_device_ptr(w_chi);
  dd_status e;
  if (hin) {
    void* p;
    if ((e = workspace(c, 44, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, chi, bytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  if (hout) {
    void* p;
    if ((e = workspace(c, 45, bytes, &p)) != DD_OK) return e;
    dout = (double*)p;
  }
  dd_status r = apply_w_dev(c, n_f, din, dout, prm, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  if (hout) DD_CUDA(c, cudaMemcpyAsync(w_chi, dout, bytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return r;
}

dd_status dd_apply_w_part(dd_ctx* c, int part, int n_f, const int* ids, int nblk, const double* in,
                          double* out, const dd_solve_params* prm, void* stream) {
  if (!c || !in || !out || !prm || n_f < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_f > 65535) return fail(c, DD_EINVAL, "n_f must be <= 65535");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  const double* din = in;
  double* dout = out;
  const bool hin = !is_device_ptr(in), hout = !is_device_ptr(out);
  dd_status e;
  if (hin) {
    void* p;
    if ((e = workspace(c, 44, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, in, bytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  if (hout) {          // the entries the stage does not write are kept
    void* p;
    if ((e = workspace(c, 45, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, out, bytes, cudaMemcpyHostToDevice, s));
    dout = (double*)p;
  }
  dd_status r = apply_w_part_dev(c, part, n_f, ids, nblk, din, dout, prm, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  if (hout) DD_CUDA(c, cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return r;
}

dd_status dd_multiboson_action(dd_ctx* c, int n_f, const double* u, const double* chi, double* S,
                               double* S_block, double* S_r, const dd_solve_params* prm,
                               void* stream) {
  if (!c || !u || !chi || !S || !S_r || !prm || n_f < 1) return fail(c, DD_EINVAL, "bad argument");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  cudaStream_t s = (cudaStream_t)stream;
  size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  const double* din = chi;
  dd_status e;
  if (!is_device_ptr(chi)) {
    void* p;
    if ((e = workspace(c, 44, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, chi, bytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  return mb_action_dev(c, n_f, u, din, S, S_block, S_r, prm, s);
}

dd_status dd_multiboson_heatbath(dd_ctx* c, int n_f, const double* u, const double* eta, double* chi,
                                 double tol, int maxiter, const dd_solve_params* prm, dd_heatbath_stats* stats,
                                 void* stream) {
  if (!c || !u || !eta || !chi || !prm || n_f < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_f > 65535) return fail(c, DD_EINVAL, "n_f must be <= 65535");
  if (!(tol > 0) || maxiter < 1) return fail(c, DD_EINVAL, "bad heat-bath tolerance or iteration cap");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  for (int f = 0; f < n_f; ++f)
    if (u[2 * f] == 0.0 && u[2 * f + 1] == 0.0) return fail(c, DD_EINVAL, "root u_k = 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = 16ULL * n_f * c->info.n_dpi * 12;
  const double* din = eta;
  double* dout = chi;
  const bool hin = !is_device_ptr(eta), hout = !is_device_ptr(chi);
  dd_status e;
  if (hin) {
    void* p;
    if ((e = workspace(c, 211, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, eta, bytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  if (hout) {
    void* p;
    if ((e = workspace(c, 212, bytes, &p)) != DD_OK) return e;
    dout = (double*)p;
  }
  std::vector<double2> uh(n_f);
  for (int f = 0; f < n_f; ++f) uh[f] = make_double2(u[2 * f], u[2 * f + 1]);
  dd_status r = heatbath_dev(c, n_f, uh.data(), (const double2*)din, (double2*)dout, tol, maxiter, prm, stats, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  if (hout) DD_CUDA(c, cudaMemcpyAsync(chi, dout, bytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return r;
}

dd_status dd_mb_force(dd_ctx* c, int n_f, const double* u, const double* chi, double* F,
                      const dd_solve_params* prm, void* stream) {
  if (!c || !u || !chi || !F || !prm || n_f < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_f > 65535) return fail(c, DD_EINVAL, "n_f must be <= 65535");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  if (c->csw != 0.0) return fail(c, DD_EINVAL, "the force does not include the clover term");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vbytes = 16ULL * n_f * c->info.n_dpi * 12;
  const size_t fbytes = sizeof(double) * 32ULL * c->V;
  dd_status e;
  const double* din = chi;
  if (!is_device_ptr(chi)) {
    void* p;
    if ((e = workspace(c, 230, vbytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, chi, vbytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  double* dF = F;
  const bool hF = !is_device_ptr(F);
  if (hF) {
    void* p;
    if ((e = workspace(c, 236, fbytes, &p)) != DD_OK) return e;
    dF = (double*)p;
  }
  bool noconv = false;
  if ((e = mb_force_dev(c, n_f, u, din, dF, false, prm, &noconv, s)) != DD_OK) return e;
  if (hF) DD_CUDA(c, cudaMemcpyAsync(F, dF, fbytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  if (noconv) return fail(c, DD_ENOCONV, "a block or frame-piece solve missed its tolerance");
  return DD_OK;
}

dd_status dd_logdet_force(dd_ctx* c, int n_noise, const double* eta, double* G, const dd_solve_params* prm,
                          void* stream) {
  if (!c || !eta || !G || !prm || n_noise < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_noise > 65535) return fail(c, DD_EINVAL, "n_noise must be <= 65535");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  if (c->csw != 0.0) return fail(c, DD_EINVAL, "the force does not include the clover term");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)c->blocks.size();
  const size_t fbytes = sizeof(double) * 32ULL * c->V;
  std::vector<int> insts(nb);
  for (int b = 0; b < nb; ++b) insts[b] = c->omega0 + b;
  Batch* ob;
  dd_status e;
  if ((e = get_batch_insts(c, insts, n_noise, &ob)) != DD_OK) return e;
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& P = *PP;
  if ((e = build_force_plan(c, P)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  const size_t vbytes = 16ULL * ob->user_tot;
  const double* din = eta;
  if (!is_device_ptr(eta)) {
    void* p;
    if ((e = workspace(c, 250, vbytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, eta, vbytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  double* dG = G;
  const bool hG = !is_device_ptr(G);
  if (hG) {
    void* p;
    if ((e = workspace(c, 251, fbytes, &p)) != DD_OK) return e;
    dG = (double*)p;
  }
  void *vrhs, *vz;
  if ((e = workspace(c, 252, vbytes, &vrhs)) || (e = workspace(c, 253, vbytes, &vz))) return e;
  // z = (D_Omega^dag)^{-1} eta = gamma_5 D_Omega^{-1} gamma_5 eta (the outer gamma_5 is
  // applied by the link kernel when it reads z)
  const long long ntot = ob->user_tot;
  DD_COUNT_LAUNCH(), k_gamma5<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(ntot, (const double2*)din,
                                                                           (double2*)vrhs);
  DD_CUDA(c, cudaGetLastError());
  dd_solve_stats st1{};
  dd_status r = solve_batch(c, *ob, (const double*)vrhs, (double*)vz, prm, &st1, s, true);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  DD_CUDA(c, cudaMemsetAsync(dG, 0, fbytes, s));
  if (P.n_al > 0) {
    // the link kernel returns -2 Re sum_k <z_k, dD eta_k>; G is its mean over the
    // noise vectors without the factor -2
    DD_COUNT_LAUNCH(), k_mb_force<<<(unsigned)((P.n_al + 127) / 128), 128, 0, s>>>(
        P.d_al, P.d_al_loc, P.n_al, n_noise, ob->d_uoff, (const double2*)c->d_U, (const double2*)din,
        (const double2*)vz, c->kappa, dG, 0);
    const long long nf = 32LL * c->V;
    DD_COUNT_LAUNCH(), k_scale<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(nf, -0.5 / n_noise, dG);
    DD_CUDA(c, cudaGetLastError());
  }
  if (hG) DD_CUDA(c, cudaMemcpyAsync(G, dG, fbytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  if (r == DD_ENOCONV) return fail(c, DD_ENOCONV, "a block solve missed its tolerance");
  return DD_OK;
}

dd_status dd_reweight_samples(dd_ctx* c, int N, double cpar, int n_src, const double* eta, double* s_out,
                              double* r_eta, const dd_solve_params* prm, void* stream) {
  if (!c || !eta || !s_out || !prm || n_src < 1) return fail(c, DD_EINVAL, "bad argument");
  if (n_src > 65535) return fail(c, DD_EINVAL, "n_src must be <= 65535");
  if (N < 2 || N % 2) return fail(c, DD_EINVAL, "N must be even and >= 2");
  if (!(cpar >= 0.0 && cpar < 1.0)) return fail(c, DD_EINVAL, "c must lie in [0, 1)");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = 16ULL * n_src * c->info.n_dpi * 12;
  const double* din = eta;
  dd_status e;
  if (!is_device_ptr(eta)) {
    void* p;
    if ((e = workspace(c, 218, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, eta, bytes, cudaMemcpyHostToDevice, s));
    din = (const double*)p;
  }
  double2* rdev = nullptr;
  dd_status r = reweight_dev(c, N, cpar, n_src, (const double2*)din, s_out, &rdev, prm, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  if (r_eta) DD_CUDA(c, cudaMemcpyAsync(r_eta, rdev, bytes, cudaMemcpyDefault, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return r;
}

dd_status dd_pf_heatbath(dd_ctx* c, const double* eta, double* phi, void* stream) {
  if (!c || !eta || !phi) return fail(c, DD_EINVAL, "bad argument");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  if (c->csw != 0.0) return fail(c, DD_EINVAL, "the molecular dynamics does not include the clover term");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)c->blocks.size();
  std::vector<int> ids(nb);
  for (int b = 0; b < nb; ++b) ids[b] = b;
  Batch* ob;
  dd_status e;
  if ((e = get_batch(c, DD_DOMAIN_OMEGA, ids.data(), nb, 1, &ob)) != DD_OK) return e;
  const long long ntot = ob->user_tot;
  const size_t bytes = 16ULL * ntot;
  void *vin, *vg, *vd;
  if ((e = workspace(c, 267, bytes, &vin)) || (e = workspace(c, 268, bytes, &vg)) ||
      (e = workspace(c, 269, bytes, &vd)))
    return e;
  DD_CUDA(c, cudaMemcpyAsync(vin, eta, bytes, cudaMemcpyDefault, s));
  const unsigned g5 = (unsigned)((ntot + 255) / 256);
  DD_COUNT_LAUNCH(), k_gamma5<<<g5, 256, 0, s>>>(ntot, (const double2*)vin, (double2*)vg);
  DD_CUDA(c, cudaGetLastError());
  if ((e = dd_apply_D_block(c, DD_DOMAIN_OMEGA, ids.data(), nb, 1, (const double*)vg, (double*)vd, DD_F64, s)) !=
      DD_OK)
    return e;
  double* dout = phi;
  if (!is_device_ptr(phi)) dout = (double*)vin;          // eta is no longer needed
  DD_COUNT_LAUNCH(), k_gamma5<<<g5, 256, 0, s>>>(ntot, (const double2*)vd, (double2*)dout);
  DD_CUDA(c, cudaGetLastError());
  if (dout != phi) DD_CUDA(c, cudaMemcpyAsync(phi, dout, bytes, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return check_device_error(c, s);
}

dd_status dd_md_trajectory(dd_ctx* c, int n_f, const double* u, const double* chi, const double* phi,
                           double* P, double tau, int nsteps, const dd_solve_params* prm,
                           dd_md_stats* stats, void* stream) {
  if (!c || !P || !prm || !stats || nsteps < 1 || n_f < 0) return fail(c, DD_EINVAL, "bad argument");
  if (n_f > 0 && (!u || !chi)) return fail(c, DD_EINVAL, "fields without roots or roots without fields");
  if (n_f == 0 && !phi) return fail(c, DD_EINVAL, "no action term: give multi-boson fields or phi");
  if (n_f > 65535) return fail(c, DD_EINVAL, "n_f must be <= 65535");
  if (!(tau == tau) || std::isinf(tau)) return fail(c, DD_EINVAL, "tau must be finite");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  if (c->csw != 0.0) return fail(c, DD_EINVAL, "the molecular dynamics does not include the clover term");
  cudaStream_t s = (cudaStream_t)stream;
  *stats = dd_md_stats{};
  dd_status e;
  const double* dchi = chi;
  if (n_f > 0 && !is_device_ptr(chi)) {
    const size_t vb = 16ULL * n_f * c->info.n_dpi * 12;
    void* p;
    if ((e = workspace(c, 270, vb, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, chi, vb, cudaMemcpyHostToDevice, s));
    dchi = (const double*)p;
  }
  const double* dphi = phi;
  if (phi && !is_device_ptr(phi)) {
    const int nb = (int)c->blocks.size();
    std::vector<int> ids(nb);
    for (int b = 0; b < nb; ++b) ids[b] = b;
    Batch* ob;
    if ((e = get_batch(c, DD_DOMAIN_OMEGA, ids.data(), nb, 1, &ob)) != DD_OK) return e;
    void* p;
    if ((e = workspace(c, 271, 16ULL * ob->user_tot, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, phi, 16ULL * ob->user_tot, cudaMemcpyHostToDevice, s));
    dphi = (const double*)p;
  }
  // the momenta of the active links (zero elsewhere) in a device copy
  WPlan* PP;
  if ((e = build_plan(c, &PP)) != DD_OK) return e;
  WPlan& PL = *PP;
  if ((e = build_force_plan(c, PL)) != DD_OK) return e;
  const size_t pbytes = sizeof(double) * 32ULL * c->V;
  void *vin, *vP;
  if ((e = workspace(c, 272, pbytes, &vin)) || (e = workspace(c, 273, pbytes, &vP))) return e;
  DD_CUDA(c, cudaMemcpyAsync(vin, P, pbytes, cudaMemcpyDefault, s));
  DD_CUDA(c, cudaMemsetAsync(vP, 0, pbytes, s));
  if (PL.n_al > 0)
    DD_COUNT_LAUNCH(), k_md_gather<<<(unsigned)((PL.n_al + 127) / 128), 128, 0, s>>>(
        PL.d_al, PL.n_al, (const double*)vin, (double*)vP);
  DD_CUDA(c, cudaGetLastError());
  dd_status r = md_dev(c, n_f, u, dchi, dphi, (double*)vP, tau, nsteps, prm, stats, s);
  if (r != DD_OK && r != DD_ENOCONV) return r;
  DD_CUDA(c, cudaMemcpyAsync(P, vP, pbytes, cudaMemcpyDefault, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  dd_status d = check_device_error(c, s);
  return d != DD_OK ? d : r;
}

}  // extern "C"
