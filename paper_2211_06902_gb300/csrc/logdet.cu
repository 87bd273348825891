// Dense verification of the block factorization of det D (paper Sec. 3,
// Eq. detD) on small lattices:
//   ln|det D| = ln|det W_1| + ln|det D_Lambda1| + sum_a [ln|det D_Omega0^a| - ln|det D_Phi1^a|].
// Every matrix is assembled on the GPU by applying the library's own
// operators to unit vectors (D_X through the stencil, W_1 = 1 - w through
// dd_apply_w) and factorised by an FP64 complex LU with partial pivoting.
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace dd {
namespace {

// identity in the caller layout [blk][rhs = unit index][site][12]: element
// (rhs r, site s, comp c) of block j is 1 iff 12 s + c == r
__global__ void k_identity(double2* out, long long n, long long nmat) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * n * nmat) return;
  long long m = t % (n * n);
  long long r = m / n, q = m % n;
  out[t] = make_double2(r == q ? 1.0 : 0.0, 0.0);
}

// A = 1 - A (for W_1 = 1 - w), all nmat n x n matrices
__global__ void k_one_minus(double2* A, long long n) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  long long r = t / n, q = t % n;
  double2 a = A[t];
  A[t] = make_double2((r == q ? 1.0 : 0.0) - a.x, -a.y);
}

// LU step k, 1: pivot search in column k (rows k..n-1) of each matrix.
// info[mat*4 + 0..3] = pivot row, pivot value re, im, A[k][k] before the swap
__global__ void k_lu_pivot(double2* A, long long n, long long matstride, int k, double* info,
                           double2* diag, int* swaps) {
  double2* M = A + blockIdx.z * matstride;
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1.0;
  int arg = k;
  for (long long i = k + threadIdx.x; i < n; i += blockDim.x) {
    double2 v = M[i + k * n];
    double a = v.x * v.x + v.y * v.y;
    if (a > best) { best = a; arg = (int)i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double b2 = bv[threadIdx.x + o];
      int i2 = bi[threadIdx.x + o];
      if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = b2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int p = bi[0];
    double2 pv = M[p + k * n];
    double* in = info + blockIdx.z * 4;
    in[0] = p;
    in[1] = pv.x;
    in[2] = pv.y;
    diag[blockIdx.z * n + k] = pv;
    if (p != k) swaps[blockIdx.z] += 1;
  }
}

// LU step k, 3: swap rows k and p in every column (one thread per column)
__global__ void k_lu_swap(double2* A, long long n, long long matstride, int k, const double* info) {
  double2* M = A + blockIdx.z * matstride;
  const int p = (int)info[blockIdx.z * 4];
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n || p == k) return;
  double2 a = M[k + t * n], b = M[p + t * n];
  M[k + t * n] = b;
  M[p + t * n] = a;
}

// LU step k, 4: multipliers l_i = a_i / pivot (i > k) from the copy of column k
// taken before the swap (after it, row p holds the old row k)
__global__ void k_lu_mult(double2* A, long long n, long long matstride, int k, const double* info,
                          double2* lcol, const double2* colk) {
  const double* in = info + blockIdx.z * 4;
  const int p = (int)in[0];
  const double2 pv = make_double2(in[1], in[2]);
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x + k + 1;
  if (i >= n) return;
  double2 a = colk[blockIdx.z * n + (i == p ? k : i)];
  double d = pv.x * pv.x + pv.y * pv.y;
  lcol[blockIdx.z * n + i] = make_double2((a.x * pv.x + a.y * pv.y) / d, (a.y * pv.x - a.x * pv.y) / d);
  (void)A;
  (void)matstride;
}

// LU step k, 2: copy of column k before the swap
__global__ void k_lu_colk(const double2* A, long long n, long long matstride, int k, double2* colk) {
  const double2* M = A + blockIdx.z * matstride;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  colk[blockIdx.z * n + i] = M[i + k * n];
}

// LU step k, 5: A[i][j] -= l_i A[k][j] for i, j > k
__global__ void k_lu_update(double2* A, long long n, long long matstride, int k, const double2* lcol) {
  double2* M = A + blockIdx.z * matstride;
  const long long m = n - k - 1;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  long long i = k + 1 + t % m, j = k + 1 + t / m;
  double2 l = lcol[blockIdx.z * n + i], u = M[k + j * n], a = M[i + j * n];
  a.x -= l.x * u.x - l.y * u.y;
  a.y -= l.x * u.y + l.y * u.x;
  M[i + j * n] = a;
}

// ln|det| and arg det of nmat n x n matrices stored column-major at A (destroyed)
dd_status batched_logdet(dd_ctx* c, double2* A, long long n, int nmat, cudaStream_t s,
                         std::vector<double>& logabs, std::vector<double>& phase) {
  void *vinfo, *vdiag, *vl, *vck, *vsw;
  dd_status e;
  if ((e = workspace(c, 60, sizeof(double) * 4 * nmat, &vinfo)) ||
      (e = workspace(c, 61, sizeof(double2) * n * nmat, &vdiag)) ||
      (e = workspace(c, 62, sizeof(double2) * n * nmat, &vl)) ||
      (e = workspace(c, 63, sizeof(double2) * n * nmat, &vck)) ||
      (e = workspace(c, 64, sizeof(int) * nmat, &vsw)))
    return e;
  DD_CUDA(c, cudaMemsetAsync(vsw, 0, sizeof(int) * nmat, s));
  const long long ms = n * n;
  for (int k = 0; k < n; ++k) {
    dim3 g1(1, 1, nmat);
    DD_COUNT_LAUNCH(), k_lu_pivot<<<g1, 256, 0, s>>>(A, n, ms, k, (double*)vinfo, (double2*)vdiag, (int*)vsw);
    dim3 gc((unsigned)((n + 255) / 256), 1, nmat);
    DD_COUNT_LAUNCH(), k_lu_colk<<<gc, 256, 0, s>>>(A, n, ms, k, (double2*)vck);
    DD_COUNT_LAUNCH(), k_lu_swap<<<gc, 256, 0, s>>>(A, n, ms, k, (const double*)vinfo);
    long long rem = n - k - 1;
    if (rem > 0) {
      dim3 gm((unsigned)((rem + 255) / 256), 1, nmat);
      DD_COUNT_LAUNCH(), k_lu_mult<<<gm, 256, 0, s>>>(A, n, ms, k, (const double*)vinfo, (double2*)vl, (const double2*)vck);
      long long tot = rem * rem;
      dim3 gu((unsigned)((tot + 255) / 256), 1, nmat);
      DD_COUNT_LAUNCH(), k_lu_update<<<gu, 256, 0, s>>>(A, n, ms, k, (const double2*)vl);
    }
  }
  DD_CUDA(c, cudaGetLastError());
  std::vector<double2> diag(n * nmat);
  std::vector<int> sw(nmat);
  DD_CUDA(c, cudaMemcpyAsync(diag.data(), vdiag, sizeof(double2) * n * nmat, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaMemcpyAsync(sw.data(), vsw, sizeof(int) * nmat, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  const double pi = 3.14159265358979323846;
  logabs.assign(nmat, 0.0);
  phase.assign(nmat, 0.0);
  for (int m = 0; m < nmat; ++m) {
    double la = 0.0, ph = (sw[m] % 2) ? pi : 0.0;
    for (long long k = 0; k < n; ++k) {
      double2 d = diag[m * n + k];
      la += 0.5 * std::log(d.x * d.x + d.y * d.y);
      ph += std::atan2(d.y, d.x);
    }
    logabs[m] = la;
    phase[m] = std::remainder(ph, 2 * pi);
  }
  return DD_OK;
}

// dense D_X for one domain instance kind/id: columns = D_X applied to unit vectors
dd_status dense_operator(dd_ctx* c, dd_domain kind, int id, cudaStream_t s, int slot, double2** A,
                         long long* n_out) {
  int inst;
  dd_status e = instance_of(c, kind, id, &inst);
  if (e != DD_OK) return e;
  const long long n = 12LL * c->inst[inst].d.nsites;
  void *I, *M;
  if ((e = workspace(c, slot, sizeof(double2) * n * n, &I)) ||
      (e = workspace(c, slot + 1, sizeof(double2) * n * n, &M)))
    return e;
  DD_COUNT_LAUNCH(), k_identity<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>((double2*)I, n, 1);
  DD_CUDA(c, cudaGetLastError());
  if ((e = dd_apply_D_block(c, kind, &id, 1, (int)n, (const double*)I, (double*)M, DD_F64, s)) != DD_OK)
    return e;
  *A = (double2*)M;
  *n_out = n;
  return DD_OK;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_logdet_check(dd_ctx* c, const dd_solve_params* prm, double* logabs_omega,
                                     double* logabs_phi, dd_logdet_report* rep, void* stream) {
  if (!c || !prm || !rep) return fail(c, DD_EINVAL, "null argument");
  if (!c->geom_ready || !c->gauge_ready) return fail(c, DD_EINVAL, "geometry and gauge field required");
  if (12LL * c->V > 8192) return fail(c, DD_EINVAL, "dense check limited to 12 V <= 8192");
  cudaStream_t s = (cudaStream_t)stream;
  dd_status e;
  std::vector<double> la, ph;
  dd_logdet_report r{};
  double2* A;
  long long n;
  // D on the full lattice
  if ((e = dense_operator(c, DD_DOMAIN_FULL, 0, s, 65, &A, &n)) != DD_OK) return e;
  if ((e = batched_logdet(c, A, n, 1, s, la, ph)) != DD_OK) return e;
  r.logabs_D = la[0];
  r.phase_D = ph[0];
  r.dim_D = (int)n;
  // D_Lambda1
  if ((e = dense_operator(c, DD_DOMAIN_LAMBDA1, 0, s, 65, &A, &n)) != DD_OK) return e;
  if ((e = batched_logdet(c, A, n, 1, s, la, ph)) != DD_OK) return e;
  r.logabs_Lambda1 = la[0];
  double phase_rhs = ph[0];
  r.dim_Lambda1 = (int)n;
  // D_Omega0^a and D_Phi1^a
  const int nb = (int)c->blocks.size();
  for (int kind = 0; kind < 2; ++kind) {
    double sum = 0.0;
    for (int b = 0; b < nb; ++b) {
      if ((e = dense_operator(c, kind ? DD_DOMAIN_PHI : DD_DOMAIN_OMEGA, b, s, 65, &A, &n)) != DD_OK)
        return e;
      if ((e = batched_logdet(c, A, n, 1, s, la, ph)) != DD_OK) return e;
      sum += la[0];
      if (kind == 0) {
        phase_rhs += ph[0];
        if (logabs_omega) logabs_omega[b] = la[0];
      } else {
        phase_rhs -= ph[0];
        if (logabs_phi) logabs_phi[b] = la[0];
      }
    }
    (kind ? r.logabs_Phi : r.logabs_Omega) = sum;
  }
  // W_1 = 1 - w on dPi: columns = w applied to unit vectors
  {
    const long long m = 12LL * c->info.n_dpi;
    void *I, *W;
    if ((e = workspace(c, 67, sizeof(double2) * m * m, &I)) ||
        (e = workspace(c, 68, sizeof(double2) * m * m, &W)))
      return e;
    DD_COUNT_LAUNCH(), k_identity<<<(unsigned)((m * m + 255) / 256), 256, 0, s>>>((double2*)I, m, 1);
    DD_CUDA(c, cudaGetLastError());
    e = dd_apply_w(c, (int)m, (const double*)I, (double*)W, prm, s);
    if (e != DD_OK) return e;
    DD_COUNT_LAUNCH(), k_one_minus<<<(unsigned)((m * m + 255) / 256), 256, 0, s>>>((double2*)W, m);
    DD_CUDA(c, cudaGetLastError());
    if ((e = batched_logdet(c, (double2*)W, m, 1, s, la, ph)) != DD_OK) return e;
    r.logabs_W1 = la[0];
    phase_rhs += ph[0];
    r.dim_W1 = (int)m;
  }
  const double pi = 3.14159265358979323846;
  r.phase_rhs = std::remainder(phase_rhs, 2 * pi);
  r.residual = r.logabs_D - (r.logabs_W1 + r.logabs_Lambda1 + r.logabs_Omega - r.logabs_Phi);
  *rep = r;
  return DD_OK;
}
