// Gauge-field set-up on the device (paper Sec. 1: links U_mu(x) in SU(3)).
//
// dd_gauge_random draws the synthetic links of the seeded input recipe
// directly on the GPU: U = exp(i eps H), H = sum_a h_a lambda_a / 2 with the
// eight Gell-Mann matrices and h_a ~ N(0, 1).  The normals come from the
// counter-based SplitMix64 stream of (seed, tag 1): draw n of stream key k is
// mix64(k + (n + 1) * 0x9E3779B97F4A7C15) with the SplitMix64 finaliser mix64
// (Steele, Lea & Flood 2014), the key is mix64(mix64(seed) ^ tag *
// 0xD1B54A32D192ED03), uniforms are ((z >> 11) + 1) 2^-53 and normals come in
// Box-Muller pairs (draw 2j: sqrt(-2 ln u_2j) cos(2 pi u_2j+1), draw 2j+1: the
// sine).  Link l = 4 * site + mu (site lexicographic, x3 fastest) takes draws
// 8l .. 8l + 7 as h_1 .. h_8.  The exponential uses scaling and squaring of
// the Taylor series (order 18 after scaling to norm <= 1/2; truncation below
// 1e-20), so the links agree with an eigen-decomposition exponential to FP64
// rounding.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace dd {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
unsigned long long mix64_host(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform53(unsigned long long key, unsigned long long n) {
  const unsigned long long z = mix64(key + (n + 1ull) * 0x9E3779B97F4A7C15ull);
  return ((double)(z >> 11) + 1.0) * 0x1p-53;
}

struct cd {
  double re, im;
};
__device__ __forceinline__ cd cmul_d(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// C = A B for 3x3 complex
__device__ __forceinline__ void mat_mul(const cd (&A)[9], const cd (&B)[9], cd (&C)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cd p = cmul_d(A[3 * i + k], B[3 * k + j]);
        s.re += p.re;
        s.im += p.im;
      }
      C[3 * i + j] = s;
    }
}

__global__ void k_gauge_random(double2* __restrict__ U, long long nlinks, double eps, unsigned long long key) {
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  double h[8];
#pragma unroll
  for (int pr = 0; pr < 4; ++pr) {
    const unsigned long long j = 4ull * (unsigned long long)l + pr;   // Box-Muller pair index
    const double u0 = uniform53(key, 2 * j), u1 = uniform53(key, 2 * j + 1);
    const double r = sqrt(-2.0 * log(u0));
    const double ang = 2.0 * M_PI * u1;
    h[2 * pr] = r * cos(ang);
    h[2 * pr + 1] = r * sin(ang);
  }
  // H = sum_a h_a lambda_a / 2 (Hermitian)
  const double s3 = 1.0 / sqrt(3.0);
  cd H[9];
  H[0] = {0.5 * (h[2] + h[7] * s3), 0.0};
  H[4] = {0.5 * (-h[2] + h[7] * s3), 0.0};
  H[8] = {0.5 * (-2.0 * h[7] * s3), 0.0};
  H[1] = {0.5 * h[0], -0.5 * h[1]};
  H[3] = {0.5 * h[0], 0.5 * h[1]};
  H[2] = {0.5 * h[3], -0.5 * h[4]};
  H[6] = {0.5 * h[3], 0.5 * h[4]};
  H[5] = {0.5 * h[5], -0.5 * h[6]};
  H[7] = {0.5 * h[5], 0.5 * h[6]};
  // A = i eps H, scaled by 2^-s to Frobenius norm <= 1/2
  double nrm = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) nrm += H[k].re * H[k].re + H[k].im * H[k].im;
  nrm = fabs(eps) * sqrt(nrm);
  int sq = 0;
  while (nrm > 0.5 && sq < 60) {
    nrm *= 0.5;
    ++sq;
  }
  const double sc = eps * ldexp(1.0, -sq);
  cd A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = {-sc * H[k].im, sc * H[k].re};
  // Taylor series by Horner: E = I + A (I + A/2 (I + A/3 (... (I + A/18))))
  cd E[9], T[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) E[k] = {(k % 4 == 0) ? 1.0 : 0.0, 0.0};
  for (int n = 18; n >= 1; --n) {
    mat_mul(A, E, T);
    const double inv = 1.0 / n;
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = {((k % 4 == 0) ? 1.0 : 0.0) + T[k].re * inv, T[k].im * inv};
  }
  for (int k = 0; k < sq; ++k) {
    mat_mul(E, E, T);
#pragma unroll
    for (int m = 0; m < 9; ++m) E[m] = T[m];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) U[l * 9 + k] = make_double2(E[k].re, E[k].im);
}

}  // namespace

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_gauge_random(dd_ctx* c, double eps, unsigned long long seed) {
  if (!c) return DD_EINVAL;
  if (!(eps == eps)) return fail(c, DD_EINVAL, "eps is NaN");
  const unsigned long long tag = 1ull;   // the gauge stream of the seeded input recipe
  const unsigned long long key = mix64_host(mix64_host(seed) ^ (tag * 0xD1B54A32D192ED03ull));
  const long long nl = 4LL * c->V;
  DD_COUNT_LAUNCH(), k_gauge_random<<<(unsigned)((nl + 127) / 128), 128>>>(c->d_U, nl, eps, key);
  DD_CUDA(c, cudaGetLastError());
  return gauge_finish(c);
}

dd_status dd_gauge_download(dd_ctx* c, double* U) {
  if (!c || !U) return fail(c, DD_EINVAL, "null argument");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not set");
  const size_t bytes = sizeof(double2) * 36ULL * c->V;
  DD_CUDA(c, cudaDeviceSynchronize());
  DD_CUDA(c, cudaMemcpy(U, c->d_U, bytes, cudaMemcpyDefault));
  // undo the folded time-boundary sign (mu = 0 links on the last time slice)
  if (c->time_bc != 1) {
    const long long spatial = c->V / c->L[0];
    double* base = U + 2 * 36 * (long long)(c->L[0] - 1) * spatial;
    for (long long x = 0; x < spatial; ++x)
      for (int k = 0; k < 18; ++k) base[72 * x + k] *= (double)c->time_bc;
  }
  return DD_OK;
}

}  // extern "C"
