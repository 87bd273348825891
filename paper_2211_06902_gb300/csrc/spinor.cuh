// Device arithmetic of the Wilson hop term on SoA even-odd spinor fields.
//
// Hop term (paper Sec. 1/3, Wilson operator, kappa normalisation):
//   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                       + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ],   D = 1 - kappa H.
// In the chiral basis gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]
// the projector (1 -/+ gamma_mu) has rank 2: the two upper spin components of
// the projected spinor (h) determine the lower two, so only h (2 spins x 3
// colours) is multiplied by the link and the lower half is rebuilt.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cstring>

namespace dd {

// ---- storage <-> compute conversions -----------------------------------------
template <class S> struct StoreTraits;
template <> struct StoreTraits<double2> { typedef double T; typedef double2 C; };
template <> struct StoreTraits<float2> { typedef float T; typedef float2 C; };
template <> struct StoreTraits<__nv_bfloat162> { typedef float T; typedef float2 C; };

__device__ __forceinline__ double2 ldc(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldc(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldc(const __nv_bfloat162* p) {
  return __bfloat1622float2(*p);
}
__device__ __forceinline__ void stc(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void stc(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void stc(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// ---- pair layout ---------------------------------------------------------------
// Work vectors and per-site link copies store, for n sites of one system and
// parity, component k of site i at complex index ((k / 2) * n + i) * 2 + k % 2:
// components come in pairs per site, so one thread loads two components with
// one 16-byte (FP32), 8-byte (BF16) or 2 x 16-byte (FP64) access.  A link
// keeps its 9 entries in 5 pairs (the 10th entry is padding).
__device__ __host__ __forceinline__ long long cidx(int k, long long n, long long i) {
  return (((long long)(k >> 1)) * n + i) * 2 + (k & 1);
}

__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = __ldg(p);
  b = __ldg(p + 1);
}
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const __nv_bfloat162* p, float2& a, float2& b) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  __nv_bfloat162 x, y;
  memcpy(&x, &v.x, 4);
  memcpy(&y, &v.y, 4);
  a = __bfloat1622float2(x);
  b = __bfloat1622float2(y);
}
// plain (coherent) loads for vectors the same kernel also writes
__device__ __forceinline__ void ld_pair(double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void ld_pair(float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(__nv_bfloat162* p, float2& a, float2& b) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 x, y;
  memcpy(&x, &v.x, 4);
  memcpy(&y, &v.y, 4);
  a = __bfloat1622float2(x);
  b = __bfloat1622float2(y);
}

__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(__nv_bfloat162* p, float2 a, float2 b) {
  __nv_bfloat162 x = __float22bfloat162_rn(a), y = __float22bfloat162_rn(b);
  uint2 v;
  memcpy(&v.x, &x, 4);
  memcpy(&v.y, &y, 4);
  *reinterpret_cast<uint2*>(p) = v;
}

// 12 components of site i (NC = 12) or any even count NC
template <int NC, class S, class C>
__device__ __forceinline__ void ld_site(const S* base, long long n, long long i, C (&v)[NC]) {
#pragma unroll
  for (int q = 0; q < NC / 2; ++q) ld_pair(base + (q * n + i) * 2, v[2 * q], v[2 * q + 1]);
}
template <int NC, class S, class C>
__device__ __forceinline__ void st_site(S* base, long long n, long long i, const C (&v)[NC]) {
#pragma unroll
  for (int q = 0; q < NC / 2; ++q) st_pair(base + (q * n + i) * 2, v[2 * q], v[2 * q + 1]);
}

// the 9 entries of a link stored at site i of a (parity, mu) block of n sites
template <class S, class C>
__device__ __forceinline__ void ld_link(const S* blk, long long n, long long i, C (&U)[9]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) ld_pair(blk + (q * n + i) * 2, U[2 * q], U[2 * q + 1]);
  U[8] = ldc(blk + (4 * n + i) * 2);
}
// offset of the (parity, mu) link block: [p][mu][10 entries][n_p]
__device__ __host__ __forceinline__ long long link_block(int p, int mu, long long n0, long long np) {
  return (p ? 40 * n0 : 0) + (long long)mu * 10 * np;
}

// ---- per-chunk link bundles -------------------------------------------------------
// For the bundle form of the hop, each output parity of an instance is cut
// into chunks of LB_CHUNK sites (the batch work items) and each chunk into
// LB_QUARTERS quarters of LB_LANES sites.  A quarter's bundle holds, for its
// 32 output sites, the 8 links the hop multiplies with (forward: U_mu(x);
// backward: U_mu(x - mu), stored undaggered) and the 8 neighbour indices:
//     links [dir 8]{ [pair 4][lane 32] x (2 S), [lane 32] x S }   then   index [dir 8][lane 32] int
// (entries 0..7 of a link in pairs, entry 8 alone: 9 complex per link, no
// padding), so one bulk copy brings a quarter into shared memory, and lanes
// read consecutive 16- and 8-byte (FP32) or 8- and 4-byte (BF16) words.
// Missing neighbours have index -1 and zero links; lanes past the end of the
// parity likewise.
constexpr int LB_LANES = 32;
constexpr int LB_QUARTERS = 4;
constexpr int LB_CHUNK = LB_LANES * LB_QUARTERS;
constexpr int LB_DIR_S = 9 * LB_LANES;     // storage elements of one direction's links
template <class S>
__device__ __host__ constexpr int lb_link_bytes() { return 8 * LB_DIR_S * (int)sizeof(S); }
template <class S>
__device__ __host__ constexpr int lb_quarter_bytes() { return lb_link_bytes<S>() + 8 * LB_LANES * 4; }
// number of quarters of parity p of an instance with n[0], n[1] sites
__device__ __host__ __forceinline__ long long lb_quarter_base(int p, int n0) {
  return p ? (long long)LB_QUARTERS * ((n0 + LB_CHUNK - 1) / LB_CHUNK) : 0;
}

// ---- complex helpers ------------------------------------------------------------
template <class C> __device__ __forceinline__ C cmk(double re, double im);
template <> __device__ __forceinline__ double2 cmk<double2>(double re, double im) {
  return make_double2(re, im);
}
template <> __device__ __forceinline__ float2 cmk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// a + i*b and a - i*b
template <class C> __device__ __forceinline__ C caddi(C a, C b) { a.x -= b.y; a.y += b.x; return a; }
template <class C> __device__ __forceinline__ C csubi(C a, C b) { a.x += b.y; a.y -= b.x; return a; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// acc += a * b and acc += conj(a) * b
template <class C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <class C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// i*a, -i*a
template <class C> __device__ __forceinline__ C cmuli(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <class C> __device__ __forceinline__ C cmulmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// ---- one hop direction ------------------------------------------------------------
// psi: the neighbour's 12 components; U: 9 link entries (row-major a*3+b);
// FWD: (1 - gamma_mu) U psi; otherwise (1 + gamma_mu) U^+ psi; accumulated into acc.
// spin projection of a neighbour spinor onto the 2-spin half spinor of hop (MU, FWD)
template <int MU, bool FWD, class C>
__device__ __forceinline__ void hop_project(const C (&psi)[12], C (&h)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const C p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
    if (MU == 0) {
      h[0][c] = FWD ? cadd(p0, p2) : csub(p0, p2);
      h[1][c] = FWD ? cadd(p1, p3) : csub(p1, p3);
    } else if (MU == 1) {
      h[0][c] = FWD ? caddi(p0, p3) : csubi(p0, p3);
      h[1][c] = FWD ? caddi(p1, p2) : csubi(p1, p2);
    } else if (MU == 2) {
      h[0][c] = FWD ? cadd(p0, p3) : csub(p0, p3);
      h[1][c] = FWD ? csub(p1, p2) : cadd(p1, p2);
    } else {
      h[0][c] = FWD ? caddi(p0, p2) : csubi(p0, p2);
      h[1][c] = FWD ? csubi(p1, p3) : caddi(p1, p3);
    }
  }
}
// row a of (U h) for both half-spinor components, rebuilt into all four spins of acc
template <int MU, bool FWD, class C>
__device__ __forceinline__ void hop_accum_row(C (&acc)[12], int a, C u0, C u1) {
  acc[a] = cadd(acc[a], u0);
  acc[3 + a] = cadd(acc[3 + a], u1);
  if (MU == 0) {
    acc[6 + a] = FWD ? cadd(acc[6 + a], u0) : csub(acc[6 + a], u0);
    acc[9 + a] = FWD ? cadd(acc[9 + a], u1) : csub(acc[9 + a], u1);
  } else if (MU == 1) {
    acc[6 + a] = FWD ? csubi(acc[6 + a], u1) : caddi(acc[6 + a], u1);
    acc[9 + a] = FWD ? csubi(acc[9 + a], u0) : caddi(acc[9 + a], u0);
  } else if (MU == 2) {
    acc[6 + a] = FWD ? csub(acc[6 + a], u1) : cadd(acc[6 + a], u1);
    acc[9 + a] = FWD ? cadd(acc[9 + a], u0) : csub(acc[9 + a], u0);
  } else {
    acc[6 + a] = FWD ? csubi(acc[6 + a], u0) : caddi(acc[6 + a], u0);
    acc[9 + a] = FWD ? caddi(acc[9 + a], u1) : csubi(acc[9 + a], u1);
  }
}
// U (forward) or U^+ (backward) times the half spinor, rebuilt into all four spins of acc
template <int MU, bool FWD, class C>
__device__ __forceinline__ void hop_apply(C (&acc)[12], const C (&h)[2][3], const C (&U)[9]) {
  C uh[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C v = cmk<C>(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (FWD) cfma(v, U[a * 3 + b], h[s][b]);
        else cfmac(v, U[b * 3 + a], h[s][b]);
      }
      uh[s][a] = v;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) hop_accum_row<MU, FWD>(acc, a, uh[0][a], uh[1][a]);
}
template <int MU, bool FWD, class C>
__device__ __forceinline__ void hop_dir(C (&acc)[12], const C (&psi)[12], const C (&U)[9]) {
  C h[2][3];
  hop_project<MU, FWD>(psi, h);
  hop_apply<MU, FWD>(acc, h, U);
}

// v <- M v for a site-local matrix in the chiral basis: two 6x6 blocks (components
// 0..5 and 6..11), M row-major [2][6][6] (the clover term A or its inverse)
__device__ __forceinline__ void clover_mul(const double2* __restrict__ M, double2 (&v)[12]) {
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    double2 w[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const double2 m = M[ch * 36 + r * 6 + c], x = v[ch * 6 + c];
        acc.x = fma(m.x, x.x, fma(-m.y, x.y, acc.x));
        acc.y = fma(m.x, x.y, fma(m.y, x.x, acc.y));
      }
      w[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) v[ch * 6 + r] = w[r];
  }
}

// The clover blocks are hermitian (A = 1 + i kappa c_sw sigma.F with i sigma.F
// hermitian, and so its inverse), so the mixed-precision tables keep half of
// each 6x6 block.  FP32 packing per chirality block: the 6 real diagonal
// entries, then the 15 entries above the diagonal (row by row) as complex:
// 36 floats (144 B), 72 floats per site.
constexpr int CLOV_H32_FLOATS = 72;
// (v_ch <- M_ch v_ch for both blocks) from an FP32 packed table
__device__ __forceinline__ void clover_mul_h(const float4* __restrict__ M, float2 (&v)[12]) {
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    float f[36];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const float4 t = __ldg(M + ch * 9 + q);
      f[4 * q] = t.x;
      f[4 * q + 1] = t.y;
      f[4 * q + 2] = t.z;
      f[4 * q + 3] = t.w;
    }
    float2 w[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) w[r] = make_float2(f[r] * v[ch * 6 + r].x, f[r] * v[ch * 6 + r].y);
    int z = 6;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r + 1; c < 6; ++c, z += 2) {
        const float2 m = make_float2(f[z], f[z + 1]), x = v[ch * 6 + c], y = v[ch * 6 + r];
        // w_r += m v_c ; w_c += conj(m) v_r
        w[r].x = fmaf(m.x, x.x, fmaf(-m.y, x.y, w[r].x));
        w[r].y = fmaf(m.x, x.y, fmaf(m.y, x.x, w[r].y));
        w[c].x = fmaf(m.x, y.x, fmaf(m.y, y.y, w[c].x));
        w[c].y = fmaf(m.x, y.y, fmaf(-m.y, y.x, w[c].y));
      }
#pragma unroll
    for (int r = 0; r < 6; ++r) v[ch * 6 + r] = w[r];
  }
}

// ---- scalar helpers of the stencil epilogue (overloaded for double-float) ---------
template <class C> struct ScalOf;
template <> struct ScalOf<float2> { typedef float type; };
template <> struct ScalOf<double2> { typedef double type; };
template <class C> __device__ __forceinline__ typename ScalOf<C>::type mkscal(double x);
template <> __device__ __forceinline__ float mkscal<float2>(double x) { return (float)x; }
template <> __device__ __forceinline__ double mkscal<double2>(double x) { return x; }
__device__ __forceinline__ float2 scale(float2 a, float s) { return cscale(a, s); }
__device__ __forceinline__ double2 scale(double2 a, double s) { return cscale(a, s); }
__device__ __forceinline__ void axpy(float2& o, float s, float2 v) {
  o.x = fma(s, v.x, o.x);
  o.y = fma(s, v.y, o.y);
}
__device__ __forceinline__ void axpy(double2& o, double s, double2 v) {
  o.x = fma(s, v.x, o.x);
  o.y = fma(s, v.y, o.y);
}
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
// |a|^2 of one component as float (norms for convergence tests)
__device__ __forceinline__ float nrm2f(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float nrm2f(double2 a) { return (float)(a.x * a.x + a.y * a.y); }

// Warp + block reduction of NV doubles (sum); result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* sh /* >= 32*NV */) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = lane < nw ? sh[lane * NV + k] : 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
}

// Block reduction of per-thread values held in the compute type T: the warp
// stage runs in T (FP32 for the FP32 / BF16 kernels, whose FP64 pipe is
// narrow on this GPU), the cross-warp stage in FP64.  Result in thread 0.
template <class T, int NV>
__device__ __forceinline__ void block_reduce_t(T (&t)[NV], double (&v)[NV], double* sh) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp * NV + k] = (double)t[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += sh[w * NV + k];
      v[k] = a;
    }
  }
}

// ---- generated shadow residual ------------------------------------------------------
// The BiCGstab shadow vector r^ only enters inner products, and any r^ with
// (r^, r_0) != 0 is admissible.  The solver generates r^ where it is used, so
// it is never stored or read: per (seed, system, even site) a 32-bit hash h
// (the "lowbias32" integer mixer, C. Wellons 2018: xorshift-multiply rounds
// with multipliers 0x7feb352d and 0x846ca68b), then the 24 real parts of the
// site's 12 components are the Weyl sequence h + m * 0x9e3779b9 (m = 0..23,
// mod 2^32) read as signed 32-bit integers times 2^-31, i.e. values in [-1, 1)
// with 24 or more significant bits.  Entries of that kind do not cancel
// exactly against the few equal-magnitude entries of a sparse right-hand side
// (a +-1 sign vector can: (r^, r_0) = 0 and the recurrence breaks down).
// Integer arithmetic and one rounding make every kernel generate the same r^.
__device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ unsigned rhat_bits(unsigned seed, int sys, int i) {
  return mix32(mix32(seed + (unsigned)sys) + (unsigned)i);
}
template <class C>
__device__ __forceinline__ C rhat_comp(unsigned h, int k) {
  const int ur = (int)(h + (unsigned)(2 * k) * 0x9e3779b9u);
  const int ui = (int)(h + (unsigned)(2 * k + 1) * 0x9e3779b9u);
  if constexpr (std::is_same<C, double2>::value) {
    return make_double2((double)ur * 0x1p-31, (double)ui * 0x1p-31);
  } else {
    return make_float2(__int2float_rn(ur) * 0x1p-31f, __int2float_rn(ui) * 0x1p-31f);
  }
}
// the 12 components of r^ at site i of system sys (from memory when seed == 0)
template <class S, class C>
__device__ __forceinline__ void ld_rhat(unsigned seed, int sys, const S* base, long long n, long long i,
                                        C (&w)[12]) {
  if (seed) {
    const unsigned h = rhat_bits(seed, sys, (int)i);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = rhat_comp<C>(h, k);
  } else {
    ld_site<12>(base, n, i, w);
  }
}
// components 2q, 2q + 1 of r^
template <class S, class C>
__device__ __forceinline__ void ld_rhat_pair(unsigned seed, int sys, const S* base, long long n,
                                             long long i, int q, C& w0, C& w1) {
  if (seed) {
    const unsigned h = rhat_bits(seed, sys, (int)i);
    w0 = rhat_comp<C>(h, 2 * q);
    w1 = rhat_comp<C>(h, 2 * q + 1);
  } else {
    ld_pair(base + ((long long)q * n + i) * 2, w0, w1);
  }
}

}  // namespace dd

#include "dfloat.cuh"
