#include <cstdint>
#include <string>
#include <cstdio>
// Learned block preconditioner: a gauge-covariant network of linear
// parallel-transport convolutions on the framed blocks Omega0^a, trained on
// the GPU on pairs (b, D_Omega^{-1} b) produced by the library's own solver,
// and used as the initial guess of the block solves.
//
// One layer maps C_in channels of colour 3-vectors to C_out channels:
//   y_c(x) = sum_{d in {0, +-mu}} sum_c' W[d][c][c'] (T_d phi_c')(x),
//   T_0 phi = phi,  T_+mu phi(x) = U_mu(x) phi(x+mu),  T_-mu phi(x) = U_mu(x-mu)^+ phi(x-mu),
// with hops leaving the block dropped (Dirichlet) and the links' time sign as
// in D.  W never touches colour, so the layer is gauge covariant.  The
// network is 4 -> 16 -> 16 -> 16 -> 4 channels: the 4 spin components of a
// spinor in, an approximation of D_Omega^{-1} b out.  Weights are kept as FP32
// masters (Adam) and used rounded to BF16; activations and accumulation are
// FP32.  Gradients use g = dL/dRe + i dL/dIm:
//   backward data:    g_phi_c' = sum_d sum_c conj(W[d][c][c']) T_d^+ g_c,  T_+mu^+ = T_-mu
//   backward weights: G[d][c][c'] = sum_x sum_a g_c(x)_a conj((T_d phi_c')(x)_a)
// Activations use the solver's SoA layout: per system and parity,
// [channel][colour][site], offset = (12-component offset) * C / 4.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "spinor.cuh"

struct dd_net {
  int nl = 0;
  int ch[8] = {0};
  std::vector<float> master;     // FP32 complex masters, [l][9][cout][cin] (re, im)
  std::vector<float> m, v;       // Adam moments
  long long adam_t = 0;
  float* d_w = nullptr;          // BF16-rounded compute weights (FP32 complex) per layer, concatenated
  float* d_wadj = nullptr;       // adjoint weights: [d'][cin][cout] = conj(W[d][cout][cin]), d' = flip(d)
  std::vector<long long> woff;   // offset (complex) of layer l in d_w / d_wadj
  bool dirty = true;
  bool tc = true;                // layers on the tensor cores (BF16 operands), else FP32 CUDA cores
};

namespace dd {
namespace {

constexpr int NT = 128;

__device__ __forceinline__ int flip_dir(int d) { return d == 0 ? 0 : (d <= 4 ? d + 4 : d - 4); }

// forward layer (also the adjoint, with adjoint weights): output parity p
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT) k_ptconv(BatchDev bd, int p, const float2* __restrict__ in0,
                                              const float2* __restrict__ in1, float2* __restrict__ out,
                                              const float2* __restrict__ W) {
  __shared__ float2 w[9 * COUT * CIN];
  for (int k = threadIdx.x; k < 9 * COUT * CIN; k += NT) w[k] = W[k];
  __syncthreads();
  const int item = blockIdx.x / bd.nrhs, r = blockIdx.x - item * bd.nrhs;
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  if ((int)threadIdx.x >= it.z) return;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const int i = it.y + threadIdx.x;
  const long long off_p = (p ? bd.off[1] : bd.off[0])[sys];
  const long long off_q = (p ? bd.off[0] : bd.off[1])[sys];
  const float2* inp = (p ? in1 : in0) + off_p / 4 * CIN;
  const float2* inq = (p ? in0 : in1) + off_q / 4 * CIN;
  float2 acc[COUT][3];
#pragma unroll
  for (int c = 0; c < COUT; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[c][a] = make_float2(0.f, 0.f);
  // centre tap
#pragma unroll 1
  for (int cp = 0; cp < CIN; ++cp) {
    float2 v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = inp[cidx(cp * 3 + a, n_out, i)];
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
      const float2 wc = w[c * CIN + cp];
#pragma unroll
      for (int a = 0; a < 3; ++a) cfma(acc[c][a], wc, v[a]);
    }
  }
  const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
  const float2* lk = dp->link32;
#pragma unroll 1
  for (int dir = 0; dir < 8; ++dir) {
    const int j = nbr[dir * n_out + i];
    if (j < 0) continue;
    const int mu = dir & 3;
    const bool fwd = dir < 4;
    float2 U[9];
    if (fwd) ld_link(lk + link_block(p, mu, n0, n_out), n_out, i, U);
    else ld_link(lk + link_block(1 - p, mu, n0, n_in), n_in, j, U);
    const float2* wd = w + (1 + dir) * COUT * CIN;
#pragma unroll 1
    for (int cp = 0; cp < CIN; ++cp) {
      float2 v[3], tv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = inq[cidx(cp * 3 + a, n_in, j)];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        tv[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) {
          if (fwd) cfma(tv[a], U[a * 3 + b2], v[b2]);
          else cfmac(tv[a], U[b2 * 3 + a], v[b2]);
        }
      }
#pragma unroll
      for (int c = 0; c < COUT; ++c) {
        const float2 wc = wd[c * CIN + cp];
#pragma unroll
        for (int a = 0; a < 3; ++a) cfma(acc[c][a], wc, tv[a]);
      }
    }
  }
  float2* o = out + off_p / 4 * COUT;
#pragma unroll
  for (int c = 0; c < COUT; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) o[cidx(c * 3 + a, n_out, i)] = acc[c][a];
}

// ---- tensor-core form of the layer (tcgen05, BF16 operands, FP32 in TMEM) ----
// The channel mixing is a GEMM per 32-site quarter of a work item: rows are
// (colour slot a, site s) = 32 a + s, 128 rows with slot 3 zero; for tap d the
// columns are the transported input channels, real and imaginary parts
// interleaved (k = 2 c' + {0, 1}); the output columns n < COUT hold Re y_n and
// COUT <= n < 2 COUT hold Im y_{n - COUT}:
//   D[row][n] = sum_d sum_k A_d[row][k] B_d[n][k],
//   B_d[c][2c'] = Re W, B_d[c][2c'+1] = -Im W, B_d[COUT+c][2c'] = Im W, B_d[COUT+c][2c'+1] = Re W.
// SIMT threads build A_d (parallel transport of the neighbour's colour vectors,
// rounded to BF16) in one of two shared-memory buffers while the previous tap's
// MMAs run; one thread issues the MMAs (K = 16 per instruction, M = 128) and
// commits them to the buffer's mbarrier.  Operands are K-major without swizzle:
// 8 x 16-byte core matrices, k-groups 128 B apart, 8-row groups SBO apart.
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ int koff(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned k = 0; k < limit; ++k) {
    uint32_t done;
    asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, P;\n}"
                 : "=r"(done)
                 : "r"(saddr(bar)), "r"(parity)
                 : "memory");
    if (done) return true;
  }
  return false;
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t ta, float (&v)[N]);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t ta, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t ta, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

template <int CIN, int COUT>
struct Shape {
  static constexpr int KT = 2 * CIN < 16 ? 16 : 2 * CIN;       // real columns per tap (>= 16)
  static constexpr int N = 2 * COUT < 16 ? 16 : 2 * COUT;      // real output columns
  static constexpr int SBO_A = 128 * (KT / 8);
  static constexpr int SBO_B = 128 * (KT / 8);
  static constexpr int A_BYTES = 16 * SBO_A;                    // 128 rows
  static constexpr int B_TAP = (N / 8) * SBO_B;
  static constexpr int SMEM = 2 * A_BYTES + 9 * B_TAP + 64;
};

constexpr unsigned WAIT_LIMIT = 1u << 22;

}  // namespace tc

template <int CIN, int COUT>
__global__ void __launch_bounds__(128, 4) k_ptconv_tc(BatchDev bd, int p, const float2* __restrict__ in0,
                                                   const float2* __restrict__ in1, float2* __restrict__ out,
                                                   const float2* __restrict__ W, int* err) {
  typedef tc::Shape<CIN, COUT> SH;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* abuf = smem;                                   // two A buffers
  unsigned char* bmat = smem + 2 * SH::A_BYTES;                 // B of the 9 taps
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(bmat + 9 * SH::B_TAP);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 2);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int item = blockIdx.x / bd.nrhs, r = blockIdx.x - item * bd.nrhs;
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  const int sys = it.x * bd.nrhs + r;
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const long long off_p = (p ? bd.off[1] : bd.off[0])[sys];
  const long long off_q = (p ? bd.off[0] : bd.off[1])[sys];
  const float2* inp = (p ? in1 : in0) + off_p / 4 * CIN;
  const float2* inq = (p ? in0 : in1) + off_q / 4 * CIN;
  // B of every tap (BF16 of the BF16-rounded weights: exact), A buffers zeroed
  for (int e = t; e < 9 * SH::N * SH::KT; e += 128) {
    const int d = e / (SH::N * SH::KT), rem = e - d * SH::N * SH::KT;
    const int n = rem / SH::KT, k = rem - n * SH::KT;
    const int j = k >> 1, part = k & 1;
    float v = 0.f;
    if (j < CIN && n < 2 * COUT) {
      const int c = n < COUT ? n : n - COUT;
      const float2 w = W[(d * COUT + c) * CIN + j];
      v = n < COUT ? (part ? -w.y : w.x) : (part ? w.x : w.y);
    }
    *reinterpret_cast<__nv_bfloat16*>(bmat + d * SH::B_TAP + tc::koff(n, k, SH::SBO_B)) = __float2bfloat16(v);
  }
  for (int e = t; e < 2 * SH::A_BYTES / 16; e += 128) reinterpret_cast<uint4*>(abuf)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tc::saddr(tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tbase;
  const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
  const float2* lk = dp->link32;
  unsigned ncommit[2] = {0, 0};          // commits issued on each buffer's barrier (uniform)
  bool ok = true;
  const int nq = (it.z + 31) / 32;
  for (int q = 0; q < nq; ++q) {
    const int s = lane;                  // the site of this thread in the quarter
    const int li = q * 32 + s;
    const bool live = li < it.z;
    const int i = it.y + (live ? li : 0);
    for (int d = 0; d < 9; ++d) {
      const int b = d & 1;
      // the buffer is free once the MMAs of its previous tap have completed
      if (ncommit[b] > 0 && !tc::bar_wait(&bar[b], (ncommit[b] - 1) & 1, tc::WAIT_LIMIT)) ok = false;
      unsigned char* A = abuf + b * SH::A_BYTES;
      int j = -1;
      float2 U[9];
      if (live) {
        if (d == 0) {
          j = i;
        } else {
          const int dir = d - 1;
          j = nbr[dir * n_out + i];
          if (j >= 0) {
            const int mu = dir & 3;
            if (dir < 4) ld_link(lk + link_block(p, mu, n0, n_out), n_out, i, U);
            else ld_link(lk + link_block(1 - p, mu, n0, n_in), n_in, j, U);
          }
        }
      }
      for (int cp = warp; cp < CIN; cp += 4) {
        float2 tv[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (j >= 0) {
          float2 v[3];
          const float2* src = d == 0 ? inp : inq;
          const int nn = d == 0 ? n_out : n_in;
#pragma unroll
          for (int a = 0; a < 3; ++a) v[a] = src[cidx(cp * 3 + a, nn, j)];
          if (d == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) tv[a] = v[a];
          } else {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b2 = 0; b2 < 3; ++b2) {
                if (d <= 4) cfma(tv[a], U[a * 3 + b2], v[b2]);
                else cfmac(tv[a], U[b2 * 3 + a], v[b2]);
              }
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          __nv_bfloat162 h = __floats2bfloat162_rn(tv[a].x, tv[a].y);
          *reinterpret_cast<__nv_bfloat162*>(A + tc::koff(a * 32 + s, 2 * cp, SH::SBO_A)) = h;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (t == 0) {
        constexpr uint32_t id = tc::idesc_bf16(128, SH::N);
#pragma unroll
        for (int ks = 0; ks < SH::KT / 16; ++ks) {
          const uint64_t da = tc::smem_desc(tc::saddr(A) + ks * 256, 128, SH::SBO_A);
          const uint64_t db = tc::smem_desc(tc::saddr(bmat + d * SH::B_TAP) + ks * 256, 128, SH::SBO_B);
          const uint32_t acc = (d > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(id), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            tc::saddr(&bar[b])));
      }
      ++ncommit[b];
    }
    // the quarter's accumulator: wait for the last tap (its commit covers every earlier MMA)
    if (!tc::bar_wait(&bar[0], (ncommit[0] - 1) & 1, tc::WAIT_LIMIT)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp < 3 && ok) {
      float v[SH::N];
      tc::tmem_ld<SH::N>(tmem + ((uint32_t)(32 * warp) << 16), v);
      if (live) {
        float2* o = out + off_p / 4 * COUT;
#pragma unroll
        for (int c = 0; c < COUT; ++c) o[cidx(c * 3 + warp, n_out, i)] = make_float2(v[c], v[COUT + c]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok) {
    if (t == 0) atomicExch(err, 1);
    // before the accumulator is released, every MMA this CTA issued has to be done
    tc::bar_wait(&bar[0], (ncommit[0] - 1) & 1, tc::WAIT_LIMIT);
    if (ncommit[1]) tc::bar_wait(&bar[1], (ncommit[1] - 1) & 1, tc::WAIT_LIMIT);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// weight gradient partials: one CTA per (item, rhs) work unit of parity p;
// partial[unit][d][c][c'] = sum over the unit's sites and colours
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_ptconv_wgrad(BatchDev bd, int p, const float2* __restrict__ in0,
                                                      const float2* __restrict__ in1,
                                                      const float2* __restrict__ g0,
                                                      const float2* __restrict__ g1,
                                                      float2* __restrict__ partial) {
  extern __shared__ float2 sm[];
  float2* sg = sm;                       // [COUT][3][NT]
  float2* st = sm + COUT * 3 * NT;       // [CIN][3][NT]
  const int item = blockIdx.x / bd.nrhs, r = blockIdx.x - item * bd.nrhs;
  const int4 it = (p ? bd.items[1] : bd.items[0])[item];
  const int sys = it.x * bd.nrhs + r;
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n0 = dp->n[0];
  const int n_out = p ? dp->n[1] : n0, n_in = p ? n0 : dp->n[1];
  const long long off_p = (p ? bd.off[1] : bd.off[0])[sys];
  const long long off_q = (p ? bd.off[0] : bd.off[1])[sys];
  const float2* inp = (p ? in1 : in0) + off_p / 4 * CIN;
  const float2* inq = (p ? in0 : in1) + off_q / 4 * CIN;
  const float2* gp = (p ? g1 : g0) + off_p / 4 * COUT;
  const int s = threadIdx.x;
  const bool live = s < NT && s < it.z;
  const int i = it.y + s;
  if (s < NT)
    for (int c = 0; c < COUT; ++c)
      for (int a = 0; a < 3; ++a)
        sg[(c * 3 + a) * NT + s] = live ? gp[cidx(c * 3 + a, n_out, i)] : make_float2(0.f, 0.f);
  const int* nbr = dp->nbr + (p ? 8LL * n0 : 0);
  const float2* lk = dp->link32;
  for (int d = 0; d < 9; ++d) {
    __syncthreads();
    if (s < NT) {
      int j = -1;
      if (live) j = d == 0 ? i : nbr[(d - 1) * n_out + i];
      for (int cp = 0; cp < CIN; ++cp) {
        float2 tv[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (j >= 0) {
          if (d == 0) {
            for (int a = 0; a < 3; ++a) tv[a] = inp[cidx(cp * 3 + a, n_out, i)];
          } else {
            const int mu = (d - 1) & 3;
            const bool fwd = d <= 4;
            float2 v[3];
            for (int a = 0; a < 3; ++a) v[a] = inq[cidx(cp * 3 + a, n_in, j)];
            for (int a = 0; a < 3; ++a)
              for (int b2 = 0; b2 < 3; ++b2) {
                if (fwd) {
                  float2 u = lk[link_block(p, mu, n0, n_out) + cidx(a * 3 + b2, n_out, i)];
                  cfma(tv[a], u, v[b2]);
                } else {
                  float2 u = lk[link_block(1 - p, mu, n0, n_in) + cidx(b2 * 3 + a, n_in, j)];
                  cfmac(tv[a], u, v[b2]);
                }
              }
          }
        }
        for (int a = 0; a < 3; ++a) st[(cp * 3 + a) * NT + s] = tv[a];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < COUT * CIN; t += blockDim.x) {
      const int c = t / CIN, cp = t % CIN;
      float2 acc = make_float2(0.f, 0.f);
      for (int a = 0; a < 3; ++a) {
        const float2* gr = sg + (c * 3 + a) * NT;
        const float2* tr = st + (cp * 3 + a) * NT;
        for (int k = 0; k < NT; ++k) cfmac(acc, tr[k], gr[k]);   // g * conj(T phi)
      }
      partial[((long long)blockIdx.x * 9 + d) * COUT * CIN + t] = acc;
    }
  }
}

// sum of the per-unit partials (fixed order, FP64): G[k] for k < n
__global__ void k_sum_partials(const float2* __restrict__ partial, long long nunit, int n, double2* G) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double2 a = make_double2(0.0, 0.0);
  for (long long u = 0; u < nunit; ++u) {
    float2 v = partial[u * n + k];
    a.x += v.x;
    a.y += v.y;
  }
  G[k] = a;
}

// loss and output gradient: y, x spinor activations (4 channels, FP32);
// L_s = |y - x|^2 / |x|^2 per system; g = 2 (y - x) / (|x|^2 S)
__global__ void k_loss_grad(BatchDev bd, int p, const float2* __restrict__ y, const float2* __restrict__ x,
                            const double* __restrict__ xn2, double invS, float2* __restrict__ g,
                            double* __restrict__ partial) {
  __shared__ double red[32];
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n = p ? dp->n[1] : dp->n[0];
  const int i = it.y + threadIdx.x;
  const long long o = (p ? bd.off[1] : bd.off[0])[sys];
  float t[1] = {0.f};
  double v[1] = {0.0};
  if ((int)threadIdx.x < it.z) {
    const double sc = xn2[sys] > 0 ? 1.0 / xn2[sys] : 0.0;
    const float f = (float)(2.0 * sc * invS);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const long long q = o + cidx(k, n, i);
      float2 a = y[q], b = x[q];
      float2 d = make_float2(a.x - b.x, a.y - b.y);
      t[0] = fmaf(d.x, d.x, fmaf(d.y, d.y, t[0]));
      if (g) g[q] = make_float2(f * d.x, f * d.y);
    }
    t[0] = (float)(t[0] * sc * invS);
  }
  block_reduce_t<float, 1>(t, v, red);
  if (threadIdx.x == 0) partial[(long long)blockIdx.x * bd.nrhs + r] = v[0];
}

// |x|^2 per system over one parity (FP32 activations) into partial
__global__ void k_norm2_act(BatchDev bd, int p, const float2* __restrict__ x, double* partial) {
  __shared__ double red[32];
  const int4 it = (p ? bd.items[1] : bd.items[0])[blockIdx.x];
  const int r = blockIdx.y;
  const int sys = it.x * bd.nrhs + r;
  const DomInst* dp = bd.inst_tab + bd.inst[it.x];
  const int n = p ? dp->n[1] : dp->n[0];
  const int i = it.y + threadIdx.x;
  float t[1] = {0.f};
  double v[1] = {0.0};
  if ((int)threadIdx.x < it.z) {
    const long long o = (p ? bd.off[1] : bd.off[0])[sys];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      float2 a = x[o + cidx(k, n, i)];
      t[0] = fmaf(a.x, a.x, fmaf(a.y, a.y, t[0]));
    }
  }
  block_reduce_t<float, 1>(t, v, red);
  if (threadIdx.x == 0) partial[(long long)blockIdx.x * bd.nrhs + r] = v[0];
}

// per-system sums of per-item partials of both parities
__global__ void k_sum_sys(const double* pe, const double* po, const int* ib0, const int* ib1, int nb,
                          int nrhs, double* out) {
  int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nb * nrhs) return;
  int j = sys / nrhs, r = sys % nrhs;
  double a = 0.0;
  for (int k = ib0[j]; k < ib0[j + 1]; ++k) a += pe[(long long)k * nrhs + r];
  for (int k = ib1[j]; k < ib1[j + 1]; ++k) a += po[(long long)k * nrhs + r];
  out[sys] = a;
}

__global__ void k_f64_to_f32(const double2* a, float2* b, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}
// double-float (re_h, im_h, re_l, im_l) -> nearest FP32 (the high parts)
__global__ void k_df_to_f32(const float4* a, float2* b, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) {
    const float4 v = a[k];
    b[k] = make_float2(v.x, v.y);
  }
}

}  // namespace

static float bf16_round(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7fffu + lsb) & 0xffff0000u;    // round to nearest even, BF16 precision
  float y;
  memcpy(&y, &u, 4);
  return y;
}

// upload BF16-rounded compute weights and their adjoints
static dd_status upload_weights(dd_ctx* c, dd_net* n) {
  if (!n->dirty) return DD_OK;
  long long tot = n->woff.back();
  std::vector<float> w(2 * tot), wa(2 * tot);
  for (int l = 0; l < n->nl; ++l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    const long long o = n->woff[l];
    for (int d = 0; d < 9; ++d)
      for (int co = 0; co < cout; ++co)
        for (int ci = 0; ci < cin; ++ci) {
          long long k = o + ((long long)d * cout + co) * cin + ci;
          float re = bf16_round(n->master[2 * k]), im = bf16_round(n->master[2 * k + 1]);
          w[2 * k] = re;
          w[2 * k + 1] = im;
          int dflip = d == 0 ? 0 : (d <= 4 ? d + 4 : d - 4);
          long long ka = o + ((long long)dflip * cin + ci) * cout + co;
          wa[2 * ka] = re;
          wa[2 * ka + 1] = -im;
        }
  }
  DD_CUDA(c, cudaMemcpy(n->d_w, w.data(), sizeof(float) * 2 * tot, cudaMemcpyHostToDevice));
  DD_CUDA(c, cudaMemcpy(n->d_wadj, wa.data(), sizeof(float) * 2 * tot, cudaMemcpyHostToDevice));
  n->dirty = false;
  return DD_OK;
}

template <int CIN, int COUT>
static void launch_tc(unsigned grid, const BatchDev& bd, int p, const float2* in0, const float2* in1, float2* out,
                      const float2* W, int* err, cudaStream_t s) {
  constexpr int smem = tc::Shape<CIN, COUT>::SMEM;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(k_ptconv_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr[dev] = true;
  }
  DD_COUNT_LAUNCH(), k_ptconv_tc<CIN, COUT><<<grid, 128, smem, s>>>(bd, p, in0, in1, out, W, err);
}

static void launch_layer(const Batch& b, const BatchDev& bd, int p, int cin, int cout, const float2* in0,
                         const float2* in1, float2* out, const float2* W, cudaStream_t s, int* err = nullptr) {
  const unsigned grid = (unsigned)((long long)b.nitems[p] * b.nrhs);
  if (!grid) return;
  if (err) {                       // tensor cores (tcgen05), BF16 operands
    if (cin == 4 && cout == 16) launch_tc<4, 16>(grid, bd, p, in0, in1, out, W, err, s);
    else if (cin == 16 && cout == 16) launch_tc<16, 16>(grid, bd, p, in0, in1, out, W, err, s);
    else launch_tc<16, 4>(grid, bd, p, in0, in1, out, W, err, s);
    return;
  }
  if (cin == 4 && cout == 16) DD_COUNT_LAUNCH(), k_ptconv<4, 16><<<grid, NT, 0, s>>>(bd, p, in0, in1, out, W);
  else if (cin == 16 && cout == 16) DD_COUNT_LAUNCH(), k_ptconv<16, 16><<<grid, NT, 0, s>>>(bd, p, in0, in1, out, W);
  else DD_COUNT_LAUNCH(), k_ptconv<16, 4><<<grid, NT, 0, s>>>(bd, p, in0, in1, out, W);
}

static dd_status launch_wgrad(dd_ctx* c, const Batch& b, const BatchDev& bd, int p, int cin, int cout,
                              const float2* in0, const float2* in1, const float2* g0, const float2* g1,
                              float2* partial, cudaStream_t s) {
  const unsigned grid = (unsigned)((long long)b.nitems[p] * b.nrhs);
  if (!grid) return DD_OK;
  const size_t smem = sizeof(float2) * (cin + cout) * 3 * NT;
  if (cin == 4 && cout == 16) {
    DD_CUDA(c, cudaFuncSetAttribute(k_ptconv_wgrad<4, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DD_COUNT_LAUNCH(), k_ptconv_wgrad<4, 16><<<grid, 256, smem, s>>>(bd, p, in0, in1, g0, g1, partial);
  } else if (cin == 16 && cout == 16) {
    DD_CUDA(c, cudaFuncSetAttribute(k_ptconv_wgrad<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DD_COUNT_LAUNCH(), k_ptconv_wgrad<16, 16><<<grid, 256, smem, s>>>(bd, p, in0, in1, g0, g1, partial);
  } else {
    DD_CUDA(c, cudaFuncSetAttribute(k_ptconv_wgrad<16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DD_COUNT_LAUNCH(), k_ptconv_wgrad<16, 4><<<grid, 256, smem, s>>>(bd, p, in0, in1, g0, g1, partial);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// activation buffers of the batch: slot base + 2*l (+0 even, +1 odd), C = ch[l]
struct Acts {
  float2* a[8][2];
};

static dd_status alloc_acts(dd_ctx* c, const Batch& b, const dd_net* n, int slot, Acts& A) {
  for (int l = 0; l <= n->nl; ++l)
    for (int p = 0; p < 2; ++p) {
      void* q;
      dd_status e = workspace(c, slot + 2 * l + p, sizeof(float2) * (b.tot[p] / 4) * n->ch[l] + 16, &q);
      if (e != DD_OK) return e;
      A.a[l][p] = (float2*)q;
    }
  return DD_OK;
}

// N(in): in = A.a[0] (4 channels, both parities) -> A.a[nl]
static dd_status net_forward(dd_ctx* c, dd_net* n, const Batch& b, const Acts& A, cudaStream_t s) {
  dd_status e;
  if ((e = upload_weights(c, n)) != DD_OK) return e;
  if ((e = sync_instances(c)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  for (int l = 0; l < n->nl; ++l) {
    const float2* W = (const float2*)n->d_w + n->woff[l];
    for (int p = 0; p < 2; ++p)
      launch_layer(b, bd, p, n->ch[l], n->ch[l + 1], A.a[l][0], A.a[l][1], A.a[l + 1][p], W, s,
                   n->tc ? c->d_err : nullptr);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

static dd_status check_net(dd_ctx* c, dd_net* n, const Batch& b) {
  for (int j = 0; j < b.nb; ++j) {
    if (c->inst[b.inst[j]].d.kind != DD_DOMAIN_OMEGA)
      return fail(c, DD_EINVAL, "the network acts on framed blocks Omega0^a");
    dd_status e = ensure_links(c, b.inst[j], DD_F32);
    if (e != DD_OK) return e;
  }
  (void)n;
  return sync_instances(c);
}

// loss and gradients for packed pairs: b in A.a[0], targets xt (FP32, 4 ch) ; G (device FP64)
static dd_status net_loss_grad(dd_ctx* c, dd_net* n, const Batch& b, const Acts& A, const Acts& Gr,
                               const float2* const xt[2], const double* xn2, double* loss,
                               double2* G, cudaStream_t s) {
  dd_status e;
  if ((e = net_forward(c, n, b, A, s)) != DD_OK) return e;
  BatchDev bd = batch_view(c, b);
  const int nsys = b.nb * b.nrhs;
  void *vpe, *vpo, *vls;
  if ((e = workspace(c, 90, sizeof(double) * std::max<long long>(1, (long long)b.nitems[0] * b.nrhs), &vpe)) ||
      (e = workspace(c, 91, sizeof(double) * std::max<long long>(1, (long long)b.nitems[1] * b.nrhs), &vpo)) ||
      (e = workspace(c, 92, sizeof(double) * nsys, &vls)))
    return e;
  const int nl = n->nl;
  for (int p = 0; p < 2; ++p) {
    if (!b.nitems[p]) continue;
    dim3 g(b.nitems[p], b.nrhs);
    DD_COUNT_LAUNCH(), k_loss_grad<<<g, 128, 0, s>>>(bd, p, A.a[nl][p], xt[p], xn2, 1.0 / nsys, Gr.a[nl][p],
                                                     (double*)(p ? vpo : vpe));
  }
  DD_COUNT_LAUNCH(), k_sum_sys<<<(nsys + 127) / 128, 128, 0, s>>>((const double*)vpe, (const double*)vpo,
                                                                   b.d_item_begin[0], b.d_item_begin[1],
                                                                   b.nb, b.nrhs, (double*)vls);
  // weight gradients and backward data, last layer first
  const long long units0 = (long long)b.nitems[0] * b.nrhs, units1 = (long long)b.nitems[1] * b.nrhs;
  for (int l = nl - 1; l >= 0; --l) {
    const int cin = n->ch[l], cout = n->ch[l + 1], nw = 9 * cin * cout;
    void* vpart;
    if ((e = workspace(c, 93, sizeof(float2) * (units0 + units1) * nw + 16, &vpart)) != DD_OK) return e;
    float2* part = (float2*)vpart;
    if ((e = launch_wgrad(c, b, bd, 0, cin, cout, A.a[l][0], A.a[l][1], Gr.a[l + 1][0], Gr.a[l + 1][1],
                          part, s)) != DD_OK)
      return e;
    if ((e = launch_wgrad(c, b, bd, 1, cin, cout, A.a[l][0], A.a[l][1], Gr.a[l + 1][0], Gr.a[l + 1][1],
                          part + units0 * nw, s)) != DD_OK)
      return e;
    DD_COUNT_LAUNCH(), k_sum_partials<<<(nw + 127) / 128, 128, 0, s>>>(part, units0 + units1, nw, G + n->woff[l]);
    if (l > 0) {
      const float2* Wa = (const float2*)n->d_wadj + n->woff[l];
      for (int p = 0; p < 2; ++p)
        launch_layer(b, bd, p, cout, cin, Gr.a[l + 1][0], Gr.a[l + 1][1], Gr.a[l][p], Wa, s,
                     n->tc ? c->d_err : nullptr);
    }
  }
  DD_CUDA(c, cudaGetLastError());
  std::vector<double> ls(nsys);
  DD_CUDA(c, cudaMemcpyAsync(ls.data(), vls, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  double L = 0.0;
  for (double v : ls) L += v;
  *loss = L;
  return DD_OK;
}

// packs caller-layout FP64 fields of the batch into FP32 4-channel activations
static dd_status pack32(dd_ctx* c, const Batch& b, const double* user, float2* e, float2* o,
                        cudaStream_t s) {
  return launch_pack(c, b, user, e, o, DD_F32, s);
}

static dd_status target_norms(dd_ctx* c, const Batch& b, const float2* const xt[2], double* xn2,
                              cudaStream_t s) {
  BatchDev bd = batch_view(c, b);
  const int nsys = b.nb * b.nrhs;
  void *vpe, *vpo;
  dd_status e;
  if ((e = workspace(c, 90, sizeof(double) * std::max<long long>(1, (long long)b.nitems[0] * b.nrhs), &vpe)) ||
      (e = workspace(c, 91, sizeof(double) * std::max<long long>(1, (long long)b.nitems[1] * b.nrhs), &vpo)))
    return e;
  for (int p = 0; p < 2; ++p) {
    if (!b.nitems[p]) continue;
    dim3 g(b.nitems[p], b.nrhs);
    DD_COUNT_LAUNCH(), k_norm2_act<<<g, 128, 0, s>>>(bd, p, xt[p], (double*)(p ? vpo : vpe));
  }
  DD_COUNT_LAUNCH(), k_sum_sys<<<(nsys + 127) / 128, 128, 0, s>>>((const double*)vpe, (const double*)vpo,
                                                                   b.d_item_begin[0], b.d_item_begin[1],
                                                                   b.nb, b.nrhs, xn2);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

// variable preconditioner of the Schur system: z_e = [N((v_e, 0))]_even.  The
// network approximates D_Omega^{-1}, whose even-even block is the inverse of the
// Schur complement 1 - k^2 H_eo H_oe.  The input and output even vectors serve
// as the first and last activations directly (same SoA layout, 4 channels).
dd_status net_precondition(dd_ctx* c, dd_net* n, const Batch& b, const float2* ve, float2* ze,
                           cudaStream_t s) {
  dd_status e = check_net(c, n, b);
  if (e != DD_OK) return e;
  Acts A;
  if ((e = alloc_acts(c, b, n, 100, A)) != DD_OK) return e;
  void* zo;
  if ((e = workspace(c, 110, sizeof(float2) * b.tot[1] + 16, &zo)) != DD_OK) return e;
  DD_CUDA(c, cudaMemsetAsync(zo, 0, sizeof(float2) * b.tot[1], s));
  A.a[0][0] = const_cast<float2*>(ve);
  A.a[0][1] = (float2*)zo;
  A.a[n->nl][0] = ze;
  return net_forward(c, n, b, A, s);
}

// initial guess for the solver: x0 = N(b) from the solver's parity vectors
// be, bo (FP64, or double-float when `df`), written as FP32 parity vectors
// xe32, xo32
dd_status net_guess(dd_ctx* c, dd_net* n, const Batch& b, const void* be, const void* bo, bool df,
                    float2* xe32, float2* xo32, cudaStream_t s) {
  dd_status e = check_net(c, n, b);
  if (e != DD_OK) return e;
  Acts A;
  if ((e = alloc_acts(c, b, n, 100, A)) != DD_OK) return e;
  // FP64 parity vectors -> FP32 activations of layer 0 (same SoA layout)
  for (int p = 0; p < 2; ++p) {
    const long long m = b.tot[p];
    if (!m) continue;
    const unsigned g = (unsigned)((m + 255) / 256);
    const void* v = p ? bo : be;
    if (df) DD_COUNT_LAUNCH(), k_df_to_f32<<<g, 256, 0, s>>>((const float4*)v, A.a[0][p], m);
    else DD_COUNT_LAUNCH(), k_f64_to_f32<<<g, 256, 0, s>>>((const double2*)v, A.a[0][p], m);
  }
  DD_CUDA(c, cudaGetLastError());
  if ((e = net_forward(c, n, b, A, s)) != DD_OK) return e;
  DD_CUDA(c, cudaMemcpyAsync(xe32, A.a[n->nl][0], sizeof(float2) * b.tot[0], cudaMemcpyDeviceToDevice, s));
  DD_CUDA(c, cudaMemcpyAsync(xo32, A.a[n->nl][1], sizeof(float2) * b.tot[1], cudaMemcpyDeviceToDevice, s));
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_net_create(dd_ctx* c, int nlayers, const int* channels, const double* weights, dd_net** out) {
  if (!c || !channels || !weights || !out) return fail(c, DD_EINVAL, "null argument");
  if (nlayers < 1 || nlayers > 7) return fail(c, DD_EINVAL, "1..7 layers");
  if (channels[0] != 4 || channels[nlayers] != 4) return fail(c, DD_EINVAL, "first and last channel counts must be 4");
  for (int l = 0; l < nlayers; ++l) {
    int a = channels[l], b = channels[l + 1];
    if (!((a == 4 && b == 16) || (a == 16 && b == 16) || (a == 16 && b == 4)))
      return fail(c, DD_EINVAL, "supported layers: 4->16, 16->16, 16->4");
  }
  dd_net* n = new dd_net();
  n->nl = nlayers;
  n->woff.push_back(0);
  for (int l = 0; l <= nlayers; ++l) n->ch[l] = channels[l];
  for (int l = 0; l < nlayers; ++l) n->woff.push_back(n->woff.back() + 9LL * channels[l] * channels[l + 1]);
  long long tot = n->woff.back();
  n->master.resize(2 * tot);
  for (long long k = 0; k < 2 * tot; ++k) n->master[k] = (float)weights[k];
  n->m.assign(2 * tot, 0.f);
  n->v.assign(2 * tot, 0.f);
  dd_status st;
  if ((st = dalloc(c, (void**)&n->d_w, sizeof(float) * 2 * tot)) != DD_OK ||
      (st = dalloc(c, (void**)&n->d_wadj, sizeof(float) * 2 * tot)) != DD_OK) {
    dfree(n->d_w);
    delete n;
    return st;
  }
  *out = n;
  return DD_OK;
}

// File format (little-endian, as written by this library on its host):
// "DD4DNET1", int32 layers, int32 channels[layers + 1], int64 Adam step,
// then FP32 masters, Adam first and second moments (2 * complex count floats each).
static const char kNetMagic[8] = {'D', 'D', '4', 'D', 'N', 'E', 'T', '1'};

dd_status dd_net_save(const dd_net* n, const char* path) {
  if (!n || !path) return DD_EINVAL;
  FILE* f = fopen(path, "wb");
  if (!f) return DD_EINVAL;
  const int32_t nl = n->nl;
  int32_t ch[8];
  for (int l = 0; l <= nl; ++l) ch[l] = n->ch[l];
  const int64_t t = n->adam_t;
  bool ok = fwrite(kNetMagic, 1, 8, f) == 8 && fwrite(&nl, 4, 1, f) == 1 &&
            fwrite(ch, 4, nl + 1, f) == (size_t)(nl + 1) && fwrite(&t, 8, 1, f) == 1;
  const size_t m = n->master.size();
  ok = ok && fwrite(n->master.data(), 4, m, f) == m && fwrite(n->m.data(), 4, m, f) == m &&
       fwrite(n->v.data(), 4, m, f) == m;
  ok = (fclose(f) == 0) && ok;
  return ok ? DD_OK : DD_EINVAL;
}

dd_status dd_net_load(dd_ctx* c, const char* path, dd_net** out) {
  if (!c || !path || !out) return fail(c, DD_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, DD_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t nl = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kNetMagic, 8) == 0 && fread(&nl, 4, 1, f) == 1 &&
            nl >= 1 && nl <= 7;
  int32_t ch[8] = {0};
  int64_t t = 0;
  ok = ok && fread(ch, 4, nl + 1, f) == (size_t)(nl + 1) && fread(&t, 8, 1, f) == 1 && t >= 0;
  long long tot = 0;
  for (int l = 0; ok && l < nl; ++l) {
    if (ch[l] < 1 || ch[l] > 64 || ch[l + 1] < 1 || ch[l + 1] > 64) ok = false;
    else tot += 9LL * ch[l] * ch[l + 1];
  }
  std::vector<float> w(ok ? 2 * tot : 0), m1(w.size()), m2(w.size());
  ok = ok && fread(w.data(), 4, w.size(), f) == w.size() && fread(m1.data(), 4, w.size(), f) == w.size() &&
       fread(m2.data(), 4, w.size(), f) == w.size();
  fclose(f);
  if (!ok) return fail(c, DD_EINVAL, std::string("not a network file of this library: ") + path);
  std::vector<double> wd(w.begin(), w.end());     // FP32 values are exact in FP64
  int chi[8];
  for (int l = 0; l <= nl; ++l) chi[l] = ch[l];
  dd_status st = dd_net_create(c, nl, chi, wd.data(), out);
  if (st != DD_OK) return st;
  (*out)->m = m1;
  (*out)->v = m2;
  (*out)->adam_t = t;
  (*out)->dirty = true;
  return DD_OK;
}

dd_status dd_net_destroy(dd_net* n) {
  if (!n) return DD_OK;
  dfree(n->d_w);
  dfree(n->d_wadj);
  delete n;
  return DD_OK;
}

dd_status dd_net_weights(const dd_net* n, double* w) {
  if (!n || !w) return DD_EINVAL;
  for (size_t k = 0; k < n->master.size(); ++k) w[k] = n->master[k];
  return DD_OK;
}

dd_status dd_net_apply(dd_ctx* c, dd_net* n, const int* ids, int nblk, int nrhs, const double* in,
                       double* out, void* stream) {
  if (!c || !n || !in || !out) return fail(c, DD_EINVAL, "null argument");
  if (!is_device_ptr(in) || !is_device_ptr(out)) return fail(c, DD_EINVAL, "device pointers required");
  cudaStream_t s = (cudaStream_t)stream;
  Batch* b;
  dd_status e = get_batch(c, DD_DOMAIN_OMEGA, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  if ((e = check_net(c, n, *b)) != DD_OK) return e;
  Acts A;
  if ((e = alloc_acts(c, *b, n, 100, A)) != DD_OK) return e;
  if ((e = pack32(c, *b, in, A.a[0][0], A.a[0][1], s)) != DD_OK) return e;
  if ((e = net_forward(c, n, *b, A, s)) != DD_OK) return e;
  return launch_unpack(c, *b, A.a[n->nl][0], A.a[n->nl][1], out, DD_F32, s);
}

dd_status dd_net_loss_grad(dd_ctx* c, dd_net* n, const int* ids, int nblk, int nrhs, const double* bv,
                           const double* xv, double* loss, double* grads, void* stream) {
  if (!c || !n || !bv || !xv || !loss) return fail(c, DD_EINVAL, "null argument");
  if (!is_device_ptr(bv) || !is_device_ptr(xv)) return fail(c, DD_EINVAL, "device pointers required");
  cudaStream_t s = (cudaStream_t)stream;
  Batch* b;
  dd_status e = get_batch(c, DD_DOMAIN_OMEGA, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  if ((e = check_net(c, n, *b)) != DD_OK) return e;
  Acts A, Gr;
  void *vx0, *vx1, *vxn, *vG;
  const long long tot = n->woff.back();
  if ((e = alloc_acts(c, *b, n, 100, A)) || (e = alloc_acts(c, *b, n, 120, Gr)) ||
      (e = workspace(c, 94, sizeof(float2) * b->tot[0] + 16, &vx0)) ||
      (e = workspace(c, 95, sizeof(float2) * b->tot[1] + 16, &vx1)) ||
      (e = workspace(c, 96, sizeof(double) * b->nb * b->nrhs, &vxn)) ||
      (e = workspace(c, 97, sizeof(double2) * tot, &vG)))
    return e;
  if ((e = pack32(c, *b, bv, A.a[0][0], A.a[0][1], s)) != DD_OK) return e;
  if ((e = pack32(c, *b, xv, (float2*)vx0, (float2*)vx1, s)) != DD_OK) return e;
  const float2* xt[2] = {(const float2*)vx0, (const float2*)vx1};
  if ((e = target_norms(c, *b, xt, (double*)vxn, s)) != DD_OK) return e;
  if ((e = net_loss_grad(c, n, *b, A, Gr, xt, (const double*)vxn, loss, (double2*)vG, s)) != DD_OK) return e;
  if (grads) {
    DD_CUDA(c, cudaMemcpyAsync(grads, vG, sizeof(double2) * tot, cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
  }
  return DD_OK;
}

dd_status dd_net_train(dd_ctx* c, dd_net* n, const int* ids, int nblk, int nrhs, const double* bv,
                       const dd_train_params* tp, dd_train_stats* ts, void* stream) {
  if (!c || !n || !bv || !tp) return fail(c, DD_EINVAL, "null argument");
  if (!is_device_ptr(bv)) return fail(c, DD_EINVAL, "device pointer required for b");
  if (tp->steps < 1 || !(tp->lr > 0)) return fail(c, DD_EINVAL, "bad training parameters");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  Batch* b;
  dd_status e = get_batch(c, DD_DOMAIN_OMEGA, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  // training targets x = D_Omega^{-1} b from the FP64 solver
  void* vx;
  if ((e = workspace(c, 98, 16ULL * b->user_tot, &vx)) != DD_OK) return e;
  dd_solve_params sp{};
  sp.tol = tp->solve_tol > 0 ? tp->solve_tol : 1e-10;
  sp.maxiter = 5000;
  sp.inner_prec = DD_F64;
  sp.max_outer = 4;
  sp.check_every = 8;
  dd_solve_stats sst{};
  e = solve_batch(c, *b, bv, (double*)vx, &sp, &sst, s, true);
  if (e != DD_OK) return e;
  if ((e = check_net(c, n, *b)) != DD_OK) return e;
  Acts A, Gr;
  void *vx0, *vx1, *vxn, *vG;
  const long long tot = n->woff.back();
  if ((e = alloc_acts(c, *b, n, 100, A)) || (e = alloc_acts(c, *b, n, 120, Gr)) ||
      (e = workspace(c, 94, sizeof(float2) * b->tot[0] + 16, &vx0)) ||
      (e = workspace(c, 95, sizeof(float2) * b->tot[1] + 16, &vx1)) ||
      (e = workspace(c, 96, sizeof(double) * b->nb * b->nrhs, &vxn)) ||
      (e = workspace(c, 97, sizeof(double2) * tot, &vG)))
    return e;
  const float2* xt[2] = {(const float2*)vx0, (const float2*)vx1};
  if ((e = pack32(c, *b, (const double*)vx, (float2*)vx0, (float2*)vx1, s)) != DD_OK) return e;
  if ((e = target_norms(c, *b, xt, (double*)vxn, s)) != DD_OK) return e;
  // Adam (Kingma & Ba 2015) on the FP32 masters, full batch per step
  const float b1 = 0.9f, b2 = 0.999f, epsA = 1e-8f;
  std::vector<double2> G(tot);
  double first = 0.0, last = 0.0;
  for (int step = 0; step < tp->steps; ++step) {
    if ((e = pack32(c, *b, bv, A.a[0][0], A.a[0][1], s)) != DD_OK) return e;
    double L;
    if ((e = net_loss_grad(c, n, *b, A, Gr, xt, (const double*)vxn, &L, (double2*)vG, s)) != DD_OK) return e;
    if (step == 0) first = L;
    last = L;
    DD_CUDA(c, cudaMemcpyAsync(G.data(), vG, sizeof(double2) * tot, cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
    n->adam_t += 1;
    const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
    for (long long k = 0; k < tot; ++k) {
      const float g2[2] = {(float)G[k].x, (float)G[k].y};
      for (int q = 0; q < 2; ++q) {
        float& m = n->m[2 * k + q];
        float& v = n->v[2 * k + q];
        m = b1 * m + (1 - b1) * g2[q];
        v = b2 * v + (1 - b2) * g2[q] * g2[q];
        n->master[2 * k + q] -= (float)tp->lr * (m / c1) / (sqrtf(v / c2) + epsA);
      }
    }
    n->dirty = true;
  }
  // loss after the last update
  if ((e = pack32(c, *b, bv, A.a[0][0], A.a[0][1], s)) != DD_OK) return e;
  double Lf;
  if ((e = net_loss_grad(c, n, *b, A, Gr, xt, (const double*)vxn, &Lf, (double2*)vG, s)) != DD_OK) return e;
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ts) {
    ts->loss_first = first;
    ts->loss_last = Lf;
    ts->steps = tp->steps;
    ts->seconds = ms * 1e-3;
    ts->pairs = b->nb * b->nrhs;
  }
  (void)last;
  return DD_OK;
}

dd_status dd_net_tensor_cores(dd_net* n, int on) {
  if (!n) return DD_EINVAL;
  n->tc = on != 0;
  return DD_OK;
}

dd_status dd_set_net(dd_ctx* c, dd_net* n) {
  if (!c) return DD_EINVAL;
  c->net = n;
  return DD_OK;
}

}  // extern "C"
