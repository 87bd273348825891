// dd_apply_D_block_noalloc: the FP64 restricted stencil out = D_X in without
// any device allocation.
//
// Who needs it: callers that must not call cudaMalloc from inside the call,
// for example code running while another component owns the allocator (a
// caching allocator that must see every allocation, or a memory budget that
// is fixed up front), code that cannot afford the implicit synchronisation
// of cudaMalloc / cudaFree, or a host that pre-plans its memory once and
// then only launches work.  dd_apply_D_block grows per-context work buffers
// on demand; this variant instead takes its scratch (the even / odd packed
// copies of the input and output and the launch descriptors) from one
// file-scope device array of DD_NOALLOC_SCRATCH_BYTES, reads the links
// straight from the context's global FP64 gauge copy, and rejects requests
// that do not fit.
//
// The array exists once per GPU that loads this module and stays allocated
// until the process exits.  Every call shares it and leaves its contents
// behind; nothing in it has to start at zero, because each call writes every
// word it later reads.  Calls whose GPU work overlaps (different streams, or
// different host threads) race on the array: serialise them.  The first call
// on a device resolves the array's device address with cudaGetSymbolAddress
// (once per device, with that device current); with lazy module loading that
// first call also loads this module on the device and commits the array, so it
// is the one call that takes device memory.
//
// The launch descriptors are written into a host staging buffer shared by all
// calls and devices and copied with cudaMemcpyAsync; a lock serialises the
// staging between host threads until the copy has taken the bytes (a copy from
// pageable memory returns once its source has been read).  A memcpy recorded
// into a CUDA graph would instead read the buffer when the graph is launched,
// after later calls may have rewritten it, so a call on a stream that is being
// captured returns DD_EINVAL.
#include <cstring>
#include <mutex>

#include "internal.h"
#include "spinor.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)DD_NOALLOC_SCRATCH_BYTES;
constexpr size_t kDescBytes = 1u << 20;      // launch descriptors (host staging size)
constexpr int kMaxDevices = 64;
constexpr int kThreads = 128;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch per device (host code must not use the symbol itself)
static void* g_scratch_addr[kMaxDevices];
// host staging of the descriptors (copied into the scratch on the call's stream),
// guarded by g_desc_lock from the first write until the copy has read it
static unsigned char g_desc_host[kDescBytes];
static std::mutex g_desc_lock;

struct NaView {
  const dd::DomInst* inst;     // [nb]
  const long long* off[2];     // [nb*nrhs] per parity (complex elements)
  const long long* uoff;       // [nb*nrhs] caller layout
  const int4* items[2];        // {j, start, count, 0}
  int nitems[2];
  int nrhs;
};

__global__ void k_na_pack(NaView v, int p, const double2* __restrict__ user, double2* __restrict__ dst) {
  const int item = blockIdx.x / v.nrhs, r = blockIdx.x - item * v.nrhs;
  const int4 it = (p ? v.items[1] : v.items[0])[item];
  if ((int)threadIdx.x >= it.z) return;
  const int sys = it.x * v.nrhs + r;
  const dd::DomInst* d = v.inst + it.x;
  const int n0 = d->n[0], np = p ? d->n[1] : n0;
  const int i = it.y + threadIdx.x;
  const int f = d->fmap[(p ? n0 : 0) + i];
  const double2* src = user + v.uoff[sys] + 12LL * f;
  double2* o = dst + (p ? v.off[1] : v.off[0])[sys] + i;
#pragma unroll
  for (int k = 0; k < 12; ++k) o[(long long)k * np] = src[k];
}

__global__ void k_na_unpack(NaView v, int p, const double2* __restrict__ src, double2* __restrict__ user) {
  const int item = blockIdx.x / v.nrhs, r = blockIdx.x - item * v.nrhs;
  const int4 it = (p ? v.items[1] : v.items[0])[item];
  if ((int)threadIdx.x >= it.z) return;
  const int sys = it.x * v.nrhs + r;
  const dd::DomInst* d = v.inst + it.x;
  const int n0 = d->n[0], np = p ? d->n[1] : n0;
  const int i = it.y + threadIdx.x;
  const int f = d->fmap[(p ? n0 : 0) + i];
  double2* o = user + v.uoff[sys] + 12LL * f;
  const double2* s = src + (p ? v.off[1] : v.off[0])[sys] + i;
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = s[(long long)k * np];
}

template <int DIR>
__device__ __forceinline__ void na_hop(double2 (&acc)[12], const double2* __restrict__ U, int gx,
                                       const int* __restrict__ glob_in, int j, int n_in,
                                       const double2* __restrict__ in_sys) {
  if (j < 0) return;
  constexpr int MU = DIR & 3;
  constexpr bool FWD = DIR < 4;
  double2 psi[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) psi[k] = in_sys[(long long)k * n_in + j];
  const int g = FWD ? gx : glob_in[j];      // U_mu(x) forward, U_mu(x - mu) backward
  const double2* l = U + (long long)g * 36 + MU * 9;
  double2 u[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) u[c] = l[c];
  dd::hop_dir<MU, FWD>(acc, psi, u);
}

// out_p = in_p - kappa H_{p,1-p} in_{1-p}, links from the global FP64 copy
__global__ void k_na_hop(NaView v, int p, const double2* __restrict__ U, const double2* __restrict__ vin_p,
                         const double2* __restrict__ vin_q, double2* __restrict__ vout, double kappa) {
  const int item = blockIdx.x / v.nrhs, r = blockIdx.x - item * v.nrhs;
  const int4 it = (p ? v.items[1] : v.items[0])[item];
  if ((int)threadIdx.x >= it.z) return;
  const int sys = it.x * v.nrhs + r;
  const dd::DomInst* d = v.inst + it.x;
  const int n0 = d->n[0];
  const int n_out = p ? d->n[1] : n0, n_in = p ? n0 : d->n[1];
  const int i = it.y + threadIdx.x;
  const int* nbr = d->nbr + (p ? 8LL * n0 : 0);
  const int gx = d->glob[(p ? n0 : 0) + i];
  const int* glob_in = d->glob + (p ? 0 : n0);
  const double2* in_sys = vin_q + (p ? v.off[0] : v.off[1])[sys];
  double2 acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = make_double2(0.0, 0.0);
  na_hop<0>(acc, U, gx, glob_in, nbr[0 * n_out + i], n_in, in_sys);
  na_hop<1>(acc, U, gx, glob_in, nbr[1 * n_out + i], n_in, in_sys);
  na_hop<2>(acc, U, gx, glob_in, nbr[2 * n_out + i], n_in, in_sys);
  na_hop<3>(acc, U, gx, glob_in, nbr[3 * n_out + i], n_in, in_sys);
  na_hop<4>(acc, U, gx, glob_in, nbr[4 * n_out + i], n_in, in_sys);
  na_hop<5>(acc, U, gx, glob_in, nbr[5 * n_out + i], n_in, in_sys);
  na_hop<6>(acc, U, gx, glob_in, nbr[6 * n_out + i], n_in, in_sys);
  na_hop<7>(acc, U, gx, glob_in, nbr[7 * n_out + i], n_in, in_sys);
  const long long o = (p ? v.off[1] : v.off[0])[sys] + i;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const double2 s = vin_p[o + (long long)k * n_out];
    vout[o + (long long)k * n_out] = make_double2(s.x - kappa * acc[k].x, s.y - kappa * acc[k].y);
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

using namespace dd;

extern "C" dd_status dd_apply_D_block_noalloc(dd_ctx* c, dd_domain kind, const int* ids, int nblk,
                                              int nrhs, const double* in, double* out,
                                              void* stream) {
  if (!c || !in || !out) return fail(c, DD_EINVAL, "null argument");
  if (nrhs < 1) return fail(c, DD_EINVAL, "nrhs must be >= 1");
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  if (c->csw != 0.0) return fail(c, DD_EINVAL, "dd_apply_D_block_noalloc has no clover term");
  if (!is_device_ptr(in) || !is_device_ptr(out))
    return fail(c, DD_EINVAL, "dd_apply_D_block_noalloc takes device pointers only");
  // instances (no lazily built ones: those would allocate)
  const int nb = (kind == DD_DOMAIN_FULL || kind == DD_DOMAIN_LAMBDA1) ? 1 : nblk;
  if (nb < 1) return fail(c, DD_EINVAL, "block list required");
  if (kind == DD_DOMAIN_PHI && c->phi0 < 0)
    return fail(c, DD_EINVAL, "Phi1 domains are built on first use by dd_apply_D_block or "
                              "dd_solve_blocks; the no-alloc entry point cannot build them");
  if (kind == DD_DOMAIN_OMEGA || kind == DD_DOMAIN_PHI) {
    if (!ids) return fail(c, DD_EINVAL, "block list required");
    if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  } else if (kind == DD_DOMAIN_LAMBDA1) {
    if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
    if (nblk != 1) return fail(c, DD_EINVAL, "LAMBDA1 takes nblk = 1");
  } else if (kind == DD_DOMAIN_FULL) {
    if (nblk != 1) return fail(c, DD_EINVAL, "FULL takes nblk = 1");
  } else {
    return fail(c, DD_EINVAL, "unknown domain kind");
  }
  // sizes and descriptor layout (host staging buffer, then one copy)
  long long tot[2] = {0, 0};
  int nitems[2] = {0, 0};
  for (int j = 0; j < nb; ++j) {
    int idx = kind == DD_DOMAIN_FULL ? 0
              : kind == DD_DOMAIN_LAMBDA1 ? c->lambda1
              : ((ids[j] < 0 || ids[j] >= (int)c->blocks.size()) ? -1
                 : (kind == DD_DOMAIN_OMEGA ? c->omega0 : c->phi0) + ids[j]);
    if (idx < 0) return fail(c, DD_EINVAL, "block id out of range");
    const DomInst& d = c->inst[idx].d;
    for (int p = 0; p < 2; ++p) {
      tot[p] += 12LL * d.n[p] * nrhs;
      nitems[p] += (d.n[p] + kThreads - 1) / kThreads;
    }
  }
  const long long nsys = (long long)nb * nrhs;
  size_t o_inst = 0;
  size_t o_off0 = align256(o_inst + sizeof(DomInst) * nb);
  size_t o_off1 = align256(o_off0 + sizeof(long long) * nsys);
  size_t o_uoff = align256(o_off1 + sizeof(long long) * nsys);
  size_t o_it0 = align256(o_uoff + sizeof(long long) * nsys);
  size_t o_it1 = align256(o_it0 + sizeof(int4) * nitems[0]);
  size_t desc = align256(o_it1 + sizeof(int4) * nitems[1]);
  size_t o_ve = desc;
  size_t o_vo = align256(o_ve + 16 * (size_t)tot[0]);
  size_t o_oe = align256(o_vo + 16 * (size_t)tot[1]);
  size_t o_oo = align256(o_oe + 16 * (size_t)tot[0]);
  size_t need = align256(o_oo + 16 * (size_t)tot[1]);
  if (desc > kDescBytes || need > kScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "request needs %zu bytes of scratch (%zu of descriptors); the no-alloc entry "
             "point has %zu (%zu)", need, desc, kScratchBytes, kDescBytes);
    return fail(c, DD_EINVAL, buf);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DD_CUDA(c, cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(c, DD_EINVAL, "dd_apply_D_block_noalloc stages its launch descriptors through a "
                              "host buffer and does not run on a stream that is being captured");
  // one-time per device: device address of the scratch array
  int dev = 0;
  DD_CUDA(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(c, DD_EINVAL, "device ordinal out of range");
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(c, e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_scratch_addr[dev];
  std::unique_lock<std::mutex> staging(g_desc_lock);
  unsigned char* h = g_desc_host;
  DomInst* hi = (DomInst*)(h + o_inst);
  long long* hoff0 = (long long*)(h + o_off0);
  long long* hoff1 = (long long*)(h + o_off1);
  long long* huoff = (long long*)(h + o_uoff);
  int4* hit0 = (int4*)(h + o_it0);
  int4* hit1 = (int4*)(h + o_it1);
  long long t0 = 0, t1 = 0, ut = 0;
  int k0 = 0, k1 = 0;
  for (int j = 0; j < nb; ++j) {
    int idx = kind == DD_DOMAIN_FULL ? 0
              : kind == DD_DOMAIN_LAMBDA1 ? c->lambda1
              : (kind == DD_DOMAIN_OMEGA ? c->omega0 : c->phi0) + ids[j];
    const DomInst& d = c->inst[idx].d;
    hi[j] = d;
    for (int r = 0; r < nrhs; ++r) {
      hoff0[j * nrhs + r] = t0;
      hoff1[j * nrhs + r] = t1;
      huoff[j * nrhs + r] = ut;
      t0 += 12LL * d.n[0];
      t1 += 12LL * d.n[1];
      ut += 12LL * d.nsites;
    }
    for (int s = 0; s < d.n[0]; s += kThreads)
      hit0[k0++] = make_int4(j, s, d.n[0] - s < kThreads ? d.n[0] - s : kThreads, 0);
    for (int s = 0; s < d.n[1]; s += kThreads)
      hit1[k1++] = make_int4(j, s, d.n[1] - s < kThreads ? d.n[1] - s : kThreads, 0);
  }
  DD_CUDA(c, cudaMemcpyAsync(base, h, desc, cudaMemcpyHostToDevice, s));
  staging.unlock();
  NaView v;
  v.inst = (const DomInst*)(base + o_inst);
  v.off[0] = (const long long*)(base + o_off0);
  v.off[1] = (const long long*)(base + o_off1);
  v.uoff = (const long long*)(base + o_uoff);
  v.items[0] = (const int4*)(base + o_it0);
  v.items[1] = (const int4*)(base + o_it1);
  v.nitems[0] = nitems[0];
  v.nitems[1] = nitems[1];
  v.nrhs = nrhs;
  double2* ve = (double2*)(base + o_ve);
  double2* vo = (double2*)(base + o_vo);
  double2* oe = (double2*)(base + o_oe);
  double2* oo = (double2*)(base + o_oo);
  for (int p = 0; p < 2; ++p)
    if (nitems[p]) DD_COUNT_LAUNCH(), k_na_pack<<<nitems[p] * nrhs, kThreads, 0, s>>>(v, p, (const double2*)in, p ? vo : ve);
  if (nitems[0]) DD_COUNT_LAUNCH(), k_na_hop<<<nitems[0] * nrhs, kThreads, 0, s>>>(v, 0, c->d_U, ve, vo, oe, c->kappa);
  if (nitems[1]) DD_COUNT_LAUNCH(), k_na_hop<<<nitems[1] * nrhs, kThreads, 0, s>>>(v, 1, c->d_U, vo, ve, oo, c->kappa);
  for (int p = 0; p < 2; ++p)
    if (nitems[p]) DD_COUNT_LAUNCH(), k_na_unpack<<<nitems[p] * nrhs, kThreads, 0, s>>>(v, p, p ? oo : oe, (double2*)out);
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}
