// C ABI entry points of the stencil and the batched block solves.
#include <algorithm>
#include <sstream>

#include "internal.h"

namespace dd {

dd_status get_batch(dd_ctx* c, dd_domain kind, const int* ids, int nblk, int nrhs, Batch** out) {
  if (nrhs < 1) return fail(c, DD_EINVAL, "nrhs must be >= 1");
  std::vector<int> inst;
  if (kind == DD_DOMAIN_FULL || kind == DD_DOMAIN_LAMBDA1) {
    if (nblk != 1) return fail(c, DD_EINVAL, "FULL and LAMBDA1 take nblk = 1");
    int i;
    dd_status st = instance_of(c, kind, 0, &i);
    if (st != DD_OK) return st;
    inst.push_back(i);
  } else {
    if (nblk < 1 || !ids) return fail(c, DD_EINVAL, "block list required");
    for (int k = 0; k < nblk; ++k) {
      int i;
      dd_status st = instance_of(c, kind, ids[k], &i);
      if (st != DD_OK) return st;
      inst.push_back(i);
    }
  }
  return get_batch_insts(c, inst, nrhs, out);
}

dd_status get_batch_insts(dd_ctx* c, const std::vector<int>& inst, int nrhs, Batch** out) {
  std::ostringstream key;
  key << nrhs << ':';
  for (int i : inst) key << i << ',';
  auto it = c->batches.find(key.str());
  if (it != c->batches.end()) {
    *out = it->second.get();
    return DD_OK;
  }
  if (c->batches.size() > 64) c->batches.clear();
  std::unique_ptr<Batch> b(new Batch());
  dd_status st = make_batch(c, inst, nrhs, *b);
  if (st != DD_OK) return st;
  *out = b.get();
  c->batches[key.str()] = std::move(b);
  return DD_OK;
}

// Stages caller buffers: device pointers are used in place, host buffers go
// through work-space slots (copied in / out around the computation).
struct Staged {
  const double* in = nullptr;
  double* out = nullptr;
  bool in_host = false, out_host = false;
};

static dd_status stage(dd_ctx* c, const double* in, double* out, size_t bytes, int slot_in,
                       int slot_out, Staged& sg, cudaStream_t s) {
  sg.in_host = in && !is_device_ptr(in);
  sg.out_host = out && !is_device_ptr(out);
  dd_status e;
  if (sg.in_host) {
    void* p;
    if ((e = workspace(c, slot_in, bytes, &p)) != DD_OK) return e;
    DD_CUDA(c, cudaMemcpyAsync(p, in, bytes, cudaMemcpyHostToDevice, s));
    sg.in = (const double*)p;
  } else {
    sg.in = in;
  }
  if (sg.out_host) {
    void* p;
    if ((e = workspace(c, slot_out, bytes, &p)) != DD_OK) return e;
    sg.out = (double*)p;
  } else {
    sg.out = out;
  }
  return DD_OK;
}

static dd_status unstage(dd_ctx* c, double* out, size_t bytes, const Staged& sg, cudaStream_t s) {
  if (sg.out_host) {
    DD_CUDA(c, cudaMemcpyAsync(out, sg.out, bytes, cudaMemcpyDeviceToHost, s));
    DD_CUDA(c, cudaStreamSynchronize(s));
  } else if (sg.in_host) {
    DD_CUDA(c, cudaStreamSynchronize(s));
  }
  return DD_OK;
}

// Host-buffer solve in up to four chunks of consecutive blocks (each a
// contiguous byte range of the caller layout).  All host-to-device copies are
// queued at once on one copy stream; chunk k is solved once its copy has
// landed, and its result goes back on a second copy stream while chunk k + 1
// is solved, so only the first copy in and the last copy out are not hidden.
static dd_status solve_pipelined(dd_ctx* c, dd_domain kind, const int* ids, int nblk, int nrhs,
                                 const double* bvec, double* x, size_t ub, const dd_solve_params* prm,
                                 dd_solve_stats* stats, cudaStream_t s) {
  dd_status e;
  const int K = (int)std::max<size_t>(2, std::min<size_t>({4, (size_t)nblk, ub / (64ULL << 20)}));
  void *din, *dout;
  if ((e = workspace(c, 30, ub, &din)) != DD_OK || (e = workspace(c, 31, ub, &dout)) != DD_OK) return e;
  if (!c->copy_in) DD_CUDA(c, cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking));
  if (!c->copy_out) DD_CUDA(c, cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));
  // (batches are looked up again right before their solve: the batch cache may
  // drop entries when it grows, so no pointer is kept across lookups)
  std::vector<int> j0(K + 1);
  std::vector<size_t> off(K + 1, 0);
  for (int k = 0; k <= K; ++k) j0[k] = (int)((long long)nblk * k / K);
  for (int k = 0; k < K; ++k) {
    Batch* bk;
    if ((e = get_batch(c, kind, ids + j0[k], j0[k + 1] - j0[k], nrhs, &bk)) != DD_OK) return e;
    off[k + 1] = off[k] + 16ULL * bk->user_tot;
  }
  if (off[K] != ub) return fail(c, DD_EINVAL, "internal: chunk sizes do not add up");
  std::vector<cudaEvent_t> ev(2 * K, nullptr);
  for (auto& v : ev) DD_CUDA(c, cudaEventCreateWithFlags(&v, cudaEventDisableTiming));
  // the copy stream must not start before work the caller queued on s
  cudaEvent_t start = nullptr;
  DD_CUDA(c, cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  DD_CUDA(c, cudaEventRecord(start, s));
  DD_CUDA(c, cudaStreamWaitEvent(c->copy_in, start, 0));
  for (int k = 0; k < K; ++k) {
    DD_CUDA(c, cudaMemcpyAsync((char*)din + off[k], (const char*)bvec + off[k], off[k + 1] - off[k],
                               cudaMemcpyHostToDevice, c->copy_in));
    DD_CUDA(c, cudaEventRecord(ev[k], c->copy_in));
  }
  dd_solve_stats tot{};
  dd_status rs = DD_OK;
  double seconds = 0.0;
  for (int k = 0; k < K && (rs == DD_OK || rs == DD_ENOCONV); ++k) {
    DD_CUDA(c, cudaStreamWaitEvent(s, ev[k], 0));
    Batch* bk;
    if ((e = get_batch(c, kind, ids + j0[k], j0[k + 1] - j0[k], nrhs, &bk)) != DD_OK) {
      rs = e;
      break;
    }
    dd_solve_stats st{};
    dd_status r = solve_batch(c, *bk, (const double*)((char*)din + off[k]), (double*)((char*)dout + off[k]),
                              prm, &st, s, true);
    if (r != DD_OK && r != DD_ENOCONV) {
      rs = r;
      break;
    }
    if (r == DD_ENOCONV) rs = DD_ENOCONV;
    DD_CUDA(c, cudaEventRecord(ev[K + k], s));
    DD_CUDA(c, cudaStreamWaitEvent(c->copy_out, ev[K + k], 0));
    DD_CUDA(c, cudaMemcpyAsync((char*)x + off[k], (char*)dout + off[k], off[k + 1] - off[k],
                               cudaMemcpyDeviceToHost, c->copy_out));
    tot.systems += st.systems;
    tot.converged += st.converged;
    tot.max_iters = std::max(tot.max_iters, st.max_iters);
    tot.outer_cycles = std::max(tot.outer_cycles, st.outer_cycles);
    tot.max_relres = std::max(tot.max_relres, st.max_relres);
    tot.hop_variant = st.hop_variant;
    seconds += st.seconds;
  }
  // every copy has finished before the caller may touch b or x again
  cudaStreamSynchronize(c->copy_in);
  cudaStreamSynchronize(c->copy_out);
  for (auto& v : ev) cudaEventDestroy(v);
  cudaEventDestroy(start);
  tot.seconds = seconds;
  if (stats) *stats = tot;
  c->last_stats = tot;
  if (rs != DD_OK && rs != DD_ENOCONV) return rs;
  if (rs == DD_ENOCONV) {
    char buf[160];
    snprintf(buf, sizeof buf, "%d of %d systems above tolerance (max relres %.3e)", tot.systems - tot.converged,
             tot.systems, tot.max_relres);
    return fail(c, DD_ENOCONV, buf);
  }
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_last_solve_stats(const dd_ctx* c, dd_solve_stats* st) {
  if (!c || !st) return DD_EINVAL;
  *st = c->last_stats;
  return DD_OK;
}

dd_status dd_apply_D_block(dd_ctx* c, dd_domain kind, const int* ids, int nblk, int nrhs,
                           const double* in, double* out, dd_prec prec, void* stream) {
  if (!c || !in || !out) return fail(c, DD_EINVAL, "null argument");
  if (prec != DD_F64 && prec != DD_F32 && prec != DD_BF16) return fail(c, DD_EINVAL, "bad precision");
  if (c->csw != 0.0 && prec != DD_F64) return fail(c, DD_EINVAL, "the clover term is applied in FP64 only");
  cudaStream_t s = (cudaStream_t)stream;
  Batch* b;
  dd_status e = get_batch(c, kind, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  for (int j = 0; j < b->nb; ++j)
    if ((e = ensure_links(c, b->inst[j], prec)) != DD_OK) return e;
  if (c->csw != 0.0 && !c->clover_ready && (e = clover_build(c)) != DD_OK) return e;
  size_t ub = 16ULL * b->user_tot;
  Staged sg;
  if ((e = stage(c, in, out, ub, 30, 31, sg, s)) != DD_OK) return e;
  size_t cb = prec_bytes(prec);
  void *ve, *vo, *oe, *oo;
  if ((e = workspace(c, 20, cb * b->tot[0], &ve)) || (e = workspace(c, 21, cb * b->tot[1], &vo)) ||
      (e = workspace(c, 22, cb * b->tot[0], &oe)) || (e = workspace(c, 23, cb * b->tot[1], &oo)))
    return e;
  if ((e = launch_pack(c, *b, sg.in, ve, vo, prec, s)) != DD_OK) return e;
  // the self term: psi, or A psi with the clover term (site-local, FP64)
  const void *se = ve, *so = vo;
  if (c->csw != 0.0) {
    void *ae, *ao;
    if ((e = workspace(c, 240, cb * b->tot[0], &ae)) || (e = workspace(c, 241, cb * b->tot[1], &ao)))
      return e;
    DD_CUDA(c, cudaMemcpyAsync(ae, ve, cb * b->tot[0], cudaMemcpyDeviceToDevice, s));
    if (b->tot[1] > 0) DD_CUDA(c, cudaMemcpyAsync(ao, vo, cb * b->tot[1], cudaMemcpyDeviceToDevice, s));
    if ((e = clover_apply(c, *b, ae, ao, false, s)) != DD_OK) return e;
    se = ae;
    so = ao;
  }
  HopArgs h{};
  h.p_out = 0; h.in = vo; h.out = oe; h.s1 = se; h.a1 = 1.0; h.b = -c->kappa;
  if ((e = launch_hop(c, *b, prec, h, s)) != DD_OK) return e;
  HopArgs g{};
  g.p_out = 1; g.in = ve; g.out = oo; g.s1 = so; g.a1 = 1.0; g.b = -c->kappa;
  if ((e = launch_hop(c, *b, prec, g, s)) != DD_OK) return e;
  if ((e = launch_unpack(c, *b, oe, oo, sg.out, prec, s)) != DD_OK) return e;
  if ((e = unstage(c, out, ub, sg, s)) != DD_OK) return e;
  // host buffers: the call has synchronised anyway, so report a bounded wait
  // that gave up (device buffers leave it to the next synchronous call)
  return (sg.in_host || sg.out_host) ? check_device_error(c, s) : DD_OK;
}

}  // extern "C"

namespace {
// FP64 FMA throughput probe: 8 independent dependency chains per thread, the
// result kept live through one conditional store
constexpr int FP64_CHAINS = 8;
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* sink) {
  double v[FP64_CHAINS];
#pragma unroll
  for (int k = 0; k < FP64_CHAINS; ++k) v[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FP64_CHAINS; ++k) v[k] = fma(v[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < FP64_CHAINS; ++k) s += v[k];
  if (s == 1.2345e-300) sink[0] = s;
}
}  // namespace

extern "C" {

dd_status dd_fp64_fma_rate(double* tflops) {
  if (!tflops) return DD_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return DD_ECUDA;
  const int blocks = nsm * 8, threads = 256, iters = 1 << 14;
  dd::EventPair ev;
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {      // the first launch warms up
    cudaEventRecord(ev.a, 0);
    DD_COUNT_LAUNCH(), k_fp64_fma<<<blocks, threads>>>(iters, 0.999999, 1e-7, nullptr);
    cudaEventRecord(ev.b, 0);
    if (cudaEventSynchronize(ev.b) != cudaSuccess) return DD_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    const double flops = 2.0 * FP64_CHAINS * (double)iters * blocks * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (cudaGetLastError() != cudaSuccess) return DD_ECUDA;
  *tflops = best;
  return DD_OK;
}

dd_status dd_solve_blocks(dd_ctx* c, dd_domain kind, const int* ids, int nblk, int nrhs,
                          const double* bvec, double* x, const dd_solve_params* prm,
                          dd_solve_stats* stats, void* stream) {
  if (!c || !bvec || !x || !prm) return fail(c, DD_EINVAL, "null argument");
  if (!(prm->tol > 0) || prm->maxiter < 1) return fail(c, DD_EINVAL, "bad solver parameters");
  if (prm->inner_prec != DD_F64 && prm->inner_prec != DD_F32 && prm->inner_prec != DD_BF16)
    return fail(c, DD_EINVAL, "bad inner precision");
  if (prm->inner_prec != DD_F64 && !(prm->inner_tol > 0 && prm->inner_tol < 1))
    return fail(c, DD_EINVAL, "inner_tol must be in (0, 1)");
  cudaStream_t s = (cudaStream_t)stream;
  Batch* b;
  dd_status e = get_batch(c, kind, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  size_t ub = 16ULL * b->user_tot;
  if ((kind == DD_DOMAIN_OMEGA || kind == DD_DOMAIN_PHI) && nblk >= 2 && is_pinned_host_ptr(bvec) &&
      is_pinned_host_ptr(x) && ((prm->flags & DD_SOLVE_PIPELINE) || ub >= (256ULL << 20)))
    return solve_pipelined(c, kind, ids, nblk, nrhs, bvec, x, ub, prm, stats, s);
  Staged sg;
  if ((e = stage(c, bvec, x, ub, 30, 31, sg, s)) != DD_OK) return e;
  dd_status rs = solve_batch(c, *b, sg.in, sg.out, prm, stats, s, true);
  if (rs != DD_OK && rs != DD_ENOCONV) return rs;
  if ((e = unstage(c, x, ub, sg, s)) != DD_OK) return e;
  return rs;
}

}  // extern "C"
