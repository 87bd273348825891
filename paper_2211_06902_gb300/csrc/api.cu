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
  cudaStream_t s = (cudaStream_t)stream;
  Batch* b;
  dd_status e = get_batch(c, kind, ids, nblk, nrhs, &b);
  if (e != DD_OK) return e;
  for (int j = 0; j < b->nb; ++j)
    if ((e = ensure_links(c, b->inst[j], prec)) != DD_OK) return e;
  size_t ub = 16ULL * b->user_tot;
  Staged sg;
  if ((e = stage(c, in, out, ub, 30, 31, sg, s)) != DD_OK) return e;
  size_t cb = prec_bytes(prec);
  void *ve, *vo, *oe, *oo;
  if ((e = workspace(c, 20, cb * b->tot[0], &ve)) || (e = workspace(c, 21, cb * b->tot[1], &vo)) ||
      (e = workspace(c, 22, cb * b->tot[0], &oe)) || (e = workspace(c, 23, cb * b->tot[1], &oo)))
    return e;
  if ((e = launch_pack(c, *b, sg.in, ve, vo, prec, s)) != DD_OK) return e;
  HopArgs h{};
  h.p_out = 0; h.in = vo; h.out = oe; h.s1 = ve; h.a1 = 1.0; h.b = -c->kappa;
  if ((e = launch_hop(c, *b, prec, h, s)) != DD_OK) return e;
  HopArgs g{};
  g.p_out = 1; g.in = ve; g.out = oo; g.s1 = vo; g.a1 = 1.0; g.b = -c->kappa;
  if ((e = launch_hop(c, *b, prec, g, s)) != DD_OK) return e;
  if ((e = launch_unpack(c, *b, oe, oo, sg.out, prec, s)) != DD_OK) return e;
  if ((e = unstage(c, out, ub, sg, s)) != DD_OK) return e;
  // host buffers: the call has synchronised anyway, so report a bounded wait
  // that gave up (device buffers leave it to the next synchronous call)
  return (sg.in_host || sg.out_host) ? check_device_error(c, s) : DD_OK;
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
  Staged sg;
  if ((e = stage(c, bvec, x, ub, 30, 31, sg, s)) != DD_OK) return e;
  dd_status rs = solve_batch(c, *b, sg.in, sg.out, prm, stats, s, true);
  if (rs != DD_OK && rs != DD_ENOCONV) return rs;
  if ((e = unstage(c, x, ub, sg, s)) != DD_OK) return e;
  return rs;
}

}  // extern "C"
