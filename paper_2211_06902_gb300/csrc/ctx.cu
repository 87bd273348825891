// Context, errors, gauge field, geometry (paper Sec. 2) and domain instances.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <sstream>

#include "internal.h"
#include "spinor.cuh"

namespace dd {

std::atomic<long long> g_launches{0};

dd_status fail(dd_ctx* c, dd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

dd_status cuda_fail(dd_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, DD_ENOMEM, m);
  return fail(c, DD_ECUDA, m);
}

dd_status dalloc(dd_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return DD_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool is_pinned_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

size_t prec_bytes(dd_prec p) { return (p == DD_F64 || p == DD_DF64) ? 16 : (p == DD_F32 ? 8 : 4); }

Batch::~Batch() {
  for (auto& g : graphs) cudaGraphExecDestroy(g.second);
  dfree(d_inst);
  dfree(d_uoff);
  for (int p = 0; p < 2; ++p) {
    dfree(d_off[p]);
    dfree(d_items[p]);
    dfree(d_item_begin[p]);
  }
  dfree(d_fitems);
}

// ---------------------------------------------------------------------------
// instance construction

namespace {

struct Shape {
  int n[2];
  std::vector<int> nbr;    // [p][8][n_p]
  std::vector<int> fmap;   // [p][n_p]
  std::vector<int> lex;    // [p][n_p]
  std::vector<int> ifm;    // [field position] -> (p << 30) | i
};

// Builds the per-parity site lists and neighbour tables of a set of sites
// inside a box of extents dims (periodic = wrap at the box edges, which is
// used only when the box is the whole lattice).  Parity is local (sum of box
// coordinates) plus parity_shift.
template <class Member>
// periodic: bit mu set = the box wraps around in direction mu (it spans the
// lattice's whole extent there); otherwise hops leaving the box are dropped
Shape build_shape(const int dims[4], int periodic, int parity_shift, Member member) {
  Shape sh;
  long long nloc = 1LL * dims[0] * dims[1] * dims[2] * dims[3];
  std::vector<int> eo(nloc, -1), par(nloc, 0);
  std::vector<int> list[2];
  int rank = 0;
  std::vector<int> fpos(nloc, -1);
  for (long long s = 0; s < nloc; ++s) {
    if (!member(s)) continue;
    int x3 = s % dims[3], x2 = (s / dims[3]) % dims[2];
    int x1 = (s / (1LL * dims[3] * dims[2])) % dims[1];
    int x0 = s / (1LL * dims[3] * dims[2] * dims[1]);
    int p = (x0 + x1 + x2 + x3 + parity_shift) & 1;
    par[s] = p;
    eo[s] = (int)list[p].size();
    list[p].push_back((int)s);
    fpos[s] = rank++;
  }
  sh.n[0] = (int)list[0].size();
  sh.n[1] = (int)list[1].size();
  sh.nbr.assign(8LL * (sh.n[0] + sh.n[1]), -1);
  sh.fmap.resize(sh.n[0] + sh.n[1]);
  sh.lex.resize(sh.n[0] + sh.n[1]);
  sh.ifm.resize(sh.n[0] + sh.n[1]);
  for (int p = 0; p < 2; ++p) {
    int np = sh.n[p];
    long long nb_base = p ? 8LL * sh.n[0] : 0;
    int m_base = p ? sh.n[0] : 0;
    for (int i = 0; i < np; ++i) {
      long long s = list[p][i];
      int x[4];
      x[3] = s % dims[3];
      x[2] = (s / dims[3]) % dims[2];
      x[1] = (s / (1LL * dims[3] * dims[2])) % dims[1];
      x[0] = s / (1LL * dims[3] * dims[2] * dims[1]);
      sh.fmap[m_base + i] = fpos[s];
      sh.lex[m_base + i] = (int)s;
      sh.ifm[fpos[s]] = (p << 30) | i;
      for (int dir = 0; dir < 8; ++dir) {
        int mu = dir & 3, step = dir < 4 ? 1 : -1;
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] += step;
        if (y[mu] < 0 || y[mu] >= dims[mu]) {
          if (!((periodic >> mu) & 1)) continue;
          y[mu] = (y[mu] + dims[mu]) % dims[mu];
        }
        long long t = ((1LL * y[0] * dims[1] + y[1]) * dims[2] + y[2]) * dims[3] + y[3];
        if (eo[t] < 0) continue;
        sh.nbr[nb_base + 1LL * dir * np + i] = eo[t];
      }
    }
  }
  return sh;
}

template <class T>
std::shared_ptr<void> upload_shared(dd_ctx* c, const std::vector<T>& h, dd_status* st) {
  void* p = nullptr;
  *st = dalloc(c, &p, h.size() * sizeof(T));
  if (*st != DD_OK) return nullptr;
  cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return std::shared_ptr<void>(p, [](void* q) { dfree(q); });
}

void free_instance(Instance& in) {
  dfree(in.glob_buf);
  dfree(in.link64_buf);
  dfree(in.link32_buf);
  dfree(in.link16_buf);
  dfree(in.linkdf_buf);
  dfree(in.lb32_buf);
  dfree(in.lb16_buf);
  in.glob_buf = in.link64_buf = in.link32_buf = in.link16_buf = in.linkdf_buf = nullptr;
  in.lb32_buf = in.lb16_buf = nullptr;
  in.nbr_buf.reset();
  in.ifm_buf.reset();
  in.fmap_buf.reset();
  in.lex_buf.reset();
}

// Creates an instance for the site set `member` inside the box (dims, origin).
template <class Member>
dd_status add_instance(dd_ctx* c, int kind, int block, const int dims[4], const int origin[4],
                       int periodic, int parity_shift, const std::string& key, Member member,
                       int* out_index) {
  Instance in;
  in.block = block;
  in.d.kind = kind;
  for (int m = 0; m < 4; ++m) {
    in.d.dims[m] = dims[m];
    in.d.origin[m] = origin[m];
  }
  dd_status st = DD_OK;
  auto it = c->shape_cache.find(key + "/nbr");
  std::vector<int> lex;
  if (key.empty() || it == c->shape_cache.end()) {
    Shape sh = build_shape(dims, periodic, parity_shift, member);
    in.d.n[0] = sh.n[0];
    in.d.n[1] = sh.n[1];
    in.nbr_buf = upload_shared(c, sh.nbr, &st);
    if (st != DD_OK) return st;
    in.fmap_buf = upload_shared(c, sh.fmap, &st);
    if (st != DD_OK) return st;
    in.lex_buf = upload_shared(c, sh.lex, &st);
    if (st != DD_OK) return st;
    in.ifm_buf = upload_shared(c, sh.ifm, &st);
    if (st != DD_OK) return st;
    in.h_fmap = sh.fmap;
    lex = sh.lex;
    if (!key.empty()) {
      c->shape_cache[key + "/nbr"] = in.nbr_buf;
      c->shape_cache[key + "/fmap"] = in.fmap_buf;
      c->shape_cache[key + "/lex"] = in.lex_buf;
      c->shape_cache[key + "/ifm"] = in.ifm_buf;
      auto* meta = new std::vector<int>();
      meta->push_back(sh.n[0]);
      meta->push_back(sh.n[1]);
      meta->insert(meta->end(), sh.fmap.begin(), sh.fmap.end());
      meta->insert(meta->end(), sh.lex.begin(), sh.lex.end());
      c->shape_cache[key + "/meta"] =
          std::shared_ptr<void>(meta, [](void* q) { delete (std::vector<int>*)q; });
    }
  } else {
    in.nbr_buf = it->second;
    in.fmap_buf = c->shape_cache[key + "/fmap"];
    in.lex_buf = c->shape_cache[key + "/lex"];
    in.ifm_buf = c->shape_cache[key + "/ifm"];
    auto* meta = (std::vector<int>*)c->shape_cache[key + "/meta"].get();
    in.d.n[0] = (*meta)[0];
    in.d.n[1] = (*meta)[1];
    int ns = in.d.n[0] + in.d.n[1];
    in.h_fmap.assign(meta->begin() + 2, meta->begin() + 2 + ns);
    lex.assign(meta->begin() + 2 + ns, meta->begin() + 2 + 2 * ns);
  }
  in.d.nsites = in.d.n[0] + in.d.n[1];
  // global site of each instance site
  in.h_glob.resize(in.d.nsites);
  for (int k = 0; k < in.d.nsites; ++k) {
    long long s = lex[k];
    int x[4];
    x[3] = s % dims[3];
    x[2] = (s / dims[3]) % dims[2];
    x[1] = (s / (1LL * dims[3] * dims[2])) % dims[1];
    x[0] = s / (1LL * dims[3] * dims[2] * dims[1]);
    int g[4];
    for (int m = 0; m < 4; ++m) g[m] = (origin[m] + x[m]) % c->L[m];
    in.h_glob[k] = ((g[0] * c->L[1] + g[1]) * c->L[2] + g[2]) * c->L[3] + g[3];
  }
  st = dalloc(c, &in.glob_buf, in.h_glob.size() * sizeof(int));
  if (st != DD_OK) return st;
  cudaMemcpy(in.glob_buf, in.h_glob.data(), in.h_glob.size() * sizeof(int),
             cudaMemcpyHostToDevice);
  in.d.nbr = (const int*)in.nbr_buf.get();
  in.d.fmap = (const int*)in.fmap_buf.get();
  in.d.lex = (const int*)in.lex_buf.get();
  in.d.ifm = (const int*)in.ifm_buf.get();
  in.d.glob = (const int*)in.glob_buf;
  *out_index = (int)c->inst.size();
  c->inst.push_back(std::move(in));
  c->inst_dirty = true;
  return DD_OK;
}

}  // namespace

dd_status sync_instances(dd_ctx* c) {
  if (!c->inst_dirty) return DD_OK;
  int n = (int)c->inst.size();
  if (n > c->d_inst_cap) {
    dfree(c->d_inst);
    c->d_inst = nullptr;
    dd_status st = dalloc(c, (void**)&c->d_inst, sizeof(DomInst) * (n + 16));
    if (st != DD_OK) return st;
    c->d_inst_cap = n + 16;
  }
  std::vector<DomInst> h(n);
  for (int i = 0; i < n; ++i) h[i] = c->inst[i].d;
  DD_CUDA(c, cudaMemcpy(c->d_inst, h.data(), sizeof(DomInst) * n, cudaMemcpyHostToDevice));
  c->inst_dirty = false;
  return DD_OK;
}

// ---------------------------------------------------------------------------
// link gathering

template <class S>
__device__ __forceinline__ S to_store(double2 v);
template <>
__device__ __forceinline__ double2 to_store<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 to_store<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <>
__device__ __forceinline__ __nv_bfloat162 to_store<__nv_bfloat162>(double2 v) {
  return __floats2bfloat162_rn((float)v.x, (float)v.y);
}
template <>
__device__ __forceinline__ df2s to_store<df2s>(double2 v) {
  const float2 r = split_d(v.x), i = split_d(v.y);
  df2s o;
  o.v = make_float4(r.x, i.x, r.y, i.y);
  return o;
}

// per-instance link copy in the pair layout [p][mu][10 entries][n_p] (entry
// 9 of each link is padding, zeroed by the caller)
template <class S>
__global__ void k_gather_links(const int* __restrict__ glob, int n0, int n1,
                               const double2* __restrict__ U, S* __restrict__ out) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long ns = n0 + n1;
  if (k >= ns * 36) return;
  int site = (int)(k % ns);
  int comp = (int)(k / ns);          // mu*9 + c
  int mu = comp / 9, c = comp % 9;
  int p = site < n0 ? 0 : 1;
  int i = p ? site - n0 : site;
  int np = p ? n1 : n0;
  int g = glob[site];
  out[link_block(p, mu, n0, np) + cidx(c, np, i)] = to_store<S>(U[(long long)g * 36 + comp]);
}

// per-chunk link bundles (layout in spinor.cuh) from the instance's gathered
// links: one thread per (quarter, direction, lane)
template <class S>
__global__ void k_build_bundle(DomInst d, const S* __restrict__ lk, unsigned char* __restrict__ out,
                               long long nquarters) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nquarters * 8 * LB_LANES) return;
  const int lane = (int)(k % LB_LANES);
  const int dir = (int)((k / LB_LANES) % 8);
  const long long qg = k / (8 * LB_LANES);
  const int n0 = d.n[0];
  const long long q1 = lb_quarter_base(1, n0);
  const int p = qg < q1 ? 0 : 1;
  const long long i = (qg - (p ? q1 : 0)) * LB_LANES + lane;
  const int n_out = d.n[p], n_in = d.n[1 - p];
  const int mu = dir & 3;
  unsigned char* qb = out + qg * lb_quarter_bytes<S>();
  S* lo = reinterpret_cast<S*>(qb);
  int* io = reinterpret_cast<int*>(qb + lb_link_bytes<S>());
  const int j = i < n_out ? d.nbr[(p ? 8LL * n0 : 0) + (long long)dir * n_out + i] : -1;
  io[dir * LB_LANES + lane] = j;
  S zero;
  memset(&zero, 0, sizeof(S));
  // pairs e = 0..3 (entries 2e, 2e + 1) two elements per lane, entry 8 one
  S* dl = lo + (long long)dir * LB_DIR_S;
  for (int e = 0; e < 5; ++e) {
    S* dst = e < 4 ? dl + (e * LB_LANES + lane) * 2 : dl + 4 * LB_LANES * 2 + lane;
    const int ne = e < 4 ? 2 : 1;
    if (j < 0) {
      for (int h = 0; h < ne; ++h) dst[h] = zero;
      continue;
    }
    const S* src = dir < 4 ? lk + link_block(p, mu, n0, n_out) + ((long long)e * n_out + i) * 2
                           : lk + link_block(1 - p, mu, n0, n_in) + ((long long)e * n_in + j) * 2;
    for (int h = 0; h < ne; ++h) dst[h] = src[h];
  }
}

__global__ void k_fold_time_sign(double2* U, int V, int L0, int spatial, int sign) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= (long long)spatial * 9) return;
  long long site = (long long)(L0 - 1) * spatial + k / 9;
  int c = (int)(k % 9);
  double2 v = U[site * 36 + c];    // mu = 0
  U[site * 36 + c] = make_double2(sign * v.x, sign * v.y);
}

dd_status ensure_links(dd_ctx* c, int i, dd_prec prec) {
  if (!c->gauge_ready) return fail(c, DD_EINVAL, "gauge field not uploaded");
  Instance& in = c->inst[i];
  void** buf = prec == DD_F64 ? &in.link64_buf
               : prec == DD_F32 ? &in.link32_buf
               : prec == DD_BF16 ? &in.link16_buf : &in.linkdf_buf;
  if (*buf && in.links_ready) return DD_OK;
  if (!in.links_ready) {
    // gauge changed: drop stale copies
    dfree(in.link64_buf);
    dfree(in.link32_buf);
    dfree(in.link16_buf);
    dfree(in.linkdf_buf);
    dfree(in.lb32_buf);
    dfree(in.lb16_buf);
    in.link64_buf = in.link32_buf = in.link16_buf = in.linkdf_buf = nullptr;
    in.lb32_buf = in.lb16_buf = nullptr;
    in.d.lb32 = nullptr;
    in.d.lb16 = nullptr;
    in.d.link64 = nullptr;
    in.d.link32 = nullptr;
    in.d.link16 = nullptr;
    in.d.linkdf = nullptr;
    in.links_ready = true;
  }
  size_t n = 40ULL * in.d.nsites;
  dd_status st = dalloc(c, buf, n * prec_bytes(prec));
  if (st != DD_OK) return st;
  DD_CUDA(c, cudaMemset(*buf, 0, n * prec_bytes(prec)));
  long long tot = 36LL * in.d.nsites;
  int th = 256;
  long long nb = (tot + th - 1) / th;
  if (prec == DD_F64)
    DD_COUNT_LAUNCH(), k_gather_links<double2><<<nb, th>>>(in.d.glob, in.d.n[0], in.d.n[1], c->d_U, (double2*)*buf);
  else if (prec == DD_F32)
    DD_COUNT_LAUNCH(), k_gather_links<float2><<<nb, th>>>(in.d.glob, in.d.n[0], in.d.n[1], c->d_U, (float2*)*buf);
  else if (prec == DD_BF16)
    DD_COUNT_LAUNCH(), k_gather_links<__nv_bfloat162><<<nb, th>>>(in.d.glob, in.d.n[0], in.d.n[1], c->d_U,
                                               (__nv_bfloat162*)*buf);
  else
    DD_COUNT_LAUNCH(), k_gather_links<df2s><<<nb, th>>>(in.d.glob, in.d.n[0], in.d.n[1], c->d_U, (df2s*)*buf);
  DD_CUDA(c, cudaGetLastError());
  // FP32 and BF16 links also get the per-chunk bundles of the bundle hop
  if (prec == DD_F32 || prec == DD_BF16) {
    const long long nq = lb_quarter_base(1, in.d.n[0]) +
                         (long long)LB_QUARTERS * ((in.d.n[1] + LB_CHUNK - 1) / LB_CHUNK);
    void** lb = prec == DD_F32 ? &in.lb32_buf : &in.lb16_buf;
    const size_t qbytes = prec == DD_F32 ? lb_quarter_bytes<float2>() : lb_quarter_bytes<__nv_bfloat162>();
    if ((st = dalloc(c, lb, std::max<size_t>(1, nq) * qbytes)) != DD_OK) return st;
    const long long tq = nq * 8 * LB_LANES;
    if (tq > 0) {
      if (prec == DD_F32)
        DD_COUNT_LAUNCH(), k_build_bundle<float2><<<(tq + th - 1) / th, th>>>(in.d, (const float2*)*buf,
                                                                             (unsigned char*)*lb, nq);
      else
        DD_COUNT_LAUNCH(), k_build_bundle<__nv_bfloat162><<<(tq + th - 1) / th, th>>>(
            in.d, (const __nv_bfloat162*)*buf, (unsigned char*)*lb, nq);
    }
    DD_CUDA(c, cudaGetLastError());
    hop_bundle_prepare();
  }
  in.d.link64 = (const double2*)in.link64_buf;
  in.d.link32 = (const float2*)in.link32_buf;
  in.d.link16 = (const __nv_bfloat162*)in.link16_buf;
  in.d.linkdf = (const df2s*)in.linkdf_buf;
  in.d.lb32 = (const unsigned char*)in.lb32_buf;
  in.d.lb16 = (const unsigned char*)in.lb16_buf;
  c->inst_dirty = true;
  return DD_OK;
}

// after new links in d_U: fold the time-boundary sign, mark every gathered
// per-domain copy stale
dd_status gauge_finish(dd_ctx* c) {
  const int spatial = c->V / c->L[0];
  if (c->time_bc != 1) {
    const long long n = 9LL * spatial;
    DD_COUNT_LAUNCH(), k_fold_time_sign<<<(n + 255) / 256, 256>>>(c->d_U, c->V, c->L[0], spatial, c->time_bc);
    DD_CUDA(c, cudaGetLastError());
  }
  DD_CUDA(c, cudaDeviceSynchronize());
  for (auto& in : c->inst) in.links_ready = false;
  c->gauge_ready = true;
  c->inst_dirty = true;
  return clover_build(c);        // no-op without the clover term
}

// after links in d_U changed on the device (a molecular-dynamics update): every
// gathered per-domain copy is stale (the stored links keep their time sign)
void gauge_touched(dd_ctx* c) {
  for (auto& in : c->inst) in.links_ready = false;
  c->inst_dirty = true;
}

dd_status check_device_error(dd_ctx* c, cudaStream_t s) {
  int h = 0;
  DD_CUDA(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  if (!h) return DD_OK;
  DD_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  DD_CUDA(c, cudaStreamSynchronize(s));
  return fail(c, DD_ETIMEOUT, "a bounded device-side wait gave up (bulk copy of a link bundle)");
}

dd_status instance_of(dd_ctx* c, dd_domain kind, int id, int* out) {
  switch (kind) {
    case DD_DOMAIN_FULL: *out = 0; return DD_OK;
    case DD_DOMAIN_LAMBDA1:
      if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
      *out = c->lambda1;
      return DD_OK;
    case DD_DOMAIN_OMEGA:
    case DD_DOMAIN_PHI: {
      if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
      if (id < 0 || id >= (int)c->blocks.size()) return fail(c, DD_EINVAL, "block id out of range");
      if (kind == DD_DOMAIN_OMEGA) {
        *out = c->omega0 + id;
        return DD_OK;
      }
      dd_status st = ensure_phi(c);
      if (st != DD_OK) return st;
      *out = c->phi0 + id;
      return DD_OK;
    }
  }
  return fail(c, DD_EINVAL, "unknown domain kind");
}

dd_status ensure_phi(dd_ctx* c) {
  if (c->phi0 >= 0) return DD_OK;
  int first = (int)c->inst.size();
  for (int b = 0; b < (int)c->blocks.size(); ++b) {
    const BlockDesc& bd = c->blocks[b];
    int lo[4], hi[4];
    for (int m = 0; m < 4; ++m) {
      lo[m] = (bd.core_lo[m] - bd.origin[m] + c->L[m]) % c->L[m];
      hi[m] = lo[m] + bd.core_hi[m] - bd.core_lo[m];
    }
    std::ostringstream key;
    key << "PHI p" << c->undecomposed;
    for (int m = 0; m < 4; ++m) key << ' ' << bd.side[m] << ' ' << lo[m] << ' ' << hi[m];
    const int* dims = bd.side;
    auto member = [&](long long s) {
      int x[4];
      x[3] = s % dims[3];
      x[2] = (s / dims[3]) % dims[2];
      x[1] = (s / (1LL * dims[3] * dims[2])) % dims[1];
      x[0] = s / (1LL * dims[3] * dims[2] * dims[1]);
      for (int m = 0; m < 4; ++m)
        if (x[m] < lo[m] || x[m] > hi[m]) return true;
      return false;
    };
    int idx;
    dd_status st = add_instance(c, DD_DOMAIN_PHI, b, bd.side, bd.origin, c->undecomposed, 0, key.str(),
                                member, &idx);
    if (st != DD_OK) return st;
  }
  c->phi0 = first;
  return DD_OK;
}

dd_status make_batch(dd_ctx* c, const std::vector<int>& inst, int nrhs, Batch& b) {
  const int CH = 128;
  if (nrhs > 65535 || inst.size() > 65535) return fail(c, DD_EINVAL, "at most 65535 rhs and instances per batch");
  b.nb = (int)inst.size();
  b.nrhs = nrhs;
  b.inst = inst;
  std::vector<long long> off[2], uoff;
  std::vector<int4> items[2];
  long long utot = 0;
  for (int p = 0; p < 2; ++p) {
    b.tot[p] = 0;
    b.item_begin[p].assign(b.nb + 1, 0);
    b.maxn[p] = 0;
  }
  for (int j = 0; j < b.nb; ++j) {
    const DomInst& d = c->inst[inst[j]].d;
    for (int r = 0; r < nrhs; ++r) {
      for (int p = 0; p < 2; ++p) {
        off[p].push_back(b.tot[p]);
        b.tot[p] += 12LL * d.n[p];
      }
      uoff.push_back(utot);
      utot += 12LL * d.nsites;
    }
    for (int p = 0; p < 2; ++p) {
      b.item_begin[p][j] = (int)items[p].size();
      for (int s = 0; s < d.n[p]; s += CH) items[p].push_back(make_int4(j, s, std::min(CH, d.n[p] - s), 0));
      b.maxn[p] = std::max(b.maxn[p], d.n[p]);
    }
  }
  for (int p = 0; p < 2; ++p) {
    b.item_begin[p][b.nb] = (int)items[p].size();
    b.nitems[p] = (int)items[p].size();
  }
  // runs of CH consecutive field positions (both parities) for the caller-layout kernels
  std::vector<int4> fitems;
  for (int j = 0; j < b.nb; ++j) {
    const int ns = c->inst[inst[j]].d.nsites;
    for (int f = 0; f < ns; f += CH) fitems.push_back(make_int4(j, f, std::min(CH, ns - f), 0));
  }
  b.nfitems = (int)fitems.size();
  b.user_tot = utot;
  dd_status st;
  if ((st = dalloc(c, (void**)&b.d_fitems, sizeof(int4) * std::max<size_t>(1, fitems.size()))) != DD_OK)
    return st;
  if (!fitems.empty())
    cudaMemcpy(b.d_fitems, fitems.data(), sizeof(int4) * fitems.size(), cudaMemcpyHostToDevice);
  if ((st = dalloc(c, (void**)&b.d_inst, sizeof(int) * b.nb)) != DD_OK) return st;
  cudaMemcpy(b.d_inst, inst.data(), sizeof(int) * b.nb, cudaMemcpyHostToDevice);
  if ((st = dalloc(c, (void**)&b.d_uoff, sizeof(long long) * uoff.size())) != DD_OK) return st;
  cudaMemcpy(b.d_uoff, uoff.data(), sizeof(long long) * uoff.size(), cudaMemcpyHostToDevice);
  for (int p = 0; p < 2; ++p) {
    if ((st = dalloc(c, (void**)&b.d_off[p], sizeof(long long) * off[p].size())) != DD_OK) return st;
    cudaMemcpy(b.d_off[p], off[p].data(), sizeof(long long) * off[p].size(), cudaMemcpyHostToDevice);
    if ((st = dalloc(c, (void**)&b.d_items[p], sizeof(int4) * std::max<size_t>(1, items[p].size()))) != DD_OK)
      return st;
    cudaMemcpy(b.d_items[p], items[p].data(), sizeof(int4) * items[p].size(), cudaMemcpyHostToDevice);
    if ((st = dalloc(c, (void**)&b.d_item_begin[p], sizeof(int) * (b.nb + 1))) != DD_OK) return st;
    cudaMemcpy(b.d_item_begin[p], b.item_begin[p].data(), sizeof(int) * (b.nb + 1),
               cudaMemcpyHostToDevice);
  }
  DD_CUDA(c, cudaGetLastError());
  return DD_OK;
}

BatchDev batch_view(dd_ctx* c, const Batch& b) {
  BatchDev v;
  v.inst_tab = c->d_inst;
  v.inst = b.d_inst;
  v.uoff = b.d_uoff;
  for (int p = 0; p < 2; ++p) {
    v.off[p] = b.d_off[p];
    v.items[p] = b.d_items[p];
    v.item_begin[p] = b.d_item_begin[p];
    v.nitems[p] = b.nitems[p];
  }
  v.fitems = b.d_fitems;
  v.nfitems = b.nfitems;
  v.nb = b.nb;
  v.nrhs = b.nrhs;
  return v;
}

}  // namespace dd

using namespace dd;

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char* dd_strerror(dd_status s) {
  switch (s) {
    case DD_OK: return "ok";
    case DD_EINVAL: return "invalid argument";
    case DD_ENOMEM: return "out of memory";
    case DD_ENOCONV: return "solver did not converge";
    case DD_ETIMEOUT: return "device wait timed out";
    case DD_ENAN: return "NaN or Inf encountered";
    case DD_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

const char* dd_last_error(const dd_ctx* c) { return c ? c->err.c_str() : "null context"; }

dd_status dd_create(dd_ctx** out, const int L[4], int time_bc, double kappa) {
  if (!out || !L) return DD_EINVAL;
  *out = nullptr;
  for (int m = 0; m < 4; ++m)
    if (L[m] < 2 || L[m] % 2) return DD_EINVAL;
  if (time_bc != 1 && time_bc != -1) return DD_EINVAL;
  long long V = 1LL * L[0] * L[1] * L[2] * L[3];
  if (V > (1LL << 30)) return DD_EINVAL;
  dd_ctx* c = new dd_ctx();
  for (int m = 0; m < 4; ++m) c->L[m] = L[m];
  c->V = (int)V;
  c->time_bc = time_bc;
  c->kappa = kappa;
  cudaGetDevice(&c->device);
  dd_status st = dalloc(c, (void**)&c->d_U, sizeof(double2) * 36ULL * V);
  if (st == DD_OK && (st = dalloc(c, (void**)&c->d_err, 2 * sizeof(int))) == DD_OK &&
      cudaMemset(c->d_err, 0, 2 * sizeof(int)) != cudaSuccess)
    st = DD_ECUDA;
  if (st != DD_OK) {
    dfree(c->d_U);
    dfree(c->d_err);
    delete c;
    return st;
  }
  int zero[4] = {0, 0, 0, 0};
  int idx;
  st = add_instance(c, DD_DOMAIN_FULL, -1, L, zero, 0xF, 0, "", [](long long) { return true; }, &idx);
  if (st != DD_OK) {
    dd_destroy(c);
    return st;
  }
  *out = c;
  return DD_OK;
}

dd_status dd_destroy(dd_ctx* c) {
  if (!c) return DD_OK;
  cudaDeviceSynchronize();
  for (auto& in : c->inst) free_instance(in);
  c->inst.clear();
  c->shape_cache.clear();
  dfree(c->d_U);
  dfree(c->d_inst);
  dfree(c->d_dpi_pos);
  dfree(c->d_dpi_kind);
  dfree(c->d_tbytes);
  dfree(c->d_err);
  dfree(c->d_clov);
  dfree(c->d_clovi);
  dfree(c->d_clovi32);
  dfree(c->d_clovi_df);
  free_workspace(c);
  free_plan(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->copy_in) cudaStreamDestroy(c->copy_in);
  if (c->copy_out) cudaStreamDestroy(c->copy_out);
  c->batches.clear();
  for (auto& r : c->trec) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete c;
  return DD_OK;
}

dd_status dd_set_kappa(dd_ctx* c, double kappa) {
  if (!c) return DD_EINVAL;
  c->kappa = kappa;
  return clover_build(c);        // A depends on kappa (no-op without the clover term)
}

dd_status dd_gauge_upload(dd_ctx* c, const double* U) {
  if (!c || !U) return fail(c, DD_EINVAL, "null argument");
  size_t bytes = sizeof(double2) * 36ULL * c->V;
  DD_CUDA(c, cudaMemcpy(c->d_U, U, bytes, cudaMemcpyDefault));
  return gauge_finish(c);
}

dd_status dd_set_geometry(dd_ctx* c, const int ncores[4], const int* core_lo, const int* core_hi,
                          dd_geom_info* info) {
  if (!c || !ncores || !core_lo || !core_hi) return fail(c, DD_EINVAL, "null argument");
  if (c->geom_ready) return fail(c, DD_EINVAL, "geometry already set for this context");
  std::vector<std::vector<int>> lo(4), hi(4);
  int k = 0;
  // ncores[m] == 0: direction m is not decomposed (one virtual core spanning its
  // whole periodic extent, no frame, no hyperplane; boxes wrap around in m)
  int und = 0, ndec = 0;
  int nc[4];
  for (int m = 0; m < 4; ++m) {
    if (ncores[m] == 0) {
      und |= 1 << m;
      lo[m].push_back(0);
      hi[m].push_back(c->L[m] - 1);
      nc[m] = 1;
      continue;
    }
    ++ndec;
    nc[m] = ncores[m];
    if (ncores[m] < 2) return fail(c, DD_EINVAL, "need at least two cores per decomposed direction");
    for (int i = 0; i < ncores[m]; ++i, ++k) {
      lo[m].push_back(core_lo[k]);
      hi[m].push_back(core_hi[k]);
      if (core_lo[k] < 0 || core_lo[k] > core_hi[k] || core_hi[k] >= c->L[m])
        return fail(c, DD_EINVAL, "core interval outside the lattice");
      if (i > 0 && core_lo[k] <= hi[m][i - 1] + 1)
        return fail(c, DD_EINVAL, "cores must be sorted and separated by a frame");
    }
    if (lo[m][0] + c->L[m] - hi[m].back() < 2)
      return fail(c, DD_EINVAL, "cores must be separated by a frame across the boundary");
  }
  if (ndec == 0) return fail(c, DD_EINVAL, "at least one direction must be decomposed");
  c->undecomposed = und;
  c->cores_lo = lo;
  c->cores_hi = hi;
  const int* L = c->L;
  int V = c->V;
  // block descriptors, lexicographic in the interval indices, direction 3 fastest
  c->blocks.clear();
  int nb = nc[0] * nc[1] * nc[2] * nc[3];
  for (int b = 0; b < nb; ++b) {
    int idx[4], r = b;
    for (int m = 3; m >= 0; --m) {
      idx[m] = r % nc[m];
      r /= nc[m];
    }
    BlockDesc bd;
    for (int m = 0; m < 4; ++m) {
      int n = nc[m];
      bd.core_lo[m] = lo[m][idx[m]];
      bd.core_hi[m] = hi[m][idx[m]];
      if ((und >> m) & 1) {
        bd.origin[m] = 0;
        bd.side[m] = L[m];
        continue;
      }
      int prev_hi = hi[m][(idx[m] + n - 1) % n];
      int next_lo = lo[m][(idx[m] + 1) % n];
      bd.origin[m] = (prev_hi + 1) % L[m];
      bd.side[m] = ((next_lo - 1 - prev_hi) % L[m] + L[m]) % L[m];
    }
    c->blocks.push_back(bd);
  }
  // site classification
  std::vector<int> core_of(V, -1);
  std::vector<char> plane(V, 0);
  std::vector<std::vector<char>> isplane(4);
  for (int m = 0; m < 4; ++m) {
    isplane[m].assign(L[m], 0);
    if (!((und >> m) & 1))
      for (int i = 0; i < nc[m]; ++i) isplane[m][lo[m][i]] = isplane[m][hi[m][i]] = 1;
  }
  std::vector<std::vector<int>> coreidx(4);
  for (int m = 0; m < 4; ++m) {
    coreidx[m].assign(L[m], -1);
    for (int i = 0; i < nc[m]; ++i)
      for (int x = lo[m][i]; x <= hi[m][i]; ++x) coreidx[m][x] = i;
  }
  for (int s = 0; s < V; ++s) {
    int x[4] = {s / (L[1] * L[2] * L[3]), (s / (L[2] * L[3])) % L[1], (s / L[3]) % L[2], s % L[3]};
    bool in0 = true;
    int b = 0;
    for (int m = 0; m < 4; ++m) {
      if (isplane[m][x[m]]) plane[s] = 1;
      if (coreidx[m][x[m]] < 0) in0 = false;
      else b = b * nc[m] + coreidx[m][x[m]];
    }
    if (in0) core_of[s] = b;
  }
  c->dpi_sites.clear();
  c->B_sites.clear();
  c->C_sites.clear();
  c->B_of_block.assign(nb, {});
  c->dpi_pos.assign(V, -1);
  std::vector<int> dpi_kind;
  int nA = 0, nL1 = 0;
  for (int s = 0; s < V; ++s) {
    if (core_of[s] < 0) nL1++;
    if (plane[s]) {
      c->dpi_pos[s] = (int)c->dpi_sites.size();
      c->dpi_sites.push_back(s);
      if (core_of[s] >= 0) {
        c->B_sites.push_back(s);
        c->B_of_block[core_of[s]].push_back(s);
        dpi_kind.push_back(core_of[s]);
      } else {
        c->C_sites.push_back(s);
        dpi_kind.push_back(-1);
      }
    } else if (core_of[s] >= 0) {
      nA++;
    }
  }
  dd_geom_info gi{};
  gi.nblocks = nb;
  gi.n_dpi = (int)c->dpi_sites.size();
  gi.n_B = (int)c->B_sites.size();
  gi.n_C = (int)c->C_sites.size();
  gi.n_lambda1 = nL1;
  gi.n_E = nL1 - gi.n_C;
  gi.n_A = nA;
  // instances: LAMBDA1 then OMEGA blocks
  dd_status st;
  int zero[4] = {0, 0, 0, 0};
  int idx;
  st = add_instance(c, DD_DOMAIN_LAMBDA1, -1, L, zero, 0xF, 0, "",
                    [&](long long s) { return core_of[s] < 0; }, &idx);
  if (st != DD_OK) return st;
  c->lambda1 = idx;
  c->omega0 = (int)c->inst.size();
  int maxo = 0, maxphi = 0;
  for (int b = 0; b < nb; ++b) {
    const BlockDesc& bd = c->blocks[b];
    std::ostringstream key;
    key << "OMEGA " << bd.side[0] << ' ' << bd.side[1] << ' ' << bd.side[2] << ' ' << bd.side[3] << " p"
        << c->undecomposed;
    st = add_instance(c, DD_DOMAIN_OMEGA, b, bd.side, bd.origin, c->undecomposed, 0, key.str(),
                      [](long long) { return true; }, &idx);
    if (st != DD_OK) return st;
    int no = c->inst[idx].d.nsites;
    int core = 1;
    for (int m = 0; m < 4; ++m) core *= bd.core_hi[m] - bd.core_lo[m] + 1;
    maxo = std::max(maxo, no);
    maxphi = std::max(maxphi, no - core);
  }
  gi.max_omega = maxo;
  gi.max_phi = maxphi;
  // device copies of dPi bookkeeping
  if ((st = dalloc(c, (void**)&c->d_dpi_pos, sizeof(int) * V)) != DD_OK) return st;
  cudaMemcpy(c->d_dpi_pos, c->dpi_pos.data(), sizeof(int) * V, cudaMemcpyHostToDevice);
  if ((st = dalloc(c, (void**)&c->d_dpi_kind, sizeof(int) * std::max(1, gi.n_dpi))) != DD_OK) return st;
  cudaMemcpy(c->d_dpi_kind, dpi_kind.data(), sizeof(int) * gi.n_dpi, cudaMemcpyHostToDevice);
  DD_CUDA(c, cudaGetLastError());
  c->info = gi;
  c->geom_ready = true;
  if (info) *info = gi;
  return DD_OK;
}

dd_status dd_geom_sites(dd_ctx* c, dd_set set, int block, int* out, int* count) {
  if (!c || !count) return fail(c, DD_EINVAL, "null argument");
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  std::vector<int> tmp;
  const std::vector<int>* v = nullptr;
  auto per_block = [&](int base) -> dd_status {
    if (block < 0 || block >= (int)c->blocks.size()) return fail(c, DD_EINVAL, "block id out of range");
    const Instance& in = c->inst[base + block];
    tmp.assign(in.d.nsites, 0);
    for (int k = 0; k < in.d.nsites; ++k) tmp[in.h_fmap[k]] = in.h_glob[k];
    v = &tmp;
    return DD_OK;
  };
  dd_status st = DD_OK;
  switch (set) {
    case DD_SET_DPI: v = &c->dpi_sites; break;
    case DD_SET_C: v = &c->C_sites; break;
    case DD_SET_B:
      if (block < 0 || block >= (int)c->blocks.size()) return fail(c, DD_EINVAL, "block id out of range");
      v = &c->B_of_block[block];
      break;
    case DD_SET_OMEGA: st = per_block(c->omega0); break;
    case DD_SET_PHI:
      if ((st = ensure_phi(c)) != DD_OK) return st;
      st = per_block(c->phi0);
      break;
    case DD_SET_LAMBDA1: {
      const Instance& in = c->inst[c->lambda1];
      tmp.assign(in.d.nsites, 0);
      for (int k = 0; k < in.d.nsites; ++k) tmp[in.h_fmap[k]] = in.h_glob[k];
      v = &tmp;
      break;
    }
    default: return fail(c, DD_EINVAL, "unknown set");
  }
  if (st != DD_OK) return st;
  if (out) {
    if (*count < (int)v->size()) return fail(c, DD_EINVAL, "output array too small");
    std::copy(v->begin(), v->end(), out);
  }
  *count = (int)v->size();
  return DD_OK;
}

dd_status dd_geom_block(dd_ctx* c, int block, int origin[4], int side[4], int core_lo[4],
                        int core_hi[4]) {
  if (!c) return DD_EINVAL;
  if (!c->geom_ready) return fail(c, DD_EINVAL, "geometry not set");
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, DD_EINVAL, "block id out of range");
  const BlockDesc& b = c->blocks[block];
  for (int m = 0; m < 4; ++m) {
    if (origin) origin[m] = b.origin[m];
    if (side) side[m] = b.side[m];
    if (core_lo) core_lo[m] = b.core_lo[m];
    if (core_hi) core_hi[m] = b.core_hi[m];
  }
  return DD_OK;
}

dd_status dd_roots(int N, double c, double* u) {
  if (!u || N < 2 || N % 2 || !(c >= 0.0 && c < 1.0)) return DD_EINVAL;
  const double pi = 3.14159265358979323846;
  double s = sqrt(1.0 - c * c);
  for (int k = 1; k <= N / 2; ++k) {
    double ph = 2.0 * pi * k / (N + 1);
    u[2 * (k - 1)] = cos(ph);
    u[2 * (k - 1) + 1] = s * sin(ph);
  }
  return DD_OK;
}

dd_status dd_launch_count(long long* n) {
  if (!n) return DD_EINVAL;
  *n = dd::g_launches.load();
  return DD_OK;
}

dd_status dd_timing_enable(dd_ctx* c, int on) {
  if (!c) return DD_EINVAL;
  c->timing = on != 0;
  return DD_OK;
}

dd_status dd_timing_get(dd_ctx* c, int which, double* ms, long long* launches, double* bytes) {
  if (!c || which < 0 || which > 3) return DD_EINVAL;
  for (auto& r : c->trec) {
    cudaEventSynchronize(r.b);
    float t = 0;
    cudaEventElapsedTime(&t, r.a, r.b);
    c->t_ms[r.which] += t;
    c->t_n[r.which] += 1;
    c->t_bytes[r.which] += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->trec.clear();
  if (c->d_tbytes) {
    double hb[3];
    cudaMemcpy(hb, c->d_tbytes, sizeof(hb), cudaMemcpyDeviceToHost);
    for (int k = 0; k < 3; ++k) c->t_bytes[k] += hb[k];
    cudaMemset(c->d_tbytes, 0, sizeof(hb));
  }
  if (ms) *ms = c->t_ms[which];
  if (launches) *launches = c->t_n[which];
  if (bytes) *bytes = c->t_bytes[which];
  c->t_ms[which] = 0;
  c->t_n[which] = 0;
  c->t_bytes[which] = 0;
  return DD_OK;
}

}  // extern "C"
