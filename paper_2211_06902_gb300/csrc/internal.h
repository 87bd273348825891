// Internal data model of libdd4d (not part of the C ABI).
//
// Every site set on which D is restricted (the full lattice, the frame
// Lambda1, each framed block Omega0^a and its frame piece Phi1^a) is a
// "domain instance".  Its sites are split by parity; within a parity they are
// numbered in increasing field order.  Per instance the library keeps
//   nbr  [p][8][n_p]  neighbour (index in the other parity) in directions
//                     +0,+1,+2,+3,-0,-1,-2,-3, or -1 when the hop leaves the set;
//   fmap [p][n_p]     position of the site in the caller's field order;
//   glob [p][n_p]     global lexicographic site index;
//   lex  [p][n_p]     local lexicographic index inside the box (boxes only);
//   links [p][mu][9][n_p]  forward links U_mu(x) of the instance's sites, with
//                     the time-boundary sign folded into U_0 at x0 = L0-1,
//                     stored complex (SoA, site fastest) in FP64, FP32, BF16.
// Boxes of the same shape share nbr/fmap/lex.  Spinor work vectors use the
// same SoA order: for one (instance, rhs) system and one parity,
// 12 components x n_p sites, component-major, component = 3*spin + colour.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dd4d.h"

namespace dd {

// internal storage precision (not in the C ABI): double-float pairs of FP32
constexpr dd_prec DD_DF64 = (dd_prec)3;
struct df2s;

struct DomInst {            // device-visible descriptor (plain data)
  int n[2];                 // sites per parity
  int dims[4];              // box extents (lattice extents for FULL / LAMBDA1)
  int origin[4];            // global coordinates of local site 0 (boxes)
  int kind;                 // dd_domain
  int nsites;               // n[0] + n[1]
  const int* nbr;           // [p][8][n_p], parity-1 table at 8*n[0]
  const int* fmap;          // [p][n_p]
  const int* glob;          // [p][n_p]
  const int* lex;           // [p][n_p] (boxes), nullptr otherwise
  const int* ifm;           // [field position] -> (parity << 30) | index in the parity
  const double2* link64;    // [p][4][9][n_p]
  const float2* link32;
  const __nv_bfloat162* link16;
  const df2s* linkdf;       // double-float copy (residual of the mixed solver)
  const unsigned char* lb32;  // per-chunk link bundles (FP32 / BF16), see spinor.cuh
  const unsigned char* lb16;
};

// Owning host record of an instance.
struct Instance {
  DomInst d{};
  int block = -1;
  std::shared_ptr<void> nbr_buf, fmap_buf, lex_buf, ifm_buf;   // shared between same-shape boxes
  void* glob_buf = nullptr;
  void* link64_buf = nullptr;
  void* link32_buf = nullptr;
  void* link16_buf = nullptr;
  void* linkdf_buf = nullptr;
  void* lb32_buf = nullptr;
  void* lb16_buf = nullptr;
  std::vector<int> h_glob;      // host copy [p][n_p]
  std::vector<int> h_fmap;      // host copy [p][n_p]
  bool links_ready = false;
};

struct BlockDesc {
  int core_lo[4], core_hi[4];
  int origin[4], side[4];
};

// A batch of systems: instances x nrhs, with per-parity work items.
struct Batch {
  int nb = 0, nrhs = 0;
  std::vector<int> inst;                    // instance index per batch position
  long long tot[2] = {0, 0};                // complex elements per parity (all systems)
  long long user_tot = 0;                   // complex elements in caller layout
  // device arrays
  int* d_inst = nullptr;
  long long* d_off[2] = {nullptr, nullptr}; // [nb*nrhs] offsets (complex elements)
  long long* d_uoff = nullptr;              // [nb*nrhs] caller-layout offsets
  int4* d_items[2] = {nullptr, nullptr};    // {j, start, count, 0}
  int nitems[2] = {0, 0};
  int* d_item_begin[2] = {nullptr, nullptr}; // [nb+1] first item of instance j
  int4* d_fitems = nullptr;                 // {j, first field position, count, 0}: 128-site runs in
  int nfitems = 0;                          // field order (caller layout), both parities together
  std::vector<int> item_begin[2];
  int maxn[2] = {0, 0};
  // tuned hop launch variant per precision (f64, f32, bf16) and CUDA graphs of
  // the inner Krylov iterations (krylov.cu), owned by the batch
  mutable int hop_variant[3] = {0, 0, 0};
  mutable bool tuned[3] = {false, false, false};
  mutable std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;
  mutable std::map<std::string, long long> graph_kernels;   // kernel nodes per replay (launch count)
  ~Batch();
};

struct BatchDev {           // device-visible view of a Batch
  const DomInst* inst_tab;  // all instances
  const int* inst;          // [nb]
  const long long* off[2];
  const long long* uoff;
  const int4* items[2];
  const int* item_begin[2];
  int nitems[2];
  const int4* fitems;
  int nfitems;
  int nb, nrhs;
};

// per-system state of the batched solver (krylov.cu, fgmres.cu), device memory
struct SysState {
  double2 rho, alpha, omega, beta;
  double rr;        // current |r|^2 of the inner recursion (or outer residual)
  double target2;   // inner stopping threshold on |r|^2
  double bnorm2;    // |b|^2 of the full (both-parity) right-hand side
  double outer2;    // outer threshold (tol |b|)^2
  int active;       // inner recursion running
  int outer_active; // outer loop still running
  int iters;        // inner iterations, summed over cycles
  int status;       // 0 ok, 1 converged, 2 breakdown
};

// two CUDA events destroyed on scope exit (also on the early error returns)
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
};

struct TimingRec {
  cudaEvent_t a, b;
  int which;
  double bytes;
};

}  // namespace dd

struct dd_ctx {
  int L[4];
  int V;
  int time_bc;
  double kappa;
  int device = 0;
  int nsm = 0;
  std::string err;
  // gauge field, FP64, [V][4][9] complex (time sign folded in)
  double2* d_U = nullptr;
  bool gauge_ready = false;
  // geometry
  bool geom_ready = false;
  std::vector<std::vector<int>> cores_lo, cores_hi;   // per direction
  std::vector<dd::BlockDesc> blocks;
  std::vector<int> dpi_sites, B_sites, C_sites;       // increasing global order
  std::vector<std::vector<int>> B_of_block;           // per block, increasing global order
  std::vector<int> dpi_pos;                            // [V] -> index in dPi or -1
  std::vector<int> block_of_B;                         // [n_B in dPi order?] unused
  dd_geom_info info{};
  // instances: 0 = FULL, 1 = LAMBDA1, then OMEGA blocks, then PHI blocks (lazy)
  std::vector<dd::Instance> inst;
  int omega0 = -1, phi0 = -1, lambda1 = -1;
  dd::DomInst* d_inst = nullptr;
  int d_inst_cap = 0;
  bool inst_dirty = true;
  std::map<std::string, std::shared_ptr<void>> shape_cache;
  // device copies of the dPi bookkeeping
  int* d_dpi_pos = nullptr;      // [V]
  int* d_dpi_kind = nullptr;     // [n_dpi] 0..nblocks-1: block of a B site; -1: C site
  // timing
  bool timing = false;
  std::vector<dd::TimingRec> trec;
  double t_ms[4] = {0, 0, 0, 0};          // per timing class (hop F64/F32/BF16, force)
  long long t_n[4] = {0, 0, 0, 0};
  double t_bytes[4] = {0, 0, 0, 0};
  double* d_tbytes = nullptr;     // device accumulators of algorithmic bytes [3]
  // clover term (clover.cu): A and A^{-1} per site, [V][2][6][6] complex FP64
  double csw = 0.0;
  double2* d_clov = nullptr;
  double2* d_clovi = nullptr;
  float4* d_clovi32 = nullptr;    // A^{-1} hermitian-packed, FP32 [V][18] float4
  float4* d_clovi_df = nullptr;   // A^{-1} hermitian-packed, double-float [V][36] float4
  bool clover_ready = false;
  double clover_cond = 1.0;          // max |A_x|_inf * max |A_x^{-1}|_inf >= cond_2(A)
  bool clover_mixed_ready = false;   // the two packed tables match A^{-1}
  bool clover_active = false;     // inside a solve: every hop applies A^{-1} (clov_inv)
  int* d_err = nullptr;           // [0]: device error word, set by kernels whose bounded waits give up;
                                  // [1]: work-queue counter of the persistent stencil
  // work space (krylov.cu) and cached batches
  void* scratch = nullptr;
  std::map<std::string, std::unique_ptr<dd::Batch>> batches;
  void* wplan = nullptr;     // gather lists of apply_w (dd.cu)
  dd_solve_stats last_stats{};   // statistics of the last batched solve
  dd_net* net = nullptr;         // learned initial guess for block solves (not owned)
  cudaStream_t capture_stream = nullptr;   // private stream for CUDA-graph capture
  int undecomposed = 0;                    // bit m: direction m not decomposed (boxes wrap in m)
  cudaStream_t copy_in = nullptr, copy_out = nullptr;   // host<->device copies of pipelined solves
  int forced_variant[3] = {-1, -1, -1};    // manual stencil launch variant per precision
  bool debug_wait_fault = false;           // test hook: see dd_debug_wait_fault
};

// ---- helpers shared by the translation units --------------------------------
namespace dd {

// process-wide count of kernel launches issued by the library
extern std::atomic<long long> g_launches;
#define DD_COUNT_LAUNCH() (dd::g_launches.fetch_add(1, std::memory_order_relaxed))

dd_status fail(dd_ctx* c, dd_status s, const std::string& msg);
dd_status cuda_fail(dd_ctx* c, cudaError_t e, const char* where);
#define DD_CUDA(ctx, call)                                         \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return dd::cuda_fail(ctx, e_, #call);   \
  } while (0)

dd_status sync_instances(dd_ctx* c);              // upload DomInst table if dirty
dd_status ensure_links(dd_ctx* c, int i, dd_prec prec);
dd_status ensure_phi(dd_ctx* c);
dd_status instance_of(dd_ctx* c, dd_domain kind, int id, int* out);
dd_status make_batch(dd_ctx* c, const std::vector<int>& inst, int nrhs, Batch& b);
BatchDev batch_view(dd_ctx* c, const Batch& b);

// Device memory: plain cudaMalloc wrappers that record failures.
dd_status dalloc(dd_ctx* c, void** p, size_t bytes);
void dfree(void* p);

// Host-or-device pointer helper: returns true when p is device-accessible memory.
bool is_device_ptr(const void* p);
bool is_pinned_host_ptr(const void* p);   // page-locked (registered or cudaHostAlloc) host memory

// stencil launches (stencil.cu)
struct HopArgs {
  int p_out;                // output parity
  const void* in;           // parity 1-p_out vector base
  void* out;                // parity p_out vector base
  const void* s1;           // optional self term (parity p_out)
  const void* s2;           // optional second self term
  double a1, a2, b;         // out = a1*s1 + a2*s2 + b*H in
  const void* dotq;         // optional: partial (dotq, out)  [complex]
  const void* dots;         // optional: partials (out, dots) and (out, out)
  bool dotqs;               // with dotq and s1: also the partial (dotq, s1) into slot 3
  unsigned rhat_seed;       // nonzero: dotq is not read but generated (rhat_comp, spinor.cuh)
  bool norm_out;            // double-float output: |out|^2 per (item, rhs) into partial slot 0
  double* partial;          // [k][nitems*nrhs] complex (2 doubles)
  const int* active;        // optional per-system flags, active[sys * active_stride]
  int active_stride;
  double* work_bytes;       // timing only: algorithmic bytes of the CTAs that ran
  double site_bytes;        // algorithmic bytes per output (site, rhs)
  int* err;                 // device error word (bounded waits that gave up)
  const void* clov_inv;     // A^{-1} of the clover term, applied to the hop sum at the output
                            // site (left-preconditioned solves): FP64 [V][72] complex for
                            // FP64 hops; hermitian-packed FP32 [V][72] floats for FP32 and
                            // BF16-storage hops; hermitian-packed double-float [V][36]
                            // float4 for the double-float residual hops
  int lb_fault;             // test hook of the bundle form (dd_debug_wait_fault): CTA 0 leaves
                            // one quarter's bulk copy unissued and waits a few microseconds
  int* queue;               // work-queue counter of the persistent bundle form
};
dd_status launch_hop(dd_ctx* c, const Batch& b, dd_prec prec, const HopArgs& a, cudaStream_t s);
int hop_variant_count(dd_prec prec);
// sets the shared-memory attributes of the bundle kernels on the current device
void hop_bundle_prepare();
// reads and clears the device error word: DD_ETIMEOUT if a bounded wait gave up
dd_status check_device_error(dd_ctx* c, cudaStream_t s);
// after new links in d_U (ctx.cu): time sign, stale per-domain copies
dd_status gauge_finish(dd_ctx* c);
// clover term (clover.cu): build A, A^{-1} from d_U (no-op at c_sw = 0), and
// v <- A v or A^{-1} v on both parity vectors of a batch (FP64)
dd_status clover_build(dd_ctx* c);
void gauge_touched(dd_ctx* c);
dd_status clover_apply(dd_ctx* c, const Batch& b, void* ve, void* vo, bool inverse, cudaStream_t s);
dd_status clover_mixed_tables(dd_ctx* c);
dd_status clover_apply_inv_df(dd_ctx* c, const Batch& b, void* ve, void* vo, cudaStream_t s);

// layout conversions (stencil.cu)
// b -> b, r = b (outer precision F64 or double-float), x = 0, in caller field order
dd_status launch_pack_init(dd_ctx* c, const Batch& b, const double* user, void* be, void* bo, void* re,
                           void* ro, void* xe, void* xo, dd_prec prec, cudaStream_t s);
dd_status launch_pack(dd_ctx* c, const Batch& b, const double* user, void* ve, void* vo,
                      dd_prec prec, cudaStream_t s);
dd_status launch_unpack(dd_ctx* c, const Batch& b, const void* ve, const void* vo, double* user,
                        dd_prec prec, cudaStream_t s);

// solver (krylov.cu)
dd_status solve_batch(dd_ctx* c, const Batch& b, const double* b_user, double* x_user,
                      const dd_solve_params* prm, dd_solve_stats* st, cudaStream_t s,
                      bool user_layout);

size_t prec_bytes(dd_prec p);

// growable per-context device work buffers (krylov.cu); slots are reused by
// every call on the context, so calls on one context must not overlap
dd_status workspace(dd_ctx* c, int slot, size_t bytes, void** out);
void free_workspace(dd_ctx* c);
void free_plan(dd_ctx* c);
dd_status get_batch(dd_ctx* c, dd_domain kind, const int* ids, int nblk, int nrhs, Batch** out);
dd_status get_batch_insts(dd_ctx* c, const std::vector<int>& inst, int nrhs, Batch** out);
// Flexible GMRES(m) for the even Schur systems of a batch (fgmres.cu): solves
// M x_e = rhs_e (x_e at the inner precision, from zero) for the systems still in
// the outer loop, to max(inner_tol2 |rhs|^2, floor_frac outer2); with `net`, the
// network is the variable right preconditioner z = [N((v, 0))]_even (FP32 only)
dd_status run_fgmres(dd_ctx* c, const Batch& b, dd_prec prec, SysState* st, const void* rhs, void* x,
                     int restart, double inner_tol2, double floor_frac, int maxiter, dd_net* net,
                     cudaStream_t s, int* iters_run);
// z_e = [N((v_e, 0))]_even on every system of the batch (net.cu), FP32 vectors
dd_status net_precondition(dd_ctx* c, dd_net* n, const Batch& b, const float2* ve, float2* ze,
                           cudaStream_t s);
// learned initial guess x0 = N(b) (net.cu) from FP64 or double-float (df)
// parity vectors, written as FP32 parity vectors
dd_status net_guess(dd_ctx* c, dd_net* n, const Batch& b, const void* be, const void* bo, bool df,
                    float2* xe32, float2* xo32, cudaStream_t s);

}  // namespace dd
