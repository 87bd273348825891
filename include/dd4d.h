/*
 * dd4d.h - C ABI of libdd4d.so, the GB300 (sm_103a) implementation of the
 * data-parallel hot path of the four-dimensional overlapping domain
 * decomposition of the lattice Wilson-Dirac operator and of the factorization
 * of det D (Saccardi & Giusti, "Four-dimensional domain decomposition for the
 * factorization of the fermion determinant", Lattice 2022).
 *
 * Conventions used by every call
 * ------------------------------
 * - Every call returns a dd_status; DD_OK is 0.  dd_strerror() names a code,
 *   dd_last_error() gives the message of the last failure on a context.  No
 *   C++ exception crosses this interface.
 * - Lattice: extents L[4], x0 is time.  Global site index is lexicographic
 *   with x3 fastest: ((x0*L1 + x1)*L2 + x2)*L3 + x3.  Boundary conditions:
 *   periodic in x1..x3; the hop across x0 = L0-1 <-> 0 is multiplied by
 *   time_bc (+1 periodic, -1 antiperiodic).
 * - Spinor fields are complex128 (interleaved re, im doubles) with 12
 *   components per site, spin-major: component = 3*spin + colour, in the
 *   chiral basis gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]],
 *   gamma_5 = diag(1,1,-1,-1).
 * - Dirac operator (paper Sec. 1 and 3; Wilson, kappa normalisation, r = 1):
 *   (D psi)(x) = psi(x) - kappa sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu)
 *                                     + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)].
 *   Restriction to a site set X: D_X = P_X D P_X (hops leaving X dropped,
 *   Dirichlet boundary).
 * - Pointers to fields may be device pointers or host pointers (pageable or
 *   pinned); the library detects which.  With host pointers the call copies
 *   in and out itself and returns after the result is on the host.  With
 *   device pointers the call is asynchronous on `stream` unless stated.
 *   Callers keep ownership of every buffer they pass; the context owns the
 *   gauge field, the geometry tables and its work space.
 * - A context is not thread-safe: one host thread at a time.
 */
#ifndef DD4D_H
#define DD4D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DD_OK = 0,
  DD_EINVAL = 1,    /* invalid argument (size, id, layout, state) */
  DD_ENOMEM = 2,    /* device or host allocation failed */
  DD_ENOCONV = 3,   /* a Krylov solve stopped before reaching its tolerance */
  DD_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  DD_ENAN = 5,      /* NaN or Inf in an input or a residual */
  DD_ECUDA = 6      /* a CUDA runtime call failed */
} dd_status;

typedef enum { DD_F64 = 0, DD_F32 = 1, DD_BF16 = 2 } dd_prec;

/* Site sets on which D can be restricted (paper Sec. 2). */
typedef enum {
  DD_DOMAIN_FULL = 0,    /* the whole lattice                                   */
  DD_DOMAIN_OMEGA = 1,   /* framed block Omega0^a = Lambda0^a u Phi1^a          */
  DD_DOMAIN_PHI = 2,     /* its frame piece Phi1^a = Omega0^a \ Lambda0^a       */
  DD_DOMAIN_LAMBDA1 = 3  /* the inactive connected frame Lambda1                */
} dd_domain;

/* Site sets that can be listed with dd_geom_sites(). */
typedef enum {
  DD_SET_DPI = 0,        /* dPi: union of the block-boundary hyperplanes        */
  DD_SET_B = 1,          /* dLambda0^a of one block (block id required)          */
  DD_SET_C = 2,          /* dPi1 = dPi \ dLambda0                               */
  DD_SET_OMEGA = 3,      /* Omega0^a of one block, in the block's field order    */
  DD_SET_PHI = 4,        /* Phi1^a of one block, in its field order              */
  DD_SET_LAMBDA1 = 5     /* Lambda1 in its field order                           */
} dd_set;

typedef struct dd_ctx dd_ctx;

typedef struct {
  int nblocks;
  int n_dpi;        /* |dPi|        */
  int n_B;          /* |dLambda0|   */
  int n_C;          /* |dPi1|       */
  int n_E;          /* |Lambda1 \ dPi1| */
  int n_A;          /* |Lambda0 \ dLambda0| (bulk of the blocks) */
  int n_lambda1;    /* |Lambda1|    */
  int max_omega;    /* largest |Omega0^a| */
  int max_phi;      /* largest |Phi1^a|   */
} dd_geom_info;

typedef struct {
  double tol;          /* stop when |b - D x| <= tol |b| per system (e.g. 1e-10); with the
                          clover term on (dd_set_clover) the solver tests the left-preconditioned
                          residual, |A^{-1}(b - D x)| <= (tol / c_A) |A^{-1} b| with
                          c_A = max_x |A_x|_inf max_x |A_x^{-1}|_inf >= cond_2(A), which keeps
                          the true residual |b - D x| <= tol |b| */
  int maxiter;         /* Krylov iterations cap per system (inner ones for mixed) */
  dd_prec inner_prec;  /* DD_F64: plain FP64 BiCGstab; DD_F32 / DD_BF16: inner
                          solve at that precision with FP64 defect correction */
  double inner_tol;    /* relative reduction per inner solve (mixed only), e.g. 1e-5 */
  int max_outer;       /* defect-correction cycles cap (mixed only) */
  int check_every;     /* iterations between host convergence checks (>= 1) */
  int flags;           /* DD_SOLVE_* below, or-ed, or 0 */
  int restart;         /* Arnoldi steps per FGMRES cycle (DD_SOLVE_FGMRES; 1..16) */
} dd_solve_params;

/* dd_solve_params.flags */
#define DD_SOLVE_GRAPH 1     /* replay the inner iterations between two host polls as one
                                captured CUDA graph (ignored while kernel timing is on) */
#define DD_SOLVE_AUTOTUNE 2  /* on a batch's first solve, time every compiled launch variant
                                of the stencil (resident CTAs per SM, persistent grid) and
                                keep the fastest for that batch */
#define DD_SOLVE_NET_GUESS 4 /* framed-block batches start from x0 = N(b), the network set
                                with dd_set_net (ignored when none is set) */
#define DD_SOLVE_PIPELINE 8  /* page-locked host b and x: always split the blocks into
                                chunks whose host<->device copies overlap the solves of
                                the other chunks (done anyway from 256 MB of b) */
#define DD_SOLVE_GRAPH_LOOP 64 /* each inner BiCGstab solve as ONE captured CUDA graph: a
                                conditional WHILE node repeats the iteration, and a
                                one-thread kernel sets its condition from the device-side
                                count of running systems (no host polls inside the inner
                                solve; ignored while kernel timing is on) */
#define DD_SOLVE_GRAPH_SOLVE 128 /* the whole mixed-precision solve (FP32 or BF16 inner BiCGstab)
                                as ONE CUDA graph launch after b is packed: conditional WHILE
                                and IF nodes run the defect-correction cycles, their inner
                                solves, the verification of an updated residual and the
                                choice between a true and an updated residual, each decided
                                by a one-thread kernel from device-side counts (no host poll
                                in the solve); taken once the launch form is tuned, and not
                                with FGMRES or while kernel timing is on */
#define DD_SOLVE_FGMRES 16   /* inner solve by flexible GMRES(restart) instead of BiCGstab
                                (FP32 or FP64 inner precision; the host checks after
                                every Arnoldi step) */
#define DD_SOLVE_NET_PRECOND 32 /* with DD_SOLVE_FGMRES and FP32 inner solves of framed
                                blocks: the network set with dd_set_net is the variable
                                right preconditioner, z = [N((v_e, 0))]_even, the even
                                block of its approximation of D_Omega^{-1} (= the inverse
                                of the Schur complement) */

typedef struct {
  int systems;         /* number of (block, rhs) systems solved */
  int converged;       /* how many reached tol */
  int max_iters;       /* largest Krylov iteration count over systems (all cycles) */
  int outer_cycles;    /* defect-correction cycles run (1 for plain FP64) */
  double max_relres;   /* largest final |b - D x|/|b|, FP64, over systems */
  double seconds;      /* device time of the call (CUDA events) */
  int hop_variant;     /* stencil launch variant used at the inner precision (autotuner) */
} dd_solve_stats;

/* ---- context --------------------------------------------------------- */

/* Creates a context for a lattice of extents L (each even, >= 2), time
 * boundary sign time_bc (+1 or -1) and hopping parameter kappa.  Uses the
 * current CUDA device. DD_EINVAL on bad sizes. */
dd_status dd_create(dd_ctx** ctx, const int L[4], int time_bc, double kappa);
dd_status dd_destroy(dd_ctx* ctx);
const char* dd_strerror(dd_status s);
const char* dd_last_error(const dd_ctx* ctx);
dd_status dd_set_kappa(dd_ctx* ctx, double kappa);

/* ---- clover term (paper Sec. 1: D may carry a site-local term) --------------
 * c_sw != 0 adds to D the Sheikholeslami-Wohlert term in kappa normalisation,
 * D = A - kappa H with A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu F_mu_nu(x),
 * sigma_mu_nu = (i/2)[gamma_mu, gamma_nu] and F_mu_nu = (Q_mu_nu - Q_mu_nu^+)/8
 * from the four plaquettes Q_mu_nu of the mu-nu plane at x (each traversed mu
 * first; the links without the time boundary sign).  A and A^{-1} (two 6x6
 * chiral blocks per site, FP64) are rebuilt on every gauge upload and kappa
 * change.  With the term on: dd_apply_D_block computes A psi - kappa H psi
 * (DD_F64 only); dd_solve_blocks and everything built on it (dd_apply_w, the
 * action, the heat-bath, the reweighting samples, dd_logdet_check) solve
 * (1 - kappa A^{-1} H) x = A^{-1} b with the even-odd Schur form
 * 1 - kappa^2 A_ee^{-1} H_eo A_oo^{-1} H_oe, to tol / c_A on the residual
 * A^{-1}(b - D x) relative to A^{-1} b (c_A: the bound of cond_2(A) from the
 * row-sum norms of the hermitian blocks of A and A^{-1}, computed with the
 * tables), so the true residual stays within tol.  Every hop of a solve applies
 * A^{-1} of its output site at its own precision: FP64 for DD_F64 solves; for
 * DD_F32 and DD_BF16 inner solves an FP32 copy of A^{-1} (each hermitian block
 * packed to its diagonal and upper triangle, 288 B per site), and for their
 * double-float residual a double-float copy (576 B per site); A^{-1} b is
 * formed once in FP64.  The two copies (1.5 times the FP64 table) are built
 * at the first mixed solve after A changes.  dd_mb_force, dd_apply_D_block at
 * DD_F32 / DD_BF16, dd_apply_D_block_noalloc and the learned network
 * (DD_SOLVE_NET_GUESS, DD_SOLVE_NET_PRECOND) return DD_EINVAL with the term
 * on.  c_sw = 0 turns it off (the default). */
dd_status dd_set_clover(dd_ctx* ctx, double c_sw);
/* c_A = max_x |A_x|_inf * max_x |A_x^{-1}|_inf, the bound of cond_2(A) the solves
 * divide their tolerance by (1 without the term). */
dd_status dd_clover_cond(dd_ctx* ctx, double* c_A);

/* Gauge links U_mu(x) in SU(3) (paper Sec. 1).  Host buffer, layout
 * [site (global index)][mu 0..3][3][3] complex128 (row-major 3x3).  The
 * stored links are not modified; the time boundary sign is applied by the
 * operator.  Rebuilds every gathered per-domain copy.  Synchronous. */
dd_status dd_gauge_upload(dd_ctx* ctx, const double* U_host);

/* Synthetic links drawn on the device (the paper's links U_mu(x) in SU(3),
 * Sec. 1; the synthetic recipe stands in for its Monte Carlo ensembles):
 * U = exp(i eps H), H = sum_a h_a lambda_a / 2 over the Gell-Mann matrices,
 * h_a ~ N(0, 1) from the counter-based SplitMix64 stream of (seed, tag 1)
 * with Box-Muller normals, link l = 4 site + mu taking draws 8l .. 8l+7.
 * Bit-for-bit the same draws as the seeded host generator; the exponential
 * agrees with an eigen-decomposition to FP64 rounding.  Synchronous. */
dd_status dd_gauge_random(dd_ctx* ctx, double eps, unsigned long long seed);

/* Copy of the current links into a host buffer of the dd_gauge_upload layout
 * (time-boundary sign not applied).  Synchronous. */
dd_status dd_gauge_download(dd_ctx* ctx, double* U_host);

/* ---- geometry (paper Sec. 2) ------------------------------------------
 * Per direction mu a sorted list of core intervals [lo, hi] (inclusive,
 * 0 <= lo <= hi < L_mu) separated by at least one frame site (periodic);
 * at least two per decomposed direction.  ncores[mu] = 0 leaves direction mu
 * undecomposed: one core spans its whole periodic extent, without frame or
 * hyperplanes, and every domain wraps around in mu (ncores = {n, 0, 0, 0} is
 * the one-dimensional decomposition in thick time slices of Sec. 3, where
 * dPi1 is empty).  At least one direction is decomposed.  ncores[mu] entries for direction mu are
 * taken in turn from core_lo / core_hi (direction 0 first).  Blocks
 * Lambda0^a are the products of one interval per direction, numbered
 * lexicographically in the interval indices with direction 3 fastest.
 * Omega0^a spans the sites strictly between the neighbouring intervals'
 * hyperplanes; its field order is local lexicographic (x3 fastest) starting
 * at the site after the previous interval.  DD_EINVAL on an invalid list. */
dd_status dd_set_geometry(dd_ctx* ctx, const int ncores[4], const int* core_lo,
                          const int* core_hi, dd_geom_info* info);

/* Global site indices of a set, in the order the library uses for fields on
 * it.  `block` selects the block for per-block sets (ignored otherwise).
 * `out` is a host array of at least *count entries; pass out = NULL to get
 * only *count.  dPi, dPi1 and Lambda1 are in increasing global order. */
dd_status dd_geom_sites(dd_ctx* ctx, dd_set set, int block, int* out, int* count);

/* Block descriptor: origin (first site of Omega0^a per direction), the side
 * of Omega0^a and the core interval, all per direction. */
dd_status dd_geom_block(dd_ctx* ctx, int block, int origin[4], int side[4],
                        int core_lo[4], int core_hi[4]);

/* ---- restricted Wilson stencil (paper Sec. 3, D_X) -----------------------
 * out = D_X in for nblk domains of kind `kind` (block ids `ids`, host array;
 * ignored for FULL and LAMBDA1, which take nblk = 1) and nrhs fields each.
 * in/out layout: [blk][rhs][site in the domain's field order][12] complex128.
 * prec selects the storage/arithmetic of the stencil (FP64, or FP32 / BF16
 * storage with FP32 arithmetic). */
dd_status dd_apply_D_block(dd_ctx* ctx, dd_domain kind, const int* ids, int nblk,
                           int nrhs, const double* in, double* out, dd_prec prec,
                           void* stream);

/* ---- batched block solves (paper Sec. 3, D_Omega^-1, D_Phi^-1, D_Lambda1^-1)
 * x = D_X^{-1} b for every (block, rhs) pair, with even-odd (site parity)
 * preconditioning and BiCGstab; plain FP64, or an FP32/BF16 inner solve with
 * defect correction whose b, x, r, residual stencil and updates are kept in
 * double-float (two FP32 numbers, about 44 significant bits).  Layout as for
 * dd_apply_D_block; b and x may be device or host memory (host buffers are
 * copied; page-locked ones of 256 MB or more, or with DD_SOLVE_PIPELINE, in
 * chunks of blocks that overlap the copies with the solves).  Synchronises
 * `stream` (the host polls convergence).  Returns DD_ENOCONV (with stats
 * filled) if some system missed params->tol. */
dd_status dd_solve_blocks(dd_ctx* ctx, dd_domain kind, const int* ids, int nblk,
                          int nrhs, const double* b, double* x,
                          const dd_solve_params* params, dd_solve_stats* stats,
                          void* stream);

/* Manual choice of the stencil launch variant (0 .. dd_hop_variants(prec)-1)
 * for every batch used afterwards on the context, overriding the autotuner;
 * v = -1 returns to the defaults.  Variants differ in launch shape (resident
 * CTAs per SM, persistent grid, rhs per thread, direction split, links staged
 * in shared memory by bulk copy), not in the per-site arithmetic; the fused
 * inner products may sum in a different order.  dd_hop_variant_name returns
 * a static description of variant v (NULL if out of range). */
dd_status dd_set_hop_variant(dd_ctx* ctx, dd_prec prec, int v);

/* Test hook of the failure path (no counterpart in the paper).  While on != 0,
 * every launch of the shared-memory bundle form of the FP32/BF16 stencil lets
 * its first CTA arm the barrier of its last link quarter without issuing the
 * bulk copy, and bounds that CTA's waits to 64 polls of about 1 us: the wait
 * gives up with nothing in flight, the kernel sets the device error word, and
 * the next synchronising call returns DD_ETIMEOUT (that CTA's output is left
 * incomplete).  on = 0 restores normal launches; the context stays usable.
 * Host-only, no sync. */
dd_status dd_debug_wait_fault(dd_ctx* ctx, int on);
int dd_hop_variants(dd_prec prec);
const char* dd_hop_variant_name(dd_prec prec, int v);

/* Statistics of the last batched solve run on the context (by any call,
 * including the block and frame solves inside dd_apply_w). */
dd_status dd_last_solve_stats(const dd_ctx* ctx, dd_solve_stats* stats);

/* ---- the operator w (paper Sec. 3, Eqs. Wz and offdiagW1) ----------------
 * w = 1 - W_1 on dPi, W_1 = diag(D^d, D^_{dPi1})^{-1} M the matrix of the second
 * Schur decomposition with the blocks the paper prints (the hopping block D^h
 * in its symmetrised form over the frame pieces Phi1^a).  For n_f fields chi on
 * dPi (layout [f][dPi site in dd_geom_sites order][12]) it is applied as
 *   Y_b = D_{Phi1^b}^{-1} D_{Phi1^b, dLambda0^b} chi           (every block b)
 *   (Q chi)(x) = sum_{b : x in Phi1^b} Y_b(x)  on dPi1,  chi' = chi - Q chi
 *   (w chi)_{dLambda0^a} = -P_{dLambda0^a} D_{Omega0^a}^{-1} D_{Omega0^a, ext} chi'
 *   (w chi)_{dPi1}       = (Q chi)_{dPi1} - P_{dPi1} D_{Lambda1}^{-1} D_{Lambda1, dLambda0} chi
 * (the block inverses of D_Phi, D_Omega and D_Lambda1 turn the printed blocks
 * into these two stages: frame pieces and frame in one batched solve, then the
 * framed blocks in a second).  W_u = u - w.  Without dPi1 (one decomposed
 * direction) Q = 0.  Solves to params->tol; dd_last_solve_stats merges both
 * stages.  Synchronises. */
dd_status dd_apply_w(dd_ctx* ctx, int n_f, const double* chi, double* w_chi,
                     const dd_solve_params* params, void* stream);

/* ---- w in stages, for a subset of blocks (paper Sec. 5: blocks on separate
 * nodes or GPUs) ------------------------------------------------------------
 * The three stages of dd_apply_w as separate calls, so that ranks owning
 * disjoint subsets of the blocks can each compute their part and combine the
 * results with sums across ranks:
 *   DD_W_FRAME_Q  in = chi; writes on every dPi1 entry of out the share of Q chi
 *                 of the listed blocks, sum over b in ids of P_{dPi1} D_{Phi1^b}^{-1}
 *                 D_{Phi1^b, dLambda0^b} chi (zero where none of their frame pieces
 *                 reaches); the sum over the ranks of these arrays is Q chi.
 *   DD_W_BLOCKS   in = chi' = chi - Q chi; writes (w chi)_{dLambda0^a} =
 *                 -P_{dLambda0^a} D_{Omega0^a}^{-1} D_{Omega0^a, ext} chi' on the
 *                 dLambda0^a entries of the listed blocks.
 *   DD_W_FRAME    in = chi (ids ignored); writes -P_{dPi1} D_{Lambda1}^{-1}
 *                 D_{Lambda1, dLambda0} chi on the dPi1 entries; adding Q chi gives
 *                 (w chi)_{dPi1}.
 * in, out: n_f fields in the layout of dd_apply_w, device or host; entries of
 * out that the stage does not write are left as they were.  ids: distinct
 * block ids.  Solves to params->tol.  Synchronises. */
#define DD_W_FRAME_Q 0
#define DD_W_BLOCKS 1
#define DD_W_FRAME 2
dd_status dd_apply_w_part(dd_ctx* ctx, int part, int n_f, const int* ids, int nblk, const double* in,
                          double* out, const dd_solve_params* params, void* stream);

/* ---- multi-boson action (paper Sec. 4, Eqs. MBaction, localMB, globalMB)
 * S = sum_k |(u_k - w) chi_k|^2 = sum_a S^a + S^r with
 * S^a = sum_k |P_{dLambda0^a}(u_k - w)chi_k|^2, S^r = sum_k |P_{dPi1}(...)|^2.
 * u: 2*n_f doubles (re, im); chi as for dd_apply_w.  S, S_r: host doubles;
 * S_block: host array of nblocks doubles or NULL.  FP64 reductions in a fixed
 * order (deterministic).  Synchronises. */
dd_status dd_multiboson_action(dd_ctx* ctx, int n_f, const double* u, const double* chi,
                               double* S, double* S_block, double* S_r,
                               const dd_solve_params* params, void* stream);

/* ---- multi-boson fields by heat-bath (paper Sec. 4, the fields of Eq. WW)
 * chi_k = W_{u_k}^{-1} eta_k for n_f fields, so that chi_k has the weight
 * exp(-|W_{u_k} chi_k|^2) when eta_k is complex Gaussian with density
 * exp(-|eta|^2).  u: 2*n_f doubles (re, im), no root zero; eta, chi: layout of
 * dd_apply_w, device or host.  BiCGstab on dPi over all fields at once, each
 * matvec one dd_apply_w batch (block and frame solves to params->tol), from
 * chi = eta / u, until |eta - W_u chi| <= tol |eta| per field or maxiter
 * iterations.  Returns DD_ENOCONV (stats filled) if a field missed tol.
 * Synchronises. */
typedef struct {
  int iterations;      /* BiCGstab iterations run (all fields together) */
  int matvecs;         /* dd_apply_w batches */
  int converged;       /* fields with relative residual <= tol */
  double max_relres;   /* largest |eta - W_u chi| / |eta| (recursive residual) */
  double seconds;      /* device time of the call */
} dd_heatbath_stats;
dd_status dd_multiboson_heatbath(dd_ctx* ctx, int n_f, const double* u, const double* eta,
                                 double* chi, double tol, int maxiter,
                                 const dd_solve_params* params, dd_heatbath_stats* stats,
                                 void* stream);

/* ---- force of the factorized multi-boson action (paper Sec. 4, Eq. localMB) --
 * The active links of block a are the links U_mu(x) with x and x + mu both in
 * its core Lambda0^a (an undecomposed direction's core is its whole periodic
 * extent).  Of S = sum_a S^a + S^r only S^a depends on them, through
 * D_{Omega0^a}.  For each active link and each generator T_t = lambda_t / 2
 * (Gell-Mann, t = 0..7) the call returns
 *   F[x][mu][t] = d S / d eps  at  U_mu(x) -> exp(i eps T_t) U_mu(x),
 * with y_k = D_Omega^{-1} D_{Omega,ext} chi'_k (chi' = chi - Q chi as in
 * dd_apply_w: frame links only), r_k = P_{dLambda0^a}(u_k chi_k + y_k),
 * z_k = (D_Omega^dag)^{-1} r_k = gamma_5 D_Omega^{-1} gamma_5 r_k and
 * dS = -2 Re sum_k <z_k, dD_Omega y_k>: a batched frame-piece solve (for Q),
 * two batched block solves (all blocks, all fields, params as for
 * dd_solve_blocks) and one thread per link (FP64).
 * u: 2*n_f doubles (re, im); chi: layout of dd_apply_w, device or host.
 * F: device or host, V*4*8 doubles, [global site (x3 fastest)][mu][t]; zero
 * on every link that is not active.  Returns DD_ENOCONV (F filled) if a block
 * solve missed its tolerance.  Synchronises. */
dd_status dd_mb_force(dd_ctx* ctx, int n_f, const double* u, const double* chi, double* F,
                      const dd_solve_params* params, void* stream);

/* ---- force of ln|det D_Omega0^a| (paper Sec. 4, Eq. SFeffN) -------------------
 * The other block-local term of the factorized effective action: for every
 * active link (as for dd_mb_force) and generator T_t, the noise estimate
 *   G[x][mu][t] = (1/n) sum_k Re <(D_Omega^dag)^{-1} eta_k, dD_Omega/d eps eta_k>
 * of d ln|det D_Omega0^a| / d eps = Re Tr[D_Omega^{-1} dD_Omega/d eps]
 * (unbiased for noise with E[eta eta^dag] = 1, e.g. complex Gaussians with
 * Re, Im ~ N(0, 1/2)).  eta: n_noise noise vectors per framed block, the caller
 * layout of dd_solve_blocks on all blocks ([block][k][Omega site][12]), device or
 * host, drawn by the caller.  One batched solve z = gamma_5 D_Omega^{-1} gamma_5 eta
 * (params as for dd_solve_blocks) and one thread per link (FP64).  G: device or
 * host, V*4*8 doubles, zero off the active links.  The block-local force of the
 * factorized effective action is dd_mb_force's F minus G.  Returns DD_ENOCONV
 * (G filled) if a solve missed its tolerance.  Synchronises. */
dd_status dd_logdet_force(dd_ctx* ctx, int n_noise, const double* eta, double* G,
                          const dd_solve_params* params, void* stream);

/* ---- block-local molecular dynamics (paper Sec. 4, Eq. SFeffN; Sec. 5) --------
 * The factorization decouples the active links of different blocks, so they
 * evolve together in one trajectory with the Hamiltonian
 *   H = 1/2 sum_{active (x,mu)} sum_t P_t(x,mu)^2 + S_MB + S_pf,
 *   S_MB = sum_k |W_{u_k} chi_k|^2 (as dd_multiboson_action; only its S^a move),
 *   S_pf = sum_a |(D_{Omega0^a}^dag)^{-1} phi_a|^2,
 * where the pseudofermion phi_a on Omega0^a stands for det(D_Omega^dag D_Omega) =
 * (det D_{Omega0^a})^2, the block determinant of Eq. SFeffN for two degenerate
 * flavours (chi then holds the multi-boson fields of both flavours).
 *
 * dd_pf_heatbath: phi_a = D_{Omega0^a}^dag eta_a = gamma_5 D_Omega gamma_5 eta_a for
 * every block (FP64), so that S_pf = |eta|^2.  eta, phi: layout of
 * dd_solve_blocks for all blocks with one rhs, [block][Omega0^a field-order
 * site][12] complex, device or host.  Synchronises.
 *
 * dd_md_trajectory: nsteps leapfrog steps of size dt = tau / nsteps from the
 * context's links and the momenta P (P -= dt/2 F; U_mu(x) -> exp(i dt sum_t P_t
 * T_t) U_mu(x), T_t = lambda_t / 2; P -= dt/2 F; merged half steps inside,
 * nsteps + 1 force evaluations), where F = dS_MB/d eps + dS_pf/d eps on the
 * active links (dd_mb_force; the pseudofermion force -2 Re <Y, dD X> with
 * Y = (D^dag)^{-1} phi, X = D^{-1} Y from two batched block solves).  The links
 * of the context are updated in place (FP64 scaling-and-squaring exponential);
 * every solve runs with `params`.  P: V*4*8 doubles, [global site][mu][t],
 * device or host, in and out; entries off the active links are ignored and
 * returned as zero.  n_f = 0 (u, chi null) drops S_MB; phi null drops S_pf;
 * at least one must be present.  stats: H and its parts at both ends.
 * DD_EINVAL with the clover term on.  Returns DD_ENOCONV (all outputs filled)
 * if a solve missed its tolerance.  Synchronises. */
typedef struct {
  double H0, H1;               /* H at the start and at the end */
  double kinetic0, kinetic1;   /* 1/2 sum P^2 over the active links */
  double s_mb0, s_mb1;         /* S_MB (0 without fields) */
  double s_pf0, s_pf1;         /* S_pf (0 without phi) */
  int steps, force_evals;
  double seconds;              /* device time of the trajectory */
} dd_md_stats;
dd_status dd_pf_heatbath(dd_ctx* ctx, const double* eta, double* phi, void* stream);
dd_status dd_md_trajectory(dd_ctx* ctx, int n_f, const double* u, const double* chi, const double* phi,
                           double* P, double tau, int nsteps, const dd_solve_params* params,
                           dd_md_stats* stats, void* stream);

/* ---- reweighting factor (paper Sec. 4, Eq. rw) ------------------------------
 * W_N = det{1 - R_{N+1}(W_1)}, W_1 = 1 - w on dPi, with the polynomial of the
 * roots below: R_{N+1}(z) = T_{N+1}((1-z)/c) / T_{N+1}(1/c) for c > 0 and
 * (1-z)^{N+1} for c = 0 (T the Chebyshev polynomials).  The paper gives no
 * estimator; this call returns, for each of n_src sources eta (complex
 * Gaussian of density exp(-|eta|^2), drawn by the caller, layout of
 * dd_apply_w, device or host), the sample
 *   s = |eta|^2 - |M eta|^2,  M = 1 - R_{N+1}(W_1),
 * whose exponential has the mean E[exp(s)] = 1/det(M^dag M) = |W_N|^-2 (finite
 * variance when every eigenvalue of M^dag M exceeds 1/2, i.e. R small: thick
 * frames).  R eta is built from N + 1 dd_apply_w batches over all sources
 * (Chebyshev recurrence in w, block and frame solves to params->tol) and s is
 * formed as 2 Re(eta, R eta) - |R eta|^2 (FP64, fixed-order sums).
 * N even >= 2, 0 <= c < 1, 1 <= n_src <= 65535.  s: host, n_src doubles.
 * r_eta: NULL, or a device or host buffer of the layout of eta that receives
 * R_{N+1}(W_1) eta.  Returns DD_ENOCONV (samples filled) if an inner solve
 * missed its tolerance.  Synchronises. */
dd_status dd_reweight_samples(dd_ctx* ctx, int N, double c, int n_src, const double* eta,
                              double* s, double* r_eta, const dd_solve_params* params,
                              void* stream);

/* ---- roots (paper Sec. 4) --------------------------------------------------
 * u_k = 1 - z_k = cos(2 pi k/(N+1)) + i sqrt(1-c^2) sin(2 pi k/(N+1)),
 * k = 1..N/2: the roots that carry the N/2 multi-boson fields (conjugates
 * u_{N+1-k} pair with them).  N even >= 2, 0 <= c < 1.  u: host, N doubles. */
dd_status dd_roots(int N, double c, double* u);

/* ---- dense check of the factorization (paper Sec. 3, Eq. detD) -------------
 * On small lattices (12 V <= 8192) assembles D, D_Lambda1, every D_Omega0^a,
 * every D_Phi1^a and W_1 = 1 - w on the GPU (the library's operators applied
 * to unit vectors; w's solves use `params`, e.g. FP64 to 1e-12) and
 * factorises each with an FP64 complex LU with partial pivoting, to check
 *   ln|det D| = ln|det W_1| + ln|det D_Lambda1| + sum_a ln|det D_Omega0^a|
 *               - sum_a ln|det D_Phi1^a|
 * and the corresponding phases.  logabs_omega / logabs_phi: host arrays of
 * nblocks doubles or NULL.  Synchronises; allocates work space. */
typedef struct {
  double logabs_D, logabs_W1, logabs_Lambda1;
  double logabs_Omega, logabs_Phi;   /* sums over the blocks */
  double phase_D;                    /* arg det D in (-pi, pi] */
  double phase_rhs;                  /* arg of det W1 det D_L1 prod det D_Omega / prod det D_Phi */
  double residual;                   /* logabs_D minus the right-hand side */
  int dim_D, dim_W1, dim_Lambda1;
} dd_logdet_report;
dd_status dd_logdet_check(dd_ctx* ctx, const dd_solve_params* params, double* logabs_omega,
                          double* logabs_phi, dd_logdet_report* report, void* stream);

/* ---- learned block preconditioner (no counterpart in the paper's method: its
 * only learning-related passage, Sec. 5 on flow-based models, is different).
 * Used as the initial guess of the framed-block solves.
 * A gauge-covariant network of linear parallel-transport convolutions on a
 * framed block Omega0^a (Dirichlet boundary): one layer maps C_in channels of
 * colour 3-vectors to C_out,
 *   y_c(x) = sum_{d in {0,+-mu}} sum_c' W[d][c][c'] (T_d phi_c')(x),
 *   T_+mu phi(x) = U_mu(x) phi(x+mu), T_-mu phi(x) = U_mu(x-mu)^+ phi(x-mu),
 * weights complex, [layer][d = 0, +0..+3, -0..-3][c_out][c_in], complex128
 * (re, im) on the host.  Supported layers 4->16, 16->16, 16->4 (input and
 * output: the 4 spin components of a spinor).  FP32 master weights (Adam),
 * BF16-rounded weights in the kernels.  The forward and backward-data layers
 * run on the tensor cores (tcgen05.mma, BF16 operands: the weights and the
 * parallel-transported activations, FP32 accumulation in tensor memory) by
 * default, or on the FP32 CUDA cores (FP32 activations and accumulation)
 * after dd_net_tensor_cores(net, 0); the weight gradients run on the CUDA
 * cores (FP32) in both cases. */
typedef struct dd_net dd_net;
typedef struct {
  int steps;          /* full-batch Adam steps */
  double lr;          /* Adam learning rate */
  double solve_tol;   /* tolerance of the FP64 solves that make the targets (e.g. 1e-10) */
} dd_train_params;
typedef struct {
  double loss_first;  /* mean |N(b) - x|^2 / |x|^2 before the first step */
  double loss_last;   /* after the last step */
  int steps, pairs;
  double seconds;     /* device time: target solves + training */
} dd_train_stats;
dd_status dd_net_create(dd_ctx* ctx, int nlayers, const int* channels, const double* weights,
                        dd_net** net);
dd_status dd_net_destroy(dd_net* net);
dd_status dd_net_weights(const dd_net* net, double* weights);  /* FP32 masters -> host */
/* Network to / from a file (the learned block preconditioner of the rows
 * above; the paper has no learned component in its method): layer channels,
 * FP32 master weights and the Adam state, so training resumes exactly.
 * dd_net_save returns DD_EINVAL if the file cannot be written; dd_net_load
 * returns DD_EINVAL (text in dd_last_error) for a missing or foreign file and
 * creates the network on ctx's device like dd_net_create. */
dd_status dd_net_save(const dd_net* net, const char* path);
dd_status dd_net_load(dd_ctx* ctx, const char* path, dd_net** net);
/* out = N(in) on framed blocks ids (device pointers, caller layout of dd_solve_blocks). */
dd_status dd_net_apply(dd_ctx* ctx, dd_net* net, const int* ids, int nblk, int nrhs,
                       const double* in, double* out, void* stream);
/* Mean loss over the (b, x) pairs and its gradient with respect to the weights
 * (dL/dRe + i dL/dIm, host, weight layout), evaluated with the BF16-rounded
 * weights.  Device pointers.  Synchronises. */
dd_status dd_net_loss_grad(dd_ctx* ctx, dd_net* net, const int* ids, int nblk, int nrhs,
                           const double* b, const double* x, double* loss, double* grads,
                           void* stream);
/* Trains on framed blocks ids: targets x = D_Omega^{-1} b from the library's FP64
 * solver for the given right-hand sides b (device pointer), then full-batch Adam
 * steps on the GPU.  Synchronises. */
dd_status dd_net_train(dd_ctx* ctx, dd_net* net, const int* ids, int nblk, int nrhs,
                       const double* b, const dd_train_params* params, dd_train_stats* stats,
                       void* stream);
/* Layers of the network on the tensor cores (on != 0, the default) or on the
 * FP32 CUDA cores (on = 0).  Host-only. */
dd_status dd_net_tensor_cores(dd_net* net, int on);
/* Network used by DD_SOLVE_NET_GUESS on this context (NULL to clear; not owned). */
dd_status dd_set_net(dd_ctx* ctx, dd_net* net);

/* ---- kernel timing -----------------------------------------------------
 * With timing on, the library brackets every launch of its stencil kernels
 * with CUDA events on the launching stream, and so every launch of the force
 * kernel of dd_mb_force.  dd_timing_get returns, for kernel class `which`
 * (0: FP64 hop, 1: FP32 hop, 2: BF16 hop, 3: force), the summed device time
 * in ms, the number of launches and the summed algorithmic bytes (class 3:
 * algorithmic FP64 flops, 576 per active link and field: 72 complex
 * multiply-adds), then clears the record.  Synchronises. */
dd_status dd_timing_enable(dd_ctx* ctx, int on);
dd_status dd_timing_get(dd_ctx* ctx, int which, double* ms, long long* launches,
                        double* bytes);

/* ---- stencil without device allocation -------------------------------------
 * The paper has no counterpart: this entry point is for callers that must not
 * allocate GPU memory during a call (a host that budgets all device memory up
 * front, an external caching allocator that must own every allocation, or
 * code that cannot take the implicit synchronisation of cudaMalloc/cudaFree).
 * It computes the same FP64 result as dd_apply_D_block(..., DD_F64, ...) with
 * the same caller layout, but takes its scratch (packed copies and launch
 * descriptors) from one static device array of DD_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library keeps until the process exits, and reads the
 * links from the context's global FP64 gauge copy.  in/out must be device
 * pointers.  Requests whose scratch exceeds the array (about 64 MiB / 384 B
 * per (site, rhs) pair) return DD_EINVAL with the size in dd_last_error.
 * Phi1 domains must have been built by an earlier dd_apply_D_block or
 * dd_solve_blocks call on them.  Every call shares the array: calls whose GPU
 * work overlaps (other streams or threads) race, so serialise them.  The first
 * call on each device resolves the array's address (cudaGetSymbolAddress);
 * with lazy module loading that first call also loads the module on the device
 * and commits the array, so it is the one call that takes device memory: make
 * it during set-up.  The launch descriptors pass through one host staging
 * buffer shared by all calls, threads and devices (a lock serialises it until
 * the copy has read it); a call on a stream that is being captured returns
 * DD_EINVAL, since a recorded copy would read that buffer only when the graph
 * runs.  Asynchronous on `stream`; calls no allocating routine. */
#define DD_NOALLOC_SCRATCH_BYTES (64u << 20)
dd_status dd_apply_D_block_noalloc(dd_ctx* ctx, dd_domain kind, const int* ids, int nblk,
                                   int nrhs, const double* in, double* out, void* stream);

/* Measured FP64 fused multiply-add rate of the current device in TFLOP/s
 * (best of three timed launches of independent FMA chains on every SM, after
 * one warm-up launch; clocks as they are).  The ALU roofline of the FP64
 * kernels (the force contraction, the plain FP64 stencil).  No counterpart in
 * the paper.  Synchronises the legacy default stream. */
dd_status dd_fp64_fma_rate(double* tflops);

/* Number of CUDA kernel launches the library has issued in this process
 * (all contexts), for launch accounting by callers.  Host-only, no sync. */
dd_status dd_launch_count(long long* n);

#ifdef __cplusplus
}
#endif
#endif /* DD4D_H */
