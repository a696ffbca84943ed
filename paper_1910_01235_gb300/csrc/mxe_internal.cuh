// mxe_internal.cuh -- types and launchers shared by the CUDA translation units
// of the MXE library (never included by the oracle, never exported).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mxe.h"
#include "ff.cuh"

namespace mxe {

constexpr int kMaxS = MXE_MAXS;
constexpr int kMaxPhiFn = MXE_MAXS * (MXE_MAXS + 1) / 2;  // distinct symmetric pair terms
constexpr int kMaxFFn = MXE_MAXS * MXE_MAXS;              // distinct density terms
constexpr int kCodeShift = 27;                            // neighbour entry: j | image code << 27
constexpr uint32_t kIdxMask = (1u << kCodeShift) - 1u;
constexpr int kReduceGroup = 1024;                        // sites per fixed-order partial sum
constexpr int kFireGroup = 256;                           // sites per partial sum of the FIRE reduction
constexpr double kKB = 8.617333262e-5;                    // eV/K
constexpr double kSqrt6 = 2.449489742783178098197284;     // node offset / sigma (App. A, r^2 = 3)
constexpr double kRMin = 0.5;                             // smallest admissible node distance
constexpr double kRhoMin = 1e-12;                         // smallest admissible static density
constexpr double kXTol = 1e-12;                           // admissible excursion of x
constexpr double kSigmaMin = 1e-3;                        // FIRE floor on sigma
constexpr double kLogFloor = 1e-300;                      // ln-argument floor of the full mu

// Device status bits (ORed by kernels, mapped to mxe_status by the host).
enum : int {
  kFlagGeometry = 1,
  kFlagNonfinite = 2,
  kFlagXRange = 4,
  kFlagBoxTooSmall = 8,
  kFlagOverflow = 16,
};

// One distinct radial term g(r) = A exp(kappa - lambda r) S(r).
//  FP64: A, kappa, lambda.  FP32: g_raw = exp2(c0 - c1 r) with
//  c0 = log2(A) + kappa log2(e), c1 = lambda log2(e).
//  Float-float: g_raw = exp(lnA_kappa - lambda r) with both constants as float pairs.
struct RadialFn {
  double A, kappa, lambda;  // kind 0: A exp(kappa - lambda r); kind 1: A ((kappa / r)^12 - (kappa / r)^6)
  float c0, c1, lam_f;
  int on;
  int kind;
  ff lnA_kappa_ff, lambda_ff;
};

// Potential in the form the kernels read (passed by value).
struct DevPot {
  int S;
  int lj;  // pair terms of kind 1 (FP64 passes only)
  int n_phi, n_f;
  RadialFn phi[kMaxPhiFn];
  RadialFn f[kMaxFFn];
  int8_t phi_of[kMaxS][kMaxS];   // species pair -> distinct phi term (-1: zero)
  int8_t f_of[kMaxS][kMaxS];     // species pair -> distinct f term (-1: zero)
  double E[kMaxS];
  int tab;                       // 1: the binary alloy pattern below, 0: general tables
  int cross_geo;                 // the cross pair term is the geometric mean of the like pairs
  // Power form (tab 1 with cross_geo): for each species s one base rate
  // beta_s with phi_ss = pw_pref_phi[2s] c_s^pw_m[s], f_s = pw_pref_f[s]
  // c_s^pw_n[s] and the cross term pw_pref_phi[1] c_0^(pw_m[0]/2)
  // c_1^(pw_m[1]/2), c_s = exp(-beta_s r): two exponentials per node
  int pw_on;
  int pw_m[2], pw_n[2];
  double pw_beta[2], pw_pref_phi[3], pw_pref_f[2];
  ff pw_beta_ff[2], pw_pref_phi_ff[3], pw_pref_f_ff[2];
  double rs, rc, inv_w;          // switch start, cutoff, 1/(rc - rs)
  float rs_f, rc_f, inv_w_f, dS_scale_f;
  ff rs_ff, inv_w_ff, dS_scale_ff;
};

// Species-pair tables known at compile time.  Pattern 1 is the usual binary
// EAM alloy: two like pair terms and one cross term, numbered in the order
// the distinct terms are found (phi_of = {{0, 1}, {1, 2}}), and a density
// that depends only on the neighbour's species (f_of[k][l] = l); the kernels
// specialised for it fold every table lookup and run no loop over absent
// terms.
template <int TAB>
struct Tables {
  static __device__ __forceinline__ int phi(const DevPot& P, int k, int l) { return P.phi_of[k][l]; }
  static __device__ __forceinline__ int f(const DevPot& P, int k, int l) { return P.f_of[k][l]; }
  static __device__ __forceinline__ int n_phi(const DevPot& P) { return P.n_phi; }
  static __device__ __forceinline__ int n_f(const DevPot& P) { return P.n_f; }
};
template <>
struct Tables<1> {
  static __device__ __forceinline__ constexpr int phi(const DevPot&, int k, int l) { return k + l; }
  static __device__ __forceinline__ constexpr int f(const DevPot&, int, int l) { return l; }
  static __device__ __forceinline__ constexpr int n_phi(const DevPot&) { return 3; }
  static __device__ __forceinline__ constexpr int n_f(const DevPot&) { return 2; }
};
// pattern 1 whose terms are also in the power form with m = 6, n = 10 (see
// DevPot::pw_on): the FP64 force pass forms them as products
template <>
struct Tables<2> : Tables<1> {};

// Box / cell grid for positions and image codes.
struct DevGrid {
  double L[3], invL[3], h[3];
  float h_f[3], h_lo[3], L_f[3], invL_f[3];  // h = h_f + h_lo (float pair)
  int nc[3];
};

// Several independent periodic systems in one context (sites of system s are
// the contiguous range [sys_off[s], sys_off[s+1])).  nsys == 0: one system,
// every kernel uses the DevGrid it receives by value.
constexpr int kMaxSystems = 1 << 20;

struct Batch {
  int nsys;
  const int* sys_of;      // [n] system of each site
  const DevGrid* grids;   // [nsys] box and cell grid of each system
  const int* cell_base;   // [nsys + 1] first global cell of each system
  const int* cell_sys;    // [ncell] system of each global cell
  const int* sys_off;     // [nsys + 1] first site of each system
};

__device__ __forceinline__ DevGrid site_grid(const DevGrid& g, const Batch& B, int64_t i) {
  return B.nsys ? B.grids[B.sys_of[i]] : g;
}

// FIRE / relaxation control block living in device memory.
struct Ctrl {
  int flags;          // kFlag* bits
  int halted;         // nonzero: remaining kernels of the chunk return at once
  int reason;         // 1 converged, 2 max_iter, 3 rebuild needed, 4 error
  int iter;           // FIRE updates done
  int n_pos;
  int max_iter;
  double dt, alpha;
  double ftol, skin;
  double sigma_max_build;
  double fmax;        // last max_i max(|g_q,i|, |g_sigma,i|)
  unsigned long long fmax_bits;   // atomicMax of non-negative doubles
  unsigned long long disp2_bits;  // max_i |q_i - q_build,i|^2 after the update
  unsigned long long smax_bits;   // max_i sigma_i after the update
  // scalars of the current update
  double keep, mix, one_minus_alpha;
  // FIRE constants
  double dt_max, f_inc, f_dec, alpha0, f_alpha;
  double sigma_lo, sigma_hi;      // box of the widths
  int n_min;
  // staggered runs captured in a graph
  int phase;          // 0: before the Euler step of the current step, 1: after it
  int steps;          // completed steps
  unsigned int red_ticket;  // blocks of the current FIRE reduction or update done (0 between launches)
};

enum { kReasonNone = 0, kReasonConverged = 1, kReasonMaxIter = 2, kReasonRebuild = 3, kReasonError = 4,
       kReasonAllDone = 5 };

// FIRE state of one system of a batch (the global Ctrl keeps the constants,
// the skin maxima and the global halt).
struct SysFire {
  int halted, reason, iter, n_pos;
  double dt, alpha, keep, mix, one_minus_alpha, fmax;
  double P, vv, ff;
};

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// scheduled while the previous kernel of its stream is finishing; it calls
// pdl_wait() before reading anything an earlier kernel wrote
// (griddepcontrol.wait returns once the prerequisite grids have completed and
// their memory is visible) and pdl_trigger() to let the next kernel be
// scheduled early in the same way.  In a kernel launched normally both are
// no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t shm, cudaStream_t s,
                              Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = shm;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Blocks of a grid-stride pass: the kernel's resident blocks on every SM (one
// wave; a launch that returns at once then costs one wave, not one block per
// work item), or fewer when the work is smaller.
int64_t resident_grid(const void* kernel, int threads, int64_t work_items);

// ---------------------------------------------------------------- launchers
// neighbours.cu
cudaError_t launch_cell_assign(const double* q, int64_t n, const DevGrid& g, const Batch& B, int* cell_of,
                               int* cell_slot, int* cell_count, int* abs_cell, float4* qf, cudaStream_t s);
cudaError_t launch_cell_place(int64_t n, const int* cell_of, const int* cell_slot, const int* cell_start,
                              int* cell_sites, cudaStream_t s);
cudaError_t launch_nbr_count(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                             const DevGrid& g, const Batch& B, const int* cell_of, const int* cell_start, const int* cell_sites,
                             double rl2, double rb2, float band, int* nb_cnt, int* bd_cnt, int* max_row,
                             cudaStream_t s);
cudaError_t launch_nbr_fill(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                            const DevGrid& g, const Batch& B, const int* cell_of, const int* cell_start, const int* cell_sites,
                            const int* abs_cell, double rl2, double rb2, float band, const int* nb_off,
                            uint32_t* nb_ent, const int* bd_off, int* bd_idx, int max_row, cudaStream_t s);
// cell-staged variants (one block per cell, candidates staged in shared memory)
cudaError_t launch_cand_max(int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, int* out,
                            cudaStream_t s);
size_t cell_stage_bytes(int cand_cap, int max_row, bool fill);
// out[t] = the last segment s with base[s] <= t, for t < count (base: nseg + 1 nondecreasing starts)
cudaError_t launch_segment_ids(const int* base, int nseg, int64_t count, int* out, cudaStream_t s);
cudaError_t launch_cell_count(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                              int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, const int* cell_sites,
                              double rl2, double rb2, float band, int cand_cap, int* nb_cnt, int* bd_cnt,
                              int* max_row, int* flags, cudaStream_t s);
cudaError_t launch_cell_fill(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                             int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, const int* cell_sites,
                             const int* abs_cell, double rl2, double rb2, float band, int cand_cap,
                             const int* nb_off, uint32_t* nb_ent, const int* bd_off, int* bd_idx, int max_row,
                             int* flags, cudaStream_t s);
// unordered-pair index of a symmetric list (rows sorted by j): n_below[i] =
// entries of row i with j < i (the head), cnt[i] = the rest (the tail, the
// pairs row i owns); after a scan of cnt into pair_off, pair p has the record
// pair_rec[p] = (i, entry of j in row i with its image code, that entry's
// index, the index of the reverse entry i in row j) (kFlagOverflow if the
// list is not symmetric)
cudaError_t launch_pair_count(const int* nb_off, const uint32_t* nb_ent, int64_t n, int* n_below, int* cnt,
                              cudaStream_t s);
cudaError_t launch_pair_fill(const int* nb_off, const uint32_t* nb_ent, int64_t n, const int* n_below,
                             const int* pair_off, int64_t npair, int4* pair_rec, int* flags, cudaStream_t s);
// fill without a count pass: rows at a fixed stride (the previous build's
// longest row plus a margin), counts and the longest row; then the scan of the
// counts and the compaction into the CSR (a longer row: count + fill instead);
// with n_below / pair_cnt (may be null) also the half-list index's head and
// tail lengths of every row
cudaError_t launch_cell_fill_direct(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask,
                                    int64_t n, int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start,
                                    const int* cell_sites, const int* abs_cell, double rl2, double rb2, float band,
                                    int cand_cap, int stride, uint32_t* rows, int* brows, int* nb_cnt, int* bd_cnt,
                                    int* n_below, int* pair_cnt, int* row_max, int* flags, cudaStream_t s);
cudaError_t launch_row_compact(const uint32_t* rows, const int* brows, int stride, int64_t n, const int* nb_off,
                               const int* bd_off, uint32_t* nb_ent, int* bd_idx, cudaStream_t s);
// exclusive scan of n int32 counts into out[0..n] (out[n] = total, int64 total in *total64)
cudaError_t launch_scan(const int* in, int* out, int64_t n, long long* total64, int* tmp, int64_t tmp_len,
                        cudaStream_t s);
int64_t scan_tmp_len(int64_t n);
cudaError_t launch_strip_codes(const uint32_t* ent, int32_t* idx, int64_t m, cudaStream_t s);
cudaError_t launch_site_max(const double* sigma, const double* q, int64_t n, unsigned long long* out_bits,
                            cudaStream_t s);

// eam.cu
// pos32/x32: FP32 records; pos32lo/x32lo (optional): the float-pair remainders
cudaError_t launch_pack(const double* q, const double* sigma, const double* x, const int* abs_cell, int64_t n,
                        int S, const DevGrid& g, const Batch& B, float4* pos32, float4* x32, float4* pos32lo,
                        float4* x32lo, cudaStream_t s);
cudaError_t init_ff_exp_table();
struct PassArgs {
  const double* q;
  const double* sigma;
  const double* x;
  const double* T;
  const float4* pos32;
  const float4* x32;
  const float4* pos32lo;  // float-float passes: remainders of pos32, x32, ab32
  const float4* x32lo;
  const int* nb_off;
  const uint32_t* nb_ent;
  int64_t n;
  int64_t n_ent;    // neighbour entries of the list (bound of every entry index)
  // pass-1 outputs / pass-2 inputs
  double* rho_bar;
  double* rho_avg;
  double* a;
  double* b;
  double* e;
  float4* ab32;     // [n][2] packed (a_k, b_k) for the mixed pass-2 gathers
  float4* ab32lo;
  // pass-2 outputs
  double* gq;
  double* gs;
  double* mu_ex;
  double* mu;
  double* site_E;   // [3][n]: E_V, F_vib, F_mix per site
  Ctrl* ctrl;       // optional: kernels return at once if ctrl->halted
  int* flags;
  int check_skin;   // pass 1 checks the rebuild criterion in ctrl first
  int lean;         // FP32 density pass of the relaxation: write only the packed (a, b)
  Batch batch;      // several systems (nsys > 0): per-site box and cell grid
  int tpb;  // threads per block of the density and gradient passes (0: 256)
  int pair_tpb;  // threads per block of the pair kernels: pairs per block (64, 128, 256; else 128)
};
cudaError_t launch_density(int precision, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a,
                           cudaStream_t s);
enum { kGradAll = 0, kGradForce = 1, kGradMu = 2, kGradForceNoE = 3 };
cudaError_t launch_gradient(int precision, int mode, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a,
                            cudaStream_t s);
// half-list accurate passes: each unordered pair's record of
// pair_record_len(P) values (float pairs: float-float node arithmetic of the
// FP32 modes; doubles: FP64 contexts) written to both of its entries, then
// the density (mu = false) or chemical-potential gather over each site's own
// row (per-site sums in float-float for MXE_FP32_FF, FP64 otherwise).  Record
// components [0, 2 n_f) (the densities) and [2 n_f, 2 n_f + n_phi) (the pair
// terms) lie in two planes when they do not fit one 32-byte group: plane A
// [cap][ca] at buf, plane B [cap][cb] at buf + b_off (cap: entries allocated),
// so that the density gather reads plane A only.
struct GeoLayout {
  int ca, cb;      // values per entry in plane A and plane B (cb 0: one plane)
  int64_t b_off;   // plane B's first value
};
int pair_record_len(const DevPot& P);
GeoLayout geo_layout(const DevPot& P, int64_t cap);
int pair_threads(const PassArgs& A);
cudaError_t launch_pair_geo(int precision, const DevPot& P, const DevGrid& g, const PassArgs& A,
                            const int4* pair_rec, int64_t npair, void* buf, int64_t cap, cudaStream_t s);
cudaError_t launch_pair_gather(int precision, bool mu, int nl, const DevPot& P, const PassArgs& A, const void* buf,
                               int64_t cap, cudaStream_t s);
// half-list relaxation passes (FP32 node math in the FP32 modes, FP64 in FP64
// contexts): the pair kernel writes each pair's record to both of its entries
// (pair_t[p], pair_rev[p]); the gather then reads its own row: density (force
// = false: a, b packed into ab32, or the FP64 arrays a, b) or forces (dF/dq,
// dF/dsigma); dens, frc: [entries] records of relax_record_bytes(precision)
bool pair_kernels_supported(const DevPot& P);
size_t relax_record_bytes(int precision);
cudaError_t launch_relax_pair(int precision, bool force, const DevPot& P, const DevGrid& g, const PassArgs& A,
                              const int4* pair_rec, int64_t npair, void* dens, void* frc, cudaStream_t s);
cudaError_t launch_relax_gather(int precision, bool force, int nl, const DevPot& P, const PassArgs& A,
                                const void* dens, const void* frc, cudaStream_t s);
// exact phase average of the embedding term (App. B.2: App. A's rule over a
// site and its neighbours inside r_cut): per-site rule data of the first pass,
// read by the second
struct EmbArgs {
  double* rhob;   // [S][n] density at the mean positions (rule members only)
  double* rown;   // [6 S][n] density at the six nodes that move the site itself
  double* fsum;   // [S][n] sum over all M nodes of F_k'(rho(node))
  double* emb;    // [S][n] <F_k(rho)>
  int* nrule;     // [n] sites of the rule (the site and its members)
};
// node arithmetic in FP64 (fp64 = true) or FP32 (per-site sums in FP64); the
// second pass adds dF/dq, dF/dsigma and dE_V/dx into A.gq, A.gs, A.mu_ex (and
// A.mu), the first adds the embedding energy into A.site_E
cudaError_t launch_emb_exact(bool second, bool fp64, int nl, const DevPot& P, const DevGrid& g, const PassArgs& A,
                             const EmbArgs& E, cudaStream_t s);
cudaError_t launch_pack_ab(const double* a, const double* b, int64_t n, int S, float4* ab32, cudaStream_t s);
cudaError_t launch_energy_reduce(const double* site_E, int64_t n, double* partials, double* F4, cudaStream_t s);
// batches: F4 [nsys][4], one block per system in a fixed order
cudaError_t launch_energy_seg(const double* site_E, int64_t n, const Batch& B, double* F4, cudaStream_t s);

// relax.cu
cudaError_t launch_fire_reduce(const double* gq, const double* gs, const double* sigma, const double* vq,
                               const double* vs, int64_t n, double* partials, Ctrl* ctrl, int* flags, cudaStream_t s);
cudaError_t launch_fire_update(double* q, double* sigma, double* vq, double* vs, const double* gq,
                               const double* gs, const double* q_build, const int* abs_cell, int64_t n,
                               const DevGrid& g, const Batch& B, float4* pos32, Ctrl* ctrl, cudaStream_t s);
// batches: one block per system reduces, one block runs every system's FIRE logic
cudaError_t launch_fire_seg_reduce(const double* gq, const double* gs, const double* sigma, const double* vq,
                                   const double* vs, int64_t n, const Batch& B, SysFire* sf, Ctrl* ctrl, int* flags,
                                   cudaStream_t s);
cudaError_t launch_fire_seg_logic(SysFire* sf, int nsys, Ctrl* ctrl, const int* flags, cudaStream_t s);
cudaError_t launch_fire_seg_update(double* q, double* sigma, double* vq, double* vs, const double* gq,
                                   const double* gs, const double* q_build, const int* abs_cell, int64_t n,
                                   const DevGrid& g, const Batch& B, const SysFire* sf, float4* pos32, Ctrl* ctrl,
                                   cudaStream_t s);
cudaError_t launch_fire_seg_init(SysFire* sf, int nsys, double dt0, double alpha0, const Ctrl* gate, cudaStream_t s);
// staggered steps captured in a graph: per-step bookkeeping (a stop for a
// rebuild or an error is kept until the host clears it)
cudaError_t launch_step_begin(Ctrl* ctrl, double dt0, double alpha0, cudaStream_t s);
cudaError_t launch_step_end(Ctrl* ctrl, cudaStream_t s);
// end of the body of a device-side loop of steps (graph while node): sets
// the loop's condition; loop [3] = bodies run, step count to reach, cap
cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const Ctrl* ctrl, int* loop, cudaStream_t s);
cudaError_t launch_fire_zero_v(double* vq, double* vs, int64_t n, const Ctrl* gate, cudaStream_t s);

// deriv.cu: forward-mode (dual-number) density and gradient passes
struct TanArgs {
  const double *q, *sigma, *x, *T;           // state
  const double *dq, *dsigma, *dx;            // tangents ([3][n], [n], [S][n]; null: zero)
  const int* nb_off;
  const uint32_t* nb_ent;
  int64_t n;
  double *a_v, *a_t, *b_v, *b_t, *e_v, *e_t;  // [S][n] embedding terms (written by the density pass)
  double *gq_v, *gq_t, *gs_v, *gs_t, *mu_v, *mu_t;  // outputs, any may be null
  double *th_v, *th_t;                       // [2 T][n] per-site term sensitivities (null: skip)
  int* flags;
  Batch batch;
};
cudaError_t launch_tangent(const DevPot& P, const DevGrid& g, const TanArgs& A, cudaStream_t s);
cudaError_t launch_col_sum(const double* col, int ncol, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_flux_vjp(const double* x, const double* T, const double* mu, const int* bd_off, const int* bd_idx,
                            int64_t n, int S, double dt, double nu0, double Qm, const double* dt_sys,
                            const int* sys_of, const double* xbar1, double* xbar0, double* mubar, cudaStream_t s);
int64_t dot_partials_len(int64_t len);
cudaError_t launch_dot(const double* a, const double* b, int64_t len, double* part, double* out, cudaStream_t s);
// y = alpha x + beta y
cudaError_t launch_axpby(double* y, const double* x, double alpha, double beta, int64_t len, cudaStream_t s);

// flux.cu
int64_t flux_scratch_len(int64_t n, int S);
// with reservoir groups (any pointer may be null); mu_eff: [S][n] scratch
cudaError_t launch_flux_res(const double* x, const double* T, const double* mu_ex, const int* bd_off,
                            const int* bd_idx, int64_t n, int S, double dt, double nu0, double Qm, double* scratch,
                            double* x_new, int* flags, const uint8_t* fix_x_mask, const double* fix_x_value,
                            const uint8_t* fix_mu_mask, const double* fix_mu_value, double* mu_eff,
                            const double* dt_sys, const int* sys_of, Ctrl* gate, cudaStream_t s);
cudaError_t launch_flux(const double* x, const double* T, const double* mu_ex, const int* bd_off, const int* bd_idx,
                        int64_t n, int S, double dt, double nu0, double Qm, double* scratch, double* x_new,
                        int* flags, cudaStream_t s);
// transport variants (host exchange, ballistic term): flux into x_new / v_new
// and a conditional commit of x and v (x is written through the commit only)
cudaError_t launch_transport_ext(double* x, const double* T, const double* mu_ex, const int* bd_off,
                                 const int* bd_idx, int64_t n, int S, double dt, double nu0, double Qm, int host,
                                 double tau, double* v, double* v_new, double* x_new, int* step_flags, int* flags,
                                 const double* dt_sys, const int* sys_of, cudaStream_t s);
// gate (optional): nothing runs while gate->halted; a range error stops the
// run (gate->reason = error), a commit sets gate->phase = 1
cudaError_t launch_commit_x(double* x, const double* x_new, int64_t count, const int* step_flags, int* flags,
                            Ctrl* gate, cudaStream_t s);

}  // namespace mxe
