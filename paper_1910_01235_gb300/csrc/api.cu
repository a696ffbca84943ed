// api.cu -- the C ABI declared in include/mxe.h: context, workspace ownership,
// call ordering and status mapping.  Every compute step is a kernel launched
// on the context's stream; this file holds host logic only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mxe_internal.cuh"

using namespace mxe;

// What a captured staggered step depends on beyond the context's own buffers.
struct StepKey {
  const double *q, *sigma, *x, *T;
  const uint8_t* sub;
  uint32_t mobile_mask;
  double dt, nu0, Qm;
  int32_t max_iter;
  double dt0, alpha0;
  int64_t list_gen;
  int32_t nl, tpb, pair_tpb;
};

inline bool same_key(const StepKey& a, const StepKey& b) {
  return a.q == b.q && a.sigma == b.sigma && a.x == b.x && a.T == b.T && a.sub == b.sub &&
         a.mobile_mask == b.mobile_mask && a.dt == b.dt && a.nu0 == b.nu0 && a.Qm == b.Qm &&
         a.max_iter == b.max_iter && a.dt0 == b.dt0 && a.alpha0 == b.alpha0 && a.list_gen == b.list_gen &&
         a.nl == b.nl && a.tpb == b.tpb && a.pair_tpb == b.pair_tpb;
}

struct mxe_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  int S = 1;
  int precision = 0;
  int nl = 8;
  mxe_box box{};
  mxe_potential pot{};
  DevPot dp{};
  DevPot dp_pair{};  // the potential with every embedding switched off (pair terms alone)
  // embedding average: 0 the Taylor form (Eq. F_taylor_mxe), 1 the exact rule
  int embedding = 0;
  double* emb_buf = nullptr;  // rule data of the exact average: (9 S) [n] doubles
  int* emb_nrule = nullptr;   // [n]
  DevGrid grid{};

  // cell grid
  int* cell_of = nullptr;
  int* cell_slot = nullptr;
  int* abs_cell = nullptr;  // [3][n]
  int* cell_count = nullptr;
  int* cell_start = nullptr;
  int* cell_sites = nullptr;
  float4* qf = nullptr;  // [2][n] FP32 positions for the neighbour prefilter: absolute, then within the cell
  int64_t ncell_cap = 0;

  // neighbour / bond CSR
  int* nb_cnt = nullptr;
  int* bd_cnt = nullptr;
  int* nb_off = nullptr;
  int* bd_off = nullptr;
  uint32_t* nb_ent = nullptr;
  int* bd_idx = nullptr;
  int64_t nb_cap = 0, bd_cap = 0;
  long long* scan_tmp = nullptr;
  int64_t scan_len = 0;
  long long* totals = nullptr;  // [4]: cells, neighbours, bonds, owned pairs
  int* max_row = nullptr;
  int cand_cap_prev = 0;  // largest stencil candidate set of the last build
  unsigned long long* smax_bits = nullptr;
  int64_t n_pairs = 0, n_bonds = 0;
  int max_row_h = 0;
  bool have_list = false;
  double r_list = 0, skin = 0.2, r_bond = 0, sigma_max_build = 0;
  double* q_build = nullptr;
  // unordered-pair index and records of the half-list passes (contexts whose
  // potential the pair kernels support)
  // per row: entries below its site (head), pairs it owns (tail), their scan
  int *n_below = nullptr, *pair_cnt = nullptr, *pair_off = nullptr;  // [n], [n], [n + 1]
  int4* pair_rec = nullptr;  // [pairs] (i, entry of j with its image code, entry index, reverse entry index)
  double* pair_buf = nullptr;  // pair_cap x pair_record_len 8-byte values (float pairs or doubles; see geo_layout)
  void *ent_dens = nullptr, *ent_frc = nullptr;  // [entries] relaxation records (relax_record_bytes each)
  bool relax_records = false;  // allocate them (first relaxation of the context, then with every list growth)
  int64_t pair_cap = 0, n_upairs = 0;
  // rows of a fill without a count pass, at a fixed stride
  uint32_t* rows_tmp = nullptr;
  int* brows_tmp = nullptr;
  int64_t rows_cap = 0;

  // per-site work arrays
  double *rho_bar = nullptr, *rho_avg = nullptr, *a = nullptr, *b = nullptr, *e = nullptr;
  float4 *pos32 = nullptr, *x32 = nullptr, *ab32 = nullptr;
  float4 *pos32lo = nullptr, *x32lo = nullptr, *ab32lo = nullptr;  // float-float remainders (FP32 modes)
  double *gq = nullptr, *gs = nullptr, *mu_ex = nullptr;
  double* site_E = nullptr;
  double* partials = nullptr;
  double* F4_tmp = nullptr;
  double *vq = nullptr, *vs = nullptr, *q0 = nullptr, *s0 = nullptr;
  double* x_new = nullptr;
  double* flux_tmp = nullptr;  // per-site factors of the Euler step
  double* mu_eff = nullptr;    // mu with the reservoir values
  // reservoir groups (caller-owned device arrays, kept until changed)
  const uint8_t* fix_x_mask = nullptr;
  const double* fix_x_value = nullptr;
  const uint8_t* fix_mu_mask = nullptr;
  const double* fix_mu_value = nullptr;
  int* flags = nullptr;
  int* step_flags = nullptr;
  Ctrl* ctrl = nullptr;

  // batch of independent systems (nsys == 0: one system, box above)
  int nsys = 0;
  std::vector<mxe_box> boxes;
  std::vector<int64_t> sys_off_h;
  int* sys_of = nullptr;        // [n]
  int* sys_off = nullptr;       // [nsys + 1]
  DevGrid* grids = nullptr;     // [nsys]
  int* cell_base = nullptr;     // [nsys + 1]
  int* cell_sys = nullptr;      // [ncell_cap]
  DevGrid* grids_h = nullptr;   // pinned staging of grids
  int* cell_base_h = nullptr;   // pinned staging of cell_base
  SysFire* sf = nullptr;        // [nsys] FIRE state of each system
  SysFire* sf_h = nullptr;      // pinned copy after a relaxation
  double* dt_sys = nullptr;     // [nsys] Euler step multipliers
  Batch B{};
  // pass shape: lanes per site and threads per block of the density/gradient
  // passes and gathers, threads (pairs) per block of the pair kernels
  int tpb = 256;
  int pair_tpb = 128;
  // captured staggered step
  int64_t list_gen = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;  // the run's loop: a while node around one captured step
  StepKey step_key{};
  int* loop_dev = nullptr;  // [3] device loop control (bodies run, step count to reach, cap)
  int* loop_h = nullptr;    // pinned staging of loop_dev
  int step_kernels = 0;     // kernel nodes of the captured step
  int run_launches = 0;     // graph launches of the last staggered run
  // second-order passes (allocated on first use)
  double* tan_buf = nullptr;   // a, b, e values and tangents: 6 [S][n]
  double* th_buf = nullptr;    // per-site term sensitivities, values and tangents: 2 x [2 T][n]
  double* th_sum = nullptr;    // [4 T]: sums of the values, then of the tangents
  double* dot_part = nullptr;  // partial sums of dot products
  double* dot_out = nullptr;   // [2]
  double* dot_h = nullptr;     // pinned [2]
  double* v_new = nullptr;     // [S][n] rates after a ballistic transport step (allocated on first use)
  // result of the last relaxation, per system (one entry without a batch)
  std::vector<int32_t> last_iters, last_reason;
  std::vector<double> last_fmax;

  // event timing (profiling): launches bracketed by events, filed by class
  bool timing = false;
  struct TimedLaunch {
    std::string cls;
    cudaEvent_t e0, e1;
  };
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;

  // pinned host mirrors
  Ctrl* ctrl_h = nullptr;
  long long* totals_h = nullptr;
  int* ints_h = nullptr;
  unsigned long long* bits_h = nullptr;
};

namespace {

struct Guard {  // keep the caller's current device, switch to the context's
  int prev = 0;
  bool ok = false;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~Guard() {
    if (ok) cudaSetDevice(prev);
  }
};

#define CK(call)                                  \
  do {                                            \
    cudaError_t _e = (call);                      \
    if (_e != cudaSuccess) return map_cuda(_e);   \
  } while (0)

mxe_status map_cuda(cudaError_t e) {
  cudaGetLastError();  // clear a non-sticky error so it does not surface in the caller's next CUDA call
  return e == cudaErrorMemoryAllocation ? MXE_ERR_OOM : MXE_ERR_CUDA;
}

cudaEvent_t take_event(mxe_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch `fn` (returning cudaError_t); with timing on, bracket it with events.
template <typename Fn>
cudaError_t timed(mxe_ctx* c, const std::string& cls, Fn&& fn) {
  if (!c->timing) return fn();
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  cudaEventRecord(e0, c->stream);
  cudaError_t e = fn();
  cudaEventRecord(e1, c->stream);
  c->timed.push_back({cls, e0, e1});
  return e;
}

const char* prec_name(int p) {
  static const char* names[] = {"fp64", "fp32_mixed", "fp32_ff", "ff"};
  return (p >= 0 && p < 4) ? names[p] : "?";
}

std::string cls_name(const char* pass, int prec, int mode = -1) {
  static const char* modes[] = {"all", "force", "mu", "force_noe"};
  std::string s = std::string(pass) + "_" + prec_name(prec);
  if (mode >= 0 && mode < 4) s += std::string("_") + modes[mode];
  return s;
}

#define TIMED(cls, call) timed(c, (cls), [&]() { return (call); })

// cudaMemcpyAsync / cudaMemsetAsync that accept an empty range with null pointers
cudaError_t copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}

template <typename T>
cudaError_t dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)count);
}

cudaError_t dalloc_bytes(void** p, int64_t bytes) {
  *p = nullptr;
  if (bytes <= 0) bytes = 16;
  return cudaMalloc(p, (size_t)bytes);
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

mxe_status map_flags(int f) {
  if (f & kFlagGeometry) return MXE_ERR_GEOMETRY;
  if (f & kFlagNonfinite) return MXE_ERR_NONFINITE;
  if (f & kFlagXRange) return MXE_ERR_X_RANGE;
  if (f & kFlagBoxTooSmall) return MXE_ERR_BOX_TOO_SMALL;
  if (f & kFlagOverflow) return MXE_ERR_NBR_OVERFLOW;
  return MXE_OK;
}

// Distinct radial terms of the potential (dedupe identical (A, kappa, lambda)).
int add_fn(RadialFn* tab, int& count, int cap, double A, double kappa, double lambda, int kind = 0) {
  if (A == 0.0) return -1;
  for (int u = 0; u < count; ++u)
    if (tab[u].A == A && tab[u].kappa == kappa && tab[u].lambda == lambda && tab[u].kind == kind) return u;
  if (count >= cap) return -2;
  RadialFn& F = tab[count];
  F.A = A;
  F.kappa = kappa;
  F.lambda = lambda;
  const double log2e = 1.4426950408889634;
  F.c0 = (float)(std::log2(A) + kappa * log2e);
  F.c1 = (float)(lambda * log2e);
  F.lam_f = (float)lambda;
  F.on = 1;
  F.kind = kind;
  F.lnA_kappa_ff = ff(std::log(A) + kappa);
  F.lambda_ff = ff(lambda);
  return count++;
}

// The power form of a binary pattern with a geometric-mean cross term: for
// each species s, integers m, n <= 16 with lambda(phi_ss) = m beta and
// lambda(f_s) = n beta (m even, so the cross term's exponent m/2 is whole),
// to 1e-15 relative (the rounding of rates computed from p / r0).  exp(c - lambda r) = exp(c) exp(-beta r)^m exactly in
// real arithmetic; the rounding of the power adds at most m ulps of the base.
void set_power_form(DevPot& d) {
  d.pw_on = 0;
  if (!(d.tab == 1 && d.cross_geo && !d.lj)) return;
  const int phi_of_s[2] = {0, 2};
  for (int s = 0; s < 2; ++s) {
    const double lp = d.phi[phi_of_s[s]].lambda, lf = d.f[s].lambda;
    if (!(lp > 0.0) || !(lf > 0.0)) return;
    int m = 0, n = 0;
    for (int nn = 1; nn <= 16 && !m; ++nn) {
      const double mm = std::nearbyint(lp / lf * nn);
      if (mm >= 1.0 && mm <= 16.0 && std::fabs(mm * lf - nn * lp) <= 1e-15 * nn * lp) {
        m = (int)mm;
        n = nn;
      }
    }
    if (!m) return;
    if (m % 2) {
      m *= 2;
      n *= 2;
    }
    if (m > 16 || n > 16) return;
    d.pw_m[s] = m;
    d.pw_n[s] = n;
    d.pw_beta[s] = lp / m;
  }
  // the cross term's rate must be the mean of the like rates (geometric mean)
  const double lx = d.phi[1].lambda, lmean = 0.5 * (d.pw_m[0] * d.pw_beta[0] + d.pw_m[1] * d.pw_beta[1]);
  if (std::fabs(lx - lmean) > 1e-15 * lx) return;
  for (int u = 0; u < 3; ++u) {
    d.pw_pref_phi[u] = d.phi[u].A * std::exp(d.phi[u].kappa);
    d.pw_pref_phi_ff[u] = ff(d.pw_pref_phi[u]);
  }
  for (int v = 0; v < 2; ++v) {
    d.pw_pref_f[v] = d.f[v].A * std::exp(d.f[v].kappa);
    d.pw_pref_f_ff[v] = ff(d.pw_pref_f[v]);
  }
  for (int s = 0; s < 2; ++s) d.pw_beta_ff[s] = ff(d.pw_beta[s]);
  d.pw_on = 1;
}

mxe_status make_devpot(const mxe_potential& p, DevPot& d) {
  std::memset(&d, 0, sizeof(d));
  const int S = p.n_species;
  if (S < 1 || S > 2) return MXE_ERR_ARG;  // kernels are instantiated for S = 1, 2
  if (!(p.r_cut > p.r_switch) || !(p.r_switch >= 0.0)) return MXE_ERR_ARG;
  d.S = S;
  for (int k = 0; k < kMaxS; ++k)
    for (int l = 0; l < kMaxS; ++l) d.phi_of[k][l] = d.f_of[k][l] = -1;
  for (int k = 0; k < S; ++k) {
    if (!(p.E[k] >= 0.0)) return MXE_ERR_ARG;
    d.E[k] = p.E[k];
    for (int l = 0; l < S; ++l) {
      if (!(p.phi_r0[k][l] > 0.0) || !(p.f_r0[k][l] > 0.0)) return MXE_ERR_ARG;
      if (p.phi_A[k][l] < 0.0 || p.f_xi[k][l] < 0.0) return MXE_ERR_ARG;
    }
  }
  d.lj = p.lj ? 1 : 0;
  for (int k = 0; k < S; ++k)
    for (int l = k; l < S && p.lj; ++l) {
      // thermalized Lennard-Jones pair terms: A = 4 eps, kappa = sigma
      const double eps = p.lj_eps[k][l], sg = p.lj_sigma[k][l];
      if (eps != p.lj_eps[l][k] || sg != p.lj_sigma[l][k] || !(eps >= 0.0) || !(sg > 0.0)) return MXE_ERR_ARG;
      int u = add_fn(d.phi, d.n_phi, kMaxPhiFn, 4.0 * eps, sg, 0.0, 1);
      if (u == -2) return MXE_ERR_ARG;
      d.phi_of[k][l] = d.phi_of[l][k] = (int8_t)u;
    }
  for (int k = 0; k < S; ++k)
    for (int l = k; l < S && !p.lj; ++l) {
      double A, kap, lam;
      if (p.cross_geomean && k != l) {
        // sqrt(phi_kk phi_ll) = sqrt(A_k A_l) exp((p_k + p_l)/2 - (p_k/r0_k + p_l/r0_l)/2 r) S(r)
        A = std::sqrt(p.phi_A[k][k] * p.phi_A[l][l]);
        kap = 0.5 * (p.phi_p[k][k] + p.phi_p[l][l]);
        lam = 0.5 * (p.phi_p[k][k] / p.phi_r0[k][k] + p.phi_p[l][l] / p.phi_r0[l][l]);
      } else {
        if (p.phi_A[k][l] != p.phi_A[l][k] || p.phi_p[k][l] != p.phi_p[l][k] || p.phi_r0[k][l] != p.phi_r0[l][k])
          return MXE_ERR_ARG;
        A = p.phi_A[k][l];
        kap = p.phi_p[k][l];
        lam = p.phi_p[k][l] / p.phi_r0[k][l];
      }
      int u = add_fn(d.phi, d.n_phi, kMaxPhiFn, A, kap, lam);
      if (u == -2) return MXE_ERR_ARG;
      d.phi_of[k][l] = d.phi_of[l][k] = (int8_t)u;
    }
  for (int k = 0; k < S; ++k)
    for (int l = 0; l < S; ++l) {
      int v = add_fn(d.f, d.n_f, kMaxFFn, p.f_xi[k][l], p.f_q[k][l], p.f_q[k][l] / p.f_r0[k][l]);
      if (v == -2) return MXE_ERR_ARG;
      d.f_of[k][l] = (int8_t)v;
    }
  d.tab = (S == 2 && d.n_phi == 3 && d.n_f == 2 && d.phi_of[0][0] == 0 && d.phi_of[0][1] == 1 &&
           d.phi_of[1][0] == 1 && d.phi_of[1][1] == 2 && d.f_of[0][0] == 0 && d.f_of[1][0] == 0 &&
           d.f_of[0][1] == 1 && d.f_of[1][1] == 1)
              ? 1
              : 0;
  d.cross_geo = (S == 2 && p.cross_geomean && !p.lj) ? 1 : 0;
  set_power_form(d);
  d.rs = p.r_switch;
  d.rc = p.r_cut;
  d.inv_w = 1.0 / (p.r_cut - p.r_switch);
  d.rs_f = (float)p.r_switch;
  d.rc_f = (float)p.r_cut;
  d.inv_w_f = (float)d.inv_w;
  d.dS_scale_f = (float)(-30.0 * d.inv_w);
  d.rs_ff = ff(d.rs);
  d.inv_w_ff = ff(d.inv_w);
  d.dS_scale_ff = ff(-30.0 * d.inv_w);
  return MXE_OK;
}

// The context keeps an unordered-pair index of its lists (and evaluates the
// pairs once) when the pair kernels support its potential.
bool has_pair_index(const mxe_ctx* c) { return pair_kernels_supported(c->dp); }

bool state_ok(const mxe_ctx* c, const mxe_state* s) {
  return s && s->n == c->n && (c->n == 0 || (s->q && s->sigma && s->x && s->T));
}

void fill_pass(mxe_ctx* c, const mxe_state* s, PassArgs& A) {
  std::memset(&A, 0, sizeof(A));
  A.q = s->q;
  A.sigma = s->sigma;
  A.x = s->x;
  A.T = s->T;
  A.pos32 = c->pos32;
  A.x32 = c->x32;
  A.pos32lo = c->pos32lo;
  A.x32lo = c->x32lo;
  A.nb_off = c->nb_off;
  A.nb_ent = c->nb_ent;
  A.n = c->n;
  A.n_ent = c->n_pairs;
  A.rho_bar = c->rho_bar;
  A.rho_avg = c->rho_avg;
  A.a = c->a;
  A.b = c->b;
  A.e = c->e;
  A.ab32 = c->ab32;
  A.ab32lo = c->ab32lo;
  A.gq = c->gq;
  A.gs = c->gs;
  A.mu_ex = c->mu_ex;
  A.mu = nullptr;
  A.site_E = c->site_E;
  A.ctrl = nullptr;
  A.flags = c->flags;
  A.check_skin = 0;
  A.batch = c->B;
  A.tpb = c->tpb;
  A.pair_tpb = c->pair_tpb;
}

mxe_status ensure_cells(mxe_ctx* c, int64_t ncell) {
  if (ncell <= c->ncell_cap) return MXE_OK;
  dfree(c->cell_count);
  dfree(c->cell_start);
  int64_t cap = ncell + ncell / 4 + 16;
  CK(dalloc(&c->cell_count, cap));
  CK(dalloc(&c->cell_start, cap + 1));
  c->ncell_cap = cap;
  if (c->nsys) {
    dfree(c->cell_sys);
    CK(dalloc(&c->cell_sys, cap));
    c->B.cell_sys = c->cell_sys;
  }
  int64_t need = std::max<int64_t>(c->n, cap) + 1;
  if (c->scan_len < scan_tmp_len(need)) {
    dfree(c->scan_tmp);
    c->scan_len = scan_tmp_len(need);
    CK(dalloc(&c->scan_tmp, c->scan_len));
  }
  return MXE_OK;
}

// Cell grid of one periodic box: cells no smaller than r_list; a sparse box
// gets coarser cells so the grid never holds more than `limit` cells.
int64_t plan_grid(const double L[3], double r_list, int64_t limit, DevGrid& g) {
  double cell_min = r_list * (1.0 + 1e-9);
  int64_t ncell = 1;
  for (int pass = 0; pass < 64; ++pass) {
    ncell = 1;
    for (int a = 0; a < 3; ++a) {
      int nc = (int)std::floor(L[a] / cell_min);
      if (nc < 3) nc = 1;
      g.nc[a] = nc;
      ncell *= nc;
    }
    if (ncell <= limit) break;
    cell_min *= 1.25;
  }
  for (int a = 0; a < 3; ++a) {
    g.L[a] = L[a];
    g.invL[a] = 1.0 / L[a];
    g.h[a] = L[a] / g.nc[a];
    g.h_f[a] = (float)g.h[a];
    g.h_lo[a] = (float)(g.h[a] - (double)g.h_f[a]);
    g.L_f[a] = (float)g.L[a];
    g.invL_f[a] = (float)g.invL[a];
  }
  return ncell;
}

mxe_status build_lists(mxe_ctx* c, const mxe_state* s, double skin, double r_bond) {
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  c->have_list = false;
  // max sigma -> r_list; max |q| -> error band of the FP32 prefilter
  CK(cudaMemsetAsync(c->smax_bits, 0, 2 * sizeof(unsigned long long), st));
  CK(TIMED("build_misc", launch_site_max(s->sigma, s->q, n, c->smax_bits, st)));
  CK(cudaMemcpyAsync(c->bits_h, c->smax_bits, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double smax, qmax;
  std::memcpy(&smax, c->bits_h, sizeof(double));
  std::memcpy(&qmax, c->bits_h + 1, sizeof(double));
  const double r_list = (c->pot.r_cut + kSqrt6 * smax) + skin;
  if (!std::isfinite(r_list)) return MXE_ERR_ARG;
  DevGrid& g = c->grid;
  double Lmax = 0.0;
  int64_t ncell = 0;
  if (c->nsys == 0) {
    for (int a = 0; a < 3; ++a) {
      if (!(c->box.L[a] >= 2.0 * r_list)) return MXE_ERR_BOX_TOO_SMALL;
      Lmax = std::max(Lmax, c->box.L[a]);
    }
    ncell = plan_grid(c->box.L, r_list, 8 * n + 4096, g);
  } else {
    // one grid per system, cells numbered system after system
    for (int b = 0; b < c->nsys; ++b) {
      for (int a = 0; a < 3; ++a) {
        if (!(c->boxes[b].L[a] >= 2.0 * r_list)) return MXE_ERR_BOX_TOO_SMALL;
        Lmax = std::max(Lmax, c->boxes[b].L[a]);
      }
      const int64_t nb = c->sys_off_h[b + 1] - c->sys_off_h[b];
      c->cell_base_h[b] = (int)ncell;
      ncell += plan_grid(c->boxes[b].L, r_list, 8 * nb + 64, c->grids_h[b]);
      if (ncell > (int64_t)1 << 30) return MXE_ERR_NBR_OVERFLOW;
    }
    c->cell_base_h[c->nsys] = (int)ncell;
    g = c->grids_h[0];  // kernels take each site's own grid from the table
  }
  // Error band of the FP32 |d|^2 (u = 2^-24): each component of d carries at
  // most delta = 6 u Qmax (rounded positions and their difference) + u Lmax
  // (rounded box length times the image count) + u r_list (last rounding),
  // doubled for a differing image choice near half a box; then
  // | |d|^2_f32 - |d|^2 | <= 2 sqrt3 r delta + 3 delta^2 + 3 u r^2, plus u r^2
  // for the rounded cutoff; the band is twice that.
  // The cell-staged kernels on grids of >= 3 cells per axis take d from
  // positions within the cell (|.| <= h) and the stencil offset times h_f:
  // per component at most 8 u h (the two rounded positions, h_f, the shifted
  // candidate, the difference) <= 8 u Lmax / 3, the second bound below.
  const double u = std::ldexp(1.0, -24);
  const double delta = std::max(2.0 * (6.0 * u * qmax + u * Lmax + u * r_list), 8.0 * u * Lmax / 3.0);
  const double band_d = 2.0 * (2.0 * std::sqrt(3.0) * r_list * delta + 3.0 * delta * delta + 4.0 * u * r_list * r_list);
  const float band = (float)(band_d * (1.0 + 1e-6));
  mxe_status ms = ensure_cells(c, ncell);
  if (ms != MXE_OK) return ms;
  if (c->nsys) {
    CK(cudaMemcpyAsync(c->grids, c->grids_h, sizeof(DevGrid) * c->nsys, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->cell_base, c->cell_base_h, sizeof(int) * (c->nsys + 1), cudaMemcpyHostToDevice, st));
    CK(TIMED("build_misc", launch_segment_ids(c->cell_base, c->nsys, ncell, c->cell_sys, st)));
  }
  const Batch& B = c->B;
  // cell lists
  CK(cudaMemsetAsync(c->cell_count, 0, sizeof(int) * ncell, st));
  CK(TIMED("build_misc", launch_cell_assign(s->q, n, g, B, c->cell_of, c->cell_slot, c->cell_count, c->abs_cell, c->qf, st)));
  CK(TIMED("build_misc", launch_scan(c->cell_count, c->cell_start, ncell, c->totals + 0, (int*)c->scan_tmp, c->scan_len, st)));
  CK(TIMED("build_misc", launch_cell_place(n, c->cell_of, c->cell_slot, c->cell_start, c->cell_sites, st)));
  // largest stencil candidate set: the cell-staged kernels hold it in shared
  // memory.  A rebuild that can skip the count pass (the previous build's
  // longest row bounds this one's) sizes it from the previous build's largest
  // stencil plus a margin and checks the true size, computed on the device
  // meanwhile, together with the totals: a larger stencil discards that fill
  // (count + fill instead).  Otherwise the host waits for the size here.
  CK(cudaMemsetAsync(c->max_row, 0, 3 * sizeof(int), st));
  CK(TIMED("build_misc", launch_cand_max(ncell, g, B, c->cell_start, c->max_row + 1, st)));
  // MXE_NEIGHBOR_PER_SITE forces the warp-per-site kernels (they are the
  // fallback for stencils too dense for shared memory; tests compare both)
  const bool per_site = std::getenv("MXE_NEIGHBOR_PER_SITE") != nullptr;
  const bool try_direct = c->max_row_h > 0 && c->max_row_h + 16 <= 256 && c->cand_cap_prev > 0 && !per_site &&
                          !std::getenv("MXE_NEIGHBOR_COUNT");
  int cand_cap;
  if (try_direct) {
    cand_cap = c->cand_cap_prev + c->cand_cap_prev / 8 + 8;
  } else {
    CK(cudaMemcpyAsync(c->ints_h + 2, c->max_row + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cand_cap = std::max(c->ints_h[2], 1);
  }
  bool staged = cell_stage_bytes(cand_cap, 256, true) <= 64 * 1024 && !per_site;
  // counts: from a fill at a fixed stride when the previous build's longest row
  // bounds it (no count pass), else a count pass before the fill
  const double rl2 = r_list * r_list, rb2 = r_bond * r_bond;
  bool direct = false;
  int stride = 0;
  if (staged && try_direct) {
    stride = (c->max_row_h + 16 + 3) & ~3;
    if ((int64_t)n * stride > c->rows_cap) {
      dfree(c->rows_tmp);
      dfree(c->brows_tmp);
      CK(dalloc(&c->rows_tmp, (int64_t)n * stride));
      CK(dalloc(&c->brows_tmp, (int64_t)n * stride));
      c->rows_cap = (int64_t)n * stride;
    }
    const bool pi = has_pair_index(c);
    // a stencil above cand_cap is cut and reported in max_row[2] (not in the
    // context's flags): the check below then discards this fill
    CK(TIMED("build_fill", launch_cell_fill_direct(s->q, c->qf, s->sublattice, s->mobile_mask, n, ncell, g, B,
                                                   c->cell_start, c->cell_sites, c->abs_cell, rl2, rb2, band, cand_cap,
                                                   stride, c->rows_tmp, c->brows_tmp, c->nb_cnt, c->bd_cnt,
                                                   pi ? c->n_below : nullptr, pi ? c->pair_cnt : nullptr,
                                                   c->max_row, c->max_row + 2, st)));
    CK(TIMED("build_misc", launch_scan(c->nb_cnt, c->nb_off, n, c->totals + 1, (int*)c->scan_tmp, c->scan_len, st)));
    CK(TIMED("build_misc", launch_scan(c->bd_cnt, c->bd_off, n, c->totals + 2, (int*)c->scan_tmp, c->scan_len, st)));
    if (pi)
      CK(TIMED("build_misc", launch_scan(c->pair_cnt, c->pair_off, n, c->totals + 3, (int*)c->scan_tmp, c->scan_len, st)));
    CK(cudaMemcpyAsync(c->totals_h, c->totals, sizeof(long long) * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->ints_h, c->max_row, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int cand_true = std::max(c->ints_h[1], 1);
    // else a row did not fit, or the stencil did not: count + fill
    direct = c->ints_h[0] <= stride && cand_true <= cand_cap;
    if (cand_true > cand_cap) {
      cand_cap = cand_true;
      staged = cell_stage_bytes(cand_cap, 256, true) <= 64 * 1024;
    }
    c->cand_cap_prev = cand_true;  // the next guess starts from the true size, not from this guess
    if (!direct) CK(cudaMemsetAsync(c->max_row, 0, sizeof(int), st));
  } else if (try_direct) {  // the guessed size did not fit shared memory: take the true one
    CK(cudaMemcpyAsync(c->ints_h + 2, c->max_row + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cand_cap = std::max(c->ints_h[2], 1);
    staged = cell_stage_bytes(cand_cap, 256, true) <= 64 * 1024;
    c->cand_cap_prev = cand_cap;
  } else {
    c->cand_cap_prev = cand_cap;  // the true size (read above)
  }
  if (direct) {
    // counts, offsets and totals are in place
  } else if (staged) {
    CK(TIMED("build_count", launch_cell_count(s->q, c->qf, s->sublattice, s->mobile_mask, n, ncell, g, B, c->cell_start,
                                              c->cell_sites, rl2, rb2, band, cand_cap, c->nb_cnt, c->bd_cnt,
                                              c->max_row, c->flags, st)));
  } else {
    CK(TIMED("build_count", launch_nbr_count(s->q, c->qf, s->sublattice, s->mobile_mask, n, g, B, c->cell_of,
                                             c->cell_start, c->cell_sites, rl2, rb2, band, c->nb_cnt, c->bd_cnt,
                                             c->max_row, st)));
  }
  if (!direct) {
    CK(TIMED("build_misc", launch_scan(c->nb_cnt, c->nb_off, n, c->totals + 1, (int*)c->scan_tmp, c->scan_len, st)));
    CK(TIMED("build_misc", launch_scan(c->bd_cnt, c->bd_off, n, c->totals + 2, (int*)c->scan_tmp, c->scan_len, st)));
    CK(cudaMemcpyAsync(c->totals_h, c->totals, sizeof(long long) * 3, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->ints_h, c->max_row, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  const long long npairs = c->totals_h[1], nbonds = c->totals_h[2];
  if (npairs > 2147483647LL || nbonds > 2147483647LL) return MXE_ERR_NBR_OVERFLOW;
  if (npairs > c->nb_cap) {
    dfree(c->nb_ent);
    int64_t cap = npairs + npairs / 8 + 64;
    CK(dalloc(&c->nb_ent, cap));
    c->nb_cap = cap;
  }
  const bool pairs = has_pair_index(c);
  if (pairs && (npairs > c->pair_cap || !c->pair_rec)) {
    dfree(c->pair_rec);
    dfree(c->pair_buf);
    const int64_t cap = std::max<int64_t>(c->nb_cap, npairs);
    CK(dalloc(&c->pair_rec, cap / 2 + 64));
    CK(dalloc(&c->pair_buf, cap * (int64_t)pair_record_len(c->dp)));  // one record per entry
    dfree(c->ent_dens);
    dfree(c->ent_frc);
    if (c->relax_records) {
      CK(dalloc_bytes(&c->ent_dens, cap * (int64_t)relax_record_bytes(c->precision)));
      CK(dalloc_bytes(&c->ent_frc, cap * (int64_t)relax_record_bytes(c->precision)));
    }
    c->pair_cap = cap;
  }
  if (nbonds > c->bd_cap) {
    dfree(c->bd_idx);
    int64_t cap = nbonds + nbonds / 8 + 64;
    CK(dalloc(&c->bd_idx, cap));
    c->bd_cap = cap;
  }
  const int max_row = c->ints_h[0];
  if ((int64_t)max_row * 5 > 200 * 1024) return MXE_ERR_NBR_OVERFLOW;
  if (direct) {
    CK(TIMED("build_misc", launch_row_compact(c->rows_tmp, c->brows_tmp, stride, n, c->nb_off, c->bd_off, c->nb_ent,
                                              c->bd_idx, st)));
  } else if (staged && max_row <= 256) {
    CK(TIMED("build_fill", launch_cell_fill(s->q, c->qf, s->sublattice, s->mobile_mask, n, ncell, g, B, c->cell_start,
                                            c->cell_sites, c->abs_cell, rl2, rb2, band, cand_cap, c->nb_off,
                                            c->nb_ent, c->bd_off, c->bd_idx, max_row, c->flags, st)));
  } else {
    CK(TIMED("build_fill", launch_nbr_fill(s->q, c->qf, s->sublattice, s->mobile_mask, n, g, B, c->cell_of,
                                           c->cell_start, c->cell_sites, c->abs_cell, rl2, rb2, band, c->nb_off,
                                           c->nb_ent, c->bd_off, c->bd_idx, max_row, st)));
  }
  if (pairs) {
    if (npairs % 2) return MXE_ERR_NBR_OVERFLOW;  // a symmetric list has every pair twice
    // every pair record is written only if the rows' tails own exactly half
    // of the entries (a symmetric list): checked before any pair kernel runs.
    // The fill without a count pass counted heads and tails already (their
    // total came with the list's); otherwise count them from the rows.
    if (!direct) {
      CK(TIMED("build_misc", launch_pair_count(c->nb_off, c->nb_ent, n, c->n_below, c->pair_cnt, st)));
      CK(TIMED("build_misc", launch_scan(c->pair_cnt, c->pair_off, n, c->totals + 3, (int*)c->scan_tmp, c->scan_len, st)));
      CK(cudaMemcpyAsync(c->totals_h + 3, c->totals + 3, sizeof(long long), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    if (c->totals_h[3] != npairs / 2) return MXE_ERR_NBR_OVERFLOW;
    CK(TIMED("build_misc", launch_pair_fill(c->nb_off, c->nb_ent, n, c->n_below, c->pair_off, npairs / 2,
                                            c->pair_rec, c->flags, st)));
    c->n_upairs = npairs / 2;
  }
  CK(copy_d2d(c->q_build, s->q, sizeof(double) * 3 * n, st));
  c->n_pairs = npairs;
  c->n_bonds = nbonds;
  c->max_row_h = max_row;
  c->r_list = r_list;
  c->skin = skin;
  c->r_bond = r_bond;
  c->sigma_max_build = smax;
  c->have_list = true;
  c->list_gen += 1;
  return MXE_OK;
}

// The force passes run on the half list: pair index and relaxation records
// present (the records are allocated by the first relaxation).
bool half_list_forces(const mxe_ctx* c) { return has_pair_index(c) && c->pair_rec && c->ent_dens && c->ent_frc; }

EmbArgs emb_args(mxe_ctx* c) {
  EmbArgs E;
  const int64_t n = c->n, S = c->S;
  E.rhob = c->emb_buf;
  E.rown = c->emb_buf + S * n;
  E.fsum = c->emb_buf + 7 * S * n;
  E.emb = c->emb_buf + 8 * S * n;
  E.nrule = c->emb_nrule;
  return E;
}

// The exact embedding average: the rule data of every site, then the
// derivatives, added to what the pair passes left in A (energies, gradients,
// chemical potentials, whichever A carries).
mxe_status enqueue_emb_exact(mxe_ctx* c, const PassArgs& A, bool fp64) {
  const EmbArgs E = emb_args(c);
  CK(TIMED(fp64 ? "emb_nodes_fp64" : "emb_nodes_fp32",
           launch_emb_exact(false, fp64, c->nl, c->dp, c->grid, A, E, c->stream)));
  if (A.gq || A.gs || A.mu_ex || A.mu)
    CK(TIMED(fp64 ? "emb_grad_fp64" : "emb_grad_fp32",
             launch_emb_exact(true, fp64, c->nl, c->dp, c->grid, A, E, c->stream)));
  return MXE_OK;
}

// Class names of the half-list kernels in the event timing.
const char* relax_pair_name(bool force, int prec) {
  if (prec == MXE_FP64) return force ? "pair64_force" : "pair64_density";
  return force ? "pair32_force" : "pair32_density";
}
const char* relax_gather_name(bool force, int prec) {
  if (prec == MXE_FP64) return force ? "gather64_force" : "gather64_density";
  if (prec == MXE_FP32_MIXED) return force ? "gather32_force_mixed" : "gather32_density_mixed";
  return force ? "gather32_force" : "gather32_density";
}
const char* accurate_gather_name(bool mu, int prec) {
  if (prec == MXE_FP64) return mu ? "mu_gather_fp64" : "density_gather_fp64";
  if (prec == MXE_FP32_MIXED) return mu ? "mu_gather_mixed" : "density_gather_mixed";
  return mu ? "mu_gather_ff" : "density_gather_ff";
}

// Free energy and gradients.  want_mu: the chemical potentials are requested.
// With a pair index, the accurate pass evaluates each unordered pair once
// (geometry records: float-float node arithmetic in the FP32 modes, FP64 in
// FP64 contexts), then gathers the densities and the chemical potentials and
// energies per site (sums in float-float for MXE_FP32_FF, FP64 otherwise):
// the flux step takes differences of neighbouring mu, so their absolute
// error must stay far below kB T * 1e-7.  Forces and the relaxation use the
// relaxation pair passes (FP32 node arithmetic in the FP32 modes).
mxe_status enqueue_passes(mxe_ctx* c, const mxe_state* s, PassArgs& A, bool want_mu) {
  cudaStream_t st = c->stream;
  const int prec = c->precision;
  const bool fp32 = prec != MXE_FP64;
  const bool hl = has_pair_index(c) && c->pair_rec;
  // with the exact embedding average the pair passes run without embedding
  const DevPot& PP = c->embedding ? c->dp_pair : c->dp;
  if (fp32)
    CK(TIMED("pack", launch_pack(s->q, s->sigma, s->x, c->abs_cell, c->n, c->S, c->grid, c->B, c->pos32, c->x32,
                   hl && want_mu ? c->pos32lo : nullptr, hl && want_mu ? c->x32lo : nullptr, st)));
  if (!hl) {  // full-list passes
    if (!fp32) {
      CK(TIMED(cls_name("density", 0), launch_density(0, c->nl, PP, c->grid, A, st)));
      CK(TIMED(cls_name("gradient", 0, want_mu ? kGradAll : kGradForce),
               launch_gradient(0, want_mu ? kGradAll : kGradForce, c->nl, PP, c->grid, A, st)));
      return c->embedding ? enqueue_emb_exact(c, A, true) : MXE_OK;
    }
    if (!want_mu) {
      CK(TIMED(cls_name("density", prec), launch_density(prec, c->nl, PP, c->grid, A, st)));
      CK(TIMED(cls_name("gradient", prec, kGradForce), launch_gradient(prec, kGradForce, c->nl, PP, c->grid, A, st)));
      return c->embedding ? enqueue_emb_exact(c, A, false) : MXE_OK;
    }
    CK(TIMED(cls_name("density", 0), launch_density(0, c->nl, PP, c->grid, A, st)));
    CK(TIMED(cls_name("gradient", 0, kGradMu), launch_gradient(0, kGradMu, c->nl, PP, c->grid, A, st)));
    CK(TIMED("pack_ab", launch_pack_ab(c->a, c->b, c->n, c->S, c->ab32, st)));
  } else {
    if (fp32 && !want_mu) {
      // forces and energies from the FP32 passes alone (energies to ~1e-6)
      CK(TIMED(cls_name("density", prec), launch_density(prec, c->nl, PP, c->grid, A, st)));
      CK(TIMED(cls_name("gradient", prec, kGradForce), launch_gradient(prec, kGradForce, c->nl, PP, c->grid, A, st)));
      return c->embedding ? enqueue_emb_exact(c, A, false) : MXE_OK;
    }
    PassArgs G = A;
    if (!fp32) {  // FP64: no packed records
      G.ab32 = nullptr;
      G.ab32lo = nullptr;
    }
    CK(TIMED(prec == MXE_FP64 ? "pair_geo64" : "pair_ff",
             launch_pair_geo(prec, PP, c->grid, G, c->pair_rec, c->n_upairs, c->pair_buf, c->pair_cap, st)));
    CK(TIMED(accurate_gather_name(false, prec),
             launch_pair_gather(prec, false, c->nl, PP, G, c->pair_buf, c->pair_cap, st)));
    CK(TIMED(accurate_gather_name(true, prec),
             launch_pair_gather(prec, true, c->nl, PP, G, c->pair_buf, c->pair_cap, st)));
  }
  if (A.gq != nullptr || A.gs != nullptr) {
    PassArgs F = A;
    F.site_E = nullptr;  // energies already come from the accurate pass
    if (half_list_forces(c)) {
      // the relaxation's force pass: each unordered pair once, then the gather
      CK(TIMED(relax_pair_name(true, prec), launch_relax_pair(prec, true, PP, c->grid, F, c->pair_rec,
                                                               c->n_upairs, c->ent_dens, c->ent_frc, st)));
      CK(TIMED(relax_gather_name(true, prec),
               launch_relax_gather(prec, true, c->nl, PP, F, c->ent_dens, c->ent_frc, st)));
    } else {
      CK(TIMED(cls_name("gradient", prec, kGradForceNoE),
               launch_gradient(prec, kGradForceNoE, c->nl, PP, c->grid, F, st)));
    }
  }
  // the accurate pass: the exact average in FP64
  return c->embedding ? enqueue_emb_exact(c, A, true) : MXE_OK;
}

mxe_fire_params fire_params_or_default(const mxe_fire_params* fire) {
  mxe_fire_params fp = {0.02, 0.1, 1.1, 0.5, 0.1, 0.99, 0.0, 5, 16};
  if (fire) fp = *fire;
  return fp;
}

// Control block at the start of a relaxation (or of a staggered run).
void init_ctrl(mxe_ctx* c, Ctrl& H, const mxe_fire_params& fp, double ftol, int max_iter) {
  std::memset(&H, 0, sizeof(Ctrl));
  H.max_iter = max_iter;
  H.dt = fp.dt0;
  H.alpha = fp.alpha0;
  H.ftol = ftol;
  H.skin = c->skin;
  H.sigma_max_build = c->sigma_max_build;
  H.dt_max = fp.dt_max;
  H.f_inc = fp.f_inc;
  H.f_dec = fp.f_dec;
  H.alpha0 = fp.alpha0;
  H.f_alpha = fp.f_alpha;
  H.n_min = fp.n_min;
  H.sigma_lo = kSigmaMin;
  H.sigma_hi = fp.sigma_max > 0.0 ? fp.sigma_max : INFINITY;
}

void relax_pass_args(mxe_ctx* c, const mxe_state* s, PassArgs& A) {
  fill_pass(c, s, A);
  A.ctrl = c->ctrl;
  A.check_skin = 1;
  A.site_E = nullptr;
  A.lean = 1;
}

// The per-entry records of the half-list relaxation passes are allocated by
// the first relaxation of a context with a pair index (outside any stream
// capture) and kept, resized with the lists, from then on.
mxe_status ensure_relax_records(mxe_ctx* c) {
  if (!has_pair_index(c) || !c->pair_rec) return MXE_OK;
  c->relax_records = true;
  if (c->ent_dens && c->ent_frc) return MXE_OK;
  dfree(c->ent_dens);
  dfree(c->ent_frc);
  const int64_t bytes = c->pair_cap * (int64_t)relax_record_bytes(c->precision);
  CK(dalloc_bytes(&c->ent_dens, bytes));
  CK(dalloc_bytes(&c->ent_frc, bytes));
  return MXE_OK;
}

// The force passes of one relaxation iteration (densities, then dF/dq and
// dF/dsigma into A.gq / A.gs): half list in float-float contexts, else the
// full-list passes.
mxe_status enqueue_force_passes(mxe_ctx* c, const PassArgs& A) {
  cudaStream_t st = c->stream;
  const DevPot& PP = c->embedding ? c->dp_pair : c->dp;
  if (half_list_forces(c)) {
    // each unordered pair once: pair kernel, then the per-site gather
    const int prec = c->precision;
    CK(TIMED(relax_pair_name(false, prec), launch_relax_pair(prec, false, PP, c->grid, A, c->pair_rec,
                                                              c->n_upairs, c->ent_dens, c->ent_frc, st)));
    CK(TIMED(relax_gather_name(false, prec),
             launch_relax_gather(prec, false, c->nl, PP, A, c->ent_dens, c->ent_frc, st)));
    CK(TIMED(relax_pair_name(true, prec), launch_relax_pair(prec, true, PP, c->grid, A, c->pair_rec,
                                                             c->n_upairs, c->ent_dens, c->ent_frc, st)));
    CK(TIMED(relax_gather_name(true, prec),
             launch_relax_gather(prec, true, c->nl, PP, A, c->ent_dens, c->ent_frc, st)));
  } else {
    CK(TIMED(cls_name("density", c->precision), launch_density(c->precision, c->nl, PP, c->grid, A, st)));
    CK(TIMED(cls_name("gradient", c->precision, kGradForceNoE), launch_gradient(c->precision, kGradForceNoE, c->nl, PP, c->grid, A, st)));
  }
  if (c->embedding) {
    PassArgs F = A;  // forces only
    F.mu_ex = nullptr;
    F.mu = nullptr;
    F.site_E = nullptr;
    return enqueue_emb_exact(c, F, c->precision == MXE_FP64);
  }
  return MXE_OK;
}

// One FIRE iteration: the force passes, then the reduction, logic and update
// (per system for a batch).
mxe_status enqueue_fire_iter(mxe_ctx* c, mxe_state* s, const PassArgs& A) {
  cudaStream_t st = c->stream;
  const int64_t n = c->n;
  mxe_status fm = enqueue_force_passes(c, A);
  if (fm != MXE_OK) return fm;
  float4* p32 = c->precision != MXE_FP64 ? c->pos32 : nullptr;
  if (c->nsys) {
    CK(TIMED("fire_reduce", launch_fire_seg_reduce(c->gq, c->gs, s->sigma, c->vq, c->vs, n, c->B, c->sf, c->ctrl, c->flags, st)));
    CK(TIMED("fire_logic", launch_fire_seg_logic(c->sf, c->nsys, c->ctrl, c->flags, st)));
    CK(TIMED("fire_update", launch_fire_seg_update(s->q, s->sigma, c->vq, c->vs, c->gq, c->gs, c->q_build, c->abs_cell, n,
                                                   c->grid, c->B, c->sf, p32, c->ctrl, st)));
  } else {
    CK(TIMED("fire_reduce", launch_fire_reduce(c->gq, c->gs, s->sigma, c->vq, c->vs, n, c->partials, c->ctrl, c->flags, st)));
    CK(TIMED("fire_update", launch_fire_update(s->q, s->sigma, c->vq, c->vs, c->gq, c->gs, c->q_build, c->abs_cell, n,
                                               c->grid, c->B, p32, c->ctrl, st)));
  }
  return MXE_OK;
}

// FIRE iterations from the current device state (control block, velocities,
// packed positions) until convergence, max_iter or an error; rebuilds the
// lists when the skin criterion fails.  H receives the final control block.
mxe_status fire_loop(mxe_ctx* c, mxe_state* s, int max_iter, int chunk, Ctrl& H) {
  cudaStream_t st = c->stream;
  PassArgs A;
  relax_pass_args(c, s, A);
  mxe_status result = MXE_OK;
  int last_iter = -1, rebuilds = 0;
  for (;;) {
    // enqueue no more iterations than can still run: max_iter updates plus the
    // final evaluation
    const int left = max_iter + 1 - H.iter;
    const int todo = std::max(1, std::min(chunk, left));
    for (int it = 0; it < todo; ++it) {
      mxe_status ms = enqueue_fire_iter(c, s, A);
      if (ms != MXE_OK) return ms;
    }
    CK(cudaMemcpyAsync(&H, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (H.reason == kReasonNone) {
      if (H.iter == last_iter) {  // no progress over a whole chunk: never expected
        result = MXE_ERR_STATE;
        break;
      }
      last_iter = H.iter;
      continue;
    }
    last_iter = H.iter;
    if (H.reason == kReasonConverged) {
      result = MXE_OK;
      break;
    }
    if (H.reason == kReasonMaxIter) {
      result = MXE_ERR_NO_CONVERGE;
      break;
    }
    if (H.reason == kReasonAllDone) {  // batches: every system converged or hit max_iter
      CK(cudaMemcpyAsync(c->sf_h, c->sf, sizeof(SysFire) * c->nsys, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      result = MXE_OK;
      for (int b = 0; b < c->nsys; ++b)
        if (c->sf_h[b].reason != kReasonConverged) result = MXE_ERR_NO_CONVERGE;
      break;
    }
    if (H.reason == kReasonError) {
      result = mxe_sync_status(c);
      if (result == MXE_OK) result = MXE_ERR_NONFINITE;
      break;
    }
    // rebuild: the skin criterion failed before the next evaluation
    if (++rebuilds > max_iter + 16) {
      result = MXE_ERR_STATE;
      break;
    }
    mxe_status ms = build_lists(c, s, c->skin, c->r_bond);
    if (ms != MXE_OK) {
      result = ms;
      break;
    }
    H.halted = 0;
    H.reason = kReasonNone;
    H.disp2_bits = 0ull;
    H.smax_bits = 0ull;
    H.sigma_max_build = c->sigma_max_build;
    CK(cudaMemcpyAsync(c->ctrl, &H, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    if (c->precision != MXE_FP64)
      CK(TIMED("pack", launch_pack(s->q, s->sigma, s->x, c->abs_cell, c->n, c->S, c->grid, c->B, c->pos32, c->x32, nullptr, nullptr, st)));
    // the rebuild may have reallocated the lists: take the current pointers
    relax_pass_args(c, s, A);
  }
  return result;
}

// Per-system outcome of the last relaxation; for a batch H.fmax becomes the
// largest fmax.
mxe_status record_relax_info(mxe_ctx* c, Ctrl& H) {
  if (c->nsys) {
    CK(cudaMemcpyAsync(c->sf_h, c->sf, sizeof(SysFire) * c->nsys, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double fm = 0.0;
    for (int b = 0; b < c->nsys; ++b) {
      c->last_iters[b] = c->sf_h[b].iter;
      c->last_fmax[b] = c->sf_h[b].fmax;
      c->last_reason[b] = c->sf_h[b].reason;
      fm = std::max(fm, c->sf_h[b].fmax);
    }
    H.fmax = fm;
  } else {
    c->last_iters[0] = H.iter;
    c->last_fmax[0] = H.fmax;
    c->last_reason[0] = H.reason;
  }
  return MXE_OK;
}

// One step of the staggered scheme (Sec. 4): excess chemical potentials, one
// Euler step of x, then max_iter + 1 FIRE evaluations (kernels after
// convergence return at once).  Every kernel obeys the control block, so the
// sequence can be captured once and replayed.
mxe_status enqueue_staggered_step(mxe_ctx* c, mxe_state* s, const StepKey& k) {
  cudaStream_t st = c->stream;
  CK(launch_step_begin(c->ctrl, k.dt0, k.alpha0, st));
  PassArgs M;
  fill_pass(c, s, M);
  M.site_E = nullptr;
  M.gq = nullptr;
  M.gs = nullptr;
  M.ctrl = c->ctrl;
  M.check_skin = 1;
  mxe_status ms = enqueue_passes(c, s, M, true);
  if (ms != MXE_OK) return ms;
  CK(cudaMemsetAsync(c->step_flags, 0, sizeof(int), st));
  CK(launch_flux_res(s->x, s->T, c->mu_ex, c->bd_off, c->bd_idx, c->n, c->S, k.dt, k.nu0, k.Qm, c->flux_tmp,
                     c->x_new, c->step_flags, c->fix_x_mask, c->fix_x_value, c->fix_mu_mask, c->fix_mu_value,
                     c->mu_eff, c->nsys ? c->dt_sys : nullptr, c->nsys ? c->sys_of : nullptr, c->ctrl, st));
  CK(launch_commit_x(s->x, c->x_new, (int64_t)c->S * c->n, c->step_flags, c->flags, c->ctrl, st));
  if (c->precision != MXE_FP64)
    CK(launch_pack(s->q, s->sigma, s->x, c->abs_cell, c->n, c->S, c->grid, c->B, c->pos32, c->x32, nullptr, nullptr, st));
  CK(launch_fire_zero_v(c->vq, c->vs, c->n, c->ctrl, st));
  if (c->nsys) CK(launch_fire_seg_init(c->sf, c->nsys, k.dt0, k.alpha0, c->ctrl, st));
  PassArgs A;
  relax_pass_args(c, s, A);
  for (int it = 0; it <= k.max_iter; ++it) {
    ms = enqueue_fire_iter(c, s, A);
    if (ms != MXE_OK) return ms;
  }
  CK(launch_step_end(c->ctrl, st));
  return MXE_OK;
}

// The staggered run as one graph: a while node whose body is one captured
// staggered step followed by the loop-control kernel, so a launch runs the
// steps on the device until the requested count is reached, a step stops for
// a list rebuild or an error, or the body count hits its cap.  The step is
// captured on a private stream (the caller's stream may be the legacy
// default stream, which cannot be captured); the graph is kept while the key
// (state pointers, step parameters, list generation, pass shape) is
// unchanged.
mxe_status ensure_step_graph(mxe_ctx* c, mxe_state* s, StepKey key) {
  key.list_gen = c->list_gen;
  if (c->step_exec && same_key(key, c->step_key)) return MXE_OK;
  if (c->step_exec) {
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!c->loop_dev) {
    CK(dalloc(&c->loop_dev, 3));
    CK(cudaMallocHost((void**)&c->loop_h, 3 * sizeof(int)));
  }
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  }
  mxe_status ms = MXE_OK;
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t user = c->stream;
    const bool timing = c->timing;
    c->stream = c->cap_stream;
    c->timing = false;
    e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      ms = enqueue_staggered_step(c, s, key);
      if (ms == MXE_OK) e = launch_loop_cond(h, c->ctrl, c->loop_dev, c->cap_stream);
      cudaGraph_t out = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &out);
      if (e == cudaSuccess) e = e2;
      // kernel nodes of one step (the loop-control kernel included)
      size_t nn = 0;
      if (e == cudaSuccess && cudaGraphGetNodes(body, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        int k = 0;
        if (cudaGraphGetNodes(body, nodes.data(), &nn) == cudaSuccess)
          for (size_t u = 0; u < nn; ++u) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[u], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
          }
        c->step_kernels = k;
      }
    }
    c->stream = user;
    c->timing = timing;
  }
  if (e == cudaSuccess && ms == MXE_OK) e = cudaGraphInstantiate(&c->step_exec, g, 0);
  cudaGraphDestroy(g);
  if (ms != MXE_OK) return ms;
  if (e != cudaSuccess) {
    c->step_exec = nullptr;
    return map_cuda(e);
  }
  c->step_key = key;
  return MXE_OK;
}

// Work timed by the autotuner: the chemical-potential passes and two FIRE
// force evaluations, as in one staggered step.
mxe_status enqueue_tune_work(mxe_ctx* c, const mxe_state* s) {
  PassArgs M;
  fill_pass(c, s, M);
  M.site_E = nullptr;
  M.gq = nullptr;
  M.gs = nullptr;
  mxe_status ms = enqueue_passes(c, s, M, true);
  if (ms != MXE_OK) return ms;
  PassArgs A;
  fill_pass(c, s, A);
  A.site_E = nullptr;
  A.lean = 1;
  if (c->precision != MXE_FP64) CK(launch_pack(s->q, s->sigma, s->x, c->abs_cell, c->n, c->S, c->grid, c->B, c->pos32, c->x32, nullptr, nullptr, c->stream));
  for (int r = 0; r < 2; ++r) {
    ms = enqueue_force_passes(c, A);
    if (ms != MXE_OK) return ms;
  }
  return MXE_OK;
}

// ---------------------------------------------------------------- second order
int n_terms(const mxe_ctx* c) { return c->dp.n_phi + c->dp.n_f; }

mxe_status ensure_tangent(mxe_ctx* c) {
  if (c->tan_buf) return MXE_OK;
  const int64_t n = c->n, S = c->S, T = n_terms(c);
  CK(dalloc(&c->tan_buf, 6 * S * n));
  CK(dalloc(&c->th_buf, 2 * 2 * T * n));
  CK(dalloc(&c->th_sum, 4 * T));
  CK(dalloc(&c->dot_part, dot_partials_len(4 * n + 1)));
  CK(dalloc(&c->dot_out, 2));
  CK(cudaMallocHost((void**)&c->dot_h, 2 * sizeof(double)));
  return MXE_OK;
}

// One forward-mode pass: values and tangents of dF/dq, dF/dsigma, mu^ex and
// (when th_out) the summed term sensitivities [values 2T | tangents 2T].
mxe_status enqueue_tangent(mxe_ctx* c, const mxe_state* s, const double* dq, const double* dsig, const double* dx,
                           double* gq_v, double* gs_v, double* mu_v, double* gq_t, double* gs_t, double* mu_t,
                           double* th_out) {
  const int64_t n = c->n, S = c->S, T = n_terms(c);
  TanArgs A;
  std::memset(&A, 0, sizeof(A));
  A.q = s->q;
  A.sigma = s->sigma;
  A.x = s->x;
  A.T = s->T;
  A.dq = dq;
  A.dsigma = dsig;
  A.dx = dx;
  A.nb_off = c->nb_off;
  A.nb_ent = c->nb_ent;
  A.n = n;
  double* b = c->tan_buf;
  A.a_v = b;
  A.a_t = b + S * n;
  A.b_v = b + 2 * S * n;
  A.b_t = b + 3 * S * n;
  A.e_v = b + 4 * S * n;
  A.e_t = b + 5 * S * n;
  A.gq_v = gq_v;
  A.gs_v = gs_v;
  A.mu_v = mu_v;
  A.gq_t = gq_t;
  A.gs_t = gs_t;
  A.mu_t = mu_t;
  if (th_out) {
    A.th_v = c->th_buf;
    A.th_t = c->th_buf + 2 * T * n;
  }
  A.flags = c->flags;
  A.batch = c->B;
  CK(TIMED("tangent", launch_tangent(c->dp, c->grid, A, c->stream)));
  if (th_out && T > 0) {
    CK(launch_col_sum(A.th_v, (int)(2 * T), n, th_out, c->stream));
    CK(launch_col_sum(A.th_t, (int)(2 * T), n, th_out + 2 * T, c->stream));
  }
  return MXE_OK;
}

// <a, b> over len doubles, returned on the host (syncs)
mxe_status dot_host(mxe_ctx* c, const double* a, const double* b, int64_t len, double& out) {
  CK(launch_dot(a, b, len, c->dot_part, c->dot_out, c->stream));
  CK(cudaMemcpyAsync(c->dot_h, c->dot_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out = c->dot_h[0];
  return MXE_OK;
}

// Conjugate gradients on H lam = rhs, H the Hessian of F in y = (q [3n],
// sigma [n]) at fixed x, applied by the forward-mode pass.  lam, r, p, Hp:
// 4n device vectors.  Stops at |r| <= tol |rhs| or max_it iterations.
mxe_status cg_solve(mxe_ctx* c, const mxe_state* s, const double* rhs, double* lam, double* r, double* p,
                    double* Hp, double tol, int max_it, int& iters, double& rel) {
  const int64_t n = c->n, m = 4 * n;
  cudaStream_t st = c->stream;
  iters = 0;
  rel = 0.0;
  if (m > 0) CK(cudaMemsetAsync(lam, 0, sizeof(double) * m, st));
  CK(copy_d2d(r, rhs, sizeof(double) * m, st));
  CK(copy_d2d(p, rhs, sizeof(double) * m, st));
  double rr = 0.0;
  mxe_status ms = dot_host(c, r, r, m, rr);
  if (ms != MXE_OK) return ms;
  const double rr0 = rr;
  if (!(rr0 > 0.0)) return MXE_OK;
  while (iters < max_it) {
    ms = enqueue_tangent(c, s, p, p + 3 * n, nullptr, nullptr, nullptr, nullptr, Hp, Hp + 3 * n, nullptr, nullptr);
    if (ms != MXE_OK) return ms;
    double pHp = 0.0;
    ms = dot_host(c, p, Hp, m, pHp);
    if (ms != MXE_OK) return ms;
    if (!(pHp > 0.0)) return MXE_ERR_NONFINITE;  // not a minimum: no implicit function
    const double alpha = rr / pHp;
    CK(launch_axpby(lam, p, alpha, 1.0, m, st));
    CK(launch_axpby(r, Hp, -alpha, 1.0, m, st));
    double rr1 = 0.0;
    ms = dot_host(c, r, r, m, rr1);
    if (ms != MXE_OK) return ms;
    ++iters;
    rel = std::sqrt(rr1 / rr0);
    if (!std::isfinite(rel)) return MXE_ERR_NONFINITE;
    if (rel <= tol) break;
    CK(launch_axpby(p, r, 1.0, rr1 / rr, m, st));  // p = r + beta p
    rr = rr1;
  }
  return MXE_OK;
}

}  // namespace

extern "C" {

const char* mxe_status_string(mxe_status s) {
  switch (s) {
    case MXE_OK: return "ok";
    case MXE_ERR_ARG: return "invalid argument";
    case MXE_ERR_CUDA: return "CUDA runtime error";
    case MXE_ERR_OOM: return "device out of memory";
    case MXE_ERR_BOX_TOO_SMALL: return "box length below 2 r_list";
    case MXE_ERR_NBR_OVERFLOW: return "neighbour list too large";
    case MXE_ERR_GEOMETRY: return "quadrature node closer than 0.5 A or static density <= 1e-12";
    case MXE_ERR_NONFINITE: return "non-finite free energy or gradient";
    case MXE_ERR_X_RANGE: return "Euler step leaves molar fractions outside [0, 1]";
    case MXE_ERR_NO_CONVERGE: return "relaxation reached max_iter";
    case MXE_ERR_STATE: return "call order violated (no neighbour list)";
  }
  return "unknown status";
}

mxe_status mxe_create(mxe_ctx** out, const mxe_box* box, const mxe_potential* pot, int64_t n,
                      mxe_precision precision, void* cuda_stream) {
  return mxe_create_batch(out, 0, box, nullptr, pot, n, precision, cuda_stream);
}

mxe_status mxe_create_batch(mxe_ctx** out, int32_t n_systems, const mxe_box* boxes, const int64_t* offsets,
                            const mxe_potential* pot, int64_t n, mxe_precision precision, void* cuda_stream) {
  if (!out) return MXE_ERR_ARG;
  *out = nullptr;
  if (n_systems < 0 || n_systems > kMaxSystems || !boxes) return MXE_ERR_ARG;
  if (n_systems > 0) {
    if (!offsets || offsets[0] != 0 || offsets[n_systems] != n) return MXE_ERR_ARG;
    for (int b = 0; b < n_systems; ++b) {
      if (offsets[b + 1] < offsets[b]) return MXE_ERR_ARG;
      for (int a = 0; a < 3; ++a)
        if (!(boxes[b].L[a] > 0.0) || !std::isfinite(boxes[b].L[a])) return MXE_ERR_ARG;
    }
  }
  const mxe_box* box = boxes;
  *out = nullptr;
  if (!box || !pot || n < 0 || n >= (int64_t)kIdxMask) return MXE_ERR_ARG;
  if (precision != MXE_FP64 && precision != MXE_FP32_MIXED && precision != MXE_FP32_FF) return MXE_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!(box->L[a] > 0.0) || !std::isfinite(box->L[a])) return MXE_ERR_ARG;
  mxe_ctx* c = new (std::nothrow) mxe_ctx();
  if (!c) return MXE_ERR_OOM;
  mxe_status ms = make_devpot(*pot, c->dp);
  if (ms == MXE_OK && c->dp.lj && precision != MXE_FP64) ms = MXE_ERR_ARG;  // FP64 passes only
  if (ms == MXE_OK) {
    c->dp_pair = c->dp;
    for (int k = 0; k < kMaxS; ++k) c->dp_pair.E[k] = 0.0;
  }
  if (ms != MXE_OK) {
    delete c;
    return ms;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return MXE_ERR_CUDA;
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->n = n;
  c->S = pot->n_species;
  c->precision = precision;
  c->box = *box;
  c->pot = *pot;
  if (const char* env = std::getenv("MXE_LANES_PER_SITE")) {
    int v = std::atoi(env);
    if (v == 4 || v == 8 || v == 16) c->nl = v;
  }
  const int64_t S = c->S;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(dalloc(&c->cell_of, n));
  A(dalloc(&c->cell_slot, n));
  A(dalloc(&c->abs_cell, 3 * n));
  A(dalloc(&c->cell_sites, n));
  A(dalloc(&c->nb_cnt, n));
  A(dalloc(&c->bd_cnt, n));
  A(dalloc(&c->nb_off, n + 1));
  A(dalloc(&c->bd_off, n + 1));
  A(dalloc(&c->totals, 4));
  A(dalloc(&c->max_row, 4));  // longest row, largest stencil, flags of a fill that may be discarded
  A(dalloc(&c->smax_bits, 2));
  A(dalloc(&c->qf, 2 * n));
  A(dalloc(&c->q_build, 3 * n));
  A(dalloc(&c->rho_bar, S * n));
  A(dalloc(&c->rho_avg, S * n));
  A(dalloc(&c->a, S * n));
  A(dalloc(&c->b, S * n));
  A(dalloc(&c->e, S * n));
  if (precision != MXE_FP64) {
    A(dalloc(&c->pos32, n));
    A(dalloc(&c->x32, n));
    A(dalloc(&c->ab32, 2 * n));
  }
  if (has_pair_index(c)) {
    A(dalloc(&c->n_below, n));
    A(dalloc(&c->pair_cnt, n));
    A(dalloc(&c->pair_off, n + 1));
    if (precision != MXE_FP64) {
      A(dalloc(&c->pos32lo, n));
      A(dalloc(&c->x32lo, n));
      A(dalloc(&c->ab32lo, 2 * n));
    }
  }
  A(init_ff_exp_table());
  A(dalloc(&c->gq, 3 * n));
  A(dalloc(&c->gs, n));
  A(dalloc(&c->mu_ex, S * n));
  A(dalloc(&c->site_E, 3 * n));
  A(dalloc(&c->partials, 3 * ((n + kFireGroup - 1) / kFireGroup + 1)));  // FIRE and energy partial sums (kFireGroup <= kReduceGroup)
  A(dalloc(&c->F4_tmp, 4));
  A(dalloc(&c->vq, 3 * n));
  A(dalloc(&c->vs, n));
  A(dalloc(&c->q0, 3 * n));
  A(dalloc(&c->s0, n));
  A(dalloc(&c->x_new, S * n));
  A(dalloc(&c->flux_tmp, flux_scratch_len(n, (int)S)));
  A(dalloc(&c->mu_eff, S * n));
  A(dalloc(&c->flags, 1));
  A(dalloc(&c->step_flags, 1));
  A(dalloc(&c->ctrl, 1));
  A(cudaMallocHost((void**)&c->ctrl_h, sizeof(Ctrl)));
  A(cudaMallocHost((void**)&c->totals_h, sizeof(long long) * 4));
  A(cudaMallocHost((void**)&c->ints_h, sizeof(int) * 4));
  A(cudaMallocHost((void**)&c->bits_h, sizeof(unsigned long long) * 2));
  const int nsys = n_systems;
  c->last_iters.assign(std::max(nsys, 1), 0);
  c->last_fmax.assign(std::max(nsys, 1), 0.0);
  c->last_reason.assign(std::max(nsys, 1), 0);
  if (nsys > 0) {
    c->nsys = nsys;
    c->boxes.assign(boxes, boxes + nsys);
    c->sys_off_h.assign(offsets, offsets + nsys + 1);
    A(dalloc(&c->sys_of, n));
    A(dalloc(&c->sys_off, nsys + 1));
    A(dalloc(&c->grids, nsys));
    A(dalloc(&c->cell_base, nsys + 1));
    A(dalloc(&c->sf, nsys));
    A(dalloc(&c->dt_sys, nsys));
    A(cudaMallocHost((void**)&c->grids_h, sizeof(DevGrid) * nsys));
    A(cudaMallocHost((void**)&c->cell_base_h, sizeof(int) * (nsys + 1)));
    A(cudaMallocHost((void**)&c->sf_h, sizeof(SysFire) * nsys));
    if (e == cudaSuccess) {
      std::vector<int> off32(offsets, offsets + nsys + 1);
      std::vector<double> ones(nsys, 1.0);
      e = cudaMemcpy(c->sys_off, off32.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c->dt_sys, ones.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = launch_segment_ids(c->sys_off, nsys, n, c->sys_of, c->stream);
    }
    c->B.nsys = nsys;
    c->B.sys_of = c->sys_of;
    c->B.grids = c->grids;
    c->B.cell_base = c->cell_base;
    c->B.cell_sys = nullptr;  // set with the cell arrays
    c->B.sys_off = c->sys_off;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    mxe_destroy(c);
    return map_cuda(e);
  }
  *out = c;
  return MXE_OK;
}

mxe_status mxe_destroy(mxe_ctx* c) {
  if (!c) return MXE_OK;
  Guard gd(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& t : c->timed) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  dfree(c->loop_dev);
  if (c->loop_h) cudaFreeHost(c->loop_h);
  dfree(c->tan_buf);
  dfree(c->emb_buf);
  dfree(c->emb_nrule);
  dfree(c->n_below);
  dfree(c->pair_cnt);
  dfree(c->pair_off);
  dfree(c->pair_rec);
  dfree(c->pair_buf);
  dfree(c->rows_tmp);
  dfree(c->brows_tmp);
  dfree(c->ent_dens);
  dfree(c->ent_frc);
  dfree(c->v_new);
  dfree(c->th_buf);
  dfree(c->th_sum);
  dfree(c->dot_part);
  dfree(c->dot_out);
  if (c->dot_h) cudaFreeHost(c->dot_h);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  dfree(c->cell_of);
  dfree(c->cell_slot);
  dfree(c->abs_cell);
  dfree(c->cell_count);
  dfree(c->cell_start);
  dfree(c->cell_sites);
  dfree(c->nb_cnt);
  dfree(c->bd_cnt);
  dfree(c->nb_off);
  dfree(c->bd_off);
  dfree(c->nb_ent);
  dfree(c->bd_idx);
  dfree(c->scan_tmp);
  dfree(c->totals);
  dfree(c->max_row);
  dfree(c->smax_bits);
  dfree(c->qf);
  dfree(c->q_build);
  dfree(c->rho_bar);
  dfree(c->rho_avg);
  dfree(c->a);
  dfree(c->b);
  dfree(c->e);
  dfree(c->pos32);
  dfree(c->x32);
  dfree(c->ab32);
  dfree(c->pos32lo);
  dfree(c->x32lo);
  dfree(c->ab32lo);
  dfree(c->gq);
  dfree(c->gs);
  dfree(c->mu_ex);
  dfree(c->site_E);
  dfree(c->partials);
  dfree(c->F4_tmp);
  dfree(c->vq);
  dfree(c->vs);
  dfree(c->q0);
  dfree(c->s0);
  dfree(c->x_new);
  dfree(c->flux_tmp);
  dfree(c->mu_eff);
  dfree(c->flags);
  dfree(c->step_flags);
  dfree(c->ctrl);
  dfree(c->sys_of);
  dfree(c->sys_off);
  dfree(c->grids);
  dfree(c->cell_base);
  dfree(c->cell_sys);
  dfree(c->sf);
  dfree(c->dt_sys);
  if (c->grids_h) cudaFreeHost(c->grids_h);
  if (c->cell_base_h) cudaFreeHost(c->cell_base_h);
  if (c->sf_h) cudaFreeHost(c->sf_h);
  if (c->ctrl_h) cudaFreeHost(c->ctrl_h);
  if (c->totals_h) cudaFreeHost(c->totals_h);
  if (c->ints_h) cudaFreeHost(c->ints_h);
  if (c->bits_h) cudaFreeHost(c->bits_h);
  delete c;
  return MXE_OK;
}

mxe_status mxe_build_neighbors(mxe_ctx* c, const mxe_state* s, double skin, double r_bond, int64_t* n_pairs_out,
                               double* r_list_out) {
  if (!c || !state_ok(c, s) || !(skin >= 0.0) || !(r_bond >= 0.0)) return MXE_ERR_ARG;
  Guard gd(c->device);
  mxe_status ms = build_lists(c, s, skin, r_bond);
  if (ms != MXE_OK) return ms;
  if (n_pairs_out) *n_pairs_out = c->n_pairs;
  if (r_list_out) *r_list_out = c->r_list;
  return MXE_OK;
}

mxe_status mxe_export_neighbors(mxe_ctx* c, int32_t* offsets_dev, int32_t* idx_dev) {
  if (!c) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  if (offsets_dev) CK(copy_d2d(offsets_dev, c->nb_off, sizeof(int32_t) * (c->n + 1), c->stream));
  if (idx_dev) CK(launch_strip_codes(c->nb_ent, idx_dev, c->n_pairs, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MXE_OK;
}

mxe_status mxe_export_bonds(mxe_ctx* c, int32_t* offsets_dev, int32_t* idx_dev, int64_t* n_bonds_out) {
  if (!c) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  if (offsets_dev) CK(copy_d2d(offsets_dev, c->bd_off, sizeof(int32_t) * (c->n + 1), c->stream));
  if (idx_dev) CK(copy_d2d(idx_dev, c->bd_idx, sizeof(int32_t) * c->n_bonds, c->stream));
  if (n_bonds_out) *n_bonds_out = c->n_bonds;
  CK(cudaStreamSynchronize(c->stream));
  return MXE_OK;
}

mxe_status mxe_set_reservoirs(mxe_ctx* c, const uint8_t* fix_x_mask_dev, const double* fix_x_value_dev,
                              const uint8_t* fix_mu_mask_dev, const double* fix_mu_value_dev) {
  if (!c) return MXE_ERR_ARG;
  if ((fix_x_mask_dev == nullptr) != (fix_x_value_dev == nullptr)) return MXE_ERR_ARG;
  if ((fix_mu_mask_dev == nullptr) != (fix_mu_value_dev == nullptr)) return MXE_ERR_ARG;
  c->fix_x_mask = fix_x_mask_dev;
  c->fix_x_value = fix_x_value_dev;
  c->fix_mu_mask = fix_mu_mask_dev;
  c->fix_mu_value = fix_mu_value_dev;
  return MXE_OK;
}

mxe_status mxe_set_dt_scale(mxe_ctx* c, const double* scale) {
  if (!c || c->nsys == 0) return MXE_ERR_ARG;
  std::vector<double> v(c->nsys, 1.0);
  if (scale) {
    for (int b = 0; b < c->nsys; ++b) {
      if (!(scale[b] >= 0.0) || !std::isfinite(scale[b])) return MXE_ERR_ARG;
      v[b] = scale[b];
    }
  }
  Guard gd(c->device);
  CK(cudaMemcpyAsync(c->dt_sys, v.data(), sizeof(double) * c->nsys, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MXE_OK;
}

mxe_status mxe_relax_info(mxe_ctx* c, int32_t n_entries, int32_t* iters, double* fmax, int32_t* converged) {
  if (!c) return MXE_ERR_ARG;
  const int m = std::max(c->nsys, 1);
  if (n_entries != m) return MXE_ERR_ARG;
  for (int b = 0; b < m; ++b) {
    if (iters) iters[b] = c->last_iters[b];
    if (fmax) fmax[b] = c->last_fmax[b];
    if (converged) converged[b] = c->last_reason[b] == kReasonConverged ? 1 : 0;
  }
  return MXE_OK;
}

mxe_status mxe_potential_terms(mxe_ctx* c, int32_t* n_phi, int32_t* n_f, double* terms, int32_t* phi_of,
                               int32_t* f_of) {
  if (!c) return MXE_ERR_ARG;
  const DevPot& P = c->dp;
  if (n_phi) *n_phi = P.n_phi;
  if (n_f) *n_f = P.n_f;
  if (terms) {
    int k = 0;
    for (int u = 0; u < P.n_phi; ++u, ++k) {
      terms[3 * k] = P.phi[u].A;
      terms[3 * k + 1] = P.phi[u].kappa;
      terms[3 * k + 2] = P.phi[u].lambda;
    }
    for (int v = 0; v < P.n_f; ++v, ++k) {
      terms[3 * k] = P.f[v].A;
      terms[3 * k + 1] = P.f[v].kappa;
      terms[3 * k + 2] = P.f[v].lambda;
    }
  }
  for (int k = 0; k < MXE_MAXS; ++k)
    for (int l = 0; l < MXE_MAXS; ++l) {
      const bool in = k < P.S && l < P.S;
      if (phi_of) phi_of[k * MXE_MAXS + l] = in ? P.phi_of[k][l] : -1;
      if (f_of) f_of[k * MXE_MAXS + l] = in && P.f_of[k][l] >= 0 ? P.n_phi + P.f_of[k][l] : -1;
    }
  return MXE_OK;
}

mxe_status mxe_element_param_grad(const mxe_potential* pot, const double* dterm, double* out) {
  if (!pot || !dterm || !out) return MXE_ERR_ARG;
  DevPot d;
  mxe_status ms = make_devpot(*pot, d);
  if (ms != MXE_OK) return ms;
  const mxe_potential& p = *pot;
  const int S = p.n_species, T = d.n_phi + d.n_f;
  if (p.lj || (S > 1 && !p.cross_geomean)) return MXE_ERR_ARG;
  // the element structure: the density from an l-neighbour is l's own term,
  // whose length scale is l's pair length scale
  for (int k = 0; k < S; ++k)
    for (int l = 0; l < S; ++l)
      if (p.f_xi[k][l] != p.f_xi[l][l] || p.f_q[k][l] != p.f_q[l][l] || p.f_r0[k][l] != p.f_r0[l][l] ||
          p.f_r0[l][l] != p.phi_r0[l][l])
        return MXE_ERR_ARG;
  for (int e = 0; e < 4 * S; ++e) out[e] = 0.0;
  std::vector<char> seen(T, 0);
  // dL/dtheta_e = sum over terms u of dL/dc_u dc_u/dtheta_e + dL/dlambda_u dlambda_u/dtheta_e
  auto add = [&](int e, double dc_dA, double dc_dp, double dc_dq, double dl_dp, double dl_dq, double dl_dr0, int u) {
    const double gc = dterm[u], gl = dterm[T + u];
    out[4 * e + 0] += gc * dc_dA;
    out[4 * e + 1] += gc * dc_dp + gl * dl_dp;
    out[4 * e + 2] += gc * dc_dq + gl * dl_dq;
    out[4 * e + 3] += gl * dl_dr0;
  };
  for (int k = 0; k < S; ++k)
    for (int l = k; l < S; ++l) {
      const int u = d.phi_of[k][l];
      if (u < 0 || seen[u]) continue;
      seen[u] = 1;
      // c = ln A_e + p_e, lambda = p_e / r0_e; the geometric-mean cross pair
      // averages the two elements' c and lambda
      const double wgt = (k == l) ? 1.0 : 0.5;
      const int els[2] = {k, l};
      for (int t = 0; t < (k == l ? 1 : 2); ++t) {
        const int e = els[t];
        const double A = p.phi_A[e][e], pe = p.phi_p[e][e], r0 = p.phi_r0[e][e];
        add(e, wgt / A, wgt, 0.0, wgt / r0, 0.0, -wgt * pe / (r0 * r0), u);
      }
    }
  for (int k = 0; k < S; ++k)
    for (int l = 0; l < S; ++l) {
      const int v = d.f_of[k][l];
      if (v < 0 || seen[d.n_phi + v]) continue;
      seen[d.n_phi + v] = 1;
      // c = ln xi_l + q_l, lambda = q_l / r0_l
      const double q = p.f_q[l][l], r0 = p.phi_r0[l][l];
      add(l, 0.0, 0.0, 1.0, 0.0, 1.0 / r0, -q / (r0 * r0), d.n_phi + v);
    }
  return MXE_OK;
}

mxe_status mxe_tangent(mxe_ctx* c, const mxe_state* s, const double* dq_dev, const double* dsigma_dev,
                       const double* dx_dev, double* dFdq_dev, double* dFdsigma_dev, double* mu_ex_dev,
                       double* dFdq_t_dev, double* dFdsigma_t_dev, double* mu_ex_t_dev, double* dterm_dev) {
  if (!c || !state_ok(c, s) || c->dp.lj || c->embedding) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  mxe_status ms = ensure_tangent(c);
  if (ms != MXE_OK) return ms;
  ms = enqueue_tangent(c, s, dq_dev, dsigma_dev, dx_dev, dFdq_dev, dFdsigma_dev, mu_ex_dev, dFdq_t_dev,
                       dFdsigma_t_dev, mu_ex_t_dev, dterm_dev);
  if (ms != MXE_OK) return ms;
  return mxe_sync_status(c);
}

mxe_status mxe_flux_vjp(mxe_ctx* c, const mxe_state* s, const double* mu_ex_dev, double dt, double nu0, double Qm,
                        const double* xbar_next_dev, double* xbar_dev, double* mubar_dev) {
  if (!c || !state_ok(c, s) || !mu_ex_dev || !xbar_next_dev || !xbar_dev || !mubar_dev) return MXE_ERR_ARG;
  if (!(dt >= 0.0) || !(nu0 >= 0.0) || !std::isfinite(Qm)) return MXE_ERR_ARG;
  if (c->fix_x_mask || c->fix_mu_mask) return MXE_ERR_ARG;  // reservoir groups are not differentiated
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  CK(launch_flux_vjp(s->x, s->T, mu_ex_dev, c->bd_off, c->bd_idx, c->n, c->S, dt, nu0, Qm,
                     c->nsys ? c->dt_sys : nullptr, c->nsys ? c->sys_of : nullptr, xbar_next_dev, xbar_dev,
                     mubar_dev, c->stream));
  return mxe_sync_status(c);
}

// The forward sweep and each checkpoint segment's recomputed relaxations are
// shared by the n_obj objectives; the reverse steps (Euler-step VJP, CG on
// H_yy, tangent pass) run per objective.
mxe_status unrolled_grad_impl(mxe_ctx* c, mxe_state* s, int32_t n_steps, double dt, double nu0, double Qm,
                              double ftol, int32_t max_iter, const mxe_fire_params* fire, int32_t every, int32_t n_obj,
                              const double* w_dev, double cg_tol, int32_t cg_max, double* dterm_host,
                              double* dx0_dev, mxe_grad_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (n_obj < 1 || n_obj > 4096) return MXE_ERR_ARG;
  if (!c || !state_ok(c, s) || n_steps < 0 || every < 1 || !w_dev || !dterm_host || !(cg_tol > 0.0) ||
      cg_max < 1 || !(dt >= 0.0) || !(nu0 >= 0.0) || !std::isfinite(Qm) || !(ftol >= 0.0) || max_iter < 0)
    return MXE_ERR_ARG;
  if (c->precision != MXE_FP64 || c->fix_x_mask || c->fix_mu_mask || c->dp.lj || c->embedding) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  mxe_status ms = ensure_tangent(c);
  if (ms != MXE_OK) return ms;
  const int64_t n = c->n, S = c->S, T = n_terms(c), ny = 4 * n, nx = S * n;
  const int nck = n_steps / every + 1;
  cudaStream_t st = c->stream;
  // work arrays (freed on return)
  std::vector<double*> owned;
  auto alloc = [&](int64_t len) -> double* {
    double* p = nullptr;
    if (dalloc(&p, len) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  };
  struct Free {
    std::vector<double*>& v;
    ~Free() {
      for (double* p : v) cudaFree(p);
    }
  } fr{owned};
  double* X = alloc((int64_t)(n_steps + 1) * nx);    // x_t, every step
  double* Y = alloc((int64_t)nck * ny);              // (q, sigma) every `every` steps
  double* seg = alloc((int64_t)every * ny);          // (q, sigma) recomputed inside a segment
  double* yT = alloc(ny);                            // final state
  double* mu = alloc(nx);
  double* xbar = alloc((int64_t)n_obj * nx);  // one cotangent of x per objective
  double* xdir = alloc(nx);
  double* mubar = alloc(nx);
  double* rhs = alloc(ny);
  double* lam = alloc(ny);
  double* r = alloc(ny);
  double* p = alloc(ny);
  double* Hp = alloc(ny);
  double* th = alloc(4 * T);
  double* mut = alloc(nx);
  if (!X || !Y || !seg || !yT || !mu || !xbar || !xdir || !mubar || !rhs || !lam || !r || !p || !Hp || !th || !mut)
    return MXE_ERR_OOM;
  auto save_y = [&](double* dst) -> mxe_status {
    CK(copy_d2d(dst, s->q, sizeof(double) * 3 * n, st));
    CK(copy_d2d(dst + 3 * n, s->sigma, sizeof(double) * n, st));
    return MXE_OK;
  };
  auto load_y = [&](const double* src) -> mxe_status {
    CK(copy_d2d(s->q, src, sizeof(double) * 3 * n, st));
    CK(copy_d2d(s->sigma, src + 3 * n, sizeof(double) * n, st));
    return MXE_OK;
  };
  auto relax = [&]() -> mxe_status {
    int32_t it = 0;
    double fm = 0.0;
    mxe_status r2 = mxe_relax(c, s, ftol, max_iter, fire, &it, &fm);
    if (info) info->relax_iters_total += it;
    return r2;
  };
  auto mu_pass = [&]() -> mxe_status {  // mu^ex at the current state into `mu`
    PassArgs A;
    fill_pass(c, s, A);
    A.site_E = nullptr;
    A.gq = nullptr;
    A.gs = nullptr;
    A.mu_ex = mu;
    mxe_status r2 = enqueue_passes(c, s, A, true);
    if (r2 != MXE_OK) return r2;
    return mxe_sync_status(c);
  };
#define RUN(expr)                      \
  do {                                 \
    mxe_status _m = (expr);            \
    if (_m != MXE_OK) return _m;       \
  } while (0)
  // ---- forward: y_0 = relax(x_0); per step mu, Euler, relax
  RUN(relax());
  CK(copy_d2d(X, s->x, sizeof(double) * nx, st));
  RUN(save_y(Y));
  for (int t = 0; t < n_steps; ++t) {
    RUN(mu_pass());
    RUN(mxe_diffuse_step(c, s, mu, dt, nu0, Qm));
    RUN(relax());
    CK(copy_d2d(X + (int64_t)(t + 1) * nx, s->x, sizeof(double) * nx, st));
    if ((t + 1) % every == 0) RUN(save_y(Y + (int64_t)((t + 1) / every) * ny));
  }
  RUN(save_y(yT));
  // ---- reverse sweep
  std::vector<double> acc((size_t)n_obj * 2 * T, 0.0), hth(4 * T, 0.0);
  CK(copy_d2d(xbar, w_dev, sizeof(double) * nx * n_obj, st));
  for (int c0 = ((n_steps - 1) / every) * every; n_steps > 0 && c0 >= 0; c0 -= every) {
    const int c1 = std::min(c0 + every, n_steps);
    // recompute the relaxed states of the segment from its checkpoint
    RUN(load_y(Y + (int64_t)(c0 / every) * ny));
    RUN(save_y(seg));
    for (int t = c0 + 1; t < c1; ++t) {
      CK(copy_d2d(s->x, X + (int64_t)t * nx, sizeof(double) * nx, st));
      RUN(build_lists(c, s, c->skin, c->r_bond));
      RUN(relax());
      RUN(save_y(seg + (int64_t)(t - c0) * ny));
      if (info) info->recomputed_steps += 1;
    }
    for (int t = c1 - 1; t >= c0; --t) {
      RUN(load_y(seg + (int64_t)(t - c0) * ny));
      CK(copy_d2d(s->x, X + (int64_t)t * nx, sizeof(double) * nx, st));
      RUN(build_lists(c, s, c->skin, c->r_bond));
      RUN(mu_pass());
      for (int o = 0; o < n_obj; ++o) {
        double* xb = xbar + (int64_t)o * nx;
        // Euler step: xbar_t (direct part) and mubar from xbar_{t+1}
        CK(launch_flux_vjp(s->x, s->T, mu, c->bd_off, c->bd_idx, n, (int)S, dt, nu0, Qm,
                           c->nsys ? c->dt_sys : nullptr, c->nsys ? c->sys_of : nullptr, xb, xdir, mubar, st));
        // relaxed state as an implicit function of x: H lam = H_yx mubar
        RUN(enqueue_tangent(c, s, nullptr, nullptr, mubar, nullptr, nullptr, nullptr, rhs, rhs + 3 * n, nullptr,
                            nullptr));
        int iters = 0;
        double rel = 0.0;
        RUN(cg_solve(c, s, rhs, lam, r, p, Hp, cg_tol, cg_max, iters, rel));
        if (info) {
          info->cg_iters_total += iters;
          info->cg_iters_max = std::max(info->cg_iters_max, iters);
          info->cg_resid_max = std::max(info->cg_resid_max, rel);
        }
        if (rel > cg_tol && iters >= cg_max) return MXE_ERR_NO_CONVERGE;
        // xbar_t = xdir + H_xx mubar - H_xy lam; thetabar += H_tx mubar - H_ty lam
        CK(launch_axpby(lam, lam, 0.0, -1.0, ny, st));
        RUN(enqueue_tangent(c, s, lam, lam + 3 * n, mubar, nullptr, nullptr, nullptr, nullptr, nullptr, mut, th));
        CK(launch_axpby(xdir, mut, 1.0, 1.0, nx, st));
        CK(copy_d2d(xb, xdir, sizeof(double) * nx, st));
        CK(cudaMemcpyAsync(hth.data(), th, sizeof(double) * 4 * T, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int u = 0; u < 2 * T; ++u) acc[(size_t)o * 2 * T + u] += hth[2 * T + u];
      }
      RUN(mxe_sync_status(c));
    }
  }
  for (size_t u = 0; u < (size_t)n_obj * 2 * T; ++u) dterm_host[u] = acc[u];
  if (dx0_dev) CK(copy_d2d(dx0_dev, xbar, sizeof(double) * nx * n_obj, st));
  // leave the state at the end of the run
  RUN(load_y(yT));
  CK(copy_d2d(s->x, X + (int64_t)n_steps * nx, sizeof(double) * nx, st));
  RUN(build_lists(c, s, c->skin, c->r_bond));
#undef RUN
  CK(cudaStreamSynchronize(st));
  return MXE_OK;
}

mxe_status mxe_unrolled_grad(mxe_ctx* c, mxe_state* s, int32_t n_steps, double dt, double nu0, double Qm,
                             double ftol, int32_t max_iter, const mxe_fire_params* fire, int32_t every,
                             const double* w_dev, double cg_tol, int32_t cg_max, double* dterm_host,
                             double* dx0_dev, mxe_grad_info* info) {
  return unrolled_grad_impl(c, s, n_steps, dt, nu0, Qm, ftol, max_iter, fire, every, 1, w_dev, cg_tol, cg_max,
                            dterm_host, dx0_dev, info);
}

mxe_status mxe_unrolled_grad_multi(mxe_ctx* c, mxe_state* s, int32_t n_steps, double dt, double nu0, double Qm,
                                   double ftol, int32_t max_iter, const mxe_fire_params* fire, int32_t every,
                                   int32_t n_obj, const double* w_dev, double cg_tol, int32_t cg_max,
                                   double* dterm_host, double* dx0_dev, mxe_grad_info* info) {
  return unrolled_grad_impl(c, s, n_steps, dt, nu0, Qm, ftol, max_iter, fire, every, n_obj, w_dev, cg_tol, cg_max,
                            dterm_host, dx0_dev, info);
}

mxe_status mxe_transport_step(mxe_ctx* c, mxe_state* s, const mxe_transport* opt, const double* mu_ex_dev,
                              double* v_dev, double dt, double nu0, double Qm) {
  if (!c || !state_ok(c, s) || !(dt >= 0.0) || !(nu0 >= 0.0) || !std::isfinite(Qm)) return MXE_ERR_ARG;
  const int host = opt ? opt->host_species : -1;
  const double tau = opt ? opt->tau_r : 0.0;
  if (host < -1 || host >= c->S || !(tau >= 0.0) || !std::isfinite(tau)) return MXE_ERR_ARG;
  if (tau > 0.0 && !v_dev) return MXE_ERR_ARG;
  if (c->fix_x_mask || c->fix_mu_mask) return MXE_ERR_ARG;  // reservoir groups belong to mxe_diffuse_step
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  cudaStream_t st = c->stream;
  mxe_status pre = mxe_sync_status(c);
  if (pre != MXE_OK) return pre;
  const double* mu = mu_ex_dev;
  if (!mu) {
    PassArgs A;
    fill_pass(c, s, A);
    A.site_E = nullptr;
    A.gq = nullptr;
    A.gs = nullptr;
    mxe_status ms = enqueue_passes(c, s, A, true);
    if (ms != MXE_OK) return ms;
    mu = c->mu_ex;
  }
  if (v_dev && !c->v_new) CK(dalloc(&c->v_new, (int64_t)c->S * c->n));
  CK(cudaMemsetAsync(c->step_flags, 0, sizeof(int), st));
  CK(TIMED("flux_ext", launch_transport_ext(s->x, s->T, mu, c->bd_off, c->bd_idx, c->n, c->S, dt, nu0, Qm, host, tau,
                                            v_dev, c->v_new, c->x_new, c->step_flags, c->flags,
                                            c->nsys ? c->dt_sys : nullptr, c->nsys ? c->sys_of : nullptr, st)));
  return mxe_sync_status(c);
}

mxe_status mxe_timing_enable(mxe_ctx* c, int32_t enable) {
  if (!c) return MXE_ERR_ARG;
  c->timing = enable != 0;
  return MXE_OK;
}

mxe_status mxe_timing_read(mxe_ctx* c, int32_t max_entries, char* names, int64_t* counts, double* total_ms,
                           int32_t* n_entries) {
  if (!c || max_entries < 0 || (max_entries > 0 && (!names || !counts || !total_ms))) return MXE_ERR_ARG;
  Guard gd(c->device);
  CK(cudaStreamSynchronize(c->stream));
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (auto& t : c->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.e0, t.e1) != cudaSuccess) cudaGetLastError();
    auto& a = agg[t.cls];
    a.first += 1;
    a.second += ms;
    c->event_pool.push_back(t.e0);
    c->event_pool.push_back(t.e1);
  }
  c->timed.clear();
  int32_t k = 0;
  for (auto& kv : agg) {
    if (k >= max_entries) break;
    std::memset(names + (size_t)k * MXE_TIMING_NAME_LEN, 0, MXE_TIMING_NAME_LEN);
    std::strncpy(names + (size_t)k * MXE_TIMING_NAME_LEN, kv.first.c_str(), MXE_TIMING_NAME_LEN - 1);
    counts[k] = kv.second.first;
    total_ms[k] = kv.second.second;
    ++k;
  }
  if (n_entries) *n_entries = k;
  return MXE_OK;
}

mxe_status mxe_sync_status(mxe_ctx* c) {
  if (!c) return MXE_ERR_ARG;
  Guard gd(c->device);
  CK(cudaMemcpyAsync(c->ints_h, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int f = c->ints_h[0];
  if (f) {
    CK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return map_flags(f);
}

mxe_status mxe_free_energy_grad_async(mxe_ctx* c, const mxe_state* s, double* F4_dev, double* dFdq_dev,
                                      double* dFdsigma_dev, double* mu_ex_dev, double* mu_dev) {
  if (!c || !state_ok(c, s) || !F4_dev) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  PassArgs A;
  fill_pass(c, s, A);
  if (dFdq_dev) A.gq = dFdq_dev;
  if (dFdsigma_dev) A.gs = dFdsigma_dev;
  if (mu_ex_dev) A.mu_ex = mu_ex_dev;
  A.mu = mu_dev;
  if (!dFdq_dev) A.gq = nullptr;
  if (!dFdsigma_dev) A.gs = nullptr;
  const bool want_mu = mu_ex_dev != nullptr || mu_dev != nullptr;
  if (!want_mu) A.mu_ex = nullptr;
  mxe_status ms = enqueue_passes(c, s, A, want_mu);
  if (ms != MXE_OK) return ms;
  if (c->nsys) CK(TIMED("energy_reduce", launch_energy_seg(c->site_E, c->n, c->B, F4_dev, c->stream)));
  else CK(TIMED("energy_reduce", launch_energy_reduce(c->site_E, c->n, c->partials, F4_dev, c->stream)));
  return MXE_OK;
}

mxe_status mxe_free_energy_grad(mxe_ctx* c, const mxe_state* s, double* F4_dev, double* dFdq_dev,
                                double* dFdsigma_dev, double* mu_ex_dev, double* mu_dev) {
  mxe_status ms = mxe_free_energy_grad_async(c, s, F4_dev, dFdq_dev, dFdsigma_dev, mu_ex_dev, mu_dev);
  if (ms != MXE_OK) return ms;
  return mxe_sync_status(c);
}

mxe_status mxe_relax(mxe_ctx* c, mxe_state* s, double ftol, int32_t max_iter, const mxe_fire_params* fire,
                     int32_t* iters_out, double* fmax_out) {
  if (!c || !state_ok(c, s) || !(ftol >= 0.0) || max_iter < 0) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  const mxe_fire_params fp = fire_params_or_default(fire);
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  // clear stale device errors from earlier asynchronous calls into this call's result
  mxe_status pre = mxe_sync_status(c);
  if (pre != MXE_OK) return pre;
  CK(copy_d2d(c->q0, s->q, sizeof(double) * 3 * n, st));
  CK(copy_d2d(c->s0, s->sigma, sizeof(double) * n, st));
  if (n > 0) {
    CK(cudaMemsetAsync(c->vq, 0, sizeof(double) * 3 * n, st));
    CK(cudaMemsetAsync(c->vs, 0, sizeof(double) * n, st));
  }
  Ctrl& H = *c->ctrl_h;
  mxe_status rr = ensure_relax_records(c);
  if (rr != MXE_OK) return rr;
  init_ctrl(c, H, fp, ftol, max_iter);
  CK(cudaMemcpyAsync(c->ctrl, &H, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  if (c->nsys) CK(launch_fire_seg_init(c->sf, c->nsys, fp.dt0, fp.alpha0, nullptr, st));
  if (c->precision != MXE_FP64)
    CK(TIMED("pack", launch_pack(s->q, s->sigma, s->x, c->abs_cell, n, c->S, c->grid, c->B, c->pos32, c->x32, nullptr, nullptr, st)));
  mxe_status result = fire_loop(c, s, max_iter, fp.check_every > 0 ? fp.check_every : 16, H);
  mxe_status info = record_relax_info(c, H);
  if (info != MXE_OK && result == MXE_OK) result = info;
  if (iters_out) *iters_out = H.iter;
  if (fmax_out) *fmax_out = H.fmax;
  if (result != MXE_OK && result != MXE_ERR_NO_CONVERGE) {
    CK(copy_d2d(s->q, c->q0, sizeof(double) * 3 * n, st));
    CK(copy_d2d(s->sigma, c->s0, sizeof(double) * n, st));
    CK(cudaStreamSynchronize(st));
    // the list was built for the discarded iterate; rebuild it for the restored state
    if (result != MXE_ERR_BOX_TOO_SMALL && result != MXE_ERR_NBR_OVERFLOW) build_lists(c, s, c->skin, c->r_bond);
    else c->have_list = false;
  }
  return result;
}

mxe_status mxe_run_staggered(mxe_ctx* c, mxe_state* s, int32_t n_steps, double dt, double nu0, double Qm,
                             double ftol, int32_t max_iter, const mxe_fire_params* fire, int32_t* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!c || !state_ok(c, s) || n_steps < 0 || !(dt >= 0.0) || !(nu0 >= 0.0) || !std::isfinite(Qm) ||
      !(ftol >= 0.0) || max_iter < 0 || max_iter > 100000)
    return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  if (n_steps == 0 || c->n == 0) {
    if (steps_done) *steps_done = n_steps;
    return MXE_OK;
  }
  Guard gd(c->device);
  const mxe_fire_params fp = fire_params_or_default(fire);
  const int chunk = fp.check_every > 0 ? fp.check_every : 16;
  cudaStream_t st = c->stream;
  mxe_status pre = mxe_sync_status(c);
  if (pre != MXE_OK) return pre;
  Ctrl& H = *c->ctrl_h;
  mxe_status rr = ensure_relax_records(c);
  if (rr != MXE_OK) return rr;
  init_ctrl(c, H, fp, ftol, max_iter);
  CK(cudaMemcpyAsync(c->ctrl, &H, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  const StepKey key{s->q, s->sigma, s->x, s->T, s->sublattice, s->mobile_mask, dt, nu0, Qm, max_iter,
                    fp.dt0, fp.alpha0, 0, c->nl, c->tpb, c->pair_tpb};
  mxe_status result = MXE_OK;
  int done = 0, stops = 0;
  c->run_launches = 0;
  while (done < n_steps) {
    mxe_status ms = ensure_step_graph(c, s, key);
    if (ms != MXE_OK) return ms;
    // one launch runs every remaining step on the device
    c->loop_h[0] = 0;
    c->loop_h[1] = n_steps;
    c->loop_h[2] = n_steps - done + 2;
    CK(cudaMemcpyAsync(c->loop_dev, c->loop_h, 3 * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaGraphLaunch(c->step_exec, st));
    c->run_launches += 1;
    CK(cudaMemcpyAsync(&H, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    done = H.steps;
    if (H.reason == kReasonError) {
      result = mxe_sync_status(c);
      if (result == MXE_OK) result = MXE_ERR_NONFINITE;
      break;
    }
    if (!(H.halted && H.reason == kReasonRebuild)) {
      if (done != n_steps) result = MXE_ERR_STATE;  // every launched step must have completed
      break;
    }
    // the skin criterion failed: rebuild, then finish the interrupted step
    if (++stops > n_steps * (max_iter + 2) + 16) {
      result = MXE_ERR_STATE;
      break;
    }
    ms = build_lists(c, s, c->skin, c->r_bond);
    if (ms != MXE_OK) {
      result = ms;
      break;
    }
    H.halted = 0;
    H.reason = kReasonNone;
    H.disp2_bits = 0ull;
    H.smax_bits = 0ull;
    H.sigma_max_build = c->sigma_max_build;
    if (H.phase == 1) {
      // the Euler step of this step is committed: continue its relaxation
      // (velocities, dt and alpha kept) outside the graph
      CK(cudaMemcpyAsync(c->ctrl, &H, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
      if (c->precision != MXE_FP64)
        CK(TIMED("pack", launch_pack(s->q, s->sigma, s->x, c->abs_cell, c->n, c->S, c->grid, c->B, c->pos32, c->x32, nullptr, nullptr, st)));
      ms = fire_loop(c, s, max_iter, chunk, H);
      if (ms != MXE_OK && ms != MXE_ERR_NO_CONVERGE) {
        result = ms;
        break;
      }
      done += 1;
      H.steps = done;
      H.phase = 0;
    }
    // phase 0: the step had not changed x; the graph runs it again from its start
    CK(cudaMemcpyAsync(c->ctrl, &H, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  }
  mxe_status info = record_relax_info(c, H);
  if (info != MXE_OK && result == MXE_OK) result = info;
  if (steps_done) *steps_done = done;
  return result;
}

mxe_status mxe_autotune(mxe_ctx* c, const mxe_state* s, int32_t* lanes_out, int32_t* threads_out) {
  if (!c || !state_ok(c, s)) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  mxe_status pre = mxe_sync_status(c);
  if (pre != MXE_OK) return pre;
  cudaStream_t st = c->stream;
  mxe_status rr = ensure_relax_records(c);
  if (rr != MXE_OK) return rr;
  const bool timing = c->timing;
  c->timing = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mxe_status result = MXE_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) result = MXE_ERR_CUDA;
  const int lanes[3] = {4, 8, 16}, threads[2] = {128, 256}, pthreads[3] = {64, 128, 256};
  int best_nl = c->nl, best_tpb = c->tpb, best_ptpb = c->pair_tpb;
  float best = INFINITY;
  for (int a = 0; a < 3 && result == MXE_OK; ++a)
    for (int b = 0; b < 2 && result == MXE_OK; ++b)
      for (int pb = 0; pb < (has_pair_index(c) ? 3 : 1) && result == MXE_OK; ++pb) {
        c->nl = lanes[a];
        c->tpb = threads[b];
        c->pair_tpb = has_pair_index(c) ? pthreads[pb] : 128;
        float total = 0.f;
        for (int rep = 0; rep < 3 && result == MXE_OK; ++rep) {  // rep 0 warms up
          if (cudaEventRecord(e0, st) != cudaSuccess) result = MXE_ERR_CUDA;
          if (result == MXE_OK) result = enqueue_tune_work(c, s);
          if (result == MXE_OK && cudaEventRecord(e1, st) != cudaSuccess) result = MXE_ERR_CUDA;
          float ms = 0.f;
          if (result == MXE_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            result = MXE_ERR_CUDA;
          if (rep > 0) total += ms;
        }
        if (result == MXE_OK && total < best) {
          best = total;
          best_nl = c->nl;
          best_tpb = c->tpb;
          best_ptpb = c->pair_tpb;
        }
      }
  c->nl = best_nl;
  c->tpb = best_tpb;
  c->pair_tpb = best_ptpb;
  c->timing = timing;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (result != MXE_OK) {
    cudaGetLastError();
    return result;
  }
  mxe_status fl = mxe_sync_status(c);
  if (fl != MXE_OK) return fl;
  if (lanes_out) *lanes_out = c->nl;
  if (threads_out) *threads_out = c->tpb;
  return MXE_OK;
}

mxe_status mxe_set_embedding(mxe_ctx* c, int32_t mode) {
  if (!c || (mode != MXE_EMBED_TAYLOR && mode != MXE_EMBED_EXACT)) return MXE_ERR_ARG;
  Guard gd(c->device);
  if (mode == MXE_EMBED_EXACT && !c->emb_buf) {
    CK(dalloc(&c->emb_buf, 9 * (int64_t)c->S * c->n));
    CK(dalloc(&c->emb_nrule, c->n));
  }
  c->embedding = mode;
  c->list_gen += 1;  // a captured staggered step is captured again
  return MXE_OK;
}

mxe_status mxe_set_pass_shape(mxe_ctx* c, int32_t lanes, int32_t threads) {
  if (!c || (lanes != 4 && lanes != 8 && lanes != 16) || (threads != 128 && threads != 256)) return MXE_ERR_ARG;
  c->nl = lanes;
  c->tpb = threads;
  return MXE_OK;
}

mxe_status mxe_run_stats(mxe_ctx* c, int32_t* graph_launches, int32_t* kernels_per_step) {
  if (!c) return MXE_ERR_ARG;
  if (graph_launches) *graph_launches = c->run_launches;
  if (kernels_per_step) *kernels_per_step = c->step_kernels;
  return MXE_OK;
}

mxe_status mxe_set_pair_block(mxe_ctx* c, int32_t pair_threads) {
  if (!c || (pair_threads != 64 && pair_threads != 128 && pair_threads != 256)) return MXE_ERR_ARG;
  c->pair_tpb = pair_threads;
  return MXE_OK;
}

mxe_status mxe_get_pass_shape(mxe_ctx* c, int32_t* lanes, int32_t* threads, int32_t* pair_threads) {
  if (!c) return MXE_ERR_ARG;
  if (lanes) *lanes = c->nl;
  if (threads) *threads = c->tpb;
  if (pair_threads) *pair_threads = c->pair_tpb;
  return MXE_OK;
}

mxe_status mxe_potential_pair_form(const mxe_potential* pot, int32_t* table_pattern, int32_t* power_form, int32_t* m,
                                   int32_t* n) {
  if (!pot) return MXE_ERR_ARG;
  DevPot d;
  const mxe_status ms = make_devpot(*pot, d);
  if (ms != MXE_OK) return ms;
  if (table_pattern) *table_pattern = d.tab;
  if (power_form) *power_form = d.pw_on;
  for (int s = 0; s < 2; ++s) {
    if (m) m[s] = d.pw_on ? d.pw_m[s] : 0;
    if (n) n[s] = d.pw_on ? d.pw_n[s] : 0;
  }
  return MXE_OK;
}

mxe_status mxe_pair_form(mxe_ctx* c, int32_t* table_pattern, int32_t* power_form) {
  if (!c) return MXE_ERR_ARG;
  if (table_pattern) *table_pattern = c->dp.tab;
  if (power_form) *power_form = c->dp.pw_on;
  return MXE_OK;
}

mxe_status mxe_diffuse_step_async(mxe_ctx* c, mxe_state* s, const double* mu_ex_dev, double dt, double nu0,
                                  double Qm) {
  if (!c || !state_ok(c, s) || !(dt >= 0.0) || !(nu0 >= 0.0) || !std::isfinite(Qm)) return MXE_ERR_ARG;
  if (!c->have_list) return MXE_ERR_STATE;
  Guard gd(c->device);
  cudaStream_t st = c->stream;
  const double* mu = mu_ex_dev;
  if (!mu) {
    PassArgs A;
    fill_pass(c, s, A);
    A.site_E = nullptr;
    A.gq = nullptr;
    A.gs = nullptr;
    mxe_status ms = enqueue_passes(c, s, A, true);
    if (ms != MXE_OK) return ms;
    mu = c->mu_ex;
  }
  CK(cudaMemsetAsync(c->step_flags, 0, sizeof(int), st));
  CK(TIMED("flux", launch_flux_res(s->x, s->T, mu, c->bd_off, c->bd_idx, c->n, c->S, dt, nu0, Qm, c->flux_tmp,
                                   c->x_new, c->step_flags, c->fix_x_mask, c->fix_x_value, c->fix_mu_mask,
                                   c->fix_mu_value, c->mu_eff, c->nsys ? c->dt_sys : nullptr,
                                   c->nsys ? c->sys_of : nullptr, nullptr, st)));
  CK(TIMED("commit", launch_commit_x(s->x, c->x_new, (int64_t)c->S * c->n, c->step_flags, c->flags, nullptr, st)));
  return MXE_OK;
}

mxe_status mxe_diffuse_step(mxe_ctx* c, mxe_state* s, const double* mu_ex_dev, double dt, double nu0, double Qm) {
  mxe_status ms = mxe_diffuse_step_async(c, s, mu_ex_dev, dt, nu0, Qm);
  if (ms != MXE_OK) return ms;
  return mxe_sync_status(c);
}

}  // extern "C"
