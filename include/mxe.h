/*
 * mxe.h -- C ABI of the GB300 MXE hot path.
 *
 * The library evaluates the mean-field, phase-averaged EAM free energy of a
 * lattice of Gaussian-smeared sites and its gradients (App. A, App. B.2,
 * Sec. 2.1 of Mendez & Ponga, "MXE: A package for simulating long-term
 * diffusive mass transport phenomena in nanoscale systems"), relaxes the mean
 * positions and widths at fixed composition (Sec. 4, dynamic relaxation; here
 * FIRE), and advances the molar fractions by one forward-Euler step of the
 * master equation (Sec. 3.1, Eq. MassTransport).
 *
 * Conventions shared by every call:
 *  - Units: Angstrom, eV, K, s.  kB = 8.617333262e-5 eV/K.
 *  - Sites i = 0..n-1; non-vacancy species k = 0..S-1 (S <= MXE_MAXS); the
 *    vacancy fraction x_iv = 1 - sum_k x_ik is implicit.
 *  - sigma_i is the per-Cartesian-component standard deviation of site i's
 *    Gaussian, sigma = (beta m)^(-1/2) / omega with the paper's omega.
 *  - Arrays are structure-of-arrays, contiguous, FP64 unless stated:
 *    q [3][n] (all x, then all y, then all z), sigma [n], x [S][n], T [n].
 *  - Every state, input and output array is a CALLER-OWNED DEVICE pointer.
 *    The context owns its own scratch (cell grid, neighbour and bond lists,
 *    per-site embedding terms, reduction buffers, FIRE state).
 *  - Every call is enqueued on the context's CUDA stream.  Calls that return
 *    host values (counts, iteration numbers, statuses found on the device)
 *    synchronise that stream before returning.
 *  - No exception crosses the ABI.  Every call returns an mxe_status.  On any
 *    error other than MXE_ERR_NO_CONVERGE, in-out arrays are left as they were.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef MXE_H
#define MXE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MXE_MAXS 4

#if defined(__GNUC__)
#define MXE_API __attribute__((visibility("default")))
#else
#define MXE_API
#endif

typedef enum {
    MXE_OK = 0,
    MXE_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, unsupported option) */
    MXE_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MXE_ERR_OOM = 3,            /* device allocation failed */
    MXE_ERR_BOX_TOO_SMALL = 4,  /* a box length is below 2 r_list */
    MXE_ERR_NBR_OVERFLOW = 5,   /* neighbour count exceeds the list's int32 range */
    MXE_ERR_GEOMETRY = 6,       /* a quadrature node closer than 0.5 A, or a static density <= 1e-12 */
    MXE_ERR_NONFINITE = 7,      /* NaN or Inf in the free energy or a gradient */
    MXE_ERR_X_RANGE = 8,        /* Euler step would give x_ik < -1e-12 or sum_k x_ik > 1 + 1e-12 */
    MXE_ERR_NO_CONVERGE = 9,    /* relaxation reached max_iter; the last iterate is returned */
    MXE_ERR_STATE = 10          /* call order violated (e.g. no neighbour list built yet) */
} mxe_status;

typedef enum {
    MXE_FP64 = 0,        /* every step in FP64 */
    MXE_FP32_MIXED = 1,  /* node arithmetic (distance, switch, exp, derivatives) in FP32;
                            each pair's 13-node partial sums added into FP64 per-site sums;
                            FP64 for per-site results, totals, mu differences, x, FIRE */
    MXE_FP32_FF = 2      /* as MXE_FP32_MIXED, but the per-site sums are carried as
                            unevaluated float pairs (float-float, >= 44-bit significand)
                            and rounded to FP64 once per site */
} mxe_precision;

/* Periodic orthorhombic box.  A free surface is a periodic axis longer than
 * the slab by more than r_list (a vacuum gap), so no pair spans the gap.    */
typedef struct {
    double L[3];
} mxe_box;

/* Analytic EAM tables (App. B.2 with pair-resolved species):
 *   phi_kl(r) = phi_A[k][l] exp(-phi_p[k][l] (r / phi_r0[k][l] - 1)) S(r)
 *   f_kl(r)   = f_xi[k][l]  exp(-f_q[k][l]  (r / f_r0[k][l]  - 1)) S(r)
 *               (electron density at a k-site from an l-neighbour)
 *   F_k(rho)  = -E[k] sqrt(rho)
 *   S(r)      = 1 - 10 t^3 + 15 t^4 - 6 t^5, t = (r - r_switch)/(r_cut - r_switch)
 *               clipped to [0, 1].
 * cross_geomean != 0: phi_kl for k != l is sqrt(phi_kk phi_ll) pointwise and
 * the off-diagonal phi entries are ignored.  Otherwise phi must be symmetric
 * (phi_kl = phi_lk), else mxe_create returns MXE_ERR_ARG.  A = 0 or xi = 0
 * switches a term off.
 * lj != 0: the pair terms are thermalized Lennard-Jones terms (App. C.1)
 *   phi_kl(r) = 4 lj_eps[k][l] ((lj_sigma[k][l] / r)^12 - (lj_sigma[k][l] / r)^6) S(r)
 * (phi_* and cross_geomean ignored; the tables must be symmetric, eps >= 0,
 * sigma > 0).  An element with E[k] = 0 has no embedding energy (no density
 * check either), so lj with E = 0 and f_xi = 0 is a pure pair potential.
 * Lennard-Jones terms are evaluated in MXE_FP64 contexts only.               */
typedef struct {
    int32_t n_species;
    int32_t cross_geomean;
    double phi_A[MXE_MAXS][MXE_MAXS], phi_p[MXE_MAXS][MXE_MAXS], phi_r0[MXE_MAXS][MXE_MAXS];
    double f_xi[MXE_MAXS][MXE_MAXS], f_q[MXE_MAXS][MXE_MAXS], f_r0[MXE_MAXS][MXE_MAXS];
    double E[MXE_MAXS];
    double r_switch, r_cut;
    int32_t lj;
    int32_t pad;
    double lj_eps[MXE_MAXS][MXE_MAXS], lj_sigma[MXE_MAXS][MXE_MAXS];
} mxe_potential;

/* Per-site state (device pointers, caller-owned).  q and sigma are in-out for
 * mxe_relax, x is in-out for mxe_diffuse_step.  sublattice may be NULL (all
 * sites on sublattice 0); bit s of mobile_mask marks sublattice s as carrying
 * mass flux (bonds only join two sites of the same mobile sublattice).      */
typedef struct {
    int64_t n;
    double *q;                 /* [3][n] */
    double *sigma;             /* [n] */
    double *x;                 /* [S][n] */
    const double *T;           /* [n] */
    const uint8_t *sublattice; /* [n] or NULL */
    uint32_t mobile_mask;
    uint32_t pad;
} mxe_state;

/* FIRE constants (Bitzek et al., PRL 97, 170201, 2006), unit masses.
 * sigma_max > 0 bounds every width from above (<= 0: no bound).  The paper's
 * free energy gives each site -3 kB T ln sigma whatever its occupancy, so the
 * width of a site with zero occupied fraction has nothing opposing it and
 * grows without bound; a finite sigma_max keeps such sites in a box.        */
typedef struct {
    double dt0, dt_max, f_inc, f_dec, alpha0, f_alpha;
    double sigma_max;
    int32_t n_min;
    int32_t check_every;  /* iterations enqueued between host checks (<= 0: 16) */
} mxe_fire_params;

typedef struct mxe_ctx mxe_ctx;

/* Human-readable name of a status code (static string, never NULL). */
MXE_API const char *mxe_status_string(mxe_status s);

/* Create a context for n sites on one box with one potential, evaluating in
 * the given precision, enqueuing on cuda_stream (a cudaStream_t; NULL = the
 * legacy default stream).  Allocates the n-sized scratch on the current
 * device.  *out is NULL on error.                                            */
MXE_API mxe_status mxe_create(mxe_ctx **out, const mxe_box *box, const mxe_potential *pot, int64_t n,
                      mxe_precision precision, void *cuda_stream);

/* Batched ensemble: n_systems independent periodic systems of one potential
 * in one context (each system is a separate instance of the problem of Sec. 4;
 * systems share no pair, bond or reduction).  Sites are concatenated system
 * after system: system b holds sites offsets[b] .. offsets[b+1]-1 (host array
 * of n_systems + 1 nondecreasing values, offsets[0] = 0, offsets[n_systems] =
 * n) in the box boxes[b] (host array of n_systems boxes); temperatures,
 * compositions and sizes may differ between systems.  Every other call takes
 * the concatenated state and works per system:
 *  - neighbour and bond sets never cross systems; each system has its own cell
 *    grid and minimum image; every box must hold 2 r_list (r_list from the
 *    largest sigma of the whole batch);
 *  - mxe_free_energy_grad writes F4_dev as [n_systems][4] (E_V, F_vib, F_mix,
 *    F of each system, each summed in a fixed order);
 *  - mxe_relax runs FIRE separately per system (own P, norms, dt, alpha,
 *    n_pos and convergence test; a converged system stops moving while the
 *    others continue).  It returns MXE_OK when every system converged,
 *    MXE_ERR_NO_CONVERGE when any reached max_iter; iters_out is the largest
 *    iteration count and fmax_out the largest fmax; mxe_relax_info gives
 *    them per system;
 *  - mxe_diffuse_step uses dt * scale_b in system b (mxe_set_dt_scale;
 *    default 1), so systems at very different temperatures each take a
 *    stable step.
 * 1 <= n_systems <= 1048576.  mxe_create is this call with n_systems = 0 (one
 * system, offsets ignored).                                                  */
MXE_API mxe_status mxe_create_batch(mxe_ctx **out, int32_t n_systems, const mxe_box *boxes, const int64_t *offsets,
                                    const mxe_potential *pot, int64_t n, mxe_precision precision,
                                    void *cuda_stream);

/* Per-system multipliers of the Euler step of a batch (host array of
 * n_systems finite values >= 0; NULL restores 1).  MXE_ERR_ARG on a
 * context without a batch.  Syncs.                                          */
MXE_API mxe_status mxe_set_dt_scale(mxe_ctx *ctx, const double *scale);

/* Outcome of the last mxe_relax per system (n_entries = n_systems, or 1 for a
 * context without a batch): FIRE updates taken, fmax at the last evaluation,
 * and whether fmax <= ftol was reached (host arrays, each may be NULL).      */
MXE_API mxe_status mxe_relax_info(mxe_ctx *ctx, int32_t n_entries, int32_t *iters, double *fmax,
                                  int32_t *converged);

/* Release every device allocation of the context.  NULL is accepted. */
MXE_API mxe_status mxe_destroy(mxe_ctx *ctx);

/* Neighbour and bond sets (Sec. 4, Algorithm 1: neighbour-list step; Sec. 3:
 * the transport sum runs over nearest neighbours).
 *   r_list = r_cut + sqrt(6) max_i sigma_i + skin  (a pair farther apart than
 *   r_cut + sqrt(6) max sigma has every quadrature node beyond r_cut).
 * Neighbours: every j != i with |d_ij| < r_list, d_ij the minimum image of
 * q_j - q_i; d and |d|^2 are formed in FP64 without FMA as
 *   d_a = (q_ja - q_ia) - L_a rint((q_ja - q_ia) (1/L_a)),
 *   |d|^2 = (d_x d_x + d_y d_y) + d_z d_z,
 * so the set is bit-reproducible.  Bonds: neighbours with |d| < r_bond on the
 * same sublattice, that sublattice mobile.  Rows are sorted by j.
 * Requires L_a >= 2 r_list on every axis (else MXE_ERR_BOX_TOO_SMALL).
 * The list stays valid while 2 max|q - q_build| + sqrt(6)(max sigma - max
 * sigma_build) <= skin; mxe_relax rebuilds it on its own when that fails.
 * Outputs (host, optional): total neighbour entries, r_list used.  Syncs.  */
MXE_API mxe_status mxe_build_neighbors(mxe_ctx *ctx, const mxe_state *state, double skin, double r_bond,
                               int64_t *n_pairs_out, double *r_list_out);

/* Copy the current neighbour CSR (offsets_dev [n+1], idx_dev [n_pairs], int32
 * device arrays, caller-owned) -- for tests; bit-identical to a brute-force
 * evaluation of the rule above.  Either pointer may be NULL.                 */
MXE_API mxe_status mxe_export_neighbors(mxe_ctx *ctx, int32_t *offsets_dev, int32_t *idx_dev);

/* Same for the bond CSR; *n_bonds_out (host) receives the entry count.     */
MXE_API mxe_status mxe_export_bonds(mxe_ctx *ctx, int32_t *offsets_dev, int32_t *idx_dev, int64_t *n_bonds_out);

/* Free energy and its three gradients (App. A third-degree rule with 12 nodes
 * per pair at +-sqrt(6) sigma along each axis for each of the two sites;
 * App. B.2 Taylor-linearised embedding; Sec. 2.1 mean-field free energy):
 *   rho_bar_i^k = sum_j sum_l x_jl f_kl(|d_ij|),  <rho_i^k> = sum_j sum_l x_jl <f_kl>_ij
 *   e_i^k = F_k(rho_bar) + F_k'(rho_bar)(<rho> - rho_bar)
 *   E_V   = sum_i [1/2 sum_j sum_kl x_ik x_jl <phi_kl>_ij + sum_k x_ik e_i^k]
 *   F_vib = -3 kB sum_i T_i ln(sigma_i / 1 A)
 *   F_mix = kB sum_i T_i (sum_k x_ik ln x_ik + x_iv ln x_iv),  0 ln 0 = 0
 *   F     = E_V + F_vib + F_mix
 * Outputs (device, caller-owned; any may be NULL except F4_dev):
 *   F4_dev [4]       = E_V, F_vib, F_mix, F (FP64, deterministic order)
 *   dFdq_dev [3][n]  = dF/dq (the force is its negative)
 *   dFdsigma_dev [n] = dF/dsigma
 *   mu_ex_dev [S][n] = dE_V/dx_ik with x_iv dependent (excess chemical potential)
 *   mu_dev [S][n]    = dF/dx_ik = mu_ex + kB T_i (ln x_ik - ln x_iv), ln arguments
 *                      floored at 1e-300
 * Requires a neighbour list built for this state.  Syncs and returns
 * MXE_ERR_GEOMETRY / MXE_ERR_NONFINITE if found.                              */
MXE_API mxe_status mxe_free_energy_grad(mxe_ctx *ctx, const mxe_state *state, double *F4_dev,
                                double *dFdq_dev, double *dFdsigma_dev, double *mu_ex_dev,
                                double *mu_dev);

/* As mxe_free_energy_grad, but only enqueues the work: device-found errors
 * are kept in the context and returned by the next mxe_sync_status.        */
MXE_API mxe_status mxe_free_energy_grad_async(mxe_ctx *ctx, const mxe_state *state, double *F4_dev,
                                      double *dFdq_dev, double *dFdsigma_dev, double *mu_ex_dev,
                                      double *mu_dev);

/* Synchronise the context's stream and return (then clear) the first error
 * recorded on the device since the last call.                               */
MXE_API mxe_status mxe_sync_status(mxe_ctx *ctx);

/* Relax (q, sigma) at fixed x (Sec. 4: the equilibrium step of the staggered
 * scheme) with FIRE:  y = (q, sigma), f = -(dF/dq, dF/dsigma), v = 0,
 * dt = dt0, alpha = alpha0.  Iteration it = 0, 1, ...:
 *   1. f(y); fmax = max_i max(|dF/dq_i|_2, |dF/dsigma_i|); stop (MXE_OK) if fmax <= ftol
 *   2. stop with MXE_ERR_NO_CONVERGE if it == max_iter
 *   3. if it > 0: P = f.v; P > 0: n_pos += 1 and, if n_pos > n_min,
 *      dt = min(f_inc dt, dt_max), alpha *= f_alpha;  P <= 0: n_pos = 0,
 *      dt *= f_dec, alpha = alpha0, v = 0
 *   4. v += dt f;  v = (1 - alpha) v + alpha |v| f / |f|   (global norms)
 *   5. y += dt v; a sigma leaving [1e-3 A, sigma_max] is set to the bound
 *      and its velocity to zero
 * The sigma force is projected on that box (zero where a bound blocks it) in
 * fmax, P, |f| and the update.
 * Neighbour lists are rebuilt whenever the skin criterion fails.
 * fire may be NULL (defaults dt0 0.02, dt_max 0.1, f_inc 1.1, f_dec 0.5,
 * alpha0 0.1, f_alpha 0.99, n_min 5, no sigma_max).  iters_out = number of FIRE updates,
 * fmax_out = fmax at the last evaluation (host, optional).  Syncs.
 * On GEOMETRY / NONFINITE the input (q, sigma) is restored.                 */
MXE_API mxe_status mxe_relax(mxe_ctx *ctx, mxe_state *state, double ftol, int32_t max_iter,
                     const mxe_fire_params *fire, int32_t *iters_out, double *fmax_out);

/* One forward-Euler step of the master equation (Sec. 3.1, Eq. MassTransport
 * with tau_r = 0, Eq. attempt_freq_mass), per species k and bond (i, j):
 *   J_{i->j} = nu0 exp(-beta_i Qm) x_ik x_jv exp(beta_i (mu_ik - mu_jk))
 *   x_ik' = x_ik + dt sum_{j in bonds(i)} (J_{j->i} - J_{i->j})
 * with mu the excess chemical potential dE_V/dx.  Each bond's net exchange
 * is formed identically from both ends, so the updates of i and j cancel
 * exactly and total mass is conserved up to the rounding of the two sums.
 * mu_ex_dev may be NULL: it is then computed first (one free-energy pass).
 * x is updated only if every x_ik' >= -1e-12 and sum_k x_ik' <= 1 + 1e-12,
 * else MXE_ERR_X_RANGE and x is unchanged.  Requires a bond list.  Syncs.   */
MXE_API mxe_status mxe_diffuse_step(mxe_ctx *ctx, mxe_state *state, const double *mu_ex_dev,
                            double dt, double nu0, double Qm);

/* As mxe_diffuse_step but enqueue-only; the range status is kept for the
 * next mxe_sync_status.  The conditional commit of x happens on the device. */
MXE_API mxe_status mxe_diffuse_step_async(mxe_ctx *ctx, mxe_state *state, const double *mu_ex_dev,
                                  double dt, double nu0, double Qm);

/* The staggered scheme (Sec. 4, Algorithm 1) for n_steps steps, each:
 *   1. excess chemical potentials mu_ex at the current state;
 *   2. one Euler step of x as mxe_diffuse_step(dt, nu0, Qm) (per-system dt
 *      scale and reservoir groups included);
 *   3. relaxation of (q, sigma) at the new x as mxe_relax(ftol, max_iter,
 *      fire): exactly max_iter + 1 force evaluations are enqueued; a system
 *      that converges earlier stops moving.  Not converging within max_iter
 *      is not an error here (the next step starts from the last iterate).
 * The step is captured once in a CUDA graph (on a private stream) as the body
 * of a while node, so one graph launch runs all the steps on the device, with
 * no host round trip between them: after each step a one-thread kernel lets
 * the loop go on while steps remain, no stop is pending and the body has run
 * fewer than (steps left + 2) times.  The graph is rebuilt when the state
 * pointers, the step parameters, the pass shape or the lists change.  When
 * the skin criterion fails, the loop stops itself; the host rebuilds the
 * lists, finishes the interrupted step and launches the loop again.  *steps_done (host, optional) receives the
 * completed steps.  On MXE_ERR_GEOMETRY / NONFINITE / X_RANGE the run stops
 * inside the failing step: steps before it are complete, and x is not
 * advanced by a step whose range check failed.  mxe_relax_info then
 * describes the relaxation of the last step.  Syncs at the end (and at each
 * rebuild).                                                                  */
MXE_API mxe_status mxe_run_staggered(mxe_ctx *ctx, mxe_state *state, int32_t n_steps, double dt, double nu0,
                                     double Qm, double ftol, int32_t max_iter, const mxe_fire_params *fire,
                                     int32_t *steps_done);

/* The last mxe_run_staggered: graph launches it made (one, plus one after
 * each list rebuild) and the kernels of one captured step (the loop-control
 * kernel included); host values, either pointer may be NULL.                */
MXE_API mxe_status mxe_run_stats(mxe_ctx *ctx, int32_t *graph_launches, int32_t *kernels_per_step);

/* Autotuner of the passes: times every pass shape -- lanes per site 4, 8, 16
 * (the chunk of a site's neighbour row each lane takes) times 128 or 256
 * threads per block of the per-site passes and gathers, times 64, 128 or 256
 * unordered pairs per block of the pair kernels (contexts with a pair index)
 * -- on the given state over one staggered step's worth of passes and keeps
 * the fastest for this context.  Results do not depend on the shape beyond
 * rounding order.  Requires a neighbour list.  lanes_out / threads_out (host,
 * optional) receive the choice; mxe_get_pass_shape reads all three.  Syncs.
 * mxe_set_pass_shape and mxe_set_pair_block set a shape directly.           */
MXE_API mxe_status mxe_autotune(mxe_ctx *ctx, const mxe_state *state, int32_t *lanes_out, int32_t *threads_out);
MXE_API mxe_status mxe_set_pass_shape(mxe_ctx *ctx, int32_t lanes, int32_t threads);
MXE_API mxe_status mxe_set_pair_block(mxe_ctx *ctx, int32_t pair_threads);
MXE_API mxe_status mxe_get_pass_shape(mxe_ctx *ctx, int32_t *lanes, int32_t *threads, int32_t *pair_threads);

/* Forms of the pair kernels this context's potential takes (host values,
 * either pointer may be NULL):
 *  table_pattern 1: two species, two like pair terms and a cross term, a
 *    density that depends on the neighbour's species only (the species tables
 *    are compile-time constants in the pair kernels); 0: general tables.
 *  power_form 1: in addition the cross term is the geometric mean of the like
 *    terms, and each species' pair and density terms are integer powers
 *    (<= 16) of one exponential exp(-beta_s r), to 1e-15 in their rates: the
 *    accurate pass evaluates two exponentials per node (App. A) and forms the
 *    terms as products; 0: one exponential per term.                        */
MXE_API mxe_status mxe_pair_form(mxe_ctx *ctx, int32_t *table_pattern, int32_t *power_form);

/* The same decision for a potential alone, on the host (no context, no GPU):
 * table_pattern and power_form as above; m, n (host arrays of 2, may be NULL)
 * receive each species' integer powers of exp(-beta_s r) for the like pair
 * term and the density term when power_form is 1 (0 otherwise).
 * MXE_ERR_ARG for a potential mxe_create would reject.                      */
MXE_API mxe_status mxe_potential_pair_form(const mxe_potential *pot, int32_t *table_pattern, int32_t *power_form,
                                           int32_t *m, int32_t *n);

/* Phase average of the embedding term (App. B.2).
 *  MXE_EMBED_TAYLOR (default): the Taylor form Eq. F_taylor_mxe,
 *    <F_k(rho_i)> ~ F_k(rho_bar_i) + F_k'(rho_bar_i)(<rho_i> - rho_bar_i).
 *  MXE_EMBED_EXACT: the third-degree rule of App. A applied to the many-body
 *    function itself (the form the paper states before replacing it by its
 *    Taylor expansion).  Site i's rule covers the N_i sites inside the
 *    potential cut-off: i and every neighbour j with |qbar_j - qbar_i| <
 *    r_cut; rho_i^k = sum over those j of sum_l x_jl f_kl(r_ij); N_q = 3 N_i
 *    coordinates, M = 2 N_q nodes of weight 1/M, each moving one site s of
 *    the rule by +-sigma_s sqrt(N_q) along one axis:
 *      <F_k(rho_i^k)> = (1/M) sum_nodes F_k(rho_i^k(node)).
 *    The rule's membership is fixed by the mean positions, so F is piecewise
 *    smooth: it jumps where a mean distance crosses r_cut.  Every call then
 *    uses this average (energies, gradients, chemical potentials, mxe_relax,
 *    mxe_run_staggered); the derivative calls (mxe_tangent,
 *    mxe_unrolled_grad) return MXE_ERR_ARG.  Allocates the rule data (9 S + 1
 *    values per site) on first use.  GEOMETRY also when a node density is
 *    <= 1e-12 for an occupied element with an embedding energy.              */
#define MXE_EMBED_TAYLOR 0
#define MXE_EMBED_EXACT 1
MXE_API mxe_status mxe_set_embedding(mxe_ctx *ctx, int32_t mode);

/* ---------------------------------------------------------------------------
 * Derivatives of the staggered scheme (second order).
 *
 * Every pair and density function of the potential is a radial term
 * A exp(kappa - lambda r) S(r) (App. B.2 analytic forms with the cut-off
 * switch).  The context holds the distinct terms: the pair terms first, then
 * the density terms.  mxe_potential_terms returns their count, (A, kappa,
 * lambda) for each (host array [3 (n_phi + n_f)]), and which term each species
 * pair uses (phi_of, f_of: host [MXE_MAXS][MXE_MAXS], -1 = none; f_of indices
 * count from n_phi).  Parameter sensitivities are reported per term with
 * respect to c = ln A + kappa and lambda (dF/dc = F, dF/dlambda = -r F); a
 * caller maps them to its own parameters by the chain rule.                 */
MXE_API mxe_status mxe_potential_terms(mxe_ctx *ctx, int32_t *n_phi, int32_t *n_f, double *terms,
                                       int32_t *phi_of, int32_t *f_of);

/* Chain rule from the term sensitivities to per-element parameters (App.
 * B.2 analytic forms).  For tables with the element structure -- element e
 * has a pair term A_e exp(-p_e (r/r0_e - 1)) S(r), the density from an
 * e-neighbour is xi_e exp(-q_e (r/r0_e - 1)) S(r) at every site (same r0_e),
 * and the cross pair of two elements is their geometric mean (S = 2) -- the
 * parameters theta_e = (A_e, p_e, q_e, r0_e) enter the radial terms only
 * through c = ln A + exponent and lambda = exponent / r0 (the cross pair: the
 * mean of the two elements' c and lambda).  Given dterm (host [2 T]:
 * dL/dc_u then dL/dlambda_u, in the term order of mxe_potential_terms, as
 * mxe_tangent and mxe_unrolled_grad report them), writes out (host [S][4])
 * = dL/d(A_e, p_e, q_e, r0_e) with the closed-form Jacobian.  Host
 * arithmetic only (no context, no device).  MXE_ERR_ARG for tables without
 * that structure (or Lennard-Jones terms).                                   */
MXE_API mxe_status mxe_element_param_grad(const mxe_potential *pot, const double *dterm, double *out);

/* Forward-mode pass (FP64 in every precision mode): the gradients of the
 * free energy and their directional derivatives along a tangent (dq [3][n],
 * dsigma [n], dx [S][n]; each may be NULL = zero) of the state:
 *   dFdq, dFdsigma, mu_ex                 values (as mxe_free_energy_grad)
 *   dFdq_t, dFdsigma_t, mu_ex_t           H v: the Hessian of F (of E_V for
 *                                         mu_ex) in (q, sigma, x) times the tangent
 *   dterm [4 T] (T = n_phi + n_f)         dE_V/dc_u, dE_V/dlambda_u (2 T values),
 *                                         then their directional derivatives (2 T)
 * Every output is a caller-owned device array and may be NULL.  Because the
 * Hessian is symmetric these products are also the vector-Jacobian products
 * of the gradients.  Requires a neighbour list.  Syncs.                      */
MXE_API mxe_status mxe_tangent(mxe_ctx *ctx, const mxe_state *state, const double *dq_dev, const double *dsigma_dev,
                               const double *dx_dev, double *dFdq_dev, double *dFdsigma_dev, double *mu_ex_dev,
                               double *dFdq_t_dev, double *dFdsigma_t_dev, double *mu_ex_t_dev, double *dterm_dev);

/* Vector-Jacobian product of the Euler step x' = x + dt R(x, mu) of
 * mxe_diffuse_step (Sec. 3.1): given the cotangent xbar_next [S][n] of x',
 * writes xbar = xbar_next + (dt dR/dx)^T xbar_next and mubar = (dt dR/dmu)^T
 * xbar_next (device [S][n] each), at the state's x and the given mu_ex.
 * Per-system step multipliers of a batch apply; reservoir groups are not
 * differentiated (MXE_ERR_ARG while any is set).  Syncs.                     */
MXE_API mxe_status mxe_flux_vjp(mxe_ctx *ctx, const mxe_state *state, const double *mu_ex_dev, double dt, double nu0,
                                double Qm, const double *xbar_next_dev, double *xbar_dev, double *mubar_dev);

typedef struct {
    int32_t relax_iters_total;  /* FIRE updates of every relaxation, forward and recomputed */
    int32_t recomputed_steps;   /* relaxations repeated from checkpoints */
    int32_t cg_iters_total;
    int32_t cg_iters_max;
    double cg_resid_max;        /* largest final |r| / |rhs| */
} mxe_grad_info;

/* Gradient of L = sum_ik w_ik x_ik(n_steps) after n_steps staggered steps
 * (Sec. 4) with respect to the radial-term parameters and the initial x.
 * Forward: y_0 = relax(x_0); per step mu_t = mu_ex(y_t, x_t), x_{t+1} =
 * x_t + dt R(x_t, mu_t), y_{t+1} = relax(x_{t+1}) from y_t, where y = (q,
 * sigma) and relax = mxe_relax(ftol, max_iter, fire), which must converge
 * (else MXE_ERR_NO_CONVERGE).  Each relaxed state is differentiated as the
 * implicit function grad_y F(y, x) = 0: the reverse sweep solves
 * H_yy lam = H_yx mubar by conjugate gradients (to |r| <= cg_tol |rhs|,
 * at most cg_max iterations, else MXE_ERR_NO_CONVERGE), with the Hessian
 * products of mxe_tangent, and accumulates
 *   xbar_t = xbar_{t+1} + (dt dR/dx)^T xbar_{t+1} + H_xx mubar - H_xy lam,
 *   thetabar += H_theta,x mubar - H_theta,y lam.
 * (q, sigma) are kept every `checkpoint_every` steps and recomputed inside a
 * segment on the way back; x is kept for every step.  Outputs: dterm_host
 * [2 T] (dL/dc_u, then dL/dlambda_u, host), dx0_dev [S][n] (dL/dx_0, device,
 * may be NULL), info (host, may be NULL); the state is left at the end of the
 * run.  FP64 contexts only, no reservoir groups.  Syncs.                     */
MXE_API mxe_status mxe_unrolled_grad(mxe_ctx *ctx, mxe_state *state, int32_t n_steps, double dt, double nu0,
                                     double Qm, double ftol, int32_t max_iter, const mxe_fire_params *fire,
                                     int32_t checkpoint_every, const double *w_dev, double cg_tol, int32_t cg_max,
                                     double *dterm_host, double *dx0_dev, mxe_grad_info *info);

/* As mxe_unrolled_grad for n_obj objectives L_o = sum_ik w_o,ik x_ik(n_steps)
 * at once (w_dev: device [n_obj][S][n], e.g. the bins of a z-profile): one
 * forward sweep, and one recomputation of each checkpoint segment's relaxed
 * states, serve every objective; the reverse steps (Euler-step VJP, the CG
 * solve on H_yy, the tangent pass) run per objective.  dterm_host: host
 * [n_obj][2 T]; dx0_dev: device [n_obj][S][n] or NULL.  1 <= n_obj <= 4096.
 * Same requirements and statuses as mxe_unrolled_grad.                       */
MXE_API mxe_status mxe_unrolled_grad_multi(mxe_ctx *ctx, mxe_state *state, int32_t n_steps, double dt, double nu0,
                                           double Qm, double ftol, int32_t max_iter, const mxe_fire_params *fire,
                                           int32_t checkpoint_every, int32_t n_obj, const double *w_dev,
                                           double cg_tol, int32_t cg_max, double *dterm_host, double *dx0_dev,
                                           mxe_grad_info *info);

/* Variants of the transport step (Sec. 3: Eq. Transport, Eq. MassTransport).
 *  host_species = -1: vacancy-mediated exchange, as mxe_diffuse_step.
 *  host_species = h:  species h is the exchange partner of every other
 *     species instead of the vacancy (a substitutional alloy whose two
 *     species are the x and 1 - x of Eq. MassTransport):
 *       J^k_{i->j} = D_i x_ik x_jh exp(beta_i (m_ik - m_jk)),  m_k = mu_k - mu_h,
 *     every k atom leaving a site is replaced by an h atom (dx_h = -sum dx_k),
 *     so each species and each site's occupied total are conserved.
 *  tau_r > 0: the ballistic term of Eq. Transport, tau_r x'' + x' = R, as
 *     x' = v, tau_r v' = R - v; over one step R is held at its start value and
 *     v is integrated exactly:
 *       v' = R + (v - R) e,  x' = x + dt R + tau_r (v - R)(1 - e),  e = exp(-dt/tau_r)
 *     (tau_r -> 0 gives the Euler step).  v_dev [S][n] (caller-owned device
 *     array, in-out) holds the rates; start it at zero (or at R).  With
 *     tau_r = 0, v_dev may be NULL; if given it receives R.              */
typedef struct {
    int32_t host_species;  /* -1: vacancy-mediated */
    int32_t pad;
    double tau_r;          /* s; 0: purely diffusive */
} mxe_transport;

/* One step of the variants above.  opt NULL = vacancy-mediated, tau_r = 0.
 * mu_ex_dev as in mxe_diffuse_step (NULL: computed first).  x (and v) are
 * updated only if every x_ik' >= -1e-12 and sum_k x_ik' <= 1 + 1e-12, else
 * MXE_ERR_X_RANGE and both are unchanged.  Per-system step multipliers of a
 * batch apply.  Reservoir groups are not combined with the variants
 * (MXE_ERR_ARG while any is set).  Syncs.                                  */
MXE_API mxe_status mxe_transport_step(mxe_ctx *ctx, mxe_state *state, const mxe_transport *opt,
                                      const double *mu_ex_dev, double *v_dev, double dt, double nu0, double Qm);

/* Reservoir groups of the Euler step (Sec. 4: fix setatomicfraction, fix
 * setchemicalpotential; Algorithm 1: applied after the mass-transport step and
 * after the force computation).  fix_mu_mask [n] (nonzero: the site is in the
 * chemical-potential group) with fix_mu_value [S][n]: in every rate of
 * mxe_diffuse_step such a site enters with the held excess chemical potential
 * in place of the computed one.  fix_x_mask [n] with fix_x_value [S][n]: after
 * the Euler step such a site has x set to the held value (the range check then
 * applies to the held value).  Caller-owned device arrays; the context keeps
 * the pointers until the next call (NULL mask and value: no group).  Mass is
 * no longer conserved when a group exchanges with the rest.                   */
MXE_API mxe_status mxe_set_reservoirs(mxe_ctx *ctx, const uint8_t *fix_x_mask_dev, const double *fix_x_value_dev,
                                      const uint8_t *fix_mu_mask_dev, const double *fix_mu_value_dev);

/* Event timing of the context's kernels, for profiling.  While enabled, every
 * kernel launch of the context is bracketed by CUDA events on the context's
 * stream and filed under its kernel class.  mxe_timing_read synchronises the
 * stream and returns, per class, the number of launches and their total
 * device time in ms; names receives the class names as consecutive
 * NUL-terminated strings of MXE_TIMING_NAME_LEN bytes each (caller-owned
 * host arrays of max_entries entries; *n_entries receives the count).
 * Reading clears the record.  Enabling allocates a small host-side pool of
 * CUDA events.                                                               */
#define MXE_TIMING_NAME_LEN 48
MXE_API mxe_status mxe_timing_enable(mxe_ctx *ctx, int32_t enable);
MXE_API mxe_status mxe_timing_read(mxe_ctx *ctx, int32_t max_entries, char *names, int64_t *counts,
                                   double *total_ms, int32_t *n_entries);

/* Euler step of the master equation that allocates no device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- a host framework whose caching allocator already holds
 * the card, a process under a fixed device-memory budget, or a
 * latency-critical loop that must not pay the device-wide synchronisation an
 * allocation can cause.  It computes exactly what mxe_diffuse_step computes,
 * without a context: the caller passes every input and output (device
 * pointers): x [S][n] in-out, T [n], mu_ex [S][n], and the bond CSR
 * (offsets [n+1], idx) that mxe_export_bonds returns.  Scratch lives in one
 * file-scope device array of MXE_NOALLOC_SCRATCH_DOUBLES doubles plus 256
 * bytes (about 4 MiB) that every device which loads the library holds until
 * the process exits; it bounds n to MXE_NOALLOC_MAX_SITES(S), and a larger n
 * (or S outside 1..2) returns MXE_ERR_ARG before any GPU work.  The first
 * call on a device looks up the array's device address with that device
 * current.  Every call ends by reading the step's status back and
 * synchronising its stream, so no call may be issued on a stream that is
 * being captured (the capture would be invalidated and the call returns
 * MXE_ERR_CUDA).  The address is
 * kept for the life of the process: a process that resets a device
 * (cudaDeviceReset) must not call this entry point on it again.  Every call shares
 * the array and it keeps the last call's contents: the flag words are cleared
 * at the start of each call and the per-site scratch is written before it is
 * read, but calls that overlap on the GPU (other streams, other host threads)
 * race on it.  Work is enqueued on cuda_stream (NULL: legacy default stream);
 * the call synchronises that stream and returns MXE_ERR_X_RANGE (x unchanged)
 * under the same rule as mxe_diffuse_step.                                    */
#define MXE_NOALLOC_SCRATCH_DOUBLES (1 << 19)
#define MXE_NOALLOC_MAX_SITES(S) ((int64_t)MXE_NOALLOC_SCRATCH_DOUBLES / (3 + 3 * (int64_t)(S)))
MXE_API mxe_status mxe_diffuse_step_noalloc(int64_t n, int32_t n_species, double *x_dev, const double *T_dev,
                                            const double *mu_ex_dev, const int32_t *bond_offsets_dev,
                                            const int32_t *bond_idx_dev, double dt, double nu0, double Qm,
                                            void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MXE_H */
