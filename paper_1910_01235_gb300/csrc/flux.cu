// flux.cu -- K4: one forward-Euler step of the master equation (Sec. 3.1,
// Eq. MassTransport with tau_r = 0; rate constant Eq. attempt_freq_mass; Euler
// integration as in Sec. 4), per species k over the nearest-neighbour bonds:
//   J_{i->j} = nu0 exp(-beta_i Qm) x_ik x_jv exp(beta_i (mu_ik - mu_jk))
//   x_ik' = x_ik + dt sum_j (J_{j->i} - J_{i->j})
// (mu = excess chemical potential, origin-site beta, vacancy fraction x_jv in
// place of (1 - x_j)).  Everything is FP64 in every precision mode: the rates
// depend on differences of neighbouring chemical potentials and the x budget
// of a whole run is 1e-7.
//
// k_flux_prep evaluates the per-site factors once: beta_i, D_i = nu0
// exp(-beta_i Qm), x_iv, and E_ik = exp(beta_i mu_ik) with its reciprocal.
// Across a bond whose two ends share the temperature, exp(beta (mu_i - mu_j))
// = E_i / E_j, so a hop costs four multiplications and no exponential; a bond
// between different temperatures, or an E outside the normal range, takes the
// exponential of the difference.  Each site gathers over its own bond row (no
// atomics, deterministic).  A bond's net exchange is always formed by the same
// function of the bond's canonical orientation (lower index first) with
// explicitly rounded operations, so site j obtains exactly the negation of
// what site i obtains: the two updates cancel and mass is conserved up to the
// rounding of the two row sums.
#include <cuda_runtime.h>

#include "mxe_internal.cuh"

namespace mxe {
namespace {

constexpr double kEMin = 1e-250, kEMax = 1e250;

// Reservoirs (Sec. 4, fix setchemicalpotential / setatomicfraction): a site
// of the chemical-potential group enters every rate with its held mu; a site of
// the molar-fraction group has x set to its held value after the step.
struct Reservoirs {
  const uint8_t* fix_x_mask;
  const double* fix_x_value;
  const uint8_t* fix_mu_mask;
  const double* fix_mu_value;
  double* mu_eff;  // [S][n] scratch: mu with the held values (when fix_mu_mask is set)
  // batches: the step of site i is dt * dt_sys[sys_of[i]] (both null: dt)
  const double* dt_sys;
  const int* sys_of;
  const Ctrl* gate;  // optional: nothing runs while gate->halted
};

template <int S>
__global__ void __launch_bounds__(256) k_flux_prep(const double* __restrict__ x, const double* __restrict__ T,
                                                   const double* __restrict__ mu, int64_t n, double nu0, double Qm,
                                                   double* __restrict__ fl, Reservoirs res) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || (res.gate && res.gate->halted)) return;
  const bool held = res.fix_mu_mask && res.fix_mu_mask[i];
  const double beta = 1.0 / (kKB * T[i]);
  double xv = 1.0;
#pragma unroll
  for (int k = 0; k < S; ++k) xv -= x[k * n + i];
  fl[i] = beta;
  fl[n + i] = nu0 * exp(-beta * Qm);
  fl[2 * n + i] = xv;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double m = held ? res.fix_mu_value[k * n + i] : mu[k * n + i];
    if (res.mu_eff) res.mu_eff[k * n + i] = m;
    const double E = exp(beta * m);
    fl[(3 + 2 * k) * n + i] = E;
    fl[(4 + 2 * k) * n + i] = 1.0 / E;
  }
}

struct Site {
  double T, beta, D, xv, x, mu, E, Einv;
};

// J_{a->b} for one species
__device__ __forceinline__ double hop(const Site& a, const Site& b, bool factorised) {
  const double e = factorised ? __dmul_rn(a.E, b.Einv) : exp(__dmul_rn(a.beta, __dsub_rn(a.mu, b.mu)));
  return __dmul_rn(__dmul_rn(__dmul_rn(a.D, a.x), b.xv), e);
}

__device__ __forceinline__ bool normal_E(const Site& s) { return s.E > kEMin && s.E < kEMax; }

template <int S>
__global__ void __launch_bounds__(256) k_flux(const double* __restrict__ x, const double* __restrict__ T,
                                              const double* __restrict__ mu_in, const double* __restrict__ fl,
                                              const int* __restrict__ bd_off, const int* __restrict__ bd_idx,
                                              int64_t n, double dt, double* __restrict__ x_new,
                                              int* __restrict__ flags, Reservoirs res) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || (res.gate && res.gate->halted)) return;
  const double* __restrict__ mu = res.mu_eff ? res.mu_eff : mu_in;
  Site si[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    si[k].T = T[i];
    si[k].beta = fl[i];
    si[k].D = fl[n + i];
    si[k].xv = fl[2 * n + i];
    si[k].x = x[k * n + i];
    si[k].mu = mu[k * n + i];
    si[k].E = fl[(3 + 2 * k) * n + i];
    si[k].Einv = fl[(4 + 2 * k) * n + i];
  }
  double rate[S];
#pragma unroll
  for (int k = 0; k < S; ++k) rate[k] = 0.0;
  const int beg = bd_off[i], end = bd_off[i + 1];
  for (int t = beg; t < end; ++t) {
    const int64_t j = bd_idx[t];
    const double Tj = T[j], bj = fl[j], Dj = fl[n + j], xvj = fl[2 * n + j];
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Site sj{Tj, bj, Dj, xvj, x[k * n + j], mu[k * n + j], fl[(3 + 2 * k) * n + j], fl[(4 + 2 * k) * n + j]};
      const bool fac = si[k].T == sj.T && normal_E(si[k]) && normal_E(sj);
      if (i < j) {
        const double net = __dsub_rn(hop(si[k], sj, fac), hop(sj, si[k], fac));
        rate[k] = __dsub_rn(rate[k], net);  // outflow from i
      } else {
        const double net = __dsub_rn(hop(sj, si[k], fac), hop(si[k], sj, fac));
        rate[k] = __dadd_rn(rate[k], net);  // inflow into i
      }
    }
  }
  double tot = 0.0;
  bool ok = true;
  const bool held_x = res.fix_x_mask && res.fix_x_mask[i];
  const double dti = res.dt_sys ? __dmul_rn(dt, res.dt_sys[res.sys_of[i]]) : dt;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double v = held_x ? res.fix_x_value[k * n + i] : __dadd_rn(si[k].x, __dmul_rn(dti, rate[k]));
    x_new[k * n + i] = v;
    tot += v;
    ok = ok && (v >= -kXTol);
  }
  ok = ok && (tot <= 1.0 + kXTol);
  if (!ok) atomicOr(flags, kFlagXRange);
}

__global__ void k_commit(double* __restrict__ x, const double* __restrict__ x_new, int64_t count,
                         const int* __restrict__ step_flags, int* __restrict__ flags, Ctrl* __restrict__ gate) {
  if (gate && gate->halted) return;
  const int sf = *step_flags;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (sf && lead) {
    atomicOr(flags, sf);  // keep the error for the status call
    if (gate && (sf & kFlagXRange)) {
      gate->reason = kReasonError;
      gate->halted = 1;
    }
  }
  if (sf & kFlagXRange) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count) x[t] = x_new[t];
  if (gate && lead) gate->phase = 1;
}

// ---------------------------------------------------------------- transport variants
// Host exchange (host >= 0): the exchange partner of species k != host is the
// host species (a binary alloy without vacancies, where x and 1 - x of Eq.
// MassTransport are two species): J^k_{a->b} = D_a x_ak x_b,host
// exp(beta_a (m_ak - m_bk)), m_k = mu_k - mu_host, and R_host = -sum R_k.
// Ballistic term (tau > 0, Eq. Transport): tau x'' + x' = R as x' = v,
// tau v' = R - v, integrated over the step with R held:
//   v' = R + (v - R) e,  x' = x + dt R + tau (v - R)(1 - e),  e = exp(-dt/tau);
// tau = 0 is the Euler step (v' = R).  Each bond's net exchange is formed in
// its canonical orientation with explicitly rounded operations, so the two
// ends cancel exactly, as in k_flux.
struct Ext {
  int host;
  double tau;
  const double* v;   // [S][n] rates at the start of the step (tau > 0)
  double* v_new;     // [S][n] (optional)
  const double* dt_sys;
  const int* sys_of;
};

__device__ __forceinline__ double ext_hop(double Da, double xak, double part_b, double beta_a, double ma, double mb) {
  return __dmul_rn(__dmul_rn(__dmul_rn(Da, xak), part_b), exp(__dmul_rn(beta_a, __dsub_rn(ma, mb))));
}

template <int S>
__device__ __forceinline__ double partner(const double* __restrict__ x, int64_t n, int64_t i, int host) {
  if (host >= 0) return x[host * n + i];
  double p = 1.0;
#pragma unroll
  for (int k = 0; k < S; ++k) p = __dsub_rn(p, x[k * n + i]);
  return p;
}

template <int S>
__global__ void __launch_bounds__(256) k_flux_ext(const double* __restrict__ x, const double* __restrict__ T,
                                                  const double* __restrict__ mu, const int* __restrict__ bd_off,
                                                  const int* __restrict__ bd_idx, int64_t n, double dt, double nu0,
                                                  double Qm, double* __restrict__ x_new, int* __restrict__ flags,
                                                  Ext e) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double bi = 1.0 / (kKB * T[i]);
  const double Di = nu0 * exp(-bi * Qm);
  const double pi = partner<S>(x, n, i, e.host);
  double m_i[S];
#pragma unroll
  for (int k = 0; k < S; ++k) m_i[k] = e.host >= 0 ? __dsub_rn(mu[k * n + i], mu[e.host * n + i]) : mu[k * n + i];
  double R[S];
#pragma unroll
  for (int k = 0; k < S; ++k) R[k] = 0.0;
  for (int t = bd_off[i]; t < bd_off[i + 1]; ++t) {
    const int64_t j = bd_idx[t];
    const double bj = 1.0 / (kKB * T[j]);
    const double Dj = nu0 * exp(-bj * Qm);
    const double pj = partner<S>(x, n, j, e.host);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      if (k == e.host) continue;
      const double m_j = e.host >= 0 ? __dsub_rn(mu[k * n + j], mu[e.host * n + j]) : mu[k * n + j];
      const double xi = x[k * n + i], xj = x[k * n + j];
      if (i < j) {  // net exchange i -> j, canonical orientation
        const double net = __dsub_rn(ext_hop(Di, xi, pj, bi, m_i[k], m_j), ext_hop(Dj, xj, pi, bj, m_j, m_i[k]));
        R[k] = __dsub_rn(R[k], net);
      } else {      // net exchange j -> i
        const double net = __dsub_rn(ext_hop(Dj, xj, pi, bj, m_j, m_i[k]), ext_hop(Di, xi, pj, bi, m_i[k], m_j));
        R[k] = __dadd_rn(R[k], net);
      }
    }
  }
  if (e.host >= 0) {
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < S; ++k)
      if (k != e.host) r = __dsub_rn(r, R[k]);
    R[e.host] = r;
  }
  const double dti = e.dt_sys ? dt * e.dt_sys[e.sys_of[i]] : dt;
  const double ex = e.tau > 0.0 ? exp(-dti / e.tau) : 0.0;
  double tot = 0.0;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int64_t a = k * n + i;
    double xv, vv;
    if (e.tau > 0.0) {
      const double dv = e.v[a] - R[k];
      xv = x[a] + dti * R[k] + e.tau * dv * (1.0 - ex);
      vv = R[k] + dv * ex;
    } else {
      xv = x[a] + dti * R[k];
      vv = R[k];
    }
    x_new[a] = xv;
    if (e.v_new) e.v_new[a] = vv;
    tot += xv;
    ok = ok && (xv >= -kXTol);
  }
  ok = ok && (tot <= 1.0 + kXTol);
  if (!ok) atomicOr(flags, kFlagXRange);
}

// commit x (and the rates) unless the step failed its range check
__global__ void k_commit_xv(double* __restrict__ x, const double* __restrict__ x_new, double* __restrict__ v,
                            const double* __restrict__ v_new, int64_t count, const int* __restrict__ step_flags,
                            int* __restrict__ flags) {
  const int sf = *step_flags;
  if (sf && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, sf);
  if (sf & kFlagXRange) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  x[t] = x_new[t];
  if (v) v[t] = v_new[t];
}

}  // namespace

int64_t flux_scratch_len(int64_t n, int S) { return (3 + 2 * (int64_t)S) * n; }

namespace {
template <int S>
void flux_kernels(unsigned blocks, const double* x, const double* T, const double* mu_ex, const int* bd_off,
                  const int* bd_idx, int64_t n, double dt, double nu0, double Qm, double* scratch, double* x_new,
                  int* flags, const Reservoirs& res, cudaStream_t s) {
  k_flux_prep<S><<<blocks, 256, 0, s>>>(x, T, mu_ex, n, nu0, Qm, scratch, res);
  k_flux<S><<<blocks, 256, 0, s>>>(x, T, mu_ex, scratch, bd_off, bd_idx, n, dt, x_new, flags, res);
}
}  // namespace

cudaError_t launch_flux_res(const double* x, const double* T, const double* mu_ex, const int* bd_off,
                            const int* bd_idx, int64_t n, int S, double dt, double nu0, double Qm, double* scratch,
                            double* x_new, int* flags, const uint8_t* fix_x_mask, const double* fix_x_value,
                            const uint8_t* fix_mu_mask, const double* fix_mu_value, double* mu_eff,
                            const double* dt_sys, const int* sys_of, Ctrl* gate, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if ((dt_sys == nullptr) != (sys_of == nullptr)) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  Reservoirs res{fix_x_mask, fix_x_value, fix_mu_mask, fix_mu_value, fix_mu_mask ? mu_eff : nullptr, dt_sys, sys_of, gate};
  switch (S) {
    case 1: flux_kernels<1>(blocks, x, T, mu_ex, bd_off, bd_idx, n, dt, nu0, Qm, scratch, x_new, flags, res, s); break;
    case 2: flux_kernels<2>(blocks, x, T, mu_ex, bd_off, bd_idx, n, dt, nu0, Qm, scratch, x_new, flags, res, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_flux(const double* x, const double* T, const double* mu_ex, const int* bd_off, const int* bd_idx,
                        int64_t n, int S, double dt, double nu0, double Qm, double* scratch, double* x_new,
                        int* flags, cudaStream_t s) {
  return launch_flux_res(x, T, mu_ex, bd_off, bd_idx, n, S, dt, nu0, Qm, scratch, x_new, flags, nullptr, nullptr,
                         nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, s);
}

cudaError_t launch_commit_x(double* x, const double* x_new, int64_t count, const int* step_flags, int* flags,
                            Ctrl* gate, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_commit<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(x, x_new, count, step_flags, flags, gate);
  return cudaGetLastError();
}

cudaError_t launch_transport_ext(double* x, const double* T, const double* mu_ex, const int* bd_off,
                                 const int* bd_idx, int64_t n, int S, double dt, double nu0, double Qm, int host,
                                 double tau, double* v, double* v_new, double* x_new, int* step_flags, int* flags,
                                 const double* dt_sys, const int* sys_of, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (host >= S || (tau > 0.0 && (!v || !v_new))) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  Ext e{host, tau, v, v ? v_new : nullptr, dt_sys, sys_of};
  switch (S) {
    case 1: k_flux_ext<1><<<blocks, 256, 0, s>>>(x, T, mu_ex, bd_off, bd_idx, n, dt, nu0, Qm, x_new, step_flags, e); break;
    case 2: k_flux_ext<2><<<blocks, 256, 0, s>>>(x, T, mu_ex, bd_off, bd_idx, n, dt, nu0, Qm, x_new, step_flags, e); break;
    default: return cudaErrorInvalidValue;
  }
  const int64_t count = (int64_t)S * n;
  k_commit_xv<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(x, x_new, v, v ? v_new : nullptr,
                                                             count, step_flags, flags);
  return cudaGetLastError();
}

}  // namespace mxe
