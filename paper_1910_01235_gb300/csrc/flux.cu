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

}  // namespace mxe
