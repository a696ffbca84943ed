// deriv.cu -- K8: second-order quantities of the free energy and the
// vector-Jacobian product of the Euler step, for differentiating the
// staggered scheme (Sec. 4) with respect to the potential's parameters.
//
// Forward-mode (dual-number) differentiation of the density and gradient
// passes: every input of the pair sums carries a tangent -- the mean
// positions q, widths sigma and fractions x -- and every output of the
// gradient pass (dF/dq, dF/dsigma, mu^ex = dE_V/dx, and the sensitivities of
// E_V to each radial term's parameters) comes out with its directional
// derivative.  With the tangent (qdot, sdot, xdot) that is the Hessian of F
// (or E_V) times that vector; because the Hessian is symmetric the same
// products are the vector-Jacobian products the reverse sweep needs.
//
// Radial terms: every pair or density function of the potential is
// A exp(kappa - lambda r) S(r) (App. B.2 analytic forms; switch S of the
// cut-off).  The parameter sensitivities are dE_V/dc_u and dE_V/dlambda_u per
// distinct term u, with c = ln A + kappa: dF/dc = F and dF/dlambda = -r F.
// The caller maps them to its own parameters (chain rule on the host).
//
// Arithmetic is FP64 in every precision mode; one thread per site gathers
// over its own neighbour row (deterministic, no atomics except error flags).
#include <cuda_runtime.h>

#include "mxe_internal.cuh"

namespace mxe {
namespace {

struct Dual {
  double v, t;
};
__device__ __forceinline__ Dual D(double v) { return Dual{v, 0.0}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.v * b.t + a.t * b.v}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual{a * b.v, a * b.t}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual{a.v * b, a.t * b}; }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual{a.v + b, a.t}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual{q, (a.t - q * b.t) / b.v};
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) {
  a = a - b;
  return a;
}
__device__ __forceinline__ Dual dexp(Dual a) {
  const double e = exp(a.v);
  return Dual{e, e * a.t};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
  const double s = sqrt(a.v);
  return Dual{s, s > 0.0 ? a.t / (2.0 * s) : 0.0};
}

__device__ __forceinline__ Dual ld(const double* v, const double* t, int64_t k) {
  return Dual{v[k], t ? t[k] : 0.0};
}

// switch S(r) and dS/dr (quintic on [r_s, r_c])
__device__ __forceinline__ void dswitch(const DevPot& P, Dual r, Dual& S, Dual& dS) {
  if (r.v <= P.rs) {
    S = D(1.0);
    dS = D(0.0);
    return;
  }
  if (r.v >= P.rc) {
    S = D(0.0);
    dS = D(0.0);
    return;
  }
  const Dual t = (r + (-P.rs)) * P.inv_w;
  const Dual t2 = t * t;
  const Dual u = D(1.0) - t;
  S = D(1.0) + t2 * t * (D(-10.0) + t * (D(15.0) + t * D(-6.0)));
  dS = (-30.0 * P.inv_w) * (t2 * (u * u));
}

// A exp(kappa - lambda r): the raw exponential of one radial term
__device__ __forceinline__ Dual draw(const RadialFn& F, Dual r) { return F.A * dexp(D(F.kappa) - F.lambda * r); }

// minimum-image separation q_j - q_i (image chosen from the values)
__device__ __forceinline__ void dsep(const DevGrid& g, const TanArgs& A, int64_t i, int64_t j, Dual d[3]) {
  const int64_t n = A.n;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double dv = A.q[a * n + j] - A.q[a * n + i];
    const double shift = -g.L[a] * rint(dv * g.invL[a]);
    d[a] = ld(A.q, A.dq, a * n + j) - ld(A.q, A.dq, a * n + i) + shift;
  }
}

// ---------------------------------------------------------------- tangent density pass
template <int S>
__global__ void __launch_bounds__(128) k_tan_density(DevPot P, DevGrid g0, TanArgs A) {
  constexpr int NF = S * S;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t n = A.n;
  const DevGrid g = site_grid(g0, A.batch, i);
  Dual rb[S], ra[S];
#pragma unroll
  for (int k = 0; k < S; ++k) rb[k] = ra[k] = D(0.0);
  const Dual s_i = kSqrt6 * ld(A.sigma, A.dsigma, i);
  int bad = 0;
  for (int t = A.nb_off[i]; t < A.nb_off[i + 1]; ++t) {
    const int64_t j = A.nb_ent[t] & kIdxMask;
    Dual d[3];
    dsep(g, A, i, j, d);
    const Dual s_j = kSqrt6 * ld(A.sigma, A.dsigma, j);
    const Dual D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    bad |= D2.v < kRMin * kRMin;
    Dual fst[NF], fav[NF];
    {
      const Dual r = dsqrt(D2);
      Dual Sw, dS;
      dswitch(P, r, Sw, dS);
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        fst[v] = v < P.n_f ? draw(P.f[v], r) * Sw : D(0.0);
        fav[v] = D(0.0);
      }
    }
    for (int site = 0; site < 2; ++site) {
      const Dual s = site == 0 ? s_i : s_j;
      for (int a = 0; a < 3; ++a)
        for (int pm = -1; pm <= 1; pm += 2) {
          Dual r2 = D(0.0);
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const Dual c = b == a ? d[b] + (double)pm * s : d[b];
            r2 += c * c;
          }
          bad |= r2.v < kRMin * kRMin;
          const Dual r = dsqrt(r2);
          Dual Sw, dS;
          dswitch(P, r, Sw, dS);
#pragma unroll
          for (int v = 0; v < NF; ++v)
            if (v < P.n_f) fav[v] += draw(P.f[v], r) * Sw;
        }
    }
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int v = P.f_of[k][l];
        if (v < 0) continue;
        const Dual xl = ld(A.x, A.dx, l * n + j);
        rb[k] += xl * fst[v];
        ra[k] += xl * fav[v] * (1.0 / 12.0);
      }
  }
  int flag = bad ? kFlagGeometry : 0;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    Dual e = D(0.0), a = D(0.0), b = D(0.0);
    if (rb[k].v > kRhoMin) {
      const Dual sq = dsqrt(rb[k]);
      const double E = P.E[k];
      const Dual F = -E * sq;
      const Dual dF = D(-E) / (2.0 * sq);
      const Dual d2F = D(E) / (4.0 * rb[k] * sq);
      const Dual xk = ld(A.x, A.dx, k * n + i);
      e = F + dF * (ra[k] - rb[k]);
      a = xk * d2F * (ra[k] - rb[k]);
      b = xk * dF;
    } else {
      flag |= kFlagGeometry;
    }
    A.e_v[k * n + i] = e.v;
    A.e_t[k * n + i] = e.t;
    A.a_v[k * n + i] = a.v;
    A.a_t[k * n + i] = a.t;
    A.b_v[k * n + i] = b.v;
    A.b_t[k * n + i] = b.t;
  }
  if (flag) atomicOr(A.flags, flag);
}

// ---------------------------------------------------------------- tangent gradient pass
// Per site i, with the embedding coefficients a, b of every site from the
// density pass:
//   dF/dq_i     = sum_j d/dq_i [ <V_ij> + A_ij(r_ij) ]
//   dF/dsigma_i = sum_j d/dsigma_i <V_ij> - 3 kB T_i / sigma_i
//   mu_ik       = sum_j sum_l x_jl <phi_kl>_ij + e_i^k
//                 + sum_j sum_k' (a_j^k' f_k'k(r_ij) + b_j^k' <f_k'k>_ij)
//   dE_V/dc_u, dE_V/dlambda_u: the i-side share of every term u
// with V_ij(r) = sum_kl x_ik x_jl phi_kl + sum_kl (b_i^k x_jl + b_j^k x_il) f_kl
// over the 12 nodes and A_ij(r) = sum_kl (a_i^k x_jl + a_j^k x_il) f_kl at the
// static point (App. B.2 with the Taylor-linearised embedding).
template <int S>
__global__ void __launch_bounds__(128) k_tan_gradient(DevPot P, DevGrid g0, TanArgs A) {
  constexpr int NF = S * S;
  constexpr int NP = S * (S + 1) / 2;
  constexpr int NT = NP + NF;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int64_t n = A.n;
  const DevGrid g = site_grid(g0, A.batch, i);
  Dual gq[3] = {D(0.0), D(0.0), D(0.0)}, gs = D(0.0), mu[S];
  Dual thc[NT], thl[NT];
#pragma unroll
  for (int k = 0; k < S; ++k) mu[k] = D(0.0);
#pragma unroll
  for (int u = 0; u < NT; ++u) thc[u] = thl[u] = D(0.0);
  Dual xi[S], ai[S], bi[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    xi[k] = ld(A.x, A.dx, k * n + i);
    ai[k] = Dual{A.a_v[k * n + i], A.a_t[k * n + i]};
    bi[k] = Dual{A.b_v[k * n + i], A.b_t[k * n + i]};
  }
  const Dual s_i = kSqrt6 * ld(A.sigma, A.dsigma, i);
  int bad = 0;
  for (int t = A.nb_off[i]; t < A.nb_off[i + 1]; ++t) {
    const int64_t j = A.nb_ent[t] & kIdxMask;
    Dual d[3];
    dsep(g, A, i, j, d);
    const Dual s_j = kSqrt6 * ld(A.sigma, A.dsigma, j);
    Dual xj[S], aj[S], bj[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
      xj[k] = ld(A.x, A.dx, k * n + j);
      aj[k] = Dual{A.a_v[k * n + j], A.a_t[k * n + j]};
      bj[k] = Dual{A.b_v[k * n + j], A.b_t[k * n + j]};
    }
    // pair weights of the distinct terms: both sides (forces) and i-side only
    Dual wphi[NP], wfa[NF], wfs[NF], wfa_i[NF], wfs_i[NF];
#pragma unroll
    for (int u = 0; u < NP; ++u) wphi[u] = D(0.0);
#pragma unroll
    for (int v = 0; v < NF; ++v) wfa[v] = wfs[v] = wfa_i[v] = wfs_i[v] = D(0.0);
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int u = P.phi_of[k][l], v = P.f_of[k][l];
        if (u >= 0) wphi[u] += xi[k] * xj[l];
        if (v >= 0) {
          wfa[v] += bi[k] * xj[l] + bj[k] * xi[l];
          wfs[v] += ai[k] * xj[l] + aj[k] * xi[l];
          wfa_i[v] += bi[k] * xj[l];
          wfs_i[v] += ai[k] * xj[l];
        }
      }
    const Dual D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    bad |= D2.v < kRMin * kRMin;
    // static point: density terms
    Dual fst[NF];
    {
      const Dual r = dsqrt(D2);
      Dual Sw, dS;
      dswitch(P, r, Sw, dS);
      Dual Ap = D(0.0);  // dA/dr
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        fst[v] = D(0.0);
        if (v < P.n_f) {
          const Dual E = draw(P.f[v], r);
          fst[v] = E * Sw;
          Ap += wfs[v] * (E * (dS - P.f[v].lambda * Sw));
          thc[NP + v] += wfs_i[v] * fst[v];
          thl[NP + v] -= wfs_i[v] * (r * fst[v]);
        }
      }
      const Dual Apr = Ap / r;
#pragma unroll
      for (int c = 0; c < 3; ++c) gq[c] -= Apr * d[c];
    }
    // 12 nodes
    Dual aphi[NP], af[NF], aphir[NP], afr[NF];
#pragma unroll
    for (int u = 0; u < NP; ++u) aphi[u] = aphir[u] = D(0.0);
#pragma unroll
    for (int v = 0; v < NF; ++v) af[v] = afr[v] = D(0.0);
    for (int site = 0; site < 2; ++site) {
      const Dual s = site == 0 ? s_i : s_j;
      for (int a = 0; a < 3; ++a)
        for (int pm = -1; pm <= 1; pm += 2) {
          Dual dn[3];
#pragma unroll
          for (int b = 0; b < 3; ++b) dn[b] = b == a ? d[b] + (double)pm * s : d[b];
          const Dual r2 = dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2];
          bad |= r2.v < kRMin * kRMin;
          const Dual r = dsqrt(r2);
          Dual Sw, dS;
          dswitch(P, r, Sw, dS);
          Dual Vp = D(0.0);  // dV/dr
#pragma unroll
          for (int u = 0; u < NP; ++u)
            if (u < P.n_phi) {
              const Dual E = draw(P.phi[u], r);
              const Dual ES = E * Sw;
              aphi[u] += ES;
              aphir[u] -= r * ES;
              Vp += wphi[u] * (E * (dS - P.phi[u].lambda * Sw));
            }
#pragma unroll
          for (int v = 0; v < NF; ++v)
            if (v < P.n_f) {
              const Dual E = draw(P.f[v], r);
              const Dual ES = E * Sw;
              af[v] += ES;
              afr[v] -= r * ES;
              Vp += wfa[v] * (E * (dS - P.f[v].lambda * Sw));
            }
          const Dual w = (1.0 / 12.0) * (Vp / r);
#pragma unroll
          for (int c = 0; c < 3; ++c) gq[c] -= w * dn[c];
          if (site == 0) gs += (w * dn[a]) * ((double)pm * kSqrt6);
        }
    }
    const double inv12 = 1.0 / 12.0;
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      thc[u] += (0.5 * inv12) * (wphi[u] * aphi[u]);
      thl[u] += (0.5 * inv12) * (wphi[u] * aphir[u]);
    }
#pragma unroll
    for (int v = 0; v < NF; ++v) {
      thc[NP + v] += inv12 * (wfa_i[v] * af[v]);
      thl[NP + v] += inv12 * (wfa_i[v] * afr[v]);
    }
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Dual m = D(0.0);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int u = P.phi_of[k][l];
        if (u >= 0) m += xj[l] * aphi[u] * inv12;
      }
#pragma unroll
      for (int kp = 0; kp < S; ++kp) {
        const int v = P.f_of[kp][k];
        if (v >= 0) m += aj[kp] * fst[v] + bj[kp] * af[v] * inv12;
      }
      mu[k] += m;
    }
  }
#pragma unroll
  for (int k = 0; k < S; ++k) mu[k] += Dual{A.e_v[k * n + i], A.e_t[k * n + i]};
  gs -= D(3.0 * kKB * A.T[i]) / ld(A.sigma, A.dsigma, i);
  // outputs: values (optional) and tangents
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (A.gq_v) A.gq_v[c * n + i] = gq[c].v;
    if (A.gq_t) A.gq_t[c * n + i] = gq[c].t;
  }
  if (A.gs_v) A.gs_v[i] = gs.v;
  if (A.gs_t) A.gs_t[i] = gs.t;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    if (A.mu_v) A.mu_v[k * n + i] = mu[k].v;
    if (A.mu_t) A.mu_t[k * n + i] = mu[k].t;
  }
  // term sensitivities per site: columns c_0..c_{T-1}, lambda_0..lambda_{T-1},
  // terms numbered phi first, then f
  const int T = P.n_phi + P.n_f;
  for (int u = 0; u < T && A.th_v; ++u) {
    const int src = u < P.n_phi ? u : NP + (u - P.n_phi);
    A.th_v[(int64_t)u * n + i] = thc[src].v;
    A.th_t[(int64_t)u * n + i] = thc[src].t;
    A.th_v[(int64_t)(T + u) * n + i] = thl[src].v;
    A.th_t[(int64_t)(T + u) * n + i] = thl[src].t;
  }
  if (bad) atomicOr(A.flags, kFlagGeometry);
}

// ---------------------------------------------------------------- column sums
// out[c] = sum_i col[c][i] in a fixed order (one block per column)
__global__ void __launch_bounds__(256) k_col_sum(const double* __restrict__ col, int64_t n,
                                                 double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += col[(int64_t)c * n + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// ---------------------------------------------------------------- Euler-step VJP
// x' = x + dt R(x, mu): given the cotangent xbar' of x', accumulate
//   xbar = xbar' + (dt dR/dx)^T xbar',  mubar = (dt dR/dmu)^T xbar'
// per site over its bond row.  For the bond (i, j) and species k the net
// outflow N = J_ij - J_ji (J_ij = D_i x_ik x_jv exp(beta_i (mu_ik - mu_jk)))
// enters x_i' with -dt and x_j' with +dt, so dL/dN = dt (xbar'_jk - xbar'_ik);
// site i takes the derivatives of N with respect to its own variables.
template <int S>
__global__ void __launch_bounds__(128) k_flux_vjp(const double* __restrict__ x, const double* __restrict__ T,
                                                  const double* __restrict__ mu, const int* __restrict__ bd_off,
                                                  const int* __restrict__ bd_idx, int64_t n, double dt, double nu0,
                                                  double Qm, const double* __restrict__ dt_sys,
                                                  const int* __restrict__ sys_of, const double* __restrict__ xbar1,
                                                  double* __restrict__ xbar0, double* __restrict__ mubar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dti = dt_sys ? dt * dt_sys[sys_of[i]] : dt;
  const double bi = 1.0 / (kKB * T[i]);
  const double Di = nu0 * exp(-bi * Qm);
  double xvi = 1.0;
#pragma unroll
  for (int k = 0; k < S; ++k) xvi -= x[k * n + i];
  double ax[S], am[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    ax[k] = xbar1[k * n + i];
    am[k] = 0.0;
  }
  for (int t = bd_off[i]; t < bd_off[i + 1]; ++t) {
    const int64_t j = bd_idx[t];
    const double bj = 1.0 / (kKB * T[j]);
    const double Dj = nu0 * exp(-bj * Qm);
    double xvj = 1.0;
#pragma unroll
    for (int k = 0; k < S; ++k) xvj -= x[k * n + j];
    double into_v = 0.0;  // d/dx_ik' of N through x_iv, summed over species
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double dmu = mu[k * n + i] - mu[k * n + j];
      const double eij = exp(bi * dmu), eji = exp(-bj * dmu);
      const double Jij = Di * x[k * n + i] * xvj * eij;
      const double Jji = Dj * x[k * n + j] * xvi * eji;
      const double c = dti * (xbar1[k * n + j] - xbar1[k * n + i]);
      ax[k] += c * Di * xvj * eij;
      into_v += c * Dj * x[k * n + j] * eji;
      am[k] += c * (bi * Jij + bj * Jji);
    }
#pragma unroll
    for (int k = 0; k < S; ++k) ax[k] += into_v;
  }
#pragma unroll
  for (int k = 0; k < S; ++k) {
    xbar0[k * n + i] = ax[k];
    mubar[k * n + i] = am[k];
  }
}

// ---------------------------------------------------------------- vectors
__global__ void k_dot_partials(const double* __restrict__ a, const double* __restrict__ b, int64_t len,
                               double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  const int64_t base = blockIdx.x * (int64_t)kReduceGroup;
  for (int r = threadIdx.x; r < kReduceGroup; r += 256) {
    const int64_t i = base + r;
    if (i < len) s += a[i] * b[i];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double alpha, double beta,
                        int64_t len) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < len) y[i] = alpha * x[i] + beta * y[i];
}

template <int S>
cudaError_t tangent_t(const DevPot& P, const DevGrid& g, const TanArgs& A, cudaStream_t s) {
  const unsigned blocks = (unsigned)((A.n + 127) / 128);
  k_tan_density<S><<<blocks, 128, 0, s>>>(P, g, A);
  k_tan_gradient<S><<<blocks, 128, 0, s>>>(P, g, A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tangent(const DevPot& P, const DevGrid& g, const TanArgs& A, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  switch (P.S) {
    case 1: return tangent_t<1>(P, g, A, s);
    case 2: return tangent_t<2>(P, g, A, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col_sum(const double* col, int ncol, int64_t n, double* out, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  k_col_sum<<<(unsigned)ncol, 256, 0, s>>>(col, n, out);
  return cudaGetLastError();
}

cudaError_t launch_flux_vjp(const double* x, const double* T, const double* mu, const int* bd_off, const int* bd_idx,
                            int64_t n, int S, double dt, double nu0, double Qm, const double* dt_sys,
                            const int* sys_of, const double* xbar1, double* xbar0, double* mubar, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  switch (S) {
    case 1:
      k_flux_vjp<1><<<blocks, 128, 0, s>>>(x, T, mu, bd_off, bd_idx, n, dt, nu0, Qm, dt_sys, sys_of, xbar1, xbar0, mubar);
      break;
    case 2:
      k_flux_vjp<2><<<blocks, 128, 0, s>>>(x, T, mu, bd_off, bd_idx, n, dt, nu0, Qm, dt_sys, sys_of, xbar1, xbar0, mubar);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int64_t dot_partials_len(int64_t len) { return (len + kReduceGroup - 1) / kReduceGroup + 1; }

cudaError_t launch_dot(const double* a, const double* b, int64_t len, double* part, double* out, cudaStream_t s) {
  const int64_t ng = (len + kReduceGroup - 1) / kReduceGroup;
  if (ng == 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
  k_dot_partials<<<(unsigned)ng, 256, 0, s>>>(a, b, len, part);
  k_col_sum<<<1, 256, 0, s>>>(part, ng, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* y, const double* x, double alpha, double beta, int64_t len, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  k_axpby<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(y, x, alpha, beta, len);
  return cudaGetLastError();
}

}  // namespace mxe
