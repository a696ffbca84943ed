// relax.cu -- K5: FIRE relaxation of (q, sigma) at fixed x (Sec. 4, the
// equilibrium step of the staggered scheme; FIRE after Bitzek et al., PRL 97,
// 170201, 2006, replacing the paper's damped Verlet).
//
// One iteration is: density pass, gradient pass (eam.cu), then
//   k_fire_reduce : per fixed group of sites, P = f.v, |v|^2, |f|^2 partial sums;
//                   max_i max(|g_q,i|, |g_sigma,i|) by an atomic max on the bit
//                   patterns of non-negative doubles (order independent);
//   k_fire_logic  : one block sums the partials in a fixed order, tests
//                   convergence / the iteration cap, and advances dt, alpha, n_pos;
//   k_fire_update : v = (1 - alpha)(keep v + dt f) + alpha |v'| f / |f|,
//                   y += dt v, sigma kept in [sigma_lo, sigma_hi] (velocity
//                   zeroed at a bound), and the maxima the skin test needs.
// The sigma force is projected on [sigma_lo, sigma_hi] (zero where a bound
// blocks it) in the reduction and the update.
// |v'|^2 = keep (|v|^2 + 2 dt f.v) + dt^2 |f|^2 is formed from the partial sums,
// so one reduction per iteration suffices.  All kernels return at once while
// ctrl->halted is set, so a chunk of iterations can be enqueued blindly.
#include <cuda_runtime.h>

#include "mxe_internal.cuh"

namespace mxe {
namespace {

constexpr int kRedThreads = kReduceGroup / 4;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  unsigned long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
    b = y > b ? y : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(addr, b);
}

// force on sigma projected on the box [lo, hi]: zero where a bound blocks it
__device__ __forceinline__ double proj_fsig(double gs, double sigma, double lo, double hi) {
  const double f = -gs;
  if (sigma >= hi && f > 0.0) return 0.0;
  if (sigma <= lo && f < 0.0) return 0.0;
  return f;
}

__global__ void __launch_bounds__(kRedThreads) k_fire_reduce(const double* __restrict__ gq,
                                                             const double* __restrict__ gs,
                                                             const double* __restrict__ sigma,
                                                             const double* __restrict__ vq,
                                                             const double* __restrict__ vs, int64_t n,
                                                             int64_t ngroups, double* __restrict__ partials,
                                                             Ctrl* __restrict__ ctrl, int* __restrict__ flags) {
  if (ctrl->halted) return;
  __shared__ double sh[3][kRedThreads];
  const int tid = threadIdx.x;
  const double lo = ctrl->sigma_lo, hi = ctrl->sigma_hi;
  double P = 0.0, vv = 0.0, ff = 0.0, fm = 0.0;
  bool finite = true;
  for (int r = 0; r < 4; ++r) {
    int64_t i = blockIdx.x * (int64_t)kReduceGroup + r * kRedThreads + tid;
    if (i >= n) continue;
    double g0 = gq[i], g1 = gq[n + i], g2 = gq[2 * n + i];
    double f3 = proj_fsig(gs[i], sigma[i], lo, hi);
    double v0 = vq[i], v1 = vq[n + i], v2 = vq[2 * n + i], v3 = vs[i];
    P += -(g0 * v0 + g1 * v1 + g2 * v2) + f3 * v3;
    vv += v0 * v0 + v1 * v1 + v2 * v2 + v3 * v3;
    ff += g0 * g0 + g1 * g1 + g2 * g2 + f3 * f3;
    double gqn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    fm = fmax(fm, fmax(gqn, fabs(f3)));
    finite = finite && isfinite(g0) && isfinite(g1) && isfinite(g2) && isfinite(gs[i]);
  }
  sh[0][tid] = P;
  sh[1][tid] = vv;
  sh[2][tid] = ff;
  if (!finite) atomicOr(flags, kFlagNonfinite);
  atomic_max_nonneg(&ctrl->fmax_bits, finite ? fm : 0.0);
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid == 0)
    for (int c = 0; c < 3; ++c) partials[c * ngroups + blockIdx.x] = sh[c][0];
}

__global__ void __launch_bounds__(256) k_fire_logic(const double* __restrict__ partials, int64_t ngroups,
                                                    Ctrl* __restrict__ ctrl, const int* __restrict__ flags) {
  if (ctrl->halted) return;
  __shared__ double sh[3][256];
  const int tid = threadIdx.x;
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    for (int64_t gi = tid; gi < ngroups; gi += 256) v += partials[c * ngroups + gi];
    sh[c][tid] = v;
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid != 0) return;
  Ctrl& C = *ctrl;
  const double P = sh[0][0], vv = sh[1][0], ff = sh[2][0];
  const double fmx = __longlong_as_double((long long)C.fmax_bits);
  C.fmax = fmx;
  if (*flags & (kFlagGeometry | kFlagNonfinite)) {
    C.halted = 1;
    C.reason = kReasonError;
    return;
  }
  if (fmx <= C.ftol) {
    C.halted = 1;
    C.reason = kReasonConverged;
    return;
  }
  if (C.iter >= C.max_iter) {
    C.halted = 1;
    C.reason = kReasonMaxIter;
    return;
  }
  double keep = 1.0;
  if (C.iter > 0) {
    if (P > 0.0) {
      C.n_pos += 1;
      if (C.n_pos > C.n_min) {
        C.dt = fmin(C.dt * C.f_inc, C.dt_max);
        C.alpha = C.alpha * C.f_alpha;
      }
    } else {
      C.n_pos = 0;
      C.dt = C.dt * C.f_dec;
      C.alpha = C.alpha0;
      keep = 0.0;
    }
  }
  const double dt = C.dt;
  const double v2 = keep * (vv + 2.0 * dt * P) + dt * dt * ff;
  const double vnorm = sqrt(fmax(v2, 0.0));
  const double fnorm = sqrt(ff);
  C.keep = keep;
  C.mix = fnorm > 0.0 ? C.alpha * vnorm / fnorm : 0.0;
  C.one_minus_alpha = 1.0 - C.alpha;
  C.iter += 1;
  C.fmax_bits = 0ull;
  C.disp2_bits = 0ull;
  C.smax_bits = 0ull;
}

__global__ void __launch_bounds__(256) k_fire_update(double* __restrict__ q, double* __restrict__ sigma,
                                                     double* __restrict__ vq, double* __restrict__ vs,
                                                     const double* __restrict__ gq, const double* __restrict__ gs,
                                                     const double* __restrict__ q_build,
                                                     const int* __restrict__ abs_cell, int64_t n, DevGrid g,
                                                     float4* __restrict__ pos32, Ctrl* __restrict__ ctrl) {
  if (ctrl->halted) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double dt = ctrl->dt, keep = ctrl->keep, mix = ctrl->mix, oma = ctrl->one_minus_alpha;
  double disp2 = 0.0, sg = 0.0;
  if (i < n) {
    double p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double f = -gq[c * n + i];
      double v = keep * vq[c * n + i] + dt * f;
      v = oma * v + mix * f;
      vq[c * n + i] = v;
      const double qn = q[c * n + i] + dt * v;
      q[c * n + i] = qn;
      const double dq = qn - q_build[c * n + i];
      disp2 += dq * dq;
      p[c] = (float)(qn - (double)abs_cell[c * n + i] * g.h[c]);
    }
    const double lo = ctrl->sigma_lo, hi = ctrl->sigma_hi;
    const double f = proj_fsig(gs[i], sigma[i], lo, hi);
    double v = keep * vs[i] + dt * f;
    v = oma * v + mix * f;
    sg = sigma[i] + dt * v;
    if (sg < lo || sg > hi) {
      sg = sg < lo ? lo : hi;
      v = 0.0;
    }
    vs[i] = v;
    sigma[i] = sg;
    if (pos32) pos32[i] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)sg);
  }
  atomic_max_nonneg(&ctrl->disp2_bits, disp2);
  atomic_max_nonneg(&ctrl->smax_bits, sg);
}

}  // namespace

cudaError_t launch_fire_reduce(const double* gq, const double* gs, const double* sigma, const double* vq,
                               const double* vs, int64_t n, double* partials, Ctrl* ctrl, int* flags, cudaStream_t s) {
  int64_t ng = (n + kReduceGroup - 1) / kReduceGroup;
  if (ng < 1) ng = 1;
  k_fire_reduce<<<(unsigned)ng, kRedThreads, 0, s>>>(gq, gs, sigma, vq, vs, n, ng, partials, ctrl, flags);
  return cudaGetLastError();
}

cudaError_t launch_fire_logic(const double* partials, int64_t n, Ctrl* ctrl, int* flags, cudaStream_t s) {
  int64_t ng = (n + kReduceGroup - 1) / kReduceGroup;
  if (ng < 1) ng = 1;
  k_fire_logic<<<1, 256, 0, s>>>(partials, ng, ctrl, flags);
  return cudaGetLastError();
}

cudaError_t launch_fire_update(double* q, double* sigma, double* vq, double* vs, const double* gq,
                               const double* gs, const double* q_build, const int* abs_cell, int64_t n,
                               const DevGrid& g, float4* pos32, Ctrl* ctrl, cudaStream_t s) {
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks == 0) blocks = 1;
  k_fire_update<<<blocks, 256, 0, s>>>(q, sigma, vq, vs, gq, gs, q_build, abs_cell, n, g, pos32, ctrl);
  return cudaGetLastError();
}

}  // namespace mxe
