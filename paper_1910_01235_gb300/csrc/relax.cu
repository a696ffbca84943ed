// relax.cu -- K5: FIRE relaxation of (q, sigma) at fixed x (Sec. 4, the
// equilibrium step of the staggered scheme; FIRE after Bitzek et al., PRL 97,
// 170201, 2006, replacing the paper's damped Verlet).
//
// One iteration is: density pass, gradient pass (eam.cu), then
//   k_fire_reduce : per fixed group of sites, P = f.v, |v|^2, |f|^2 partial sums;
//                   max_i max(|g_q,i|, |g_sigma,i|) by an atomic max on the bit
//                   patterns of non-negative doubles (order independent); the
//                   launch's last block then sums the partials in a fixed
//                   order, tests convergence / the iteration cap, and advances
//                   dt, alpha, n_pos;
//   k_fire_update : v = (1 - alpha)(keep v + dt f) + alpha |v'| f / |f|,
//                   y += dt v, sigma kept in [sigma_lo, sigma_hi] (velocity
//                   zeroed at a bound), and the maxima the skin test needs;
//                   the launch's last block then tests the rebuild criterion,
//                   so a halted next evaluation returns at once.
// The sigma force is projected on [sigma_lo, sigma_hi] (zero where a bound
// blocks it) in the reduction and the update.
// |v'|^2 = keep (|v|^2 + 2 dt f.v) + dt^2 |f|^2 is formed from the partial sums,
// so one reduction per iteration suffices.  All kernels return at once while
// ctrl->halted is set, so a chunk of iterations can be enqueued blindly.
#include <cuda_runtime.h>

#include "mxe_internal.cuh"

namespace mxe {
namespace {

// FIRE reduction: one site per thread, kFireGroup sites per partial sum
// (many small blocks keep the SMs busy on a pass this short)
constexpr int kRedThreads = kFireGroup;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  unsigned long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
    b = y > b ? y : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(addr, b);
}

// The block's maximum of non-negative doubles, then one atomic per block (a
// global atomic per warp serialises thousands of updates of one word).
// Every thread of the block must call it.
__device__ __forceinline__ void block_max_bits(unsigned long long* addr, unsigned long long b) {
  __shared__ unsigned long long s_max;
  if (threadIdx.x == 0) s_max = 0ull;
  __syncthreads();
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
    b = y > b ? y : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(&s_max, b);
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(addr, s_max);
}
__device__ __forceinline__ void block_max_nonneg(unsigned long long* addr, double v) {
  block_max_bits(addr, (unsigned long long)__double_as_longlong(v));
}

// Tests on bit patterns (integer instructions; GB300's FP64 pipe is narrow):
// finiteness, and the projection below for positive sigma, lo, hi, whose order
// is that of their bits.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}
__device__ __forceinline__ double proj_fsig_bits(double gs, double sigma, long long lo_b, long long hi_b) {
  const double f = -gs;
  const long long fb = __double_as_longlong(f), sb = __double_as_longlong(sigma);
  if (sb >= hi_b && fb > 0) return 0.0;                              // f > 0
  if (sb <= lo_b && fb < 0 && fb != (long long)0x8000000000000000ull) return 0.0;  // f < 0 (not -0)
  return f;
}

// force on sigma projected on the box [lo, hi]: zero where a bound blocks it
__device__ __forceinline__ double proj_fsig(double gs, double sigma, double lo, double hi) {
  const double f = -gs;
  if (sigma >= hi && f > 0.0) return 0.0;
  if (sigma <= lo && f < 0.0) return 0.0;
  return f;
}

// The FIRE logic of one iteration, run by the last block of k_fire_reduce
// (blockDim = kRedThreads): the partial sums in a fixed order (the same
// result whichever block runs it), the convergence and iteration-cap tests,
// and the advance of dt, alpha, n_pos.  Partials, the force maximum and the
// flags are written by other blocks of the same launch, so they are read past
// L1 (__ldcg).
__device__ void fire_logic_block(const double* __restrict__ partials, int64_t ngroups, Ctrl* __restrict__ ctrl,
                                 const int* __restrict__ flags, double (*sh)[kRedThreads]) {
  const int tid = threadIdx.x;
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    for (int64_t gi = tid; gi < ngroups; gi += kRedThreads) v += __ldcg(&partials[c * ngroups + gi]);
    sh[c][tid] = v;
  }
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid != 0) return;
  Ctrl& C = *ctrl;
  const double P = sh[0][0], vv = sh[1][0], ff = sh[2][0];
  const double fmx = sqrt(__longlong_as_double((long long)__ldcg(&C.fmax_bits)));
  C.fmax = fmx;
  if (__ldcg(flags) & (kFlagGeometry | kFlagNonfinite)) {
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

// Partial sums per group of kFireGroup sites; the last block to finish
// (a ticket counted in the control block) then runs the logic, so an
// iteration needs no separate single-block launch.
__global__ void __launch_bounds__(kRedThreads) k_fire_reduce(const double* __restrict__ gq,
                                                             const double* __restrict__ gs,
                                                             const double* __restrict__ sigma,
                                                             const double* __restrict__ vq,
                                                             const double* __restrict__ vs, int64_t n,
                                                             int64_t ngroups, double* __restrict__ partials,
                                                             Ctrl* __restrict__ ctrl, int* __restrict__ flags) {
  pdl_wait();
  pdl_trigger();
  if (ctrl->halted) return;  // the same for every block: nothing in this launch changes it before the logic
  __shared__ double sh[3][kRedThreads];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const long long lo_b = __double_as_longlong(ctrl->sigma_lo), hi_b = __double_as_longlong(ctrl->sigma_hi);
  double P = 0.0, vv = 0.0, ff = 0.0;
  unsigned long long fmb = 0ull;
  bool finite = true;
  const int64_t i = blockIdx.x * (int64_t)kFireGroup + tid;
  if (i < n) {
    const double g0 = gq[i], g1 = gq[n + i], g2 = gq[2 * n + i], gsi = gs[i];
    const double f3 = proj_fsig_bits(gsi, sigma[i], lo_b, hi_b);
    const double v0 = vq[i], v1 = vq[n + i], v2 = vq[2 * n + i], v3 = vs[i];
    P = -(g0 * v0 + g1 * v1 + g2 * v2) + f3 * v3;
    vv = v0 * v0 + v1 * v1 + v2 * v2 + v3 * v3;
    const double gg = g0 * g0 + g1 * g1 + g2 * g2, f33 = f3 * f3;
    ff = gg + f33;
    finite = finite_bits(g0) && finite_bits(g1) && finite_bits(g2) && finite_bits(gsi);
    // the largest squared force component norm (maximum of non-negative
    // doubles = maximum of their bits); its square root is taken once, by
    // the logic (sqrt is monotone and correctly rounded, so sqrt(max) ==
    // max(sqrt)); a site with a non-finite gradient enters as 0 (flagged)
    const unsigned long long a = __double_as_longlong(gg), b = __double_as_longlong(f33);
    fmb = finite ? (a > b ? a : b) : 0ull;
  }
  sh[0][tid] = P;
  sh[1][tid] = vv;
  sh[2][tid] = ff;
  if (!finite) atomicOr(flags, kFlagNonfinite);
  block_max_bits(&ctrl->fmax_bits, fmb);
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    for (int c = 0; c < 3; ++c) partials[c * ngroups + blockIdx.x] = sh[c][0];
    __threadfence();  // partials, flags and the maximum before the ticket
    s_last = atomicAdd(&ctrl->red_ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  fire_logic_block(partials, ngroups, ctrl, flags, sh);
  if (tid == 0) ctrl->red_ticket = 0u;
}

// One FIRE update of site i with the given scalars; returns |q - q_build|^2 and sigma.
__device__ __forceinline__ void fire_site(double* __restrict__ q, double* __restrict__ sigma, double* __restrict__ vq,
                                          double* __restrict__ vs, const double* __restrict__ gq,
                                          const double* __restrict__ gs, const double* __restrict__ q_build,
                                          const int* __restrict__ abs_cell, int64_t n, int64_t i, const DevGrid& g,
                                          float4* __restrict__ pos32, double dt, double keep, double mix, double oma,
                                          double lo, double hi, double& disp2, double& sg) {
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
  const double f = proj_fsig_bits(gs[i], sigma[i], __double_as_longlong(lo), __double_as_longlong(hi));
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

__global__ void __launch_bounds__(256) k_fire_update(double* __restrict__ q, double* __restrict__ sigma,
                                                     double* __restrict__ vq, double* __restrict__ vs,
                                                     const double* __restrict__ gq, const double* __restrict__ gs,
                                                     const double* __restrict__ q_build,
                                                     const int* __restrict__ abs_cell, int64_t n, DevGrid g0,
                                                     Batch B, float4* __restrict__ pos32, Ctrl* __restrict__ ctrl) {
  pdl_wait();
  pdl_trigger();
  if (ctrl->halted) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double dt = ctrl->dt, keep = ctrl->keep, mix = ctrl->mix, oma = ctrl->one_minus_alpha;
  double disp2 = 0.0, sg = 0.0;
  if (i < n) {
    const DevGrid g = site_grid(g0, B, i);
    fire_site(q, sigma, vq, vs, gq, gs, q_build, abs_cell, n, i, g, pos32, dt, keep, mix, oma, ctrl->sigma_lo,
              ctrl->sigma_hi, disp2, sg);
  }
  block_max_nonneg(&ctrl->disp2_bits, disp2);
  block_max_nonneg(&ctrl->smax_bits, sg);
  // The last block to finish (a ticket in the control block) tests the
  // rebuild criterion on this update's maxima, so that every kernel of the
  // next evaluation returns at once when the lists must be rebuilt (the same
  // test as the first pass's, which then finds the flag already set).
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl->red_ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    ctrl->red_ticket = 0u;
    const double disp = sqrt(__longlong_as_double((long long)__ldcg(&ctrl->disp2_bits)));
    const double smax = __longlong_as_double((long long)__ldcg(&ctrl->smax_bits));
    if (2.0 * disp + kSqrt6 * (smax - ctrl->sigma_max_build) > ctrl->skin) {
      ctrl->reason = kReasonRebuild;
      ctrl->halted = 1;
    }
  }
}

// ---------------------------------------------------------------- batches
__global__ void __launch_bounds__(256) k_fire_seg_reduce(const double* __restrict__ gq,
                                                         const double* __restrict__ gs,
                                                         const double* __restrict__ sigma,
                                                         const double* __restrict__ vq,
                                                         const double* __restrict__ vs, int64_t n, Batch B,
                                                         SysFire* __restrict__ sf, Ctrl* __restrict__ ctrl,
                                                         int* __restrict__ flags) {
  if (ctrl->halted) return;
  const int sys = blockIdx.x;
  if (sf[sys].halted) return;
  __shared__ double sh[4][256];
  const int tid = threadIdx.x;
  const double lo = ctrl->sigma_lo, hi = ctrl->sigma_hi;
  double P = 0.0, vv = 0.0, ff = 0.0, fm = 0.0;
  bool finite = true;
  for (int64_t i = B.sys_off[sys] + tid; i < B.sys_off[sys + 1]; i += 256) {
    const double g0 = gq[i], g1 = gq[n + i], g2 = gq[2 * n + i];
    const double f3 = proj_fsig(gs[i], sigma[i], lo, hi);
    const double v0 = vq[i], v1 = vq[n + i], v2 = vq[2 * n + i], v3 = vs[i];
    P += -(g0 * v0 + g1 * v1 + g2 * v2) + f3 * v3;
    vv += v0 * v0 + v1 * v1 + v2 * v2 + v3 * v3;
    ff += g0 * g0 + g1 * g1 + g2 * g2 + f3 * f3;
    fm = fmax(fm, fmax(g0 * g0 + g1 * g1 + g2 * g2, f3 * f3));  // squared; one sqrt per system below
    finite = finite && isfinite(g0) && isfinite(g1) && isfinite(g2) && isfinite(gs[i]);
  }
  if (!finite) atomicOr(flags, kFlagNonfinite);
  sh[0][tid] = P;
  sh[1][tid] = vv;
  sh[2][tid] = ff;
  sh[3][tid] = fm;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) {
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
      sh[3][tid] = fmax(sh[3][tid], sh[3][tid + w]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    sf[sys].P = sh[0][0];
    sf[sys].vv = sh[1][0];
    sf[sys].ff = sh[2][0];
    sf[sys].fmax = sqrt(sh[3][0]);
  }
}

__global__ void __launch_bounds__(256) k_fire_seg_logic(SysFire* __restrict__ sf, int nsys, Ctrl* __restrict__ ctrl,
                                                        const int* __restrict__ flags) {
  if (ctrl->halted) return;
  __shared__ int active[256];
  const Ctrl& C = *ctrl;
  if (*flags & (kFlagGeometry | kFlagNonfinite)) {
    if (threadIdx.x == 0) {
      ctrl->halted = 1;
      ctrl->reason = kReasonError;
    }
    return;
  }
  int act = 0;
  for (int s = threadIdx.x; s < nsys; s += 256) {
    SysFire& F = sf[s];
    if (F.halted) continue;
    if (F.fmax <= C.ftol) {
      F.halted = 1;
      F.reason = kReasonConverged;
      continue;
    }
    if (F.iter >= C.max_iter) {
      F.halted = 1;
      F.reason = kReasonMaxIter;
      continue;
    }
    double keep = 1.0;
    if (F.iter > 0) {
      if (F.P > 0.0) {
        F.n_pos += 1;
        if (F.n_pos > C.n_min) {
          F.dt = fmin(F.dt * C.f_inc, C.dt_max);
          F.alpha = F.alpha * C.f_alpha;
        }
      } else {
        F.n_pos = 0;
        F.dt = F.dt * C.f_dec;
        F.alpha = C.alpha0;
        keep = 0.0;
      }
    }
    const double dt = F.dt;
    const double v2 = keep * (F.vv + 2.0 * dt * F.P) + dt * dt * F.ff;
    const double fnorm = sqrt(F.ff);
    F.keep = keep;
    F.mix = fnorm > 0.0 ? F.alpha * sqrt(fmax(v2, 0.0)) / fnorm : 0.0;
    F.one_minus_alpha = 1.0 - F.alpha;
    F.iter += 1;
    act += 1;
  }
  active[threadIdx.x] = act;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) active[threadIdx.x] += active[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ctrl& G = *ctrl;
    if (active[0] == 0) {
      G.halted = 1;  // the maxima of the last update stay for the skin test
      G.reason = kReasonAllDone;
    } else {
      G.iter += 1;  // updates of the longest-running system
      G.disp2_bits = 0ull;
      G.smax_bits = 0ull;
    }
  }
}

__global__ void __launch_bounds__(256) k_fire_seg_update(double* __restrict__ q, double* __restrict__ sigma,
                                                         double* __restrict__ vq, double* __restrict__ vs,
                                                         const double* __restrict__ gq,
                                                         const double* __restrict__ gs,
                                                         const double* __restrict__ q_build,
                                                         const int* __restrict__ abs_cell, int64_t n, DevGrid g0,
                                                         Batch B, const SysFire* __restrict__ sf,
                                                         float4* __restrict__ pos32, Ctrl* __restrict__ ctrl) {
  if (ctrl->halted) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double disp2 = 0.0, sg = 0.0;
  if (i < n) {
    const SysFire& F = sf[B.sys_of[i]];
    if (!F.halted) {
      const DevGrid g = site_grid(g0, B, i);
      fire_site(q, sigma, vq, vs, gq, gs, q_build, abs_cell, n, i, g, pos32, F.dt, F.keep, F.mix, F.one_minus_alpha,
                ctrl->sigma_lo, ctrl->sigma_hi, disp2, sg);
    } else {  // a stopped system still counts in the skin test
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double dq = q[c * n + i] - q_build[c * n + i];
        disp2 += dq * dq;
      }
      sg = sigma[i];
    }
  }
  atomic_max_nonneg(&ctrl->disp2_bits, disp2);
  atomic_max_nonneg(&ctrl->smax_bits, sg);
}

__global__ void k_fire_seg_init(SysFire* __restrict__ sf, int nsys, double dt0, double alpha0,
                                const Ctrl* __restrict__ gate) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || (gate && gate->halted)) return;
  SysFire F;
  F.halted = 0;
  F.reason = kReasonNone;
  F.iter = 0;
  F.n_pos = 0;
  F.dt = dt0;
  F.alpha = alpha0;
  F.keep = F.mix = F.one_minus_alpha = F.fmax = 0.0;
  F.P = F.vv = F.ff = 0.0;
  sf[s] = F;
}

// ------------------------------------------------------- staggered steps in a graph
// A stop for a rebuild or an error stays until the host clears it: every
// later kernel of the captured steps then returns at once.
__device__ __forceinline__ bool run_stopped(const Ctrl& C) {
  return C.halted && (C.reason == kReasonRebuild || C.reason == kReasonError);
}

__global__ void k_step_begin(Ctrl* __restrict__ ctrl, double dt0, double alpha0) {
  Ctrl& C = *ctrl;
  if (run_stopped(C)) return;
  C.halted = 0;
  C.reason = kReasonNone;
  C.iter = 0;
  C.n_pos = 0;
  C.dt = dt0;
  C.alpha = alpha0;
  C.fmax_bits = 0ull;
  C.phase = 0;
}

__global__ void k_step_end(Ctrl* __restrict__ ctrl) {
  Ctrl& C = *ctrl;
  if (run_stopped(C)) return;
  C.steps += 1;
  C.phase = 0;
}

// The staggered run replayed on the device: after each step the condition of
// the graph's while node is set to repeat the step while steps remain, no
// stop (rebuild or error) is pending and the body has run fewer than `cap`
// times, so the loop always ends.  loop[0]: bodies run, loop[1]: the step
// count to reach, loop[2]: the cap (set by the host before each launch).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const Ctrl* __restrict__ ctrl, int* __restrict__ loop) {
  const int runs = loop[0] + 1;
  loop[0] = runs;
  const bool more = ctrl->steps < loop[1] && !run_stopped(*ctrl) && runs < loop[2];
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_fire_zero_v(double* __restrict__ vq, double* __restrict__ vs, int64_t n,
                                                     const Ctrl* __restrict__ gate) {
  if (gate->halted) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  vq[i] = 0.0;
  vq[n + i] = 0.0;
  vq[2 * n + i] = 0.0;
  vs[i] = 0.0;
}

}  // namespace

cudaError_t launch_step_begin(Ctrl* ctrl, double dt0, double alpha0, cudaStream_t s) {
  k_step_begin<<<1, 1, 0, s>>>(ctrl, dt0, alpha0);
  return cudaGetLastError();
}

cudaError_t launch_step_end(Ctrl* ctrl, cudaStream_t s) {
  k_step_end<<<1, 1, 0, s>>>(ctrl);
  return cudaGetLastError();
}

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const Ctrl* ctrl, int* loop, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(h, ctrl, loop);
  return cudaGetLastError();
}

cudaError_t launch_fire_zero_v(double* vq, double* vs, int64_t n, const Ctrl* gate, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_fire_zero_v<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vq, vs, n, gate);
  return cudaGetLastError();
}

cudaError_t launch_fire_reduce(const double* gq, const double* gs, const double* sigma, const double* vq,
                               const double* vs, int64_t n, double* partials, Ctrl* ctrl, int* flags, cudaStream_t s) {
  int64_t ng = (n + kFireGroup - 1) / kFireGroup;
  if (ng < 1) ng = 1;
  return launch_pdl(k_fire_reduce, dim3((unsigned)ng), dim3(kRedThreads), 0, s, gq, gs, sigma, vq, vs, n, ng, partials,
                    ctrl, flags);
}

cudaError_t launch_fire_update(double* q, double* sigma, double* vq, double* vs, const double* gq,
                               const double* gs, const double* q_build, const int* abs_cell, int64_t n,
                               const DevGrid& g, const Batch& B, float4* pos32, Ctrl* ctrl, cudaStream_t s) {
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks == 0) blocks = 1;
  return launch_pdl(k_fire_update, dim3(blocks), dim3(256), 0, s, q, sigma, vq, vs, gq, gs, q_build, abs_cell, n, g, B,
                    pos32, ctrl);
}

cudaError_t launch_fire_seg_reduce(const double* gq, const double* gs, const double* sigma, const double* vq,
                                   const double* vs, int64_t n, const Batch& B, SysFire* sf, Ctrl* ctrl, int* flags,
                                   cudaStream_t s) {
  if (B.nsys <= 0) return cudaErrorInvalidValue;
  k_fire_seg_reduce<<<(unsigned)B.nsys, 256, 0, s>>>(gq, gs, sigma, vq, vs, n, B, sf, ctrl, flags);
  return cudaGetLastError();
}

cudaError_t launch_fire_seg_logic(SysFire* sf, int nsys, Ctrl* ctrl, const int* flags, cudaStream_t s) {
  k_fire_seg_logic<<<1, 256, 0, s>>>(sf, nsys, ctrl, flags);
  return cudaGetLastError();
}

cudaError_t launch_fire_seg_update(double* q, double* sigma, double* vq, double* vs, const double* gq,
                                   const double* gs, const double* q_build, const int* abs_cell, int64_t n,
                                   const DevGrid& g, const Batch& B, const SysFire* sf, float4* pos32, Ctrl* ctrl,
                                   cudaStream_t s) {
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks == 0) blocks = 1;
  k_fire_seg_update<<<blocks, 256, 0, s>>>(q, sigma, vq, vs, gq, gs, q_build, abs_cell, n, g, B, sf, pos32, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_fire_seg_init(SysFire* sf, int nsys, double dt0, double alpha0, const Ctrl* gate, cudaStream_t s) {
  if (nsys <= 0) return cudaSuccess;
  k_fire_seg_init<<<(unsigned)((nsys + 255) / 256), 256, 0, s>>>(sf, nsys, dt0, alpha0, gate);
  return cudaGetLastError();
}

}  // namespace mxe
