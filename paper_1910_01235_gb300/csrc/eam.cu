// eam.cu -- K7 pack, K2 density/embedding pass, K3 gradient pass, K6 energy reduction.
//
// Thermalized EAM (App. B.2) averaged with the third-degree rule of App. A:
// for a pair (i, j) the 12 nodes move one of the two sites by +-sqrt(6) sigma
// along one axis, each with weight 1/12; the static point is the mean
// separation.  Embedding: Taylor-linearised about the static density
// (Eq. F_taylor_mxe), so pass 1 needs rho_bar and <rho> of every site and pass
// 2 needs the per-site coefficients a = x F''(rho_bar)(<rho> - rho_bar) and
// b = x F'(rho_bar) of every neighbour.
//
// Work split: a team of NL consecutive lanes owns one site and strides over
// its neighbour row; each lane evaluates the 13 points of a pair unrolled in
// registers; the team reduces its per-site sums with warp shuffles.  The
// neighbour rows are contiguous (CSR), so a team's index loads coalesce, and
// the neighbours' packed float4 records are L1/L2-resident gathers.
//
// Precision variants (template PREC):
//   0  FP64 everywhere.
//   1  node arithmetic in FP32 from cell-relative FP32 positions (the pair
//      separation is rebuilt from the image code, never from absolute FP32
//      coordinates); each pair's 13-node partial sums are added into FP64
//      per-site accumulators.
//   2  as 1, with the per-site sums carried as float-float pairs (TwoSum).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ff.cuh"
#include "mxe_internal.cuh"

namespace mxe {

__constant__ FFExpTable c_exp_table;  // 2^(j/32) as float pairs

cudaError_t init_ff_exp_table() {
  FFExpTable T;
  for (int j = 0; j < 32; ++j) {
    const double v = std::exp2((double)j / 32.0);
    T.hi[j] = (float)v;
    T.lo[j] = (float)(v - (double)T.hi[j]);
  }
  return cudaMemcpyToSymbol(c_exp_table, &T, sizeof(T));
}

namespace {

// ---------------------------------------------------------------- accumulators
struct AccD {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(float x) { v += (double)x; }
  __device__ __forceinline__ void add(ff x) { v += ff_to_double(x); }
  __device__ __forceinline__ double get() const { return v; }
  __device__ __forceinline__ float2 get_pair() const {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
  __device__ __forceinline__ void team_reduce(int nl) {
    for (int o = nl >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
};

// Unevaluated sum hi + lo of floats; TwoSum (Knuth) keeps the rounding error
// of every addition, so the pair carries about twice the float significand.
struct AccFF {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float s = hi + x;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ float2 get_pair() const { return make_float2(hi, lo); }
  __device__ __forceinline__ void team_reduce(int nl) {
    for (int o = nl >> 1; o > 0; o >>= 1) {
      float oh = __shfl_xor_sync(0xffffffffu, hi, o);
      float ol = __shfl_xor_sync(0xffffffffu, lo, o);
      add(oh);
      lo += ol;
    }
  }
};

template <int PREC>
struct Traits;
template <>
struct Traits<0> {
  using R = double;
  using Acc = AccD;
};
template <>
struct Traits<1> {
  using R = float;
  using Acc = AccD;
};
template <>
struct Traits<2> {
  using R = float;
  using Acc = AccFF;
};
// 3: float-float node arithmetic (about 48 bits), for the chemical-potential
// passes of the FP32 modes; pair sums are added into FP64 per-site sums.
template <>
struct Traits<3> {
  using R = ff;
  using Acc = AccD;
};

// ---------------------------------------------------------------- math
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/r and r from r^2
__device__ __forceinline__ void r_from_r2(float r2, float& r, float& rinv) {
  rinv = rsqrt_approx(r2);
  r = r2 * rinv;
}
__device__ __forceinline__ void r_from_r2(double r2, double& r, double& rinv) {
  // one reciprocal square root (CUDA's rsqrt, 1 ulp) and a product: r and
  // 1/r to about 2 ulps, against a square root and a division on the FP64 pipe
  rinv = rsqrt(r2);
  r = r2 * rinv;
}

__device__ __forceinline__ void r_from_r2(ff r2, ff& r, ff& rinv) {
  r = ff_sqrt(r2);
  rinv = ff_recip(r);
}

// quintic switch S(r) and dS/dr
__device__ __forceinline__ void sw(const DevPot& P, float r, float& S, float& dS) {
  // clamp to [0, 1] as a saturating multiply (no separate min/max)
  float t = __saturatef((r - P.rs_f) * P.inv_w_f);
  float t2 = t * t;
  float u = 1.f - t;
  S = fmaf(t2 * t, fmaf(t, fmaf(-6.f, t, 15.f), -10.f), 1.f);
  dS = (t2 * (u * u)) * P.dS_scale_f;
}
__device__ __forceinline__ void sw(const DevPot& P, double r, double& S, double& dS) {
  double t = fmin(fmax((r - P.rs) * P.inv_w, 0.0), 1.0);
  double t2 = t * t;
  double u = 1.0 - t;
  S = fma(t2 * t, fma(t, fma(-6.0, t, 15.0), -10.0), 1.0);
  dS = (t2 * (u * u)) * (-30.0 * P.inv_w);
}

__device__ __forceinline__ void sw(const DevPot& P, ff r, ff& S, ff& dS) {
  if (r.hi <= P.rs_f && !(r.hi == P.rs_f && r.lo > 0.f)) {  // r <= r_switch: S = 1
    S = ff(1.0f, 0.f);
    dS = ff(0.f, 0.f);
    return;
  }
  ff t = (r - P.rs_ff) * P.inv_w_ff;
  if (!(t < ff(1.0f, 0.f))) {
    S = ff(0.f, 0.f);
    dS = ff(0.f, 0.f);
    return;
  }
  const ff t2 = t * t;
  const ff u = ff_add_f(-t, 1.0f);
  S = ff_add_f(t2 * t * ff_add_f(t * ff_add_f(ff_mul_f(t, -6.0f), 15.0f), -10.0f), 1.0f);
  dS = t2 * (u * u) * P.dS_scale_ff;
}

// raw exponential part of a radial term
__device__ __forceinline__ float rad_raw(const RadialFn& F, float r) { return ex2_approx(fmaf(-F.c1, r, F.c0)); }
__device__ __forceinline__ double rad_raw(const RadialFn& F, double r) { return F.A * exp(F.kappa - F.lambda * r); }
__device__ __forceinline__ ff rad_raw(const RadialFn& F, ff r) {
  return ff_exp(F.lnA_kappa_ff - F.lambda_ff * r, c_exp_table);
}
__device__ __forceinline__ ff rad_lam(const RadialFn& F, ff) { return F.lambda_ff; }
__device__ __forceinline__ float rad_lam(const RadialFn& F, float) { return F.lam_f; }
__device__ __forceinline__ double rad_lam(const RadialFn& F, double) { return F.lambda; }

// A pair term and minus its derivative (FP64 passes): exponential terms, or
// thermalized Lennard-Jones terms A ((s / r)^12 - (s / r)^6) (kind 1).
__device__ __forceinline__ void rad_pair(const RadialFn& F, double r, double& e, double& mde) {
  if (F.kind == 1) {
    const double x = F.kappa / r, x2 = x * x, x6 = x2 * x2 * x2;
    e = F.A * (x6 * x6 - x6);
    mde = F.A * (12.0 * x6 * x6 - 6.0 * x6) / r;
  } else {
    e = F.A * exp(F.kappa - F.lambda * r);
    mde = F.lambda * e;
  }
}

template <typename T>
__device__ __forceinline__ T sqrt6();
template <>
__device__ __forceinline__ float sqrt6<float>() { return 2.44948974f; }
template <>
__device__ __forceinline__ double sqrt6<double>() { return kSqrt6; }
template <>
__device__ __forceinline__ ff sqrt6<ff>() { return ff(kSqrt6); }

// ---------------------------------------------------------------- site data
template <int PREC, int S>
struct SiteData {
  using R = typename Traits<PREC>::R;
  R p[3];     // FP64: absolute position; FP32: cell-relative position
  R sig;
  R x[S];
};

template <int S>
__device__ __forceinline__ void load_site(const PassArgs& A, int64_t j, SiteData<0, S>& d) {
  const int64_t n = A.n;
  d.p[0] = A.q[j];
  d.p[1] = A.q[n + j];
  d.p[2] = A.q[2 * n + j];
  d.sig = A.sigma[j];
#pragma unroll
  for (int k = 0; k < S; ++k) d.x[k] = A.x[k * n + j];
}
template <int S>
__device__ __forceinline__ void load_site(const PassArgs& A, int64_t j, SiteData<3, S>& d) {
  const float4 P = __ldg(&A.pos32[j]), Pl = __ldg(&A.pos32lo[j]);
  d.p[0] = ff(P.x, Pl.x);
  d.p[1] = ff(P.y, Pl.y);
  d.p[2] = ff(P.z, Pl.z);
  d.sig = ff(P.w, Pl.w);
  const float4 X = __ldg(&A.x32[j]), Xl = __ldg(&A.x32lo[j]);
  const float xs[4] = {X.x, X.y, X.z, X.w}, xl[4] = {Xl.x, Xl.y, Xl.z, Xl.w};
#pragma unroll
  for (int k = 0; k < S; ++k) d.x[k] = ff(xs[k], xl[k]);
}
template <int PREC, int S>
__device__ __forceinline__ void load_site(const PassArgs& A, int64_t j, SiteData<PREC, S>& d) {
  float4 P = __ldg(&A.pos32[j]);
  d.p[0] = P.x;
  d.p[1] = P.y;
  d.p[2] = P.z;
  d.sig = P.w;
  float4 X = __ldg(&A.x32[j]);
  float xs[4] = {X.x, X.y, X.z, X.w};
#pragma unroll
  for (int k = 0; k < S; ++k) d.x[k] = xs[k];
}

// separation d = q_j - q_i
template <int S>
__device__ __forceinline__ void separation(const DevGrid& g, const SiteData<0, S>& si, const SiteData<0, S>& sj,
                                           uint32_t, double d[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double da = sj.p[a] - si.p[a];
    d[a] = da - g.L[a] * rint(da * g.invL[a]);
  }
}
template <int PREC, int S>
__device__ __forceinline__ void separation(const DevGrid& g, const SiteData<PREC, S>& si,
                                           const SiteData<PREC, S>& sj, uint32_t code, float d[3]) {
  int c = (int)(code);
  int s[3] = {c / 9 - 1, (c / 3) % 3 - 1, c % 3 - 1};
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = (sj.p[a] - si.p[a]) + (float)s[a] * g.h_f[a];
}

template <int S>
__device__ __forceinline__ void separation(const DevGrid& g, const SiteData<3, S>& si, const SiteData<3, S>& sj,
                                           uint32_t code, ff d[3]) {
  const int c = (int)(code);
  const float s[3] = {(float)(c / 9 - 1), (float)((c / 3) % 3 - 1), (float)(c % 3 - 1)};
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = (sj.p[a] - si.p[a]) + ff(s[a] * g.h_f[a], s[a] * g.h_lo[a]);
}

// neighbours' embedding coefficients for pass 2
template <int S>
__device__ __forceinline__ void load_ab(const PassArgs& A, int64_t j, double a[S], double b[S],
                                        SiteData<0, S>*) {
#pragma unroll
  for (int k = 0; k < S; ++k) {
    a[k] = A.a[k * A.n + j];
    b[k] = A.b[k * A.n + j];
  }
}
template <int S>
__device__ __forceinline__ void load_ab(const PassArgs& A, int64_t j, ff a[S], ff b[S], SiteData<3, S>*) {
  const float4 v0 = __ldg(&A.ab32[2 * j]), l0 = __ldg(&A.ab32lo[2 * j]);
  a[0] = ff(v0.x, l0.x);
  b[0] = ff(v0.y, l0.y);
  if (S > 1) {
    a[1 < S ? 1 : 0] = ff(v0.z, l0.z);
    b[1 < S ? 1 : 0] = ff(v0.w, l0.w);
  }
}
template <int PREC, int S>
__device__ __forceinline__ void load_ab(const PassArgs& A, int64_t j, float a[S], float b[S],
                                        SiteData<PREC, S>*) {
  float4 v0 = __ldg(&A.ab32[2 * j]);
  a[0] = v0.x;
  b[0] = v0.y;
  if (S > 1) {
    a[1 < S ? 1 : 0] = v0.z;
    b[1 < S ? 1 : 0] = v0.w;
  }
  if (S > 2) {
    float4 v1 = __ldg(&A.ab32[2 * j + 1]);
    a[2 < S ? 2 : 0] = v1.x;
    b[2 < S ? 2 : 0] = v1.y;
    if (S > 3) {
      a[3 < S ? 3 : 0] = v1.z;
      b[3 < S ? 3 : 0] = v1.w;
    }
  }
}

__device__ __forceinline__ bool skin_violated(const Ctrl* c) {
  double disp = sqrt(__longlong_as_double((long long)c->disp2_bits));
  double smax = __longlong_as_double((long long)c->smax_bits);
  return 2.0 * disp + kSqrt6 * (smax - c->sigma_max_build) > c->skin;
}

// Uniform early exit of the relaxation chunk.  Returns true if the kernel must
// stop.  The skin test runs once per launch, on thread 0 of block 0 (on the
// 1:64 FP64 pipe a test per block kept the FP64 pipe a quarter busy and held
// every block at the barrier behind it); each block reads the halt flag
// through one thread.  Blocks that start before block 0 sets the flag run the
// pass on the old lists (valid arrays, so every access stays in bounds); a
// halted pass is always evaluated again after the rebuild, so that output is
// never used.  Every thread of the block must call this before any early
// return.
__device__ __forceinline__ bool chunk_halted(const PassArgs& A) {
  if (A.ctrl == nullptr) return false;
  __shared__ int halt;
  if (threadIdx.x == 0) {
    int h = A.ctrl->halted ? 1 : 0;
    if (!h && blockIdx.x == 0 && A.check_skin && skin_violated(A.ctrl)) {
      A.ctrl->reason = kReasonRebuild;
      A.ctrl->halted = 1;
      h = 1;
    }
    halt = h;
  }
  __syncthreads();
  return halt != 0;
}

// ---------------------------------------------------------------- K2: density pass
// Minimum resident blocks per SM for the two passes (0: let the compiler choose
// the register budget); set at build time.
#ifndef MXE_DENSITY_MIN_BLOCKS
#define MXE_DENSITY_MIN_BLOCKS 0
#endif
#ifndef MXE_GRADIENT_MIN_BLOCKS
#define MXE_GRADIENT_MIN_BLOCKS 0
#endif

template <int PREC, int S, int NL>
__global__ void __launch_bounds__(256, MXE_DENSITY_MIN_BLOCKS) k_density(DevPot P, DevGrid g, PassArgs A) {
  using R = typename Traits<PREC>::R;
  using Acc = typename Traits<PREC>::Acc;
  constexpr int NF = S * S;
  if (chunk_halted(A)) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc rb[S], ra[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    rb[k].zero();
    ra[k].zero();
  }
  int bad = 0;
  if (active) {
    const DevGrid gs = site_grid(g, A.batch, i);
    SiteData<PREC, S> si;
    load_site(A, i, si);
    const R s_i = sqrt6<R>() * si.sig;
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
    for (int t = beg + lane; t < end; t += NL) {
      const uint32_t ent = __ldg(&A.nb_ent[t]);
      const int64_t j = ent & kIdxMask;
      SiteData<PREC, S> sj;
      load_site(A, j, sj);
      R d[3];
      separation(gs, si, sj, ent >> kCodeShift, d);
      const R s_j = sqrt6<R>() * sj.sig;
      const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      // every node lies at least |d| - max(s_i, s_j) from the origin site:
      // only a pair closer than 0.5 A + that shift needs its nodes checked
      constexpr bool kNodeCheck = PREC == 0 || PREC == 3;
      const R s_max = s_i < s_j ? s_j : s_i;
      const R near = (R)kRMin + s_max;
      const bool close = D2 < near * near;
      R fst[NF], fav[NF];
      // static point
      {
        R r, rinv, Sw, dS;
        r_from_r2(D2, r, rinv);
        bad |= D2 < (R)(kRMin * kRMin);
        sw(P, r, Sw, dS);
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          fst[v] = (v < P.n_f) ? rad_raw(P.f[v], r) * Sw : (R)0;
          fav[v] = (R)0;
        }
      }
      // 12 nodes: site i moved (base_i), site j moved (base_j), each +-s along each axis
      // float-float node arithmetic is long: keep its node loops rolled so the
      // kernel fits the instruction cache
#pragma unroll(PREC == 3 ? 1 : 2)
      for (int site = 0; site < 2; ++site) {
        const R s = site == 0 ? s_i : s_j;
        const R base = D2 + s * s;
#pragma unroll(PREC == 3 ? 1 : 3)
        for (int a = 0; a < 3; ++a) {
          const R tw = (R)2 * s * d[a];
#pragma unroll
          for (int pm = 0; pm < 2; ++pm) {
            const R r2 = pm == 0 ? base + tw : base - tw;
            R r, rinv, Sw, dS;
            r_from_r2(r2, r, rinv);
            if (kNodeCheck) bad |= r2 < (R)(kRMin * kRMin);
            sw(P, r, Sw, dS);
#pragma unroll
            for (int v = 0; v < NF; ++v)
              if (v < P.n_f) fav[v] += rad_raw(P.f[v], r) * Sw;
          }
        }
      }
      if (!kNodeCheck && close) {  // rare: the exact node distances
        for (int site = 0; site < 2; ++site) {
          const R s = site == 0 ? s_i : s_j;
          for (int a = 0; a < 3; ++a) {
            const R base = D2 + s * s, tw = (R)2 * s * d[a];
            bad |= (base + tw) < (R)(kRMin * kRMin);
            bad |= (base - tw) < (R)(kRMin * kRMin);
          }
        }
      }
      // rho_i^k += sum_l x_jl f_kl
#pragma unroll
      for (int k = 0; k < S; ++k) {
        R sb = (R)0, sa = (R)0;
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const int fo = P.f_of[k][l];
#pragma unroll
          for (int v = 0; v < NF; ++v)
            if (fo == v) {
              sb += sj.x[l] * fst[v];
              sa += sj.x[l] * fav[v];
            }
        }
        rb[k].add(sb);
        ra[k].add(sa);
      }
    }
  }
  if (NL > 1) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      rb[k].team_reduce(NL);
      ra[k].team_reduce(NL);
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
  }
  if (!active || lane != 0) {
    if (bad && active) atomicOr(A.flags, kFlagGeometry);
    return;
  }
  const int64_t n = A.n;
  int flag = bad ? kFlagGeometry : 0;
  float ab[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if constexpr (PREC == 1 || PREC == 2) {
    if (A.lean) {
      // relaxation loop: only the packed FP32 (a, b) are needed; all in FP32
      const float4 X = A.x32[i];
      const float xs[4] = {X.x, X.y, X.z, X.w};
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const float2 b2 = rb[k].get_pair(), a2 = ra[k].get_pair();
        const float rf = b2.x + b2.y;
        const float df = fmaf(a2.x, 1.0f / 12.0f, -b2.x) + fmaf(a2.y, 1.0f / 12.0f, -b2.y);
        if (P.E[k] == 0.0) {
          // no embedding energy for this element
        } else if (rf > (float)kRhoMin) {
          const float Ef = (float)P.E[k];
          const float isq = rsqrt_approx(rf);
          const float dF = -0.5f * Ef * isq;
          const float d2F = 0.25f * Ef * isq * isq * isq;
          ab[2 * k] = xs[k] * d2F * df;
          ab[2 * k + 1] = xs[k] * dF;
        } else {
          flag |= kFlagGeometry;
        }
      }
      A.ab32[2 * i] = make_float4(ab[0], ab[1], ab[2], ab[3]);
      if (S > 2) A.ab32[2 * i + 1] = make_float4(ab[4], ab[5], ab[6], ab[7]);
      if (flag) atomicOr(A.flags, flag);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double rbar = rb[k].get();
    const double ravg = ra[k].get() * (1.0 / 12.0);
    const double xk = A.x[k * n + i];
    double e = 0.0, ak = 0.0, bk = 0.0;
    if (P.E[k] == 0.0) {
      // no embedding energy for this element
    } else if (rbar > kRhoMin) {
      if (PREC == 0 || PREC == 3) {
        const double sq = sqrt(rbar);
        const double F = -P.E[k] * sq;
        const double dF = -P.E[k] / (2.0 * sq);
        const double d2F = P.E[k] / (4.0 * rbar * sq);
        e = F + dF * (ravg - rbar);
        ak = xk * d2F * (ravg - rbar);
        bk = xk * dF;
      } else {
        // embedding arithmetic in FP32 (the difference <rho> - rho_bar is taken
        // in FP64 first: it is small against rho)
        const float rf = (float)rbar, df = (float)(ravg - rbar), Ef = (float)P.E[k], xf = (float)xk;
        const float isq = rsqrt_approx(rf);
        const float sq = rf * isq;
        const float dF = -0.5f * Ef * isq;
        const float d2F = 0.25f * Ef * isq * isq * isq;
        e = (double)(-Ef * sq) + (double)(dF * df);
        ak = (double)(xf * d2F * df);
        bk = (double)(xf * dF);
      }
    } else {
      flag |= kFlagGeometry;
    }
    A.rho_bar[k * n + i] = rbar;
    A.rho_avg[k * n + i] = ravg;
    A.e[k * n + i] = e;
    A.a[k * n + i] = ak;
    A.b[k * n + i] = bk;
    ab[2 * k] = (float)ak;
    ab[2 * k + 1] = (float)bk;
  }
  if (PREC != 0) {
    A.ab32[2 * i] = make_float4(ab[0], ab[1], ab[2], ab[3]);
    if (S > 2) A.ab32[2 * i + 1] = make_float4(ab[4], ab[5], ab[6], ab[7]);
  }
  if (PREC == 3) {
    float lo[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double av = k < S ? A.a[k * n + i] : 0.0, bv = k < S ? A.b[k * n + i] : 0.0;
      lo[2 * k] = (float)(av - (double)(float)av);
      lo[2 * k + 1] = (float)(bv - (double)(float)bv);
    }
    A.ab32lo[2 * i] = make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
  if (flag) atomicOr(A.flags, flag);
}

// ---------------------------------------------------------------- K3: gradient pass
// MODE kGradAll: dF/dq, dF/dsigma, mu, energies; kGradForce: dF/dq, dF/dsigma,
// energies (no mu); kGradForceNoE: dF/dq, dF/dsigma only (relaxation loop);
// kGradMu: mu and energies only (no derivatives).
// Without mu, the derivative of the pair's weighted radial terms at a node is
// formed as G = dS sum_u c_u E_u - S sum_u (c_u lambda_u) E_u (E_u the raw
// exponentials), three FP32 operations per term.
template <int PREC, int S, int NL, int MODE>
__global__ void __launch_bounds__(256, MXE_GRADIENT_MIN_BLOCKS) k_gradient(DevPot P, DevGrid g, PassArgs A) {
  constexpr bool DER = MODE != kGradMu;
  constexpr bool MU = MODE == kGradAll || MODE == kGradMu;
  constexpr bool EN = MODE != kGradForceNoE;
  using R = typename Traits<PREC>::R;
  using Acc = typename Traits<PREC>::Acc;
  constexpr int NF = S * S;
  constexpr int NP = S * (S + 1) / 2;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc gacc[3], gsig, mu[S], epair;
#pragma unroll
  for (int c = 0; c < 3; ++c) gacc[c].zero();
  gsig.zero();
  epair.zero();
#pragma unroll
  for (int k = 0; k < S; ++k) mu[k].zero();
  if (active) {
    const DevGrid gs = site_grid(g, A.batch, i);
    SiteData<PREC, S> si;
    load_site(A, i, si);
    R ai[S], bi[S];
    load_ab(A, i, ai, bi, (SiteData<PREC, S>*)nullptr);
    const R s_i = sqrt6<R>() * si.sig;
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
    for (int t = beg + lane; t < end; t += NL) {
      const uint32_t ent = __ldg(&A.nb_ent[t]);
      const int64_t j = ent & kIdxMask;
      SiteData<PREC, S> sj;
      load_site(A, j, sj);
      R aj[S], bj[S];
      load_ab(A, j, aj, bj, (SiteData<PREC, S>*)nullptr);
      R d[3];
      separation(gs, si, sj, ent >> kCodeShift, d);
      const R s_j = sqrt6<R>() * sj.sig;
      const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      // pair weights of the distinct radial terms
      R cphi[NP], cfa[NF], cfs[NF];
#pragma unroll
      for (int u = 0; u < NP; ++u) cphi[u] = (R)0;
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        cfa[v] = (R)0;
        cfs[v] = (R)0;
      }
#pragma unroll
      for (int k = 0; k < S; ++k)
#pragma unroll
        for (int l = 0; l < S; ++l) {
          // table entries read once (compared inside the unrolled loops they
          // sent a copy of the tables to the stack)
          const int po = P.phi_of[k][l], fo = P.f_of[k][l];
#pragma unroll
          for (int u = 0; u < NP; ++u)
            if (po == u) cphi[u] += si.x[k] * sj.x[l];
#pragma unroll
          for (int v = 0; v < NF; ++v)
            if (fo == v) {
              cfa[v] += bi[k] * sj.x[l] + bj[k] * si.x[l];
              cfs[v] += ai[k] * sj.x[l] + aj[k] * si.x[l];
            }
        }
      R clphi[NP], clf[NF];  // weights times decay rates (factored derivative)
#pragma unroll
      for (int u = 0; u < NP; ++u) clphi[u] = cphi[u] * rad_lam(P.phi[u], s_i);
#pragma unroll
      for (int v = 0; v < NF; ++v) clf[v] = cfa[v] * rad_lam(P.f[v], s_i);
      R epn = (R)0;  // sum over nodes of S sum_u c_u E_u (pair energy, factored path)
      // static point: density terms only
      R fst[NF], Gs;
      {
        R r, rinv, Sw, dS;
        r_from_r2(D2, r, rinv);
        sw(P, r, Sw, dS);
        Gs = (R)0;
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          fst[v] = (R)0;
          if (v < P.n_f) {
            const R e = rad_raw(P.f[v], r);
            fst[v] = e * Sw;
            Gs += cfs[v] * (e * (dS - rad_lam(P.f[v], r) * Sw));
          }
        }
        Gs *= rinv;
      }
      // 12 nodes
      R aphi[NP], af[NF];
#pragma unroll
      for (int u = 0; u < NP; ++u) aphi[u] = (R)0;
#pragma unroll
      for (int v = 0; v < NF; ++v) af[v] = (R)0;
      R T = (R)0, U[3] = {(R)0, (R)0, (R)0}, Vs = (R)0;
      // float-float node arithmetic is long: keep its node loops rolled so the
      // kernel fits the instruction cache
#pragma unroll(PREC == 3 ? 1 : 2)
      for (int site = 0; site < 2; ++site) {
        const R s = site == 0 ? s_i : s_j;
        const R base = D2 + s * s;
#pragma unroll(PREC == 3 ? 1 : 3)
        for (int a = 0; a < 3; ++a) {
          const R tw = (R)2 * s * d[a];
          R w2[2];
#pragma unroll
          for (int pm = 0; pm < 2; ++pm) {
            const R r2 = pm == 0 ? base + tw : base - tw;
            R r, rinv, Sw, dS;
            r_from_r2(r2, r, rinv);
            sw(P, r, Sw, dS);
            R G = (R)0;
            if constexpr (!MU) {
              R A1p = (R)0, A1f = (R)0, A2 = (R)0;
#pragma unroll
              for (int u = 0; u < NP; ++u)
                if (u < P.n_phi) {
                  if constexpr (PREC == 0) {
                    double e, mde;
                    rad_pair(P.phi[u], r, e, mde);
                    A1p += cphi[u] * e;
                    A2 += cphi[u] * mde;
                  } else {
                    const R e = rad_raw(P.phi[u], r);
                    A1p += cphi[u] * e;
                    A2 += clphi[u] * e;
                  }
                }
#pragma unroll
              for (int v = 0; v < NF; ++v)
                if (v < P.n_f) {
                  const R e = rad_raw(P.f[v], r);
                  A1f += cfa[v] * e;
                  A2 += clf[v] * e;
                }
              G = (A1p + A1f) * dS - A2 * Sw;
              if (EN) epn += A1p * Sw;
            } else {
#pragma unroll
              for (int u = 0; u < NP; ++u)
                if (u < P.n_phi) {
                  if constexpr (PREC == 0) {
                    double e, mde;
                    rad_pair(P.phi[u], r, e, mde);
                    aphi[u] += e * Sw;
                    if (DER) G += cphi[u] * (e * dS - mde * Sw);
                  } else {
                    const R e = rad_raw(P.phi[u], r);
                    aphi[u] += e * Sw;
                    if (DER) G += cphi[u] * (e * (dS - rad_lam(P.phi[u], r) * Sw));
                  }
                }
#pragma unroll
              for (int v = 0; v < NF; ++v)
                if (v < P.n_f) {
                  const R e = rad_raw(P.f[v], r);
                  af[v] += e * Sw;
                  if (DER) G += cfa[v] * (e * (dS - rad_lam(P.f[v], r) * Sw));
                }
            }
            w2[pm] = G * rinv;
          }
          T += w2[0] + w2[1];
          U[a] += s * (w2[0] - w2[1]);
          if (site == 0) Vs += sqrt6<R>() * ((d[a] + s) * w2[0] - (d[a] - s) * w2[1]);
        }
      }
      const R inv12 = (R)(1.0 / 12.0);
      if (DER) {
        const R Tt = T * inv12 + Gs;
#pragma unroll
        for (int c = 0; c < 3; ++c) gacc[c].add(-(d[c] * Tt + U[c] * inv12));
        gsig.add(Vs * inv12);
      }
      if constexpr (!MU) {
        if (EN) epair.add((R)0.5 * inv12 * epn);
      } else {
        R ep = (R)0;
#pragma unroll
        for (int u = 0; u < NP; ++u) ep += cphi[u] * aphi[u];
        epair.add((R)0.5 * inv12 * ep);
      }
#pragma unroll
      for (int k = 0; k < S; ++k) {
        if (!MU) break;
        R m = (R)0;
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const int po = P.phi_of[k][l], fo = P.f_of[l][k];
#pragma unroll
          for (int u = 0; u < NP; ++u)
            if (po == u) m += sj.x[l] * aphi[u] * inv12;
          // density at j of species l from this site holding species k: f_lk
#pragma unroll
          for (int v = 0; v < NF; ++v)
            if (fo == v) m += aj[l] * fst[v] + bj[l] * af[v] * inv12;
        }
        mu[k].add(m);
      }
    }
  }
  if (NL > 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) gacc[c].team_reduce(NL);
    gsig.team_reduce(NL);
    epair.team_reduce(NL);
#pragma unroll
    for (int k = 0; k < S; ++k) mu[k].team_reduce(NL);
  }
  if (!active || lane != 0) return;
  const int64_t n = A.n;
  const double kT = kKB * A.T[i];
  const double sg = A.sigma[i];
  int flag = 0;
  double g0 = gacc[0].get(), g1 = gacc[1].get(), g2 = gacc[2].get();
  double gs;
  if constexpr (PREC == 1 || PREC == 2) {
    // FP32 modes: the thermal term in FP32 (no FP64 division)
    const float2 gp = gsig.get_pair();
    const float th = 3.0f * (float)kKB * (float)A.T[i] / (float)sg;
    gs = (double)((gp.x - th) + gp.y);
  } else {
    gs = gsig.get() - 3.0 * kT / sg;
  }
  if (DER && A.gq) {
    A.gq[i] = g0;
    A.gq[n + i] = g1;
    A.gq[2 * n + i] = g2;
  }
  if (DER && A.gs) A.gs[i] = gs;
  bool finite = !DER || (isfinite(g0) && isfinite(g1) && isfinite(g2) && isfinite(gs));
  if (MU) {
    double xv = 1.0;
#pragma unroll
    for (int k = 0; k < S; ++k) xv -= A.x[k * n + i];
    const double lv = log(fmax(xv, kLogFloor));
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double m = mu[k].get() + A.e[k * n + i];
      finite = finite && isfinite(m);
      if (A.mu_ex) A.mu_ex[k * n + i] = m;
      if (A.mu) A.mu[k * n + i] = m + kT * (log(fmax(A.x[k * n + i], kLogFloor)) - lv);
    }
  }
  if (A.site_E) {  // the relaxation loop asks for no energies: skip their FP64 logarithms
    double xv = 1.0, mix = 0.0, emb = 0.0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double xk = A.x[k * n + i];
      xv -= xk;
      if (xk > 0.0) mix += xk * log(xk);
      emb += xk * A.e[k * n + i];
    }
    if (xv > 0.0) mix += xv * log(xv);
    const double EV = epair.get() + emb;
    const double Fv = -3.0 * kT * log(sg);
    const double Fm = kT * mix;
    A.site_E[i] = EV;
    A.site_E[n + i] = Fv;
    A.site_E[2 * n + i] = Fm;
    finite = finite && isfinite(EV) && isfinite(Fv) && isfinite(Fm);
  }
  if (!finite) flag |= kFlagNonfinite;
  if (flag) atomicOr(A.flags, flag);
}

// ---------------------------------------------------------------- half-list accurate passes
// The averages <phi_u>_ij, <f_v>_ij and the static f_v(r_ij) of a pair depend
// only on its geometry and are the same from both ends (the node set of
// App. A is symmetric in i and j).  k_pair_geo evaluates them once per
// unordered pair (one thread per pair) into a record of C values, written
// to both entries of the pair:
// [f_v static (n_f) | sum over the 12 nodes of f_v (n_f) | of phi_u (n_phi)];
// k_pair_density / k_pair_mu gather the records over every site's full row
// in row order and finish exactly as the density and chemical-potential
// passes do.  Node arithmetic R: float-float (records of
// float pairs; the FP32 modes) or FP64 (records of doubles).
// The record of unordered pair p: owner site i, the entry of j in row i (j with
// its image code), that entry's index tp and the index tr of the reverse
// entry (i in row j).  The records are built from the current lists, so they
// are consistent with them by construction; every index is still bounded
// (a bad record sets the overflow flag and the pair is skipped).  Building
// with MXE_DEBUG_CHECKS also checks that tp and tr lie in their rows.
struct PairRef {
  int64_t i, j;
  uint32_t code;
  int tp, tr;
};
__device__ __forceinline__ bool load_pair(const PassArgs& A, const int4* __restrict__ rec, int64_t p, PairRef& r) {
  const int4 v = __ldg(&rec[p]);
  r.i = v.x;
  r.j = (uint32_t)v.y & kIdxMask;
  r.code = (uint32_t)v.y >> kCodeShift;
  r.tp = v.z;
  r.tr = v.w;
  bool ok = (uint64_t)(uint32_t)v.x < (uint64_t)A.n && (uint64_t)r.j < (uint64_t)A.n &&
            (uint64_t)(uint32_t)v.z < (uint64_t)A.n_ent && (uint64_t)(uint32_t)v.w < (uint64_t)A.n_ent;
#ifdef MXE_DEBUG_CHECKS
  ok = ok && r.tp >= A.nb_off[r.i] && r.tp < A.nb_off[r.i + 1] && A.nb_ent[r.tp] == (uint32_t)v.y &&
       r.tr >= A.nb_off[r.j] && r.tr < A.nb_off[r.j + 1] && (A.nb_ent[r.tr] & kIdxMask) == (uint32_t)r.i;
#endif
  if (!ok) atomicOr(A.flags, kFlagOverflow);
  return ok;
}

template <typename R>
struct GeoRec;
template <>
struct GeoRec<ff> {
  using T = float2;
  static __device__ __forceinline__ T put(ff v) { return make_float2(v.hi, v.lo); }
  static __device__ __forceinline__ ff get(const T* __restrict__ rec, int c) {
    const float2 v = __ldg(&rec[c]);
    return ff(v.x, v.y);
  }
};
template <>
struct GeoRec<double> {
  using T = double;
  static __device__ __forceinline__ T put(double v) { return v; }
  static __device__ __forceinline__ double get(const T* __restrict__ rec, int c) { return __ldg(&rec[c]); }
};

// site data of the accurate passes: float-float records (PREC 3) or FP64 state
template <typename R>
struct GeoPrec;
template <>
struct GeoPrec<ff> {
  static constexpr int P = 3;
};
template <>
struct GeoPrec<double> {
  static constexpr int P = 0;
};

// a radial term at a node: exponential terms in R (float-float: with the
// exponential's table in shared memory); thermalized Lennard-Jones pair terms
// (FP64 contexts only) through rad_pair
__device__ __forceinline__ ff geo_term(const RadialFn& F, ff r, const float2* T) {
  return ff_exp(F.lnA_kappa_ff - F.lambda_ff * r, T);
}
__device__ __forceinline__ double geo_term(const RadialFn& F, double r, const float2*) { return rad_raw(F, r); }
__device__ __forceinline__ ff pair_term(const RadialFn& F, ff r, const float2* T) { return geo_term(F, r, T); }
__device__ __forceinline__ double pair_term(const RadialFn& F, double r, const float2*) {
  double e, mde;
  rad_pair(F, r, e, mde);
  return e;
}

// the power form's pieces in the node arithmetic R
__device__ __forceinline__ ff geo_exp(ff x, const float2* T) { return ff_exp(x, T); }
__device__ __forceinline__ double geo_exp(double x, const float2*) { return exp(x); }
__device__ __forceinline__ ff pw_beta(const DevPot& P, int s, ff) { return P.pw_beta_ff[s]; }
__device__ __forceinline__ double pw_beta(const DevPot& P, int s, double) { return P.pw_beta[s]; }
__device__ __forceinline__ ff pw_pref_phi(const DevPot& P, int u, ff) { return P.pw_pref_phi_ff[u]; }
__device__ __forceinline__ double pw_pref_phi(const DevPot& P, int u, double) { return P.pw_pref_phi[u]; }
__device__ __forceinline__ ff pw_pref_f(const DevPot& P, int v, ff) { return P.pw_pref_f_ff[v]; }
__device__ __forceinline__ double pw_pref_f(const DevPot& P, int v, double) { return P.pw_pref_f[v]; }

// c^e for 1 <= e <= 31 from the squares sq[b] = c^(2^b) (the bits of e are
// uniform over the warp: the exponents are the potential's)
template <typename R>
__device__ __forceinline__ R pow_from_squares(const R sq[5], int e) {
  R r = (R)1;
  bool first = true;
#pragma unroll
  for (int b = 0; b < 5; ++b)
    if ((e >> b) & 1) {
      r = first ? sq[b] : r * sq[b];
      first = false;
    }
  return r;
}

// sqrt(a b) of two positive values (the cross term of a geometric-mean pair)
__device__ __forceinline__ ff cross_mean(ff a, ff b) { return ff_sqrt(a * b); }
__device__ __forceinline__ double cross_mean(double a, double b) { return sqrt(a * b); }

// PW 1: the power form with the exponents fixed at compile time, m = 6 and
// n = 10 for both species (pair rate 3/r0, density rate 5/r0: c_s =
// exp(-r / (2 r0_s))); PW 2: the power form with the exponents read at run
// time; PW 0: the general form (no power-form code: fewer registers).
template <int S, typename R, int PW>
__global__ void __launch_bounds__(256) k_pair_geo(DevPot P, DevGrid g0, PassArgs A,
                                                  const int4* __restrict__ pair_rec, int64_t npair,
                                                  typename GeoRec<R>::T* __restrict__ buf, GeoLayout L) {
  constexpr int PR = GeoPrec<R>::P;
  // the float-float exponential's table, in shared memory (read by the
  // halt check's barrier below before any use)
  __shared__ float2 s_exp[32];
  if (threadIdx.x < 32) s_exp[threadIdx.x] = make_float2(c_exp_table.hi[threadIdx.x], c_exp_table.lo[threadIdx.x]);
  if (A.ctrl == nullptr) __syncthreads();
  if (chunk_halted(A)) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npair) return;
  PairRef pr_;
  if (!load_pair(A, pair_rec, p, pr_)) return;
  const int64_t i = pr_.i, j = pr_.j;
  const DevGrid gs = site_grid(g0, A.batch, i);
  SiteData<PR, S> si, sj;
  load_site(A, i, si);
  load_site(A, j, sj);
  R d[3];
  separation(gs, si, sj, pr_.code, d);
  const R s_i = sqrt6<R>() * si.sig, s_j = sqrt6<R>() * sj.sig;
  const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  int bad = D2 < (R)(kRMin * kRMin);
  // component c of the record, at both entries of the pair (plane A below
  // L.ca, plane B above)
  typename GeoRec<R>::T* oa = buf + pr_.tp * (int64_t)L.ca;
  typename GeoRec<R>::T* oa2 = buf + pr_.tr * (int64_t)L.ca;
  typename GeoRec<R>::T* ob = buf + L.b_off + pr_.tp * (int64_t)L.cb;
  typename GeoRec<R>::T* ob2 = buf + L.b_off + pr_.tr * (int64_t)L.cb;
  auto put = [&](int c, R v) {
    const typename GeoRec<R>::T w = GeoRec<R>::put(v);
    if (c < L.ca) {
      oa[c] = w;
      oa2[c] = w;
    } else {
      ob[c - L.ca] = w;
      ob2[c - L.ca] = w;
    }
  };
  if constexpr (PW != 0) {
    // power form: per point its distance and switch, the two bases c_s =
    // exp(-beta_s r) and the terms as their integer powers (prefactors
    // applied to the sums); no per-point arrays
    R af[2] = {(R)0, (R)0}, aphi[3] = {(R)0, (R)0, (R)0}, st[2];
    const int top0 = max(P.pw_m[0], P.pw_n[0]), top1 = max(P.pw_m[1], P.pw_n[1]);
#pragma unroll 1
    for (int k = 0; k < 13; ++k) {
      R r2 = D2;  // point 12: the static point
      if (k < 12) {
        const int site = k / 6, a = (k / 2) % 3, pm = k & 1;
        const R s = site == 0 ? s_i : s_j;
        const R tw = (R)2 * s * d[a];
        const R base = D2 + s * s;
        r2 = pm == 0 ? base + tw : base - tw;
        bad |= r2 < (R)(kRMin * kRMin);
      }
      R r, rinv, Sw, dS;
      r_from_r2(r2, r, rinv);
      sw(P, r, Sw, dS);
      const R c0 = geo_exp(-(pw_beta(P, 0, R()) * r), s_exp);
      const R c1 = geo_exp(-(pw_beta(P, 1, R()) * r), s_exp);
      R f0, f1, h0, h1;  // c^n and c^(m/2) of each species
      if constexpr (PW == 1) {
        const R c0_2 = c0 * c0, c1_2 = c1 * c1;
        h0 = c0_2 * c0;
        h1 = c1_2 * c1;
        const R c0_5 = h0 * c0_2, c1_5 = h1 * c1_2;
        f0 = c0_5 * c0_5;
        f1 = c1_5 * c1_5;
      } else {
        R sq0[5], sq1[5];
        sq0[0] = c0;
        sq1[0] = c1;
#pragma unroll
        for (int b = 1; b < 5; ++b) {
          if ((top0 >> b) != 0) sq0[b] = sq0[b - 1] * sq0[b - 1];
          if ((top1 >> b) != 0) sq1[b] = sq1[b - 1] * sq1[b - 1];
        }
        f0 = pow_from_squares(sq0, P.pw_n[0]);
        f1 = pow_from_squares(sq1, P.pw_n[1]);
        h0 = pow_from_squares(sq0, P.pw_m[0] / 2);
        h1 = pow_from_squares(sq1, P.pw_m[1] / 2);
      }
      if (k == 12) {  // the static point: densities only
        st[0] = f0 * Sw;
        st[1] = f1 * Sw;
        break;
      }
      af[0] += f0 * Sw;
      af[1] += f1 * Sw;
      aphi[0] += (h0 * h0) * Sw;
      aphi[2] += (h1 * h1) * Sw;
      aphi[1] += (h0 * h1) * Sw;
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      put(v, pw_pref_f(P, v, R()) * st[v]);
      put(2 + v, pw_pref_f(P, v, R()) * af[v]);
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) put(4 + u, pw_pref_phi(P, u, R()) * aphi[u]);
    if (bad) atomicOr(A.flags, kFlagGeometry);
    return;
  }
  // the 13 points once: r and S(r) of the 12 nodes (0..11) and the static point (12)
  R pr[13], pw[13];
  {
    R rinv, dS;
    r_from_r2(D2, pr[12], rinv);
    sw(P, pr[12], pw[12], dS);
  }
#pragma unroll 1
  for (int k = 0; k < 12; ++k) {
    const int site = k / 6, a = (k / 2) % 3, pm = k & 1;
    const R s = site == 0 ? s_i : s_j;
    const R tw = (R)2 * s * d[a];
    const R base = D2 + s * s;
    const R r2 = pm == 0 ? base + tw : base - tw;
    bad |= r2 < (R)(kRMin * kRMin);
    R rinv, dS;
    r_from_r2(r2, pr[k], rinv);
    sw(P, pr[k], pw[k], dS);
  }
  // general form: one term at a time over the points (rolled: one copy of
  // the float-float exponential in the loop body).  The record goes to both
  // entries of the pair (every value is symmetric in i and j), so the gathers
  // read rows in order.
#pragma unroll 1
  for (int v = 0; v < P.n_f; ++v) {
    R acc = (R)0;
#pragma unroll 1
    for (int k = 0; k < 12; ++k) acc += geo_term(P.f[v], pr[k], s_exp) * pw[k];
    const R st = geo_term(P.f[v], pr[12], s_exp) * pw[12];
    put(v, st);
    put(P.n_f + v, acc);
  }
  if (P.tab == 1 && P.cross_geo) {
    // binary pattern with a geometric-mean cross pair: terms 0 and 2 are the
    // like pairs and term 1's exponential is exactly the square root of their
    // product (its c and lambda are their means), so a node costs two
    // exponentials and a square root instead of three exponentials
    R a0 = (R)0, a1 = (R)0, a2 = (R)0;
#pragma unroll 1
    for (int k = 0; k < 12; ++k) {
      const R e0 = pair_term(P.phi[0], pr[k], s_exp), e2 = pair_term(P.phi[2], pr[k], s_exp);
      a0 += e0 * pw[k];
      a2 += e2 * pw[k];
      a1 += cross_mean(e0, e2) * pw[k];
    }
    put(2 * P.n_f + 0, a0);
    put(2 * P.n_f + 1, a1);
    put(2 * P.n_f + 2, a2);
  } else {
#pragma unroll 1
    for (int u = 0; u < P.n_phi; ++u) {
      R acc = (R)0;
#pragma unroll 1
      for (int k = 0; k < 12; ++k) acc += pair_term(P.phi[u], pr[k], s_exp) * pw[k];
      put(2 * P.n_f + u, acc);
    }
  }
  if (bad) atomicOr(A.flags, kFlagGeometry);
}

// per-site sums of the float-float gathers in float-float on the FP32 pipe (a
// conversion to FP64 per term would load GB300's slow FP64 pipe); the mixed
// and FP64 contexts sum in FP64 (AccD)
struct AccF2 {
  ff v;
  __device__ __forceinline__ void zero() { v = ff(0.f, 0.f); }
  __device__ __forceinline__ void add(ff x) { v = v + x; }
  __device__ __forceinline__ double get() const { return ff_to_double(v); }
  __device__ __forceinline__ void team_reduce(int nl) {
    for (int o = nl >> 1; o > 0; o >>= 1) {
      const ff w(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
      v = v + w;
    }
  }
};

// molar fractions of a neighbour in the accurate passes
template <int S>
__device__ __forceinline__ void load_x(const PassArgs& A, int64_t j, ff x[S]) {
  const float4 X = __ldg(&A.x32[j]), Xl = __ldg(&A.x32lo[j]);
  const float xs[4] = {X.x, X.y, X.z, X.w}, xl[4] = {Xl.x, Xl.y, Xl.z, Xl.w};
#pragma unroll
  for (int k = 0; k < S; ++k) x[k] = ff(xs[k], xl[k]);
}
template <int S>
__device__ __forceinline__ void load_x(const PassArgs& A, int64_t j, double x[S]) {
#pragma unroll
  for (int k = 0; k < S; ++k) x[k] = __ldg(&A.x[k * A.n + j]);
}

template <int S, int NL, typename R, typename Acc>
__global__ void __launch_bounds__(256) k_pair_density(DevPot P, PassArgs A,
                                                      const typename GeoRec<R>::T* __restrict__ buf, GeoLayout GL) {
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc rb[S], ra[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    rb[k].zero();
    ra[k].zero();
  }
  if (active) {
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
#pragma unroll 4
    for (int t = beg + lane; t < end; t += NL) {
      const int64_t j = __ldg(&A.nb_ent[t]) & kIdxMask;
      const typename GeoRec<R>::T* rec = buf + (int64_t)t * GL.ca;  // densities: plane A
      R xj[S];
      load_x<S>(A, j, xj);
#pragma unroll
      for (int k = 0; k < S; ++k) {
        R sb = (R)0, sa = (R)0;
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const int v = P.f_of[k][l];
          if (v < 0) continue;
          sb += xj[l] * GeoRec<R>::get(rec, v);
          sa += xj[l] * GeoRec<R>::get(rec, P.n_f + v);
        }
        rb[k].add(sb);
        ra[k].add(sa);
      }
    }
  }
  if (NL > 1) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      rb[k].team_reduce(NL);
      ra[k].team_reduce(NL);
    }
  }
  // Per-site tail: team lane k < S takes species k (the FP64 square root and
  // divisions then issue once per warp, not S times); the sums are those of
  // team lane 0, so the result does not depend on which lane finishes it.
  // Every lane reaches every shuffle.
  static_assert(S <= 2 && NL >= S, "one team lane per species");
  const int src = (int)(threadIdx.x & 31) - lane;
  double rbar = 0.0, rsum = 0.0;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double wb = __shfl_sync(0xffffffffu, rb[k].get(), src);
    const double wa = __shfl_sync(0xffffffffu, ra[k].get(), src);
    if (lane == k) {
      rbar = wb;
      rsum = wa;
    }
  }
  const int64_t n = A.n;
  const bool mine = active && lane < S;
  float abk = 0.f, bbk = 0.f, lak = 0.f, lbk = 0.f;
  if (mine) {
    const int k = lane;
    const double Ek = (S > 1 && k == 1) ? P.E[S > 1 ? 1 : 0] : P.E[0];
    const double ravg = rsum * (1.0 / 12.0);
    const double xk = A.x[k * n + i];
    double e = 0.0, ak = 0.0, bk = 0.0;
    if (Ek == 0.0) {
      // no embedding energy for this element
    } else if (rbar > kRhoMin) {
      const double sq = sqrt(rbar);
      const double F = -Ek * sq;
      const double dF = -Ek / (2.0 * sq);
      const double d2F = Ek / (4.0 * rbar * sq);
      e = F + dF * (ravg - rbar);
      ak = xk * d2F * (ravg - rbar);
      bk = xk * dF;
    } else {
      atomicOr(A.flags, kFlagGeometry);
    }
    A.rho_bar[k * n + i] = rbar;
    A.rho_avg[k * n + i] = ravg;
    A.e[k * n + i] = e;
    A.a[k * n + i] = ak;
    A.b[k * n + i] = bk;
    abk = (float)ak;
    bbk = (float)bk;
    lak = (float)(ak - (double)abk);
    lbk = (float)(bk - (double)bbk);
  }
  if (A.ab32 == nullptr) return;  // FP64 contexts: no packed records
  // the packed FP32 (a, b) records of both species, written by team lane 0
  float ab[4] = {abk, bbk, 0.f, 0.f}, lo[4] = {lak, lbk, 0.f, 0.f};
  if (S > 1) {
    ab[2] = __shfl_sync(0xffffffffu, abk, src + 1);
    ab[3] = __shfl_sync(0xffffffffu, bbk, src + 1);
    lo[2] = __shfl_sync(0xffffffffu, lak, src + 1);
    lo[3] = __shfl_sync(0xffffffffu, lbk, src + 1);
  }
  if (!active || lane != 0) return;
  A.ab32[2 * i] = make_float4(ab[0], ab[1], ab[2], ab[3]);
  if (A.ab32lo) A.ab32lo[2 * i] = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

template <int S, int NL, typename R, typename Acc>
__global__ void __launch_bounds__(256) k_pair_mu(DevPot P, PassArgs A,
                                                 const typename GeoRec<R>::T* __restrict__ buf, GeoLayout GL) {
  constexpr int PR = GeoPrec<R>::P;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc mu[S], epair;
  epair.zero();
#pragma unroll
  for (int k = 0; k < S; ++k) mu[k].zero();
  if (active) {
    R xi[S];
    load_x<S>(A, i, xi);
    const R inv12 = (R)(1.0 / 12.0);
    const R half = (R)0.5;
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
    for (int t = beg + lane; t < end; t += NL) {
      const int64_t j = __ldg(&A.nb_ent[t]) & kIdxMask;
      const typename GeoRec<R>::T* rec = buf + (int64_t)t * GL.ca;
      // pair terms: plane B when the record is split, else after the densities
      const typename GeoRec<R>::T* recp = GL.cb ? buf + GL.b_off + (int64_t)t * GL.cb : rec + 2 * P.n_f;
      R xj[S];
      load_x<S>(A, j, xj);
      R aj[S], bj[S];
      load_ab(A, j, aj, bj, (SiteData<PR, S>*)nullptr);
      R ep = (R)0;
#pragma unroll
      for (int k = 0; k < S; ++k) {
        R m = (R)0;
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const int u = P.phi_of[k][l];
          if (u >= 0) {
            const R ph = GeoRec<R>::get(recp, u);
            m += xj[l] * ph * inv12;
            ep += xi[k] * xj[l] * ph;
          }
          // density at j of species l from this site holding species k: f_lk
          const int v = P.f_of[l][k];
          if (v >= 0) m += aj[l] * GeoRec<R>::get(rec, v) + bj[l] * GeoRec<R>::get(rec, P.n_f + v) * inv12;
        }
        mu[k].add(m);
      }
      epair.add(half * inv12 * ep);
    }
  }
  if (NL > 1) {
    epair.team_reduce(NL);
#pragma unroll
    for (int k = 0; k < S; ++k) mu[k].team_reduce(NL);
  }
  // Per-site tail on the first S + 2 team lanes, one FP64 logarithm each:
  // lane k < S ln x_k (with the floor of the chemical potential), lane S
  // ln x_v, lane S + 1 ln sigma; x ln x of the mixing entropy reuses them
  // (a separate logarithm only for 0 < x below the floor).  The sums are
  // those of team lane 0; every lane reaches every shuffle.
  static_assert(NL >= S + 2, "one team lane per logarithm");
  const int src = (int)(threadIdx.x & 31) - lane;
  double mk = 0.0;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double w = __shfl_sync(0xffffffffu, mu[k].get(), src);
    if (lane == k) mk = w;
  }
  const int64_t n = A.n;
  double xk = 0.0, xv = 1.0;
  if (active) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double v = A.x[k * n + i];
      xv -= v;
      if (lane == k) xk = v;
    }
  }
  double arg = 1.0;
  if (active) {
    if (lane < S) arg = fmax(xk, kLogFloor);
    else if (lane == S) arg = fmax(xv, kLogFloor);
    else if (lane == S + 1 && A.site_E) arg = A.sigma[i];
  }
  const double L = log(arg);
  const double lv = __shfl_sync(0xffffffffu, L, src + S);
  bool finite = true;
  if (active && lane < S) {
    const double kT = kKB * A.T[i];
    const double m = mk + A.e[lane * n + i];
    finite = isfinite(m);
    if (A.mu_ex) A.mu_ex[lane * n + i] = m;
    if (A.mu) A.mu[lane * n + i] = m + kT * (L - lv);
  }
  if (A.site_E) {
    const double xs = lane < S ? xk : xv;
    double t = 0.0;
    if (active && lane <= S && xs > 0.0) t = xs * (xs >= kLogFloor ? L : log(xs));
    double tk[S + 1];
#pragma unroll
    for (int k = 0; k <= S; ++k) tk[k] = __shfl_sync(0xffffffffu, t, src + k);
    const double Ls = __shfl_sync(0xffffffffu, L, src + S + 1);
    const double ept = __shfl_sync(0xffffffffu, epair.get(), src);
    if (active && lane == 0) {
      const double kT = kKB * A.T[i];
      double mix = 0.0, emb = 0.0;
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const double x = A.x[k * n + i];
        if (x > 0.0) mix += tk[k];
        emb += x * A.e[k * n + i];
      }
      if (xv > 0.0) mix += tk[S];
      const double EV = ept + emb;
      const double Fv = -3.0 * kT * Ls;
      const double Fm = kT * mix;
      A.site_E[i] = EV;
      A.site_E[n + i] = Fv;
      A.site_E[2 * n + i] = Fm;
      finite = finite && isfinite(EV) && isfinite(Fv) && isfinite(Fm);
    }
  }
  if (!finite) atomicOr(A.flags, kFlagNonfinite);
}

// ---------------------------------------------------------------- half-list relaxation passes
// The relaxation's density and force passes, each unordered pair evaluated
// once (PREC 1, 2: FP32 node arithmetic, float4 records; PREC 0: FP64, records
// of four doubles):
//  k_pair_rdensity: f_v(r_ij) and the sum of f_v over the 12 nodes (both
//    symmetric in i, j), weighted by the other site's fractions, written to
//    both entries of the pair;
//  k_gather_rdensity: per site the sums over its row (float-float in PREC 2,
//    FP64 otherwise), then the embedding coefficients (a, b): packed FP32
//    records (PREC 1, 2) or the FP64 arrays (PREC 0);
//  k_pair_rforce: with the pair's weights (x, a, b of both sites) the force
//    on the row-owner site i, F_i = -(d T + U / 12), d = q_j - q_i (the other
//    site receives -F_i: the pair functions are symmetric), and the width
//    derivatives of both sites (over the nodes that move i and those that
//    move j), written to the two entries of the pair;
//  k_gather_rforce: per site the sums over its row, then the thermal term.
struct alignas(32) Dbl4 {
  double x, y, z, w;
};

template <typename R>
struct Rec4;
template <>
struct Rec4<float> {
  using T = float4;
  static __device__ __forceinline__ T make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
  static __device__ __forceinline__ void load(const T* __restrict__ p, float v[4]) {
    const float4 r = __ldg(p);
    v[0] = r.x;
    v[1] = r.y;
    v[2] = r.z;
    v[3] = r.w;
  }
};
template <>
struct Rec4<double> {
  using T = Dbl4;
  static __device__ __forceinline__ T make(double a, double b, double c, double d) { return Dbl4{a, b, c, d}; }
  static __device__ __forceinline__ void load(const T* __restrict__ p, double v[4]) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 r0 = __ldg(q), r1 = __ldg(q + 1);
    v[0] = r0.x;
    v[1] = r0.y;
    v[2] = r1.x;
    v[3] = r1.y;
  }
};

// value type of the relaxation records: FP32 in PREC 2 (float-float sums);
// doubles in PREC 0 and in PREC 1, whose FP32 node values are converted to
// FP64 by the pair kernel (its FP64 pipe is idle) rather than by the gathers
// (bound by the FP64 pipe: a conversion and an add per component)
template <int PREC>
struct RelaxRec {
  using V = double;
};
template <>
struct RelaxRec<2> {
  using V = float;
};

// per-site sums of the relaxation gathers: float-float in PREC 2, FP64 otherwise
template <int PREC>
struct RelaxAcc {
  using T = AccD;
};
template <>
struct RelaxAcc<2> {
  using T = AccFF;
};

template <int PREC, int S, int TAB>
__device__ __forceinline__ void pair_rdensity_one(const DevPot& P, const DevGrid& g0, const PassArgs& A,
                                                const int4* __restrict__ pair_rec, int64_t p,
                                                typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ dens);

// grid-stride over the unordered pairs (a resident grid: see resident_grid)
template <int PREC, int S, int TAB>
__global__ void __launch_bounds__(256) k_pair_rdensity(DevPot P, DevGrid g0, PassArgs A,
                                                       const int4* __restrict__ pair_rec, int64_t npair,
                                                       typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ dens) {
  pdl_wait();
  pdl_trigger();
  if (chunk_halted(A)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npair; p += stride)
    pair_rdensity_one<PREC, S, TAB>(P, g0, A, pair_rec, p, dens);
}

template <int PREC, int S, int TAB>
__device__ __forceinline__ void pair_rdensity_one(const DevPot& P, const DevGrid& g0, const PassArgs& A,
                                                const int4* __restrict__ pair_rec, int64_t p,
                                                typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ dens) {
  using R = typename Traits<PREC>::R;
  using RT = Rec4<typename RelaxRec<PREC>::V>;
  using TB = Tables<TAB>;
  constexpr int NF = S * S;
  PairRef pr_;
  if (!load_pair(A, pair_rec, p, pr_)) return;
  const int64_t i = pr_.i, j = pr_.j;
  const int tp = pr_.tp, tr = pr_.tr;
  const DevGrid gs = site_grid(g0, A.batch, i);
  SiteData<PREC, S> si, sj;
  load_site(A, i, si);
  load_site(A, j, sj);
  R d[3];
  separation(gs, si, sj, pr_.code, d);
  const R s_i = sqrt6<R>() * si.sig, s_j = sqrt6<R>() * sj.sig;
  const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const R near = (R)kRMin + (s_i < s_j ? s_j : s_i);
  R fst[NF], fav[NF];
  {
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
#pragma unroll
    for (int v = 0; v < NF; ++v) {
      fst[v] = v < TB::n_f(P) ? rad_raw(P.f[v], r) * Sw : (R)0;
      fav[v] = (R)0;
    }
  }
#pragma unroll
  for (int site = 0; site < 2; ++site) {
    const R s = site == 0 ? s_i : s_j;
    const R base = D2 + s * s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R tw = (R)2 * s * d[a];
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        const R r2 = pm == 0 ? base + tw : base - tw;
        R r, rinv, Sw, dS;
        r_from_r2(r2, r, rinv);
        sw(P, r, Sw, dS);
#pragma unroll
        for (int v = 0; v < NF; ++v)
          if (v < TB::n_f(P)) fav[v] += rad_raw(P.f[v], r) * Sw;
      }
    }
  }
  int bad = D2 < (R)(kRMin * kRMin);
  if (D2 < near * near) {  // rare: the exact node distances
    for (int site = 0; site < 2; ++site) {
      const R s = site == 0 ? s_i : s_j;
      for (int a = 0; a < 3; ++a) {
        const R base = D2 + s * s, tw = (R)2 * s * d[a];
        bad |= (base + tw) < (R)(kRMin * kRMin);
        bad |= (base - tw) < (R)(kRMin * kRMin);
      }
    }
  }
  // each entry receives its own site's density contributions from the other
  // site: (rho_bar^0, rho_bar^1, <rho>^0, <rho>^1) x 12 for the average
  R ci[4] = {(R)0, (R)0, (R)0, (R)0}, cj[4] = {(R)0, (R)0, (R)0, (R)0};
#pragma unroll
  for (int k = 0; k < S; ++k)
#pragma unroll
    for (int l = 0; l < S; ++l) {
      const int v = TB::f(P, k, l);
#pragma unroll
      for (int w = 0; w < NF; ++w)
        if (v == w) {
          ci[k] += sj.x[l] * fst[w];
          ci[2 + k] += sj.x[l] * fav[w];
          cj[k] += si.x[l] * fst[w];
          cj[2 + k] += si.x[l] * fav[w];
        }
    }
  using RV = typename RelaxRec<PREC>::V;
  dens[tp] = RT::make((RV)ci[0], (RV)ci[1], (RV)ci[2], (RV)ci[3]);
  dens[tr] = RT::make((RV)cj[0], (RV)cj[1], (RV)cj[2], (RV)cj[3]);
  if (bad) atomicOr(A.flags, kFlagGeometry);
}

template <int PREC, int S, int NL>
__global__ void __launch_bounds__(256) k_gather_rdensity(DevPot P, PassArgs A,
                                                         const typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ dens) {
  pdl_wait();
  pdl_trigger();
  using R = typename Traits<PREC>::R;
  using Acc = typename RelaxAcc<PREC>::T;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc rb[S], ra[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    rb[k].zero();
    ra[k].zero();
  }
  if (active) {
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
#pragma unroll 4
    for (int t = beg + lane; t < end; t += NL) {
      typename RelaxRec<PREC>::V rec[4];
      Rec4<typename RelaxRec<PREC>::V>::load(&dens[t], rec);
      rb[0].add(rec[0]);
      ra[0].add(rec[2]);
      if (S > 1) {
        rb[S > 1 ? 1 : 0].add(rec[1]);
        ra[S > 1 ? 1 : 0].add(rec[3]);
      }
    }
  }
  if (NL > 1) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      rb[k].team_reduce(NL);
      ra[k].team_reduce(NL);
    }
  }
  if (!active || lane != 0) return;
  int flag = 0;
  const int64_t n = A.n;
  if constexpr (PREC == 0) {
    // FP64 embedding coefficients, as the FP64 density pass forms them
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double rbar = rb[k].get();
      const double ravg = ra[k].get() * (1.0 / 12.0);
      const double xk = A.x[k * n + i];
      double ak = 0.0, bk = 0.0;
      if (P.E[k] == 0.0) {
        // no embedding energy for this element
      } else if (rbar > kRhoMin) {
        const double sq = sqrt(rbar);
        const double dF = -P.E[k] / (2.0 * sq);
        const double d2F = P.E[k] / (4.0 * rbar * sq);
        ak = xk * d2F * (ravg - rbar);
        bk = xk * dF;
      } else {
        flag |= kFlagGeometry;
      }
      A.a[k * n + i] = ak;
      A.b[k * n + i] = bk;
    }
  } else {
    float ab[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float4 X = A.x32[i];
    const float xs[4] = {X.x, X.y, X.z, X.w};
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const float2 b2 = rb[k].get_pair(), a2 = ra[k].get_pair();
      const float rf = b2.x + b2.y;
      const float df = fmaf(a2.x, 1.0f / 12.0f, -b2.x) + fmaf(a2.y, 1.0f / 12.0f, -b2.y);
      if (P.E[k] == 0.0) {
        // no embedding energy for this element
      } else if (rf > (float)kRhoMin) {
        const float Ef = (float)P.E[k];
        const float isq = rsqrt_approx(rf);
        const float dF = -0.5f * Ef * isq;
        const float d2F = 0.25f * Ef * isq * isq * isq;
        ab[2 * k] = xs[k] * d2F * df;
        ab[2 * k + 1] = xs[k] * dF;
      } else {
        flag |= kFlagGeometry;
      }
    }
    A.ab32[2 * i] = make_float4(ab[0], ab[1], ab[2], ab[3]);
  }
  if (flag) atomicOr(A.flags, flag);
}

template <int PREC, int S, int TAB>
__device__ __forceinline__ void pair_rforce_one(const DevPot& P, const DevGrid& g0, const PassArgs& A,
                                                const int4* __restrict__ pair_rec, int64_t p,
                                                typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ frc);

// one thread per unordered pair (a grid-stride loop here held 48 registers
// against 40 and ran 9 % slower)
template <int PREC, int S, int TAB>
__global__ void __launch_bounds__(256) k_pair_rforce(DevPot P, DevGrid g0, PassArgs A,
                                                       const int4* __restrict__ pair_rec, int64_t npair,
                                                       typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ frc) {
  pdl_wait();
  pdl_trigger();
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < npair) pair_rforce_one<PREC, S, TAB>(P, g0, A, pair_rec, p, frc);
}

template <int PREC, int S, int TAB>
__device__ __forceinline__ void pair_rforce_one(const DevPot& P, const DevGrid& g0, const PassArgs& A,
                                                const int4* __restrict__ pair_rec, int64_t p,
                                                typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ frc) {
  using R = typename Traits<PREC>::R;
  using RT = Rec4<typename RelaxRec<PREC>::V>;
  using TB = Tables<TAB>;
  constexpr int NF = S * S;
  constexpr int NP = S * (S + 1) / 2;
  PairRef pr_;
  if (!load_pair(A, pair_rec, p, pr_)) return;
  const int64_t i = pr_.i, j = pr_.j;
  const int tp = pr_.tp, tr = pr_.tr;
  const DevGrid gs = site_grid(g0, A.batch, i);
  SiteData<PREC, S> si, sj;
  load_site(A, i, si);
  load_site(A, j, sj);
  R ai[S], bi[S], aj[S], bj[S];
  load_ab(A, i, ai, bi, (SiteData<PREC, S>*)nullptr);
  load_ab(A, j, aj, bj, (SiteData<PREC, S>*)nullptr);
  R d[3];
  separation(gs, si, sj, pr_.code, d);
  const R s_i = sqrt6<R>() * si.sig, s_j = sqrt6<R>() * sj.sig;
  const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  R cphi[NP], cfa[NF], cfs[NF];
#pragma unroll
  for (int u = 0; u < NP; ++u) cphi[u] = (R)0;
#pragma unroll
  for (int v = 0; v < NF; ++v) cfa[v] = cfs[v] = (R)0;
#pragma unroll
  for (int k = 0; k < S; ++k)
#pragma unroll
    for (int l = 0; l < S; ++l) {
      // table entries read once (compared inside the unrolled loops they
      // sent a copy of the tables to the stack)
      const int po = TB::phi(P, k, l), fo = TB::f(P, k, l);
#pragma unroll
      for (int u = 0; u < NP; ++u)
        if (po == u) cphi[u] += si.x[k] * sj.x[l];
#pragma unroll
      for (int v = 0; v < NF; ++v)
        if (fo == v) {
          cfa[v] += bi[k] * sj.x[l] + bj[k] * si.x[l];
          cfs[v] += ai[k] * sj.x[l] + aj[k] * si.x[l];
        }
    }
  R clphi[NP], clf[NF];  // weights times decay rates (factored derivative)
#pragma unroll
  for (int u = 0; u < NP; ++u) clphi[u] = cphi[u] * rad_lam(P.phi[u], s_i);
#pragma unroll
  for (int v = 0; v < NF; ++v) clf[v] = cfa[v] * rad_lam(P.f[v], s_i);
  R Gs;
  {
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
    Gs = (R)0;
#pragma unroll
    for (int v = 0; v < NF; ++v)
      if (v < TB::n_f(P)) {
        const R e = rad_raw(P.f[v], r);
        Gs += cfs[v] * (e * (dS - rad_lam(P.f[v], r) * Sw));
      }
    Gs *= rinv;
  }
  R T = (R)0, U[3] = {(R)0, (R)0, (R)0}, Vs[2] = {(R)0, (R)0};
#pragma unroll
  for (int site = 0; site < 2; ++site) {
    const R s = site == 0 ? s_i : s_j;
    const R base = D2 + s * s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R tw = (R)2 * s * d[a];
      R w2[2];
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        const R r2 = pm == 0 ? base + tw : base - tw;
        R r, rinv, Sw, dS;
        r_from_r2(r2, r, rinv);
        sw(P, r, Sw, dS);
        R A1 = (R)0, A2 = (R)0;
        if constexpr (TAB == 2) {
          // power form (FP64): two exponentials, the five terms as products;
          // minus a term's derivative is its rate times the term
          const R c0 = exp(-P.pw_beta[0] * r), c1 = exp(-P.pw_beta[1] * r);
          const R c0_2 = c0 * c0, c1_2 = c1 * c1;
          const R h0 = c0_2 * c0, h1 = c1_2 * c1;
          const R c0_5 = h0 * c0_2, c1_5 = h1 * c1_2;
          const R ephi[3] = {P.pw_pref_phi[0] * (h0 * h0), P.pw_pref_phi[1] * (h0 * h1),
                             P.pw_pref_phi[2] * (h1 * h1)};
          const R ef[2] = {P.pw_pref_f[0] * (c0_5 * c0_5), P.pw_pref_f[1] * (c1_5 * c1_5)};
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            A1 += cphi[u] * ephi[u];
            A2 += clphi[u] * ephi[u];
          }
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            A1 += cfa[v] * ef[v];
            A2 += clf[v] * ef[v];
          }
        } else {
#pragma unroll
        for (int u = 0; u < NP; ++u)
          if (u < TB::n_phi(P)) {
            if constexpr (PREC == 0) {
              double e, mde;  // exponential or Lennard-Jones term and minus its derivative
              rad_pair(P.phi[u], r, e, mde);
              A1 += cphi[u] * e;
              A2 += cphi[u] * mde;
            } else {
              const R e = rad_raw(P.phi[u], r);
              A1 += cphi[u] * e;
              A2 += clphi[u] * e;
            }
          }
#pragma unroll
        for (int v = 0; v < NF; ++v)
          if (v < TB::n_f(P)) {
            const R e = rad_raw(P.f[v], r);
            A1 += cfa[v] * e;
            A2 += clf[v] * e;
          }
        }
        w2[pm] = (A1 * dS - A2 * Sw) * rinv;
      }
      T += w2[0] + w2[1];
      U[a] += s * (w2[0] - w2[1]);
      Vs[site] += sqrt6<R>() * ((d[a] + s) * w2[0] - (d[a] - s) * w2[1]);
    }
  }
  const R inv12 = (R)(1.0 / 12.0);
  const R Tt = T * inv12 + Gs;
  // this entry: the force on i and its width derivative; the reverse entry:
  // the force on j (Newton's third law) and j's width derivative
  const R Fx = -(d[0] * Tt + U[0] * inv12), Fy = -(d[1] * Tt + U[1] * inv12), Fz = -(d[2] * Tt + U[2] * inv12);
  using RV = typename RelaxRec<PREC>::V;
  const RV fx = (RV)Fx, fy = (RV)Fy, fz = (RV)Fz;
  frc[tp] = RT::make(fx, fy, fz, (RV)(Vs[0] * inv12));
  frc[tr] = RT::make(-fx, -fy, -fz, (RV)(Vs[1] * inv12));
}

template <int PREC, int S, int NL>
__global__ void __launch_bounds__(256) k_gather_rforce(PassArgs A,
                                                       const typename Rec4<typename RelaxRec<PREC>::V>::T* __restrict__ frc) {
  pdl_wait();
  pdl_trigger();
  using R = typename Traits<PREC>::R;
  using Acc = typename RelaxAcc<PREC>::T;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  Acc g[3], gsig;
#pragma unroll
  for (int c = 0; c < 3; ++c) g[c].zero();
  gsig.zero();
  if (active) {
    const int beg = A.nb_off[i], end = A.nb_off[i + 1];
#pragma unroll 4
    for (int t = beg + lane; t < end; t += NL) {
      typename RelaxRec<PREC>::V f[4];
      Rec4<typename RelaxRec<PREC>::V>::load(&frc[t], f);
      g[0].add(f[0]);
      g[1].add(f[1]);
      g[2].add(f[2]);
      gsig.add(f[3]);
    }
  }
  if (NL > 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c].team_reduce(NL);
    gsig.team_reduce(NL);
  }
  // Per-site tail: team lanes 0-2 the force components, lane 3 the width
  // derivative with its thermal term, so the conversions and the FP64 division
  // issue once per warp.  After the butterfly every team lane holds the whole
  // sum (a lane's own rounding order: fixed, so runs repeat exactly).
  static_assert(NL >= 4, "one team lane per output");
  if (!active || lane > 3) return;
  const int64_t n = A.n;
  double v;
  if constexpr (PREC == 0) {
    v = lane == 0 ? g[0].get() : lane == 1 ? g[1].get() : lane == 2 ? g[2].get()
                  : gsig.get() - 3.0 * kKB * A.T[i] / A.sigma[i];
  } else {
    float2 h = g[0].get_pair();
    if (lane == 1) h = g[1].get_pair();
    else if (lane == 2) h = g[2].get_pair();
    else if (lane == 3) {
      // FP32 modes: the thermal term in FP32 (no FP64 division)
      const float2 gp = gsig.get_pair();
      const float th = 3.0f * (float)kKB * (float)A.T[i] / (float)A.sigma[i];
      h = make_float2((gp.x - th) + gp.y, 0.f);
    }
    v = (double)h.x + (double)h.y;
  }
  if (lane < 3) {
    if (A.gq) A.gq[lane * n + i] = v;
  } else if (A.gs) {
    A.gs[i] = v;
  }
  if (!isfinite(v)) atomicOr(A.flags, kFlagNonfinite);
}

// ---------------------------------------------------------------- exact embedding average
// App. B.2 (before Eq. F_taylor): the third-degree rule of App. A applied to the
// many-body function F_k(rho_i^k), rho_i^k = sum_{j in J_i} sum_l x_jl f_kl(r_ij),
// over the N_i sites of site i's rule: i and its neighbours J_i closer than
// r_cut at the mean positions.  N_q = 3 N_i, M_i = 2 N_q nodes of weight 1/M_i,
// each moving one site s by +-sigma_s sqrt(N_q) along one axis.  The pair terms
// come from the ordinary passes with the embedding switched off; these two
// passes add the embedding terms.
//  k_emb_nodes (per site i): N_i, rho_bar_i (rule members at the mean), the six
//    densities at the nodes that move i, then over the members j the six nodes
//    that move j (rho = rho_bar - x_j f(r_bar) + x_j f(r_node)): <F_k> and the
//    sum of F_k' over all M_i nodes.
//  k_emb_grad (per site m, a gather): the derivatives of sum_i x_ik <F_k(rho_i^k)>
//    w.r.t. q_m, sigma_m and x_m from m's own rule and from the rule of every
//    member j of J_m (m is a member of J_j): in j's rule only the nodes that
//    move j (densities stored by the first pass) or m (recomputed) change r_jm;
//    every other node leaves r_jm at its mean and contributes F' summed as
//    the stored total minus those twelve.
template <typename R>
struct EmbPrec {
  static constexpr int P = 0;
};
template <>
struct EmbPrec<float> {
  static constexpr int P = 1;
};

// density term f_kl(r) and its derivative
template <typename R>
__device__ __forceinline__ void f_val(const DevPot& P, int v, R r, R Sw, R dS, R& f, R& df) {
  const R e = rad_raw(P.f[v], r);
  f = e * Sw;
  df = e * (dS - rad_lam(P.f[v], r) * Sw);
}

// F_k(rho) = -E_k sqrt(rho) and F_k'(rho)
__device__ __forceinline__ void embed_F(double E, double rho, double& F, double& dF) {
  const double sq = sqrt(rho);
  F = -E * sq;
  dF = -E / (2.0 * sq);
}
__device__ __forceinline__ void embed_F(double E, float rho, double& F, double& dF) {
  const float is = rsqrt_approx(rho);
  F = (double)(-(float)E * rho * is);
  dF = (double)(-0.5f * (float)E * is);
}

template <int S, int NL, typename R>
__global__ void __launch_bounds__(256) k_emb_nodes(DevPot P, DevGrid g0, PassArgs A, EmbArgs E) {
  constexpr int PR = EmbPrec<R>::P;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = i < A.n;
  const R rc2 = (R)(P.rc * P.rc);
  const R rmin2 = (R)(kRMin * kRMin);
  int bad = 0;
  SiteData<PR, S> si;
  DevGrid gs = g0;
  int beg = 0, end = 0;
  if (active) {
    gs = site_grid(g0, A.batch, i);
    load_site(A, i, si);
    beg = A.nb_off[i];
    end = A.nb_off[i + 1];
  }
  // members of the rule
  int cnt = 0;
  for (int t = beg + lane; t < end; t += NL) {
    const uint32_t ent = __ldg(&A.nb_ent[t]);
    SiteData<PR, S> sj;
    load_site(A, ent & kIdxMask, sj);
    R d[3];
    separation(gs, si, sj, ent >> kCodeShift, d);
    cnt += (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < rc2;
  }
  for (int o = NL >> 1; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  const int N = cnt + 1;
  const R hs = sqrt((R)(3 * N));
  const R hi = active ? si.sig * hs : (R)0;
  // densities at the mean and at the six nodes that move i
  double rb[S], ro[S][6];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    rb[k] = 0.0;
#pragma unroll
    for (int v = 0; v < 6; ++v) ro[k][v] = 0.0;
  }
  for (int t = beg + lane; t < end; t += NL) {
    const uint32_t ent = __ldg(&A.nb_ent[t]);
    SiteData<PR, S> sj;
    load_site(A, ent & kIdxMask, sj);
    R d[3];
    separation(gs, si, sj, ent >> kCodeShift, d);
    const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(D2 < rc2)) continue;
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
    bad |= D2 < rmin2;
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int v = P.f_of[k][l];
        if (v < 0) continue;
        R f, df;
        f_val(P, v, r, Sw, dS, f, df);
        rb[k] += (double)(sj.x[l] * f);
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        const R h = pm == 0 ? hi : -hi;  // node: q_i + h e_a, so d_a -> d_a - h
        const R r2 = D2 - (R)2 * h * d[a] + h * h;
        bad |= r2 < rmin2;
        R rn, rinvn, Swn, dSn;
        r_from_r2(r2, rn, rinvn);
        sw(P, rn, Swn, dSn);
#pragma unroll
        for (int k = 0; k < S; ++k)
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const int v = P.f_of[k][l];
            if (v < 0) continue;
            R f, df;
            f_val(P, v, rn, Swn, dSn, f, df);
            ro[k][2 * a + pm] += (double)(sj.x[l] * f);
          }
      }
  }
  for (int o = NL >> 1; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      rb[k] += __shfl_xor_sync(0xffffffffu, rb[k], o);
#pragma unroll
      for (int v = 0; v < 6; ++v) ro[k][v] += __shfl_xor_sync(0xffffffffu, ro[k][v], o);
    }
  }
  // the nodes that move a member j: rho = rho_bar - x_j f(r_bar) + x_j f(r_node)
  double Fs[S], Ts[S];
#pragma unroll
  for (int k = 0; k < S; ++k) Fs[k] = Ts[k] = 0.0;
  double xi[S];
#pragma unroll
  for (int k = 0; k < S; ++k) xi[k] = active ? A.x[k * A.n + i] : 0.0;
  for (int t = beg + lane; t < end; t += NL) {
    const uint32_t ent = __ldg(&A.nb_ent[t]);
    SiteData<PR, S> sj;
    load_site(A, ent & kIdxMask, sj);
    R d[3];
    separation(gs, si, sj, ent >> kCodeShift, d);
    const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(D2 < rc2)) continue;
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
    double base[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
      base[k] = rb[k];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int v = P.f_of[k][l];
        if (v < 0) continue;
        R f, df;
        f_val(P, v, r, Sw, dS, f, df);
        base[k] -= (double)(sj.x[l] * f);
      }
    }
    const R hj = sj.sig * hs;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        const R h = pm == 0 ? hj : -hj;  // node: q_j + h e_a
        const R r2 = D2 + (R)2 * h * d[a] + h * h;
        bad |= r2 < rmin2;
        R rn, rinvn, Swn, dSn;
        r_from_r2(r2, rn, rinvn);
        sw(P, rn, Swn, dSn);
#pragma unroll
        for (int k = 0; k < S; ++k) {
          if (P.E[k] == 0.0) continue;
          double rho = base[k];
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const int v = P.f_of[k][l];
            if (v < 0) continue;
            R f, df;
            f_val(P, v, rn, Swn, dSn, f, df);
            rho += (double)(sj.x[l] * f);
          }
          if (rho > kRhoMin) {
            double F, dF;
            embed_F(P.E[k], (R)rho, F, dF);
            Fs[k] += F;
            Ts[k] += dF;
          } else if (xi[k] > 0.0) {
            bad = 1;
          }
        }
      }
  }
  for (int o = NL >> 1; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Fs[k] += __shfl_xor_sync(0xffffffffu, Fs[k], o);
      Ts[k] += __shfl_xor_sync(0xffffffffu, Ts[k], o);
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (!active || lane != 0) return;
  const int64_t n = A.n;
  const double invM = 1.0 / (6.0 * N);
  double eV = 0.0;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    double F = Fs[k], T = Ts[k];
    if (P.E[k] != 0.0) {
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        if (ro[k][v] > kRhoMin) {
          double Fo, dFo;
          embed_F(P.E[k], (R)ro[k][v], Fo, dFo);
          F += Fo;
          T += dFo;
        } else if (xi[k] > 0.0) {
          bad = 1;
        }
      }
    }
    E.rhob[k * n + i] = rb[k];
#pragma unroll
    for (int v = 0; v < 6; ++v) E.rown[(6 * k + v) * n + i] = ro[k][v];
    E.fsum[k * n + i] = T;
    E.emb[k * n + i] = F * invM;
    eV += xi[k] * F * invM;
  }
  E.nrule[i] = N;
  if (A.site_E) A.site_E[i] += eV;
  if (bad) atomicOr(A.flags, kFlagGeometry);
}

template <int S, int NL, typename R>
__global__ void __launch_bounds__(256) k_emb_grad(DevPot P, DevGrid g0, PassArgs A, EmbArgs E) {
  constexpr int PR = EmbPrec<R>::P;
  if (A.ctrl != nullptr && A.ctrl->halted) return;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t m = tid / NL;
  const int lane = (int)(tid % NL);
  const bool active = m < A.n;
  const int64_t n = A.n;
  const R rc2 = (R)(P.rc * P.rc);
  SiteData<PR, S> sm;
  DevGrid gs = g0;
  int beg = 0, end = 0, Nm = 1;
  double xm[S], rbm[S], wown[S][6];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    xm[k] = rbm[k] = 0.0;
#pragma unroll
    for (int v = 0; v < 6; ++v) wown[k][v] = 0.0;
  }
  if (active) {
    gs = site_grid(g0, A.batch, m);
    load_site(A, m, sm);
    beg = A.nb_off[m];
    end = A.nb_off[m + 1];
    Nm = E.nrule[m];
    const double invM = 1.0 / (6.0 * Nm);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      xm[k] = A.x[k * n + m];
      rbm[k] = E.rhob[k * n + m];
      if (P.E[k] == 0.0) continue;
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        const double ro = E.rown[(6 * k + v) * n + m];
        double F = 0.0, dF = 0.0;
        if (ro > kRhoMin) embed_F(P.E[k], (R)ro, F, dF);
        wown[k][v] = xm[k] * dF * invM;  // weight of the node in d/dq
      }
    }
  }
  const R hsm = sqrt((R)(3 * Nm));
  const R hm = active ? sm.sig * hsm : (R)0;
  const double invMm = 1.0 / (6.0 * Nm);
  // static density gradient G_m^k = sum_{j in J_m} sum_l x_jl f_kl'(r) d / r
  double G[S][3];
#pragma unroll
  for (int k = 0; k < S; ++k) G[k][0] = G[k][1] = G[k][2] = 0.0;
  for (int t = beg + lane; t < end; t += NL) {
    const uint32_t ent = __ldg(&A.nb_ent[t]);
    SiteData<PR, S> sj;
    load_site(A, ent & kIdxMask, sj);
    R d[3];
    separation(gs, sm, sj, ent >> kCodeShift, d);
    const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(D2 < rc2)) continue;
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      R s = (R)0;
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int v = P.f_of[k][l];
        if (v < 0) continue;
        R f, df;
        f_val(P, v, r, Sw, dS, f, df);
        s += sj.x[l] * df;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) G[k][c] += (double)(s * d[c] * rinv);
    }
  }
  for (int o = NL >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) G[k][c] += __shfl_xor_sync(0xffffffffu, G[k][c], o);
  double g[3] = {0.0, 0.0, 0.0}, gsig = 0.0, mu[S], wsum[S];
#pragma unroll
  for (int k = 0; k < S; ++k) mu[k] = wsum[k] = 0.0;
  for (int t = beg + lane; t < end; t += NL) {
    const uint32_t ent = __ldg(&A.nb_ent[t]);
    const int64_t j = ent & kIdxMask;
    SiteData<PR, S> sj;
    load_site(A, j, sj);
    R d[3];  // q_j - q_m
    separation(gs, sm, sj, ent >> kCodeShift, d);
    const R D2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(D2 < rc2)) continue;
    R r, rinv, Sw, dS;
    r_from_r2(D2, r, rinv);
    sw(P, r, Sw, dS);
    // f_kl(r_bar), f_kl'(r_bar) for every species pair
    R fb[S][S], dfb[S][S];
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int l = 0; l < S; ++l) {
        const int v = P.f_of[k][l];
        fb[k][l] = dfb[k][l] = (R)0;
        if (v >= 0) f_val(P, v, r, Sw, dS, fb[k][l], dfb[k][l]);
      }
    // (1) m's rule, the nodes that move m: q_m + h e_a, so d_a -> d_a - h
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        const R h = pm == 0 ? hm : -hm;
        R v3[3] = {d[0], d[1], d[2]};
        v3[a] -= h;
        const R r2 = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
        R rn, rinvn, Swn, dSn;
        r_from_r2(r2, rn, rinvn);
        sw(P, rn, Swn, dSn);
        double w = 0.0;  // sum_k w_own sum_l x_jl f_kl'(r_node) / r_node
#pragma unroll
        for (int k = 0; k < S; ++k) {
          R s = (R)0;
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const int v = P.f_of[k][l];
            if (v < 0) continue;
            R f, df;
            f_val(P, v, rn, Swn, dSn, f, df);
            s += sj.x[l] * df;
          }
          w += wown[k][2 * a + pm] * (double)(s * rinvn);
        }
        // d rho / d q_m = -sum x f' v / r;  d/dsigma_m along a: times +-sqrt(N_q)
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] -= w * (double)v3[c];
        gsig -= w * (double)v3[a] * (double)(pm == 0 ? hsm : -hsm);
      }
    // (2) m's rule, the nodes that move j: q_j + h e_a, h = sigma_j sqrt(3 N_m)
    {
      const R hj = sj.sig * hsm;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int pm = 0; pm < 2; ++pm) {
          const R h = pm == 0 ? hj : -hj;
          R v3[3] = {d[0], d[1], d[2]};
          v3[a] += h;
          const R r2 = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
          R rn, rinvn, Swn, dSn;
          r_from_r2(r2, rn, rinvn);
          sw(P, rn, Swn, dSn);
#pragma unroll
          for (int k = 0; k < S; ++k) {
            if (P.E[k] == 0.0) continue;
            double rho = rbm[k];
            R sn = (R)0, sb = (R)0;
#pragma unroll
            for (int l = 0; l < S; ++l) {
              const int v = P.f_of[k][l];
              if (v < 0) continue;
              R f, df;
              f_val(P, v, rn, Swn, dSn, f, df);
              rho += (double)(sj.x[l] * (f - fb[k][l]));
              sn += sj.x[l] * df;
              sb += sj.x[l] * dfb[k][l];
            }
            double F = 0.0, dF = 0.0;
            if (rho > kRhoMin) embed_F(P.E[k], (R)rho, F, dF);
            const double w = xm[k] * dF * invMm;
            wsum[k] += w;  // times -G_m^k after the row
            // + x_j f'(r_bar) d / r_bar - x_j f'(r_node) v / r_node
#pragma unroll
            for (int c = 0; c < 3; ++c) g[c] += w * (double)(sb * d[c] * rinv - sn * v3[c] * rinvn);
          }
        }
    }
    // j's rule (m is a member): its data from the first pass
    const int Nj = E.nrule[j];
    const R hsj = sqrt((R)(3 * Nj));
    const double invMj = 1.0 / (6.0 * Nj);
    double xj[S];
#pragma unroll
    for (int k = 0; k < S; ++k) xj[k] = A.x[k * n + j];
#pragma unroll
    for (int k = 0; k < S; ++k) {
      if (P.E[k] == 0.0 || xj[k] == 0.0) continue;
      double used = 0.0;  // F' of the twelve nodes handled here
      // (3) the nodes that move j: q_j + h e_a; from m's side the separation
      // q_m - q_j(node) = -(d + h e_a), so r from d_a + h
      const R hjj = sj.sig * hsj;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int pm = 0; pm < 2; ++pm) {
          const R h = pm == 0 ? hjj : -hjj;
          R v3[3] = {-d[0], -d[1], -d[2]};  // q_m - q_j at the node
          v3[a] -= h;
          const R r2 = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
          R rn, rinvn, Swn, dSn;
          r_from_r2(r2, rn, rinvn);
          sw(P, rn, Swn, dSn);
          const double ro = E.rown[(6 * k + 2 * a + pm) * n + j];
          double F = 0.0, dF = 0.0;
          if (ro > kRhoMin) embed_F(P.E[k], (R)ro, F, dF);
          used += dF;
          const double w = xj[k] * dF * invMj;
          R sn = (R)0;
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const int v = P.f_of[k][l];
            if (v < 0) continue;
            R f, df;
            f_val(P, v, rn, Swn, dSn, f, df);
            sn += (R)xm[l] * df;
            mu[l] += w * (double)f;
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) g[c] += w * (double)(sn * v3[c] * rinvn);
        }
      // (4) the nodes that move m in j's rule: q_m + h e_a, h = sigma_m sqrt(3 N_j)
      const double rbj = E.rhob[k * n + j];
      const R hmj = sm.sig * hsj;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int pm = 0; pm < 2; ++pm) {
          const R h = pm == 0 ? hmj : -hmj;
          R v3[3] = {-d[0], -d[1], -d[2]};
          v3[a] += h;
          const R r2 = v3[0] * v3[0] + v3[1] * v3[1] + v3[2] * v3[2];
          R rn, rinvn, Swn, dSn;
          r_from_r2(r2, rn, rinvn);
          sw(P, rn, Swn, dSn);
          double rho = rbj;
          R sn = (R)0;
          R fn[S];
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const int v = P.f_of[k][l];
            fn[l] = (R)0;
            if (v < 0) continue;
            R f, df;
            f_val(P, v, rn, Swn, dSn, f, df);
            fn[l] = f;
            rho += xm[l] * (double)(f - fb[k][l]);
            sn += (R)xm[l] * df;
          }
          double F = 0.0, dF = 0.0;
          if (rho > kRhoMin) embed_F(P.E[k], (R)rho, F, dF);
          used += dF;
          const double w = xj[k] * dF * invMj;
#pragma unroll
          for (int l = 0; l < S; ++l) mu[l] += w * (double)fn[l];
#pragma unroll
          for (int c = 0; c < 3; ++c) g[c] += w * (double)(sn * v3[c] * rinvn);
          gsig += w * (double)(sn * v3[a] * rinvn) * (double)(pm == 0 ? hsj : -hsj);
        }
      // (5) every other node of j's rule: r_jm at its mean
      const double w = xj[k] * (E.fsum[k * n + j] - used) * invMj;
      R sb = (R)0;
#pragma unroll
      for (int l = 0; l < S; ++l) {
        sb += (R)xm[l] * dfb[k][l];
        mu[l] += w * (double)fb[k][l];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] -= w * (double)(sb * d[c] * rinv);
    }
  }
  for (int o = NL >> 1; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] += __shfl_xor_sync(0xffffffffu, g[c], o);
    gsig += __shfl_xor_sync(0xffffffffu, gsig, o);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      mu[k] += __shfl_xor_sync(0xffffffffu, mu[k], o);
      wsum[k] += __shfl_xor_sync(0xffffffffu, wsum[k], o);
    }
  }
  if (!active || lane != 0) return;
#pragma unroll
  for (int k = 0; k < S; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] -= wsum[k] * G[k][c];
  bool finite = isfinite(g[0]) && isfinite(g[1]) && isfinite(g[2]) && isfinite(gsig);
  if (A.gq) {
#pragma unroll
    for (int c = 0; c < 3; ++c) A.gq[c * n + m] += g[c];
  }
  if (A.gs) A.gs[m] += gsig;
  if (A.mu_ex || A.mu) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const double v = mu[k] + E.emb[k * n + m];
      finite = finite && isfinite(v);
      if (A.mu_ex) A.mu_ex[k * n + m] += v;
      if (A.mu) A.mu[k * n + m] += v;
    }
  }
  if (!finite) atomicOr(A.flags, kFlagNonfinite);
}

// ---------------------------------------------------------------- K7: pack
__global__ void k_pack(const double* __restrict__ q, const double* __restrict__ sigma, const double* __restrict__ x,
                       const int* __restrict__ abs_cell, int64_t n, int S, DevGrid g0, Batch B,
                       float4* __restrict__ pos32, float4* __restrict__ x32, float4* __restrict__ pos32lo,
                       float4* __restrict__ x32lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DevGrid g = site_grid(g0, B, i);
  double pd[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) pd[a] = q[a * n + i] - (double)abs_cell[a * n + i] * g.h[a];
  pd[3] = sigma[i];
  float p[4], pl[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    p[a] = (float)pd[a];
    pl[a] = (float)(pd[a] - (double)p[a]);
  }
  pos32[i] = make_float4(p[0], p[1], p[2], p[3]);
  float xs[4] = {0, 0, 0, 0}, xl[4] = {0, 0, 0, 0};
  for (int k = 0; k < S && k < 4; ++k) {
    const double xv = x[k * n + i];
    xs[k] = (float)xv;
    xl[k] = (float)(xv - (double)xs[k]);
  }
  x32[i] = make_float4(xs[0], xs[1], xs[2], xs[3]);
  if (pos32lo) {
    pos32lo[i] = make_float4(pl[0], pl[1], pl[2], pl[3]);
    x32lo[i] = make_float4(xl[0], xl[1], xl[2], xl[3]);
  }
}

// FP64 embedding coefficients -> the packed FP32 records the FP32 gradient pass gathers
__global__ void k_pack_ab(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int S,
                          float4* __restrict__ ab32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < S && k < 4; ++k) {
    v[2 * k] = (float)a[k * n + i];
    v[2 * k + 1] = (float)b[k * n + i];
  }
  ab32[2 * i] = make_float4(v[0], v[1], v[2], v[3]);
  if (S > 2) ab32[2 * i + 1] = make_float4(v[4], v[5], v[6], v[7]);
}

// ---------------------------------------------------------------- K6: energy totals
// Fixed grouping (kReduceGroup sites per partial, fixed tree inside a group,
// groups summed in order by one block), so the totals do not depend on any
// launch shape.
__global__ void k_energy_partials(const double* __restrict__ site_E, int64_t n, int64_t ngroups,
                                  double* __restrict__ partials) {
  __shared__ double sh[3][kReduceGroup / 4];
  const int64_t grp = blockIdx.x;
  const int tid = threadIdx.x;  // blockDim = kReduceGroup / 4
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    for (int r = 0; r < 4; ++r) {
      int64_t i = grp * kReduceGroup + r * (kReduceGroup / 4) + tid;
      if (i < n) v += site_E[c * n + i];
    }
    sh[c][tid] = v;
  }
  __syncthreads();
  for (int w = kReduceGroup / 8; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid == 0)
    for (int c = 0; c < 3; ++c) partials[c * ngroups + grp] = sh[c][0];
}

__global__ void k_energy_final(const double* __restrict__ partials, int64_t ngroups, double* __restrict__ F4) {
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
  if (tid == 0) {
    F4[0] = sh[0][0];
    F4[1] = sh[1][0];
    F4[2] = sh[2][0];
    F4[3] = (sh[0][0] + sh[1][0]) + sh[2][0];
  }
}

// Batches: one block per system sums its own sites with a fixed stride and
// tree, F4 laid out [nsys][4].
__global__ void __launch_bounds__(256) k_energy_seg(const double* __restrict__ site_E, int64_t n,
                                                    const int* __restrict__ sys_off, double* __restrict__ F4) {
  __shared__ double sh[3][256];
  const int sys = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t beg = sys_off[sys], end = sys_off[sys + 1];
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    for (int64_t i = beg + tid; i < end; i += 256) v += site_E[c * n + i];
    sh[c][tid] = v;
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c][tid] += sh[c][tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    double* o = F4 + 4 * (int64_t)sys;
    o[0] = sh[0][0];
    o[1] = sh[1][0];
    o[2] = sh[2][0];
    o[3] = (sh[0][0] + sh[1][0]) + sh[2][0];
  }
}

template <int PREC, int S, int NL>
cudaError_t launch_density_t(const DevPot& P, const DevGrid& g, const PassArgs& a, cudaStream_t s) {
  const int threads = a.tpb > 0 ? a.tpb : 256;
  const int64_t work = a.n * NL;
  k_density<PREC, S, NL><<<(unsigned)((work + threads - 1) / threads), threads, 0, s>>>(P, g, a);
  return cudaGetLastError();
}
template <int PREC, int S, int NL>
cudaError_t launch_gradient_t(int mode, const DevPot& P, const DevGrid& g, const PassArgs& a, cudaStream_t s) {
  const int threads = a.tpb > 0 ? a.tpb : 256;
  const int64_t work = a.n * NL;
  const unsigned blocks = (unsigned)((work + threads - 1) / threads);
  if constexpr (PREC == 3) {  // float-float: chemical potentials and energies only
    if (mode != kGradMu) return cudaErrorInvalidValue;
    k_gradient<3, S, NL, kGradMu><<<blocks, threads, 0, s>>>(P, g, a);
  } else if constexpr (PREC == 0) {
    if (mode == kGradForce)
      k_gradient<0, S, NL, kGradForce><<<blocks, threads, 0, s>>>(P, g, a);
    else if (mode == kGradForceNoE)
      k_gradient<0, S, NL, kGradForceNoE><<<blocks, threads, 0, s>>>(P, g, a);
    else if (mode == kGradAll)
      k_gradient<0, S, NL, kGradAll><<<blocks, threads, 0, s>>>(P, g, a);
    else
      k_gradient<0, S, NL, kGradMu><<<blocks, threads, 0, s>>>(P, g, a);
  } else {  // FP32 node arithmetic: forces (and energies)
    if (mode == kGradForce)
      k_gradient<PREC, S, NL, kGradForce><<<blocks, threads, 0, s>>>(P, g, a);
    else if (mode == kGradForceNoE)
      k_gradient<PREC, S, NL, kGradForceNoE><<<blocks, threads, 0, s>>>(P, g, a);
    else
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// mode < 0: density pass; otherwise the gradient pass in that mode
template <int PREC, int S>
cudaError_t dispatch_nl(int mode, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a, cudaStream_t s) {
  switch (nl) {
    case 4: return mode >= 0 ? launch_gradient_t<PREC, S, 4>(mode, P, g, a, s) : launch_density_t<PREC, S, 4>(P, g, a, s);
    case 8: return mode >= 0 ? launch_gradient_t<PREC, S, 8>(mode, P, g, a, s) : launch_density_t<PREC, S, 8>(P, g, a, s);
    case 16:
      return mode >= 0 ? launch_gradient_t<PREC, S, 16>(mode, P, g, a, s) : launch_density_t<PREC, S, 16>(P, g, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int PREC>
cudaError_t dispatch_s(int mode, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a, cudaStream_t s) {
  switch (P.S) {
    case 1: return dispatch_nl<PREC, 1>(mode, nl, P, g, a, s);
    case 2: return dispatch_nl<PREC, 2>(mode, nl, P, g, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch(int mode, int precision, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a,
                     cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.tpb < 0 || a.tpb > 256 || a.tpb % 32 != 0) return cudaErrorInvalidValue;
  switch (precision) {
    case 0: return dispatch_s<0>(mode, nl, P, g, a, s);
    case 1: return dispatch_s<1>(mode, nl, P, g, a, s);
    case 2: return dispatch_s<2>(mode, nl, P, g, a, s);
    case 3: return dispatch_s<3>(mode, nl, P, g, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_pack(const double* q, const double* sigma, const double* x, const int* abs_cell, int64_t n,
                        int S, const DevGrid& g, const Batch& B, float4* pos32, float4* x32, float4* pos32lo,
                        float4* x32lo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, sigma, x, abs_cell, n, S, g, B, pos32, x32, pos32lo, x32lo);
  return cudaGetLastError();
}

cudaError_t launch_density(int precision, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a,
                           cudaStream_t s) {
  return dispatch(-1, precision, nl, P, g, a, s);
}

cudaError_t launch_gradient(int precision, int mode, int nl, const DevPot& P, const DevGrid& g, const PassArgs& a,
                            cudaStream_t s) {
  return dispatch(mode, precision, nl, P, g, a, s);
}

cudaError_t launch_pack_ab(const double* a, const double* b, int64_t n, int S, float4* ab32, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_pack_ab<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n, S, ab32);
  return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const double* site_E, int64_t n, double* partials, double* F4, cudaStream_t s) {
  int64_t ng = (n + kReduceGroup - 1) / kReduceGroup;
  if (ng < 1) ng = 1;
  k_energy_partials<<<(unsigned)ng, kReduceGroup / 4, 0, s>>>(site_E, n, ng, partials);
  k_energy_final<<<1, 256, 0, s>>>(partials, ng, F4);
  return cudaGetLastError();
}

cudaError_t launch_energy_seg(const double* site_E, int64_t n, const Batch& B, double* F4, cudaStream_t s) {
  if (B.nsys <= 0) return cudaSuccess;
  k_energy_seg<<<(unsigned)B.nsys, 256, 0, s>>>(site_E, n, B.sys_off, F4);
  return cudaGetLastError();
}

namespace {
bool geo_split(const DevPot& P) { return 2 * P.n_f + P.n_phi > 4; }
}  // namespace
int pair_record_len(const DevPot& P) {
  if (geo_split(P)) return ((2 * P.n_f + 3) & ~3) + ((P.n_phi + 3) & ~3);
  return (2 * P.n_f + P.n_phi + 3) & ~3;
}
GeoLayout geo_layout(const DevPot& P, int64_t cap) {
  if (!geo_split(P)) return GeoLayout{pair_record_len(P), 0, 0};
  const int ca = (2 * P.n_f + 3) & ~3;
  return GeoLayout{ca, (P.n_phi + 3) & ~3, cap * ca};
}

// threads per block of the pair kernels: the unordered pairs one block takes
int pair_threads(const PassArgs& A) { return A.pair_tpb == 64 || A.pair_tpb == 256 ? A.pair_tpb : 128; }

namespace {
template <typename R>
cudaError_t pair_geo_t(const DevPot& P, const DevGrid& g, const PassArgs& A, const int4* pair_rec, int64_t npair,
                       void* buf, int64_t cap, cudaStream_t s) {
  const GeoLayout C = geo_layout(P, cap);
  const int pt = pair_threads(A);
  const unsigned blocks = (unsigned)((npair + pt - 1) / pt);
  using T = typename GeoRec<R>::T;
  switch (P.S) {
    case 1: k_pair_geo<1, R, 0><<<blocks, pt, 0, s>>>(P, g, A, pair_rec, npair, (T*)buf, C); break;
    case 2:
      if (P.pw_on && P.pw_m[0] == 6 && P.pw_n[0] == 10 && P.pw_m[1] == 6 && P.pw_n[1] == 10)
        k_pair_geo<2, R, 1><<<blocks, pt, 0, s>>>(P, g, A, pair_rec, npair, (T*)buf, C);
      else if (P.pw_on)
        k_pair_geo<2, R, 2><<<blocks, pt, 0, s>>>(P, g, A, pair_rec, npair, (T*)buf, C);
      else
        k_pair_geo<2, R, 0><<<blocks, pt, 0, s>>>(P, g, A, pair_rec, npair, (T*)buf, C);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_pair_geo(int precision, const DevPot& P, const DevGrid& g, const PassArgs& A,
                            const int4* pair_rec, int64_t npair, void* buf, int64_t cap, cudaStream_t s) {
  if (npair == 0) return cudaSuccess;
  if (precision == 0) return pair_geo_t<double>(P, g, A, pair_rec, npair, buf, cap, s);
  if (P.lj) return cudaErrorInvalidValue;  // Lennard-Jones terms: FP64 passes only
  return pair_geo_t<ff>(P, g, A, pair_rec, npair, buf, cap, s);
}

namespace {
template <int S, int NL, typename R, typename Acc>
cudaError_t pair_gather_t(bool mu, const DevPot& P, const PassArgs& A, const void* buf, GeoLayout C, cudaStream_t s) {
  const int threads = A.tpb > 0 ? A.tpb : 256;
  const unsigned blocks = (unsigned)((A.n * NL + threads - 1) / threads);
  using T = typename GeoRec<R>::T;
  if (mu) k_pair_mu<S, NL, R, Acc><<<blocks, threads, 0, s>>>(P, A, (const T*)buf, C);
  else k_pair_density<S, NL, R, Acc><<<blocks, threads, 0, s>>>(P, A, (const T*)buf, C);
  return cudaGetLastError();
}
template <int S, int NL>
cudaError_t pair_gather_p(int precision, bool mu, const DevPot& P, const PassArgs& A, const void* buf, GeoLayout C,
                          cudaStream_t s) {
  switch (precision) {
    case 0: return pair_gather_t<S, NL, double, AccD>(mu, P, A, buf, C, s);
    case 1: return pair_gather_t<S, NL, ff, AccD>(mu, P, A, buf, C, s);
    case 2: return pair_gather_t<S, NL, ff, AccF2>(mu, P, A, buf, C, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int S>
cudaError_t pair_gather_s(int precision, bool mu, int nl, const DevPot& P, const PassArgs& A, const void* buf, GeoLayout C,
                          cudaStream_t s) {
  switch (nl) {
    case 4: return pair_gather_p<S, 4>(precision, mu, P, A, buf, C, s);
    case 8: return pair_gather_p<S, 8>(precision, mu, P, A, buf, C, s);
    case 16: return pair_gather_p<S, 16>(precision, mu, P, A, buf, C, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_pair_gather(int precision, bool mu, int nl, const DevPot& P, const PassArgs& A, const void* buf,
                               int64_t cap, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  const GeoLayout C = geo_layout(P, cap);
  switch (P.S) {
    case 1: return pair_gather_s<1>(precision, mu, nl, P, A, buf, C, s);
    case 2: return pair_gather_s<2>(precision, mu, nl, P, A, buf, C, s);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
template <int PREC, int S, int NL>
cudaError_t relax_gather_t(bool force, const DevPot& P, const PassArgs& A, const void* dens, const void* frc,
                           cudaStream_t s) {
  using T = typename Rec4<typename RelaxRec<PREC>::V>::T;
  const int threads = A.tpb > 0 ? A.tpb : 256;
  const unsigned blocks = (unsigned)((A.n * NL + threads - 1) / threads);
  if (force) return launch_pdl(k_gather_rforce<PREC, S, NL>, dim3(blocks), dim3(threads), 0, s, A, (const T*)frc);
  return launch_pdl(k_gather_rdensity<PREC, S, NL>, dim3(blocks), dim3(threads), 0, s, P, A, (const T*)dens);
}
template <int PREC, int S>
cudaError_t relax_gather_s(bool force, int nl, const DevPot& P, const PassArgs& A, const void* dens, const void* frc,
                           cudaStream_t s) {
  switch (nl) {
    case 4: return relax_gather_t<PREC, S, 4>(force, P, A, dens, frc, s);
    case 8: return relax_gather_t<PREC, S, 8>(force, P, A, dens, frc, s);
    case 16: return relax_gather_t<PREC, S, 16>(force, P, A, dens, frc, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int PREC>
cudaError_t relax_gather_p(bool force, int nl, const DevPot& P, const PassArgs& A, const void* dens, const void* frc,
                           cudaStream_t s) {
  if (P.S == 1) return relax_gather_s<PREC, 1>(force, nl, P, A, dens, frc, s);
  return relax_gather_s<PREC, 2>(force, nl, P, A, dens, frc, s);
}
template <int PREC>
cudaError_t relax_pair_p(bool force, const DevPot& P, const DevGrid& g, const PassArgs& A, const int4* pair_rec,
                         int64_t npair, void* dens, void* frc, cudaStream_t s) {
  using T = typename Rec4<typename RelaxRec<PREC>::V>::T;
  const int pt = pair_threads(A);
  // the density pass strides over a resident grid in a single system; the
  // force pass, and every pass of a batch (a stride would take each thread
  // across systems, reloading a system's grid per pair: 55 -> 62 ms per
  // ensemble step), take one thread per pair
  auto run = [&](auto kernel, T* out, bool resident) {
    const int64_t blocks = resident ? resident_grid((const void*)kernel, pt, npair) : (npair + pt - 1) / pt;
    if (blocks < 0 || blocks > 0x7fffffff) return cudaErrorInvalidValue;
    return launch_pdl(kernel, dim3((unsigned)blocks), dim3(pt), 0, s, P, g, A, pair_rec, npair, out);
  };
  if (force) {
    if (P.S == 1) return run(k_pair_rforce<PREC, 1, 0>, (T*)frc, false);
    if constexpr (PREC == 0) {
      if (P.tab == 1 && P.pw_on && P.pw_m[0] == 6 && P.pw_n[0] == 10 && P.pw_m[1] == 6 && P.pw_n[1] == 10)
        return run(k_pair_rforce<PREC, 2, 2>, (T*)frc, false);
    }
    if (P.tab == 1) return run(k_pair_rforce<PREC, 2, 1>, (T*)frc, false);
    return run(k_pair_rforce<PREC, 2, 0>, (T*)frc, false);
  }
  if (P.S == 1) return run(k_pair_rdensity<PREC, 1, 0>, (T*)dens, A.batch.nsys == 0);
  if (P.tab == 1) return run(k_pair_rdensity<PREC, 2, 1>, (T*)dens, A.batch.nsys == 0);
  return run(k_pair_rdensity<PREC, 2, 0>, (T*)dens, A.batch.nsys == 0);
}
}  // namespace

namespace {
template <int S, int NL, typename R>
cudaError_t emb_t(bool second, const DevPot& P, const DevGrid& g, const PassArgs& A, const EmbArgs& E,
                  cudaStream_t s) {
  const int threads = A.tpb > 0 ? A.tpb : 256;
  const unsigned blocks = (unsigned)((A.n * NL + threads - 1) / threads);
  if (second) k_emb_grad<S, NL, R><<<blocks, threads, 0, s>>>(P, g, A, E);
  else k_emb_nodes<S, NL, R><<<blocks, threads, 0, s>>>(P, g, A, E);
  return cudaGetLastError();
}
template <int S, typename R>
cudaError_t emb_nl(bool second, int nl, const DevPot& P, const DevGrid& g, const PassArgs& A, const EmbArgs& E,
                   cudaStream_t s) {
  switch (nl) {
    case 4: return emb_t<S, 4, R>(second, P, g, A, E, s);
    case 8: return emb_t<S, 8, R>(second, P, g, A, E, s);
    case 16: return emb_t<S, 16, R>(second, P, g, A, E, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_emb_exact(bool second, bool fp64, int nl, const DevPot& P, const DevGrid& g, const PassArgs& A,
                             const EmbArgs& E, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  if (P.S == 1) return fp64 ? emb_nl<1, double>(second, nl, P, g, A, E, s) : emb_nl<1, float>(second, nl, P, g, A, E, s);
  if (P.S == 2) return fp64 ? emb_nl<2, double>(second, nl, P, g, A, E, s) : emb_nl<2, float>(second, nl, P, g, A, E, s);
  return cudaErrorInvalidValue;
}

bool pair_kernels_supported(const DevPot& P) { return P.S <= 2 && P.n_f <= 2; }

int64_t resident_grid(const void* kernel, int threads, int64_t work_items) {
  struct Entry {
    const void* k;
    int threads, device, blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  int wave = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
      if (e.k == kernel && e.threads == threads && e.device == dev) wave = e.blocks;
    if (wave == 0) {
      int per_sm = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
      wave = std::max(per_sm, 1) * std::max(sms, 1);
      cache.push_back(Entry{kernel, threads, dev, wave});
    }
  }
  const int64_t need = (work_items + threads - 1) / threads;
  return std::max<int64_t>(1, std::min<int64_t>(need, wave));
}

size_t relax_record_bytes(int precision) { return precision == 2 ? sizeof(float4) : sizeof(Dbl4); }

cudaError_t launch_relax_pair(int precision, bool force, const DevPot& P, const DevGrid& g, const PassArgs& A,
                              const int4* pair_rec, int64_t npair, void* dens, void* frc, cudaStream_t s) {
  if (A.n == 0 || npair == 0) return cudaSuccess;
  if (!pair_kernels_supported(P)) return cudaErrorInvalidValue;
  switch (precision) {
    case 0: return relax_pair_p<0>(force, P, g, A, pair_rec, npair, dens, frc, s);
    case 1: return relax_pair_p<1>(force, P, g, A, pair_rec, npair, dens, frc, s);
    case 2: return relax_pair_p<2>(force, P, g, A, pair_rec, npair, dens, frc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_relax_gather(int precision, bool force, int nl, const DevPot& P, const PassArgs& A,
                                const void* dens, const void* frc, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  if (!pair_kernels_supported(P)) return cudaErrorInvalidValue;
  switch (precision) {
    case 0: return relax_gather_p<0>(force, nl, P, A, dens, frc, s);
    case 1: return relax_gather_p<1>(force, nl, P, A, dens, frc, s);
    case 2: return relax_gather_p<2>(force, nl, P, A, dens, frc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mxe
