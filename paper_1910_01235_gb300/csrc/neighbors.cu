// neighbors.cu -- K1: cell-list neighbour and bond builder (Sec. 4, Algorithm 1,
// neighbour-list step; Sec. 3: the transport sum runs over nearest neighbours).
//
// Membership is decided in FP64 with explicitly rounded operations (no FMA):
//   d_a = (q_ja - q_ia) - L_a rint((q_ja - q_ia) * invL_a),  |d|^2 = (dx dx + dy dy) + dz dz
// so the set is bit-reproducible against any IEEE evaluation of the same rule.
// GB300 runs FP64 at 1/73 of the FP32 rate, so every candidate is first tested
// in FP32 from rounded positions; only a candidate whose FP32 |d|^2 lies
// inside a rigorous error band around the cutoff is decided by the FP64 rule
// (the band bounds the position rounding, the image choice and the rounding
// of |d|^2; outside it the FP32 and FP64 decisions agree).
// One warp handles one site: lanes sweep the candidates of the distinct
// neighbouring cells, accepted entries are compacted into shared memory with
// ballots and placed in j order (a bitonic sort in registers; rank counting
// for rows longer than 128).  Each entry stores j in the
// low 27 bits and the periodic image code (cell offset in {-1,0,1}^3) above it,
// which the FP32 kernels use to rebuild d from cell-relative positions.
#include <cuda_runtime.h>

#include "mxe_internal.cuh"

namespace mxe {
namespace {

__global__ void k_cell_assign(const double* __restrict__ q, int64_t n, DevGrid g0, Batch B, int* __restrict__ cell_of,
                              int* __restrict__ cell_slot, int* __restrict__ cell_count, int* __restrict__ abs_cell,
                              float4* __restrict__ qf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DevGrid g = site_grid(g0, B, i);
  const int base = B.nsys ? B.cell_base[B.sys_of[i]] : 0;
  qf[i] = make_float4((float)q[i], (float)q[n + i], (float)q[2 * n + i], 0.f);
  int c3[3];
  float rel[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double u = q[a * n + i] * g.invL[a];
    double w = floor(u);
    int c = (int)((u - w) * g.nc[a]);
    c = c < 0 ? 0 : (c >= g.nc[a] ? g.nc[a] - 1 : c);
    c3[a] = c;
    const int ac = (int)w * g.nc[a] + c;
    abs_cell[a * n + i] = ac;
    rel[a] = (float)(q[a * n + i] - (double)ac * g.h[a]);  // position within its cell
  }
  qf[n + i] = make_float4(rel[0], rel[1], rel[2], 0.f);
  int cell = base + (c3[0] * g.nc[1] + c3[1]) * g.nc[2] + c3[2];
  cell_of[i] = cell;
  cell_slot[i] = atomicAdd(&cell_count[cell], 1);
}

__global__ void k_cell_place(int64_t n, const int* __restrict__ cell_of, const int* __restrict__ cell_slot,
                             const int* __restrict__ cell_start, int* __restrict__ cell_sites) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  cell_sites[cell_start[cell_of[i]] + cell_slot[i]] = (int)i;
}

// The distinct cells of the 3x3x3 stencil around `cell` (duplicates removed
// when an axis has fewer than 3 cells).
struct Stencil {
  int off[3][3];
  int cnt[3];
};

__device__ __forceinline__ Stencil make_stencil(int cell, const DevGrid& g) {
  Stencil st;
  int c3[3] = {cell / (g.nc[1] * g.nc[2]), (cell / g.nc[2]) % g.nc[1], cell % g.nc[2]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    st.cnt[a] = 0;
    for (int o = -1; o <= 1; ++o) {
      int v = ((c3[a] + o) % g.nc[a] + g.nc[a]) % g.nc[a];
      bool dup = false;
      for (int t = 0; t < st.cnt[a]; ++t) dup |= st.off[a][t] == v;
      if (!dup) st.off[a][st.cnt[a]++] = v;
    }
  }
  return st;
}

struct PairTest {
  double r2;
  double k[3];
};

__device__ __forceinline__ PairTest pair_test(const double qi[3], const double* __restrict__ q, int64_t n, int j,
                                              const DevGrid& g) {
  PairTest t;
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double da = __dsub_rn(q[a * n + j], qi[a]);
    double k = rint(__dmul_rn(da, g.invL[a]));
    d[a] = __dsub_rn(da, __dmul_rn(g.L[a], k));
    t.k[a] = k;
  }
  t.r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return t;
}

// FP32 estimate of the minimum-image |d|^2 and image counts
struct PairTestF {
  float r2;
  float k[3];
  bool near_half;  // a component near half a box length: take the FP64 image
};

__device__ __forceinline__ PairTestF pair_test_f(const float4& qi, const float4& qj, const DevGrid& g) {
  PairTestF t;
  const float dq[3] = {qj.x - qi.x, qj.y - qi.y, qj.z - qi.z};
  float r2 = 0.f;
  t.near_half = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float u = dq[a] * g.invL_f[a];
    const float k = rintf(u);
    const float d = fmaf(-g.L_f[a], k, dq[a]);
    t.near_half |= fabsf(u - k) > 0.45f;
    t.k[a] = k;
    r2 = fmaf(d, d, r2);
  }
  t.r2 = r2;
  return t;
}

// Decision for one cutoff: 1 inside, 0 outside, -1 undecided in FP32.
__device__ __forceinline__ int decide_f(float r2f, float cut2f, float band) {
  if (r2f < cut2f - band) return 1;
  if (r2f > cut2f + band) return 0;
  return -1;
}

__global__ void k_nbr_count(const double* __restrict__ q, const float4* __restrict__ qf,
                            const uint8_t* __restrict__ sub, uint32_t mobile_mask, int64_t n, DevGrid g0, Batch B,
                            const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                            const int* __restrict__ cell_sites, double rl2, double rb2, float band,
                            int* __restrict__ nb_cnt, int* __restrict__ bd_cnt, int* __restrict__ max_row) {
  const int lane = threadIdx.x & 31;
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double qi[3] = {q[i], q[n + i], q[2 * n + i]};
  const float4 qfi = qf[i];
  const float rl2f = (float)rl2, rb2f = (float)rb2;
  int si = sub ? sub[i] : 0;
  bool mob = (mobile_mask >> si) & 1u;
  const DevGrid g = site_grid(g0, B, i);
  const int base = B.nsys ? B.cell_base[B.sys_of[i]] : 0;
  Stencil st = make_stencil(cell_of[i] - base, g);
  int cnt = 0, bcnt = 0;
  for (int ax = 0; ax < st.cnt[0]; ++ax)
    for (int ay = 0; ay < st.cnt[1]; ++ay)
      for (int az = 0; az < st.cnt[2]; ++az) {
        int c = base + (st.off[0][ax] * g.nc[1] + st.off[1][ay]) * g.nc[2] + st.off[2][az];
        int beg = cell_start[c], end = cell_start[c + 1];
        for (int t0 = beg; t0 < end; t0 += 32) {
          int t = t0 + lane;
          bool in = false, bond = false;
          if (t < end) {
            int j = cell_sites[t];
            if (j != (int)i) {
              const PairTestF pf = pair_test_f(qfi, __ldg(&qf[j]), g);
              int din = decide_f(pf.r2, rl2f, band);
              int dbo = decide_f(pf.r2, rb2f, band);
              if (din < 0 || (din > 0 && dbo < 0)) {
                const PairTest pt = pair_test(qi, q, n, j, g);
                din = pt.r2 < rl2;
                dbo = pt.r2 < rb2;
              }
              in = din > 0;
              int sj = sub ? sub[j] : 0;
              bond = in && mob && sj == si && dbo > 0;
            }
          }
          cnt += __popc(__ballot_sync(0xffffffffu, in));
          bcnt += __popc(__ballot_sync(0xffffffffu, bond));
        }
      }
  if (lane == 0) {
    nb_cnt[i] = cnt;
    bd_cnt[i] = bcnt;
    atomicMax(max_row, cnt);
  }
}

__global__ void k_nbr_fill(const double* __restrict__ q, const float4* __restrict__ qf,
                           const uint8_t* __restrict__ sub, uint32_t mobile_mask, int64_t n, DevGrid g0, Batch B,
                           const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                           const int* __restrict__ cell_sites, const int* __restrict__ abs_cell, double rl2,
                           double rb2, float band, const int* __restrict__ nb_off, uint32_t* __restrict__ nb_ent,
                           const int* __restrict__ bd_off, int* __restrict__ bd_idx, int max_row) {
  extern __shared__ unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint32_t* buf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * max_row;
  uint8_t* isb = reinterpret_cast<uint8_t*>(reinterpret_cast<uint32_t*>(smem) + (size_t)(blockDim.x >> 5) * max_row) +
                 (size_t)warp * max_row;
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double qi[3] = {q[i], q[n + i], q[2 * n + i]};
  const float4 qfi = qf[i];
  const float rl2f = (float)rl2, rb2f = (float)rb2;
  int Ai[3] = {abs_cell[i], abs_cell[n + i], abs_cell[2 * n + i]};
  int si = sub ? sub[i] : 0;
  bool mob = (mobile_mask >> si) & 1u;
  const DevGrid g = site_grid(g0, B, i);
  const int base = B.nsys ? B.cell_base[B.sys_of[i]] : 0;
  Stencil st = make_stencil(cell_of[i] - base, g);
  int m = 0;
  for (int ax = 0; ax < st.cnt[0]; ++ax)
    for (int ay = 0; ay < st.cnt[1]; ++ay)
      for (int az = 0; az < st.cnt[2]; ++az) {
        int c = base + (st.off[0][ax] * g.nc[1] + st.off[1][ay]) * g.nc[2] + st.off[2][az];
        int beg = cell_start[c], end = cell_start[c + 1];
        for (int t0 = beg; t0 < end; t0 += 32) {
          int t = t0 + lane;
          bool in = false, bond = false;
          uint32_t ent = 0;
          if (t < end) {
            int j = cell_sites[t];
            if (j != (int)i) {
              const PairTestF pf = pair_test_f(qfi, __ldg(&qf[j]), g);
              int din = decide_f(pf.r2, rl2f, band);
              int dbo = decide_f(pf.r2, rb2f, band);
              float kk[3] = {pf.k[0], pf.k[1], pf.k[2]};
              if (din < 0 || (din > 0 && (dbo < 0 || pf.near_half))) {
                const PairTest pt = pair_test(qi, q, n, j, g);
                din = pt.r2 < rl2;
                dbo = pt.r2 < rb2;
                kk[0] = (float)pt.k[0];
                kk[1] = (float)pt.k[1];
                kk[2] = (float)pt.k[2];
              }
              in = din > 0;
              if (in) {
                int sj = sub ? sub[j] : 0;
                bond = mob && sj == si && dbo > 0;
                int code = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  int s = abs_cell[a * n + j] - Ai[a] - g.nc[a] * (int)kk[a];
                  s = s < -1 ? -1 : (s > 1 ? 1 : s);
                  code = code * 3 + (s + 1);
                }
                ent = (uint32_t)j | ((uint32_t)code << kCodeShift);
              }
            }
          }
          unsigned msk = __ballot_sync(0xffffffffu, in);
          if (in) {
            int pos = m + __popc(msk & ((1u << lane) - 1u));
            if (pos < max_row) {
              buf[pos] = ent;
              isb[pos] = bond ? 1 : 0;
            }
          }
          m += __popc(msk);
        }
      }
  __syncwarp();
  if (m > max_row) m = max_row;  // cannot happen: max_row is the counted maximum
  const int off = nb_off[i];
  const int boff = bd_off[i];
  for (int e = lane; e < m; e += 32) {
    uint32_t je = buf[e] & kIdxMask;
    int rank = 0, brank = 0;
    for (int f = 0; f < m; ++f) {
      uint32_t jf = buf[f] & kIdxMask;
      int less = jf < je;
      rank += less;
      brank += less & isb[f];
    }
    nb_ent[off + rank] = buf[e];
    if (isb[e]) bd_idx[boff + brank] = (int)je;
  }
}

// ---------------------------------------------------------------- cell-staged build
// One block per cell: the block stages the candidates of the cell's distinct
// stencil cells (FP32 position, index) in shared memory once, then each warp
// takes one home site of the cell at a time and tests it against the staged
// candidates with the same rule as above.  The warp-per-site kernels above are
// the fallback when a stencil holds more candidates than shared memory fits.
constexpr int kCellThreads = 128;

struct CellStage {
  int ncand;
  // Every axis has >= 3 cells of width >= r_list: then a pair within r_list
  // has one image, that of the stencil cell, and the staged candidates carry
  // their image code (cj = j | code << kCodeShift) and their position in the
  // home cell's frame (cell-relative position + offset x cell width).
  bool fast;
};

__device__ __forceinline__ CellStage stage_cell(int cell, int base, const DevGrid& g, int64_t n,
                                                const int* __restrict__ cell_start,
                                                const int* __restrict__ cell_sites, const float4* __restrict__ qf,
                                                float4* cq, int* cj, int* s_off, int* s_beg, float* s_sh,
                                                int cand_cap, int* __restrict__ flags) {
  const bool fast = g.nc[0] >= 3 && g.nc[1] >= 3 && g.nc[2] >= 3;
  if (threadIdx.x < 32) {
    // one stencil cell per lane (its first site and count; lanes past the
    // stencil count nothing), then an exclusive scan of the counts: the
    // cells' loads are in flight together
    const int lane = threadIdx.x;
    const Stencil st = make_stencil(cell - base, g);
    const int n1 = st.cnt[1], n2 = st.cnt[2], nk = st.cnt[0] * n1 * n2;
    int cntk = 0;
    if (lane < nk) {
      const int ax = lane / (n1 * n2), ay = (lane / n2) % n1, az = lane % n2;
      const int c = base + (st.off[0][ax] * g.nc[1] + st.off[1][ay]) * g.nc[2] + st.off[2][az];
      const int b0 = cell_start[c];
      s_beg[lane] = b0;
      cntk = cell_start[c + 1] - b0;
      // without duplicates index t of an axis is the offset t - 1, and k the image code
      s_sh[3 * lane + 0] = (float)(ax - 1) * g.h_f[0];
      s_sh[3 * lane + 1] = (float)(ay - 1) * g.h_f[1];
      s_sh[3 * lane + 2] = (float)(az - 1) * g.h_f[2];
    }
    int incl = cntk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane < 28) s_off[lane] = incl - cntk;  // lanes >= nk: the total
  }
  __syncthreads();
  int ncand = s_off[27];
  if (ncand > cand_cap) {  // cannot happen: cand_cap is the measured maximum
    if (threadIdx.x == 0) atomicOr(flags, kFlagOverflow);
    ncand = cand_cap;
  }
  // the candidates' indices, then their positions: the loads of each pass do
  // not depend on one another, so a thread has all of its candidates' loads
  // in flight (a thread reads back only what it wrote)
#pragma unroll 4
  for (int t = threadIdx.x; t < ncand; t += blockDim.x) {
    int k = 0;
    while (t >= s_off[k + 1]) ++k;
    const int j = cell_sites[s_beg[k] + (t - s_off[k])];
    cj[t] = fast ? (int)((uint32_t)j | ((uint32_t)k << kCodeShift)) : j;
  }
#pragma unroll 4
  for (int t = threadIdx.x; t < ncand; t += blockDim.x) {
    const uint32_t e = (uint32_t)cj[t];
    const int j = (int)(e & kIdxMask);
    if (fast) {
      const int k = (int)(e >> kCodeShift);
      const float4 r = qf[n + j];
      cq[t] = make_float4(r.x + s_sh[3 * k], r.y + s_sh[3 * k + 1], r.z + s_sh[3 * k + 2], 0.f);
    } else {
      cq[t] = qf[j];
    }
  }
  __syncthreads();
  return CellStage{ncand, fast};
}

// Decisions for home site i against staged candidate t (FP64 rule inside the band).
struct CandResult {
  bool in, bond;
  float k[3];
};

__device__ __forceinline__ CandResult test_cand(int64_t i, const double qi[3], const float4& qfi, int j,
                                                const float4& qfj, const double* __restrict__ q, int64_t n,
                                                const DevGrid& g, float rl2f, float rb2f, float band, double rl2,
                                                double rb2, bool mob, int si, const uint8_t* __restrict__ sub,
                                                bool need_k) {
  CandResult r{false, false, {0.f, 0.f, 0.f}};
  if (j == (int)i) return r;
  const PairTestF pf = pair_test_f(qfi, qfj, g);
  int din = decide_f(pf.r2, rl2f, band);
  int dbo = decide_f(pf.r2, rb2f, band);
  r.k[0] = pf.k[0];
  r.k[1] = pf.k[1];
  r.k[2] = pf.k[2];
  if (din < 0 || (din > 0 && (dbo < 0 || (need_k && pf.near_half)))) {
    const PairTest pt = pair_test(qi, q, n, j, g);
    din = pt.r2 < rl2;
    dbo = pt.r2 < rb2;
    r.k[0] = (float)pt.k[0];
    r.k[1] = (float)pt.k[1];
    r.k[2] = (float)pt.k[2];
  }
  r.in = din > 0;
  if (r.in && mob) {
    const int sj = sub ? sub[j] : 0;
    r.bond = sj == si && dbo > 0;
  }
  return r;
}

// The same decisions from home-frame FP32 positions (CellStage::fast): the
// image is the stencil cell's, so no image search; FP64 inside the band.
__device__ __forceinline__ CandResult test_cand_rel(int64_t i, const double qi[3], const float4& ri, int j,
                                                    const float4& rj, const double* __restrict__ q, int64_t n,
                                                    const DevGrid& g, float rl2f, float rb2f, float band, double rl2,
                                                    double rb2, bool mob, int si, const uint8_t* __restrict__ sub) {
  CandResult r{false, false, {0.f, 0.f, 0.f}};
  if (j == (int)i) return r;
  const float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  int din = decide_f(r2, rl2f, band);
  int dbo = decide_f(r2, rb2f, band);
  if (din < 0 || (din > 0 && dbo < 0)) {
    const PairTest pt = pair_test(qi, q, n, j, g);
    din = pt.r2 < rl2;
    dbo = pt.r2 < rb2;
  }
  r.in = din > 0;
  if (r.in && mob) {
    const int sj = sub ? sub[j] : 0;
    r.bond = sj == si && dbo > 0;
  }
  return r;
}

// Row order by a bitonic sort in registers: KPL keys per lane (32 KPL >= m),
// element e = 32 h + lane in register h.  A key packs the entry's j, its image
// code and its bond flag, (j << 6) | (code << 1) | bond, so the sort by key is
// the sort by j (j is unique in a row); it needs j < 2^26.  Pads (e >= m) are
// 0xFFFFFFFF and sort last.  The sorted entries go to ent_out[0, m) and the
// bonds, in the same order, to bond_out (ballot-compacted).
constexpr int64_t kSortKeySites = (int64_t)1 << 26;

template <int KPL>
__device__ __forceinline__ void warp_sort_row(const uint32_t* __restrict__ buf, const uint32_t* __restrict__ kw, int m,
                                              int lane, uint32_t* __restrict__ ent_out,
                                              int* __restrict__ bond_out) {
  uint32_t v[KPL];
#pragma unroll
  for (int h = 0; h < KPL; ++h) {
    const int e = 32 * h + lane;
    v[h] = 0xFFFFFFFFu;
    if (e < m) {
      const uint32_t ent = buf[e];
      v[h] = ((ent & kIdxMask) << 6) | ((ent >> kCodeShift) << 1) | (kw[e] & 1u);
    }
  }
#pragma unroll
  for (int k = 2; k <= 32 * KPL; k <<= 1) {
#pragma unroll
    for (int s = k >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
        // partner in the same lane, register h ^ (s / 32)
#pragma unroll
        for (int h = 0; h < KPL; ++h) {
          const int hp = h ^ (s / 32);
          if (hp > h) {
            const bool asc = ((32 * h + lane) & k) == 0;
            const uint32_t lo = min(v[h], v[hp]), hi = max(v[h], v[hp]);
            v[h] = asc ? lo : hi;
            v[hp] = asc ? hi : lo;
          }
        }
      } else {
        const bool lower = (lane & s) == 0;
#pragma unroll
        for (int h = 0; h < KPL; ++h) {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, v[h], s);
          const bool asc = ((32 * h + lane) & k) == 0;
          v[h] = (asc == lower) ? min(v[h], o) : max(v[h], o);
        }
      }
    }
  }
  int nb = 0;
#pragma unroll
  for (int h = 0; h < KPL; ++h) {
    const int e = 32 * h + lane;
    const uint32_t key = v[h];
    const uint32_t j = key >> 6;
    if (e < m) ent_out[e] = j | (((key >> 1) & 31u) << kCodeShift);
    const bool bond = e < m && (key & 1u);
    const unsigned bm = __ballot_sync(0xffffffffu, bond);
    if (bond) bond_out[nb + __popc(bm & ((1u << lane) - 1u))] = (int)j;
    nb += __popc(bm);
  }
}

__global__ void __launch_bounds__(kCellThreads) k_cell_count(
    const double* __restrict__ q, const float4* __restrict__ qf, const uint8_t* __restrict__ sub, uint32_t mobile_mask,
    int64_t n, DevGrid g0, Batch B, const int* __restrict__ cell_start, const int* __restrict__ cell_sites, double rl2,
    double rb2, float band, int cand_cap, int* __restrict__ nb_cnt, int* __restrict__ bd_cnt,
    int* __restrict__ max_row, int* __restrict__ flags) {
  extern __shared__ unsigned char smem[];
  __shared__ int s_off[28], s_beg[27];
  __shared__ float s_sh[27 * 3];
  float4* cq = reinterpret_cast<float4*>(smem);
  int* cj = reinterpret_cast<int*>(cq + cand_cap);
  const int cell = blockIdx.x;
  const int hbeg = cell_start[cell], hend = cell_start[cell + 1];
  if (hbeg == hend) return;  // uniform over the block
  const int sys = B.nsys ? B.cell_sys[cell] : 0;
  const DevGrid g = B.nsys ? B.grids[sys] : g0;
  const int base = B.nsys ? B.cell_base[sys] : 0;
  __shared__ int s_rowmax;  // the block's longest row: one global atomic per block
  if (threadIdx.x == 0) s_rowmax = 0;
  const CellStage cs =
      stage_cell(cell, base, g, n, cell_start, cell_sites, qf, cq, cj, s_off, s_beg, s_sh, cand_cap, flags);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float rl2f = (float)rl2, rb2f = (float)rb2;
  for (int h = hbeg + warp; h < hend; h += nwarps) {
    const int64_t i = cell_sites[h];
    const double qi[3] = {q[i], q[n + i], q[2 * n + i]};
    const float4 qfi = cs.fast ? qf[n + i] : qf[i];
    const int si = sub ? sub[i] : 0;
    const bool mob = (mobile_mask >> si) & 1u;
    int cnt = 0, bcnt = 0;
    for (int t0 = 0; t0 < cs.ncand; t0 += 32) {
      const int t = t0 + lane;
      CandResult r{false, false, {0.f, 0.f, 0.f}};
      if (t < cs.ncand) {
        const int j = (int)((uint32_t)cj[t] & kIdxMask);
        r = cs.fast ? test_cand_rel(i, qi, qfi, j, cq[t], q, n, g, rl2f, rb2f, band, rl2, rb2, mob, si, sub)
                    : test_cand(i, qi, qfi, j, cq[t], q, n, g, rl2f, rb2f, band, rl2, rb2, mob, si, sub, false);
      }
      cnt += __popc(__ballot_sync(0xffffffffu, r.in));
      bcnt += __popc(__ballot_sync(0xffffffffu, r.bond));
    }
    if (lane == 0) {
      nb_cnt[i] = cnt;
      bd_cnt[i] = bcnt;
      atomicMax(&s_rowmax, cnt);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(max_row, s_rowmax);
}

// DIRECT: no count pass before: row i goes to nb_ent[i * max_row ...] (max_row
// = the stride, from the previous build) with its counts in nb_cnt / bd_cnt
// and the longest row in *row_max; a row longer than the stride is cut and
// its true length reported, so the caller can fall back to count + fill.
template <bool DIRECT>
__global__ void __launch_bounds__(kCellThreads, 8) k_cell_fill(
    const double* __restrict__ q, const float4* __restrict__ qf, const uint8_t* __restrict__ sub, uint32_t mobile_mask,
    int64_t n, DevGrid g0, Batch B, const int* __restrict__ cell_start, const int* __restrict__ cell_sites,
    const int* __restrict__ abs_cell, double rl2, double rb2, float band, int cand_cap,
    const int* __restrict__ nb_off, uint32_t* __restrict__ nb_ent, const int* __restrict__ bd_off,
    int* __restrict__ bd_idx, int max_row, int* __restrict__ nb_cnt, int* __restrict__ bd_cnt,
    int* __restrict__ n_below, int* __restrict__ pair_cnt, int* __restrict__ row_max, int* __restrict__ flags) {
  extern __shared__ unsigned char smem[];
  __shared__ int s_off[28], s_beg[27];
  __shared__ float s_sh[27 * 3];
  float4* cq = reinterpret_cast<float4*>(smem);
  int* cj = reinterpret_cast<int*>(cq + cand_cap);
  const int cell = blockIdx.x;
  const int hbeg = cell_start[cell], hend = cell_start[cell + 1];
  if (hbeg == hend) return;
  const int sys = B.nsys ? B.cell_sys[cell] : 0;
  const DevGrid g = B.nsys ? B.grids[sys] : g0;
  const int base = B.nsys ? B.cell_base[sys] : 0;
  // the longest row of the block, then one global maximum per block (a global
  // atomic per site serialises 256,000 updates of one word)
  __shared__ int s_rowmax;
  if (threadIdx.x == 0) s_rowmax = 0;
  const CellStage cs =
      stage_cell(cell, base, g, n, cell_start, cell_sites, qf, cq, cj, s_off, s_beg, s_sh, cand_cap, flags);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // per warp: the row's entries and its sort keys (j << 1 | bond), 16-byte aligned
  const int stride = (max_row + 3) & ~3;
  uint32_t* rows = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(cj + cand_cap) + 15) & ~uintptr_t(15));
  uint32_t* buf = rows + (size_t)warp * stride;
  uint32_t* kw = rows + (size_t)(nwarps + warp) * stride;
  // Octant lists (home-frame stencils): cells are at least r_list wide, so a
  // home site in the lower half of its cell along an axis has no neighbour
  // beyond 1.5 cell widths on that axis, and one in the upper half none below
  // -0.5; list o holds the candidates the home sites of octant o can reach
  // (about (5/6)^3 of the stencil).  The cut has a margin of 1e-4 h against
  // the FP32 rounding of the home-frame positions (below 1e-6 h); the row
  // order is set by the sort below, so the lists' order does not matter.
  uint16_t* olist = reinterpret_cast<uint16_t*>(rows + (size_t)2 * nwarps * stride);
  __shared__ int s_ocnt[8];
  if (threadIdx.x < 8) s_ocnt[threadIdx.x] = 0;
  __syncthreads();
  if (cs.fast) {
    float lo_cut[3], hi_cut[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo_cut[a] = 1.5f * g.h_f[a] + 1e-4f * g.h_f[a];
      hi_cut[a] = -0.5f * g.h_f[a] - 1e-4f * g.h_f[a];
    }
    for (int t = threadIdx.x; t < cs.ncand; t += blockDim.x) {
      const float4 u = cq[t];
      const bool lo_x = u.x < lo_cut[0], lo_y = u.y < lo_cut[1], lo_z = u.z < lo_cut[2];
      const bool hi_x = u.x >= hi_cut[0], hi_y = u.y >= hi_cut[1], hi_z = u.z >= hi_cut[2];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const bool need = ((o & 4) ? hi_x : lo_x) && ((o & 2) ? hi_y : lo_y) && ((o & 1) ? hi_z : lo_z);
        if (need) olist[o * cand_cap + atomicAdd(&s_ocnt[o], 1)] = (uint16_t)t;
      }
    }
    __syncthreads();
  }
  const float rl2f = (float)rl2, rb2f = (float)rb2;
  for (int h = hbeg + warp; h < hend; h += nwarps) {
    const int64_t i = cell_sites[h];
    const double qi[3] = {q[i], q[n + i], q[2 * n + i]};
    const float4 qfi = cs.fast ? qf[n + i] : qf[i];
    const int si = sub ? sub[i] : 0;
    const bool mob = (mobile_mask >> si) & 1u;
    int m = 0, nbond = 0, nlow = 0;
    const int oct = cs.fast ? ((qfi.x >= 0.5f * g.h_f[0]) << 2) | ((qfi.y >= 0.5f * g.h_f[1]) << 1) |
                                  (int)(qfi.z >= 0.5f * g.h_f[2])
                            : 0;
    const int nc = cs.fast ? s_ocnt[oct] : cs.ncand;
    const uint16_t* ol = olist + oct * cand_cap;
    for (int t0 = 0; t0 < nc; t0 += 32) {
      const int tt = t0 + lane;
      CandResult r{false, false, {0.f, 0.f, 0.f}};
      uint32_t ent = 0;
      int j = 0;
      if (tt < nc) {
        const int t = cs.fast ? (int)ol[tt] : tt;
        ent = (uint32_t)cj[t];
        j = (int)(ent & kIdxMask);
        r = cs.fast ? test_cand_rel(i, qi, qfi, j, cq[t], q, n, g, rl2f, rb2f, band, rl2, rb2, mob, si, sub)
                    : test_cand(i, qi, qfi, j, cq[t], q, n, g, rl2f, rb2f, band, rl2, rb2, mob, si, sub, true);
      }
      if (r.in && !cs.fast) {
        int code = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          int sh = abs_cell[a * n + j] - abs_cell[a * n + i] - g.nc[a] * (int)r.k[a];
          sh = sh < -1 ? -1 : (sh > 1 ? 1 : sh);
          code = code * 3 + (sh + 1);
        }
        ent = (uint32_t)j | ((uint32_t)code << kCodeShift);
      }
      const unsigned msk = __ballot_sync(0xffffffffu, r.in);
      if (r.in) {
        const int pos = m + __popc(msk & ((1u << lane) - 1u));
        if (pos < max_row) {
          buf[pos] = ent;
          kw[pos] = ((uint32_t)j << 1) | (r.bond ? 1u : 0u);
        }
      }
      m += __popc(msk);
      if (DIRECT) {
        nbond += __popc(__ballot_sync(0xffffffffu, r.bond));
        if (n_below) nlow += __popc(__ballot_sync(0xffffffffu, r.in && (int64_t)j < i));
      }
    }
    if (DIRECT && lane == 0) {
      nb_cnt[i] = m;
      bd_cnt[i] = nbond;
      if (n_below) {  // the half-list index: entries below i, pairs owned by i
        n_below[i] = nlow;
        pair_cnt[i] = m - nlow;
      }
      atomicMax(&s_rowmax, m);
    }
    if (m > max_row) m = max_row;  // count + fill: cannot happen (max_row is the counted maximum)
    __syncwarp();
    const int64_t off = DIRECT ? i * (int64_t)max_row : (int64_t)nb_off[i];
    const int64_t boff = DIRECT ? i * (int64_t)max_row : (int64_t)bd_off[i];
    if (m <= 64 && n <= kSortKeySites) {
      warp_sort_row<2>(buf, kw, m, lane, nb_ent + off, bd_idx + boff);
      __syncwarp();
      continue;
    }
    if (m <= 128 && n <= kSortKeySites) {
      warp_sort_row<4>(buf, kw, m, lane, nb_ent + off, bd_idx + boff);
      __syncwarp();
      continue;
    }
    // longer rows: rank counting against the row
    const int m4 = (m + 3) >> 2;
    for (int e = m + lane; e < 4 * m4; e += 32) kw[e] = 0xFFFFFFFFu;  // pads rank after every key
    __syncwarp();
    const uint4* k4 = reinterpret_cast<const uint4*>(kw);
    for (int e = lane; e < m; e += 32) {
      const uint32_t ke = kw[e] & ~1u;  // j << 1: keys of smaller j are below it
      int rank = 0, brank = 0;
      for (int f = 0; f < m4; ++f) {
        const uint4 v = k4[f];
        const uint32_t l0 = v.x < ke, l1 = v.y < ke, l2 = v.z < ke, l3 = v.w < ke;
        rank += (int)(l0 + l1 + l2 + l3);
        brank += (int)((l0 & v.x) + (l1 & v.y) + (l2 & v.z) + (l3 & v.w));
      }
      nb_ent[off + rank] = buf[e];
      if (kw[e] & 1u) bd_idx[boff + brank] = (int)(ke >> 1);
    }
    __syncwarp();
  }
  if (DIRECT) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(row_max, s_rowmax);
  }
}

// Largest number of candidates of any cell's stencil.
__global__ void k_cand_max(int64_t ncell, DevGrid g0, Batch B, const int* __restrict__ cell_start,
                           int* __restrict__ out) {
  const int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c0 >= ncell) return;
  const int sys = B.nsys ? B.cell_sys[c0] : 0;
  const DevGrid g = B.nsys ? B.grids[sys] : g0;
  const int base = B.nsys ? B.cell_base[sys] : 0;
  const Stencil st = make_stencil((int)c0 - base, g);
  int tot = 0;
  for (int ax = 0; ax < st.cnt[0]; ++ax)
    for (int ay = 0; ay < st.cnt[1]; ++ay)
      for (int az = 0; az < st.cnt[2]; ++az) {
        const int c = base + (st.off[0][ax] * g.nc[1] + st.off[1][ay]) * g.nc[2] + st.off[2][az];
        tot += cell_start[c + 1] - cell_start[c];
      }
  atomicMax(out, tot);
}

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanBlock = kScanThreads * kScanPer;

__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int64_t n,
                              long long* __restrict__ block_tot) {
  __shared__ long long warp_tot[kScanThreads / 32];
  int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x * kScanPer;
  long long v[kScanPer];
  long long run = 0;
#pragma unroll
  for (int t = 0; t < kScanPer; ++t) {
    long long x = (base + t < n) ? in[base + t] : 0;
    v[t] = run;
    run += x;
  }
  // exclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  long long wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
  long long excl = wbase + incl - run;
#pragma unroll
  for (int t = 0; t < kScanPer; ++t)
    if (base + t < n) out[base + t] = (int)(excl + v[t]);
  if (threadIdx.x == kScanThreads - 1) block_tot[blockIdx.x] = excl + run;
}

// Exclusive scan of the block totals by one block of kScanThreads threads:
// chunks of kScanThreads totals, each scanned with warp shuffles and the
// warps' sums, carried from chunk to chunk (nblk is n / 2048: a few chunks).
__global__ void __launch_bounds__(kScanThreads) k_scan_tops(long long* __restrict__ block_tot, int64_t nblk,
                                                             long long* __restrict__ total64) {
  __shared__ long long warp_sum[kScanThreads / 32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nblk; c0 += kScanThreads) {
    const int64_t b = c0 + threadIdx.x;
    const long long v = b < nblk ? block_tot[b] : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    long long before = carry;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    if (b < nblk) block_tot[b] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total64 = carry;
}

__global__ void k_scan_add(int* __restrict__ out, int64_t n, const long long* __restrict__ block_tot,
                           const long long* __restrict__ total64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)((long long)out[i] + block_tot[i / kScanBlock]);
  if (i == n) out[n] = (int)(*total64);
}

__global__ void k_strip(const uint32_t* __restrict__ ent, int32_t* __restrict__ idx, int64_t m) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) idx[t] = (int32_t)(ent[t] & kIdxMask);
}

// out[0] = max sigma, out[1] = max |q| component (maxima of non-negative doubles =
// maxima of their bit patterns; warp maximum, then one atomic per warp)
__device__ __forceinline__ void warp_max_bits(unsigned long long* addr, double v) {
  unsigned long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
    b = y > b ? y : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(addr, b);
}

__global__ void k_site_max(const double* __restrict__ sigma, const double* __restrict__ q, int64_t n,
                           unsigned long long* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double vs = 0.0, vq = 0.0;
  if (i < n) {
    vs = fmax(sigma[i], 0.0);
    vq = fmax(fabs(q[i]), fmax(fabs(q[n + i]), fabs(q[2 * n + i])));
    if (!(vq <= 1e300)) vq = 1e300;  // NaN / Inf positions
  }
  warp_max_bits(&out[0], vs);
  warp_max_bits(&out[1], vq);
}

inline unsigned grid_for(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

// segment of each index by binary search over the segment starts (empty
// segments share their start with the next one and are skipped)
__global__ void k_segment_ids(const int* __restrict__ base, int nseg, int64_t count, int* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int lo = 0, hi = nseg - 1;  // invariant: base[lo] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)base[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  out[t] = lo;
}

// ---------------------------------------------------------------- pair index
// Rows are sorted by j, so the entries of row i with j > i (each unordered
// pair once, in the row of its lower-index site) are the tail of the row.
__device__ __forceinline__ int first_above(const uint32_t* __restrict__ ent, int beg, int end, uint32_t i) {
  int lo = beg, hi = end;  // first t in [beg, end) with (ent[t] & mask) > i
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((ent[mid] & kIdxMask) > i) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// n_below[i]: the length of row i's head (entries below i); cnt[i]: of its tail
__global__ void k_pair_count(const int* __restrict__ nb_off, const uint32_t* __restrict__ nb_ent, int64_t n,
                             int* __restrict__ n_below, int* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int beg = nb_off[i], end = nb_off[i + 1];
  const int fg = first_above(nb_ent, beg, end, (uint32_t)i);
  n_below[i] = fg - beg;
  cnt[i] = end - fg;
}

// Pair records rec[p] = (i, entry of j in row i with its image code, that
// entry's index, the index of the reverse entry i in row j): one warp per row
// i, lanes over the row's tail (the pairs it owns); the reverse entry is
// found by binary search in the head of row j (its entries below j, where i
// lies since i < j), and the lane writes the whole record with one store.
__device__ __forceinline__ int first_not_below(const uint32_t* __restrict__ ent, int beg, int end, uint32_t i) {
  int lo = beg, hi = end;  // first t in [beg, end) with (ent[t] & mask) >= i
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((ent[mid] & kIdxMask) >= i) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void k_pair_fill(const int* __restrict__ nb_off, const uint32_t* __restrict__ nb_ent, int64_t n,
                            const int* __restrict__ n_below, const int* __restrict__ pair_off, int64_t npair,
                            int4* __restrict__ rec, int* __restrict__ flags) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w == 0 && lane == 0 && pair_off[n] != npair) atomicOr(flags, kFlagOverflow);  // lists must be symmetric
  if (w >= n) return;
  const int64_t i = w;
  const int end = nb_off[i + 1], fg = nb_off[i] + n_below[i], p0 = pair_off[i];
  for (int t = fg + lane; t < end; t += 32) {
    const uint32_t e = nb_ent[t];
    const int64_t j = e & kIdxMask;
    const int p = p0 + (t - fg);
    const int jb = nb_off[j], jh = jb + n_below[j];
    const int tr = first_not_below(nb_ent, jb, jh, (uint32_t)i);
    if (p < npair && tr < jh && (nb_ent[tr] & kIdxMask) == (uint32_t)i) {
      rec[p] = make_int4((int)i, (int)e, t, tr);
    } else {
      atomicOr(flags, kFlagOverflow);
    }
  }
}


// rows written at a fixed stride -> CSR (one warp per row; a thread per slot
// of the strided layout measured 0.10 ms per rebuild against 0.064 ms)
__global__ void k_row_compact(const uint32_t* __restrict__ rows, const int* __restrict__ brows, int stride, int64_t n,
                              const int* __restrict__ nb_off, const int* __restrict__ bd_off,
                              uint32_t* __restrict__ nb_ent, int* __restrict__ bd_idx) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int m = nb_off[i + 1] - nb_off[i], b = bd_off[i + 1] - bd_off[i];
  const uint32_t* src = rows + i * (int64_t)stride;
  const int* bsrc = brows + i * (int64_t)stride;
  for (int e = lane; e < m; e += 32) nb_ent[nb_off[i] + e] = src[e];
  for (int e = lane; e < b; e += 32) bd_idx[bd_off[i] + e] = bsrc[e];
}
}  // namespace

cudaError_t launch_cell_assign(const double* q, int64_t n, const DevGrid& g, const Batch& B, int* cell_of,
                               int* cell_slot, int* cell_count, int* abs_cell, float4* qf, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_cell_assign<<<grid_for(n, 256), 256, 0, s>>>(q, n, g, B, cell_of, cell_slot, cell_count, abs_cell, qf);
  return cudaGetLastError();
}

cudaError_t launch_cell_place(int64_t n, const int* cell_of, const int* cell_slot, const int* cell_start,
                              int* cell_sites, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_cell_place<<<grid_for(n, 256), 256, 0, s>>>(n, cell_of, cell_slot, cell_start, cell_sites);
  return cudaGetLastError();
}

cudaError_t launch_nbr_count(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                             const DevGrid& g, const Batch& B, const int* cell_of, const int* cell_start, const int* cell_sites,
                             double rl2, double rb2, float band, int* nb_cnt, int* bd_cnt, int* max_row,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_nbr_count<<<grid_for(n * 32, 256), 256, 0, s>>>(q, qf, sub, mobile_mask, n, g, B, cell_of, cell_start, cell_sites,
                                                    rl2, rb2, band, nb_cnt, bd_cnt, max_row);
  return cudaGetLastError();
}

cudaError_t launch_nbr_fill(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                            const DevGrid& g, const Batch& B, const int* cell_of, const int* cell_start, const int* cell_sites,
                            const int* abs_cell, double rl2, double rb2, float band, const int* nb_off,
                            uint32_t* nb_ent, const int* bd_off, int* bd_idx, int max_row, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (max_row < 1) max_row = 1;
  const size_t per_warp = (size_t)max_row * 5;
  int warps = (int)((200 * 1024) / per_warp);
  if (warps > 8) warps = 8;
  if (warps < 1) return cudaErrorInvalidValue;
  size_t shm = per_warp * warps + 16;
  cudaError_t e = cudaFuncSetAttribute(k_nbr_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  int threads = warps * 32;
  k_nbr_fill<<<grid_for(n * 32, threads), threads, shm, s>>>(q, qf, sub, mobile_mask, n, g, B, cell_of, cell_start,
                                                             cell_sites, abs_cell, rl2, rb2, band, nb_off, nb_ent,
                                                             bd_off, bd_idx, max_row);
  return cudaGetLastError();
}

cudaError_t launch_cand_max(int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, int* out,
                            cudaStream_t s) {
  if (ncell == 0) return cudaSuccess;
  k_cand_max<<<grid_for(ncell, 256), 256, 0, s>>>(ncell, g, B, cell_start, out);
  return cudaGetLastError();
}

size_t cell_stage_bytes(int cand_cap, int max_row, bool fill) {
  size_t b = (size_t)cand_cap * (sizeof(float4) + sizeof(int));
  if (fill)
    b += 16 + (size_t)(kCellThreads / 32) * 2 * (size_t)((max_row + 3) & ~3) * sizeof(uint32_t) +
         (size_t)8 * cand_cap * sizeof(uint16_t);  // rows and sort keys per warp, octant lists
  return b + 16;
}

cudaError_t launch_cell_count(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                              int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, const int* cell_sites,
                              double rl2, double rb2, float band, int cand_cap, int* nb_cnt, int* bd_cnt,
                              int* max_row, int* flags, cudaStream_t s) {
  if (n == 0 || ncell == 0) return cudaSuccess;
  const size_t shm = cell_stage_bytes(cand_cap, 0, false);
  cudaError_t e = cudaFuncSetAttribute(k_cell_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  k_cell_count<<<(unsigned)ncell, kCellThreads, shm, s>>>(q, qf, sub, mobile_mask, n, g, B, cell_start, cell_sites, rl2,
                                                          rb2, band, cand_cap, nb_cnt, bd_cnt, max_row, flags);
  return cudaGetLastError();
}

cudaError_t launch_cell_fill(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask, int64_t n,
                             int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start, const int* cell_sites,
                             const int* abs_cell, double rl2, double rb2, float band, int cand_cap,
                             const int* nb_off, uint32_t* nb_ent, const int* bd_off, int* bd_idx, int max_row,
                             int* flags, cudaStream_t s) {
  if (n == 0 || ncell == 0) return cudaSuccess;
  if (max_row < 1) max_row = 1;
  const size_t shm = cell_stage_bytes(cand_cap, max_row, true);
  cudaError_t e = cudaFuncSetAttribute(k_cell_fill<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  k_cell_fill<false><<<(unsigned)ncell, kCellThreads, shm, s>>>(q, qf, sub, mobile_mask, n, g, B, cell_start,
                                                                cell_sites, abs_cell, rl2, rb2, band, cand_cap, nb_off,
                                                                nb_ent, bd_off, bd_idx, max_row, nullptr, nullptr,
                                                                nullptr, nullptr, nullptr, flags);
  return cudaGetLastError();
}

cudaError_t launch_cell_fill_direct(const double* q, const float4* qf, const uint8_t* sub, uint32_t mobile_mask,
                                    int64_t n, int64_t ncell, const DevGrid& g, const Batch& B, const int* cell_start,
                                    const int* cell_sites, const int* abs_cell, double rl2, double rb2, float band,
                                    int cand_cap, int stride, uint32_t* rows, int* brows, int* nb_cnt, int* bd_cnt,
                                    int* n_below, int* pair_cnt, int* row_max, int* flags, cudaStream_t s) {
  if (n == 0 || ncell == 0) return cudaSuccess;
  const size_t shm = cell_stage_bytes(cand_cap, stride, true);
  cudaError_t e = cudaFuncSetAttribute(k_cell_fill<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  k_cell_fill<true><<<(unsigned)ncell, kCellThreads, shm, s>>>(q, qf, sub, mobile_mask, n, g, B, cell_start,
                                                               cell_sites, abs_cell, rl2, rb2, band, cand_cap, nullptr,
                                                               rows, nullptr, brows, stride, nb_cnt, bd_cnt, n_below,
                                                               pair_cnt, row_max, flags);
  return cudaGetLastError();
}

cudaError_t launch_row_compact(const uint32_t* rows, const int* brows, int stride, int64_t n, const int* nb_off,
                               const int* bd_off, uint32_t* nb_ent, int* bd_idx, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_row_compact<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(rows, brows, stride, n, nb_off, bd_off, nb_ent,
                                                                  bd_idx);
  return cudaGetLastError();
}

int64_t scan_tmp_len(int64_t n) { return (n + kScanBlock) / kScanBlock + 2; }

cudaError_t launch_scan(const int* in, int* out, int64_t n, long long* total64, int* tmp, int64_t tmp_len,
                        cudaStream_t s) {
  int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
  if (nblk < 1) nblk = 1;
  if (nblk + 1 > tmp_len) return cudaErrorInvalidValue;
  long long* bt = reinterpret_cast<long long*>(tmp);
  k_scan_blocks<<<(unsigned)nblk, kScanThreads, 0, s>>>(in, out, n, bt);
  k_scan_tops<<<1, kScanThreads, 0, s>>>(bt, nblk, total64);
  k_scan_add<<<grid_for(n + 1, 256), 256, 0, s>>>(out, n, bt, total64);
  return cudaGetLastError();
}

cudaError_t launch_strip_codes(const uint32_t* ent, int32_t* idx, int64_t m, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  k_strip<<<grid_for(m, 256), 256, 0, s>>>(ent, idx, m);
  return cudaGetLastError();
}

cudaError_t launch_site_max(const double* sigma, const double* q, int64_t n, unsigned long long* out_bits,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_site_max<<<grid_for(n, 256), 256, 0, s>>>(sigma, q, n, out_bits);
  return cudaGetLastError();
}

cudaError_t launch_segment_ids(const int* base, int nseg, int64_t count, int* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (nseg <= 0) return cudaErrorInvalidValue;
  k_segment_ids<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(base, nseg, count, out);
  return cudaGetLastError();
}

cudaError_t launch_pair_count(const int* nb_off, const uint32_t* nb_ent, int64_t n, int* n_below, int* cnt,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_pair_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nb_off, nb_ent, n, n_below, cnt);
  return cudaGetLastError();
}

cudaError_t launch_pair_fill(const int* nb_off, const uint32_t* nb_ent, int64_t n, const int* n_below,
                             const int* pair_off, int64_t npair, int4* pair_rec, int* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_pair_fill<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(nb_off, nb_ent, n, n_below, pair_off, npair,
                                                               pair_rec, flags);
  return cudaGetLastError();
}

}  // namespace mxe
