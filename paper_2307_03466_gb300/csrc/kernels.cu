// sm_103a kernels of the PDHG hot path of Scylla (arXiv 2307.03466, Algorithm 1,
// Sections 2.1-2.2 and 2.4).
//
// One PDHG attempt is two launches:
//   k_primal : (A^T y)_j by a warp-tile gather over the stored transpose, fused with
//              x'_j = proj_[l,u](x_j + tau_x (A^T y - c)_j)  (Algorithm 1, primal
//              step), the pending iterate-average update and ||x' - x||^2.
//   k_dual   : (A x')_i by the same gather over A, fused with the extrapolated dual
//              step y'_i = prox(y_i + tau_y (b - A(2x' - x))_i)  (Algorithm 1, dual
//              step), the average update, ||y' - y||^2 and (y'-y).(A x' - A x); its
//              last block takes the adaptive step-size decision.
// Every n_check attempts two check launches evaluate the current and the averaged
// iterate in FP64 (Section 2.2: relative KKT error, termination; PDLP restarts)
// and refresh the cached products A x and A^T y from FP64 matrix values.
// All decisions live in the device control block; launches read it and return
// early once the solve is done, so the loop can run inside one CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "device_common.cuh"
#include "internal.h"

namespace scylla {

// lanes that sum one row of a multi-row tile of nr rows: the largest power of two
// L with L * nr <= 32 (a tile of up to 16 rows splits each row over 2+ lanes, whose
// partial sums are combined by a shuffle tree, in a fixed order); 1 from 32 rows on
// (a wide tile of up to 32 * RPL rows gives each lane rows lane, lane + 32, ...)
__device__ __forceinline__ int row_lanes(int nr) {
  if (nr >= 32) return 1;
  const int l = 32 / (nr > 0 ? nr : 1);
  return 1 << (31 - __clz(l));
}

// The tiles of a warp: tile t goes to block t mod G and, within the block, to warp
// (t div G) mod 8, so every block holds the same number of tiles (within one) and
// each SM the same share when the grid is a whole number of waves of resident
// blocks; costly tiles (long rows, often stored together) spread over the blocks.
// The gathers of a launch are bound by each SM's L1TEX throughput (and the checks
// by its FP64 pipe), so the busiest SM sets the time.
struct WarpTiles {
  int first, end, step;
};
__device__ __forceinline__ WarpTiles warp_tiles(int ntiles) {
  const int G = int(gridDim.x), wpb = int(blockDim.x >> 5);
  return WarpTiles{int(blockIdx.x) + int(threadIdx.x >> 5) * G, ntiles, wpb * G};
}

// Sum of one long row (p1 - p0 > kTileNnz nonzeros) over a warp: lane l takes the
// vectors base + (32 i + l) kVec, i = 0, 1, ...  The column indices and values of
// step i + 1 are loaded before the gathers of step i are issued, so the loads of a
// row overlap its gathers (a 500-entry row: five dependent latencies, not eight);
// each lane accumulates its entries in the same order as an unpipelined loop.
template <int NV, bool kStream, typename Acc, typename V, typename Gather>
__device__ __forceinline__ void long_row_sum(int p0, int p1, const int* __restrict__ cols,
                                             const V* __restrict__ vals, Gather& gat, Acc (&s)[NV]) {
  constexpr int kStep = 32 * kVec;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = Acc(0);
  int p = (p0 & ~(kVec - 1)) + lane * kVec;
  int cc[4] = {0, 0, 0, 0};
  V vv[4] = {V(0), V(0), V(0), V(0)};
  if (p < p1) {
    ld4_as<kStream>(cols + p, cc);
    ld4_as<kStream>(vals + p, vv);
  }
  for (; p < p1; p += kStep) {
    int cn[4] = {0, 0, 0, 0};
    V vn[4] = {V(0), V(0), V(0), V(0)};
    if (p + kStep < p1) {
      ld4_as<kStream>(cols + p + kStep, cn);
      ld4_as<kStream>(vals + p + kStep, vn);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int q = p + e;
      if (q >= p0 && q < p1) {
        Acc g[NV];
        gat(cc[e], g);
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] = fma_t<Acc>(Acc(vv[e]), g[k], s[k]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      cc[e] = cn[e];
      vv[e] = vn[e];
    }
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = warp_sum(s[k]);
}

// --------------------------------------------------------------- the SpMV core ---
// Warp-tile CSR gather.  Each warp takes tiles round-robin.  A multi-row tile (at
// most kTileNnz nonzeros and 32 rows) is read with 16-byte vector loads of column
// indices and values, aligned down to the vector boundary and masked: every lane
// first issues all of its (at most three) vector loads, then all of its gathers, so
// up to 12 gathers per lane are in flight.  Products go to a skewed per-warp
// shared buffer and lane r sums row r in CSR order.  A single long row is reduced
// across the warp with shuffles.  The epilogue has two halves: load(row) is issued
// before the gathers, and finish(row, sum, pre) runs once the row sum is known, on
// the lane that owns the row.
//
// pro() runs once per thread before the first gather (it waits for the preceding
// kernel and sets up the gather and the epilogue; false ends the launch).  With PF
// the immutable part of the warp's first tile (bounds, row ranges, column indices,
// values) is loaded before pro(), so those loads overlap the wait.
template <int NV, bool PF, typename Acc, typename V, typename Gather, typename Epi, typename Pro, int RPL = 1>
__device__ __forceinline__ bool spmv_tiles(const int2* __restrict__ tiles, int ntiles,
                                           const int* __restrict__ rowptr, const int* __restrict__ cols,
                                           const V* __restrict__ vals, Gather& gat, Epi& epi,
                                           Acc* __restrict__ sm, Pro&& pro) {
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  // wide tiles serve DRAM-resident problems: stream the matrix past the caches so
  // that the gathered vector stays in L2
  constexpr bool kStream = RPL > 1;
  int r0 = 0, r1 = 0, p0 = 0, p1 = 0;
  int q0[RPL], q1[RPL];
  bool longrow = false;
  // p1 - base <= kTileNnz + kVec - 1 < 3 * 32 * kVec: three vector steps cover a tile
  int c[3][4];
  V v[3][4];
  // row of slot j of this lane in a multi-row tile of nr rows (nr when none): row
  // lane / L when rows are split over L lanes, else rows lane, lane + 32, ...
  auto slot_row = [&](int nr, int L, int j) { return L > 1 ? (j == 0 ? lane / L : nr) : lane + 32 * j; };
  // wide tiles (several per warp): the bounds of the warp's next tile are loaded one
  // tile ahead, so that a tile's row pointers and vector loads wait for one latency,
  // not two.  32-row tiles serve L2-resident problems with about one tile per warp.
  constexpr bool kAhead = RPL > 1;
  int2 nta = make_int2(0, 0), ntb = make_int2(0, 0);
  auto load_bounds = [&](int t) {
    if (t < wt.end) {
      nta = __ldg(tiles + t);
      ntb = __ldg(tiles + t + 1);
    }
  };
  auto fetch = [&](int t) {
    int2 ta, tb;
    if (kAhead) {
      ta = nta;
      tb = ntb;
      load_bounds(t + wt.step);
    } else {
      ta = __ldg(tiles + t);
      tb = __ldg(tiles + t + 1);
    }
    r0 = ta.x;
    r1 = tb.x;
    p0 = ta.y;
    p1 = tb.y;
    longrow = r1 - r0 == 1 && p1 - p0 > kTileNnz;
    if (!longrow) {
      const int nr = r1 - r0, L = row_lanes(nr);
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        q0[j] = q1[j] = 0;
        const int rl = slot_row(nr, L, j);
        if (rl < nr) {
          q0[j] = __ldg(rowptr + r0 + rl) - p0;
          q1[j] = __ldg(rowptr + r0 + rl + 1) - p0;
        }
      }
      const int base = p0 & ~(kVec - 1);
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
        if (p < p1) {
          ld4_as<kStream>(cols + p, c[it]);
          ld4_as<kStream>(vals + p, v[it]);
        }
      }
    }
  };
  if (kAhead) load_bounds(wt.first);
  if (PF && wt.first < wt.end) fetch(wt.first);
  if (!pro()) return false;
  for (int t = wt.first; t < wt.end; t += wt.step) {
    if (!PF || t != wt.first) fetch(t);
    const int base = p0 & ~(kVec - 1);
    if (longrow) {
      const typename Epi::Pre pre = epi.load(r0);
      Acc s[NV];
      long_row_sum<NV, kStream>(p0, p1, cols, vals, gat, s);
      if (lane == 0) epi.finish(r0, s, pre);
    } else {
      const int nr = r1 - r0, L = row_lanes(nr), sub = L > 1 ? lane % L : 0;
      typename Epi::Pre pre[RPL];
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int rl = slot_row(nr, L, j);
        pre[j] = typename Epi::Pre{};
        if (rl < nr && sub == 0) pre[j] = epi.load(r0 + rl);
      }
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          if (q >= p0 && q < p1) {
            Acc g[NV];
            gat(c[it][e], g);
            const int o = skew(q - p0);
#pragma unroll
            for (int k = 0; k < NV; ++k) sm[k * kSmemPerWarp + o] = Acc(v[it][e]) * g[k];
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int rl = slot_row(nr, L, j);
        Acc s[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] = Acc(0);
        if (rl < nr) {
          for (int q = q0[j] + sub; q < q1[j]; q += L) {
            const int o = skew(q);
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] += sm[k * kSmemPerWarp + o];
          }
        }
        if (j == 0)
          for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
        if (rl < nr && sub == 0) epi.finish(r0 + rl, s, pre[j]);
      }
      __syncwarp();
    }
  }
  return true;
}

struct NoPro {
  __device__ __forceinline__ bool operator()() const { return true; }
};

// Check form of the gather over FP32 iterates: the multi-row path stores each FP64
// value and the gathered FP32 entries, and every row sum is a chain of FP64 fused
// multiply-adds of a value and an exactly converted entry, in CSR order (one FP64
// instruction per nonzero and vector instead of a conversion, a product and a sum).
// smw holds kSmemPerWarp doubles, then NV * kSmemPerWarp floats.
template <int NV, typename Gather, typename Epi>
__device__ __forceinline__ void spmv_tiles_fma(const int2* __restrict__ tiles, int ntiles,
                                               const int* __restrict__ rowptr, const int* __restrict__ cols,
                                               const double* __restrict__ vals, Gather& gat, Epi& epi,
                                               double* __restrict__ smw) {
  float* __restrict__ sg = reinterpret_cast<float*>(smw + kSmemPerWarp);
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  for (int t = wt.first; t < wt.end; t += wt.step) {
    const int2 ta = __ldg(tiles + t), tb = __ldg(tiles + t + 1);
    const int r0 = ta.x, r1 = tb.x, p0 = ta.y, p1 = tb.y;
    const int base = p0 & ~(kVec - 1);
    if (r1 - r0 == 1 && p1 - p0 > kTileNnz) {
      const typename Epi::Pre pre = epi.load(r0);
      double s[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = 0.0;
      for (int p = base + lane * kVec; p < p1; p += 32 * kVec) {
        int cc[4];
        double vv[4];
        ld4(cols + p, cc);
        ld4(vals + p, vv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          if (q >= p0 && q < p1) {
            float g[NV];
            gat(cc[e], g);
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] = __fma_rn(vv[e], to_f64(g[k]), s[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = warp_sum(s[k]);
      if (lane == 0) epi.finish(r0, s, pre);
    } else {
      const int L = row_lanes(r1 - r0), rl = lane / L, sub = lane - rl * L;
      const bool mine = rl < r1 - r0, lead = mine && sub == 0;
      const int row = r0 + rl;
      int q0 = 0, q1 = 0;
      typename Epi::Pre pre{};
      if (mine) {
        q0 = __ldg(rowptr + row) - p0;
        q1 = __ldg(rowptr + row + 1) - p0;
      }
      if (lead) pre = epi.load(row);
      int c[3][4];
      double v[3][4];
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
        if (p < p1) {
          ld4(cols + p, c[it]);
          ld4(vals + p, v[it]);
        }
      }
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          if (q >= p0 && q < p1) {
            float g[NV];
            gat(c[it][e], g);
            const int o = skew(q - p0);
            smw[o] = v[it][e];
#pragma unroll
            for (int k = 0; k < NV; ++k) sg[k * kSmemPerWarp + o] = g[k];
          }
        }
      }
      __syncwarp();
      double s[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = 0.0;
      if (mine) {
        for (int q = q0 + sub; q < q1; q += L) {
          const int o = skew(q);
          const double a = smw[o];
#pragma unroll
          for (int k = 0; k < NV; ++k) s[k] = __fma_rn(a, to_f64(sg[k * kSmemPerWarp + o]), s[k]);
        }
      }
      for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
      if (lead) epi.finish(row, s, pre);
      __syncwarp();
    }
  }
}

// Programmatic dependent launch: each per-attempt kernel is launched while its
// predecessor still runs; it waits here for the predecessor's completion (and
// memory) before touching any mutable data, then lets its own successor launch.
// Without the launch attribute both calls return at once.
__device__ __forceinline__ void pdl_enter() {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
}

// resident blocks per SM the per-attempt kernels are compiled for: FP32 SpMVs are
// bound by the bytes in flight (more warps), FP64 ones by the FP64 pipe
template <typename T>
struct MinBlocks {
  static constexpr int value = 4;
};
template <>
struct MinBlocks<double> {
  static constexpr int value = 2;
};
// the wide-tile form holds up to four rows' epilogue values per lane
template <typename T, int F>
struct MinBlocksOf {
  static constexpr int value = (F == kFormWide && sizeof(T) == 4) ? 3 : MinBlocks<T>::value;
};


// gathered vectors: read-only path within one launch; L2-coherent loads inside the
// persistent kernel, where other SMs wrote them earlier in the same launch
template <bool Coh, typename T>
__device__ __forceinline__ T gload(const T* p) {
  if (Coh) return __ldcg(p);
  return __ldg(p);
}
// load of a vector the same kernel writes elsewhere: L2 only when blocks of one
// launch hand the data to one another (a persistent kernel whose work moves between
// blocks), a plain load otherwise
template <bool Coh, typename T>
__device__ __forceinline__ T eload(const T* p) {
  if (Coh) return __ldcg(p);
  return *p;
}

// the control values one attempt or check needs, read once per phase; the step
// sizes and averaging weights come already derived and converted to T
template <typename T>
struct SlotView {
  int cur, nxt, avg, ia_cur, ia_avg;
  T tau, sigma, w, w1;
  bool do_avg;
  int copy_lr, aty_valid;
};
__device__ __forceinline__ void view_steps(const Control* c, SlotView<float>& v) {
  v.tau = c->tau_f;
  v.sigma = c->sigma_f;
  v.w = c->w_f;
  v.w1 = c->w1_f;
}
__device__ __forceinline__ void view_steps(const Control* c, SlotView<double>& v) {
  v.tau = c->tau_d;
  v.sigma = c->sigma_d;
  v.w = c->w_d;
  v.w1 = c->w1_d;
}
template <typename T>
__device__ __forceinline__ SlotView<T> make_view(const Control* c) {
  SlotView<T> v;
  v.cur = c->ix_cur;
  v.nxt = c->ix_next;
  v.avg = c->ix_avg;
  v.ia_cur = c->ia_cur;
  v.ia_avg = c->ia_avg;
  view_steps(c, v);
  v.do_avg = c->avg_on != 0;
  v.copy_lr = c->copy_lr;
  v.aty_valid = c->aty_valid;
  return v;
}

// rows of every tile owned by this warp, without a gather: the same row-to-lane
// map as spmv_tiles, so the epilogue sums accumulate in the same lanes and order
template <typename T, typename Epi>
__device__ __forceinline__ void tiles_rows(const int2* __restrict__ tiles, int ntiles, const T* __restrict__ src,
                                           Epi& epi) {
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  for (int t = wt.first; t < wt.end; t += wt.step) {
    const int2 ta = __ldg(tiles + t), tb = __ldg(tiles + t + 1);
    const int nr = tb.x - ta.x, L = row_lanes(nr);
    if (L > 1) {
      if (lane % L == 0 && lane / L < nr) {
        const int row = ta.x + lane / L;
        const T s[1] = {src[row]};
        epi.finish(row, s, epi.load(row));
      }
    } else {
      for (int rl = lane; rl < nr; rl += 32) {
        const int row = ta.x + rl;
        const T s[1] = {src[row]};
        epi.finish(row, s, epi.load(row));
      }
    }
  }
}

// ------------------------------------------------- asynchronous tile staging ---
// The 32-row tiles with the warp's next tile staged in shared memory by
// asynchronous copies (cp.async) while the warp gathers for the current tile: the
// column indices and values, the row pointers and the epilogue operands of the next
// tile are in flight one tile ahead, and none of them holds a register until the
// tile starts.  Products, row sums and epilogues are those of spmv_tiles on the same
// tiles, in the same order, so the two forms give identical results.  A single row
// longer than a tile reads global memory directly.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cpa16(void* dst, const void* src, unsigned long long pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                   unsigned(__cvta_generic_to_shared(dst))),
               "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(unsigned(__cvta_generic_to_shared(dst))), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one warp's stage: a tile's indices and values (three vector steps of 32 lanes),
// the row pointers of its rows and five epilogue vectors over its rows
template <typename V>
struct AsyncStage {
  static constexpr int kN = 3 * 32 * kVec;
  int col[kN];
  V val[kN];
  int rp[32];
  V pre[5][32];
};

template <typename V, typename Gather, typename Epi>
__device__ __forceinline__ void spmv_tiles_async(const int2* __restrict__ tiles, int ntiles,
                                                 const int* __restrict__ rowptr, const int* __restrict__ cols,
                                                 const V* __restrict__ vals, Gather& gat, Epi& epi,
                                                 V* __restrict__ sm, AsyncStage<V>& S, int vec_mask) {
  static_assert(sizeof(V) == 4, "the asynchronous-copy form stages FP32 values");
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  if (wt.first >= wt.end) return;
  const unsigned long long pol = l2_policy_evict_first();
  auto longrow_of = [](int2 a, int2 b) { return b.x - a.x == 1 && b.y - a.y > kTileNnz; };
  // the copies of one tile into the stage (none for a long row), as one group
  auto issue = [&](int2 ta, int2 tb) {
    if (!longrow_of(ta, tb)) {
      const int base = ta.y & ~(kVec - 1);
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int o = (it * 32 + lane) * kVec, p = base + o;
        if (p < tb.y) {
          cpa16(&S.col[o], cols + p, pol);
          cpa16(&S.val[o], vals + p, pol);
        }
      }
      if (lane < tb.x - ta.x) {
        cpa4(&S.rp[lane], rowptr + ta.x + lane);
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if (vec_mask & (1 << k)) cpa4(&S.pre[k][lane], epi.stage_vec(k) + ta.x + lane);
      }
    }
    cpa_commit();
  };
  int2 ca = __ldg(tiles + wt.first), cb = __ldg(tiles + wt.first + 1);
  int2 na = make_int2(0, 0), nb = make_int2(0, 0), la = make_int2(0, 0), lb = make_int2(0, 0);
  if (wt.first + wt.step < wt.end) {
    na = __ldg(tiles + wt.first + wt.step);
    nb = __ldg(tiles + wt.first + wt.step + 1);
  }
  issue(ca, cb);
  for (int t = wt.first; t < wt.end; t += wt.step) {
    const int t2 = t + 2 * wt.step;
    if (t2 < wt.end) {  // bounds two tiles ahead, for the copies issued at the next tile
      la = __ldg(tiles + t2);
      lb = __ldg(tiles + t2 + 1);
    }
    const int r0 = ca.x, r1 = cb.x, p0 = ca.y, p1 = cb.y;
    const int base = p0 & ~(kVec - 1);
    cpa_wait_all();
    __syncwarp();
    if (longrow_of(ca, cb)) {
      __syncwarp();
      if (t + wt.step < wt.end) issue(na, nb);
      const typename Epi::Pre pre = epi.load(r0);
      V s[1];
      long_row_sum<1, true>(p0, p1, cols, vals, gat, s);
      if (lane == 0) epi.finish(r0, s, pre);
    } else {
      const int nr = r1 - r0, L = row_lanes(nr), sub = L > 1 ? lane % L : 0;
      const int rl = L > 1 ? lane / L : lane;
      int q0 = 0, q1 = 0;
      typename Epi::Pre pre{};
      if (rl < nr) {
        q0 = S.rp[rl] - p0;
        q1 = (rl + 1 < nr ? S.rp[rl + 1] : p1) - p0;
        if (sub == 0) pre = epi.stage_pre(&S.pre[0][0], 32, rl);
      }
      // the gathers take their indices from the stage; the values wait in registers
      // for the products, so the stage is free once every gather is issued
      V v[3][4], g[3][4];
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int o = (it * 32 + lane) * kVec, p = base + o;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          v[it][e] = V(0);
          g[it][e] = V(0);
          if (q >= p0 && q < p1) {
            V gg[1];
            gat(S.col[o + e], gg);
            g[it][e] = gg[0];
            v[it][e] = S.val[o + e];
          }
        }
      }
      __syncwarp();  // every lane has read the stage before it is refilled
      if (t + wt.step < wt.end) issue(na, nb);
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          if (q >= p0 && q < p1) sm[skew(q - p0)] = v[it][e] * g[it][e];
        }
      }
      __syncwarp();
      V sum = V(0);
      if (rl < nr)
        for (int q = q0 + sub; q < q1; q += L) sum += sm[skew(q)];
      for (int o = L >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
      const V sv[1] = {sum};
      if (rl < nr && sub == 0) epi.finish(r0 + rl, sv, pre);
      __syncwarp();
    }
    ca = na;
    cb = nb;
    na = la;
    nb = lb;
  }
  cpa_wait_all();
}

// ---------------------------------------------------------------- PDHG slot ---
template <typename T, bool Coh = false>
struct PrimalEpi {
  typedef typename AccOf<T>::type A;
  struct Pre {
    T x, c, l, u, xa;
  };
  const T* __restrict__ xc;
  T* __restrict__ xn;
  T* __restrict__ xa;
  T* __restrict__ aty;
  T* __restrict__ xlr;
  const T* __restrict__ cc;
  const T* __restrict__ ll;
  const T* __restrict__ uu;
  const T* __restrict__ qq;  // scaled Hessian diagonal of a quadratic objective, or null
  T tau, w, w1;
  bool do_avg, copy_lr, store_aty, use_cached;
  A acc;
  __device__ __forceinline__ Pre load(int j) const {
    return Pre{eload<Coh>(xc + j), cc[j], ll[j], uu[j], do_avg ? eload<Coh>(xa + j) : T(0)};
  }
  // staged form: the five vectors of load(), in its order, staged in shared memory
  __device__ __forceinline__ const T* stage_vec(int k) const {
    return k == 0 ? xc : k == 1 ? cc : k == 2 ? ll : k == 3 ? uu : xa;
  }
  __device__ __forceinline__ Pre stage_pre(const T* sv, int stride, int o) const {
    return Pre{sv[o], sv[stride + o], sv[2 * stride + o], sv[3 * stride + o], do_avg ? sv[4 * stride + o] : T(0)};
  }
  __device__ __forceinline__ void finish(int j, const T (&s)[1], const Pre& p) {
    const T aty_j = use_cached ? eload<Coh>(aty + j) : s[0];
    if (store_aty) aty[j] = aty_j;
    if (do_avg) xa[j] = blend(p.xa, p.x, w1, w);
    if (copy_lr) xlr[j] = p.x;
    T z = p.x + tau * (aty_j - p.c);
    // quadratic objective: the prox of tau/2 q x^2 scales the step by 1 / (1 + tau q)
    if (qq) z = z / (T(1) + tau * qq[j]);
    const T v = clampv<T>(z, p.l, p.u);
    xn[j] = v;
    const A dx = A(v) - A(p.x);
    acc += dx * dx;
  }
};

// primal step of Algorithm 1 over all columns; block partial of ||x' - x||^2 to part
template <typename T>
__device__ __forceinline__ void setup_primal(PrimalEpi<T>& epi, const DevLP<T>& d, const SlotView<T>& v) {
  epi.xc = d.X[v.cur];
  epi.xn = d.X[v.nxt];
  epi.xa = d.X[v.avg];
  epi.aty = d.ATY[v.ia_cur];
  epi.xlr = d.XLR;
  epi.cc = d.c;
  epi.ll = d.l;
  epi.uu = d.u;
  epi.qq = d.q;
  epi.tau = v.tau;
  epi.w = v.w;
  epi.w1 = v.w1;
  epi.do_avg = v.do_avg;
  epi.copy_lr = v.copy_lr != 0;
  epi.store_aty = !v.aty_valid;
  epi.use_cached = false;
  epi.acc = 0;
}

// RPL > 1: the wide tiles
template <typename T, bool Coh, int RPL = 1>
__device__ __forceinline__ void primal_phase(const DevLP<T>& d, const SlotView<T>& v, T* sm,
                                             typename AccOf<T>::type* part) {
  PrimalEpi<T> epi;
  setup_primal(epi, d, v);
  const int2* tiles = RPL > 1 ? d.t_tiles_w : d.t_tiles;
  const int ntiles = RPL > 1 ? d.t_ntiles_w : d.t_ntiles;
  if (v.aty_valid) {
    tiles_rows<T>(tiles, ntiles, epi.aty, epi);  // retry: A^T y is cached
  } else {
    const T* __restrict__ yc = d.Y[v.cur];
    auto gat = [&](int i, T(&g)[1]) { g[0] = gload<Coh>(yc + i); };
    spmv_tiles<1, false, T, T, decltype(gat), PrimalEpi<T>, NoPro, RPL>(
        tiles, ntiles, d.t_rowptr, d.t_cols, d.t_vals, gat, epi, sm + (threadIdx.x >> 5) * kSmemPerWarp, NoPro());
  }
  const typename AccOf<T>::type acc[kNP] = {epi.acc};
  block_store_partials<kNP>(acc, part);
}

template <typename T, bool Coh = false>
struct DualEpi {
  typedef typename AccOf<T>::type A;
  struct Pre {
    T ax, y, lo, hi, ya;
  };
  const T* __restrict__ axc;
  T* __restrict__ axn;
  const T* __restrict__ yc;
  T* __restrict__ yn;
  T* __restrict__ ya;
  T* __restrict__ ylr;
  const T* __restrict__ lo;
  const T* __restrict__ hi;
  T sigma, w, w1;
  bool do_avg, copy_lr;
  A acc0, acc1;
  __device__ __forceinline__ Pre load(int i) const {
    return Pre{eload<Coh>(axc + i), eload<Coh>(yc + i), lo[i], hi[i], do_avg ? eload<Coh>(ya + i) : T(0)};
  }
  __device__ __forceinline__ const T* stage_vec(int k) const {
    return k == 0 ? axc : k == 1 ? yc : k == 2 ? lo : k == 3 ? hi : ya;
  }
  __device__ __forceinline__ Pre stage_pre(const T* sv, int stride, int o) const {
    return Pre{sv[o], sv[stride + o], sv[2 * stride + o], sv[3 * stride + o], do_avg ? sv[4 * stride + o] : T(0)};
  }
  __device__ __forceinline__ void finish(int i, const T (&s)[1], const Pre& p) {
    const T ax_new = s[0];
    if (do_avg) ya[i] = blend(p.ya, p.y, w1, w);
    if (copy_lr) ylr[i] = p.y;
    const T axt = T(2) * ax_new - p.ax;
    const T v = dual_prox<T>(p.y, sigma, axt, p.lo, p.hi);
    yn[i] = v;
    axn[i] = ax_new;
    const A dy = A(v) - A(p.y);
    acc0 += dy * dy;
    acc1 += dy * (A(ax_new) - A(p.ax));
  }
};

// extrapolated dual step of Algorithm 1 over all rows; block partials of ||y' - y||^2
// and (y' - y).(A x' - A x) to part
template <typename T>
__device__ __forceinline__ void setup_dual(DualEpi<T>& epi, const DevLP<T>& d, const SlotView<T>& v) {
  epi.axc = d.AX[v.cur];
  epi.axn = d.AX[v.nxt];
  epi.yc = d.Y[v.cur];
  epi.yn = d.Y[v.nxt];
  epi.ya = d.Y[v.avg];
  epi.ylr = d.YLR;
  epi.lo = d.lo;
  epi.hi = d.hi;
  epi.sigma = v.sigma;
  epi.w = v.w;
  epi.w1 = v.w1;
  epi.do_avg = v.do_avg;
  epi.copy_lr = v.copy_lr != 0;
  epi.acc0 = 0;
  epi.acc1 = 0;
}

template <typename T, bool Coh, int RPL = 1>
__device__ __forceinline__ void dual_phase(const DevLP<T>& d, const SlotView<T>& v, T* sm,
                                           typename AccOf<T>::type* part) {
  DualEpi<T> epi;
  setup_dual(epi, d, v);
  const T* __restrict__ xn = d.X[v.nxt];
  auto gat = [&](int j, T(&g)[1]) { g[0] = gload<Coh>(xn + j); };
  spmv_tiles<1, false, T, T, decltype(gat), DualEpi<T>, NoPro, RPL>(
      RPL > 1 ? d.a_tiles_w : d.a_tiles, RPL > 1 ? d.a_ntiles_w : d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals, gat,
      epi, sm + (threadIdx.x >> 5) * kSmemPerWarp, NoPro());
  const typename AccOf<T>::type acc[kND] = {epi.acc0, epi.acc1};
  block_store_partials<kND>(acc, part);
}

// The per-attempt kernels: with programmatic dependent launch they are resident
// while their predecessor drains, and wait for it before touching any data.
// block partials of the per-attempt sums, in the bulk accumulator type
template <typename T>
__device__ __forceinline__ typename AccOf<T>::type* acc_part(double* p) {
  return reinterpret_cast<typename AccOf<T>::type*>(p);
}

// F: kFormPlain (32-row tiles), kFormPrefetch (32-row tiles, first tile loaded
// before the dependency wait), kFormWide (wide tiles, plain loads)
template <typename T, int F>
__global__ void __launch_bounds__(kThreads, (MinBlocksOf<T, F>::value)) k_primal(DevLP<T> d) {
  Control* ctl = d.ctl;
  __shared__ T sm[kWarpsPerBlock * kSmemPerWarp];
  if (F != kFormPrefetch) {
    pdl_enter();
    if (ctl->done || ctl->k >= ctl->iter_limit) return;
    if (F == kFormWide) primal_phase<T, false, kWideRPL>(d, make_view<T>(ctl), sm, acc_part<T>(d.part_p));
    else primal_phase<T, false, 1>(d, make_view<T>(ctl), sm, acc_part<T>(d.part_p));
    return;
  }
  // prefetching form: the gather of A^T y is taken even when A^T y is cached (a
  // retry), and its result is then ignored
  PrimalEpi<T> epi;
  const T* __restrict__ yc = nullptr;
  bool cached = false;
  auto gat = [&](int i, T(&g)[1]) { g[0] = cached ? T(0) : __ldg(yc + i); };
  auto pro = [&]() -> bool {
    pdl_enter();
    if (ctl->done || ctl->k >= ctl->iter_limit) return false;
    const SlotView<T> v = make_view<T>(ctl);
    setup_primal(epi, d, v);
    cached = v.aty_valid != 0;
    epi.use_cached = cached;
    yc = d.Y[v.cur];
    return true;
  };
  if (!spmv_tiles<1, true, T, T>(d.t_tiles, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals, gat, epi,
                                 sm + (threadIdx.x >> 5) * kSmemPerWarp, pro))
    return;
  const typename AccOf<T>::type acc[kNP] = {epi.acc};
  block_store_partials<kNP>(acc, acc_part<T>(d.part_p));
}

// The last block to finish reduces all block partials (warps 1..) while thread 0
// gathers the decision's other inputs, then takes the step-size decision.
template <typename T, int F>
__global__ void __launch_bounds__(kThreads, (MinBlocksOf<T, F>::value)) k_dual(DevLP<T> d) {
  typedef typename AccOf<T>::type A;
  Control* ctl = d.ctl;
  __shared__ T sm[kWarpsPerBlock * kSmemPerWarp];
  if (F != kFormPrefetch) {
    pdl_enter();
    if (ctl->done || ctl->k >= ctl->iter_limit) return;
    if (F == kFormWide) dual_phase<T, false, kWideRPL>(d, make_view<T>(ctl), sm, acc_part<T>(d.part_d));
    else dual_phase<T, false, 1>(d, make_view<T>(ctl), sm, acc_part<T>(d.part_d));
  } else {
    DualEpi<T> epi;
    const T* __restrict__ xn = nullptr;
    auto gat = [&](int j, T(&g)[1]) { g[0] = __ldg(xn + j); };
    auto pro = [&]() -> bool {
      pdl_enter();
      if (ctl->done || ctl->k >= ctl->iter_limit) return false;
      const SlotView<T> v = make_view<T>(ctl);
      setup_dual(epi, d, v);
      xn = d.X[v.nxt];
      return true;
    };
    if (!spmv_tiles<1, true, T, T>(d.a_tiles, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals, gat, epi,
                                   sm + (threadIdx.x >> 5) * kSmemPerWarp, pro))
      return;
    const A acc[kND] = {epi.acc0, epi.acc1};
    block_store_partials<kND>(acc, acc_part<T>(d.part_d));
  }
  if (!is_last_block(&ctl->cnt_dual)) return;
  __shared__ StepPre pre;  // in shared memory: nothing stays live in registers across the reduction
  if (threadIdx.x == 0) pre = step_pre<A>(ctl, d.step_fac, d.n_check);
  __shared__ A red[kNP + kND];
  static_assert(3 * (kThreads - 32) * sizeof(A) <= sizeof(sm), "reduction scratch");
  reduce_step<A>(acc_part<T>(d.part_p), d.grid_p, acc_part<T>(d.part_d), d.grid_d, reinterpret_cast<A*>(sm), red);
  if (threadIdx.x == 0) {
    step_control<A>(ctl, pre, red[0], red[1], red[2], d.trace_steps, d.trace_cap);
    ctl->cnt_dual = 0;
  }
}

// ------------------------------------------------------------ staged SpMV ---
// Form of the per-attempt kernels for matrices that do not stay in L2 between
// attempts (the kernels are then bound by the bytes in flight, not by latency).
// Each warp owns a ring of two shared-memory stages; a stage holds one wide
// tile's column indices and values, its row pointers and the five epilogue
// vectors of its rows, each brought in by one cp.async.bulk copy (16-byte aligned
// ranges, rounded outwards) that completes on the stage's mbarrier.  The warp
// processes tile i while the copies of tiles i+1 .. i+S-1 are in flight, then
// re-arms the stage with tile i+S.  A single row longer than a tile is read from
// global memory directly.  Products, row sums and epilogues are those of
// spmv_tiles on the same wide tiles, in the same order, so the staged and the
// plain-load forms give identical results.  Every
// mbarrier wait is bounded; a wait that runs out stops the warp's work and
// returns false (the caller then ends the solve with SCYLLA_DEVICE_TIMEOUT).
template <typename T>
struct Staged {
  static constexpr int kStages = 2;
  static constexpr int kNnz = kTileNnz + 8;   // a tile's nonzeros from its aligned start, rounded up
  static constexpr int kRows = kWideRows + 8;  // row pointers / rows of a wide tile from the aligned start, rounded up
  static constexpr int kVecs = 5;
  static constexpr int kColsOff = 0;
  static constexpr int kValsOff = kColsOff + kNnz * 4;
  static constexpr int kRpOff = kValsOff + kNnz * int(sizeof(T));
  static constexpr int kVecOff = kRpOff + kRows * 4;
  static constexpr int kStageBytes = kVecOff + kVecs * kRows * int(sizeof(T));
  static constexpr int kWarpBytes = kStages * kStageBytes + 64;  // + the stages' mbarriers
  static constexpr int kBlockBytes = kWarpsPerBlock * kWarpBytes;
  static_assert(kValsOff % 16 == 0 && kRpOff % 16 == 0 && kVecOff % 16 == 0 && kStageBytes % 16 == 0, "align");
  static_assert((kRows * int(sizeof(T))) % 16 == 0, "vector slots");
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase of parity `parity` to complete
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, unsigned long long limit_ns) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = clock_ns();
  while (!mbar_test(b, parity))
    if (clock_ns() - t0 > limit_ns) return false;
  return true;
}

struct TileBounds {
  int r0, r1, p0, p1;
  __device__ __forceinline__ bool longrow() const { return r1 - r0 == 1 && p1 - p0 > kTileNnz; }
};

// one staged tile: lane 0 arms the stage's mbarrier with the total byte count and
// issues the copies; vec_mask selects the epilogue vectors to stage
template <typename T, typename Epi>
__device__ __forceinline__ void stage_issue(char* st, unsigned long long* bar, const TileBounds& tb,
                                            const int* rowptr, const int* cols, const T* vals, const Epi& epi,
                                            int vec_mask) {
  typedef Staged<T> S;
  const int base = tb.p0 & ~(kVec - 1);
  const int ncv = (tb.p1 - base + kVec - 1) & ~(kVec - 1);
  const int rb = tb.r0 & ~3;
  const int nrp = (tb.r1 + 1 - rb + 3) & ~3;
  const int nv = (tb.r1 - rb + 3) & ~3;
  unsigned bytes = unsigned(nrp * 4);
  if (ncv > 0) bytes += unsigned(ncv * (4 + int(sizeof(T))));
#pragma unroll
  for (int k = 0; k < S::kVecs; ++k)
    if (vec_mask & (1 << k)) bytes += unsigned(nv * int(sizeof(T)));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the warp's reads of this stage come first
  mbar_arm(bar, bytes);
  if (ncv > 0) {
    bulk_copy(st + S::kColsOff, cols + base, unsigned(ncv * 4), bar);
    bulk_copy(st + S::kValsOff, vals + base, unsigned(ncv * int(sizeof(T))), bar);
  }
  bulk_copy(st + S::kRpOff, rowptr + rb, unsigned(nrp * 4), bar);
#pragma unroll
  for (int k = 0; k < S::kVecs; ++k)
    if (vec_mask & (1 << k))
      bulk_copy(st + S::kVecOff + k * S::kRows * int(sizeof(T)), epi.stage_vec(k) + rb, unsigned(nv * int(sizeof(T))),
                bar);
}

// the warp's tiles (warp_tiles); gather(c) returns the gathered entry
// (skip_gather: the row sums are not needed, as for a primal retry)
template <typename T, typename Gather, typename Epi>
__device__ bool staged_tiles(const int2* __restrict__ tiles, int ntiles, const int* __restrict__ rowptr,
                             const int* __restrict__ cols, const T* __restrict__ vals, Gather& gat, Epi& epi,
                             int vec_mask, bool skip_gather, char* wsm, unsigned long long limit_ns) {
  typedef Staged<T> S;
  constexpr int NS = S::kStages;
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(wsm + NS * S::kStageBytes);
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto bounds = [&](int t) {
    const int2 ta = __ldg(tiles + t), tb2 = __ldg(tiles + t + 1);
    return TileBounds{ta.x, tb2.x, ta.y, tb2.y};
  };
  // stage s holds the warp's tiles i = s, s + NS, ... (tile wt.first + i * wt.step); `armed` marks
  // stages with copies in flight, `par` their current phase parity
  unsigned armed = 0, par = 0;
  TileBounds tb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int t = wt.first + s * wt.step;
    if (t < wt.end) {
      tb[s] = bounds(t);
      if (!tb[s].longrow()) {
        if (lane == 0) stage_issue<T>(wsm + s * S::kStageBytes, &bars[s], tb[s], rowptr, cols, vals, epi, vec_mask);
        armed |= 1u << s;
      }
    }
  }
  bool ok = true;
  int i = 0;
  for (int t = wt.first; t < wt.end; t += wt.step, ++i) {
    const int s = i % NS;
    const TileBounds b = tb[s];
    char* st = wsm + s * S::kStageBytes;
    if (b.longrow()) {
      // a single long row, straight from global memory
      const int base = b.p0 & ~(kVec - 1);
      const typename Epi::Pre pre = epi.load(b.r0);
      T acc = T(0);
      if (!skip_gather) {
        for (int p = base + lane * kVec; p < b.p1; p += 32 * kVec) {
          int cc[4];
          T vv[4];
          ld4(cols + p, cc);
          ld4(vals + p, vv);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = p + e;
            if (q >= b.p0 && q < b.p1) acc = fma_t<T>(vv[e], gat(cc[e]), acc);
          }
        }
      }
      acc = warp_sum(acc);
      const T sv[1] = {acc};
      if (lane == 0) epi.finish(b.r0, sv, pre);
    } else {
      if (!mbar_wait(&bars[s], (par >> s) & 1u, limit_ns)) {
        ok = false;
        break;
      }
      par ^= 1u << s;
      armed &= ~(1u << s);
      const int base = b.p0 & ~(kVec - 1), off = b.p0 - base, len = b.p1 - b.p0;
      const int rb = b.r0 & ~3;
      const int* scol = reinterpret_cast<const int*>(st + S::kColsOff);
      T* sval = reinterpret_cast<T*>(st + S::kValsOff);
      const int* srp = reinterpret_cast<const int*>(st + S::kRpOff);
      const T* svec = reinterpret_cast<const T*>(st + S::kVecOff);
      // rows as in spmv_tiles on wide tiles: slot j of a lane is row lane / L (rows
      // split over L lanes) or row lane + 32 j
      const int nr = b.r1 - b.r0, L = row_lanes(nr), sub = L > 1 ? lane % L : 0;
      int q0[kWideRPL], q1[kWideRPL];
      typename Epi::Pre pre[kWideRPL];
#pragma unroll
      for (int j = 0; j < kWideRPL; ++j) {
        const int rl = L > 1 ? (j == 0 ? lane / L : nr) : lane + 32 * j;
        q0[j] = q1[j] = 0;
        pre[j] = typename Epi::Pre{};
        if (rl < nr) {
          q0[j] = srp[b.r0 + rl - rb] - b.p0;
          q1[j] = srp[b.r0 + rl + 1 - rb] - b.p0;
          if (sub == 0) pre[j] = epi.stage_pre(svec, S::kRows, b.r0 + rl - rb);
        }
      }
      if (!skip_gather) {
        // products in place of the values; up to eight gathers per lane in flight
        T g[kTileNnz / 32];
#pragma unroll
        for (int j = 0; j < kTileNnz / 32; ++j) {
          const int k = lane + 32 * j;
          g[j] = k < len ? gat(scol[off + k]) : T(0);
        }
#pragma unroll
        for (int j = 0; j < kTileNnz / 32; ++j) {
          const int k = lane + 32 * j;
          if (k < len) sval[off + k] = sval[off + k] * g[j];
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kWideRPL; ++j) {
        const int rl = L > 1 ? (j == 0 ? lane / L : nr) : lane + 32 * j;
        T acc = T(0);
        if (rl < nr && !skip_gather)
          for (int q = q0[j] + sub; q < q1[j]; q += L) acc += sval[off + q];
        if (j == 0)
          for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        const T sv[1] = {acc};
        if (rl < nr && sub == 0) epi.finish(b.r0 + rl, sv, pre[j]);
      }
      __syncwarp();
    }
    // re-arm this stage with the warp's tile NS steps ahead
    const int tn = t + NS * wt.step;
    if (tn < wt.end) {
      tb[s] = bounds(tn);
      if (!tb[s].longrow()) {
        if (lane == 0) stage_issue<T>(st, &bars[s], tb[s], rowptr, cols, vals, epi, vec_mask);
        armed |= 1u << s;
      }
    }
  }
  if (!ok) {
    // let the copies in flight land (bounded) before the shared memory is released
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (armed & (1u << s)) mbar_wait(&bars[s], (par >> s) & 1u, limit_ns);
  }
  return ok;
}

template <typename T>
__device__ __forceinline__ void staged_timeout(Control* ctl) {
  ctl->status = SCYLLA_DEVICE_TIMEOUT;
  ctl->done = 1;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_primal_st(DevLP<T> d) {
  extern __shared__ __align__(128) char dsm[];
  Control* ctl = d.ctl;
  pdl_enter();
  if (ctl->done || ctl->k >= ctl->iter_limit) return;
  const SlotView<T> v = make_view<T>(ctl);
  PrimalEpi<T> epi;
  setup_primal(epi, d, v);
  const bool cached = v.aty_valid != 0;
  epi.use_cached = cached;
  const T* __restrict__ yc = d.Y[v.cur];
  auto gat = [&](int i) { return __ldg(yc + i); };
  char* wsm = dsm + (threadIdx.x >> 5) * Staged<T>::kWarpBytes;
  const bool ok = staged_tiles<T>(d.t_tiles_w, d.t_ntiles_w, d.t_rowptr, d.t_cols, d.t_vals, gat, epi,
                                  v.do_avg ? 31 : 15, cached, wsm, d.wait_ns);
  if (!ok && (threadIdx.x & 31) == 0) staged_timeout<T>(ctl);
  const typename AccOf<T>::type acc[kNP] = {epi.acc};
  block_store_partials<kNP>(acc, acc_part<T>(d.part_p));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dual_st(DevLP<T> d) {
  typedef typename AccOf<T>::type A;
  extern __shared__ __align__(128) char dsm[];
  Control* ctl = d.ctl;
  pdl_enter();
  if (ctl->done || ctl->k >= ctl->iter_limit) return;
  const SlotView<T> v = make_view<T>(ctl);
  DualEpi<T> epi;
  setup_dual(epi, d, v);
  const T* __restrict__ xn = d.X[v.nxt];
  auto gat = [&](int j) { return __ldg(xn + j); };
  char* wsm = dsm + (threadIdx.x >> 5) * Staged<T>::kWarpBytes;
  const bool ok = staged_tiles<T>(d.a_tiles_w, d.a_ntiles_w, d.a_rowptr, d.a_cols, d.a_vals, gat, epi,
                                  v.do_avg ? 31 : 15, false, wsm, d.wait_ns);
  if (!ok && (threadIdx.x & 31) == 0) staged_timeout<T>(ctl);
  const A acc[kND] = {epi.acc0, epi.acc1};
  block_store_partials<kND>(acc, acc_part<T>(d.part_d));
  if (!is_last_block(&ctl->cnt_dual)) return;
  __shared__ StepPre pre;
  if (threadIdx.x == 0) pre = step_pre<A>(ctl, d.step_fac, d.n_check);
  __shared__ A red[kNP + kND];
  static_assert(3 * (kThreads - 32) * sizeof(A) <= Staged<T>::kBlockBytes, "reduction scratch");
  reduce_step<A>(acc_part<T>(d.part_p), d.grid_p, acc_part<T>(d.part_d), d.grid_d, reinterpret_cast<A*>(dsm), red);
  if (threadIdx.x == 0) {
    if (!ctl->done) step_control<A>(ctl, pre, red[0], red[1], red[2], d.trace_steps, d.trace_cap);
    ctl->cnt_dual = 0;
  }
}

// The asynchronous-copy form (FP32): the per-attempt kernels over 32-row tiles with
// the warp's next tile staged in shared memory (spmv_tiles_async); a primal retry
// (A^T y cached) takes the rows without a gather, as the other forms do.
__global__ void __launch_bounds__(kThreads, 3) k_primal_as(DevLP<float> d) {
  Control* ctl = d.ctl;
  __shared__ float sm[kWarpsPerBlock * kSmemPerWarp];
  __shared__ __align__(16) AsyncStage<float> stg[kWarpsPerBlock];
  pdl_enter();
  if (ctl->done || ctl->k >= ctl->iter_limit) return;
  const SlotView<float> v = make_view<float>(ctl);
  PrimalEpi<float> epi;
  setup_primal(epi, d, v);
  if (v.aty_valid) {
    tiles_rows<float>(d.t_tiles, d.t_ntiles, epi.aty, epi);
  } else {
    const float* __restrict__ yc = d.Y[v.cur];
    auto gat = [&](int i, float(&g)[1]) { g[0] = __ldg(yc + i); };
    const int w = threadIdx.x >> 5;
    spmv_tiles_async<float>(d.t_tiles, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals, gat, epi, sm + w * kSmemPerWarp,
                            stg[w], v.do_avg ? 31 : 15);
  }
  const float acc[kNP] = {epi.acc};
  block_store_partials<kNP>(acc, acc_part<float>(d.part_p));
}

__global__ void __launch_bounds__(kThreads, 3) k_dual_as(DevLP<float> d) {
  typedef AccOf<float>::type A;
  Control* ctl = d.ctl;
  __shared__ float sm[kWarpsPerBlock * kSmemPerWarp];
  __shared__ __align__(16) AsyncStage<float> stg[kWarpsPerBlock];
  pdl_enter();
  if (ctl->done || ctl->k >= ctl->iter_limit) return;
  const SlotView<float> v = make_view<float>(ctl);
  DualEpi<float> epi;
  setup_dual(epi, d, v);
  const float* __restrict__ xn = d.X[v.nxt];
  auto gat = [&](int j, float(&g)[1]) { g[0] = __ldg(xn + j); };
  const int w = threadIdx.x >> 5;
  spmv_tiles_async<float>(d.a_tiles, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals, gat, epi, sm + w * kSmemPerWarp,
                          stg[w], v.do_avg ? 31 : 15);
  const A acc[kND] = {epi.acc0, epi.acc1};
  block_store_partials<kND>(acc, acc_part<float>(d.part_d));
  if (!is_last_block(&ctl->cnt_dual)) return;
  __shared__ StepPre pre;
  if (threadIdx.x == 0) pre = step_pre<A>(ctl, d.step_fac, d.n_check);
  __shared__ A red[kNP + kND];
  static_assert(3 * (kThreads - 32) * sizeof(A) <= sizeof(sm), "reduction scratch");
  reduce_step<A>(acc_part<float>(d.part_p), d.grid_p, acc_part<float>(d.part_d), d.grid_d, sm, red);
  if (threadIdx.x == 0) {
    step_control<A>(ctl, pre, red[0], red[1], red[2], d.trace_steps, d.trace_cap);
    ctl->cnt_dual = 0;
  }
}

// the two-vector FP64 gather of a check: FP32 iterates take the fused form; FP64
// iterates the product form (their gathered entries need no conversion)
template <typename Gather, typename Epi>
__device__ __forceinline__ void check_gather(const int2* tiles, int ntiles, const int* rowptr, const int* cols,
                                             const double* vals, Gather& gat, Epi& epi, double* smw,
                                             const float* /*tag*/) {
  spmv_tiles_fma<2>(tiles, ntiles, rowptr, cols, vals, gat, epi, smw);
}
template <typename Gather, typename Epi>
__device__ __forceinline__ void check_gather(const int2* tiles, int ntiles, const int* rowptr, const int* cols,
                                             const double* vals, Gather& gat, Epi& epi, double* smw,
                                             const double* /*tag*/) {
  auto gat64 = [&](int i, double(&g)[2]) { gat(i, g); };
  spmv_tiles<2, false, double, double>(tiles, ntiles, rowptr, cols, vals, gat64, epi, smw, NoPro());
}

// QP: 0 an LP (no Hessian terms compiled in), 1 a quadratic objective (qq set), 2
// either, decided per column from qq (the persistent kernel, to keep one body)
template <typename T, int QP = 0, bool Coh = false>
struct CheckColsEpi {
  struct Pre {};
  const T* __restrict__ xc;
  T* __restrict__ xa;
  T* __restrict__ aty_c;
  T* __restrict__ aty_a;
  const T* __restrict__ xlr;
  const double *C, *invC, *c64, *l64, *u64;
  const double* qq;  // scaled Hessian diagonal of a quadratic objective, or null
  const unsigned char* int_mask;
  T w, w1;
  bool do_avg;
  double acc[kNC1];
  unsigned long long h;
  __device__ __forceinline__ Pre load(int) const { return Pre{}; }
  __device__ __forceinline__ void finish(int j, const double (&s)[2], const Pre&) {
    const T x = eload<Coh>(xc + j);
    T xav = eload<Coh>(xa + j);
    if (do_avg) {
      xav = blend(xav, x, w1, w);
      xa[j] = xav;
    }
    aty_c[j] = T(s[0]);
    aty_a[j] = T(s[1]);
    const double Cj = C[j], iCj = invC[j], cj = c64[j], lj = l64[j], uj = u64[j], xl = to_f64(eload<Coh>(xlr + j));
    const double xs[2] = {to_f64(x), to_f64(xav)};
    const bool has_q = QP == 1 || (QP == 2 && qq != nullptr);
    const double qj = has_q ? qq[j] : 0.0;
    // with both bounds finite the projection returns r itself, the dual residual
    // r - lambda is exactly 0 and its two squared norms are left as they are (the
    // same sums, without four FP64 instructions per iterate)
    const bool boxed = above_neg_inf(lj) && below_pos_inf(uj);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      // quadratic objective: reduced cost c + q x - A^T y; +-1/2 q x^2 in the objectives
      const double r = has_q ? (cj + qj * xs[q]) - s[q] : cj - s[q];
      const double lam = rc_proj(r, lj, uj);
      if (!boxed) {
        const double rd = r - lam;
        acc[5 * q + 0] += rd * rd;
        const double rdu = rd * iCj;
        acc[5 * q + 1] += rdu * rdu;
      }
      acc[5 * q + 2] += cj * xs[q];
      acc[5 * q + 3] += bound_term(lam, lj, uj);
      if (has_q) {
        const double hq = 0.5 * (qj * xs[q]) * xs[q];
        acc[5 * q + 2] += hq;
        acc[5 * q + 3] -= hq;
      }
      const double dd = xs[q] - xl;
      acc[5 * q + 4] += dd * dd;
    }
    if (int_mask[j]) h += round_hash(j, xs[0] * Cj);
  }
};

// FP64 column half of a check (Section 2.2): A^T y of the current and of the
// averaged dual from FP64 values, reduced costs, dual residuals, objectives, the
// rounding hash; block partials to part, hash into *hash
template <typename T, bool Coh, int QP = 0>
__device__ __forceinline__ void check_cols_phase(const DevLP<T>& d, const SlotView<T>& v, double* sm, double* part,
                                                 unsigned long long* hash) {
  const T w = v.w, w1 = v.w1;
  const bool do_avg = v.do_avg;
  const T* __restrict__ yc = d.Y[v.cur];
  const T* __restrict__ ya = d.Y[v.avg];
  CheckColsEpi<T, QP> epi;
  epi.xc = d.X[v.cur];
  epi.xa = d.X[v.avg];
  epi.aty_c = d.ATY[v.ia_cur];
  epi.aty_a = d.ATY[v.ia_avg];
  epi.xlr = d.XLR;
  epi.C = d.C;
  epi.invC = d.invC;
  epi.c64 = d.c64;
  epi.l64 = d.l64;
  epi.u64 = d.u64;
  epi.qq = d.q64;
  epi.int_mask = d.int_mask;
  epi.w = w;
  epi.w1 = w1;
  epi.do_avg = do_avg;
#pragma unroll
  for (int k = 0; k < kNC1; ++k) epi.acc[k] = 0.0;
  epi.h = 0ULL;
  auto gat = [&](int i, T(&g)[2]) {
    const T y = gload<Coh>(yc + i);
    T av = gload<Coh>(ya + i);
    if (do_avg) av = blend(av, y, w1, w);
    g[0] = y;
    g[1] = av;
  };
  check_gather(d.t_tiles, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals64, gat, epi,
               sm + (threadIdx.x >> 5) * 2 * kSmemPerWarp, static_cast<const T*>(nullptr));
  block_store_partials<kNC1>(epi.acc, part);
  const unsigned long long h = warp_sum_u64(epi.h);
  if ((threadIdx.x & 31) == 0 && h != 0ULL) atomicAdd(hash, h);
}

template <typename T, bool Coh = false>
struct CheckRowsEpi {
  struct Pre {};
  const T* __restrict__ yc;
  T* __restrict__ ya;
  T* __restrict__ ax_c;
  T* __restrict__ ax_a;
  const T* __restrict__ ylr;
  const double *invR, *lo64, *hi64;
  T w, w1;
  bool do_avg;
  double acc[kNC2];
  __device__ __forceinline__ Pre load(int) const { return Pre{}; }
  __device__ __forceinline__ void finish(int i, const double (&s)[2], const Pre&) {
    const T y = eload<Coh>(yc + i);
    T yav = eload<Coh>(ya + i);
    if (do_avg) {
      yav = blend(yav, y, w1, w);
      ya[i] = yav;
    }
    ax_c[i] = T(s[0]);
    ax_a[i] = T(s[1]);
    const double iRi = invR[i], lo = lo64[i], hi = hi64[i], yl = to_f64(eload<Coh>(ylr + i));
    const double ys[2] = {to_f64(y), to_f64(yav)};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double rps = s[q] - clampv<double>(s[q], lo, hi);
      acc[4 * q + 0] += rps * rps;
      const double rp = rps * iRi;
      acc[4 * q + 1] += rp * rp;
      acc[4 * q + 2] += bound_term(ys[q], lo, hi);
      const double dd = ys[q] - yl;
      acc[4 * q + 3] += dd * dd;
    }
  }
};

// FP64 row half of a check: A x of the current and averaged primal from FP64
// values (refreshing the cached products), primal residuals, dual objective rows
template <typename T, bool Coh>
__device__ __forceinline__ void check_rows_phase(const DevLP<T>& d, const SlotView<T>& v, double* sm, double* part) {
  const T* __restrict__ xc = d.X[v.cur];
  const T* __restrict__ xa = d.X[v.avg];
  CheckRowsEpi<T> epi;
  epi.yc = d.Y[v.cur];
  epi.ya = d.Y[v.avg];
  epi.ax_c = d.AX[v.cur];
  epi.ax_a = d.AX[v.avg];
  epi.ylr = d.YLR;
  epi.invR = d.invR;
  epi.lo64 = d.lo64;
  epi.hi64 = d.hi64;
  epi.w = v.w;
  epi.w1 = v.w1;
  epi.do_avg = v.do_avg;
#pragma unroll
  for (int k = 0; k < kNC2; ++k) epi.acc[k] = 0.0;
  auto gat = [&](int j, T(&g)[2]) {
    g[0] = gload<Coh>(xc + j);
    g[1] = gload<Coh>(xa + j);
  };
  check_gather(d.a_tiles, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals64, gat, epi,
               sm + (threadIdx.x >> 5) * 2 * kSmemPerWarp, static_cast<const T*>(nullptr));
  block_store_partials<kNC2>(epi.acc, part);
}

// QP = 1: the objective has a Hessian (d.q64 set); the LP variant (0) carries none of
// its terms
template <typename T, int QP = 0>
__global__ void __launch_bounds__(kThreads) k_check_cols(DevLP<T> d) {
  Control* ctl = d.ctl;
  pdl_enter();
  if (ctl->done) return;
  __shared__ double sm[2 * kWarpsPerBlock * kSmemPerWarp];
  check_cols_phase<T, false, QP>(d, make_view<T>(ctl), sm, d.part_c1, &ctl->hash_accum);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_check_rows(DevLP<T> d) {
  Control* ctl = d.ctl;
  pdl_enter();
  if (ctl->done) return;
  // the column check's block partials, one value per block, while the row blocks run
  for (int k = blockIdx.x; k < kNC1; k += gridDim.x) {
    const double v = block_column_sum<kNC1>(d.part_c1, d.grid_c1, k);
    if (threadIdx.x == 0) d.red_c1[k] = v;
  }
  __shared__ double sm[2 * kWarpsPerBlock * kSmemPerWarp];
  check_rows_phase<T, false>(d, make_view<T>(ctl), sm, d.part_c2);
  if (!is_last_block(&ctl->cnt_c2)) return;
  __shared__ double red[kNC1 + kNC2];
  static_assert(kNC2 * (kThreads - 32) <= 2 * kWarpsPerBlock * kSmemPerWarp, "reduction scratch");
  if (threadIdx.x < kNC1) red[threadIdx.x] = __ldcg(d.red_c1 + threadIdx.x);
  reduce_one<kNC2>(d.part_c2, d.grid_c2, sm, red + kNC1);
  fill_step_factors<T>(ctl, d.step_fac, d.n_check);
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0 && std::is_same<T, float>::value) sync_step_state(ctl);
    __syncwarp();
    check_control_warp(ctl, red, d.trace_checks, d.trace_cap);
    if (threadIdx.x == 0) ctl->cnt_c2 = 0;
  }
}

// ------------------------------------------------------ persistent solve kernel ---
// The whole solve in one cooperative launch (all blocks co-resident): per attempt a
// primal phase and a dual phase separated by grid barriers; after the dual barrier
// every block reduces the block partials itself, in the same fixed order, and so
// takes the same step-size decision on its own shared copy of the control block
// (no third barrier, no serial tail).  Checks run as two more phases.  Partials of
// consecutive attempts alternate between two buffers, so a block that is still
// reducing attempt s never sees attempt s+1's partials.  Every barrier wait is
// bounded by a time limit; on expiry the kernel records SCYLLA_DEVICE_TIMEOUT and
// all blocks return.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(GridBar* b, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (*verr) ok = 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_solve_persistent(DevLP<T> d, GridBar* bar,
                                                                  unsigned long long limit_ns) {
  extern __shared__ double psm[];  // 2 * kPWarps * kSmemPerWarp doubles
  __shared__ Control sc;
  __shared__ double fac[3 * kMaxNcheckPersistent];  // FP64 factors, then FP32 copies
  __shared__ double red[kNC1 + kNC2];
  typedef typename AccOf<T>::type A;
  __shared__ A sred[kNP + kND];
  __shared__ StepPre spre;
  const int nb = gridDim.x;
  double* pp = d.pp_part;  // [2][nb] primal, [2][2nb] dual, [10 nb] cols, [8 nb] rows
  double* part_p[2] = {pp, pp + nb};
  double* part_d[2] = {pp + 2 * nb, pp + 4 * nb};
  double* part_c1 = pp + 6 * nb;
  double* part_c2 = pp + 16 * nb;
  unsigned long long* hash = d.p_hash;  // two slots, alternating between checks
  if (threadIdx.x == 0) sc = *d.ctl;
  __syncthreads();
  const bool lead = blockIdx.x == 0;
  int hslot = 0;
  bool ok = true;
  long long since = 0;  // attempts since the last check
  bool do_check = true;  // the start point is evaluated first
  while (ok) {
    if (do_check) {
      const SlotView<T> v = make_view<T>(&sc);
      check_cols_phase<T, true, 2>(d, v, psm, part_c1, &hash[hslot]);
      ok = grid_sync(bar, limit_ns);
      if (!ok) break;
      check_rows_phase<T, true>(d, v, psm, part_c2);
      ok = grid_sync(bar, limit_ns);
      if (!ok) break;
      static_assert((kNC1 + kNC2) * (kPThreads - 32) <= 2 * kPWarps * kSmemPerWarp, "reduction scratch");
      reduce_two<kNC1, kNC2>(part_c1, nb, part_c2, nb, psm, red);
      fill_step_factors<T>(&sc, fac, d.n_check);
      if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
          sc.hash_accum = __ldcg(&hash[hslot]);
          if (std::is_same<T, float>::value) sync_step_state(&sc);
          if (lead) hash[hslot ^ 1] = 0ULL;  // the next check's slot; nobody reads it now
        }
        __syncwarp();
        check_control_warp(&sc, red, lead ? d.trace_checks : nullptr, d.trace_cap);
      }
      __syncthreads();
      hslot ^= 1;
      since = 0;
      do_check = false;
    }
    if (sc.done) break;
    if (sc.k >= sc.iter_limit || since == d.n_check) {
      do_check = true;
      continue;
    }
    const int par = int(sc.k & 1);
    const SlotView<T> v = make_view<T>(&sc);
    primal_phase<T, true>(d, v, reinterpret_cast<T*>(psm), acc_part<T>(part_p[par]));
    ok = grid_sync(bar, limit_ns);
    if (!ok) break;
    dual_phase<T, true>(d, v, reinterpret_cast<T*>(psm), acc_part<T>(part_d[par]));
    ok = grid_sync(bar, limit_ns);
    if (!ok) break;
    if (threadIdx.x == 0) spre = step_pre<A>(&sc, fac, d.n_check);
    reduce_step<A>(acc_part<T>(part_p[par]), nb, acc_part<T>(part_d[par]), nb, reinterpret_cast<A*>(psm), sred);
    if (threadIdx.x == 0) step_control<A>(&sc, spre, sred[0], sred[1], sred[2], lead ? d.trace_steps : nullptr,
                                          d.trace_cap);
    __syncthreads();
    ++since;
  }
  if (lead && threadIdx.x == 0) {
    if (!ok) {
      sc.done = 1;
      sc.status = SCYLLA_DEVICE_TIMEOUT;
    }
    *d.ctl = sc;
  }
}

__global__ void k_loop_ctl(Control* c, cudaGraphConditionalHandle h) {
  c->chunks++;
  if (!c->done && c->chunks >= c->max_chunks) {
    // safety net: the check at the iteration limit ends every solve before this
    c->done = 1;
    c->status = SCYLLA_ITER_LIMIT;
  }
  cudaGraphSetConditional(h, c->done ? 0u : 1u);
}

__global__ void k_solve_init(Control* c, double tol, long long iter_limit, int stall_checks,
                             long long max_chunks) {
  c->tol = tol;
  c->iter_limit = iter_limit;
  c->stall_checks = stall_checks;
  c->max_chunks = max_chunks;
  c->k = 0;
  c->k_lr = 0;
  c->wsum = 0.0;
  c->avg_w = 0.0;
  c->done = 0;
  c->status = -1;
  c->used_avg = 0;
  c->accepted = c->rejected = c->restarts = 0;
  c->chunks = 0;
  c->n_ctrace = 0;
  c->initial = 1;
  c->aty_valid = 0;
  c->copy_lr = 0;
  c->hash_accum = 0ULL;
  c->same_hash = 0;
  c->cnt_dual = c->cnt_c2 = c->cnt_misc = c->cnt_inf = 0;
  c->inf_tested = 0;
  c->inf_gap = -INFINITY;
  c->inf_scale = 0.0;
  derive_steps(c);
}

// ------------------------------------------------------------ state access ---
template <typename T>
__global__ void k_get_x(DevLP<T> d, double* out, int count) {
  const T* x = d.X[d.ctl->ix_cur];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x)
    out[j] = double(x[j]) * d.C[j];
}
template <typename T>
__global__ void k_get_y(DevLP<T> d, double* out, int count) {
  const T* y = d.Y[d.ctl->ix_cur];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = double(y[i]) * d.R[i];
}
template <typename T>
__global__ void k_set_xy(DevLP<T> d, const double* x, const double* y) {
  T* xc = d.X[d.ctl->ix_cur];
  T* yc = d.Y[d.ctl->ix_cur];
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) xc[j] = T(x[j] / d.C[j]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) yc[i] = T(y[i] / d.R[i]);
}
// x = proj_[l,u](0), y = 0 (Algorithm 1 initialisation, x projected onto its box)
template <typename T>
__global__ void k_init_point(DevLP<T> d) {
  T* xc = d.X[d.ctl->ix_cur];
  T* yc = d.Y[d.ctl->ix_cur];
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride)
    xc[j] = T(clampv<double>(0.0, d.l64[j], d.u64[j]));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) yc[i] = T(0);
}

// ------------------------------------------------------------ scaled vectors ---
// c~ = C c, [l~, u~] = [l, u] / C, [lo~, hi~] = R [lo, hi], and 1/R, 1/C when asked.
__global__ void k_scale_vectors(DevVecs v) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += stride) {
    const double cj = v.C[j];
    const double c = v.c[j] * cj, l = v.l[j] / cj, u = v.u[j] / cj;
    if (v.invC) v.invC[j] = 1.0 / cj;
    v.c64[j] = c;
    v.l64[j] = l;
    v.u64[j] = u;
    if (v.c32) {
      v.c32[j] = float(c);
      v.l32[j] = float(l);
      v.u32[j] = float(u);
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.m; i += stride) {
    const double ri = v.R[i];
    const double lo = v.lo[i] * ri, hi = v.hi[i] * ri;
    if (v.invR) v.invR[i] = 1.0 / ri;
    v.lo64[i] = lo;
    v.hi64[i] = hi;
    if (v.lo32) {
      v.lo32[i] = float(lo);
      v.hi32[i] = float(hi);
    }
  }
}

// ------------------------------------------------------- objective update ---
// The end of both objective kernels: the block's partials (offset terms, sum
// c_hat^2, sum of squared row-bound magnitudes) are summed in thread order into
// o.red[3 b + k]; the last block to finish reduces them over the blocks in a fixed
// order (reduce_one) and writes ||b|| (largest finite |lo|, |hi| per row), ||c_hat||
// and the offset (the reduced offset terms, or offset_base) to the control block.
__device__ void objective_finish(const DevObjective& o, double off, double c2, double b2, double offset_base,
                                 bool use_offset_terms) {
  __shared__ double sh[3][kThreads];
  sh[0][threadIdx.x] = off;
  sh[1][threadIdx.x] = c2;
  sh[2][threadIdx.x] = b2;
  __syncthreads();
  if (threadIdx.x < 3) {
    double a = 0.0;
    for (int q = 0; q < int(blockDim.x); ++q) a += sh[threadIdx.x][q];
    o.red[3 * blockIdx.x + threadIdx.x] = a;
    __threadfence();  // each writer publishes its partial before the block's ticket
  }
  if (!is_last_block(&o.ctl->cnt_misc)) return;
  __shared__ double scratch[3 * (kThreads - 32)];
  __shared__ double out[3];
  reduce_one<3>(o.red, int(gridDim.x), scratch, out);
  if (threadIdx.x == 0) {
    o.ctl->bnorm = sqrt(out[2]);
    o.ctl->cnorm = sqrt(out[1]);
    o.ctl->offset = use_offset_terms ? out[0] : offset_base;
    o.ctl->cnt_misc = 0;
  }
}

// squared magnitude of the largest finite bound of a row
__device__ __forceinline__ double row_bound2(double lo, double hi) {
  const double inf = pos_inf<double>();
  const double a = lo > -inf ? fabs(lo) : 0.0, b = hi < inf ? fabs(hi) : 0.0;
  const double v = fmax(a, b);
  return v * v;
}

// c_hat_j = alpha^K s c_j + (1 - alpha^K) g_j (Algorithm 1, Section 2.4): g_j = +1
// when xhat_j = l_j and -1 when xhat_j = u_j on integer columns with u - l = 1; a
// general integer column keeps alpha^K s c_j and its auxiliary column gets cost
// (1 - alpha^K) with auxiliary rows d - x >= -xhat_j, d + x >= xhat_j.
// The squared row-bound magnitudes are summed over the original rows here and, for
// the auxiliary rows (lo = -xhat_j, xhat_j; hi = +inf), where they are written.
// l2 mode (o.l2): c_hat_j = t c_j - om xhat_j, q_j = om on integer columns, c_hat_j =
// t c_j, q_j = 0 elsewhere; offset terms om/2 xhat_j^2 (no auxiliary columns).
__global__ void k_objective_cols(DevObjective o, double t, double om) {
  double off = 0.0, c2 = 0.0, b2 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < o.n; j += stride) {
    double ch;
    if (o.l2) {
      double qv = 0.0;
      if (j < o.n_orig && o.kind[j] >= 1) {
        const double xh = o.xhat[j];
        ch = __dadd_rn(__dmul_rn(t, o.c_orig[j]), -__dmul_rn(om, xh));
        qv = om;
        off += 0.5 * om * xh * xh;
      } else {
        ch = j < o.n_orig ? __dmul_rn(t, o.c_orig[j]) : 0.0;
      }
      const double Cj = o.C[j], qs = (qv * Cj) * Cj;
      o.q_un[j] = qv;
      o.q64[j] = qs;
      if (o.q32) o.q32[j] = float(qs);
    } else if (j < o.n_orig) {
      double g = 0.0;
      const int kd = o.kind[j];
      if (kd == 1) {
        const double xh = o.xhat[j];
        if (xh == o.l_orig[j]) {
          g = 1.0;
          off -= om * o.l_orig[j];
        } else if (xh == o.u_orig[j]) {
          g = -1.0;
          off += om * o.u_orig[j];
        }
      } else if (kd == 2) {
        const int tq = o.aux_of[j];
        const double xh = o.xhat[j];
        const int r0 = o.m_orig + 2 * tq;
        o.lo_unscaled[r0] = -xh;
        o.lo_unscaled[r0 + 1] = xh;
        b2 += row_bound2(-xh, o.hi_unscaled[r0]) + row_bound2(xh, o.hi_unscaled[r0 + 1]);
        const double l0 = -xh * o.R[r0], l1 = xh * o.R[r0 + 1];
        o.lo64[r0] = l0;
        o.lo64[r0 + 1] = l1;
        if (o.lo32) {
          o.lo32[r0] = float(l0);
          o.lo32[r0 + 1] = float(l1);
        }
      }
      ch = __dadd_rn(__dmul_rn(t, o.c_orig[j]), __dmul_rn(om, g));
    } else {
      ch = om;
    }
    o.chat[j] = ch;
    const double cs = ch * o.C[j];
    o.c64[j] = cs;
    if (o.c32) o.c32[j] = float(cs);
    c2 += ch * ch;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < o.m_orig; i += stride)
    b2 += row_bound2(o.lo_unscaled[i], o.hi_unscaled[i]);
  objective_finish(o, off, c2, b2, 0.0, true);
}

// the norms at create time without a change of c_hat: ||c_hat|| and ||b|| over all
// rows, offset = offset_base
__global__ void k_cnorm_cols(DevObjective o, double offset_base) {
  double c2 = 0.0, b2 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < o.n; j += stride) {
    const double ch = o.chat[j];
    c2 += ch * ch;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < o.m; i += stride)
    b2 += row_bound2(o.lo_unscaled[i], o.hi_unscaled[i]);
  objective_finish(o, 0.0, c2, b2, offset_base, false);
}

// ------------------------------------------------------------ batched solve ---
// Many LPs as one block-diagonal problem (the batched pattern of the pump: many
// relaxations of uneven size in one launch sequence).  Tiles never cross an LP
// boundary and carry their LP's index; every LP has its own control block, so its
// step size, pool roles, restarts and termination are its own.  Tiles of LPs that
// are finished (or waiting at their iteration limit) are skipped.  Sums are kept per
// tile and reduced per LP in a fixed order: for the step decision by the warp that
// finishes the LP's last tile of the dual step, for the checks by one warp per LP in
// the check control kernel; both run the same step and check logic as the single-LP
// path.

// One warp tile of the batched kernels (a multi-row tile or one long row): the
// products into the warp's skewed shared buffer, then each lane sums its row in CSR
// order and hands it to the epilogue.
template <int NV, typename Acc, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void batch_tile_at(int2 ta, int2 tb, const int* __restrict__ rowptr,
                                              const int* __restrict__ cols, const V* __restrict__ vals, Gather& gat,
                                              Epi& epi, Acc* __restrict__ sm) {
  const int lane = threadIdx.x & 31;
  const int r0 = ta.x, r1 = tb.x, p0 = ta.y, p1 = tb.y;
  const int base = p0 & ~(kVec - 1);
  if (r1 - r0 == 1 && p1 - p0 > kTileNnz) {
    const typename Epi::Pre pre = epi.load(r0);
    Acc s[NV];
    long_row_sum<NV, false>(p0, p1, cols, vals, gat, s);
    if (lane == 0) epi.finish(r0, s, pre);
  } else {
    const bool mine = lane < r1 - r0;
    const int row = r0 + lane;
    int q0 = 0, q1 = 0;
    typename Epi::Pre pre{};
    if (mine) {
      q0 = __ldg(rowptr + row) - p0;
      q1 = __ldg(rowptr + row + 1) - p0;
      pre = epi.load(row);
    }
    int c[3][4];
    V v[3][4];
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const int p = base + (it * 32 + lane) * kVec;
      if (p < p1) {
        ld4(cols + p, c[it]);
        ld4(vals + p, v[it]);
      }
    }
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const int p = base + (it * 32 + lane) * kVec;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int q = p + e;
        if (q >= p0 && q < p1) {
          Acc g[NV];
          gat(c[it][e], g);
          const int o = skew(q - p0);
#pragma unroll
          for (int k = 0; k < NV; ++k) sm[k * kSmemPerWarp + o] = Acc(v[it][e]) * g[k];
        }
      }
    }
    __syncwarp();
    if (mine) {
      Acc s[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = Acc(0);
      for (int q = q0; q < q1; ++q) {
        const int o = skew(q);
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += sm[k * kSmemPerWarp + o];
      }
      epi.finish(row, s, pre);
    }
    __syncwarp();
  }
}

// tile t of a batch: its bounds, then batch_tile_at
template <int NV, typename Acc, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void batch_tile(int t, const int2* __restrict__ tiles, const int* __restrict__ rowptr,
                                           const int* __restrict__ cols, const V* __restrict__ vals, Gather& gat,
                                           Epi& epi, Acc* __restrict__ sm) {
  batch_tile_at<NV, Acc, V>(__ldg(tiles + t), __ldg(tiles + t + 1), rowptr, cols, vals, gat, epi, sm);
}

// warp-tile loop of the batched kernels over a static deal of the tiles:
// begin(lp, t) decides per tile (uniformly over the warp) whether the tile's LP
// takes part, end(t) flushes the tile's sums.  The LP index and the bounds of the
// warp's next tile are loaded together, one tile ahead, so that neither waits on
// the other nor on the current tile's work.
template <int NV, typename Acc, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void spmv_tiles_batch(const int2* __restrict__ tiles, const int* __restrict__ tile_lp,
                                                 int ntiles, const int* __restrict__ rowptr,
                                                 const int* __restrict__ cols, const V* __restrict__ vals,
                                                 Gather& gat, Epi& epi, Acc* __restrict__ sm) {
  const WarpTiles wt = warp_tiles(ntiles);
  int lp_n = 0;
  int2 ta_n = make_int2(0, 0), tb_n = make_int2(0, 0);
  auto ahead = [&](int t) {
    if (t < wt.end) {
      lp_n = __ldg(tile_lp + t);
      ta_n = __ldg(tiles + t);
      tb_n = __ldg(tiles + t + 1);
    }
  };
  ahead(wt.first);
  for (int t = wt.first; t < wt.end; t += wt.step) {
    const int lp = lp_n;
    const int2 ta = ta_n, tb = tb_n;
    ahead(t + wt.step);
    if (!epi.begin(lp, t)) continue;
    batch_tile_at<NV, Acc, V>(ta, tb, rowptr, cols, vals, gat, epi, sm);
    epi.end(t);
  }
}

// The static deal of the batched kernels with the warp's next tile staged in shared
// memory by asynchronous copies, as spmv_tiles_async does for one LP: the next
// tile's LP index and bounds come a tile ahead, its LP's pool roles are read (an L2
// load, in the shadow of the current tile's gathers) when its copies are issued, and
// a tile of an LP that takes no part is neither staged nor computed.  Every tile's
// products, row sums and epilogue are those of batch_tile_at.
template <typename V, typename Gather, typename Epi>
__device__ __forceinline__ void spmv_tiles_batch_async(const int2* __restrict__ tiles,
                                                       const int* __restrict__ tile_lp, int ntiles,
                                                       const int* __restrict__ rowptr, const int* __restrict__ cols,
                                                       const V* __restrict__ vals, Gather& gat, Epi& epi,
                                                       V* __restrict__ sm, AsyncStage<V>& S) {
  static_assert(sizeof(V) == 4, "the asynchronous-copy form stages FP32 values");
  const int lane = threadIdx.x & 31;
  const WarpTiles wt = warp_tiles(ntiles);
  if (wt.first >= wt.end) return;
  const unsigned long long pol = l2_policy_evict_first();
  auto longrow_of = [](int2 a, int2 b) { return b.x - a.x == 1 && b.y - a.y > kTileNnz; };
  auto issue = [&](int lp, int2 ta, int2 tb) {
    const V* pv[5];
    const int mask = longrow_of(ta, tb) ? 0 : epi.stage_ptrs(lp, pv);
    if (mask) {
      const int base = ta.y & ~(kVec - 1);
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int o = (it * 32 + lane) * kVec, p = base + o;
        if (p < tb.y) {
          cpa16(&S.col[o], cols + p, pol);
          cpa16(&S.val[o], vals + p, pol);
        }
      }
      if (lane < tb.x - ta.x) {
        cpa4(&S.rp[lane], rowptr + ta.x + lane);
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if (mask & (1 << k)) cpa4(&S.pre[k][lane], pv[k] + ta.x + lane);
      }
    }
    cpa_commit();
  };
  int lc = __ldg(tile_lp + wt.first), ln = 0, ll = 0;
  int2 ca = __ldg(tiles + wt.first), cb = __ldg(tiles + wt.first + 1);
  int2 na = make_int2(0, 0), nb = make_int2(0, 0), la = make_int2(0, 0), lb = make_int2(0, 0);
  if (wt.first + wt.step < wt.end) {
    ln = __ldg(tile_lp + wt.first + wt.step);
    na = __ldg(tiles + wt.first + wt.step);
    nb = __ldg(tiles + wt.first + wt.step + 1);
  }
  issue(lc, ca, cb);
  for (int t = wt.first; t < wt.end; t += wt.step) {
    const int t2 = t + 2 * wt.step;
    if (t2 < wt.end) {
      ll = __ldg(tile_lp + t2);
      la = __ldg(tiles + t2);
      lb = __ldg(tiles + t2 + 1);
    }
    const int r0 = ca.x, r1 = cb.x, p0 = ca.y, p1 = cb.y;
    const int base = p0 & ~(kVec - 1);
    cpa_wait_all();
    __syncwarp();
    const bool on = epi.begin(lc, t);
    if (!on) {
      __syncwarp();
      if (t + wt.step < wt.end) issue(ln, na, nb);
    } else if (longrow_of(ca, cb)) {
      __syncwarp();
      if (t + wt.step < wt.end) issue(ln, na, nb);
      const typename Epi::Pre pre = epi.load(r0);
      V s[1];
      long_row_sum<1, false>(p0, p1, cols, vals, gat, s);
      if (lane == 0) epi.finish(r0, s, pre);
      epi.end(t);
    } else {
      const int nr = r1 - r0;
      const bool mine = lane < nr;
      int q0 = 0, q1 = 0;
      typename Epi::Pre pre{};
      if (mine) {
        q0 = S.rp[lane] - p0;
        q1 = (lane + 1 < nr ? S.rp[lane + 1] : p1) - p0;
        pre = epi.stage_pre(&S.pre[0][0], 32, lane);
      }
      V v[3][4], g[3][4];
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int o = (it * 32 + lane) * kVec, p = base + o;
        int4 ci = make_int4(0, 0, 0, 0);
        float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < p1) {
          ci = *reinterpret_cast<const int4*>(&S.col[o]);
          vi = *reinterpret_cast<const float4*>(&S.val[o]);
        }
        const int cc[4] = {ci.x, ci.y, ci.z, ci.w};
        const V vv[4] = {vi.x, vi.y, vi.z, vi.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          v[it][e] = V(0);
          g[it][e] = V(0);
          if (q >= p0 && q < p1) {
            V gg[1];
            gat(cc[e], gg);
            g[it][e] = gg[0];
            v[it][e] = vv[e];
          }
        }
      }
      __syncwarp();  // every lane has read the stage before it is refilled
      if (t + wt.step < wt.end) issue(ln, na, nb);
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const int p = base + (it * 32 + lane) * kVec;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int q = p + e;
          if (q >= p0 && q < p1) sm[skew(q - p0)] = v[it][e] * g[it][e];
        }
      }
      __syncwarp();
      if (mine) {
        V sum = V(0);
        for (int q = q0; q < q1; ++q) sum += sm[skew(q)];
        const V sv[1] = {sum};
        epi.finish(r0 + lane, sv, pre);
      }
      __syncwarp();
      epi.end(t);
    }
    lc = ln;
    ca = na;
    cb = nb;
    ln = ll;
    na = la;
    nb = lb;
  }
  cpa_wait_all();
}

// per-LP values of one attempt: L2 loads when the writer may be another block of
// the same launch (the persistent solve)
template <bool Coh, typename T>
__device__ __forceinline__ BatchSlot<T> read_slot(const BatchSlot<T>* p) {
  if (!Coh) return *p;
  BatchSlot<T> s;
  s.tau = __ldcg(&p->tau);
  s.sigma = __ldcg(&p->sigma);
  s.w = __ldcg(&p->w);
  s.w1 = __ldcg(&p->w1);
  s.cur = __ldcg(&p->cur);
  s.nxt = __ldcg(&p->nxt);
  s.avg = __ldcg(&p->avg);
  s.ia_cur = __ldcg(&p->ia_cur);
  s.ia_avg = __ldcg(&p->ia_avg);
  s.flags = __ldcg(&p->flags);
  return s;
}

template <typename T, bool Coh = false>
struct BPrimalEpi : PrimalEpi<T, Coh> {
  const DevBatch<T>* B;
  const T* ysrc;
  bool cached;
  __device__ __forceinline__ bool begin(int b, int) {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    if (!(s.flags & kSlotActive)) return false;
    const DevLP<T>& d = B->d;
    this->xc = d.X[s.cur];
    this->xn = d.X[s.nxt];
    this->xa = d.X[s.avg];
    this->aty = d.ATY[s.ia_cur];
    this->tau = s.tau;
    this->w = s.w;
    this->w1 = s.w1;
    this->do_avg = (s.flags & kSlotAvg) != 0;
    this->copy_lr = (s.flags & kSlotCopyLr) != 0;
    cached = (s.flags & kSlotCached) != 0;
    this->use_cached = cached;
    this->store_aty = !cached;
    ysrc = d.Y[s.cur];
    return true;
  }
  __device__ __forceinline__ void end(int t) {
    const typename AccOf<T>::type a = warp_sum(this->acc);
    if ((threadIdx.x & 31) == 0) B->tp_p[t] = double(a);
    this->acc = 0;
  }
  // the epilogue vectors of LP b in stage_vec's order, and the mask of those to
  // stage (0 when the LP takes no part)
  __device__ __forceinline__ int stage_ptrs(int b, const T* (&p)[5]) const {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    if (!(s.flags & kSlotActive)) return 0;
    const DevLP<T>& d = B->d;
    p[0] = d.X[s.cur];
    p[1] = this->cc;
    p[2] = this->ll;
    p[3] = this->uu;
    p[4] = d.X[s.avg];
    return (s.flags & kSlotAvg) ? 31 : 15;
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_bprimal(DevBatch<T> B) {
  __shared__ T sm[kWarpsPerBlock * kSmemPerWarp];
  const DevLP<T>& d = B.d;
  if (blockIdx.x == 0 && threadIdx.x == 0) ++*B.kglob;  // attempt counter of the LPs still running
  BPrimalEpi<T> epi;
  epi.B = &B;
  epi.xlr = d.XLR;
  epi.cc = d.c;
  epi.ll = d.l;
  epi.uu = d.u;
  epi.qq = nullptr;  // the batched solve takes LPs only
  epi.acc = 0;
  auto gat = [&](int i, T(&g)[1]) { g[0] = epi.cached ? T(0) : __ldg(epi.ysrc + i); };
  spmv_tiles_batch<1, T, T>(d.t_tiles, B.t_tile_lp, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals, gat, epi,
                            sm + (threadIdx.x >> 5) * kSmemPerWarp);
}

// device-scope release increment and acquire fence (the per-LP completion counters
// of the persistent batched kernel)
__device__ __forceinline__ unsigned int atom_add_release_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// a control block into a warp's shared copy (L2 loads) and back, word by word
__device__ __forceinline__ void ctl_in(Control* dst, const Control* src) {
  static_assert(sizeof(Control) % 4 == 0, "word copy");
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < int(sizeof(Control) / 4); i += 32)
    reinterpret_cast<int*>(dst)[i] = __ldcg(reinterpret_cast<const int*>(src) + i);
  __syncwarp();
}
__device__ __forceinline__ void ctl_out(Control* dst, const Control* src) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < int(sizeof(Control) / 4); i += 32)
    reinterpret_cast<int*>(dst)[i] = reinterpret_cast<const int*>(src)[i];
  __syncwarp();
}

// the decision of one LP on its shared control copy: out of line, so that its
// registers do not count against the matrix phases of the persistent kernel
template <typename T>
__device__ __noinline__ void bq_decide(Control* sc, double s0, double s1, double s2, const double* fac, int n_check,
                                       BatchSlot<T>* slot, int* n_done) {
  step_control(sc, s0, s1, s2, fac, n_check, nullptr, 0);
  if (sc->done) atomicAdd(n_done, 1);
  write_slot(slot, sc);
}

// Sum over an LP's tiles of one per-tile value (part[t * stride + off], t in
// [beg, end)), by one warp: each lane keeps four running sums over its tiles
// (t = beg + lane, + 32, ...), taken round-robin, so four loads per lane are in
// flight; then the four in a fixed order and a fixed shuffle tree.  Per-tile sums are
// written in the same launch, so they are read from L2.
__device__ __forceinline__ double lp_tile_sum(const double* part, int stride, int off, int beg, int end) {
  const int lane = threadIdx.x & 31;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  int t = beg + lane;
  for (; t + 96 < end; t += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] += __ldcg(part + size_t(t + 32 * u) * stride + off);
  }
  for (int u = 0; t < end; t += 32, ++u) a[u & 3] += __ldcg(part + size_t(t) * stride + off);
  return warp_sum((a[0] + a[1]) + (a[2] + a[3]));
}

// The step decision of LP lp by one warp, from its per-tile sums of this attempt:
// out of line, so its registers do not count against the dual step's tile loop.
// sc: a shared-memory copy for the control block (the persistent kernel, where
// another block may have written it), or null (read and written in place).
template <typename T>
__device__ __noinline__ void lp_step_decision(const DevBatch<T>* B, int lp, Control* sc) {
  const int lane = threadIdx.x & 31;
  const int tb = __ldg(B->t_tile_beg + lp), te = __ldg(B->t_tile_beg + lp + 1);
  const int ab = __ldg(B->a_tile_beg + lp), ae = __ldg(B->a_tile_beg + lp + 1);
  const double s0 = lp_tile_sum(B->tp_p, 1, 0, tb, te);
  const double s1 = lp_tile_sum(B->tp_d, 2, 0, ab, ae);
  const double s2 = lp_tile_sum(B->tp_d, 2, 1, ab, ae);
  if (sc) {
    ctl_in(sc, B->ctl + lp);
    if (lane == 0) bq_decide<T>(sc, s0, s1, s2, B->d.step_fac, B->d.n_check, &B->slot[lp], B->n_done);
    ctl_out(B->ctl + lp, sc);
  } else if (lane == 0) {
    Control* c = &B->ctl[lp];
    step_control(c, s0, s1, s2, B->d.step_fac, B->d.n_check, nullptr, 0);
    if (c->done) atomicAdd(B->n_done, 1);
    write_slot(&B->slot[lp], c);
  }
  if (lane == 0) B->lp_cnt[lp] = 0u;
}

template <typename T, bool Coh = false>
struct BDualEpi : DualEpi<T, Coh> {
  const DevBatch<T>* B;
  const T* xsrc;
  int lp;
  Control* sc;  // a shared-memory copy for the decision (the persistent kernel), or null
  __device__ __forceinline__ bool begin(int b, int) {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    lp = b;
    if (!(s.flags & kSlotActive)) return false;
    const DevLP<T>& d = B->d;
    this->axc = d.AX[s.cur];
    this->axn = d.AX[s.nxt];
    this->yc = d.Y[s.cur];
    this->yn = d.Y[s.nxt];
    this->ya = d.Y[s.avg];
    this->sigma = s.sigma;
    this->w = s.w;
    this->w1 = s.w1;
    this->do_avg = (s.flags & kSlotAvg) != 0;
    this->copy_lr = (s.flags & kSlotCopyLr) != 0;
    xsrc = d.X[s.nxt];
    return true;
  }
  // the tile's sums; in the persistent kernel (Coh) the warp that finishes the
  // LP's last tile of this attempt takes the LP's step decision (its primal sums are
  // complete since the primal step came before): the tile's sums are released to the
  // LP's counter by its increment, and the last one acquires them all
  __device__ __forceinline__ void end(int t) {
    const typename AccOf<T>::type a0 = warp_sum(this->acc0), a1 = warp_sum(this->acc1);
    const int lane = threadIdx.x & 31;
    int last = 0;
    if (lane == 0) {
      B->tp_d[2 * t] = double(a0);
      B->tp_d[2 * t + 1] = double(a1);
      if (Coh) {
        const unsigned int ntiles = unsigned(__ldg(B->a_tile_beg + lp + 1) - __ldg(B->a_tile_beg + lp));
        last = atom_add_release_gpu(B->lp_cnt + lp, 1u) == ntiles - 1u;
      }
    }
    this->acc0 = 0;
    this->acc1 = 0;
    if (!Coh || !__shfl_sync(0xffffffffu, last, 0)) return;
    fence_acquire_gpu();
    lp_step_decision<T>(B, lp, sc);
  }
  __device__ __forceinline__ int stage_ptrs(int b, const T* (&p)[5]) const {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    if (!(s.flags & kSlotActive)) return 0;
    const DevLP<T>& d = B->d;
    p[0] = d.AX[s.cur];
    p[1] = d.Y[s.cur];
    p[2] = this->lo;
    p[3] = this->hi;
    p[4] = d.Y[s.avg];
    return (s.flags & kSlotAvg) ? 31 : 15;
  }
};

// one warp per LP: its tiles' sums in a fixed order, then the step decision (the
// launch-per-phase path)
template <typename T>
__global__ void k_bstep_control(DevBatch<T> B) {
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B.nlp) return;
  if (!(B.slot[b].flags & kSlotActive)) return;
  lp_step_decision<T>(&B, b, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_bdual(DevBatch<T> B) {
  __shared__ T sm[kWarpsPerBlock * kSmemPerWarp];
  const DevLP<T>& d = B.d;
  BDualEpi<T> epi;
  epi.B = &B;
  epi.sc = nullptr;
  epi.ylr = d.YLR;
  epi.lo = d.lo;
  epi.hi = d.hi;
  epi.acc0 = 0;
  epi.acc1 = 0;
  auto gat = [&](int j, T(&g)[1]) { g[0] = __ldg(epi.xsrc + j); };
  spmv_tiles_batch<1, T, T>(d.a_tiles, B.a_tile_lp, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals, gat, epi,
                            sm + (threadIdx.x >> 5) * kSmemPerWarp);
}

// the attempt kernels of the static deal with asynchronous-copy staging (FP32)
__global__ void __launch_bounds__(kThreads, 3) k_bprimal_as(DevBatch<float> B) {
  __shared__ float sm[kWarpsPerBlock * kSmemPerWarp];
  __shared__ __align__(16) AsyncStage<float> stg[kWarpsPerBlock];
  const DevLP<float>& d = B.d;
  if (blockIdx.x == 0 && threadIdx.x == 0) ++*B.kglob;  // attempt counter of the LPs still running
  BPrimalEpi<float> epi;
  epi.B = &B;
  epi.xlr = d.XLR;
  epi.cc = d.c;
  epi.ll = d.l;
  epi.uu = d.u;
  epi.qq = nullptr;
  epi.acc = 0;
  auto gat = [&](int i, float(&g)[1]) { g[0] = epi.cached ? 0.f : __ldg(epi.ysrc + i); };
  const int w = threadIdx.x >> 5;
  spmv_tiles_batch_async<float>(d.t_tiles, B.t_tile_lp, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals, gat, epi,
                                sm + w * kSmemPerWarp, stg[w]);
}

__global__ void __launch_bounds__(kThreads, 3) k_bdual_as(DevBatch<float> B) {
  __shared__ float sm[kWarpsPerBlock * kSmemPerWarp];
  __shared__ __align__(16) AsyncStage<float> stg[kWarpsPerBlock];
  const DevLP<float>& d = B.d;
  BDualEpi<float> epi;
  epi.B = &B;
  epi.sc = nullptr;
  epi.ylr = d.YLR;
  epi.lo = d.lo;
  epi.hi = d.hi;
  epi.acc0 = 0;
  epi.acc1 = 0;
  auto gat = [&](int j, float(&g)[1]) { g[0] = __ldg(epi.xsrc + j); };
  const int w = threadIdx.x >> 5;
  spmv_tiles_batch_async<float>(d.a_tiles, B.a_tile_lp, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals, gat, epi,
                                sm + w * kSmemPerWarp, stg[w]);
}

template <typename T, bool Coh = false>
struct BCheckColsEpi : CheckColsEpi<T, 0, Coh> {
  const DevBatch<T>* B;
  const T* ycur;
  const T* yavg;
  T bw, bw1;
  bool bavg;
  int lp;
  __device__ __forceinline__ bool begin(int b, int) {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    if (!(s.flags & kSlotCheck)) return false;
    const DevLP<T>& d = B->d;
    this->xc = d.X[s.cur];
    this->xa = d.X[s.avg];
    this->aty_c = d.ATY[s.ia_cur];
    this->aty_a = d.ATY[s.ia_avg];
    this->w = s.w;
    this->w1 = s.w1;
    this->do_avg = (s.flags & kSlotAvg) != 0;
    bw = s.w;
    bw1 = s.w1;
    bavg = this->do_avg;
    ycur = d.Y[s.cur];
    yavg = d.Y[s.avg];
    lp = b;
    return true;
  }
  __device__ __forceinline__ void end(int t) {
#pragma unroll
    for (int k = 0; k < kNC1; ++k) {
      const double a = warp_sum(this->acc[k]);
      if ((threadIdx.x & 31) == 0) B->tp_c1[kNC1 * t + k] = a;
      this->acc[k] = 0.0;
    }
    const unsigned long long h = warp_sum_u64(this->h);
    if ((threadIdx.x & 31) == 0 && h != 0ULL) atomicAdd(&B->ctl[lp].hash_accum, h);
    this->h = 0ULL;
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bcheck_cols(DevBatch<T> B) {
  __shared__ double sm[2 * kWarpsPerBlock * kSmemPerWarp];
  const DevLP<T>& d = B.d;
  BCheckColsEpi<T> epi;
  epi.B = &B;
  epi.xlr = d.XLR;
  epi.C = d.C;
  epi.invC = d.invC;
  epi.c64 = d.c64;
  epi.l64 = d.l64;
  epi.u64 = d.u64;
  epi.qq = d.q64;
  epi.int_mask = d.int_mask;
#pragma unroll
  for (int k = 0; k < kNC1; ++k) epi.acc[k] = 0.0;
  epi.h = 0ULL;
  auto gat = [&](int i, double(&g)[2]) {
    const T y = epi.ycur[i];
    T av = epi.yavg[i];
    if (epi.bavg) av = blend(av, y, epi.bw1, epi.bw);
    g[0] = double(y);
    g[1] = double(av);
  };
  spmv_tiles_batch<2, double, double>(d.t_tiles, B.t_tile_lp, d.t_ntiles, d.t_rowptr, d.t_cols, d.t_vals64, gat,
                                      epi, sm + (threadIdx.x >> 5) * 2 * kSmemPerWarp);
}

template <typename T, bool Coh = false>
struct BCheckRowsEpi : CheckRowsEpi<T, Coh> {
  const DevBatch<T>* B;
  const T* xcur;
  const T* xavg;
  __device__ __forceinline__ bool begin(int b, int) {
    const BatchSlot<T> s = read_slot<Coh>(B->slot + b);
    if (!(s.flags & kSlotCheck)) return false;
    const DevLP<T>& d = B->d;
    this->yc = d.Y[s.cur];
    this->ya = d.Y[s.avg];
    this->ax_c = d.AX[s.cur];
    this->ax_a = d.AX[s.avg];
    this->w = s.w;
    this->w1 = s.w1;
    this->do_avg = (s.flags & kSlotAvg) != 0;
    xcur = d.X[s.cur];
    xavg = d.X[s.avg];
    return true;
  }
  __device__ __forceinline__ void end(int t) {
#pragma unroll
    for (int k = 0; k < kNC2; ++k) {
      const double a = warp_sum(this->acc[k]);
      if ((threadIdx.x & 31) == 0) B->tp_c2[kNC2 * t + k] = a;
      this->acc[k] = 0.0;
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bcheck_rows(DevBatch<T> B) {
  __shared__ double sm[2 * kWarpsPerBlock * kSmemPerWarp];
  const DevLP<T>& d = B.d;
  BCheckRowsEpi<T> epi;
  epi.B = &B;
  epi.ylr = d.YLR;
  epi.invR = d.invR;
  epi.lo64 = d.lo64;
  epi.hi64 = d.hi64;
#pragma unroll
  for (int k = 0; k < kNC2; ++k) epi.acc[k] = 0.0;
  auto gat = [&](int j, double(&g)[2]) {
    g[0] = double(epi.xcur[j]);
    g[1] = double(epi.xavg[j]);
  };
  spmv_tiles_batch<2, double, double>(d.a_tiles, B.a_tile_lp, d.a_ntiles, d.a_rowptr, d.a_cols, d.a_vals64, gat,
                                      epi, sm + (threadIdx.x >> 5) * 2 * kSmemPerWarp);
}

// one warp per LP: its check sums in a fixed order, then termination / stalling /
// restart (check_control); block 0 also refills the shared step-size factor table
// for the next n_check attempts (every LP still running is at the same attempt)
template <typename T>
__global__ void k_bcheck_control(DevBatch<T> B) {
  if (blockIdx.x == 0) {
    const long long k = *B.kglob;
    for (int i = threadIdx.x; i < B.d.n_check; i += blockDim.x) {
      const double kk = double(k + 1 + i + 1);
      B.d.step_fac[2 * i] = 1.0 - pow(kk, -B.exp_red);
      B.d.step_fac[2 * i + 1] = 1.0 + pow(kk, -B.exp_grow);
    }
  }
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= B.nlp) return;
  if (!(B.slot[b].flags & kSlotCheck)) return;
  double r[kNC1 + kNC2];
#pragma unroll
  for (int k = 0; k < kNC1 + kNC2; ++k) r[k] = 0.0;
  for (int t = B.t_tile_beg[b] + lane; t < B.t_tile_beg[b + 1]; t += 32)
#pragma unroll
    for (int k = 0; k < kNC1; ++k) r[k] += B.tp_c1[kNC1 * t + k];
  for (int t = B.a_tile_beg[b] + lane; t < B.a_tile_beg[b + 1]; t += 32)
#pragma unroll
    for (int k = 0; k < kNC2; ++k) r[kNC1 + k] += B.tp_c2[kNC2 * t + k];
#pragma unroll
  for (int k = 0; k < kNC1 + kNC2; ++k) r[k] = warp_sum(r[k]);
  if (lane == 0) {
    Control* c = &B.ctl[b];
    c->k_fac = *B.kglob;
    check_control(c, r, nullptr, 0);
    if (c->done) atomicAdd(B.n_done, 1);
    write_slot(&B.slot[b], c);
  }
}

// cold start of every LP: solve-init fields, slots
template <typename T>
__global__ void k_binit(DevBatch<T> B, double tol, long long iter_limit, int stall_checks) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    *B.kglob = 0;
    *B.n_done = 0;
  }
  if (b >= B.nlp) return;
  B.lp_cnt[b] = 0u;
  Control* c = &B.ctl[b];
  c->tol = tol;
  c->iter_limit = iter_limit;
  c->stall_checks = stall_checks;
  c->k = 0;
  c->k_lr = 0;
  c->k_fac = 0;
  c->wsum = 0.0;
  c->avg_w = 0.0;
  c->done = 0;
  c->status = -1;
  c->used_avg = 0;
  c->accepted = c->rejected = c->restarts = 0;
  c->initial = 1;
  c->aty_valid = 0;
  c->copy_lr = 0;
  c->hash_accum = 0ULL;
  c->same_hash = 0;
  derive_steps(c);
  write_slot(&B.slot[b], c);
}

template <typename T>
__global__ void k_bget_x(DevBatch<T> B, int b, int col0, int count, double* out) {
  const T* x = B.d.X[B.ctl[b].ix_cur];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x)
    out[j] = double(x[col0 + j]) * B.d.C[col0 + j];
}

template <typename T>
__global__ void k_binit_point(DevBatch<T> B) {
  const DevLP<T>& d = B.d;
  const int stride = gridDim.x * blockDim.x;
  // every LP starts with the same pool roles (0 current, 1 next, 2 average)
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride)
    d.X[0][j] = T(clampv<double>(0.0, d.l64[j], d.u64[j]));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) d.Y[0][i] = T(0);
}


// ------------------------------------- persistent batched solve over a work queue ---
// One cooperative launch runs the attempts between two checks.  The two phases of
// an attempt (primal; dual with the step decisions) are separated by bounded grid
// barriers.  In the matrix phases warps take the tiles of a list of the tiles of
// the LPs still running: a contiguous share each, then the rest in chunks of
// kQChunk from a shared counter, so the work is balanced over the grid whatever the
// sizes of the LPs; after every check the LPs that finished are dropped from the
// lists (compaction), so their tiles are not visited again.  The
// arithmetic per tile and the per-LP reduction of the per-tile sums are those of
// the launch-per-phase path (same functions, same order), so the two give
// identical results.  Work moves between blocks from one phase to the next, so
// every load of data written during the launch goes to L2 (ld.global.cg): the
// vectors, slots, control blocks, per-tile sums and lists.
constexpr int kQChunk = 4;          // tiles a warp takes from a queue at once

// The tiles of a work list for one phase: each warp first works through its own
// contiguous share of the first three quarters of the list (no atomics), then the
// warps take the last quarter kQChunk tiles at a time from the shared counter, which
// evens out the finishing times whatever the tiles' costs.
template <int NV, typename Acc, typename V, typename Gather, typename Epi>
__device__ __forceinline__ void queue_tiles(const int* list, int count, unsigned int* ctr, const int2* tiles,
                                            const int* tile_lp, const int* rowptr, const int* cols, const V* vals,
                                            Gather& gat, Epi& epi, Acc* sm) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  auto one = [&](int v) {
    const int t = __ldcg(list + v);
    if (!epi.begin(__ldg(tile_lp + t), t)) return;
    batch_tile<NV, Acc, V>(t, tiles, rowptr, cols, vals, gat, epi, sm);
    epi.end(t);
  };
  const int per = int((3LL * count) / (4LL * nw));
  for (int v = gw * per; v < (gw + 1) * per; ++v) one(v);
  const int head = per * nw;
  for (;;) {
    int v0 = 0;
    if (lane == 0) v0 = head + int(atomicAdd(ctr, unsigned(kQChunk)));
    v0 = __shfl_sync(0xffffffffu, v0, 0);
    if (v0 >= count) break;
    const int v1 = min(count, v0 + kQChunk);
    for (int v = v0; v < v1; ++v) one(v);
  }
}

template <typename T>
__device__ __forceinline__ void bq_primal(const DevBatch<T>& B, int count, T* sm) {
  const DevLP<T>& d = B.d;
  BPrimalEpi<T, true> epi;
  epi.B = &B;
  epi.xlr = d.XLR;
  epi.cc = d.c;
  epi.ll = d.l;
  epi.uu = d.u;
  epi.qq = nullptr;
  epi.acc = 0;
  auto gat = [&](int i, T(&g)[1]) { g[0] = epi.cached ? T(0) : __ldcg(epi.ysrc + i); };
  queue_tiles<1, T, T>(B.q_t, count, B.q_ctr + 0, d.t_tiles, B.t_tile_lp, d.t_rowptr, d.t_cols, d.t_vals, gat, epi,
                       sm);
}

template <typename T>
__device__ __forceinline__ void bq_dual(const DevBatch<T>& B, int count, T* sm, Control* sc) {
  const DevLP<T>& d = B.d;
  BDualEpi<T, true> epi;
  epi.B = &B;
  epi.sc = sc;
  epi.ylr = d.YLR;
  epi.lo = d.lo;
  epi.hi = d.hi;
  epi.acc0 = 0;
  epi.acc1 = 0;
  auto gat = [&](int j, T(&g)[1]) { g[0] = __ldcg(epi.xsrc + j); };
  queue_tiles<1, T, T>(B.q_a, count, B.q_ctr + 1, d.a_tiles, B.a_tile_lp, d.a_rowptr, d.a_cols, d.a_vals, gat, epi,
                       sm);
}

template <typename T>
__device__ __forceinline__ void bq_check_cols(const DevBatch<T>& B, int count, double* sm) {
  const DevLP<T>& d = B.d;
  BCheckColsEpi<T, true> epi;
  epi.B = &B;
  epi.xlr = d.XLR;
  epi.C = d.C;
  epi.invC = d.invC;
  epi.c64 = d.c64;
  epi.l64 = d.l64;
  epi.u64 = d.u64;
  epi.qq = nullptr;
  epi.int_mask = d.int_mask;
#pragma unroll
  for (int k = 0; k < kNC1; ++k) epi.acc[k] = 0.0;
  epi.h = 0ULL;
  auto gat = [&](int i, double(&g)[2]) {
    const T y = __ldcg(epi.ycur + i);
    T av = __ldcg(epi.yavg + i);
    if (epi.bavg) av = blend(av, y, epi.bw1, epi.bw);
    g[0] = double(y);
    g[1] = double(av);
  };
  queue_tiles<2, double, double>(B.q_t, count, B.q_ctr + 2, d.t_tiles, B.t_tile_lp, d.t_rowptr, d.t_cols, d.t_vals64,
                                 gat, epi, sm);
}

template <typename T>
__device__ __forceinline__ void bq_check_rows(const DevBatch<T>& B, int count, double* sm) {
  const DevLP<T>& d = B.d;
  BCheckRowsEpi<T, true> epi;
  epi.B = &B;
  epi.ylr = d.YLR;
  epi.invR = d.invR;
  epi.lo64 = d.lo64;
  epi.hi64 = d.hi64;
#pragma unroll
  for (int k = 0; k < kNC2; ++k) epi.acc[k] = 0.0;
  auto gat = [&](int j, double(&g)[2]) {
    g[0] = double(__ldcg(epi.xcur + j));
    g[1] = double(__ldcg(epi.xavg + j));
  };
  queue_tiles<2, double, double>(B.q_a, count, B.q_ctr + 3, d.a_tiles, B.a_tile_lp, d.a_rowptr, d.a_cols, d.a_vals64,
                                 gat, epi, sm);
}

// termination, stalling and restarts of every LP in the list; block 0 refills the
// shared step-size factor table for the next n_check attempts
template <typename T>
__device__ __forceinline__ void bq_check_control(const DevBatch<T>& B, int nl, Control* sc) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const long long k = __ldcg(B.kglob);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < B.d.n_check; i += blockDim.x) {
      const double kk = double(k + 1 + i + 1);
      B.d.step_fac[2 * i] = 1.0 - pow(kk, -B.exp_red);
      B.d.step_fac[2 * i + 1] = 1.0 + pow(kk, -B.exp_grow);
    }
  for (int q = gw; q < nl; q += nw) {
    const int b = __ldcg(B.q_lps + q);
    if (!(__ldcg(&B.slot[b].flags) & kSlotCheck)) continue;
    double r[kNC1 + kNC2];
#pragma unroll
    for (int s = 0; s < kNC1 + kNC2; ++s) r[s] = 0.0;
    for (int t = __ldg(B.t_tile_beg + b) + lane; t < __ldg(B.t_tile_beg + b + 1); t += 32)
#pragma unroll
      for (int s = 0; s < kNC1; ++s) r[s] += __ldcg(B.tp_c1 + kNC1 * t + s);
    for (int t = __ldg(B.a_tile_beg + b) + lane; t < __ldg(B.a_tile_beg + b + 1); t += 32)
#pragma unroll
      for (int s = 0; s < kNC2; ++s) r[kNC1 + s] += __ldcg(B.tp_c2 + kNC2 * t + s);
#pragma unroll
    for (int s = 0; s < kNC1 + kNC2; ++s) r[s] = warp_sum(r[s]);
    ctl_in(sc, B.ctl + b);
    if (lane == 0) {
      sc->k_fac = k;
      check_control(sc, r, nullptr, 0);
      if (sc->done) atomicAdd(B.n_done, 1);
      write_slot(&B.slot[b], sc);
    }
    ctl_out(B.ctl + b, sc);
  }
}

// block-wide exclusive prefix sums of three counts (blockDim.x threads); returns
// the block totals
__device__ __forceinline__ int3 block_scan3(int3 v, int3& excl) {
  __shared__ int3 wsum[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int3 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, inc.x, o), b = __shfl_up_sync(0xffffffffu, inc.y, o),
              c = __shfl_up_sync(0xffffffffu, inc.z, o);
    if (lane >= o) {
      inc.x += a;
      inc.y += b;
      inc.z += c;
    }
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int3 off = make_int3(0, 0, 0), tot = make_int3(0, 0, 0);
  for (int q = 0; q < int(blockDim.x >> 5); ++q) {
    if (q < w) {
      off.x += wsum[q].x;
      off.y += wsum[q].y;
      off.z += wsum[q].z;
    }
    tot.x += wsum[q].x;
    tot.y += wsum[q].y;
    tot.z += wsum[q].z;
  }
  excl = make_int3(off.x + inc.x - v.x, off.y + inc.y - v.y, off.z + inc.z - v.z);
  __syncthreads();
  return tot;
}

// compaction (block 0): the LPs of the list that are not finished, in list order,
// with prefix sums of their tile counts; the chunk counters rearmed
template <typename T>
__device__ __forceinline__ void bq_compact_lps(const DevBatch<T>& B, int nl) {
  int kept = 0, na = 0, nt = 0;
  int* pre_a = B.q_pre;
  int* pre_t = B.q_pre + (B.nlp + 1);
  for (int base = 0; base < nl; base += blockDim.x) {
    const int q = base + threadIdx.x;
    int b = -1;
    int3 v = make_int3(0, 0, 0);
    if (q < nl) {
      b = __ldcg(B.q_lps + q);
      if (__ldcg(&B.slot[b].flags) & kSlotCheck) {
        v.x = 1;
        v.y = __ldg(B.a_tile_beg + b + 1) - __ldg(B.a_tile_beg + b);
        v.z = __ldg(B.t_tile_beg + b + 1) - __ldg(B.t_tile_beg + b);
      }
    }
    int3 ex;
    const int3 tot = block_scan3(v, ex);  // its barriers also order the reads above before the writes below
    if (v.x) {
      B.q_lps[kept + ex.x] = b;
      pre_a[kept + ex.x] = na + ex.y;
      pre_t[kept + ex.x] = nt + ex.z;
    }
    kept += tot.x;
    na += tot.y;
    nt += tot.z;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pre_a[kept] = na;
    pre_t[kept] = nt;
    B.q_cnt[0] = kept;
    B.q_cnt[1] = na;
    B.q_cnt[2] = nt;
    for (int c = 0; c < 4; ++c) B.q_ctr[c] = 0u;
  }
}

// the tile lists of the compacted LP list: a warp per LP copies its tile ranges
template <typename T>
__device__ __forceinline__ void bq_fill_tiles(const DevBatch<T>& B, int nl) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int* pre_a = B.q_pre;
  const int* pre_t = B.q_pre + (B.nlp + 1);
  for (int q = gw; q < nl; q += nw) {
    const int b = __ldcg(B.q_lps + q);
    const int a0 = __ldg(B.a_tile_beg + b), a1 = __ldg(B.a_tile_beg + b + 1);
    const int t0 = __ldg(B.t_tile_beg + b), t1 = __ldg(B.t_tile_beg + b + 1);
    const int da = __ldcg(pre_a + q), dt = __ldcg(pre_t + q);
    for (int i = lane; i < a1 - a0; i += 32) B.q_a[da + i] = a0 + i;
    for (int i = lane; i < t1 - t0; i += 32) B.q_t[dt + i] = t0 + i;
  }
}

// The attempts between two checks in one cooperative launch: primal phase, dual
// phase and step decisions per attempt, separated by bounded grid barriers, until
// n_check attempts are made or the iteration limit is reached.  The checks, and the
// compaction of the work lists after them, run as ordinary kernels between launches.
template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value)
    k_battempts_persistent(DevBatch<T> B, GridBar* bar, long long iter_limit, unsigned long long limit_ns) {
  __shared__ T sm[kWarpsPerBlock * kSmemPerWarp];
  __shared__ Control sctl[kWarpsPerBlock];
  const int w = threadIdx.x >> 5;
  T* smw = sm + w * kSmemPerWarp;
  const int nl = __ldcg(B.q_cnt + 0), na = __ldcg(B.q_cnt + 1), nt = __ldcg(B.q_cnt + 2);
  if (nl == 0) return;
  // attempts before this launch (a previous launch wrote it).  Every block reads it
  // before its first barrier and block 0 counts an attempt only after that barrier,
  // so all blocks see the same value and make the same number of attempts.
  const long long k0 = __ldcg(B.kglob);
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  for (int since = 0; since < B.d.n_check && k0 + since < iter_limit; ++since) {
    // the primal step (block 0 rearms the dual counter, which nobody takes from
    // until after the next barrier)
    if (lead) B.q_ctr[1] = 0u;
    bq_primal<T>(B, nt, smw);
    if (!grid_sync(bar, limit_ns)) return;
    // the dual step, whose last tile of each LP takes that LP's step decision; block
    // 0 counts the attempt (read only by the check after this launch)
    if (lead) {
      B.q_ctr[0] = 0u;
      ++*B.kglob;
    }
    bq_dual<T>(B, na, smw, &sctl[w]);
    if (!grid_sync(bar, limit_ns)) return;
  }
}

// after a check: the LP list without the LPs that finished (one block), then the
// tile lists of the LPs kept (every block)
template <typename T>
__global__ void k_bcompact(DevBatch<T> B) {
  bq_compact_lps<T>(B, B.q_cnt[0]);
}
template <typename T>
__global__ void k_bfill_tiles(DevBatch<T> B) {
  bq_fill_tiles<T>(B, B.q_cnt[0]);
}

// every LP and every tile in the work lists (in order), counters zeroed
template <typename T>
__global__ void k_bqueue_reset(DevBatch<T> B) {
  const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int na = B.d.a_ntiles, nt = B.d.t_ntiles;
  for (int i = t0; i < B.nlp; i += stride) {
    B.q_lps[i] = i;
    B.q_pre[i] = B.a_tile_beg[i];
    B.q_pre[B.nlp + 1 + i] = B.t_tile_beg[i];
  }
  for (int i = t0; i < na; i += stride) B.q_a[i] = i;
  for (int i = t0; i < nt; i += stride) B.q_t[i] = i;
  if (t0 == 0) {
    B.q_pre[B.nlp] = na;
    B.q_pre[2 * B.nlp + 1] = nt;
    B.q_cnt[0] = B.nlp;
    B.q_cnt[1] = na;
    B.q_cnt[2] = nt;
    for (int c = 0; c < 4; ++c) B.q_ctr[c] = 0u;
  }
}

// ----------------------------------------------------------------- launchers ---
static int g_sms = 0;
int device_sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

static int ew_grid(long long count) {
  long long g = (count + kThreads - 1) / kThreads;
  const long long cap = 4LL * device_sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return int(g);
}

cudaError_t launch_scale_vectors(const DevVecs& v, cudaStream_t st) {
  k_scale_vectors<<<ew_grid(v.m > v.n ? v.m : v.n), kThreads, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_objective_update(const DevObjective& o, double t_scale, double one_minus_aK,
                                    cudaStream_t st) {
  k_objective_cols<<<o.red_blocks, kThreads, 0, st>>>(o, t_scale, one_minus_aK);
  return cudaGetLastError();
}

cudaError_t launch_objective_norms(const DevObjective& o, double offset, cudaStream_t st) {
  k_cnorm_cols<<<o.red_blocks, kThreads, 0, st>>>(o, offset);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_init(const DevLP<T>& d, double tol, long long iter_limit, int stall_checks,
                              long long max_chunks, cudaStream_t st) {
  k_solve_init<<<1, 1, 0, st>>>(d.ctl, tol, iter_limit, stall_checks, max_chunks);
  return cudaGetLastError();
}

// launch of a per-attempt kernel, with the programmatic-serialization attribute when
// d.pdl is set (the kernel then overlaps its launch with its predecessor's tail)
template <typename T>
static cudaError_t launch_step_kernel(void (*kernel)(DevLP<T>), int grid, const DevLP<T>& d, cudaStream_t st,
                                      int smem = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = size_t(smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = d.pdl ? attr : nullptr;
  cfg.numAttrs = d.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, d);
}

template <typename T>
cudaError_t launch_check(const DevLP<T>& d, cudaStream_t st) {
  cudaError_t e = launch_step_kernel<T>(d.q64 ? k_check_cols<T, 1> : k_check_cols<T, 0>, d.grid_c1, d, st);
  // infeasibility detection: the ray's terms, before the row half takes the decision
  if (e == cudaSuccess && d.inf_cand) e = launch_infeas<T>(d, st);
  if (e == cudaSuccess) e = launch_step_kernel<T>(k_check_rows<T>, d.grid_c2, d, st);
  return e;
}

template <typename T>
cudaError_t launch_primal(const DevLP<T>& d, cudaStream_t st) {
  switch (d.form_p) {
    case kFormStaged: return launch_step_kernel<T>(k_primal_st<T>, d.grid_p, d, st, Staged<T>::kBlockBytes);
    case kFormAsync:
      if constexpr (std::is_same<T, float>::value) return launch_step_kernel<float>(k_primal_as, d.grid_p, d, st);
      return cudaErrorInvalidValue;
    case kFormPrefetch: return launch_step_kernel<T>(k_primal<T, kFormPrefetch>, d.grid_p, d, st);
    case kFormWide: return launch_step_kernel<T>(k_primal<T, kFormWide>, d.grid_p, d, st);
    default: return launch_step_kernel<T>(k_primal<T, kFormPlain>, d.grid_p, d, st);
  }
}
template <typename T>
cudaError_t launch_dual(const DevLP<T>& d, cudaStream_t st) {
  switch (d.form_d) {
    case kFormStaged: return launch_step_kernel<T>(k_dual_st<T>, d.grid_d, d, st, Staged<T>::kBlockBytes);
    case kFormAsync:
      if constexpr (std::is_same<T, float>::value) return launch_step_kernel<float>(k_dual_as, d.grid_d, d, st);
      return cudaErrorInvalidValue;
    case kFormPrefetch: return launch_step_kernel<T>(k_dual<T, kFormPrefetch>, d.grid_d, d, st);
    case kFormWide: return launch_step_kernel<T>(k_dual<T, kFormWide>, d.grid_d, d, st);
    default: return launch_step_kernel<T>(k_dual<T, kFormPlain>, d.grid_d, d, st);
  }
}

template <typename T>
cudaError_t launch_slot(const DevLP<T>& d, cudaStream_t st) {
  cudaError_t e = launch_primal<T>(d, st);
  if (e == cudaSuccess) e = launch_dual<T>(d, st);
  return e;
}
template <typename T>
cudaError_t launch_check_cols(const DevLP<T>& d, cudaStream_t st) {
  return launch_step_kernel<T>(d.q64 ? k_check_cols<T, 1> : k_check_cols<T, 0>, d.grid_c1, d, st);
}
template <typename T>
cudaError_t launch_check_rows(const DevLP<T>& d, cudaStream_t st) {
  return launch_step_kernel<T>(k_check_rows<T>, d.grid_c2, d, st);
}

cudaError_t launch_loop_ctl(Control* ctl, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_loop_ctl<<<1, 1, 0, st>>>(ctl, h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_get_x(const DevLP<T>& d, double* out, int count, cudaStream_t st) {
  k_get_x<T><<<ew_grid(count), kThreads, 0, st>>>(d, out, count);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_get_y(const DevLP<T>& d, double* out, int count, cudaStream_t st) {
  k_get_y<T><<<ew_grid(count), kThreads, 0, st>>>(d, out, count);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_set_xy(const DevLP<T>& d, const double* x, const double* y, cudaStream_t st) {
  k_set_xy<T><<<ew_grid(d.m > d.n ? d.m : d.n), kThreads, 0, st>>>(d, x, y);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_init_point(const DevLP<T>& d, cudaStream_t st) {
  k_init_point<T><<<ew_grid(d.m > d.n ? d.m : d.n), kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

constexpr size_t kPersistentSmem = sizeof(double) * 2 * kPWarps * kSmemPerWarp;

template <typename T>
int persistent_blocks_per_sm() {
  if (cudaFuncSetAttribute(k_solve_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(kPersistentSmem)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_persistent<T>, kPThreads, kPersistentSmem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

template <typename T>
cudaError_t launch_persistent(const DevLP<T>& d, void* grid_bar, int grid, double wait_limit_s, cudaStream_t st) {
  GridBar* bar = static_cast<GridBar*>(grid_bar);
  unsigned long long limit_ns = (unsigned long long)(wait_limit_s * 1e9);
  DevLP<T> dd = d;
  void* args[] = {&dd, &bar, &limit_ns};
  return cudaLaunchCooperativeKernel((const void*)k_solve_persistent<T>, dim3(grid), dim3(kPThreads), args,
                                     kPersistentSmem, st);
}

// grid of a per-attempt kernel (side 0: primal, 1: dual) of form `form`, or of a
// check kernel (side 2: columns, 3: rows): resident blocks per SM times the SMs,
// at most one warp per tile
template <typename T>
int occupancy_grid(int side, int form, int work_tiles) {
  int per_sm = 1;
  int smem = 0;
  void (*k)(DevLP<T>) = nullptr;
  if (side == 2) k = k_check_cols<T, 0>;
  else if (side == 3) k = k_check_rows<T>;
  else if (form == kFormStaged) {
    k = side == 0 ? k_primal_st<T> : k_dual_st<T>;
    smem = Staged<T>::kBlockBytes;
  } else if (form == kFormAsync) {
    if constexpr (std::is_same<T, float>::value) k = side == 0 ? k_primal_as : k_dual_as;
    else k = side == 0 ? k_primal<T, kFormPlain> : k_dual<T, kFormPlain>;
  } else if (form == kFormWide) k = side == 0 ? k_primal<T, kFormWide> : k_dual<T, kFormWide>;
  else if (form == kFormPrefetch) k = side == 0 ? k_primal<T, kFormPrefetch> : k_dual<T, kFormPrefetch>;
  else k = side == 0 ? k_primal<T, kFormPlain> : k_dual<T, kFormPlain>;
  cudaError_t e = cudaSuccess;
  if (smem > 0) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  // a whole wave of resident blocks (every SM the same number, and with warp_tiles
  // the same share of the tiles), or one block per tile on small problems
  long long need = work_tiles;
  if (need < 1) need = 1;
  const long long cap = (long long)per_sm * device_sm_count();
  return int(need < cap ? need : cap);
}

#define SCYLLA_INSTANTIATE(T)                                                                              \
  template cudaError_t launch_solve_init<T>(const DevLP<T>&, double, long long, int, long long, cudaStream_t); \
  template cudaError_t launch_check<T>(const DevLP<T>&, cudaStream_t);                                    \
  template cudaError_t launch_slot<T>(const DevLP<T>&, cudaStream_t);                                     \
  template cudaError_t launch_primal<T>(const DevLP<T>&, cudaStream_t);                                   \
  template cudaError_t launch_dual<T>(const DevLP<T>&, cudaStream_t);                                     \
  template cudaError_t launch_check_cols<T>(const DevLP<T>&, cudaStream_t);                               \
  template cudaError_t launch_check_rows<T>(const DevLP<T>&, cudaStream_t);                               \
  template cudaError_t launch_get_x<T>(const DevLP<T>&, double*, int, cudaStream_t);                      \
  template cudaError_t launch_get_y<T>(const DevLP<T>&, double*, int, cudaStream_t);                      \
  template cudaError_t launch_set_xy<T>(const DevLP<T>&, const double*, const double*, cudaStream_t);     \
  template cudaError_t launch_init_point<T>(const DevLP<T>&, cudaStream_t);                               \
  template int occupancy_grid<T>(int, int, int);                                                           \
  template int persistent_blocks_per_sm<T>();                                                             \
  template cudaError_t launch_persistent<T>(const DevLP<T>&, void*, int, double, cudaStream_t);

SCYLLA_INSTANTIATE(double)
SCYLLA_INSTANTIATE(float)

// ----------------------------------------------------------- batched launchers ---
template <typename T>
cudaError_t launch_batch_init(const DevBatch<T>& B, double tol, long long iter_limit, int stall_checks,
                              cudaStream_t st) {
  k_binit<T><<<(B.nlp + 127) / 128, 128, 0, st>>>(B, tol, iter_limit, stall_checks);
  return cudaGetLastError();
}
static void batch_attempt_kernels(const DevBatch<float>& B, cudaStream_t st, int part) {
  if (part != 1) {
    if (B.async_p) k_bprimal_as<<<B.grid_pa, kThreads, 0, st>>>(B);
    else k_bprimal<float><<<B.grid_p, kThreads, 0, st>>>(B);
  }
  if (part != 0) {
    if (B.async_d) k_bdual_as<<<B.grid_da, kThreads, 0, st>>>(B);
    else k_bdual<float><<<B.grid_d, kThreads, 0, st>>>(B);
  }
}
static void batch_attempt_kernels(const DevBatch<double>& B, cudaStream_t st, int part) {
  if (part != 1) k_bprimal<double><<<B.grid_p, kThreads, 0, st>>>(B);
  if (part != 0) k_bdual<double><<<B.grid_d, kThreads, 0, st>>>(B);
}
template <typename T>
cudaError_t launch_batch_slot(const DevBatch<T>& B, cudaStream_t st) {
  batch_attempt_kernels(B, st, -1);
  k_bstep_control<T><<<B.grid_ctl, kThreads, 0, st>>>(B);
  return cudaGetLastError();
}
// one kernel of an attempt on its own (measurement): 0 primal, 1 dual, 2 step control
template <typename T>
cudaError_t launch_batch_part(const DevBatch<T>& B, int part, cudaStream_t st) {
  if (part == 0 || part == 1) batch_attempt_kernels(B, st, part);
  else k_bstep_control<T><<<B.grid_ctl, kThreads, 0, st>>>(B);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_check(const DevBatch<T>& B, cudaStream_t st) {
  k_bcheck_cols<T><<<B.grid_c1, kThreads, 0, st>>>(B);
  k_bcheck_rows<T><<<B.grid_c2, kThreads, 0, st>>>(B);
  k_bcheck_control<T><<<B.grid_ctl, kThreads, 0, st>>>(B);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_batch_get_x(const DevBatch<T>& B, int b, int col0, int count, double* out, cudaStream_t st) {
  k_bget_x<T><<<ew_grid(count), kThreads, 0, st>>>(B, b, col0, count, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_batch_init_point(const DevBatch<T>& B, cudaStream_t st) {
  k_binit_point<T><<<ew_grid(B.d.m > B.d.n ? B.d.m : B.d.n), kThreads, 0, st>>>(B);
  return cudaGetLastError();
}
template <typename T>
int batch_persistent_blocks_per_sm() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_battempts_persistent<T>, kThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

template <typename T>
cudaError_t launch_batch_queue_reset(const DevBatch<T>& B, cudaStream_t st) {
  const int items = B.d.a_ntiles > B.d.t_ntiles ? B.d.a_ntiles : B.d.t_ntiles;
  k_bqueue_reset<T><<<ew_grid(items > B.nlp ? items : B.nlp), kThreads, 0, st>>>(B);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_persistent(const DevBatch<T>& B, void* grid_bar, long long iter_limit, double wait_limit_s,
                                    cudaStream_t st) {
  if (B.grid_q < 1) return cudaErrorInvalidConfiguration;
  GridBar* bar = static_cast<GridBar*>(grid_bar);
  unsigned long long limit_ns = (unsigned long long)(wait_limit_s * 1e9);
  DevBatch<T> bb = B;
  void* args[] = {&bb, &bar, &iter_limit, &limit_ns};
  return cudaLaunchCooperativeKernel((const void*)k_battempts_persistent<T>, dim3(B.grid_q), dim3(kThreads), args, 0,
                                     st);
}

template <typename T>
cudaError_t launch_batch_compact(const DevBatch<T>& B, cudaStream_t st) {
  k_bcompact<T><<<1, kThreads, 0, st>>>(B);
  k_bfill_tiles<T><<<ew_grid(32LL * B.nlp), kThreads, 0, st>>>(B);
  return cudaGetLastError();
}

template <typename T>
void batch_grids(DevBatch<T>& B) {
  auto grid = [](const void* k, int tiles, size_t smem) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    long long need = tiles;  // a whole wave, or one block per tile (as occupancy_grid)
    if (need < 1) need = 1;
    const long long cap = (long long)per_sm * device_sm_count();
    return int(need < cap ? need : cap);
  };
  B.grid_p = grid((const void*)k_bprimal<T>, B.d.t_ntiles, 0);
  B.grid_d = grid((const void*)k_bdual<T>, B.d.a_ntiles, 0);
  if constexpr (std::is_same<T, float>::value) {
    B.grid_pa = grid((const void*)k_bprimal_as, B.d.t_ntiles, 0);
    B.grid_da = grid((const void*)k_bdual_as, B.d.a_ntiles, 0);
  } else {
    B.grid_pa = B.grid_p;
    B.grid_da = B.grid_d;
  }
  B.grid_c1 = grid((const void*)k_bcheck_cols<T>, B.d.t_ntiles, 0);
  B.grid_c2 = grid((const void*)k_bcheck_rows<T>, B.d.a_ntiles, 0);
  B.grid_ctl = (B.nlp * 32 + kThreads - 1) / kThreads;
  if (B.grid_ctl < 1) B.grid_ctl = 1;
}

#define SCYLLA_INSTANTIATE_BATCH(T)                                                                   \
  template cudaError_t launch_batch_init<T>(const DevBatch<T>&, double, long long, int, cudaStream_t); \
  template cudaError_t launch_batch_slot<T>(const DevBatch<T>&, cudaStream_t);                         \
  template cudaError_t launch_batch_check<T>(const DevBatch<T>&, cudaStream_t);                        \
  template cudaError_t launch_batch_part<T>(const DevBatch<T>&, int, cudaStream_t);                    \
  template cudaError_t launch_batch_get_x<T>(const DevBatch<T>&, int, int, int, double*, cudaStream_t); \
  template cudaError_t launch_batch_init_point<T>(const DevBatch<T>&, cudaStream_t);                   \
  template void batch_grids<T>(DevBatch<T>&);                                                            \
  template int batch_persistent_blocks_per_sm<T>();                                                       \
  template cudaError_t launch_batch_queue_reset<T>(const DevBatch<T>&, cudaStream_t);                     \
  template cudaError_t launch_batch_persistent<T>(const DevBatch<T>&, void*, long long, double, cudaStream_t); \
  template cudaError_t launch_batch_compact<T>(const DevBatch<T>&, cudaStream_t);

SCYLLA_INSTANTIATE_BATCH(double)
SCYLLA_INSTANTIATE_BATCH(float)

}  // namespace scylla
