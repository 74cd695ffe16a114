// K pump objectives of one LP solved together (the feasibility-pump fan-out):
// K independent PDHG runs (Algorithm 1 inner loop) that share A, A^T and the
// bounds and differ only in the objective, done as sparse-times-tall-skinny
// products so A is read once per K objectives.
//
// Layout: every K-wide vector is row-major with 64 slots per row (row j holds the
// values of objectives 0..63 contiguously, 256 bytes in FP32), so a nonzero a_ij
// gathers one contiguous K-wide row.  The objective of column k is generated on the
// fly from the base c and two bit planes (target at the lower / upper bound) instead
// of being stored K times: c_hat_jk = alpha^K s c_j + (1 - alpha^K) g_jk
// (Section 2.4).
//
// Pool roles are shared by every objective: X[cur], Y[cur], AX[cur] hold the
// current points, [1 - cur] the next ones, [2] the running averages, ATY[0] and
// ATY[1] the check's A^T y of the current and averaged points.  Every attempt
// writes the next point of every slot and swaps cur.  An objective whose attempt was
// rejected, or that restarts to (or finishes with) its average, has its slices
// copied back into the current pool by k_fcopy before the next attempt (a few
// scattered 4-byte columns); a finished objective is carried along unchanged
// by zero step sizes.  So the SpMMs treat all 64 slots of a row alike and move them
// with vector loads: a lane holds VEC consecutive objectives, CHUNK / VEC lanes
// cover a row's CHUNK slots, and a warp works on 32 VEC / CHUNK rows at once
// (64 / CHUNK sweeps over the matrix).  (VEC, CHUNK) is the tile shape the
// create-time autotuner picks per SpMM.
//
// Every objective has its own control block (step size, primal weight, restarts,
// termination); sums are per block and per objective, reduced per objective by one
// warp in the control kernels, which apply the same logic as the single-LP path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace scylla {

constexpr int kFK = 64;  // slots of a K-wide row
constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;

__device__ __forceinline__ double fwarp_sum(double v) { return warp_sum(v); }

// sum over the row's nonzeros of a_rp * src[col][k] for the lane's two objectives;
// the (index, value) pairs are loaded 32 at a time and broadcast by shuffles, four
// nonzeros per step so eight gathers per lane are in flight.  Lanes past the row end
// carry (column 0, value 0), which adds exactly zero, so the four-wide steps need
// no bounds test and the summation order stays the CSR order.
template <typename Acc, typename V, typename Src>
__device__ __forceinline__ void row_gather(int p0, int p1, const int* __restrict__ cols, const V* __restrict__ vals,
                                           Src src, Acc (&s)[2]) {
  const int lane = threadIdx.x & 31;
  s[0] = Acc(0);
  s[1] = Acc(0);
  for (int b = p0; b < p1; b += 32) {
    const int p = b + lane;
    int cl = 0;
    V vl = V(0);
    if (p < p1) {
      cl = __ldg(cols + p);
      vl = __ldg(vals + p);
    }
    const int cnt = p1 - b < 32 ? p1 - b : 32;
    for (int e = 0; e < cnt; e += 4) {
      int c[4];
      Acc a[4];
      Acc g[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __shfl_sync(0xffffffffu, cl, e + u);
        a[u] = Acc(__shfl_sync(0xffffffffu, vl, e + u));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) src(c[u], g[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s[0] = fma_t<Acc>(a[u], g[u][0], s[0]);
        s[1] = fma_t<Acc>(a[u], g[u][1], s[1]);
      }
    }
  }
}

// The FP32-mixed checks' form of row_gather: the same sums over the row in CSR order,
// each an FP32 pair (s, c) with s + c the value, so that they take the FP32 pipe and
// not the FP64 one (64 times slower on this part, and the bound of these kernels).
// The FP64 entry a is split once per warp step into a_hi = fl32(a) and
// a_lo = fl32(a - a_hi); per term, a_hi g is formed exactly as p + e (an FMA gives the
// product's rounding error), a_lo g is added to e, and p joins s by Knuth's two-sum,
// whose rounding error joins c with e.  The pair holds the FP64 sum to about 2^-44 of
// the sum of the terms' magnitudes (the FP64 form: 2^-53).  Every operation is an
// explicitly rounded intrinsic, so no multiply is contracted into a following add.
template <typename Src>
__device__ __forceinline__ void row_gather_pair(int p0, int p1, const int* __restrict__ cols,
                                                const double* __restrict__ vals, Src src, float (&s)[2],
                                                float (&c)[2]) {
  const int lane = threadIdx.x & 31;
  s[0] = s[1] = c[0] = c[1] = 0.0f;
  for (int b = p0; b < p1; b += 32) {
    const int p = b + lane;
    int cl = 0;
    float hl = 0.0f, ll = 0.0f;
    if (p < p1) {
      cl = __ldg(cols + p);
      const double a = __ldg(vals + p);
      hl = __double2float_rn(a);
      ll = __double2float_rn(a - to_f64(hl));
    }
    const int cnt = p1 - b < 32 ? p1 - b : 32;
    for (int e = 0; e < cnt; e += 4) {
      int ci[4];
      float ah[4], al[4], g[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ci[u] = __shfl_sync(0xffffffffu, cl, e + u);
        ah[u] = __shfl_sync(0xffffffffu, hl, e + u);
        al[u] = __shfl_sync(0xffffffffu, ll, e + u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) src(ci[u], g[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          // lanes past the row end carry (column 0, 0, 0): every term is an exact zero
          const float pr = __fmul_rn(ah[u], g[u][q]);
          float er = __fmaf_rn(ah[u], g[u][q], -pr);
          er = __fmaf_rn(al[u], g[u][q], er);
          const float t = __fadd_rn(s[q], pr);
          const float z = __fsub_rn(t, s[q]);
          const float ts = __fadd_rn(__fsub_rn(s[q], __fsub_rn(t, z)), __fsub_rn(pr, z));
          c[q] = __fadd_rn(c[q], __fadd_rn(ts, er));
          s[q] = t;
        }
    }
  }
}

// A check's products of one row for the lane's two objectives: out in FP64 for the
// check's sums, ref in the iterates' precision for the refresh of the cached products
// (FP64: the FP64 sums; FP32-mixed: the FP32 pairs of row_gather_pair, ref their
// rounded value).  src(col, g) gives the two gathered entries in T.
template <typename T, typename Src>
__device__ __forceinline__ void check_gather(int p0, int p1, const int* __restrict__ cols,
                                             const double* __restrict__ vals, Src src, double (&out)[2],
                                             T (&ref)[2]) {
  if constexpr (sizeof(T) == 4) {
    float s[2], c[2];
    row_gather_pair(p0, p1, cols, vals, src, s, c);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      out[q] = to_f64(s[q]) + to_f64(c[q]);
      ref[q] = __fadd_rn(s[q], c[q]);
    }
  } else {
    row_gather<double, double>(p0, p1, cols, vals, src, out);
#pragma unroll
    for (int q = 0; q < 2; ++q) ref[q] = out[q];
  }
}

template <typename T>
__device__ __forceinline__ void store_block_sums(const typename AccOf<T>::type* acc /*[2][N]*/, int N, double* part,
                                                 double* sh /*[kFWarps][N*kFK]*/) {
  // per objective and sum: warp partials to shared memory, then block sums
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < 2; ++q)
    for (int s = 0; s < N; ++s) sh[(w * N + s) * kFK + lane + 32 * q] = double(acc[q * N + s]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * kFK; idx += blockDim.x) {
    double t = 0.0;
    for (int v = 0; v < kFWarps; ++v) t += sh[v * N * kFK + idx];
    part[blockIdx.x * N * kFK + idx] = t;  // [block][sum][objective]
  }
}

// pool of the current points (the next points are in the other of pools 0 and 1)
template <typename T>
__device__ __forceinline__ int fan_cur(const DevFan<T>& F) {
  return int(F.state->att & 1ULL);
}

// ---------------------------------------------------------------- vectors ---
template <typename T, int N>
struct FVec;
template <>
struct FVec<float, 4> {
  typedef float4 V;
};
template <>
struct FVec<float, 2> {
  typedef float2 V;
};
template <>
struct FVec<double, 2> {
  typedef double2 V;
};

template <typename T, int N>
union VecU {
  typename FVec<T, N>::V v;
  T e[N];
};

template <typename T, int N>
__device__ __forceinline__ void vld_nc(const T* p, T (&o)[N]) {
  VecU<T, N> u;
  u.v = __ldg(reinterpret_cast<const typename FVec<T, N>::V*>(p));
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = u.e[i];
}
// streaming accesses (read or written once per attempt and not gathered by the next
// kernel): evict-first in L2, so the vector the next kernel gathers (x' written by
// the primal, y' by the dual) and the one this kernel gathers keep their lines
template <typename T, int N>
__device__ __forceinline__ void vld_cs(const T* p, T (&o)[N]) {
  VecU<T, N> u;
  u.v = __ldcs(reinterpret_cast<const typename FVec<T, N>::V*>(p));
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = u.e[i];
}
template <typename T, int N>
__device__ __forceinline__ void vst_cs(T* p, const T (&o)[N]) {
  VecU<T, N> u;
#pragma unroll
  for (int i = 0; i < N; ++i) u.e[i] = o[i];
  __stcs(reinterpret_cast<typename FVec<T, N>::V*>(p), u.v);
}
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T* p, T (&o)[N]) {
  VecU<T, N> u;
  u.v = *reinterpret_cast<const typename FVec<T, N>::V*>(p);
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = u.e[i];
}
template <typename T, int N>
__device__ __forceinline__ void vst(T* p, const T (&o)[N]) {
  VecU<T, N> u;
#pragma unroll
  for (int i = 0; i < N; ++i) u.e[i] = o[i];
  *reinterpret_cast<typename FVec<T, N>::V*>(p) = u.v;
}

// Asynchronous copies of a lane's VEC entries of an epilogue vector into shared
// memory (zero-filled when off), so that the next row group's operands are in flight
// while the warp gathers for the current one, without holding registers (the dual
// SpMM).  Each lane
// reads back only the slots it copied, so a wait on its own copies is all the
// synchronisation needed.  16-byte copies bypass L1.
// The copies carry an evict-first L2 policy (pol, from l2_evict_first()): the
// operands are read once per attempt, and the vector the kernel gathers should keep
// its lines.
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
template <int BYTES>
__device__ __forceinline__ void cp_async_lane(void* dst, const void* src, bool on, unsigned long long pol) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  const int n = on ? BYTES : 0;
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(d), "l"(src), "r"(n),
                 "l"(pol)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3, %4;" ::"r"(d), "l"(src), "n"(BYTES),
                 "r"(n), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// two stages of three epilogue vectors per lane, per warp of a block
template <typename T, int VEC>
struct FanStage {
  typename FVec<T, VEC>::V v[kFWarps][2][3][32];
};
template <typename T, int VEC>
__device__ __forceinline__ void stage_read(const FanStage<T, VEC>& S, int w, int st, int q, int lane, T (&o)[VEC]) {
  VecU<T, VEC> u;
  u.v = S.v[w][st][q][lane];
#pragma unroll
  for (int i = 0; i < VEC; ++i) o[i] = u.e[i];
}

// the tile shapes by number: (objectives per lane, slots per sweep) = 1: (4, 64),
// 2: (2, 64), 3: (4, 32), 4: (2, 32)
__host__ __device__ constexpr int fan_shape_vec(int s) { return (s == 1 || s == 3) ? 4 : 2; }
__host__ __device__ constexpr int fan_shape_chunk(int s) { return (s == 3 || s == 4) ? 32 : 64; }

// ---------------------------------------------------------- per-objective ---
// The per-objective values of one attempt, copied to shared memory by every block
// (structure of arrays, so a lane reads its VEC objectives from consecutive words).
template <typename T>
struct FanShared {
  T tau[kFK], sigma[kFK], w[kFK], w1[kFK];
  int flags[kFK];
};

template <typename T>
__device__ __forceinline__ void load_fan_shared(const DevFan<T>& F, FanShared<T>& S) {
  for (int k = threadIdx.x; k < kFK; k += blockDim.x) {
    FanSlot<T> s;
    if (k < F.K) {
      s = F.slot[k];
    } else {  // unused slots are carried like finished objectives
      s.tau = s.sigma = s.w = T(0);
      s.w1 = T(1);
      s.flags = 0;
    }
    S.tau[k] = s.tau;
    S.sigma[k] = s.sigma;
    S.w[k] = s.w;
    S.w1[k] = s.w1;
    S.flags[k] = s.flags;
  }
  __syncthreads();
}

// c_hat_jk in the scaled space, C_j (t c_j + om g_jk), g_jk in {-1, 0, 1}: the
// column's three possible values are formed once per column and selected per
// objective.  FP32 from the per-column pair (t c_j C_j, om C_j) prepared at create;
// FP64 as (t c_j + om g) C_j, the same rounding for each g as written out.
template <typename T>
struct FanCostCol {
  T c0, cp, cm;  // g = 0, +1, -1
  __device__ __forceinline__ T at(int gi) const { return gi > 0 ? cp : (gi < 0 ? cm : c0); }
};
template <typename T>
__device__ __forceinline__ FanCostCol<T> fan_cost_col(const DevFan<T>& F, int j);
template <>
__device__ __forceinline__ FanCostCol<float> fan_cost_col<float>(const DevFan<float>& F, int j) {
  const float2 w = __ldg(F.cw + j);
  return FanCostCol<float>{w.x, w.x + w.y, w.x - w.y};
}
// FP64 (the FP64 SpMMs, and the checks' triples of every precision): every
// operation explicitly rounded, so that no multiply is contracted into the following
// add (a contraction the compiler may take in one kernel or tile shape and not in
// another)
__device__ __forceinline__ FanCostCol<double> fan_cost_col64(double t, double om, double c, double Cj) {
  const double tc = __dmul_rn(t, c);
  return FanCostCol<double>{__dmul_rn(tc, Cj), __dmul_rn(__dadd_rn(tc, om), Cj), __dmul_rn(__dsub_rn(tc, om), Cj)};
}
template <>
__device__ __forceinline__ FanCostCol<double> fan_cost_col<double>(const DevFan<double>& F, int j) {
  return fan_cost_col64(F.t, F.om, __ldg(F.c_orig + j), __ldg(F.d.C + j));
}

// ------------------------------------------------------------ SpMM sweeps ---
// Geometry of a tile shape: LPR lanes per row, RPW rows per warp, NSW sweeps.
template <int VEC, int CHUNK>
struct FanGeo {
  static constexpr int LPR = CHUNK / VEC;
  static constexpr int RPW = 32 / LPR;
  static constexpr int NSW = kFK / CHUNK;
  static constexpr int NOBJ = NSW * VEC;  // objectives per lane over all sweeps
};

// One row's sum s[v] = sum_p a_p src(col_p)[v] in CSR order for the lane's VEC
// objectives.  The segment's lanes hold the row's (index, value) pairs LPR at a time
// (the first LPR loaded ahead in cl, vl) and broadcast them by shuffles within the
// segment, 16 / VEC nonzeros per step so that many vector gathers per lane are in flight.
// The warp loops to the longest of its rows; a segment past its row's end issues no
// load and adds nothing.
template <typename T, int VEC, int LPR, typename Src>
__device__ __forceinline__ void fan_vgather(int p0, int p1, int cl, T vl, const int* __restrict__ cols,
                                            const T* __restrict__ vals, Src src, T (&s)[VEC]) {
  const int sl = threadIdx.x & (LPR - 1);
  // nonzeros per step: 16 entries of the gathered vector per lane in flight
  constexpr int U = 16 / VEC;
#pragma unroll
  for (int v = 0; v < VEC; ++v) s[v] = T(0);
  const int cnt = p1 - p0;
  int maxcnt = cnt;
#pragma unroll
  for (int o = LPR; o < 32; o <<= 1) maxcnt = max(maxcnt, __shfl_xor_sync(0xffffffffu, maxcnt, o));
  for (int b = 0; b < maxcnt; b += LPR) {
    if (b != 0) {
      cl = 0;
      vl = T(0);
      if (b + sl < cnt) {
        cl = __ldg(cols + p0 + b + sl);
        vl = __ldg(vals + p0 + b + sl);
      }
    }
    const int lim = min(LPR, maxcnt - b);
    for (int e = 0; e < lim; e += U) {
      int c[U];
      T a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        c[u] = __shfl_sync(0xffffffffu, cl, (e + u) & (LPR - 1), LPR);
        a[u] = __shfl_sync(0xffffffffu, vl, (e + u) & (LPR - 1), LPR);
      }
      T g[U][VEC];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (b + e + u < cnt) {
          src(c[u], g[u]);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) g[u][v] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (b + e + u < cnt)
#pragma unroll
          for (int v = 0; v < VEC; ++v) s[v] = fma_t<T>(a[u], g[u][v], s[v]);
    }
  }
}

// per-block sums of the per-lane accumulators acc[t][o] (sum t; the lane's o-th
// objective is slot (o / VEC) CHUNK + sl VEC + o % VEC) into
// part[t][objective][block]; the segments of a warp hold the same objectives
template <typename A, int VEC, int CHUNK, int NSUM>
__device__ __forceinline__ void fan_block_sums(A (&acc)[NSUM][FanGeo<VEC, CHUNK>::NOBJ], double* part,
                                               double* sh /*[kFWarps][NSUM][kFK]*/) {
  typedef FanGeo<VEC, CHUNK> G;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, sl = lane & (G::LPR - 1);
#pragma unroll
  for (int t = 0; t < NSUM; ++t)
#pragma unroll
    for (int o = 0; o < G::NOBJ; ++o) {
      A v = acc[t][o];
#pragma unroll
      for (int off = G::LPR; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      acc[t][o] = v;
    }
  if (lane < G::LPR)
#pragma unroll
    for (int t = 0; t < NSUM; ++t)
#pragma unroll
      for (int o = 0; o < G::NOBJ; ++o)
        sh[(w * NSUM + t) * kFK + (o / VEC) * CHUNK + sl * VEC + (o % VEC)] = double(acc[t][o]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < NSUM * kFK; idx += blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < kFWarps; ++v) s += sh[v * NSUM * kFK + idx];
    part[idx * int(gridDim.x) + int(blockIdx.x)] = s;  // [sum][objective][block]
  }
}

// Primal SpMM of one attempt for every objective (Algorithm 1, primal step):
// x'_jk = proj_[l_j,u_j](x_jk + tau_k ((A^T Y)_jk - c_hat_jk)), the running average
// and ||x' - x||^2 per objective.  Row groups are dealt gw, gw + nw, ...; while a
// warp works on one group it has the row pointers of the group after the next and
// the first (index, value) pairs of the next group in flight, and it loads the
// group's epilogue operands before its gathers.
template <typename T, int VEC, int CHUNK>
__global__ void __launch_bounds__(kFThreads, sizeof(T) == 4 ? 4 : 3) k_fprimal(DevFan<T> F) {
  typedef typename AccOf<T>::type A;
  typedef FanGeo<VEC, CHUNK> G;
  __shared__ double sh[kFWarps * 1 * kFK];
  __shared__ __align__(16) FanShared<T> S;
  load_fan_shared(F, S);
  const DevLP<T>& d = F.d;
  const int lane = threadIdx.x & 31, seg = lane / G::LPR, sl = lane & (G::LPR - 1);
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = d.n, cur = fan_cur(F);
  const T* __restrict__ Xc = F.X[cur];
  T* __restrict__ Xn = F.X[1 - cur];
  T* __restrict__ Xa = F.X[2];
  const T* __restrict__ Yc = F.Y[cur];
  const T* __restrict__ At = F.ATY[0];
  A acc[1][G::NOBJ];
#pragma unroll
  for (int o = 0; o < G::NOBJ; ++o) acc[0][o] = A(0);
  const int ngroups = (n + G::RPW - 1) / G::RPW;
#pragma unroll
  for (int sw = 0; sw < G::NSW; ++sw) {
    const int k0 = sw * CHUNK + sl * VEC;  // the lane's first objective in this sweep
    bool cached = false, avg = false, lr = false;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int f = S.flags[k0 + v];
      cached |= (f & kSlotCached) != 0;
      avg |= (f & kSlotAvg) != 0;
      lr |= (f & kSlotCopyLr) != 0;
    }
    const T* ysrc = Yc + k0;
    auto src = [&](int i, T(&g)[VEC]) { vld_nc<T, VEC>(ysrc + size_t(i) * kFK, g); };
    auto rowp = [&](int gidx, int& a, int& b) {
      const int j = gidx * G::RPW + seg;
      a = b = 0;
      if (gidx < ngroups && j < n) {
        a = __ldg(d.t_rowptr + j);
        b = __ldg(d.t_rowptr + j + 1);
      }
    };
    int g = gw;
    int p0, p1, pn0, pn1, cl = 0;
    T vl = T(0);
    rowp(g, p0, p1);
    if (p0 + sl < p1) {
      cl = __ldg(d.t_cols + p0 + sl);
      vl = __ldg(d.t_vals + p0 + sl);
    }
    rowp(g + nw, pn0, pn1);
    while (g < ngroups) {
      int pnn0, pnn1, cln = 0;
      T vln = T(0);
      rowp(g + 2 * nw, pnn0, pnn1);
      if (pn0 + sl < pn1) {
        cln = __ldg(d.t_cols + pn0 + sl);
        vln = __ldg(d.t_vals + pn0 + sl);
      }
      const int j = g * G::RPW + seg;
      const bool live = j < n;
      const size_t o = size_t(live ? j : 0) * kFK + k0;
      T x[VEC], xa[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) x[v] = xa[v] = T(0);
      if (live) {
        vld_cs<T, VEC>(Xc + o, x);
        if (avg) vld_cs<T, VEC>(Xa + o, xa);
      }
      T s[VEC];
      fan_vgather<T, VEC, G::LPR>(p0, p1, cl, vl, d.t_cols, d.t_vals, src, s);
      if (live) {
        // the per-objective values from shared memory here rather than in registers
        // across the gathers (fewer registers, one more resident block per SM)
        T tau[VEC], w[VEC], w1[VEC], at[VEC];
        int fl[VEC];
        lds_vec<T, VEC>(S.tau + k0, tau);
        lds_vec<T, VEC>(S.w + k0, w);
        lds_vec<T, VEC>(S.w1 + k0, w1);
#pragma unroll
        for (int v = 0; v < VEC; ++v) fl[v] = S.flags[k0 + v];
#pragma unroll
        for (int v = 0; v < VEC; ++v) at[v] = T(0);
        if (cached) vld_cs<T, VEC>(At + o, at);
        const unsigned long long lob = __ldg(F.lo_bits + j) >> k0, upb = __ldg(F.up_bits + j) >> k0;
        const T lj = __ldg(d.l + j), uj = __ldg(d.u + j);
        const FanCostCol<T> cc = fan_cost_col<T>(F, j);
        T xn[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          // A^T y: the gathered sum, or the check's FP64 refresh of it (the checks of
          // Section 2.2 recompute the products; the next attempt starts from them)
          const T a = (fl[v] & kSlotCached) ? at[v] : s[v];
          const T cs = cc.at(int((lob >> v) & 1ULL) - int((upb >> v) & 1ULL));
          // one explicit fused multiply-add, so that every slot of the lane rounds
          // alike; an objective that does not attempt has tau = 0 and keeps its point
          // (the checks keep the average inside [l, u], so the clamp is exact too)
          xn[v] = clampv<T>(fma_t<T>(tau[v], a - cs, x[v]), lj, uj);
          const A dx = A(xn[v]) - A(x[v]);
          acc[0][sw * VEC + v] += dx * dx;
          if (avg) xa[v] = blend(xa[v], x[v], w1[v], w[v]);
        }
        vst<T, VEC>(Xn + o, xn);
        if (avg) vst_cs<T, VEC>(Xa + o, xa);
        if (lr)
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            if (fl[v] & kSlotCopyLr) __stcs(F.XLR + o + v, x[v]);
      }
      g += nw;
      p0 = pn0;
      p1 = pn1;
      pn0 = pnn0;
      pn1 = pnn1;
      cl = cln;
      vl = vln;
    }
  }
  fan_block_sums<A, VEC, CHUNK, 1>(acc, F.part_p, sh);
}

// Dual SpMM of one attempt for every objective (Algorithm 1, dual step with the
// extrapolation A(2x' - x) = 2 A x' - A x from the cached A x): y', A x', the
// running average, ||y' - y||^2 and (y' - y).(A x' - A x) per objective, with the
// primal SpMM's look-ahead of row pointers and (index, value) pairs; the next row
// group's epilogue operands (A x, y, the average) are staged in shared memory by
// asynchronous copies while the warp gathers for the current group (measured: the
// dual 5% faster; the same staging made the primal slower, so it loads directly).
template <typename T, int VEC, int CHUNK>
__global__ void __launch_bounds__(kFThreads, sizeof(T) == 4 && !(VEC == 4 && CHUNK == 32) ? 4 : 3) k_fdual(DevFan<T> F) {
  typedef typename AccOf<T>::type A;
  typedef FanGeo<VEC, CHUNK> G;
  __shared__ double sh[kFWarps * 2 * kFK];
  __shared__ __align__(16) FanShared<T> S;
  __shared__ __align__(16) FanStage<T, VEC> E;
  constexpr int kB = VEC * int(sizeof(T));
  const unsigned long long pol = l2_evict_first();
  load_fan_shared(F, S);
  const DevLP<T>& d = F.d;
  const int lane = threadIdx.x & 31, seg = lane / G::LPR, sl = lane & (G::LPR - 1), wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int m = d.m, cur = fan_cur(F);
  const T* __restrict__ Xn = F.X[1 - cur];
  const T* __restrict__ Yc = F.Y[cur];
  T* __restrict__ Yn = F.Y[1 - cur];
  T* __restrict__ Ya = F.Y[2];
  const T* __restrict__ AXc = F.AX[cur];
  T* __restrict__ AXn = F.AX[1 - cur];
  A acc[2][G::NOBJ];
#pragma unroll
  for (int o = 0; o < G::NOBJ; ++o) acc[0][o] = acc[1][o] = A(0);
  const int ngroups = (m + G::RPW - 1) / G::RPW;
#pragma unroll
  for (int sw = 0; sw < G::NSW; ++sw) {
    const int k0 = sw * CHUNK + sl * VEC;
    bool avg = false, lr = false;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int f = S.flags[k0 + v];
      avg |= (f & kSlotAvg) != 0;
      lr |= (f & kSlotCopyLr) != 0;
    }
    const T* xsrc = Xn + k0;
    auto src = [&](int jc, T(&g)[VEC]) { vld_nc<T, VEC>(xsrc + size_t(jc) * kFK, g); };
    auto rowp = [&](int gidx, int& a, int& b) {
      const int i = gidx * G::RPW + seg;
      a = b = 0;
      if (gidx < ngroups && i < m) {
        a = __ldg(d.a_rowptr + i);
        b = __ldg(d.a_rowptr + i + 1);
      }
    };
    // the epilogue operands (A x, y, the average) of row group gg into stage st
    auto issue = [&](int gg, int st) {
      const int ii = gg * G::RPW + seg;
      const bool lv = gg < ngroups && ii < m;
      const size_t oo = size_t(lv ? ii : 0) * kFK + k0;
      cp_async_lane<kB>(&E.v[wib][st][0][lane], AXc + oo, lv, pol);
      cp_async_lane<kB>(&E.v[wib][st][1][lane], Yc + oo, lv, pol);
      if (avg) cp_async_lane<kB>(&E.v[wib][st][2][lane], Ya + oo, lv, pol);
      cp_async_commit();
    };
    int g = gw, stg = 0;
    int p0, p1, pn0, pn1, cl = 0;
    T vl = T(0);
    rowp(g, p0, p1);
    if (p0 + sl < p1) {
      cl = __ldg(d.a_cols + p0 + sl);
      vl = __ldg(d.a_vals + p0 + sl);
    }
    rowp(g + nw, pn0, pn1);
    issue(g, 0);
    while (g < ngroups) {
      int pnn0, pnn1, cln = 0;
      T vln = T(0);
      rowp(g + 2 * nw, pnn0, pnn1);
      if (pn0 + sl < pn1) {
        cln = __ldg(d.a_cols + pn0 + sl);
        vln = __ldg(d.a_vals + pn0 + sl);
      }
      issue(g + nw, stg ^ 1);
      const int i = g * G::RPW + seg;
      const bool live = i < m;
      const size_t o = size_t(live ? i : 0) * kFK + k0;
      T s[VEC];
      fan_vgather<T, VEC, G::LPR>(p0, p1, cl, vl, d.a_cols, d.a_vals, src, s);
      cp_async_wait<1>();  // this group's operands (the next group's may still be in flight)
      T ax[VEC], y[VEC], ya[VEC];
      stage_read<T, VEC>(E, wib, stg, 0, lane, ax);
      stage_read<T, VEC>(E, wib, stg, 1, lane, y);
      if (avg) stage_read<T, VEC>(E, wib, stg, 2, lane, ya);
      if (live) {
        const T lo = __ldg(d.lo + i), hi = __ldg(d.hi + i);
        T sig[VEC], w[VEC], w1[VEC];
        int fl[VEC];
        lds_vec<T, VEC>(S.sigma + k0, sig);
        lds_vec<T, VEC>(S.w + k0, w);
        lds_vec<T, VEC>(S.w1 + k0, w1);
#pragma unroll
        for (int v = 0; v < VEC; ++v) fl[v] = S.flags[k0 + v];
        T yn[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T axt = T(2) * s[v] - ax[v];
          yn[v] = dual_prox<T>(y[v], sig[v], axt, lo, hi);  // sig = 0 keeps y
          const A dy = A(yn[v]) - A(y[v]);
          acc[0][sw * VEC + v] += dy * dy;
          acc[1][sw * VEC + v] += dy * (A(s[v]) - A(ax[v]));
          if (avg) ya[v] = blend(ya[v], y[v], w1[v], w[v]);
        }
        vst<T, VEC>(Yn + o, yn);
        vst_cs<T, VEC>(AXn + o, s);
        if (avg) vst_cs<T, VEC>(Ya + o, ya);
        if (lr)
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            if (fl[v] & kSlotCopyLr) __stcs(F.YLR + o + v, y[v]);
      }
      g += nw;
      stg ^= 1;
      p0 = pn0;
      p1 = pn1;
      pn0 = pnn0;
      pn1 = pnn1;
      cl = cln;
      vl = vln;
    }
    cp_async_wait<0>();  // the copies issued past the last group land before the stages are reused
  }
  // part_d is [sum][objective][block] with sum 0 = ||dy||^2, 1 = dy.(A x' - A x)
  fan_block_sums<A, VEC, CHUNK, 2>(acc, F.part_d, sh);
}

// ---------------------------------------------------------------- control ---
// slot of one objective for the next attempt: an objective that does not attempt
// (finished, or at its iteration limit until the next check ends it) is carried by
// zero step sizes and no averaging, which leaves x, y and the average unchanged
template <typename T>
__device__ __forceinline__ void write_fan_slot(FanSlot<T>* s, const Control* c) {
  // FP32-mixed: the decision's FP32 copies (set by step_control<float>, or by
  // derive_steps after a check); FP64: from the FP64 fields
  constexpr bool f32 = sizeof(T) == 4;
  const double aw = f32 ? double(c->w_f) : c->avg_w;
  FanSlot<T> v;
  const bool active = !c->done && c->k < c->iter_limit;
  if (active) {
    v.tau = f32 ? T(c->tau_f) : T(c->eta / c->omega);
    v.sigma = f32 ? T(c->sigma_f) : T(c->eta * c->omega);
    v.w = f32 ? T(c->w_f) : T(c->avg_w);
    v.w1 = f32 ? T(c->w1_f) : T(1.0 - c->avg_w);
    int f = kSlotActive | kSlotCheck;
    if (c->copy_lr) f |= kSlotCopyLr;
    if (c->aty_valid) f |= kSlotCached;
    if (aw > 0.0) f |= kSlotAvg;
    v.flags = f;
  } else if (c->done) {
    v.tau = v.sigma = v.w = T(0);
    v.w1 = T(1);
    v.flags = 0;
  } else {
    // at its iteration limit, waiting for the check that ends it: carried by zero
    // step sizes, but the average still takes the last accepted point (the next
    // attempt or the check blends it in; k_fstep_control then clears the weight)
    v.tau = v.sigma = T(0);
    v.w = f32 ? T(c->w_f) : T(c->avg_w);
    v.w1 = f32 ? T(c->w1_f) : T(1.0 - c->avg_w);
    v.flags = kSlotCheck | (aw > 0.0 ? kSlotAvg : 0) | (c->copy_lr ? kSlotCopyLr : 0);
  }
  *s = v;
}

// One warp per objective: block sums in a fixed order, then the step decision;
// rej[k] says whether objective k's attempt was rejected (k_fcopy_rej restores its
// pair).  Block 0 counts the attempt, which swaps the pool roles of every objective.
template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fstep_control(DevFan<T> F) {
  FanState* st = F.state;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ++*F.kglob;
    ++st->att;
  }
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= F.K) return;
  const int flags = F.slot[k].flags;
  if (!(flags & kSlotActive)) {
    if (lane == 0) {
      st->rej[k] = 0;
      if (flags & kSlotCheck) {  // carried: the pending average update is now applied
        Control* c = &F.ctl[k];
        c->avg_w = 0.0;
        c->w_f = 0.0f;
        c->w1_f = 1.0f;
        c->avg_on = 0;
        c->copy_lr = 0;
        write_fan_slot(&F.slot[k], c);
      }
    }
    return;
  }
  const int G = F.grid_p, H = F.grid_d;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  // the partials are [sum][objective][block]: a warp's loads are consecutive
  const double* pp = F.part_p + size_t(k) * G;
  const double* pd0 = F.part_d + size_t(k) * H;
  const double* pd1 = F.part_d + size_t(kFK + k) * H;
  for (int b = lane; b < G; b += 32) s0 += pp[b];
  for (int b = lane; b < H; b += 32) {
    s1 += pd0[b];
    s2 += pd1[b];
  }
  s0 = fwarp_sum(s0);
  s1 = fwarp_sum(s1);
  s2 = fwarp_sum(s2);
  if (lane == 0) {
    Control* c = &F.ctl[k];
    const long long rej0 = c->rejected;
    if constexpr (sizeof(T) == 4) {
      // FP32-mixed: the single-LP path's FP32 decision (no FP64 division on the
      // per-attempt path); the FP64 sums are rounded once
      const StepPre p = step_pre<float>(c, F.d.step_fac, F.d.n_check);
      step_control<float>(c, p, float(s0), float(s1), float(s2), nullptr, 0);
    } else {
      step_control(c, s0, s1, s2, F.d.step_fac, F.d.n_check, nullptr, 0);
    }
    st->rej[k] = c->rejected != rej0 ? 1 : 0;
    if (c->done) atomicAdd(F.n_done, 1);
    write_fan_slot(&F.slot[k], c);
    // the primal SpMM keeps no copy of A^T y: a retry after a rejected attempt (y
    // restored by k_fcopy_rej) gathers it again
    F.slot[k].flags &= ~kSlotCached;
  }
}

// Column half of a check for every objective: A^T y of the current and the averaged
// dual (FP64 sums, or in FP32-mixed the FP32 pairs of check_gather), reduced costs
// against c_hat_k, residuals, objectives, hash, all in FP64.  Lane q of a warp works
// on objectives q and q + 32 of one column.  FP32 entries widen to FP64 by the exact
// bit-level conversion on the integer pipe (an FP32-to-FP64 conversion instruction
// would take the FP64 pipe, the bound of these kernels on this part).
template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fcheck_cols(DevFan<T> F) {
  __shared__ double sh[kFWarps * kNC1 * kFK];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int cur = fan_cur(F);
  bool on[2], hs[2];
  int fl[2];
  T w[2], w1[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = lane + 32 * q;
    fl[q] = k < F.K ? F.slot[k].flags : 0;
    on[q] = (fl[q] & kSlotCheck) != 0;
    w[q] = k < F.K ? F.slot[k].w : T(0);
    w1[q] = k < F.K ? F.slot[k].w1 : T(1);
    // the hash of the rounded point only feeds the stall test
    hs[q] = k < F.K && F.ctl[k].stall_checks > 0;
  }
  double acc[2 * kNC1];
#pragma unroll
  for (int q = 0; q < 2 * kNC1; ++q) acc[q] = 0.0;
  unsigned long long h[2] = {0ULL, 0ULL};
  const T* yc = F.Y[cur];
  const T* ya = F.Y[2];
  T* Xc = F.X[cur];
  T* Xa = F.X[2];
  for (int j = gw; j < d.n; j += nw) {
    double sc[2], sa[2];
    T rc[2], ra[2];
    auto srcc = [&](int i, T(&g)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) g[q] = on[q] ? yc[size_t(i) * kFK + lane + 32 * q] : T(0);
    };
    auto srca = [&](int i, T(&g)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!on[q]) {
          g[q] = T(0);
          continue;
        }
        const size_t o = size_t(i) * kFK + lane + 32 * q;
        T v = ya[o];
        if (fl[q] & kSlotAvg) v = blend(v, yc[o], w1[q], w[q]);
        g[q] = v;
      }
    };
    check_gather<T>(d.t_rowptr[j], d.t_rowptr[j + 1], d.t_cols, d.t_vals64, srcc, sc, rc);
    check_gather<T>(d.t_rowptr[j], d.t_rowptr[j + 1], d.t_cols, d.t_vals64, srca, sa, ra);
    const double Cj = d.C[j], iCj = d.invC[j], lj = d.l64[j], uj = d.u64[j];
    const T ljT = d.l[j], ujT = d.u[j];
    const unsigned long long lob = F.lo_bits[j], upb = F.up_bits[j];
    const FanCostCol<double> cc{F.cc64[3 * size_t(j)], F.cc64[3 * size_t(j) + 1], F.cc64[3 * size_t(j) + 2]};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(j) * kFK + k;
      const T x = Xc[o];
      // the average of points in [l, u] can leave it by a rounding: it is kept in the
      // box the iterates are clamped to, so that the point a check evaluates is the
      // one an objective finishing with it keeps (and returns)
      const T x0 = Xa[o];
      T xav = x0;
      if (fl[q] & kSlotAvg) xav = blend(xav, x, w1[q], w[q]);
      xav = clampv<T>(xav, ljT, ujT);
      if (xav != x0) Xa[o] = xav;
      F.ATY[0][o] = rc[q];
      F.ATY[1][o] = ra[q];
      const double cs = cc.at(int((lob >> k) & 1ULL) - int((upb >> k) & 1ULL));
      const double xl = to_f64(F.XLR[o]);
      const double xs[2] = {to_f64(x), to_f64(xav)};
      const double ss[2] = {sc[q], sa[q]};
      const bool boxed = above_neg_inf(lj) && below_pos_inf(uj);  // then r - lambda = 0 exactly
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double r = cs - ss[c];
        const double lam = rc_proj(r, lj, uj);
        double* a = acc + q * kNC1 + 5 * c;
        if (!boxed) {
          const double rd = r - lam;
          a[0] += rd * rd;
          const double rdu = rd * iCj;
          a[1] += rdu * rdu;
        }
        a[2] += cs * xs[c];
        a[3] += bound_term(lam, lj, uj);
        const double dd = xs[c] - xl;
        a[4] += dd * dd;
      }
      if (hs[q] && d.int_mask[j]) h[q] += round_hash(j, xs[0] * Cj);
    }
  }
  store_block_sums<double>(acc, kNC1, F.part_c1, sh);
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (on[q] && h[q]) atomicAdd(&F.ctl[lane + 32 * q].hash_accum, h[q]);
}

template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fcheck_rows(DevFan<T> F) {
  __shared__ double sh[kFWarps * kNC2 * kFK];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int cur = fan_cur(F);
  bool on[2];
  int fl[2];
  T w[2], w1[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = lane + 32 * q;
    fl[q] = k < F.K ? F.slot[k].flags : 0;
    on[q] = (fl[q] & kSlotCheck) != 0;
    w[q] = k < F.K ? F.slot[k].w : T(0);
    w1[q] = k < F.K ? F.slot[k].w1 : T(1);
  }
  double acc[2 * kNC2];
#pragma unroll
  for (int q = 0; q < 2 * kNC2; ++q) acc[q] = 0.0;
  const T* xc = F.X[cur];
  const T* xa = F.X[2];
  T* Yc = F.Y[cur];
  T* Ya = F.Y[2];
  for (int i = gw; i < d.m; i += nw) {
    double sc[2], sa[2];
    T rc[2], ra[2];
    auto srcc = [&](int j, T(&g)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) g[q] = on[q] ? xc[size_t(j) * kFK + lane + 32 * q] : T(0);
    };
    auto srca = [&](int j, T(&g)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) g[q] = on[q] ? xa[size_t(j) * kFK + lane + 32 * q] : T(0);
    };
    check_gather<T>(d.a_rowptr[i], d.a_rowptr[i + 1], d.a_cols, d.a_vals64, srcc, sc, rc);
    check_gather<T>(d.a_rowptr[i], d.a_rowptr[i + 1], d.a_cols, d.a_vals64, srca, sa, ra);
    const double iRi = d.invR[i], lo = d.lo64[i], hi = d.hi64[i];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(i) * kFK + k;
      const T y = Yc[o];
      T yav = Ya[o];
      if (fl[q] & kSlotAvg) {
        yav = blend(yav, y, w1[q], w[q]);
        Ya[o] = yav;
      }
      F.AX[cur][o] = rc[q];
      F.AX[2][o] = ra[q];
      const double yl = to_f64(F.YLR[o]);
      const double ys[2] = {to_f64(y), to_f64(yav)};
      const double ss[2] = {sc[q], sa[q]};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double rps = ss[c] - clampv<double>(ss[c], lo, hi);
        double* a = acc + q * kNC2 + 4 * c;
        a[0] += rps * rps;
        const double rp = rps * iRi;
        a[1] += rp * rp;
        a[2] += bound_term(ys[c], lo, hi);
        const double dd = ys[c] - yl;
        a[3] += dd * dd;
      }
    }
  }
  store_block_sums<double>(acc, kNC2, F.part_c2, sh);
}

// One warp per objective: check sums in a fixed order, then check_control.  An
// objective that restarts to its average or finishes with it (the single-LP path
// swaps its pool roles) gets rst[k] = 1 instead, and k_fcopy_rst copies the
// average into the current pool.  Block 0 refills the step-size factor table
// shared by the objectives still running.
template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fcheck_control(DevFan<T> F) {
  FanState* st = F.state;
  const long long k0 = *F.kglob;
  constexpr bool f32 = sizeof(T) == 4;
  // the step-size factors of attempts k0 + 1 .. k0 + n_check (entry i: attempt
  // k0 + 1 + i), shared by the objectives still running: FP64 for the FP64 decision,
  // FP32 (after the FP64 entries) for the FP32-mixed one
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < F.d.n_check; i += blockDim.x) {
      if (f32) {
        float* facf = reinterpret_cast<float*>(F.d.step_fac + 2 * F.d.n_check);
        const float kk = float(k0 + 1 + i + 1);
        facf[2 * i] = 1.0f - powf(kk, -float(F.exp_red));
        facf[2 * i + 1] = 1.0f + powf(kk, -float(F.exp_grow));
      } else {
        const double kk = double(k0 + 1 + i + 1);
        F.d.step_fac[2 * i] = 1.0 - pow(kk, -F.exp_red);
        F.d.step_fac[2 * i + 1] = 1.0 + pow(kk, -F.exp_grow);
      }
    }
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= F.K) return;
  if (!(F.slot[k].flags & kSlotCheck)) {
    if (lane == 0) st->rst[k] = 0;
    return;
  }
  double r[kNC1 + kNC2];
#pragma unroll
  for (int s = 0; s < kNC1 + kNC2; ++s) r[s] = 0.0;
  for (int b = lane; b < F.grid_c1; b += 32)
#pragma unroll
    for (int s = 0; s < kNC1; ++s) r[s] += F.part_c1[(b * kNC1 + s) * kFK + k];
  for (int b = lane; b < F.grid_c2; b += 32)
#pragma unroll
    for (int s = 0; s < kNC2; ++s) r[kNC1 + s] += F.part_c2[(b * kNC2 + s) * kFK + k];
#pragma unroll
  for (int s = 0; s < kNC1 + kNC2; ++s) r[s] = fwarp_sum(r[s]);
  if (lane == 0) {
    Control* c = &F.ctl[k];
    const int ix0 = c->ix_cur, ia0 = c->ia_cur;
    c->k_fac = k0;
    if (f32) {
      sync_step_state(c);  // eta and the weight sum from their FP32 copies
      const float kk = float(k0 + 2);  // attempt k0 + 1's factors, as the table's entry 0
      c->fr_f = 1.0f - powf(kk, -float(F.exp_red));
      c->fg_f = 1.0f + powf(kk, -float(F.exp_grow));
    }
    check_control(c, r, nullptr, 0);
    st->rst[k] = 0;
    if (c->ix_cur != ix0) {  // to the average: copy instead of swapping roles
      st->rst[k] = 1;
      c->ix_avg = c->ix_cur;
      c->ix_cur = ix0;
      c->ia_avg = c->ia_cur;
      c->ia_cur = ia0;
    }
    if (c->done) atomicAdd(F.n_done, 1);
    write_fan_slot(&F.slot[k], c);
  }
}

// Copies into the current pool, after the control kernels: RST = false, the
// objectives whose attempt was rejected get back the point they attempted from (now
// in the next pool: x, y, A x); RST = true, the ones that restart to or finish
// with their average get the average (x, y, A x and the check's A^T y).  A thread
// per (row, flagged objective) pair; nothing to do unless a flag is set.
template <typename T, bool RST>
__global__ void __launch_bounds__(kFThreads) k_fcopy(DevFan<T> F) {
  const FanState* st = F.state;
  const unsigned char* flag = RST ? st->rst : st->rej;
  // the flagged objectives, ascending
  __shared__ int list[kFK];
  __shared__ int cnt;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const bool a = lane < F.K && flag[lane] != 0, b = lane + 32 < F.K && flag[lane + 32] != 0;
    const unsigned ma = __ballot_sync(0xffffffffu, a), mb = __ballot_sync(0xffffffffu, b);
    const unsigned below = (1u << lane) - 1u;
    if (a) list[__popc(ma & below)] = lane;
    if (b) list[__popc(ma) + __popc(mb & below)] = lane + 32;
    if (lane == 0) cnt = __popc(ma) + __popc(mb);
  }
  __syncthreads();
  const int R = cnt;
  if (R == 0) return;
  const int cur = fan_cur(F), from = RST ? 2 : 1 - cur;
  const int n = F.d.n, m = F.d.m;
  const long long rows = n > m ? n : m, total = rows * R;
  const long long stride = (long long)gridDim.x * blockDim.x;
  T* __restrict__ xc = F.X[cur];
  const T* __restrict__ xf = F.X[from];
  T* __restrict__ yc = F.Y[cur];
  const T* __restrict__ yf = F.Y[from];
  T* __restrict__ axc = F.AX[cur];
  const T* __restrict__ axf = F.AX[from];
  T* __restrict__ atc = F.ATY[0];
  const T* __restrict__ atf = F.ATY[1];
  // (row, objective) pairs, four per thread and step: every load of a step is issued
  // before its stores, so the copies are bound by bandwidth, not by latency
  constexpr int U = 4;
  for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x; base < total; base += U * stride) {
    T vx[U], vy[U], vax[U], vat[U];
    size_t off[U];
    bool rx[U], ry[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long idx = base + u * stride;
      const int r = int(idx / R), k = list[int(idx % R)];
      off[u] = size_t(r) * kFK + k;
      rx[u] = idx < total && r < n;
      ry[u] = idx < total && r < m;
      if (rx[u]) {
        vx[u] = xf[off[u]];
        if (RST) vat[u] = atf[off[u]];
      }
      if (ry[u]) {
        vy[u] = yf[off[u]];
        vax[u] = axf[off[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (rx[u]) {
        xc[off[u]] = vx[u];
        if (RST) atc[off[u]] = vat[u];
      }
      if (ry[u]) {
        yc[off[u]] = vy[u];
        axc[off[u]] = vax[u];
      }
    }
  }
}

template <typename T>
__global__ void k_finit(DevFan<T> F, double tol, long long iter_limit, int stall_checks) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    *F.kglob = 0;
    *F.n_done = 0;
  }
  if (k >= F.K) return;
  Control* c = &F.ctl[k];
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
  write_fan_slot(&F.slot[k], c);
}

// every slot starts from the same pair x0, y0 (scaled, length n / m) in pool 0
template <typename T>
__global__ void k_fseed(DevFan<T> F, const T* x0, const T* y0) {
  const size_t nk = size_t(F.d.n) * kFK, mk = size_t(F.d.m) * kFK;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  const size_t t0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t0 < 64) {
    if (t0 == 0) F.state->att = 0ULL;
    F.state->rej[t0] = 0;
    F.state->rst[t0] = 0;
  }
  for (size_t o = t0; o < nk; o += stride) F.X[0][o] = x0[o / kFK];
  for (size_t o = t0; o < mk; o += stride) F.Y[0][o] = y0[o / kFK];
}

// FP32 objective pairs (t c_j C_j, om C_j) of the scaled space, one per column
// and the checks' FP64 triples (cw null in FP64)
template <typename T>
__global__ void k_fcw(DevFan<T> F, float2* cw, double* cc64) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < F.d.n; j += gridDim.x * blockDim.x) {
    const double Cj = F.d.C[j];
    if (cw) cw[j] = make_float2(float(F.t * F.c_orig[j] * Cj), float(F.om * Cj));
    const FanCostCol<double> cc = fan_cost_col64(F.t, F.om, F.c_orig[j], Cj);
    cc64[3 * size_t(j)] = cc.c0;
    cc64[3 * size_t(j) + 1] = cc.cp;
    cc64[3 * size_t(j) + 2] = cc.cm;
  }
}

template <typename T>
__global__ void k_fget_x(DevFan<T> F, int k, double* out) {
  const T* x = F.X[fan_cur(F)];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < F.d.n; j += gridDim.x * blockDim.x)
    out[j] = double(x[size_t(j) * kFK + k]) * F.d.C[j];
}

template <typename T>
__global__ void k_fget_y(DevFan<T> F, int k, double* out) {
  const T* y = F.Y[fan_cur(F)];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.d.m; i += gridDim.x * blockDim.x)
    out[i] = double(y[size_t(i) * kFK + k]) * F.d.R[i];
}

// ----------------------------------------------------------------- launchers ---
// kernel of a tile shape (see fan_shape_vec); FP64 takes shapes 2 and 4
template <typename T>
const void* fan_spmm_kernel(int side, int shape);
template <>
const void* fan_spmm_kernel<float>(int side, int shape) {
  switch (shape) {
    case 1: return side == 0 ? (const void*)k_fprimal<float, 4, 64> : (const void*)k_fdual<float, 4, 64>;
    case 3: return side == 0 ? (const void*)k_fprimal<float, 4, 32> : (const void*)k_fdual<float, 4, 32>;
    case 4: return side == 0 ? (const void*)k_fprimal<float, 2, 32> : (const void*)k_fdual<float, 2, 32>;
    default: return side == 0 ? (const void*)k_fprimal<float, 2, 64> : (const void*)k_fdual<float, 2, 64>;
  }
}
template <>
const void* fan_spmm_kernel<double>(int side, int shape) {
  if (shape == 4) return side == 0 ? (const void*)k_fprimal<double, 2, 32> : (const void*)k_fdual<double, 2, 32>;
  return side == 0 ? (const void*)k_fprimal<double, 2, 64> : (const void*)k_fdual<double, 2, 64>;
}

template <typename T>
cudaError_t launch_spmm(const DevFan<T>& F, int side, cudaStream_t st) {
  DevFan<T> arg = F;
  void* args[] = {&arg};
  const int grid = side == 0 ? F.grid_p : F.grid_d;
  return cudaLaunchKernel(fan_spmm_kernel<T>(side, side == 0 ? F.shape_p : F.shape_d), dim3(grid), dim3(kFThreads),
                          args, 0, st);
}

template <typename T>
cudaError_t launch_fan_init(const DevFan<T>& F, double tol, long long iter_limit, int stall_checks, cudaStream_t st) {
  k_finit<T><<<1, kFK, 0, st>>>(F, tol, iter_limit, stall_checks);
  return cudaGetLastError();
}

// one kernel of an attempt or a check on its own (measurement): 0 primal, 1 dual,
// 2 step control, 3 column check, 4 row check, 5 check control, 6 copies after the
// step control, 7 copies after the check control
template <typename T>
cudaError_t launch_fan_part(const DevFan<T>& F, int part, cudaStream_t st) {
  const int ctl_grid = (F.K * 32 + kFThreads - 1) / kFThreads;
  switch (part) {
    case 0: return launch_spmm<T>(F, 0, st);
    case 1: return launch_spmm<T>(F, 1, st);
    case 2: k_fstep_control<T><<<ctl_grid, kFThreads, 0, st>>>(F); break;
    case 3: k_fcheck_cols<T><<<F.grid_c1, kFThreads, 0, st>>>(F); break;
    case 4: k_fcheck_rows<T><<<F.grid_c2, kFThreads, 0, st>>>(F); break;
    case 5: k_fcheck_control<T><<<ctl_grid, kFThreads, 0, st>>>(F); break;
    case 6: k_fcopy<T, false><<<F.grid_copy, kFThreads, 0, st>>>(F); break;
    default: k_fcopy<T, true><<<F.grid_copy, kFThreads, 0, st>>>(F); break;
  }
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_slot(const DevFan<T>& F, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int part : {0, 1, 2, 6})
    if (e == cudaSuccess) e = launch_fan_part<T>(F, part, st);
  return e;
}
template <typename T>
cudaError_t launch_fan_check(const DevFan<T>& F, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int part : {3, 4, 5, 7})
    if (e == cudaSuccess) e = launch_fan_part<T>(F, part, st);
  return e;
}
template <typename T>
cudaError_t launch_fan_seed(const DevFan<T>& F, const void* x0, const void* y0, cudaStream_t st) {
  k_fseed<T><<<4 * device_sm_count(), kFThreads, 0, st>>>(F, static_cast<const T*>(x0), static_cast<const T*>(y0));
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_cw(const DevFan<T>& F, float2* cw, double* cc64, cudaStream_t st) {
  k_fcw<T><<<2 * device_sm_count(), kFThreads, 0, st>>>(F, cw, cc64);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_get_x(const DevFan<T>& F, int k, double* out, cudaStream_t st) {
  k_fget_x<T><<<4 * device_sm_count(), kFThreads, 0, st>>>(F, k, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_get_y(const DevFan<T>& F, int k, double* out, cudaStream_t st) {
  k_fget_y<T><<<4 * device_sm_count(), kFThreads, 0, st>>>(F, k, out);
  return cudaGetLastError();
}
template <typename T>
bool fan_shape_valid(int shape) {
  return sizeof(T) == 4 ? (shape >= 1 && shape <= 4) : (shape == 2 || shape == 4);
}
template <typename T>
void fan_grids(DevFan<T>& F) {
  auto grid = [](const void* k, long long units) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFThreads, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    long long need = (units + kFWarps - 1) / kFWarps;
    if (need < 1) need = 1;
    const long long cap = (long long)per_sm * device_sm_count();
    return int(need < cap ? need : cap);
  };
  // rows per warp of a shape: 32 VEC / CHUNK
  const int rpw_p = 32 * fan_shape_vec(F.shape_p) / fan_shape_chunk(F.shape_p);
  const int rpw_d = 32 * fan_shape_vec(F.shape_d) / fan_shape_chunk(F.shape_d);
  F.grid_p = grid(fan_spmm_kernel<T>(0, F.shape_p), (F.d.n + rpw_p - 1) / rpw_p);
  F.grid_d = grid(fan_spmm_kernel<T>(1, F.shape_d), (F.d.m + rpw_d - 1) / rpw_d);
  F.grid_c1 = grid((const void*)k_fcheck_cols<T>, F.d.n);
  F.grid_c2 = grid((const void*)k_fcheck_rows<T>, F.d.m);
  F.grid_copy = grid((const void*)k_fcopy<T, false>, F.d.n > F.d.m ? F.d.n : F.d.m);
}

#define SCYLLA_INSTANTIATE_FAN(T)                                                                      \
  template cudaError_t launch_fan_init<T>(const DevFan<T>&, double, long long, int, cudaStream_t);     \
  template cudaError_t launch_fan_slot<T>(const DevFan<T>&, cudaStream_t);                             \
  template cudaError_t launch_fan_check<T>(const DevFan<T>&, cudaStream_t);                            \
  template cudaError_t launch_fan_part<T>(const DevFan<T>&, int, cudaStream_t);                        \
  template cudaError_t launch_fan_seed<T>(const DevFan<T>&, const void*, const void*, cudaStream_t);   \
  template cudaError_t launch_fan_get_x<T>(const DevFan<T>&, int, double*, cudaStream_t);              \
  template cudaError_t launch_fan_get_y<T>(const DevFan<T>&, int, double*, cudaStream_t);              \
  template cudaError_t launch_fan_cw<T>(const DevFan<T>&, float2*, double*, cudaStream_t);            \
  template bool fan_shape_valid<T>(int);                                                               \
  template void fan_grids<T>(DevFan<T>&);

SCYLLA_INSTANTIATE_FAN(double)
SCYLLA_INSTANTIATE_FAN(float)

}  // namespace scylla
