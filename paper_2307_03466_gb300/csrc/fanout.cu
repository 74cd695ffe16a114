// K pump objectives of one LP solved together (the feasibility-pump fan-out):
// K independent PDHG runs (Algorithm 1 inner loop) that share A, A^T and the
// bounds and differ only in the objective, done as sparse-times-tall-skinny
// products so A is read once per K objectives.
//
// Layout: every K-wide vector is row-major (row j holds its K values contiguously),
// so a nonzero a_ij gathers one contiguous K-wide row.  A warp owns a row of A (or
// A^T); lane q owns objectives q and q + 32, so each lane keeps the step sizes and
// flags of its objectives in registers.  The warp streams the row's (index, value)
// pairs with one coalesced load per 32 nonzeros and broadcasts them with shuffles.
// The objective of column k is generated on the fly from the base c and two bit
// planes (target at the lower / upper bound) instead of being stored K times:
// c_hat_jk = alpha^K s c_j + (1 - alpha^K) g_jk (Section 2.4).
//
// Every objective has its own control block (step size, primal weight, restarts,
// termination) and pool roles; sums are per block and per objective, reduced per
// objective by one warp in the control kernels, which apply the same logic as the
// single-LP path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace scylla {

constexpr int kFK = 64;       // objectives per fan-out (two per lane)
constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;

__device__ __forceinline__ double fwarp_sum(double v) { return warp_sum(v); }

template <typename T>
struct FanLane {  // the per-objective values of one lane's two objectives
  T tau[2], sigma[2], w[2], w1[2];
  int cur[2], nxt[2], avg[2], ia_cur[2], ia_avg[2], flags[2];
  bool on[2];
};

template <typename T>
__device__ __forceinline__ void load_lane(const DevFan<T>& F, FanLane<T>& L, bool check) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = lane + 32 * q;
    if (k < F.K) {
      const BatchSlot<T> s = F.slot[k];
      L.tau[q] = s.tau;
      L.sigma[q] = s.sigma;
      L.w[q] = s.w;
      L.w1[q] = s.w1;
      L.cur[q] = s.cur;
      L.nxt[q] = s.nxt;
      L.avg[q] = s.avg;
      L.ia_cur[q] = s.ia_cur;
      L.ia_avg[q] = s.ia_avg;
      L.flags[q] = s.flags;
      L.on[q] = (s.flags & (check ? 16 : 1)) != 0;
    } else {
      L.on[q] = false;
      L.flags[q] = 0;
      L.cur[q] = L.nxt[q] = L.avg[q] = L.ia_cur[q] = L.ia_avg[q] = 0;
      L.tau[q] = L.sigma[q] = L.w[q] = L.w1[q] = T(0);
    }
  }
}

// g_jk of the l1 distance: +1 target at l_j, -1 target at u_j, 0 otherwise
__device__ __forceinline__ double fan_g(const unsigned long long* lo_bits, const unsigned long long* up_bits, int j,
                                        int k) {
  const unsigned long long b = 1ULL << k;
  if (lo_bits[j] & b) return 1.0;
  if (up_bits[j] & b) return -1.0;
  return 0.0;
}

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

template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fprimal(DevFan<T> F) {
  typedef typename AccOf<T>::type A;
  __shared__ double sh[kFWarps * 1 * kFK];
  FanLane<T> L;
  load_lane(F, L, false);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int K = F.K;
  A acc[2] = {A(0), A(0)};
  const T* ysrc[2] = {F.Y[L.cur[0]], F.Y[L.cur[1]]};
  auto src = [&](int i, T(&g)[2]) {
    g[0] = L.on[0] ? __ldg(ysrc[0] + size_t(i) * K + lane) : T(0);
    g[1] = L.on[1] ? __ldg(ysrc[1] + size_t(i) * K + lane + 32) : T(0);
  };
  for (int j = gw; j < d.n; j += nw) {
    T s[2];
    row_gather<T, T>(d.t_rowptr[j], d.t_rowptr[j + 1], d.t_cols, d.t_vals, src, s);
    const double Cj = d.C[j], cj = F.c_orig[j];
    const T lj = d.l[j], uj = d.u[j];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!L.on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(j) * K + k;
      const bool cached = (L.flags[q] & 4) != 0;
      T* aty = F.ATY[L.ia_cur[q]];
      const T a = cached ? aty[o] : s[q];
      if (!cached) aty[o] = a;
      const T x = F.X[L.cur[q]][o];
      if (L.flags[q] & 8) F.X[L.avg[q]][o] = blend(F.X[L.avg[q]][o], x, L.w1[q], L.w[q]);
      if (L.flags[q] & 2) F.XLR[o] = x;
      const T cs = T((F.t * cj + F.om * fan_g(F.lo_bits, F.up_bits, j, k)) * Cj);
      const T v = clampv<T>(x + L.tau[q] * (a - cs), lj, uj);
      F.X[L.nxt[q]][o] = v;
      const A dx = A(v) - A(x);
      acc[q] += dx * dx;
    }
  }
  store_block_sums<T>(acc, 1, F.part_p, sh);
}

template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fdual(DevFan<T> F) {
  typedef typename AccOf<T>::type A;
  __shared__ double sh[kFWarps * 2 * kFK];
  FanLane<T> L;
  load_lane(F, L, false);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int K = F.K;
  A acc[4] = {A(0), A(0), A(0), A(0)};  // [q][dy2, inter]
  const T* xsrc[2] = {F.X[L.nxt[0]], F.X[L.nxt[1]]};
  auto src = [&](int j, T(&g)[2]) {
    g[0] = L.on[0] ? __ldg(xsrc[0] + size_t(j) * K + lane) : T(0);
    g[1] = L.on[1] ? __ldg(xsrc[1] + size_t(j) * K + lane + 32) : T(0);
  };
  for (int i = gw; i < d.m; i += nw) {
    T s[2];
    row_gather<T, T>(d.a_rowptr[i], d.a_rowptr[i + 1], d.a_cols, d.a_vals, src, s);
    const T lo = d.lo[i], hi = d.hi[i];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!L.on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(i) * K + k;
      const T ax = F.AX[L.cur[q]][o];
      const T y = F.Y[L.cur[q]][o];
      if (L.flags[q] & 8) F.Y[L.avg[q]][o] = blend(F.Y[L.avg[q]][o], y, L.w1[q], L.w[q]);
      if (L.flags[q] & 2) F.YLR[o] = y;
      const T axt = T(2) * s[q] - ax;
      const T v = dual_prox<T>(y, L.sigma[q], axt, lo, hi);
      F.Y[L.nxt[q]][o] = v;
      F.AX[L.nxt[q]][o] = s[q];
      const A dy = A(v) - A(y);
      acc[2 * q] += dy * dy;
      acc[2 * q + 1] += dy * (A(s[q]) - A(ax));
    }
  }
  store_block_sums<T>(acc, 2, F.part_d, sh);
}

// one warp per objective: block sums in a fixed order, then the step decision
template <typename T>
__global__ void k_fstep_control(DevFan<T> F) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ++*F.kglob;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= F.K) return;
  if (!(F.slot[k].flags & 1)) return;
  const int G = F.grid_p, H = F.grid_d;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int b = lane; b < G; b += 32) s0 += F.part_p[b * kFK + k];
  for (int b = lane; b < H; b += 32) {
    s1 += F.part_d[(b * 2 + 0) * kFK + k];
    s2 += F.part_d[(b * 2 + 1) * kFK + k];
  }
  s0 = fwarp_sum(s0);
  s1 = fwarp_sum(s1);
  s2 = fwarp_sum(s2);
  if (lane == 0) {
    Control* c = &F.ctl[k];
    step_control(c, s0, s1, s2, F.d.step_fac, F.d.n_check, nullptr, 0);
    if (c->done) atomicAdd(F.n_done, 1);
    write_fan_slot(&F.slot[k], c);
  }
}

// FP64 column half of a check for every objective: A^T y of the current and the
// averaged dual, reduced costs against c_hat_k, residuals, objectives, hash
template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fcheck_cols(DevFan<T> F) {
  __shared__ double sh[kFWarps * kNC1 * kFK];
  FanLane<T> L;
  load_lane(F, L, true);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int K = F.K;
  double acc[2 * kNC1];
#pragma unroll
  for (int q = 0; q < 2 * kNC1; ++q) acc[q] = 0.0;
  unsigned long long h[2] = {0ULL, 0ULL};
  const T* yc[2] = {F.Y[L.cur[0]], F.Y[L.cur[1]]};
  const T* ya[2] = {F.Y[L.avg[0]], F.Y[L.avg[1]]};
  for (int j = gw; j < d.n; j += nw) {
    double sc[2], sa[2];
    auto srcc = [&](int i, double(&g)[2]) {
      g[0] = L.on[0] ? double(yc[0][size_t(i) * K + lane]) : 0.0;
      g[1] = L.on[1] ? double(yc[1][size_t(i) * K + lane + 32]) : 0.0;
    };
    auto srca = [&](int i, double(&g)[2]) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!L.on[q]) {
          g[q] = 0.0;
          continue;
        }
        const size_t o = size_t(i) * K + lane + 32 * q;
        T v = ya[q][o];
        if (L.flags[q] & 8) v = blend(v, yc[q][o], L.w1[q], L.w[q]);
        g[q] = double(v);
      }
    };
    row_gather<double, double>(d.t_rowptr[j], d.t_rowptr[j + 1], d.t_cols, d.t_vals64, srcc, sc);
    row_gather<double, double>(d.t_rowptr[j], d.t_rowptr[j + 1], d.t_cols, d.t_vals64, srca, sa);
    const double Cj = d.C[j], cj = F.c_orig[j], lj = d.l64[j], uj = d.u64[j];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!L.on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(j) * K + k;
      const T x = F.X[L.cur[q]][o];
      T xav = F.X[L.avg[q]][o];
      if (L.flags[q] & 8) {
        xav = blend(xav, x, L.w1[q], L.w[q]);
        F.X[L.avg[q]][o] = xav;
      }
      F.ATY[L.ia_cur[q]][o] = T(sc[q]);
      F.ATY[L.ia_avg[q]][o] = T(sa[q]);
      const double cs = (F.t * cj + F.om * fan_g(F.lo_bits, F.up_bits, j, k)) * Cj;
      const double xl = double(F.XLR[o]);
      const double xs[2] = {double(x), double(xav)};
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
          const double rdu = rd / Cj;
          a[1] += rdu * rdu;
        }
        a[2] += cs * xs[c];
        a[3] += bound_term(lam, lj, uj);
        const double dd = xs[c] - xl;
        a[4] += dd * dd;
      }
      if (d.int_mask[j]) h[q] += round_hash(j, double(x) * Cj);
    }
  }
  store_block_sums<double>(acc, kNC1, F.part_c1, sh);
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (L.on[q] && h[q]) atomicAdd(&F.ctl[lane + 32 * q].hash_accum, h[q]);
}

template <typename T>
__global__ void __launch_bounds__(kFThreads) k_fcheck_rows(DevFan<T> F) {
  __shared__ double sh[kFWarps * kNC2 * kFK];
  FanLane<T> L;
  load_lane(F, L, true);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const DevLP<T>& d = F.d;
  const int K = F.K;
  double acc[2 * kNC2];
#pragma unroll
  for (int q = 0; q < 2 * kNC2; ++q) acc[q] = 0.0;
  const T* xc[2] = {F.X[L.cur[0]], F.X[L.cur[1]]};
  const T* xa[2] = {F.X[L.avg[0]], F.X[L.avg[1]]};
  for (int i = gw; i < d.m; i += nw) {
    double sc[2], sa[2];
    auto srcc = [&](int j, double(&g)[2]) {
      g[0] = L.on[0] ? double(xc[0][size_t(j) * K + lane]) : 0.0;
      g[1] = L.on[1] ? double(xc[1][size_t(j) * K + lane + 32]) : 0.0;
    };
    auto srca = [&](int j, double(&g)[2]) {
      g[0] = L.on[0] ? double(xa[0][size_t(j) * K + lane]) : 0.0;
      g[1] = L.on[1] ? double(xa[1][size_t(j) * K + lane + 32]) : 0.0;
    };
    row_gather<double, double>(d.a_rowptr[i], d.a_rowptr[i + 1], d.a_cols, d.a_vals64, srcc, sc);
    row_gather<double, double>(d.a_rowptr[i], d.a_rowptr[i + 1], d.a_cols, d.a_vals64, srca, sa);
    const double Ri = d.R[i], lo = d.lo64[i], hi = d.hi64[i];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!L.on[q]) continue;
      const int k = lane + 32 * q;
      const size_t o = size_t(i) * K + k;
      const T y = F.Y[L.cur[q]][o];
      T yav = F.Y[L.avg[q]][o];
      if (L.flags[q] & 8) {
        yav = blend(yav, y, L.w1[q], L.w[q]);
        F.Y[L.avg[q]][o] = yav;
      }
      F.AX[L.cur[q]][o] = T(sc[q]);
      F.AX[L.avg[q]][o] = T(sa[q]);
      const double yl = double(F.YLR[o]);
      const double ys[2] = {double(y), double(yav)};
      const double ss[2] = {sc[q], sa[q]};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double rps = ss[c] - clampv<double>(ss[c], lo, hi);
        double* a = acc + q * kNC2 + 4 * c;
        a[0] += rps * rps;
        const double rp = rps / Ri;
        a[1] += rp * rp;
        a[2] += bound_term(ys[c], lo, hi);
        const double dd = ys[c] - yl;
        a[3] += dd * dd;
      }
    }
  }
  store_block_sums<double>(acc, kNC2, F.part_c2, sh);
}

// one warp per objective: check sums in a fixed order, then check_control; block 0
// refills the step-size factor table shared by the objectives still running
template <typename T>
__global__ void k_fcheck_control(DevFan<T> F) {
  if (blockIdx.x == 0) {
    const long long k0 = *F.kglob;
    for (int i = threadIdx.x; i < F.d.n_check; i += blockDim.x) {
      const double kk = double(k0 + 1 + i + 1);
      F.d.step_fac[2 * i] = 1.0 - pow(kk, -F.exp_red);
      F.d.step_fac[2 * i + 1] = 1.0 + pow(kk, -F.exp_grow);
    }
  }
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= F.K) return;
  if (!(F.slot[k].flags & 16)) return;
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
    c->k_fac = *F.kglob;
    check_control(c, r, nullptr, 0);
    if (c->done) atomicAdd(F.n_done, 1);
    write_fan_slot(&F.slot[k], c);
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

// every objective starts from the same pair: x0, y0 (scaled, length n / m), roles 0
template <typename T>
__global__ void k_fseed(DevFan<T> F, const T* x0, const T* y0) {
  const int K = F.K;
  const size_t nk = size_t(F.d.n) * K, mk = size_t(F.d.m) * K;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t o = size_t(blockIdx.x) * blockDim.x + threadIdx.x; o < nk; o += stride) F.X[0][o] = x0[o / K];
  for (size_t o = size_t(blockIdx.x) * blockDim.x + threadIdx.x; o < mk; o += stride) F.Y[0][o] = y0[o / K];
}

template <typename T>
__global__ void k_fget_x(DevFan<T> F, int k, double* out) {
  const T* x = F.X[F.ctl[k].ix_cur];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < F.d.n; j += gridDim.x * blockDim.x)
    out[j] = double(x[size_t(j) * F.K + k]) * F.d.C[j];
}

// ----------------------------------------------------------------- launchers ---
template <typename T>
cudaError_t launch_fan_init(const DevFan<T>& F, double tol, long long iter_limit, int stall_checks, cudaStream_t st) {
  k_finit<T><<<1, kFK, 0, st>>>(F, tol, iter_limit, stall_checks);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_slot(const DevFan<T>& F, cudaStream_t st) {
  k_fprimal<T><<<F.grid_p, kFThreads, 0, st>>>(F);
  k_fdual<T><<<F.grid_d, kFThreads, 0, st>>>(F);
  k_fstep_control<T><<<(F.K * 32 + kFThreads - 1) / kFThreads, kFThreads, 0, st>>>(F);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_check(const DevFan<T>& F, cudaStream_t st) {
  k_fcheck_cols<T><<<F.grid_c1, kFThreads, 0, st>>>(F);
  k_fcheck_rows<T><<<F.grid_c2, kFThreads, 0, st>>>(F);
  k_fcheck_control<T><<<(F.K * 32 + kFThreads - 1) / kFThreads, kFThreads, 0, st>>>(F);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_seed(const DevFan<T>& F, const void* x0, const void* y0, cudaStream_t st) {
  k_fseed<T><<<4 * device_sm_count(), kFThreads, 0, st>>>(F, static_cast<const T*>(x0), static_cast<const T*>(y0));
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fan_get_x(const DevFan<T>& F, int k, double* out, cudaStream_t st) {
  k_fget_x<T><<<4 * device_sm_count(), kFThreads, 0, st>>>(F, k, out);
  return cudaGetLastError();
}
template <typename T>
void fan_grids(DevFan<T>& F) {
  auto grid = [](const void* k, int rows) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFThreads, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    long long need = (rows + kFWarps - 1) / kFWarps;
    if (need < 1) need = 1;
    const long long cap = (long long)per_sm * device_sm_count();
    return int(need < cap ? need : cap);
  };
  F.grid_p = grid((const void*)k_fprimal<T>, F.d.n);
  F.grid_d = grid((const void*)k_fdual<T>, F.d.m);
  F.grid_c1 = grid((const void*)k_fcheck_cols<T>, F.d.n);
  F.grid_c2 = grid((const void*)k_fcheck_rows<T>, F.d.m);
}

#define SCYLLA_INSTANTIATE_FAN(T)                                                                      \
  template cudaError_t launch_fan_init<T>(const DevFan<T>&, double, long long, int, cudaStream_t);     \
  template cudaError_t launch_fan_slot<T>(const DevFan<T>&, cudaStream_t);                             \
  template cudaError_t launch_fan_check<T>(const DevFan<T>&, cudaStream_t);                            \
  template cudaError_t launch_fan_seed<T>(const DevFan<T>&, const void*, const void*, cudaStream_t);   \
  template cudaError_t launch_fan_get_x<T>(const DevFan<T>&, int, double*, cudaStream_t);              \
  template void fan_grids<T>(DevFan<T>&);

SCYLLA_INSTANTIATE_FAN(double)
SCYLLA_INSTANTIATE_FAN(float)

}  // namespace scylla
