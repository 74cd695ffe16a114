// Device helpers shared by the CUDA translation units of the PDHG path: warp and
// block reductions, the proximal steps of Algorithm 1, the rounding hash, and the
// control logic (adaptive step size, checks, restarts, termination) that the
// single-LP, batched and multi-objective kernels all apply to a Control block.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace scylla {

// ------------------------------------------------------------------ helpers ---
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void ld4(const int* p, int (&o)[4]) {
  const int4 t = __ldg(reinterpret_cast<const int4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// The same loads with the streaming cache hint (ld.global.cs: lines allocated
// evict-first in L1 and L2), for matrix data read once per launch while the gathered
// vector should stay in L2.
__device__ __forceinline__ void ld4s(const int* p, int (&o)[4]) {
  const int4 t = __ldcs(reinterpret_cast<const int4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4s(const float* p, float (&o)[4]) {
  const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4s(const double* p, double (&o)[4]) {
  const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <bool kStream, typename V>
__device__ __forceinline__ void ld4_as(const V* p, V (&o)[4]) {
  if constexpr (kStream) ld4s(p, o);
  else ld4(p, o);
}

// float -> double without the FP64 pipe (where a conversion costs as much as an FP64
// add): sign, exponent rebiased by 1023 - 127, mantissa shifted into place; exact for
// zeros and normal numbers, which is all the iterates hold; subnormals, infinities and
// NaNs take the hardware conversion
__device__ __forceinline__ double to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xffu, man = b & 0x7fffffu;
  if (e == 0xffu || (e == 0u && man != 0u)) return double(f);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long body =
      e == 0u ? 0ULL : ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)man << 29);
  return __longlong_as_double((long long)(sign | body));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

__device__ __forceinline__ int skew(int q) { return q + (q >> 5); }

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  v = v < lo ? lo : v;
  return v > hi ? hi : v;
}
template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// running average x_avg <- (1-w) x_avg + w x, in one fixed rounding sequence
template <typename T>
__device__ __forceinline__ T blend(T a, T x, T w1, T w) { return fma_t<T>(w1, a, w * x); }

template <typename T>
__device__ __forceinline__ T pos_inf();
template <>
__device__ __forceinline__ double pos_inf<double>() { return __longlong_as_double(0x7ff0000000000000ULL); }
template <>
__device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }

// Dual step of Algorithm 1 for a row with bounds [lo, hi] (the proximal step of
// the row-bound support function); lo = b, hi = +inf gives max(0, y + s (b - axt)).
template <typename T>
__device__ __forceinline__ T dual_prox(T y, T sigma, T axt, T lo, T hi) {
  const T inf = pos_inf<T>();
  if (lo > -inf) {
    const T t = y + sigma * (lo - axt);
    if (t > T(0)) return t;
  }
  if (hi < inf) {
    const T t = y + sigma * (hi - axt);
    if (t < T(0)) return t;
  }
  return T(0);
}

// Sign and finiteness tests of non-NaN doubles on their bit patterns (integer
// instructions; an FP64 comparison occupies the slow FP64 pipe of this part):
// v > 0 iff the bits are positive as a signed integer; v < 0 iff they are negative
// and v is not -0; v > -inf and v < +inf iff the bits differ from those of -inf, +inf.
__device__ __forceinline__ bool pos_bits(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool neg_bits(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool above_neg_inf(double v) {
  return __double_as_longlong(v) != (long long)0xFFF0000000000000ULL;
}
__device__ __forceinline__ bool below_pos_inf(double v) { return __double_as_longlong(v) != 0x7FF0000000000000LL; }

// FP64 dual step with the sign and finiteness tests on the integer pipe (the same
// result as the generic form for every non-NaN value; a NaN t is passed on instead of
// being replaced by 0, so the step-size reduction reports it)
template <>
__device__ __forceinline__ double dual_prox<double>(double y, double sigma, double axt, double lo, double hi) {
  if (above_neg_inf(lo)) {
    const double t = y + sigma * (lo - axt);
    if (pos_bits(t)) return t;
  }
  if (below_pos_inf(hi)) {
    const double t = y + sigma * (hi - axt);
    if (neg_bits(t)) return t;
  }
  return 0.0;
}

// lambda = projection of the reduced cost r onto the sign cone of the column bounds
__device__ __forceinline__ double rc_proj(double r, double l, double u) {
  const bool lf = above_neg_inf(l), uf = below_pos_inf(u);
  if (lf && uf) return r;
  if (lf) return pos_bits(r) ? r : 0.0;
  if (uf) return neg_bits(r) ? r : 0.0;
  return 0.0;
}

// The bound term of a multiplier v against a bound pair: a v when v > 0, b v when
// v < 0, 0 otherwise; the same value as (v > 0 ? a v : 0) - (v < 0 ? b (-v) : 0) in
// one product.
__device__ __forceinline__ double bound_term(double v, double a, double b) {
  const double s = pos_bits(v) ? a : (neg_bits(v) ? b : 0.0);
  return s * v;
}

// SplitMix64 output function (Steele, Lea, Flood 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long round_hash(long long j, double v) {
  double r = floor(v + 0.5);
  const double lim = 4611686018427387904.0;  // 2^62
  r = r < -lim ? -lim : (r > lim ? lim : r);
  const unsigned long long key =
      (unsigned long long)j * 0x9E3779B97F4A7C15ULL + (unsigned long long)(long long)r;
  return mix64(key);
}

// per-block reduction of N partial sums into part[blockIdx.x * N + k], fixed order,
// in the accumulator type A (FP32 sums of the FP32 bulk stay on the FP32 pipe)
template <int N, typename A>
__device__ __forceinline__ void block_store_partials(const A (&v)[N], A* __restrict__ part) {
  __shared__ A sh[kMaxWarps][N];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const A t = warp_sum(v[k]);
    if (lane == 0) sh[w][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    A s = A(0);
    for (int i = 0; i < nw; ++i) s += sh[i][threadIdx.x];
    part[blockIdx.x * N + threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool is_last_block(unsigned int* counter) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    if (last) __threadfence();
  }
  __syncthreads();
  return last != 0;
}

// sums of two partial arrays (NA values over na blocks, NB over nb) by warps 1.. of
// the (last) block, in a fixed order: each thread loads a strided subset (the first
// two blocks' values before summing any), the per-thread sums go to scratch
// (N * (blockDim.x - 32) doubles), then each warp reduces whole columns across its
// lanes.  Warp 0 is left free; every thread leaves with out[0..N-1] valid.
template <int NA, int NB>
static __device__ void reduce_two(const double* pa, int na, const double* pb, int nb, double* scratch,
                                  double* out) {
  constexpr int N = NA + NB;
  const int nt = blockDim.x - 32, t = threadIdx.x - 32;
  if (t >= 0) {
    double s[N];
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = 0.0;
    constexpr int kR = 2;
    double va[kR][NA], vb[kR][NB];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const int b = t + r * nt;
#pragma unroll
      for (int k = 0; k < NA; ++k) va[r][k] = b < na ? __ldcg(pa + b * NA + k) : 0.0;
#pragma unroll
      for (int k = 0; k < NB; ++k) vb[r][k] = b < nb ? __ldcg(pb + b * NB + k) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
#pragma unroll
      for (int k = 0; k < NA; ++k) s[k] += va[r][k];
#pragma unroll
      for (int k = 0; k < NB; ++k) s[NA + k] += vb[r][k];
    }
    for (int b = t + kR * nt; b < na; b += nt)
#pragma unroll
      for (int k = 0; k < NA; ++k) s[k] += __ldcg(pa + b * NA + k);
    for (int b = t + kR * nt; b < nb; b += nt)
#pragma unroll
      for (int k = 0; k < NB; ++k) s[NA + k] += __ldcg(pb + b * NB + k);
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[k * nt + t] = s[k];
    asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    const int w = t >> 5, lane = t & 31, nw = nt >> 5;
    for (int k = w; k < N; k += nw) {
      double v = 0.0;
      for (int i = lane; i < nt; i += 32) v += scratch[k * nt + i];
      v = warp_sum(v);
      if (lane == 0) out[k] = v;
    }
  }
  __syncthreads();
}

// sums of one partial array (N values over np blocks) by warps 1.., like reduce_two
template <int N>
static __device__ void reduce_one(const double* p, int np, double* scratch, double* out) {
  const int nt = blockDim.x - 32, t = threadIdx.x - 32;
  if (t >= 0) {
    double s[N];
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = 0.0;
    constexpr int kR = 2;
    double v[kR][N];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const int b = t + r * nt;
#pragma unroll
      for (int k = 0; k < N; ++k) v[r][k] = b < np ? __ldcg(p + b * N + k) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r)
#pragma unroll
      for (int k = 0; k < N; ++k) s[k] += v[r][k];
    for (int b = t + kR * nt; b < np; b += nt)
#pragma unroll
      for (int k = 0; k < N; ++k) s[k] += __ldcg(p + b * N + k);
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[k * nt + t] = s[k];
    asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    const int w = t >> 5, lane = t & 31, nw = nt >> 5;
    for (int k = w; k < N; k += nw) {
      double x = 0.0;
      for (int i = lane; i < nt; i += 32) x += scratch[k * nt + i];
      x = warp_sum(x);
      if (lane == 0) out[k] = x;
    }
  }
  __syncthreads();
}

// column k of a partial array (N values over np blocks) by the whole block, in a
// fixed order; thread 0 returns the sum
template <int N>
static __device__ double block_column_sum(const double* p, int np, int k) {
  __shared__ double sh[kMaxWarps];
  double x = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) x += __ldcg(p + b * N + k);
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ float ldcg_t(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_t(const double* p) { return __ldcg(p); }

// The three sums of an attempt (||dx||^2 from na primal-block partials; ||dy||^2 and
// the interaction from nb dual-block partials) by warps 1.. of the block, in a fixed
// order: strided per-thread sums to scratch (3 * (blockDim.x - 32) values), then
// warp 1 + k sums column k and reduces it across its lanes.  Warp 0 is left free for
// the caller (it prefetches the decision's inputs meanwhile); every thread leaves
// with out[0..2] valid.
template <typename A>
static __device__ void reduce_step(const A* pa, int na, const A* pb, int nb, A* scratch, A* out) {
  const int nt = blockDim.x - 32, t = threadIdx.x - 32;
  if (t >= 0) {
    // the first kR values of each thread are loaded before any is summed
    constexpr int kR = 6;
    A va[kR], vb[kR], vc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const int ba = t + r * nt, bb = t + r * nt;
      va[r] = ba < na ? ldcg_t(pa + ba) : A(0);
      vb[r] = bb < nb ? ldcg_t(pb + 2 * bb) : A(0);
      vc[r] = bb < nb ? ldcg_t(pb + 2 * bb + 1) : A(0);
    }
    A s0 = A(0), s1 = A(0), s2 = A(0);
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      s0 += va[r];
      s1 += vb[r];
      s2 += vc[r];
    }
    for (int b = t + kR * nt; b < na; b += nt) s0 += ldcg_t(pa + b);
    for (int b = t + kR * nt; b < nb; b += nt) {
      s1 += ldcg_t(pb + 2 * b);
      s2 += ldcg_t(pb + 2 * b + 1);
    }
    scratch[t] = s0;
    scratch[nt + t] = s1;
    scratch[2 * nt + t] = s2;
    asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    const int w = t >> 5, lane = t & 31;
    if (w < 3) {
      A v = A(0);
      for (int i = lane; i < nt; i += 32) v += scratch[w * nt + i];
      v = warp_sum(v);
      if (lane == 0) out[w] = v;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------- step control ---
// Adaptive step (PDLP): eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy.A dx|);
// eta' = min((1 - (k+1)^-0.3) eta_max, (1 + (k+1)^-0.6) eta), k the 1-based attempt
// number; the attempt is accepted when eta <= eta_max.  The two powers come from
// a table that the check kernel fills for the next n_check attempts (FP64
// transcendentals are slow on this part; in the table they run in parallel).
//
// The decision is split in two: step_pre gathers and prepares everything that
// does not depend on the attempt's sums (it runs while they are being reduced),
// step_control finishes once they are known.  C is the type of the decision
// arithmetic: double in the FP64 mode; float in the FP32-mixed mode, whose sums
// are FP32 already (every FP64 instruction is a long serial step on this part).

// tau, sigma and the averaging weights of the next attempt from eta, omega, avg_w
__device__ __forceinline__ void derive_steps(Control* c) {
  const double eta = c->eta, om = c->omega, w = c->avg_w;
  c->inv_omega = 1.0 / om;
  c->tau_d = eta * c->inv_omega;
  c->sigma_d = eta * om;
  c->w_d = w;
  c->w1_d = 1.0 - w;
  c->tau_f = float(c->tau_d);
  c->sigma_f = float(c->sigma_d);
  c->w_f = float(w);
  c->w1_f = float(c->w1_d);
  c->avg_on = w > 0.0 ? 1 : 0;
  c->eta_f = float(eta);
  c->om_f = float(om);
  c->iom_f = float(c->inv_omega);
  c->wsum_f = float(c->wsum);
}

// FP32-mixed mode, before a check: the FP64 step-size state from its FP32 copies
__device__ __forceinline__ void sync_step_state(Control* c) {
  c->eta = double(c->eta_f);
  c->wsum = double(c->wsum_f);
}

struct StepPre {
  long long k1;
  double eta, om, inv_om, fr, fg, wsum_new, w_acc;  // FP64 mode
  float eta_f, om_f, iom_f, fr_f, fg_f, wsum_new_f, w_acc_f, fr_next, fg_next;  // FP32 mode
  int adaptive;
};

// FP64 mode: this attempt's factors from the table
static __device__ void step_factors(const Control* c, const double* fac, int n_check, long long k1, double& fr,
                                    double& fg) {
  const long long idx = k1 - 1 - c->k_fac;
  if (idx >= 0 && idx < n_check) {
    fr = fac[2 * idx];
    fg = fac[2 * idx + 1];
  } else {
    const double kk = double(k1 + 1);
    fr = 1.0 - pow(kk, -c->exp_red);
    fg = 1.0 + pow(kk, -c->exp_grow);
  }
}

template <typename C>
static __device__ StepPre step_pre(const Control* c, const double* fac, int n_check);

template <>
__device__ StepPre step_pre<double>(const Control* c, const double* fac, int n_check) {
  StepPre p;
  p.k1 = c->k + 1;
  p.eta = c->eta;
  p.om = c->omega;
  p.inv_om = c->inv_omega;
  p.adaptive = c->adaptive;
  p.wsum_new = c->wsum + p.eta;
  p.w_acc = p.eta / p.wsum_new;  // the averaging weight if the attempt is accepted
  p.fr = 1.0;
  p.fg = 1.0;
  if (p.adaptive) step_factors(c, fac, n_check, p.k1, p.fr, p.fg);
  return p;
}

// FP32 mode: everything from the FP32 copies; this attempt's factors were stored by
// the previous decision (or the check), the next attempt's come from the FP32 table
template <>
__device__ StepPre step_pre<float>(const Control* c, const double* fac, int n_check) {
  StepPre p;
  p.k1 = c->k + 1;
  p.eta_f = c->eta_f;
  p.om_f = c->om_f;
  p.iom_f = c->iom_f;
  p.adaptive = c->adaptive;
  p.fr_f = c->fr_f;
  p.fg_f = c->fg_f;
  p.wsum_new_f = c->wsum_f + p.eta_f;
  p.w_acc_f = p.eta_f / p.wsum_new_f;
  const long long idx = p.k1 - c->k_fac;  // table index of attempt k1 + 1
  if (idx >= 0 && idx < n_check) {
    const float* facf = reinterpret_cast<const float*>(fac + 2 * n_check);
    p.fr_next = facf[2 * idx];
    p.fg_next = facf[2 * idx + 1];
  } else {
    double fr, fg;
    step_factors(c, fac, n_check, p.k1 + 1, fr, fg);
    p.fr_next = float(fr);
    p.fg_next = float(fg);
  }
  return p;
}

template <typename C>
static __device__ void step_control(Control* c, const StepPre& p, C dx2, C dy2, C inter, double* trace, int cap);

// FP64 mode
template <>
__device__ void step_control<double>(Control* c, const StepPre& p, double dx2, double dy2, double inter,
                                     double* trace, int cap) {
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(inter)) {
    c->done = 1;
    c->status = SCYLLA_NUMERICAL;
    return;
  }
  bool accept = true;
  double eta_next = p.eta;
  double eta_max = pos_inf<double>();
  if (p.adaptive) {
    const double mv = p.om * dx2 + dy2 * p.inv_om;
    eta_max = inter != 0.0 ? mv / (2.0 * fabs(inter)) : pos_inf<double>();
    eta_next = fmin(p.fr * eta_max, p.fg * p.eta);
    accept = p.eta <= eta_max;
  }
  const long long k1 = p.k1;
  if (trace && k1 <= cap) {
    double* t = trace + 4 * (k1 - 1);
    t[0] = p.eta;
    t[1] = eta_max;
    t[2] = accept ? 1.0 : 0.0;
    t[3] = eta_next;
  }
  c->tau_d = eta_next * p.inv_om;
  c->sigma_d = eta_next * p.om;
  c->w_d = accept ? p.w_acc : 0.0;
  c->w1_d = accept ? 1.0 - p.w_acc : 1.0;
  c->avg_on = accept ? 1 : 0;
  c->k = k1;
  c->eta_used = p.eta;
  c->eta = eta_next;
  c->copy_lr = 0;
  if (accept) {
    const int t = c->ix_cur;
    c->ix_cur = c->ix_next;
    c->ix_next = t;
    c->aty_valid = 0;
    c->wsum = p.wsum_new;
    c->avg_w = p.w_acc;
    c->accepted++;
  } else {
    c->aty_valid = 1;
    c->avg_w = 0.0;
    c->rejected++;
  }
}

// FP32 mode: no FP64 instruction; eta and wsum live in their FP32 copies until
// the next check
template <>
__device__ void step_control<float>(Control* c, const StepPre& p, float dx2, float dy2, float inter,
                                    double* trace, int cap) {
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(inter)) {
    c->done = 1;
    c->status = SCYLLA_NUMERICAL;
    sync_step_state(c);
    return;
  }
  bool accept = true;
  float eta_next = p.eta_f;
  float eta_max = pos_inf<float>();
  if (p.adaptive) {
    const float mv = p.om_f * dx2 + dy2 * p.iom_f;
    eta_max = inter != 0.0f ? mv / (2.0f * fabsf(inter)) : pos_inf<float>();
    eta_next = fminf(p.fr_f * eta_max, p.fg_f * p.eta_f);
    accept = p.eta_f <= eta_max;
  }
  const long long k1 = p.k1;
  if (trace && k1 <= cap) {
    double* t = trace + 4 * (k1 - 1);
    t[0] = double(p.eta_f);
    t[1] = double(eta_max);
    t[2] = accept ? 1.0 : 0.0;
    t[3] = double(eta_next);
  }
  c->tau_f = eta_next * p.iom_f;
  c->sigma_f = eta_next * p.om_f;
  c->w_f = accept ? p.w_acc_f : 0.0f;
  c->w1_f = accept ? 1.0f - p.w_acc_f : 1.0f;
  c->avg_on = accept ? 1 : 0;
  c->eta_f = eta_next;
  c->fr_f = p.fr_next;
  c->fg_f = p.fg_next;
  c->k = k1;
  c->copy_lr = 0;
  if (accept) {
    const int t = c->ix_cur;
    c->ix_cur = c->ix_next;
    c->ix_next = t;
    c->aty_valid = 0;
    c->wsum_f = p.wsum_new_f;
    c->accepted++;
  } else {
    c->aty_valid = 1;
    c->rejected++;
  }
}

// the whole decision at once (control kernels of the batched and fan-out solves)
static __device__ void step_control(Control* c, double dx2, double dy2, double inter, const double* fac, int n_check,
                                    double* trace, int cap) {
  const StepPre p = step_pre<double>(c, fac, n_check);
  step_control<double>(c, p, dx2, dy2, inter, trace, cap);
}

// step-size factor table for attempts k+1 .. k+n_check (by the whole last block):
// 2 n_check FP64 values, then 2 n_check FP32 values; attempt k+1's FP32 factors also
// go to the control block.  The FP32-mixed mode needs only the FP32 table, from
// powf; the FP64 mode computes one FP64 power per thread (each is a long serial
// chain on this part) and rounds it for the FP32 copy.
template <typename T>
static __device__ void fill_step_factors(Control* c, double* fac, int n_check);

template <>
__device__ void fill_step_factors<float>(Control* c, double* fac, int n_check) {
  const long long k = c->k;
  const float er = float(c->exp_red), eg = float(c->exp_grow);
  float* facf = reinterpret_cast<float*>(fac + 2 * n_check);
  for (int i = threadIdx.x; i < n_check; i += blockDim.x) {
    const float kk = float(k + 1 + i + 1);
    const float fr = 1.0f - powf(kk, -er), fg = 1.0f + powf(kk, -eg);
    facf[2 * i] = fr;
    facf[2 * i + 1] = fg;
    if (i == 0) {
      c->fr_f = fr;
      c->fg_f = fg;
    }
  }
  if (threadIdx.x == 0) c->k_fac = k;
}

template <>
__device__ void fill_step_factors<double>(Control* c, double* fac, int n_check) {
  const long long k = c->k;
  float* facf = reinterpret_cast<float*>(fac + 2 * n_check);
  for (int q = threadIdx.x; q < 2 * n_check; q += blockDim.x) {
    const double kk = double(k + 1 + (q >> 1) + 1);
    const double v = (q & 1) ? 1.0 + pow(kk, -c->exp_grow) : 1.0 - pow(kk, -c->exp_red);
    fac[q] = v;
    facf[q] = float(v);
    if (q == 0) c->fr_f = float(v);
    if (q == 1) c->fg_f = float(v);
  }
  if (threadIdx.x == 0) c->k_fac = k;
}

// ------------------------------------------------------------------ checks ---
struct Eval {
  double rp_s2, rd_s2, rp2, rd2, pobj, dobj, dx2, dy2;
  double eps_p, eps_d, eps_g, rel;
};

__device__ __forceinline__ double weighted_kkt(const Eval& e, double om) {
  const double g = e.pobj - e.dobj;
  return sqrt(om * om * e.rp_s2 + e.rd_s2 / (om * om) + g * g);
}

static __device__ void finish(Control* c, int status, bool out_avg, const Eval& e) {
  c->done = 1;
  c->status = status;
  c->used_avg = out_avg ? 1 : 0;
  c->eps_p = e.eps_p;
  c->eps_d = e.eps_d;
  c->eps_g = e.eps_g;
  c->rel_kkt = e.rel;
  c->pobj = e.pobj;
  c->dobj = e.dobj;
  if (out_avg) {
    int t = c->ix_cur;
    c->ix_cur = c->ix_avg;
    c->ix_avg = t;
    t = c->ia_cur;
    c->ia_cur = c->ia_avg;
    c->ia_avg = t;
  }
}

// Evaluation q (0: current point, 1: averaged point) of a check from the 18 reduced
// sums of the two check kernels: relative KKT parts (Section 2.2) and the quantities
// the restart rule needs.
__device__ __forceinline__ Eval make_eval(const Control* c, const double* r, int q) {
  Eval e;
  const double* cs = r + 5 * q;
  const double* rs = r + kNC1 + 4 * q;
  e.rd_s2 = cs[0];
  e.rd2 = cs[1];
  e.pobj = cs[2] + c->offset;
  e.dobj = (rs[2] + cs[3]) + c->offset;
  e.dx2 = cs[4];
  e.rp_s2 = rs[0];
  e.rp2 = rs[1];
  e.dy2 = rs[3];
  e.eps_p = sqrt(e.rp2) / (1.0 + c->bnorm);
  e.eps_d = sqrt(e.rd2) / (1.0 + c->cnorm);
  e.eps_g = fabs(e.pobj - e.dobj) / (1.0 + fabs(e.pobj) + fabs(e.dobj));
  e.rel = fmax(e.eps_p, fmax(e.eps_d, e.eps_g));
  return e;
}

// Termination (Section 2.2), stalling (Algorithm 1) and restarts (PDLP) from the two
// evaluations and their weighted KKT errors wk[q] at the current primal weight.
static __device__ void check_control_impl(Control* c, const Eval* e, const double* wk, double* trace, int cap) {
  const unsigned long long h = c->hash_accum;
  c->hash_accum = 0ULL;
  c->aty_valid = 1;
  const bool inf_tested = c->inf_tested != 0;  // a candidate dual ray was tested at this check
  c->inf_tested = 0;
  if (c->initial) {
    c->initial = 0;
    c->avg_w = 0.0;
    const double kc = wk[0];
    c->kkt_lr = kc;
    c->kkt_prev = kc;
    c->k_lr = 0;
    c->copy_lr = 1;
    c->last_hash = h;
    c->same_hash = 0;
    c->eps_p = e[0].eps_p; c->eps_d = e[0].eps_d; c->eps_g = e[0].eps_g;
    c->rel_kkt = e[0].rel; c->pobj = e[0].pobj; c->dobj = e[0].dobj;
    if (isnan(e[0].rel)) finish(c, SCYLLA_NUMERICAL, false, e[0]);
    else if (e[0].rel <= c->tol) finish(c, SCYLLA_CONVERGED, false, e[0]);
    else if (c->iter_limit <= 0) finish(c, SCYLLA_ITER_LIMIT, false, e[0]);
    return;
  }
  const bool has_avg = c->wsum > 0.0;
  c->avg_w = 0.0;
  const bool out_avg = has_avg && e[1].rel < e[0].rel;
  const Eval& eo = out_avg ? e[1] : e[0];
  c->eps_p = eo.eps_p; c->eps_d = eo.eps_d; c->eps_g = eo.eps_g;
  c->rel_kkt = eo.rel; c->pobj = eo.pobj; c->dobj = eo.dobj;
  if (isnan(e[0].rel)) { finish(c, SCYLLA_NUMERICAL, false, e[0]); return; }
  if (eo.rel <= c->tol) { finish(c, SCYLLA_CONVERGED, out_avg, eo); return; }
  if (c->k >= c->iter_limit) { finish(c, SCYLLA_ITER_LIMIT, out_avg, eo); return; }
  c->same_hash = (h == c->last_hash) ? c->same_hash + 1 : 0;
  c->last_hash = h;
  if (c->stall_checks > 0 && c->same_hash >= c->stall_checks) { finish(c, SCYLLA_STALLED, out_avg, eo); return; }
  // the ray proves the LP infeasible (weak duality; the margin is far above the
  // rounding of D, which is <= 0 on every feasible LP)
  if (inf_tested && c->inf_gap > kInfeasMargin * c->inf_scale) { finish(c, SCYLLA_INFEASIBLE, out_avg, eo); return; }
  if (!c->restarts_on) return;
  const double om = c->omega;
  const double kc_cur = wk[0];
  const bool cand_avg = has_avg && wk[1] < kc_cur;
  const Eval& ec = cand_avg ? e[1] : e[0];
  const double kc = cand_avg ? wk[1] : wk[0];
  const bool restart = kc <= c->beta_s * c->kkt_lr || (kc <= c->beta_n * c->kkt_lr && kc > c->kkt_prev) ||
                       double(c->k - c->k_lr) >= c->beta_a * double(c->k);
  double* rec = nullptr;
  if (trace && c->n_ctrace < cap) {
    rec = trace + 5 * c->n_ctrace;
    c->n_ctrace++;
    rec[0] = double(c->k);
    rec[1] = restart ? 1.0 : 0.0;
    rec[2] = cand_avg ? 1.0 : 0.0;
    rec[3] = c->omega;
    rec[4] = kc;
  }
  if (!restart) {
    c->kkt_prev = kc;
    return;
  }
  c->restarts++;
  if (c->pw_update) {
    // omega' = exp(theta log(ddy / ddx) + (1 - theta) log omega); for theta = 1/2 this
    // is sqrt((ddy / ddx) omega), without the slow FP64 logarithms and exponential
    const double ddx = sqrt(ec.dx2), ddy = sqrt(ec.dy2);
    if (ddx > 1e-10 && ddy > 1e-10) {
      if (c->theta == 0.5) c->omega = sqrt((ddy / ddx) * om);
      else c->omega = exp(c->theta * log(ddy / ddx) + (1.0 - c->theta) * log(om));
    }
  }
  if (cand_avg) {
    int t = c->ix_cur;
    c->ix_cur = c->ix_avg;
    c->ix_avg = t;
    t = c->ia_cur;
    c->ia_cur = c->ia_avg;
    c->ia_avg = t;
  }
  c->k_lr = c->k;
  c->wsum = 0.0;
  c->copy_lr = 1;
  c->kkt_lr = c->omega == om ? kc : weighted_kkt(ec, c->omega);
  c->kkt_prev = c->kkt_lr;
  if (rec) rec[3] = c->omega;
}

// single-thread form (control kernels of the batched and fan-out solves)
static __device__ void check_control(Control* c, const double* r, double* trace, int cap) {
  const Eval e[2] = {make_eval(c, r, 0), make_eval(c, r, 1)};
  const double wk[2] = {weighted_kkt(e[0], c->omega), weighted_kkt(e[1], c->omega)};
  check_control_impl(c, e, wk, trace, cap);
  derive_steps(c);
}

// warp form: lanes 0 and 1 evaluate the two points side by side (their square roots
// and divisions are long FP64 chains), lane 0 decides.  Called by a whole warp.
// The control block is worked on in a shared-memory copy that the warp loads and
// stores with coalesced word accesses (the decision logic's many field accesses
// are then shared-memory ones).
static __device__ void check_control_warp(Control* c, const double* r, double* trace, int cap) {
  __shared__ Eval se[2];
  __shared__ double swk[2];
  __shared__ Control sc;
  static_assert(sizeof(Control) % 4 == 0, "word copy");
  const int lane = threadIdx.x & 31;
  constexpr int kWords = int(sizeof(Control) / 4);
  for (int i = lane; i < kWords; i += 32) reinterpret_cast<int*>(&sc)[i] = reinterpret_cast<const int*>(c)[i];
  __syncwarp();
  if (lane < 2) {
    const Eval e = make_eval(&sc, r, lane);
    se[lane] = e;
    swk[lane] = weighted_kkt(e, sc.omega);
  }
  __syncwarp();
  if (lane == 0) {
    check_control_impl(&sc, se, swk, trace, cap);
    derive_steps(&sc);
  }
  __syncwarp();
  for (int i = lane; i < kWords; i += 32) reinterpret_cast<int*>(c)[i] = reinterpret_cast<const int*>(&sc)[i];
  __syncwarp();
}

// per-thread accumulator type of the bulk kernels
template <typename T>
struct AccOf {
  typedef T type;
};

// flags of a per-LP / per-objective slot
constexpr int kSlotActive = 1, kSlotCopyLr = 2, kSlotCached = 4, kSlotAvg = 8, kSlotCheck = 16;

template <typename T>
__device__ __forceinline__ void write_slot(BatchSlot<T>* s, const Control* c) {
  BatchSlot<T> v;
  v.tau = T(c->eta / c->omega);
  v.sigma = T(c->eta * c->omega);
  v.w = T(c->avg_w);
  v.w1 = T(1.0 - c->avg_w);
  v.cur = c->ix_cur;
  v.nxt = c->ix_next;
  v.avg = c->ix_avg;
  v.ia_cur = c->ia_cur;
  v.ia_avg = c->ia_avg;
  int f = 0;
  if (!c->done && c->k < c->iter_limit) f |= kSlotActive;
  if (!c->done) f |= kSlotCheck;
  if (c->copy_lr) f |= kSlotCopyLr;
  if (c->aty_valid) f |= kSlotCached;
  if (c->avg_w > 0.0) f |= kSlotAvg;
  v.flags = f;
  *s = v;
}


}  // namespace scylla
