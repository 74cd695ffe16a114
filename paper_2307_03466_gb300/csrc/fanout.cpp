// Host side of the K-objective fan-out (scylla_fanout_* of scylla.h): K pump
// objectives of one LP (Section 2.4 objective update around K rounding targets)
// solved together by the SpMM kernels of fanout.cu, which share the base LP
// handle's device matrices, bounds and scaling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "lp_handle.h"

using namespace scylla;

#define CKF(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? SCYLLA_ERR_OOM : SCYLLA_ERR_CUDA;          \
    }                                                                                     \
  } while (0)

struct scylla_fanout {
  scylla_lp* lp = nullptr;
  int K = 0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<Control> ctl0;
  Control* h_ctl = nullptr;
  int* h_done = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_chunk[2] = {nullptr, nullptr};
  DevFan<double> f64{};
  DevFan<float> f32{};
  double* io = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float last_ms = 0.f;
  // the autotuner's measurements: ms per launch of the primal SpMM in tile shapes
  // 1..4, then of the dual SpMM (0 where a shape was not timed)
  double tune_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  void* pools = nullptr;  // the iterate pools (X, Y, AX, ATY, XLR, YLR), contiguous in the arena
  size_t pools_bytes = 0;

  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    if (arena) cudaFree(arena);
    arena = nullptr;
    if (h_ctl) cudaFreeHost(h_ctl);
    h_ctl = nullptr;
    if (h_done) cudaFreeHost(h_done);
    h_done = nullptr;
    for (cudaEvent_t* e : {&ev0, &ev1, &ev_chunk[0], &ev_chunk[1]}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
  }
};

namespace {

template <typename T>
int seed_state(scylla_fanout* f, DevFan<T>& F) {
  scylla_lp* lp = f->lp;
  cudaStream_t st = lp->st;
  CKF(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  const Control base = *lp->h_ctl;
  for (int k = 0; k < f->K; ++k) {
    Control& c = f->ctl0[k];
    c.eta = base.eta;
    c.omega = base.omega;
  }
  CKF(cudaMemcpyAsync(F.ctl, f->ctl0.data(), sizeof(Control) * f->K, cudaMemcpyHostToDevice, st));
  CKF(launch_fan_seed<T>(F, lp->X[base.ix_cur], lp->Y[base.ix_cur], st));
  CKF(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

template <typename T>
int fan_solve_impl(scylla_fanout* f, DevFan<T>& F, double tol, int64_t iter_limit) {
  scylla_lp* lp = f->lp;
  cudaStream_t st = lp->st;
  const long long nchk = lp->p.n_check;
  const long long max_chunks = (iter_limit + nchk - 1) / nchk + 2;
  CKF(cudaEventRecord(f->ev0, st));
  CKF(launch_fan_init<T>(F, tol, (long long)iter_limit, lp->p.stall_checks, st));
  CKF(launch_fan_check<T>(F, st));
  if (!f->exec) {
    CKF(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < lp->p.n_check && e == cudaSuccess; ++s) e = launch_fan_slot<T>(F, st);
    if (e == cudaSuccess) e = launch_fan_check<T>(F, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    CKF(e);
    CKF(e2);
    f->graph = g;
    CKF(cudaGraphInstantiate(&f->exec, g, 0));
  }
  auto enqueue = [&](long long c) -> cudaError_t {
    cudaError_t e = cudaGraphLaunch(f->exec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f->h_done[c & 1], F.n_done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(f->ev_chunk[c & 1], st);
    return e;
  };
  CKF(cudaMemcpyAsync(&f->h_done[1], F.n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  if (f->h_done[1] < f->K) {
    CKF(enqueue(0));
    for (long long c = 0; c < max_chunks; ++c) {
      if (c + 1 < max_chunks) CKF(enqueue(c + 1));
      CKF(cudaEventSynchronize(f->ev_chunk[c & 1]));
      if (f->h_done[c & 1] >= f->K) break;
    }
  }
  CKF(cudaEventRecord(f->ev1, st));
  CKF(cudaMemcpyAsync(f->h_ctl, F.ctl, sizeof(Control) * f->K, cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  cudaEventElapsedTime(&f->last_ms, f->ev0, f->ev1);
  return SCYLLA_OK;
}

// Tile-shape autotuner of the fan-out: for each SpMM (primal, dual) every valid tile
// shape (objectives per lane VEC, slots per sweep CHUNK; so 32 VEC / CHUNK rows per
// warp and 64 / CHUNK sweeps over the matrix) is timed on this fan-out's own matrix
// and the fastest kept; shape 1..4 forces one instead (0: time them all).  Every
// shape gives identical results (the same per-objective sums in the same order).
// The timed launches run from the seeded state, which is zeroed and seeded again
// afterwards.
template <typename T>
int fan_tune(scylla_fanout* f, DevFan<T>& F, int shape_p, int shape_d) {
  cudaStream_t st = f->lp->st;
  for (int side = 0; side < 2; ++side) {
    const int forced = side == 0 ? shape_p : shape_d;
    for (int q = 0; q < 4; ++q) f->tune_ms[4 * side + q] = 0.0;
    if (forced != 0) {
      (side == 0 ? F.shape_p : F.shape_d) = forced;
      continue;
    }
    CKF(launch_fan_init<T>(F, 0.0, 1LL << 40, 0, st));
    CKF(launch_fan_check<T>(F, st));
    double best = 0.0;
    int best_shape = 0;
    for (int shape = 1; shape <= 4; ++shape) {
      if (!fan_shape_valid<T>(shape)) continue;
      (side == 0 ? F.shape_p : F.shape_d) = shape;
      fan_grids<T>(F);
      CKF(launch_fan_part<T>(F, side, st));  // warm-up
      CKF(cudaEventRecord(f->ev0, st));
      for (int r = 0; r < 3; ++r) CKF(launch_fan_part<T>(F, side, st));
      CKF(cudaEventRecord(f->ev1, st));
      CKF(cudaEventSynchronize(f->ev1));
      float ms = 0.f;
      CKF(cudaEventElapsedTime(&ms, f->ev0, f->ev1));
      const double per = double(ms) / 3.0;
      f->tune_ms[4 * side + shape - 1] = per;
      if (best_shape == 0 || per < best) {
        best = per;
        best_shape = shape;
      }
    }
    (side == 0 ? F.shape_p : F.shape_d) = best_shape;
  }
  fan_grids<T>(F);
  if (f->exec) {  // the captured graph holds the old launch configuration
    cudaGraphExecDestroy(f->exec);
    cudaGraphDestroy(f->graph);
    f->exec = nullptr;
    f->graph = nullptr;
  }
  CKF(cudaMemsetAsync(f->pools, 0, f->pools_bytes, st));
  return seed_state<T>(f, F);
}

int create_fan(scylla_lp* lp, int K, const double* targets, int round_K, scylla_fanout* f) {
  f->lp = lp;
  f->K = K;
  const bool mixed = lp->p.precision == SCYLLA_PREC_MIXED;
  const int n = lp->n, m = lp->m;
  const int64_t n0 = lp->n0;
  for (cudaEvent_t* e : {&f->ev0, &f->ev1}) CKF(cudaEventCreate(e));
  for (int q = 0; q < 2; ++q) CKF(cudaEventCreateWithFlags(&f->ev_chunk[q], cudaEventDisableTiming));
  CKF(cudaMallocHost(&f->h_done, 2 * sizeof(int)));
  CKF(cudaMallocHost(&f->h_ctl, sizeof(Control) * K));
  // the objective of target k (Section 2.4, round round_K): c_hat = t c + om g_k
  const double aK = std::pow(lp->p.alpha, double(round_K));
  const double s = lp->c0norm > 0.0 ? std::sqrt(double(lp->n_int)) / lp->c0norm : 0.0;
  const double t = aK * s, om = 1.0 - aK;
  std::vector<unsigned long long> lo_bits(n, 0ULL), up_bits(n, 0ULL);
  std::vector<double> offset(K, 0.0), cn2(K, 0.0);
  for (int k = 0; k < K; ++k) {
    const double* x = targets + size_t(k) * n0;
    for (int64_t j = 0; j < n0; ++j) {
      double g = 0.0;
      if (lp->int0[j]) {
        if (x[j] == lp->l0[j]) {
          lo_bits[j] |= 1ULL << k;
          g = 1.0;
          offset[k] -= om * lp->l0[j];
        } else if (x[j] == lp->u0[j]) {
          up_bits[j] |= 1ULL << k;
          g = -1.0;
          offset[k] += om * lp->u0[j];
        }
      }
      const double ch = t * lp->c0[j] + om * g;
      cn2[k] += ch * ch;
    }
  }
  // arena
  const size_t vs = mixed ? sizeof(float) : sizeof(double);
  char *X[3], *Y[3], *AX[3], *ATY[2], *XLR, *YLR;
  unsigned long long *lob, *upb;
  float2* cw;
  double* cc64;
  Control* ctl;
  void* slot;
  FanState* state;
  double *pp, *pd, *pc1, *pc2, *fac;
  int* n_done;
  long long* kglob;
  DevFan<double> g64{};
  DevFan<float> g32{};
  if (mixed) {
    g32.d = lp->d32;
    g32.K = K;
    g32.shape_p = g32.shape_d = 1;
    fan_grids<float>(g32);
  } else {
    g64.d = lp->d64;
    g64.K = K;
    g64.shape_p = g64.shape_d = 2;
    fan_grids<double>(g64);
  }
  // the block partial arrays hold the largest grid of any tile shape
  int gp = mixed ? g32.grid_p : g64.grid_p, gd = mixed ? g32.grid_d : g64.grid_d;
  for (int shape = 1; shape <= 4; ++shape) {
    if (mixed) {
      DevFan<float> t = g32;
      t.shape_p = t.shape_d = shape;
      fan_grids<float>(t);
      gp = std::max(gp, t.grid_p);
      gd = std::max(gd, t.grid_d);
    } else if (fan_shape_valid<double>(shape)) {
      DevFan<double> t = g64;
      t.shape_p = t.shape_d = shape;
      fan_grids<double>(t);
      gp = std::max(gp, t.grid_p);
      gd = std::max(gd, t.grid_d);
    }
  }
  const int gc1 = mixed ? g32.grid_c1 : g64.grid_c1, gc2 = mixed ? g32.grid_c2 : g64.grid_c2;
  const size_t nk = size_t(n) * kFanMaxK, mk = size_t(m) * kFanMaxK;
  for (int pass = 0; pass < 2; ++pass) {
    Arena ar;
    if (pass == 1) {
      CKF(cudaMalloc(&f->arena, f->arena_bytes));
      ar.base = static_cast<char*>(f->arena);
    }
    for (int q = 0; q < 3; ++q) {
      X[q] = ar.take<char>(vs * nk);
      Y[q] = ar.take<char>(vs * mk);
      AX[q] = ar.take<char>(vs * mk);
    }
    for (int q = 0; q < 2; ++q) ATY[q] = ar.take<char>(vs * nk);
    XLR = ar.take<char>(vs * nk);
    YLR = ar.take<char>(vs * mk);
    cw = ar.take<float2>(n);
    cc64 = ar.take<double>(3 * size_t(n));
    lob = ar.take<unsigned long long>(n);
    upb = ar.take<unsigned long long>(n);
    ctl = ar.take<Control>(K);
    slot = ar.take<char>(sizeof(FanSlot<double>) * K);
    state = ar.take<FanState>(1);
    pp = ar.take<double>(size_t(gp) * 1 * kFanMaxK);
    pd = ar.take<double>(size_t(gd) * 2 * kFanMaxK);
    pc1 = ar.take<double>(size_t(gc1) * kNC1 * kFanMaxK);
    pc2 = ar.take<double>(size_t(gc2) * kNC2 * kFanMaxK);
    fac = ar.take<double>(3 * size_t(lp->p.n_check));  // FP64 factor pairs, then FP32 pairs
    n_done = ar.take<int>(1);
    kglob = ar.take<long long>(1);
    f->io = ar.take<double>(n > m ? n : m);
    if (pass == 0) f->arena_bytes = ar.off + 256;
  }
  cudaStream_t st = lp->st;
  CKF(cudaMemsetAsync(f->arena, 0, f->arena_bytes, st));
  CKF(cudaMemcpyAsync(lob, lo_bits.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st));
  CKF(cudaMemcpyAsync(upb, up_bits.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st));
  CKF(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  const Control base = *lp->h_ctl;
  f->ctl0.assign(K, Control{});
  for (int k = 0; k < K; ++k) {
    Control& c = f->ctl0[k];
    c.eta = base.eta;
    c.omega = base.omega;
    c.ix_cur = 0; c.ix_next = 1; c.ix_avg = 2; c.ia_cur = 0; c.ia_avg = 1;
    c.adaptive = base.adaptive; c.restarts_on = base.restarts_on; c.pw_update = base.pw_update;
    c.beta_s = base.beta_s; c.beta_n = base.beta_n; c.beta_a = base.beta_a;
    c.theta = base.theta; c.exp_red = base.exp_red; c.exp_grow = base.exp_grow;
    c.bnorm = base.bnorm;
    c.cnorm = std::sqrt(cn2[k]);
    c.offset = offset[k];
    c.done = 1;
  }
  auto fill = [&](auto& F, auto tag) {
    using TT = decltype(tag);
    for (int q = 0; q < 3; ++q) {
      F.X[q] = reinterpret_cast<TT*>(X[q]);
      F.Y[q] = reinterpret_cast<TT*>(Y[q]);
      F.AX[q] = reinterpret_cast<TT*>(AX[q]);
    }
    for (int q = 0; q < 2; ++q) F.ATY[q] = reinterpret_cast<TT*>(ATY[q]);
    F.XLR = reinterpret_cast<TT*>(XLR);
    F.YLR = reinterpret_cast<TT*>(YLR);
    F.c_orig = lp->c_orig;
    F.lo_bits = lob;
    F.up_bits = upb;
    F.cw = cw;
    F.cc64 = cc64;
    F.t = t;
    F.om = om;
    F.ctl = ctl;
    F.slot = static_cast<FanSlot<TT>*>(slot);
    F.state = state;
    F.part_p = pp;
    F.part_d = pd;
    F.part_c1 = pc1;
    F.part_c2 = pc2;
    F.n_done = n_done;
    F.kglob = kglob;
    F.exp_red = lp->p.step_reduction_exp;
    F.exp_grow = lp->p.step_growth_exp;
    F.d.step_fac = fac;  // the fan-out's own factor table
  };
  f->pools = X[0];
  f->pools_bytes = size_t(YLR + vs * mk - X[0]);
  if (mixed) {
    fill(g32, float{});
    f->f32 = g32;
    CKF(launch_fan_cw<float>(f->f32, cw, cc64, st));
    const int rc = seed_state<float>(f, f->f32);
    return rc != SCYLLA_OK ? rc : fan_tune<float>(f, f->f32, 0, 0);
  }
  fill(g64, double{});
  f->f64 = g64;
  CKF(launch_fan_cw<double>(f->f64, nullptr, cc64, st));
  const int rc = seed_state<double>(f, f->f64);
  return rc != SCYLLA_OK ? rc : fan_tune<double>(f, f->f64, 0, 0);
}

}  // namespace

extern "C" int scylla_fanout_create(scylla_lp* lp, int32_t K, const double* targets, int32_t round_K,
                                    scylla_fanout** out) {
  if (!out) {
    set_error("out is null");
    return SCYLLA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!lp || !targets || K < 1 || K > kFanMaxK || round_K < 1) {
    set_error("need a handle, targets, 1 <= K <= 64 and round >= 1");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (lp->qp_active || lp->p.distance == 2) {
    set_error("the fan-out takes LP objectives (no quadratic objective, distance = 1)");
    return SCYLLA_ERR_UNSUPPORTED;
  }
  if (lp->n_aux != 0) {
    set_error("the fan-out needs an LP without auxiliary distance columns (create it with aux_general_integers = 0)");
    return SCYLLA_ERR_UNSUPPORTED;
  }
  const int rv = lp->ensure_host_vectors();
  if (rv != SCYLLA_OK) return rv;
  for (int k = 0; k < K; ++k)
    for (int64_t j = 0; j < lp->n0; ++j) {
      const double v = targets[size_t(k) * lp->n0 + j];
      if (!std::isfinite(v) || (lp->int0[j] && (v != std::floor(v) || v < lp->l0[j] || v > lp->u0[j]))) {
        set_error("target " + std::to_string(k) + " not integral within bounds at column " + std::to_string(j));
        return SCYLLA_ERR_INVALID_ARG;
      }
    }
  scylla_fanout* f = nullptr;
  int rc = SCYLLA_OK;
  try {
    f = new scylla_fanout();
    rc = create_fan(lp, K, targets, round_K, f);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    rc = SCYLLA_ERR_OOM;
  }
  if (rc != SCYLLA_OK) {
    if (f) {
      f->release();
      delete f;
    }
    return rc;
  }
  *out = f;
  return SCYLLA_OK;
}

extern "C" void scylla_fanout_destroy(scylla_fanout* f) {
  if (!f) return;
  cudaStreamSynchronize(f->lp->st);
  f->release();
  delete f;
}

extern "C" int scylla_fanout_solve(scylla_fanout* f, double tol, int64_t iter_limit, scylla_pdhg_result* results,
                                   double* seconds) {
  if (!f || !results || !(tol >= 0.0) || iter_limit < 0) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const bool mixed = f->lp->p.precision == SCYLLA_PREC_MIXED;
  const int rc = mixed ? fan_solve_impl<float>(f, f->f32, tol, iter_limit)
                       : fan_solve_impl<double>(f, f->f64, tol, iter_limit);
  if (rc != SCYLLA_OK) return rc;
  for (int k = 0; k < f->K; ++k) {
    const Control& c = f->h_ctl[k];
    scylla_pdhg_result& r = results[k];
    std::memset(&r, 0, sizeof(r));
    r.status = c.status;
    r.used_average = c.used_avg;
    r.iterations = c.k;
    r.accepted = c.accepted;
    r.rejected = c.rejected;
    r.restarts = c.restarts;
    r.eps_p = c.eps_p;
    r.eps_d = c.eps_d;
    r.eps_g = c.eps_g;
    r.rel_kkt = c.rel_kkt;
    r.pobj = c.pobj;
    r.dobj = c.dobj;
    r.eta = c.eta;
    r.omega = c.omega;
    r.seconds = f->last_ms * 1e-3;
  }
  if (seconds) *seconds = f->last_ms * 1e-3;
  return SCYLLA_OK;
}

namespace {
// the fan-out's kernels as separate launches with CUDA events around each (see
// scylla_fanout_time_kernels)
template <typename T>
int fan_time_impl(scylla_fanout* f, DevFan<T>& F, int attempts, double* ms) {
  scylla_lp* lp = f->lp;
  cudaStream_t st = lp->st;
  const int nchk = lp->p.n_check;
  std::vector<std::pair<int, cudaEvent_t>> marks;  // (part, start); its end is the next entry's event
  std::vector<cudaEvent_t> evs;
  auto mark = [&](int part) -> cudaError_t {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    evs.push_back(e0);
    evs.push_back(e1);
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_fan_part<T>(F, part, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    marks.push_back({part, e0});
    return e;
  };
  cudaError_t e = launch_fan_init<T>(F, 0.0, (long long)attempts + 1, 0, st);
  if (e == cudaSuccess) e = launch_fan_check<T>(F, st);
  for (int a = 0; a < attempts && e == cudaSuccess; ++a) {
    for (int part = 0; part < 3 && e == cudaSuccess; ++part) e = mark(part);
    if ((a + 1) % nchk == 0)
      for (int part = 3; part < 6 && e == cudaSuccess; ++part) e = mark(part);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  double sum[6] = {0, 0, 0, 0, 0, 0};
  int cnt[6] = {0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess)
    for (size_t i = 0; i < marks.size(); ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, evs[2 * i], evs[2 * i + 1]);
      sum[marks[i].first] += t;
      cnt[marks[i].first]++;
    }
  for (cudaEvent_t x : evs) cudaEventDestroy(x);
  CKF(e);
  for (int k = 0; k < 6; ++k) ms[k] = cnt[k] ? sum[k] / cnt[k] : 0.0;
  return SCYLLA_OK;
}
}  // namespace

extern "C" int scylla_fanout_time_kernels(scylla_fanout* f, int32_t attempts, double* ms) {
  if (!f || !ms || attempts < 1) {
    set_error("need a fan-out, ms[6] and attempts >= 1");
    return SCYLLA_ERR_INVALID_ARG;
  }
  return f->lp->p.precision == SCYLLA_PREC_MIXED ? fan_time_impl<float>(f, f->f32, attempts, ms)
                                                 : fan_time_impl<double>(f, f->f64, attempts, ms);
}

extern "C" int scylla_fanout_tune(scylla_fanout* f, int32_t shape_primal, int32_t shape_dual) {
  if (!f) {
    set_error("null fan-out");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const bool mixed = f->lp->p.precision == SCYLLA_PREC_MIXED;
  for (const int s : {shape_primal, shape_dual})
    if (s != 0 && !(mixed ? fan_shape_valid<float>(s) : fan_shape_valid<double>(s))) {
      set_error("tile shape must be 0 (time all) or 1..4 (FP64: 2 or 4)");
      return SCYLLA_ERR_INVALID_ARG;
    }
  return mixed ? fan_tune<float>(f, f->f32, shape_primal, shape_dual)
               : fan_tune<double>(f, f->f64, shape_primal, shape_dual);
}

extern "C" int scylla_fanout_info(const scylla_fanout* f, int32_t* shape_primal, int32_t* shape_dual,
                                  double* tune_ms) {
  if (!f) {
    set_error("null fan-out");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const bool mixed = f->lp->p.precision == SCYLLA_PREC_MIXED;
  if (shape_primal) *shape_primal = mixed ? f->f32.shape_p : f->f64.shape_p;
  if (shape_dual) *shape_dual = mixed ? f->f32.shape_d : f->f64.shape_d;
  if (tune_ms)
    for (int q = 0; q < 8; ++q) tune_ms[q] = f->tune_ms[q];
  return SCYLLA_OK;
}

extern "C" int scylla_fanout_get_primal(const scylla_fanout* f, int32_t k, double* x) {
  if (!f || !x || k < 0 || k >= f->K) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  cudaStream_t st = f->lp->st;
  if (f->lp->p.precision == SCYLLA_PREC_MIXED) CKF(launch_fan_get_x<float>(f->f32, k, f->io, st));
  else CKF(launch_fan_get_x<double>(f->f64, k, f->io, st));
  CKF(cudaMemcpyAsync(x, f->io, sizeof(double) * f->lp->n0, cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

extern "C" int scylla_fanout_get_dual(const scylla_fanout* f, int32_t k, double* y) {
  if (!f || !y || k < 0 || k >= f->K) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  cudaStream_t st = f->lp->st;
  if (f->lp->p.precision == SCYLLA_PREC_MIXED) CKF(launch_fan_get_y<float>(f->f32, k, f->io, st));
  else CKF(launch_fan_get_y<double>(f->f64, k, f->io, st));
  CKF(cudaMemcpyAsync(y, f->io, sizeof(double) * f->lp->m0, cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

extern "C" int scylla_fanout_reset_state(scylla_fanout* f) {
  if (!f) {
    set_error("null handle");
    return SCYLLA_ERR_INVALID_ARG;
  }
  return f->lp->p.precision == SCYLLA_PREC_MIXED ? seed_state<float>(f, f->f32) : seed_state<double>(f, f->f64);
}
