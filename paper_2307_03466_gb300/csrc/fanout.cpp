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
  Control* ctl;
  void* slot;
  double *pp, *pd, *pc1, *pc2, *fac;
  int* n_done;
  long long* kglob;
  DevFan<double> g64{};
  DevFan<float> g32{};
  if (mixed) {
    g32.d = lp->d32;
    g32.K = K;
    fan_grids<float>(g32);
  } else {
    g64.d = lp->d64;
    g64.K = K;
    fan_grids<double>(g64);
  }
  const int gp = mixed ? g32.grid_p : g64.grid_p, gd = mixed ? g32.grid_d : g64.grid_d;
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
    lob = ar.take<unsigned long long>(n);
    upb = ar.take<unsigned long long>(n);
    ctl = ar.take<Control>(K);
    slot = ar.take<char>(sizeof(BatchSlot<double>) * K);
    pp = ar.take<double>(size_t(gp) * 1 * kFanMaxK);
    pd = ar.take<double>(size_t(gd) * 2 * kFanMaxK);
    pc1 = ar.take<double>(size_t(gc1) * kNC1 * kFanMaxK);
    pc2 = ar.take<double>(size_t(gc2) * kNC2 * kFanMaxK);
    fac = ar.take<double>(2 * size_t(lp->p.n_check));
    n_done = ar.take<int>(1);
    kglob = ar.take<long long>(1);
    f->io = ar.take<double>(n);
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
    F.t = t;
    F.om = om;
    F.ctl = ctl;
    F.slot = static_cast<BatchSlot<TT>*>(slot);
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
  if (mixed) {
    fill(g32, float{});
    f->f32 = g32;
    return seed_state<float>(f, f->f32);
  }
  fill(g64, double{});
  f->f64 = g64;
  return seed_state<double>(f, f->f64);
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

extern "C" int scylla_fanout_reset_state(scylla_fanout* f) {
  if (!f) {
    set_error("null handle");
    return SCYLLA_ERR_INVALID_ARG;
  }
  return f->lp->p.precision == SCYLLA_PREC_MIXED ? seed_state<float>(f, f->f32) : seed_state<double>(f, f->f64);
}
