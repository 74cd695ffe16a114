// Batched PDHG: many LP relaxations of uneven size solved together (the C ABI
// scylla_batch_* of scylla.h).  The LPs are stored as one block-diagonal LP; the
// kernels of kernels.cu walk a shared list of warp tiles in which no tile crosses
// an LP boundary, and every LP keeps its own control block (step size, primal
// weight, restarts, termination; Sections 2.1-2.2 of the paper per LP).  Finished
// LPs drop out: their tiles are skipped.  One CUDA graph holds n_check attempts and
// a check; a pipelined host loop replays it until every LP is done.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace scylla;

#define CKB(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? SCYLLA_ERR_OOM : SCYLLA_ERR_CUDA;          \
    }                                                                                     \
  } while (0)

struct scylla_batch {
  scylla_params p{};
  cudaStream_t st = nullptr;
  cudaStream_t user_st = nullptr;
  cudaEvent_t ev_user = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
  int* h_done = nullptr;  // pinned, two slots
  int nlp = 0;
  std::vector<int> row_off, col_off;  // per LP (nlp + 1)
  int m = 0, n = 0, nnz = 0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<Control> ctl0;  // control blocks at create (cold restart)
  Control* h_ctl = nullptr;   // pinned mirror of the control array
  double* io = nullptr;       // device staging for primal output
  DevBatch<double> b64{};
  DevBatch<float> b32{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float last_ms = 0.f;
  bool persistent = false;   // attempts in persistent launches over the work queue (batch_launch)
  // graphs whose primal / dual attempt kernels stage the next tile by asynchronous copies (FP32)
  bool async_p = false, async_d = false;
  double tune_kernel_ms[4] = {0.0, 0.0, 0.0, 0.0};  // ms per launch: primal, dual plain; primal, dual async
  // automatic choice: ms of n_check attempts in each form (graphs, persistent, graphs with asynchronous copies)
  double tune_ms[3] = {0.0, 0.0, 0.0};
  void* grid_bar = nullptr;  // the persistent launches' barrier (device)
  int* h_err = nullptr;      // pinned copy of its error flag

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
    if (h_err) cudaFreeHost(h_err);
    h_err = nullptr;
    for (cudaEvent_t* e : {&ev_user, &ev0, &ev1, &ev_chunk[0], &ev_chunk[1]}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
    if (st) cudaStreamDestroy(st);
    st = nullptr;
  }
};

namespace {

template <typename T>
void fill_batch(DevBatch<T>& B, DevLP<T>& d, scylla_batch* h, char* X[3], char* Y[3], char* AX[3], char* ATY[2],
                char* XLR, char* YLR) {
  for (int k = 0; k < 3; ++k) {
    d.X[k] = reinterpret_cast<T*>(X[k]);
    d.Y[k] = reinterpret_cast<T*>(Y[k]);
    d.AX[k] = reinterpret_cast<T*>(AX[k]);
  }
  for (int k = 0; k < 2; ++k) d.ATY[k] = reinterpret_cast<T*>(ATY[k]);
  d.XLR = reinterpret_cast<T*>(XLR);
  d.YLR = reinterpret_cast<T*>(YLR);
  B.d = d;
  B.nlp = h->nlp;
  B.exp_red = h->p.step_reduction_exp;
  B.exp_grow = h->p.step_growth_exp;
  batch_grids<T>(B);
}

// The persistent form: the start point's check and the compaction of the work
// lists, then per chunk one cooperative launch of the attempts up to the next check,
// the check kernels and the compaction, replayed by a pipelined host loop until
// every LP is done.  A barrier wait that runs out ends the solve with
// SCYLLA_ERR_TIMEOUT and the LPs still running marked SCYLLA_DEVICE_TIMEOUT.
template <typename T>
int batch_solve_persistent(scylla_batch* h, DevBatch<T>& B, double tol, int64_t iter_limit) {
  cudaStream_t st = h->st;
  const long long nchk = h->p.n_check;
  const long long max_chunks = (iter_limit + nchk - 1) / nchk + 2;
  CKB(cudaEventRecord(h->ev0, st));
  CKB(cudaMemsetAsync(h->grid_bar, 0, 16, st));
  CKB(launch_batch_init<T>(B, tol, (long long)iter_limit, h->p.stall_checks, st));
  CKB(launch_batch_queue_reset<T>(B, st));
  CKB(launch_batch_check<T>(B, st));  // every LP's start point
  CKB(launch_batch_compact<T>(B, st));
  auto enqueue = [&](long long c) -> cudaError_t {
    cudaError_t e = launch_batch_persistent<T>(B, h->grid_bar, (long long)iter_limit, h->p.device_wait_limit_s, st);
    if (e == cudaSuccess) e = launch_batch_check<T>(B, st);
    if (e == cudaSuccess) e = launch_batch_compact<T>(B, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->h_done[c & 1], B.n_done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_chunk[c & 1], st);
    return e;
  };
  CKB(cudaMemcpyAsync(&h->h_done[1], B.n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  if (h->h_done[1] < h->nlp) {
    CKB(enqueue(0));
    for (long long c = 0; c < max_chunks; ++c) {
      if (c + 1 < max_chunks) CKB(enqueue(c + 1));
      CKB(cudaEventSynchronize(h->ev_chunk[c & 1]));
      if (h->h_done[c & 1] >= h->nlp) break;
    }
  }
  CKB(cudaEventRecord(h->ev1, st));
  CKB(cudaMemcpyAsync(h->h_ctl, B.ctl, sizeof(Control) * h->nlp, cudaMemcpyDeviceToHost, st));
  // GridBar: {count, gen, err}
  CKB(cudaMemcpyAsync(h->h_err, static_cast<char*>(h->grid_bar) + 8, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  cudaEventElapsedTime(&h->last_ms, h->ev0, h->ev1);
  if (*h->h_err) {
    for (int b = 0; b < h->nlp; ++b)
      if (!h->h_ctl[b].done) {
        h->h_ctl[b].done = 1;
        h->h_ctl[b].status = SCYLLA_DEVICE_TIMEOUT;
      }
    set_error("a grid barrier wait of the persistent batched solve ran out (device_wait_limit_s)");
    return SCYLLA_ERR_TIMEOUT;
  }
  return SCYLLA_OK;
}

// the graph form's attempt kernels: asynchronous-copy tiles or not (FP32); the
// captured graph holds the launches, so it is dropped when the form changes
void set_async_tiles(scylla_batch* h, bool p, bool d) {
  if (h->async_p == p && h->async_d == d) return;
  h->async_p = p;
  h->async_d = d;
  h->b32.async_p = p ? 1 : 0;
  h->b32.async_d = d ? 1 : 0;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
}

// device ms per launch of one attempt kernel (part 0 primal, 1 dual) in the current
// tile forms, over `reps` launches after one untimed
template <typename T>
int time_batch_part(scylla_batch* h, DevBatch<T>& B, int part, int reps, double* ms) {
  cudaStream_t st = h->st;
  CKB(launch_batch_part<T>(B, part, st));
  CKB(cudaEventRecord(h->ev0, st));
  for (int r = 0; r < reps; ++r) CKB(launch_batch_part<T>(B, part, st));
  CKB(cudaEventRecord(h->ev1, st));
  CKB(cudaEventSynchronize(h->ev1));
  float t = 0.f;
  CKB(cudaEventElapsedTime(&t, h->ev0, h->ev1));
  *ms = double(t) / reps;
  return SCYLLA_OK;
}

template <typename T>
int batch_solve_impl(scylla_batch* h, DevBatch<T>& B, double tol, int64_t iter_limit) {
  if (h->persistent) return batch_solve_persistent<T>(h, B, tol, iter_limit);
  cudaStream_t st = h->st;
  const long long nchk = h->p.n_check;
  const long long max_chunks = (iter_limit + nchk - 1) / nchk + 2;
  CKB(cudaEventRecord(h->ev0, st));
  CKB(launch_batch_init<T>(B, tol, (long long)iter_limit, h->p.stall_checks, st));
  CKB(launch_batch_check<T>(B, st));  // every LP's start point
  if (!h->exec) {
    CKB(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < h->p.n_check && e == cudaSuccess; ++s) e = launch_batch_slot<T>(B, st);
    if (e == cudaSuccess) e = launch_batch_check<T>(B, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    CKB(e);
    CKB(e2);
    h->graph = g;
    CKB(cudaGraphInstantiate(&h->exec, g, 0));
  }
  auto enqueue = [&](long long c) -> cudaError_t {
    cudaError_t e = cudaGraphLaunch(h->exec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->h_done[c & 1], B.n_done, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_chunk[c & 1], st);
    return e;
  };
  // the initial check may already finish every LP
  CKB(cudaMemcpyAsync(&h->h_done[1], B.n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  if (h->h_done[1] < h->nlp) {
    CKB(enqueue(0));
    for (long long c = 0; c < max_chunks; ++c) {
      if (c + 1 < max_chunks) CKB(enqueue(c + 1));
      CKB(cudaEventSynchronize(h->ev_chunk[c & 1]));
      if (h->h_done[c & 1] >= h->nlp) break;
    }
  }
  CKB(cudaEventRecord(h->ev1, st));
  CKB(cudaMemcpyAsync(h->h_ctl, B.ctl, sizeof(Control) * h->nlp, cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  cudaEventElapsedTime(&h->last_ms, h->ev0, h->ev1);
  return SCYLLA_OK;
}

int create_batch(int32_t count, const scylla_csr* A, const double* const* c, const double* const* lo,
                 const double* const* hi, const double* const* l, const double* const* u, const scylla_params* pin,
                 void* stream, scylla_batch* h) {
  h->p = *pin;
  if (h->p.n_check < 1) {
    set_error("n_check must be >= 1");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (h->p.batch_launch < 0 || h->p.batch_launch > 3) {
    set_error("batch_launch must be 0..3");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (h->p.batch_launch == 3 && h->p.precision != SCYLLA_PREC_MIXED) {
    set_error("batch_launch = 3 (asynchronous-copy tiles) is for FP32-mixed precision");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (h->p.infeasibility_checks != 0) {
    set_error("infeasibility_checks applies to single-LP solves; a batch does not test rays");
    return SCYLLA_ERR_UNSUPPORTED;
  }
  const bool mixed = h->p.precision == SCYLLA_PREC_MIXED;
  h->nlp = count;
  h->user_st = static_cast<cudaStream_t>(stream);
  CKB(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&h->ev_user, &h->ev0, &h->ev1}) CKB(cudaEventCreate(e));
  for (int k = 0; k < 2; ++k) CKB(cudaEventCreateWithFlags(&h->ev_chunk[k], cudaEventDisableTiming));
  CKB(cudaMallocHost(&h->h_done, 2 * sizeof(int)));
  CKB(cudaMallocHost(&h->h_err, sizeof(int)));

  // ---- block-diagonal LP
  h->row_off.assign(count + 1, 0);
  h->col_off.assign(count + 1, 0);
  int64_t nnz = 0;
  for (int b = 0; b < count; ++b) {
    h->row_off[b + 1] = h->row_off[b] + int(A[b].m);
    h->col_off[b + 1] = h->col_off[b] + int(A[b].n);
    nnz += A[b].nnz;
  }
  const int m = h->row_off[count], n = h->col_off[count];
  const int64_t lim = (int64_t(1) << 31) - 64;
  if (int64_t(m) >= lim / 2 || int64_t(n) >= lim / 2 || nnz >= lim / 2) {
    set_error("batch beyond the 32-bit index range");
    return SCYLLA_ERR_UNSUPPORTED;
  }
  h->m = m;
  h->n = n;
  h->nnz = int(nnz);
  std::vector<int> rp(m + 1, 0), ci(nnz);
  std::vector<double> va(nnz), cA(n), lA(n), uA(n), loA(m), hiA(m);
  {
    int64_t q = 0;
    for (int b = 0; b < count; ++b) {
      const int r0 = h->row_off[b], c0 = h->col_off[b];
      for (int64_t i = 0; i < A[b].m; ++i) {
        for (int64_t p = A[b].rowptr[i]; p < A[b].rowptr[i + 1]; ++p, ++q) {
          ci[q] = c0 + A[b].cols[p];
          va[q] = A[b].vals[p];
        }
        rp[r0 + i + 1] = int(q);
        loA[r0 + i] = lo[b][i];
        hiA[r0 + i] = hi[b][i];
      }
      for (int64_t j = 0; j < A[b].n; ++j) {
        cA[c0 + j] = c[b][j];
        lA[c0 + j] = l[b][j];
        uA[c0 + j] = u[b][j];
      }
    }
  }
  // transpose (rows ascending within a column); block diagonal like A
  std::vector<int> tp(n + 1, 0), tr(nnz);
  std::vector<double> tv(nnz);
  for (int64_t p = 0; p < nnz; ++p) tp[ci[p] + 1]++;
  for (int j = 0; j < n; ++j) tp[j + 1] += tp[j];
  {
    std::vector<int> cur(tp.begin(), tp.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int q = cur[ci[p]]++;
        tr[q] = i;
        tv[q] = va[p];
      }
  }
  // tiles per LP, so none crosses an LP boundary
  std::vector<int2> at, tt;
  std::vector<int> alp, tlp, abeg(count + 1, 0), tbeg(count + 1, 0);
  for (int b = 0; b < count; ++b) {
    std::vector<int2> x = build_tiles_range(rp, h->row_off[b], h->row_off[b + 1]);
    abeg[b] = int(at.size());
    for (size_t q = 0; q + 1 < x.size(); ++q) {
      at.push_back(x[q]);
      alp.push_back(b);
    }
    std::vector<int2> y = build_tiles_range(tp, h->col_off[b], h->col_off[b + 1]);
    tbeg[b] = int(tt.size());
    for (size_t q = 0; q + 1 < y.size(); ++q) {
      tt.push_back(y[q]);
      tlp.push_back(b);
    }
  }
  abeg[count] = int(at.size());
  tbeg[count] = int(tt.size());
  at.push_back(make_int2(m, rp[m]));
  tt.push_back(make_int2(n, tp[n]));
  const int a_nt = int(at.size()) - 1, t_nt = int(tt.size()) - 1;
  const size_t vs = mixed ? sizeof(float) : sizeof(double);

  // ---- device arena
  DevLP<double> d64{};
  DevLP<float> d32{};
  char *X[3], *Y[3], *AX[3], *ATY[2], *XLR, *YLR;
  int *a_rowptr, *a_cols, *t_rowptr, *t_cols, *a_tlp, *t_tlp, *a_beg, *t_beg, *n_done;
  int2 *a_tiles, *t_tiles;
  double *a_vals64, *t_vals64, *c_un, *l_un, *u_un, *lo_un, *hi_un, *c64, *l64, *u64, *lo64, *hi64;
  double *R, *C, *invR, *invC, *R2, *C2, *red, *step_fac, *tp_p, *tp_d, *tp_c1, *tp_c2;
  float *a_vals32 = nullptr, *t_vals32 = nullptr, *c32 = nullptr, *l32 = nullptr, *u32 = nullptr, *lo32 = nullptr,
        *hi32 = nullptr;
  uint8_t* int_mask;
  Control* ctl;
  void* slot;
  long long* kglob;
  int *q_lps, *q_a, *q_t, *q_pre, *q_cnt;
  unsigned int *q_ctr, *lp_cnt;
  void* gbar;
  const int red_blocks = std::max(1, std::min(4 * device_sm_count(), (std::max(m, n) + kThreads - 1) / kThreads));
  for (int pass = 0; pass < 2; ++pass) {
    Arena ar;
    if (pass == 1) {
      CKB(cudaMalloc(&h->arena, h->arena_bytes));
      ar.base = static_cast<char*>(h->arena);
    }
    a_rowptr = ar.take<int>(m + 1);
    a_cols = ar.take<int>(padded_len(nnz));
    a_tiles = ar.take<int2>(at.size());
    t_rowptr = ar.take<int>(n + 1);
    t_cols = ar.take<int>(padded_len(nnz));
    t_tiles = ar.take<int2>(tt.size());
    a_tlp = ar.take<int>(a_nt);
    t_tlp = ar.take<int>(t_nt);
    a_beg = ar.take<int>(count + 1);
    t_beg = ar.take<int>(count + 1);
    a_vals64 = ar.take<double>(padded_len(nnz));
    t_vals64 = ar.take<double>(padded_len(nnz));
    if (mixed) {
      a_vals32 = ar.take<float>(padded_len(nnz));
      t_vals32 = ar.take<float>(padded_len(nnz));
      c32 = ar.take<float>(n);
      l32 = ar.take<float>(n);
      u32 = ar.take<float>(n);
      lo32 = ar.take<float>(m);
      hi32 = ar.take<float>(m);
    }
    c_un = ar.take<double>(n);
    l_un = ar.take<double>(n);
    u_un = ar.take<double>(n);
    lo_un = ar.take<double>(m);
    hi_un = ar.take<double>(m);
    c64 = ar.take<double>(n);
    l64 = ar.take<double>(n);
    u64 = ar.take<double>(n);
    lo64 = ar.take<double>(m);
    hi64 = ar.take<double>(m);
    R = ar.take<double>(m);
    C = ar.take<double>(n);
    invR = ar.take<double>(m);
    invC = ar.take<double>(n);
    R2 = ar.take<double>(std::max(m, n));
    C2 = ar.take<double>(std::max(m, n));
    red = ar.take<double>(2 * size_t(red_blocks));
    step_fac = ar.take<double>(2 * size_t(h->p.n_check));
    int_mask = ar.take<uint8_t>(n);
    for (int k = 0; k < 3; ++k) {
      X[k] = ar.take<char>(vs * n);
      Y[k] = ar.take<char>(vs * m);
      AX[k] = ar.take<char>(vs * m);
    }
    for (int k = 0; k < 2; ++k) ATY[k] = ar.take<char>(vs * n);
    XLR = ar.take<char>(vs * n);
    YLR = ar.take<char>(vs * m);
    tp_p = ar.take<double>(size_t(kNP) * t_nt);
    tp_d = ar.take<double>(size_t(kND) * a_nt);
    tp_c1 = ar.take<double>(size_t(kNC1) * t_nt);
    tp_c2 = ar.take<double>(size_t(kNC2) * a_nt);
    ctl = ar.take<Control>(count);
    slot = ar.take<char>(sizeof(BatchSlot<double>) * count);
    n_done = ar.take<int>(1);
    kglob = ar.take<long long>(1);
    q_lps = ar.take<int>(count);
    q_a = ar.take<int>(a_nt);
    q_t = ar.take<int>(t_nt);
    q_pre = ar.take<int>(2 * size_t(count + 1));
    q_cnt = ar.take<int>(4);
    q_ctr = ar.take<unsigned int>(4);
    lp_cnt = ar.take<unsigned int>(count);
    gbar = ar.take<char>(16);
    h->io = ar.take<double>(n);
    if (pass == 0) h->arena_bytes = ar.off + 256;
  }
  cudaStream_t st = h->st;
  CKB(cudaMemsetAsync(h->arena, 0, h->arena_bytes, st));
  CKB(cudaMallocHost(&h->h_ctl, sizeof(Control) * count));
  CKB(cudaMemcpyAsync(a_rowptr, rp.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(a_cols, ci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(a_tiles, at.data(), sizeof(int2) * at.size(), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_rowptr, tp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_cols, tr.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_tiles, tt.data(), sizeof(int2) * tt.size(), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(a_tlp, alp.data(), sizeof(int) * a_nt, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_tlp, tlp.data(), sizeof(int) * t_nt, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(a_beg, abeg.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_beg, tbeg.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(a_vals64, va.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(t_vals64, tv.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(c_un, cA.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(l_un, lA.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(u_un, uA.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(lo_un, loA.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
  CKB(cudaMemcpyAsync(hi_un, hiA.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
  // preconditioning of the block-diagonal LP is preconditioning of every LP
  DevSetup s{};
  s.m = m; s.n = n; s.n_orig = n; s.m_orig = m; s.nnz = int(nnz);
  s.a_rowptr = a_rowptr; s.a_cols = a_cols; s.t_rowptr = t_rowptr; s.t_cols = t_cols;
  s.a_tiles = a_tiles; s.a_ntiles = a_nt; s.t_tiles = t_tiles; s.t_ntiles = t_nt;
  s.a_vals64 = a_vals64; s.t_vals64 = t_vals64; s.a_vals32 = a_vals32; s.t_vals32 = t_vals32;
  s.R = R; s.C = C; s.R2 = R2; s.C2 = C2; s.red = red; s.red_blocks = red_blocks;
  CKB(launch_precondition(s, h->p.ruiz_iters, h->p.pock_chambolle != 0, st));
  CKB(launch_scale_values(s, st));
  DevVecs v{};
  v.c = c_un; v.lo = lo_un; v.hi = hi_un; v.l = l_un; v.u = u_un;
  v.c64 = c64; v.lo64 = lo64; v.hi64 = hi64; v.l64 = l64; v.u64 = u64;
  v.c32 = c32; v.lo32 = lo32; v.hi32 = hi32; v.l32 = l32; v.u32 = u32;
  v.R = R; v.C = C; v.invR = invR; v.invC = invC; v.m = m; v.n = n;
  CKB(launch_scale_vectors(v, st));
  // per-LP initial step size and primal weight from the scaled data, and the norms
  // of the relative KKT error from the original data
  std::vector<double> sv(nnz), sc(n), slo(m), shi(m);
  CKB(cudaMemcpyAsync(sv.data(), a_vals64, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
  CKB(cudaMemcpyAsync(sc.data(), c64, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CKB(cudaMemcpyAsync(slo.data(), lo64, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
  CKB(cudaMemcpyAsync(shi.data(), hi64, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  auto bnd = [](double a, double b) {
    const double x = std::isfinite(a) ? std::fabs(a) : 0.0, y = std::isfinite(b) ? std::fabs(b) : 0.0;
    return std::max(x, y);
  };
  h->ctl0.assign(count, Control{});
  for (int b = 0; b < count; ++b) {
    double amax = 0.0, fro2 = 0.0, cn = 0.0, qn = 0.0, cn_un = 0.0, bn_un = 0.0;
    for (int p = rp[h->row_off[b]]; p < rp[h->row_off[b + 1]]; ++p) {
      amax = std::max(amax, std::fabs(sv[p]));
      fro2 += sv[p] * sv[p];
    }
    for (int j = h->col_off[b]; j < h->col_off[b + 1]; ++j) {
      cn += sc[j] * sc[j];
      cn_un += cA[j] * cA[j];
    }
    for (int i = h->row_off[b]; i < h->row_off[b + 1]; ++i) {
      const double q = bnd(slo[i], shi[i]), qu = bnd(loA[i], hiA[i]);
      qn += q * q;
      bn_un += qu * qu;
    }
    cn = std::sqrt(cn);
    qn = std::sqrt(qn);
    Control& cb = h->ctl0[b];
    cb.eta = h->p.adaptive_step ? (amax > 0.0 ? 1.0 / amax : 1.0)
                                : (fro2 > 0.0 ? h->p.fixed_step_factor / std::sqrt(fro2) : 1.0);
    cb.omega = (cn > 0.0 && qn > 0.0) ? cn / qn : 1.0;
    cb.ix_cur = 0; cb.ix_next = 1; cb.ix_avg = 2; cb.ia_cur = 0; cb.ia_avg = 1;
    cb.adaptive = h->p.adaptive_step ? 1 : 0;
    cb.restarts_on = h->p.restarts ? 1 : 0;
    cb.pw_update = h->p.primal_weight_update ? 1 : 0;
    cb.beta_s = h->p.beta_sufficient; cb.beta_n = h->p.beta_necessary; cb.beta_a = h->p.beta_artificial;
    cb.theta = h->p.pw_smoothing; cb.exp_red = h->p.step_reduction_exp; cb.exp_grow = h->p.step_growth_exp;
    cb.cnorm = std::sqrt(cn_un);
    cb.bnorm = std::sqrt(bn_un);
    cb.offset = 0.0;
    cb.done = 1;
  }
  CKB(cudaMemcpyAsync(ctl, h->ctl0.data(), sizeof(Control) * count, cudaMemcpyHostToDevice, st));

  auto fill_common = [&](auto& d) {
    d.m = m;
    d.n = n;
    d.a_rowptr = a_rowptr; d.a_cols = a_cols; d.a_tiles = a_tiles; d.a_ntiles = a_nt;
    d.t_rowptr = t_rowptr; d.t_cols = t_cols; d.t_tiles = t_tiles; d.t_ntiles = t_nt;
    d.a_vals64 = a_vals64; d.t_vals64 = t_vals64;
    d.c64 = c64; d.l64 = l64; d.u64 = u64; d.lo64 = lo64; d.hi64 = hi64; d.R = R; d.C = C; d.invR = invR; d.invC = invC;
    d.int_mask = int_mask;
    d.step_fac = step_fac;
    d.n_check = h->p.n_check;
  };
  auto fill_b = [&](auto& B) {
    B.a_tile_lp = a_tlp; B.t_tile_lp = t_tlp; B.a_tile_beg = a_beg; B.t_tile_beg = t_beg;
    B.ctl = ctl;
    B.tp_p = tp_p; B.tp_d = tp_d; B.tp_c1 = tp_c1; B.tp_c2 = tp_c2;
    B.n_done = n_done;
    B.kglob = kglob;
    B.q_lps = q_lps; B.q_a = q_a; B.q_t = q_t; B.q_pre = q_pre; B.q_cnt = q_cnt; B.q_ctr = q_ctr;
    B.lp_cnt = lp_cnt;
  };
  if (mixed) {
    fill_common(d32);
    d32.a_vals = a_vals32; d32.t_vals = t_vals32;
    d32.c = c32; d32.l = l32; d32.u = u32; d32.lo = lo32; d32.hi = hi32;
    fill_b(h->b32);
    h->b32.slot = static_cast<BatchSlot<float>*>(slot);
    fill_batch<float>(h->b32, d32, h, X, Y, AX, ATY, XLR, YLR);
    CKB(launch_batch_init_point<float>(h->b32, st));
  } else {
    fill_common(d64);
    d64.a_vals = a_vals64; d64.t_vals = t_vals64;
    d64.c = c64; d64.l = l64; d64.u = u64; d64.lo = lo64; d64.hi = hi64;
    fill_b(h->b64);
    h->b64.slot = static_cast<BatchSlot<double>*>(slot);
    fill_batch<double>(h->b64, d64, h, X, Y, AX, ATY, XLR, YLR);
    CKB(launch_batch_init_point<double>(h->b64, st));
  }
  // persistent form: one co-resident grid (cooperative launch) where it fits
  h->grid_bar = gbar;
  {
    int coop = 0, dev = 0;
    CKB(cudaGetDevice(&dev));
    CKB(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const int per_sm = mixed ? batch_persistent_blocks_per_sm<float>() : batch_persistent_blocks_per_sm<double>();
    const int grid = (coop && per_sm > 0) ? per_sm * device_sm_count() : 0;
    h->b32.grid_q = h->b64.grid_q = grid;
    if (h->p.batch_launch == 2 && grid == 0) {
      set_error("batch_launch = 2: the persistent batched kernel cannot be made co-resident here");
      return SCYLLA_ERR_UNSUPPORTED;
    }
    h->persistent = grid > 0 && h->p.batch_launch == 2;
  }
  set_async_tiles(h, h->p.batch_launch == 3, h->p.batch_launch == 3);
  CKB(cudaStreamSynchronize(st));
  // automatic form: n_check attempts from the cold start in each form, timed on the
  // device; the fastest is kept (all give identical results) and the LPs go back to
  // the cold start.  The asynchronous-copy graphs take, for each of the two attempt
  // kernels, the tile form with the shorter launch (timed separately).
  if (h->p.batch_launch == 0) {
    const bool can_persist = (mixed ? h->b32.grid_q : h->b64.grid_q) > 0;
    bool ap = false, ad = false;
    if (mixed) {
      // every LP taking part, as at the start of a solve
      CKB(launch_batch_init<float>(h->b32, 0.0, 1LL << 40, 0, st));
      CKB(launch_batch_check<float>(h->b32, st));
      for (int q = 0; q < 2; ++q) {
        set_async_tiles(h, q == 1, q == 1);
        for (int part = 0; part < 2; ++part) {
          const int rc = time_batch_part<float>(h, h->b32, part, 8, &h->tune_kernel_ms[2 * q + part]);
          if (rc != SCYLLA_OK) return rc;
        }
      }
      ap = h->tune_kernel_ms[2] < h->tune_kernel_ms[0];
      ad = h->tune_kernel_ms[3] < h->tune_kernel_ms[1];
    }
    int best = 0;
    for (int form = 0; form < 3; ++form) {
      if ((form == 1 && !can_persist) || (form == 2 && !(ap || ad))) continue;
      h->persistent = form == 1;
      if (form == 2) set_async_tiles(h, ap, ad);
      else set_async_tiles(h, false, false);
      CKB(cudaMemcpyAsync(ctl, h->ctl0.data(), sizeof(Control) * count, cudaMemcpyHostToDevice, st));
      if (mixed) CKB(launch_batch_init_point<float>(h->b32, st));
      else CKB(launch_batch_init_point<double>(h->b64, st));
      const int rc = mixed ? batch_solve_impl<float>(h, h->b32, 0.0, h->p.n_check)
                           : batch_solve_impl<double>(h, h->b64, 0.0, h->p.n_check);
      if (rc != SCYLLA_OK) return rc;
      h->tune_ms[form] = h->last_ms;
      if (h->tune_ms[form] < h->tune_ms[best]) best = form;
    }
    h->persistent = best == 1;
    if (best == 2) set_async_tiles(h, ap, ad);
    else set_async_tiles(h, false, false);
    CKB(cudaMemcpyAsync(ctl, h->ctl0.data(), sizeof(Control) * count, cudaMemcpyHostToDevice, st));
    if (mixed) CKB(launch_batch_init_point<float>(h->b32, st));
    else CKB(launch_batch_init_point<double>(h->b64, st));
    CKB(cudaStreamSynchronize(st));
  }
  return SCYLLA_OK;
}

}  // namespace

extern "C" int scylla_batch_create(int32_t count, const scylla_csr* A, const double* const* c,
                                   const double* const* row_lo, const double* const* row_hi,
                                   const double* const* col_lo, const double* const* col_hi,
                                   const scylla_params* p, void* cuda_stream, scylla_batch** out) {
  if (!out) {
    set_error("out is null");
    return SCYLLA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (count < 1 || !A || !c || !row_lo || !row_hi || !col_lo || !col_hi) {
    set_error("need count >= 1 and non-null arrays");
    return SCYLLA_ERR_INVALID_ARG;
  }
  for (int b = 0; b < count; ++b) {
    std::vector<uint8_t> zeros(A[b].n > 0 ? size_t(A[b].n) : 1, 0);
    const int rc = validate_lp(&A[b], c[b], row_lo[b], row_hi[b], col_lo[b], col_hi[b], zeros.data());
    if (rc != SCYLLA_OK) {
      set_error("LP " + std::to_string(b) + ": " + get_error());
      return rc;
    }
  }
  scylla_params dp;
  scylla_default_params(&dp);
  scylla_batch* h = nullptr;
  int rc = SCYLLA_OK;
  try {
    h = new scylla_batch();
    rc = create_batch(count, A, c, row_lo, row_hi, col_lo, col_hi, p ? p : &dp, cuda_stream, h);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    rc = SCYLLA_ERR_OOM;
  }
  if (rc != SCYLLA_OK) {
    if (h) {
      h->release();
      delete h;
    }
    return rc;
  }
  *out = h;
  return SCYLLA_OK;
}

extern "C" void scylla_batch_destroy(scylla_batch* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  h->release();
  delete h;
}

extern "C" int scylla_batch_solve(scylla_batch* h, double tol, int64_t iter_limit, scylla_pdhg_result* results,
                                  double* seconds) {
  if (!h || !results) {
    set_error("null argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (!(tol >= 0.0) || iter_limit < 0) {
    set_error("need tol >= 0 and iter_limit >= 0");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (h->user_st) {
    CKB(cudaEventRecord(h->ev_user, h->user_st));
    CKB(cudaStreamWaitEvent(h->st, h->ev_user, 0));
  }
  const int rc = h->p.precision == SCYLLA_PREC_MIXED ? batch_solve_impl<float>(h, h->b32, tol, iter_limit)
                                                     : batch_solve_impl<double>(h, h->b64, tol, iter_limit);
  if (rc != SCYLLA_OK) return rc;
  for (int b = 0; b < h->nlp; ++b) {
    const Control& c = h->h_ctl[b];
    scylla_pdhg_result& r = results[b];
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
    r.seconds = h->last_ms * 1e-3;
  }
  if (seconds) *seconds = h->last_ms * 1e-3;
  return SCYLLA_OK;
}

namespace {
// the graph form's per-attempt kernels as separate launches with CUDA events around
// each, from the cold start, every LP taking part (see scylla_batch_time_kernels)
template <typename T>
int batch_time_impl(scylla_batch* h, DevBatch<T>& B, int attempts, double* ms) {
  cudaStream_t st = h->st;
  std::vector<cudaEvent_t> ev;
  std::vector<int> which;
  cudaError_t e = launch_batch_init<T>(B, 0.0, (long long)attempts + 1, 0, st);
  if (e == cudaSuccess) e = launch_batch_check<T>(B, st);
  for (int a = 0; a < attempts && e == cudaSuccess; ++a)
    for (int part = 0; part < 3 && e == cudaSuccess; ++part) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      e = cudaEventCreate(&e0);
      if (e == cudaSuccess) e = cudaEventCreate(&e1);
      if (e != cudaSuccess) break;
      ev.push_back(e0);
      ev.push_back(e1);
      which.push_back(part);
      e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = launch_batch_part<T>(B, part, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  double sum[3] = {0, 0, 0};
  int cnt[3] = {0, 0, 0};
  if (e == cudaSuccess)
    for (size_t i = 0; i < which.size(); ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      sum[which[i]] += t;
      cnt[which[i]]++;
    }
  for (cudaEvent_t x : ev) cudaEventDestroy(x);
  CKB(e);
  for (int k = 0; k < 3; ++k) ms[k] = cnt[k] ? sum[k] / cnt[k] : 0.0;
  return SCYLLA_OK;
}
}  // namespace

extern "C" int scylla_batch_time_kernels(scylla_batch* h, int32_t attempts, double* ms) {
  if (!h || !ms || attempts < 1) {
    set_error("need a batch, ms[3] and attempts >= 1");
    return SCYLLA_ERR_INVALID_ARG;
  }
  return h->p.precision == SCYLLA_PREC_MIXED ? batch_time_impl<float>(h, h->b32, attempts, ms)
                                             : batch_time_impl<double>(h, h->b64, attempts, ms);
}

extern "C" int scylla_batch_info(const scylla_batch* h, int32_t* form, double* tune_ms) {
  if (!h) {
    set_error("null handle");
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (form) *form = h->persistent ? 2 : ((h->async_p || h->async_d) ? 3 : 1);
  if (tune_ms)
    for (int q = 0; q < 3; ++q) tune_ms[q] = h->tune_ms[q];
  return SCYLLA_OK;
}

extern "C" int scylla_batch_get_primal(const scylla_batch* h, int32_t b, double* x) {
  if (!h || !x || b < 0 || b >= h->nlp) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const int c0 = h->col_off[b], cnt = h->col_off[b + 1] - h->col_off[b];
  cudaStream_t st = h->st;
  if (h->p.precision == SCYLLA_PREC_MIXED) CKB(launch_batch_get_x<float>(h->b32, b, c0, cnt, h->io, st));
  else CKB(launch_batch_get_x<double>(h->b64, b, c0, cnt, h->io, st));
  CKB(cudaMemcpyAsync(x, h->io, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

// y of LP b from its current pool (the pair a finished LP returns, whose errors its
// result reports), unscaled on the host: y_i = y~_i R_i in FP64, as the primal's
// getter does on the device
extern "C" int scylla_batch_get_dual(const scylla_batch* h, int32_t b, double* y) {
  if (!h || !y || b < 0 || b >= h->nlp) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const int r0 = h->row_off[b], cnt = h->row_off[b + 1] - h->row_off[b];
  if (cnt == 0) return SCYLLA_OK;
  cudaStream_t st = h->st;
  const bool mixed = h->p.precision == SCYLLA_PREC_MIXED;
  const Control* dctl = mixed ? h->b32.ctl : h->b64.ctl;
  int cur = -1;
  CKB(cudaMemcpyAsync(&cur, &dctl[b].ix_cur, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKB(cudaStreamSynchronize(st));
  if (cur < 0 || cur > 2) {
    set_error("pool index out of range");
    return SCYLLA_ERR_CUDA;
  }
  std::vector<double> R(static_cast<size_t>(cnt));
  const double* Rd = mixed ? h->b32.d.R : h->b64.d.R;
  CKB(cudaMemcpyAsync(R.data(), Rd + r0, sizeof(double) * size_t(cnt), cudaMemcpyDeviceToHost, st));
  if (mixed) {
    std::vector<float> v(static_cast<size_t>(cnt));
    CKB(cudaMemcpyAsync(v.data(), h->b32.d.Y[cur] + r0, sizeof(float) * size_t(cnt), cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    for (int i = 0; i < cnt; ++i) y[i] = double(v[size_t(i)]) * R[size_t(i)];
  } else {
    CKB(cudaMemcpyAsync(y, h->b64.d.Y[cur] + r0, sizeof(double) * size_t(cnt), cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    for (int i = 0; i < cnt; ++i) y[i] *= R[size_t(i)];
  }
  return SCYLLA_OK;
}

extern "C" int scylla_batch_reset_state(scylla_batch* h) {
  if (!h) {
    set_error("null handle");
    return SCYLLA_ERR_INVALID_ARG;
  }
  cudaStream_t st = h->st;
  const DevBatch<double>& B64 = h->b64;
  const DevBatch<float>& B32 = h->b32;
  Control* ctl = h->p.precision == SCYLLA_PREC_MIXED ? B32.ctl : B64.ctl;
  CKB(cudaMemcpyAsync(ctl, h->ctl0.data(), sizeof(Control) * h->nlp, cudaMemcpyHostToDevice, st));
  if (h->p.precision == SCYLLA_PREC_MIXED) CKB(launch_batch_init_point<float>(B32, st));
  else CKB(launch_batch_init_point<double>(B64, st));
  CKB(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}
