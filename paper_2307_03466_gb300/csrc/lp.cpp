// Host runtime of the Scylla PDHG library: the C ABI of scylla.h for creating an
// LP handle, solving, objective updates and state access.  Everything numeric on
// the PDHG path runs in the kernels of kernels.cu; this file validates input,
// builds the auxiliary columns, the transposed CSR and the warp tiles, owns the
// device memory (one arena per handle) and drives the solve as one CUDA graph
// whose device-side while loop runs until the device control block says done.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "host_par.h"
#include "lp_handle.h"

namespace scylla {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

}  // namespace scylla

using namespace scylla;

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                      \
      return e_ == cudaErrorMemoryAllocation ? SCYLLA_ERR_OOM : SCYLLA_ERR_CUDA;          \
    }                                                                                     \
  } while (0)

#define FAIL(code, msg)       \
  do {                        \
    set_error(msg);           \
    return (code);            \
  } while (0)

static const double kInf = std::numeric_limits<double>::infinity();

// a kernel form in scylla_params.prefetch's numbering
static int api_form(int f) { return f == kFormPlain ? 4 : f == kFormAsync ? 5 : f; }

extern "C" void scylla_default_params(scylla_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->precision = SCYLLA_PREC_FP64;
  p->n_check = 64;
  p->ruiz_iters = 10;
  p->pock_chambolle = 1;
  p->adaptive_step = 1;
  p->restarts = 1;
  p->primal_weight_update = 1;
  p->stall_checks = 0;
  p->aux_general_integers = 1;
  p->use_graph = 1;
  p->fixed_step_factor = 0.9;
  p->beta_sufficient = 0.2;
  p->beta_necessary = 0.8;
  p->beta_artificial = 0.36;
  p->pw_smoothing = 0.5;
  p->step_reduction_exp = 0.3;
  p->step_growth_exp = 0.6;
  p->alpha = 0.9;
  p->eps1 = 0.01;
  p->beta = 0.98;
  p->eps_floor = 1e-8;
  p->max_rounds = 100;
  p->iter_limit = 20000;
  p->total_iter_cap = 1000000000LL;
  p->run_stall_checks = 5;
  p->trace_capacity = 0;
  p->seed = 0;
  p->time_limit_s = 0.0;
  p->device_wait_limit_s = 5.0;
  p->pdl = 1;
  p->prefetch = 0;
  p->host_transpose = 0;
  p->repair_iters = 0;
  p->repair_tol = 1e-7;
  p->repair_rounds = 8;
  p->distance = 1;
  p->batch_launch = 0;
  p->autotune = 1;
  p->infeasibility_checks = 0;
  p->dual_form = 0;
}

extern "C" const char* scylla_last_error(void) { return get_error(); }

namespace {

size_t padded(size_t nnz) { return scylla::padded_len(nnz); }

// A stream-ordered memory pool per device for the handles' arenas and set-up
// scratch.  It keeps the memory of destroyed handles for the next ones (release
// threshold: all of it), so creating and destroying handles in a loop needs no
// cudaMalloc or synchronizing cudaFree.
cudaError_t handle_pool(int device, cudaMemPool_t* out) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0) return cudaErrorInvalidDevice;
  if (size_t(device) >= pools.size()) pools.resize(size_t(device) + 1, nullptr);
  if (!pools[size_t(device)]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ULL;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    pools[size_t(device)] = pool;
  }
  *out = pools[size_t(device)];
  return cudaSuccess;
}

// Pinned host blocks of kPinnedBlock bytes (a handle's control-block mirror and
// done flags), kept on a free list for reuse instead of cudaFreeHost.
constexpr size_t kPinnedBlock = sizeof(scylla::Control) + 64;
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;

cudaError_t pinned_acquire(void** p) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (!g_pinned_free.empty()) {
      *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost(p, kPinnedBlock);
}

void pinned_release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.push_back(p);
}

// Warp tiles of a CSR structure.  Above kTileSpan rows the rows are cut into spans
// of kTileSpan rows, tiled independently on the host threads and concatenated: a
// tile never crosses a span boundary, so the tiles depend on the structure alone.
constexpr int kTileSpan = 1 << 17;
std::vector<int2> build_tiles(const std::vector<int>& rowptr, int max_rows = scylla::kTileRows) {
  const int m = int(rowptr.size()) - 1;
  if (m <= kTileSpan) return scylla::build_tiles_range(rowptr, 0, m, max_rows);
  const int spans = (m + kTileSpan - 1) / kTileSpan;
  std::vector<std::vector<int2>> part(static_cast<size_t>(spans));
  scylla::fork_join(spans, [&](int k) {
    const int b = k * kTileSpan, e = std::min(m, b + kTileSpan);
    part[size_t(k)] = scylla::build_tiles_range(rowptr, b, e, max_rows);
  });
  size_t total = 1;
  for (const auto& v : part) total += v.size() - 1;
  std::vector<int2> t;
  t.reserve(total);
  for (int k = 0; k < spans; ++k) t.insert(t.end(), part[size_t(k)].begin(), part[size_t(k)].end() - 1);
  t.push_back(part.back().back());
  return t;
}

}  // namespace

namespace scylla {

size_t padded_len(size_t nnz) { return ((nnz + 3) & ~size_t(3)) + 4; }

// contiguous row ranges of [r_begin, r_end) with at most kTileNnz nonzeros and
// max_rows rows; a longer row is a tile of its own.  Each boundary is stored as
// (row, rowptr[row]).
std::vector<int2> build_tiles_range(const std::vector<int>& rowptr, int r_begin, int m, int max_rows) {
  std::vector<int2> t;
  t.reserve((m - r_begin) / 4 + 2);
  t.push_back(make_int2(r_begin, rowptr[r_begin]));
  int r = r_begin;
  while (r < m) {
    const int len = rowptr[r + 1] - rowptr[r];
    if (len > kTileNnz) {
      ++r;
      t.push_back(make_int2(r, rowptr[r]));
      continue;
    }
    int cnt = 0, nz = 0;
    while (r < m && cnt < max_rows) {
      const int l2 = rowptr[r + 1] - rowptr[r];
      if (nz + l2 > kTileNnz) break;
      nz += l2;
      ++r;
      ++cnt;
    }
    t.push_back(make_int2(r, rowptr[r]));
  }
  return t;
}

}  // namespace scylla

namespace {

template <typename T>
void fill_dev(DevLP<T>& d, scylla_lp* lp);
template <typename T>
int autotune_form(scylla_lp* lp);

}  // namespace

int scylla_lp::ensure_host_vectors() const {
  if (host_vectors_ready) return SCYLLA_OK;
  c0.resize(size_t(n0));
  l0.resize(size_t(n0));
  u0.resize(size_t(n0));
  int0.resize(size_t(n0));
  lo0.resize(size_t(m0));
  hi0.resize(size_t(m0));
  CK(cudaMemcpyAsync(c0.data(), c_orig, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(l0.data(), l_orig, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(u0.data(), u_orig, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(int0.data(), int_mask, n0, cudaMemcpyDeviceToHost, st));
  if (m0 > 0) {
    // the original rows come first; only the auxiliary rows' bounds change later
    CK(cudaMemcpyAsync(lo0.data(), lo_un, sizeof(double) * m0, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hi0.data(), hi_un, sizeof(double) * m0, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  host_vectors_ready = true;
  return SCYLLA_OK;
}

int scylla_lp::ensure_host_matrix() const {
  if (host_matrix_ready) return SCYLLA_OK;
  const int rv = ensure_host_vectors();
  if (rv != SCYLLA_OK) return rv;
  std::vector<int> rp(size_t(m0) + 1);
  cols0.resize(size_t(nnz0));
  vals0.resize(size_t(nnz0));
  CK(cudaMemcpyAsync(rp.data(), a_rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, st));
  if (nnz0 > 0) {
    CK(cudaMemcpyAsync(cols0.data(), a_cols, sizeof(int32_t) * nnz0, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(vals0.data(), a_vals0, sizeof(double) * nnz0, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  rowptr0.assign(rp.begin(), rp.end());
  host_matrix_ready = true;
  return SCYLLA_OK;
}

void scylla_lp::ensure_columns() const {
  if (columns_ready) return;
  if (ensure_host_matrix() != SCYLLA_OK) return;
  scylla::transpose_csr(m0, n0, rowptr0.data(), cols0.data(), vals0.data(), colptr0, colrows0, &colvals0);
  columns_ready = true;
}

// --------------------------------------------------------------- validation ---
int scylla::validate_lp(const scylla_csr* A, const double* c, const double* lo, const double* hi, const double* l,
                    const double* u, const uint8_t* is_int) {
  if (!A || !c || !lo || !hi || !l || !u || !is_int) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (A->m < 0 || A->n < 1 || A->nnz < 0) FAIL(SCYLLA_ERR_INVALID_ARG, "need m >= 0, n >= 1, nnz >= 0");
  const int64_t lim = (int64_t(1) << 31) - 64;
  if (A->m >= lim / 2 || A->n >= lim / 2 || A->nnz >= lim / 2)
    FAIL(SCYLLA_ERR_UNSUPPORTED, "dimensions or nnz beyond the 32-bit index range");
  if (!A->rowptr || (A->nnz > 0 && (!A->cols || !A->vals))) FAIL(SCYLLA_ERR_INVALID_ARG, "null CSR array");
  if (A->rowptr[0] != 0 || A->rowptr[A->m] != A->nnz) FAIL(SCYLLA_ERR_INVALID_ARG, "rowptr[0] != 0 or rowptr[m] != nnz");
  for (int64_t i = 0; i < A->m; ++i)
    if (A->rowptr[i + 1] < A->rowptr[i]) FAIL(SCYLLA_ERR_INVALID_ARG, "rowptr not non-decreasing at row " + std::to_string(i));
  // rows in parallel slices; the first failing row is reported
  {
    const int64_t mm = A->m;
    const int T = threads_for(A->nnz + mm);
    std::vector<int64_t> bad(size_t(T), mm);
    std::vector<int> why(size_t(T), 0);
    fork_join(T, [&](int t) {
      for (int64_t i = mm * t / T; i < mm * (t + 1) / T; ++i) {
        const int64_t p0 = A->rowptr[i], p1 = A->rowptr[i + 1];
        int w = 0;
        for (int64_t p = p0; p < p1 && !w; ++p) {
          const int32_t j = A->cols[p];
          if (j < 0 || j >= A->n) w = 1;
          else if (p > p0 && A->cols[p - 1] >= j) w = 2;
          else if (!std::isfinite(A->vals[p])) w = 3;
        }
        if (w) {
          bad[size_t(t)] = i;
          why[size_t(t)] = w;
          return;
        }
      }
    });
    for (int t = 0; t < T; ++t) {
      if (!why[size_t(t)]) continue;
      const std::string row = std::to_string(bad[size_t(t)]);
      if (why[size_t(t)] == 1) FAIL(SCYLLA_ERR_INVALID_ARG, "column index out of range in row " + row);
      if (why[size_t(t)] == 2) FAIL(SCYLLA_ERR_INVALID_ARG, "column indices not strictly increasing in row " + row);
      FAIL(SCYLLA_ERR_INVALID_ARG, "non-finite matrix value in row " + row);
    }
  }
  // row bounds and columns in parallel slices; the first failing index is reported
  {
    const int64_t mm = A->m, nn = A->n;
    const int T = threads_for(2 * (mm + nn));
    std::vector<int64_t> bad_row(size_t(T), mm), bad_col(size_t(T), nn);
    std::vector<int> why(size_t(T), 0);
    fork_join(T, [&](int t) {
      for (int64_t i = mm * t / T; i < mm * (t + 1) / T; ++i)
        if (std::isnan(lo[i]) || std::isnan(hi[i]) || lo[i] > hi[i] || lo[i] == kInf || hi[i] == -kInf) {
          bad_row[size_t(t)] = i;
          break;
        }
      for (int64_t j = nn * t / T; j < nn * (t + 1) / T; ++j) {
        int w = 0;
        if (!std::isfinite(c[j])) w = 1;
        else if (std::isnan(l[j]) || std::isnan(u[j]) || l[j] > u[j] || l[j] == kInf || u[j] == -kInf) w = 2;
        else if (is_int[j] > 1) w = 3;
        else if (is_int[j] && ((std::isfinite(l[j]) && l[j] != std::floor(l[j])) ||
                               (std::isfinite(u[j]) && u[j] != std::floor(u[j]))))
          w = 4;
        if (w) {
          bad_col[size_t(t)] = j;
          why[size_t(t)] = w;
          break;
        }
      }
    });
    for (int t = 0; t < T; ++t)
      if (bad_row[size_t(t)] < mm)
        FAIL(SCYLLA_ERR_INVALID_ARG, "invalid row bounds at row " + std::to_string(bad_row[size_t(t)]));
    for (int t = 0; t < T; ++t) {
      const std::string j = std::to_string(bad_col[size_t(t)]);
      switch (why[size_t(t)]) {
        case 1: FAIL(SCYLLA_ERR_INVALID_ARG, "non-finite objective at column " + j);
        case 2: FAIL(SCYLLA_ERR_INVALID_ARG, "invalid column bounds at column " + j);
        case 3: FAIL(SCYLLA_ERR_INVALID_ARG, "is_integer must be 0 or 1");
        case 4: FAIL(SCYLLA_ERR_INVALID_ARG, "integer column with a fractional bound: " + j);
        default: break;
      }
    }
  }
  return SCYLLA_OK;
}

// ------------------------------------------------------------------ create ---
static int create_impl(const scylla_csr* A, const double* c, const double* lo, const double* hi, const double* l,
                       const double* u, const uint8_t* is_int, const scylla_params* pin, void* cuda_stream,
                       scylla_lp* lp) {
  lp->p = *pin;
  if (lp->p.n_check < 1) FAIL(SCYLLA_ERR_INVALID_ARG, "n_check must be >= 1");
  if (lp->p.trace_capacity < 0) FAIL(SCYLLA_ERR_INVALID_ARG, "trace_capacity must be >= 0");
  if (lp->p.use_graph < 0 || lp->p.use_graph > 3) FAIL(SCYLLA_ERR_INVALID_ARG, "use_graph must be 0..3");
  if (!(lp->p.device_wait_limit_s > 0.0)) FAIL(SCYLLA_ERR_INVALID_ARG, "device_wait_limit_s must be > 0");
  if (lp->p.prefetch < 0 || lp->p.prefetch > 5) FAIL(SCYLLA_ERR_INVALID_ARG, "prefetch must be 0..5");
  if (lp->p.host_transpose < 0 || lp->p.host_transpose > 1) FAIL(SCYLLA_ERR_INVALID_ARG, "host_transpose must be 0 or 1");
  if (lp->p.repair_iters < 0 || !(lp->p.repair_tol >= 0.0) || lp->p.repair_rounds < 1)
    FAIL(SCYLLA_ERR_INVALID_ARG, "need repair_iters >= 0, repair_tol >= 0 and repair_rounds >= 1");
  if (lp->p.distance != 1 && lp->p.distance != 2) FAIL(SCYLLA_ERR_INVALID_ARG, "distance must be 1 or 2");
  if (lp->p.infeasibility_checks != 0 && lp->p.infeasibility_checks != 1)
    FAIL(SCYLLA_ERR_INVALID_ARG, "infeasibility_checks must be 0 or 1");
  if (lp->p.dual_form < 0 || lp->p.dual_form > 5) FAIL(SCYLLA_ERR_INVALID_ARG, "dual_form must be 0..5");
  if (lp->p.precision != SCYLLA_PREC_MIXED && (lp->p.prefetch == 5 || lp->p.dual_form == 5))
    FAIL(SCYLLA_ERR_INVALID_ARG, "the asynchronous-copy form (5) is for FP32-mixed precision");
  if (lp->p.precision != SCYLLA_PREC_FP64 && lp->p.precision != SCYLLA_PREC_MIXED)
    FAIL(SCYLLA_ERR_INVALID_ARG, "unknown precision");
  CK(cudaGetDevice(&lp->device));
  lp->user_st = static_cast<cudaStream_t>(cuda_stream);
  CK(cudaStreamCreateWithFlags(&lp->st, cudaStreamNonBlocking));
  CK(cudaEventCreate(&lp->ev_user));
  CK(cudaEventCreate(&lp->ev0));
  CK(cudaEventCreate(&lp->ev1));

  // ---- the original MIP: ||c||, the integer count and the general integers that
  // get auxiliary columns, in one pass over the caller's arrays in a number of
  // chunks fixed by n (so ||c|| does not depend on the host's thread count).  The
  // host copies of the vectors are fetched from the device on first use.
  const int64_t m0 = A->m, n0 = A->n, nnz0 = A->nnz;
  lp->m0 = m0;
  lp->n0 = n0;
  lp->nnz0 = nnz0;
  // the l2 distance needs no auxiliary columns
  const bool aux_on = lp->p.aux_general_integers != 0 && lp->p.distance == 1;
  {
    const int chunks = int(std::max<int64_t>(1, std::min<int64_t>(64, n0 / 65536)));
    std::vector<double> c2(size_t(chunks), 0.0);
    std::vector<int64_t> nint(size_t(chunks), 0);
    std::vector<std::vector<int32_t>> gen(static_cast<size_t>(chunks));
    fork_join(chunks, [&](int t) {
      double s2 = 0.0;
      int64_t k = 0;
      for (int64_t j = n0 * t / chunks; j < n0 * (t + 1) / chunks; ++j) {
        s2 += c[j] * c[j];
        if (!is_int[j]) continue;
        ++k;
        if (aux_on && u[j] - l[j] != 1.0) gen[size_t(t)].push_back(int32_t(j));
      }
      c2[size_t(t)] = s2;
      nint[size_t(t)] = k;
    });
    double s2 = 0.0;
    lp->n_int = 0;
    lp->gen_int.clear();
    for (int t = 0; t < chunks; ++t) {
      s2 += c2[size_t(t)];
      lp->n_int += nint[size_t(t)];
      lp->gen_int.insert(lp->gen_int.end(), gen[size_t(t)].begin(), gen[size_t(t)].end());
    }
    lp->c0norm = std::sqrt(s2);
  }
  const int64_t na = int64_t(lp->gen_int.size());
  lp->n_aux = na;
  const int64_t m = m0 + 2 * na, n = n0 + na, nnz = nnz0 + 4 * na;
  lp->m = int(m);
  lp->n = int(n);
  lp->nnz = int(nnz);

  // the iterated LP's CSR: the original rows (used in place when there are no
  // auxiliary columns), then two rows per auxiliary column
  std::vector<int> rp(m + 1), ci_aux;
  std::vector<double> va_aux;
  for (int64_t i = 0; i <= m0; ++i) rp[i] = int(A->rowptr[i]);
  const int* ci = A->cols;
  const double* va = A->vals;
  if (na > 0) {
    ci_aux.resize(nnz);
    va_aux.resize(nnz);
    std::copy(A->cols, A->cols + nnz0, ci_aux.begin());
    std::copy(A->vals, A->vals + nnz0, va_aux.begin());
    for (int64_t t = 0; t < na; ++t) {
      const int j = lp->gen_int[t];
      const int64_t r0 = m0 + 2 * t, p = nnz0 + 4 * t;
      ci_aux[p] = j; va_aux[p] = -1.0;
      ci_aux[p + 1] = int(n0 + t); va_aux[p + 1] = 1.0;
      ci_aux[p + 2] = j; va_aux[p + 2] = 1.0;
      ci_aux[p + 3] = int(n0 + t); va_aux[p + 3] = 1.0;
      rp[r0 + 1] = int(p + 2);
      rp[r0 + 2] = int(p + 4);
    }
    ci = ci_aux.data();
    va = va_aux.data();
  }
  // the iterated LP's vectors: the caller's arrays, extended for auxiliary columns
  std::vector<double> cA, loA, hiA, lA, uA;
  std::vector<uint8_t> imask;
  const double *cP = c, *loP = lo, *hiP = hi, *lP = l, *uP = u;
  const uint8_t* imP = is_int;
  if (na > 0) {
    cA.assign(c, c + n0);
    lA.assign(l, l + n0);
    uA.assign(u, u + n0);
    loA.assign(lo, lo + m0);
    hiA.assign(hi, hi + m0);
    imask.assign(is_int, is_int + n0);
    for (int64_t t = 0; t < na; ++t) {
      const int j = lp->gen_int[t];
      cA.push_back(0.0);
      lA.push_back(0.0);
      uA.push_back(u[j] - l[j]);
      imask.push_back(0);
    }
    loA.resize(size_t(m), -kInf);
    hiA.resize(size_t(m), kInf);
    cP = cA.data(); loP = loA.data(); hiP = hiA.data(); lP = lA.data(); uP = uA.data(); imP = imask.data();
  }

  // ---- stored transpose (rows ascending within each column): a stable radix sort
  // by column on the device after the upload of A, or a counting sort on the host
  // threads (scylla_params.host_transpose); its tiles are built once the column
  // pointers are known
  const bool host_tp = lp->p.host_transpose != 0;
  std::vector<int> tp, tr;
  std::vector<double> tv;
  if (host_tp) transpose_csr(m, n, rp.data(), ci, va, tp, tr, &tv);
  const std::vector<int2> at = build_tiles(rp);
  lp->a_ntiles = int(at.size()) - 1;

  // ---- grid sizes and scratch
  const bool mixed = lp->p.precision == SCYLLA_PREC_MIXED;
  // form of the per-attempt kernels.  When A, A^T and the vectors fit in half of L2
  // they stay there between attempts and the kernels are latency-bound: 32-row
  // tiles, 64 registers, four blocks per SM (measured: loading the first tile before
  // the dependency wait gains nothing there).  Otherwise they are bound by the bytes
  // in flight: wide tiles (up to kWideRows rows, several per lane; several times the
  // bytes of a 32-row tile on short rows) and 80 registers, which keep more loads in
  // flight per warp.  prefetch = 1 .. 4 force a form.
  std::vector<int2> atw, ttw;
  {
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, lp->device));
    const double vb = mixed ? 4.0 : 8.0;
    const double bytes = 2.0 * double(nnz) * (4.0 + vb) + 12.0 * double(m + n) * vb;
    const bool fits = bytes <= 0.5 * double(l2);
    const int pf = lp->p.prefetch;
    int form = kFormPlain;
    auto forced = [](int v) {
      return v == 1 ? kFormPrefetch : v == 2 ? kFormWide : v == 3 ? kFormStaged : v == 5 ? kFormAsync : kFormPlain;
    };
    if (pf == 0) form = fits ? kFormPlain : kFormWide;
    else form = forced(pf);
    lp->form_p = form;
    lp->form_d = (pf != 0 && lp->p.dual_form != 0) ? forced(lp->p.dual_form) : form;
    lp->form_rule = pf == 0 ? form : (fits ? kFormPlain : kFormWide);
    lp->tune = pf == 0 && lp->p.autotune != 0;
    auto wide_form = [](int f) { return f == kFormWide || f == kFormStaged; };
    if (wide_form(lp->form_p) || wide_form(lp->form_d) || lp->tune) atw = build_tiles(rp, kWideRows);
  }
  // wide tiles are built for the wide forms, and for the autotuner, which times both
  const bool wide_p = lp->form_p == kFormWide || lp->form_p == kFormStaged || lp->tune;
  const bool wide_d = lp->form_d == kFormWide || lp->form_d == kFormStaged || lp->tune;
  lp->a_ntiles_w = wide_d ? int(atw.size()) - 1 : lp->a_ntiles;
  auto grid_of = [&](int side, int form, int tiles) {
    return mixed ? occupancy_grid<float>(side, form, tiles) : occupancy_grid<double>(side, form, tiles);
  };
  auto form_tiles_d = [&](int form) {
    return (form == kFormWide || form == kFormStaged) ? lp->a_ntiles_w : lp->a_ntiles;
  };
  // the block partials are sized for the largest grid of the forms in play (the
  // transpose's tile counts come later)
  int cap_p = grid_of(0, lp->form_p, 1 << 30), cap_d = grid_of(1, lp->form_d, form_tiles_d(lp->form_d));
  const int cap_c1 = grid_of(2, 0, 1 << 30);
  if (lp->tune) {
    cap_p = std::max(grid_of(0, kFormPlain, 1 << 30), grid_of(0, kFormWide, 1 << 30));
    cap_d = std::max(grid_of(1, kFormPlain, lp->a_ntiles), grid_of(1, kFormWide, lp->a_ntiles_w));
    if (mixed) {
      cap_p = std::max(cap_p, grid_of(0, kFormAsync, 1 << 30));
      cap_d = std::max(cap_d, grid_of(1, kFormAsync, lp->a_ntiles));
    }
  }
  lp->grid_d = grid_of(1, lp->form_d, form_tiles_d(lp->form_d));
  lp->grid_c2 = grid_of(3, 0, lp->a_ntiles);
  // persistent cooperative solve: one grid of co-resident blocks, if it fits
  {
    const int per_sm = mixed ? persistent_blocks_per_sm<float>() : persistent_blocks_per_sm<double>();
    lp->p_grid = (per_sm >= 1 && lp->p.n_check <= kMaxNcheckPersistent) ? per_sm * device_sm_count() : 0;
  }
  // the primal kernel also runs the elementwise retry path over n columns
  lp->red_blocks = std::max(1, std::min(4 * device_sm_count(), int((std::max(m, n) + kThreads - 1) / kThreads)));
  const size_t vs = mixed ? sizeof(float) : sizeof(double);

  // ---- device arena: pass 1 sizes, pass 2 carves
  for (int pass = 0; pass < 2; ++pass) {
    Arena ar;
    if (pass == 1) {
      cudaMemPool_t pool = nullptr;
      CK(handle_pool(lp->device, &pool));
      CK(cudaMallocFromPoolAsync(&lp->arena, lp->arena_bytes, pool, lp->st));
      ar.base = static_cast<char*>(lp->arena);
    }
    lp->a_rowptr = ar.take<int>(m + 1);
    lp->a_cols = ar.take<int>(padded(nnz));
    lp->a_tiles = ar.take<int2>(at.size());
    lp->a_tiles_w = wide_d ? ar.take<int2>(atw.size()) : lp->a_tiles;
    lp->t_rowptr = ar.take<int>(n + 1);
    lp->t_cols = ar.take<int>(padded(nnz));
    lp->t_tiles = ar.take<int2>(size_t(n) + 2);  // at most one tile per column, plus the end
    lp->t_tiles_w = wide_p ? ar.take<int2>(size_t(n) + 2) : lp->t_tiles;
    lp->a_vals64 = ar.take<double>(padded(nnz));
    lp->a_vals0 = ar.take<double>(size_t(nnz));
    lp->t_vals64 = ar.take<double>(padded(nnz));
    lp->a_vals32 = mixed ? ar.take<float>(padded(nnz)) : nullptr;
    lp->t_vals32 = mixed ? ar.take<float>(padded(nnz)) : nullptr;
    lp->c_un = ar.take<double>(n);
    lp->l_un = ar.take<double>(n);
    lp->u_un = ar.take<double>(n);
    lp->lo_un = ar.take<double>(m);
    lp->hi_un = ar.take<double>(m);
    lp->c64 = ar.take<double>(n);
    lp->l64 = ar.take<double>(n);
    lp->u64 = ar.take<double>(n);
    lp->lo64 = ar.take<double>(m);
    lp->hi64 = ar.take<double>(m);
    lp->c32 = mixed ? ar.take<float>(n) : nullptr;
    lp->l32 = mixed ? ar.take<float>(n) : nullptr;
    lp->u32 = mixed ? ar.take<float>(n) : nullptr;
    lp->lo32 = mixed ? ar.take<float>(m) : nullptr;
    lp->hi32 = mixed ? ar.take<float>(m) : nullptr;
    lp->R = ar.take<double>(m);
    lp->C = ar.take<double>(n);
    lp->invR = ar.take<double>(m);
    lp->invC = ar.take<double>(n);
    lp->q_un = ar.take<double>(n);
    lp->q64 = ar.take<double>(n);
    lp->q32 = mixed ? ar.take<float>(n) : nullptr;
    lp->R2 = ar.take<double>(std::max(m, n));
    lp->C2 = ar.take<double>(std::max(m, n));
    lp->int_mask = ar.take<uint8_t>(n);
    lp->c_orig = ar.take<double>(n0);
    lp->l_orig = ar.take<double>(n0);
    lp->u_orig = ar.take<double>(n0);
    lp->xhat_d = ar.take<double>(n0);
    lp->kind_d = ar.take<int>(n0);
    lp->aux_of_d = ar.take<int>(n0);
    for (int k = 0; k < 3; ++k) {
      lp->X[k] = ar.take<char>(vs * n);
      lp->Y[k] = ar.take<char>(vs * m);
      lp->AX[k] = ar.take<char>(vs * m);
    }
    for (int k = 0; k < 2; ++k) lp->ATY[k] = ar.take<char>(vs * n);
    lp->XLR = ar.take<char>(vs * n);
    lp->YLR = ar.take<char>(vs * m);
    lp->part_p = ar.take<double>(size_t(kNP) * std::max(cap_p, 1));
    lp->part_d = ar.take<double>(size_t(kND) * std::max(cap_d, 1));
    lp->part_c1 = ar.take<double>(size_t(kNC1) * std::max(cap_c1, 1));
    lp->part_c2 = ar.take<double>(size_t(kNC2) * std::max(lp->grid_c2, 1));
    lp->red_c1 = ar.take<double>(kNC1);
    lp->red = ar.take<double>(4 * size_t(lp->red_blocks));
    lp->io_x = ar.take<double>(n);
    lp->io_y = ar.take<double>(m);
    lp->ctl = ar.take<Control>(1);
    lp->step_fac = ar.take<double>(3 * size_t(lp->p.n_check));  // FP64 factors, then FP32 copies
    lp->pp_part = ar.take<double>(size_t(kPersistentPartials) * std::max(lp->p_grid, 1));
    lp->p_hash = ar.take<unsigned long long>(2);
    lp->grid_bar = ar.take<char>(kGridBarBytes);
    const size_t tc = size_t(lp->p.trace_capacity);
    lp->trace_steps = tc ? ar.take<double>(4 * tc) : nullptr;
    lp->trace_checks = tc ? ar.take<double>(5 * tc) : nullptr;
    const bool inf = lp->p.infeasibility_checks != 0;
    lp->inf_anchor = inf ? ar.take<char>(vs * size_t(std::max(m, int64_t(1)))) : nullptr;
    lp->inf_cand = inf ? ar.take<double>(size_t(std::max(m, int64_t(1)))) : nullptr;
    lp->inf_part = inf ? ar.take<double>(size_t(kNIR + kNIC) * size_t(lp->red_blocks)) : nullptr;
    if (pass == 0) lp->arena_bytes = ar.off + 256;
  }
  cudaStream_t st = lp->st;
  CK(cudaMemsetAsync(lp->arena, 0, lp->arena_bytes, st));
  {
    // one pinned block: the control block's host copy, then the two done flags
    void* pin = nullptr;
    CK(pinned_acquire(&pin));
    lp->h_ctl = static_cast<Control*>(pin);
    lp->h_done = reinterpret_cast<int*>(static_cast<char*>(pin) + sizeof(Control));
  }
  CK(cudaEventCreateWithFlags(&lp->ev_chunk[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&lp->ev_chunk[1], cudaEventDisableTiming));

  CK(cudaMemcpyAsync(lp->a_rowptr, rp.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->a_cols, ci, sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->a_tiles, at.data(), sizeof(int2) * at.size(), cudaMemcpyHostToDevice, st));
  if (wide_d) CK(cudaMemcpyAsync(lp->a_tiles_w, atw.data(), sizeof(int2) * atw.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->a_vals64, va, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  if (nnz > 0) CK(cudaMemcpyAsync(lp->a_vals0, lp->a_vals64, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, st));
  if (host_tp) {
    CK(cudaMemcpyAsync(lp->t_rowptr, tp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lp->t_cols, tr.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lp->t_vals64, tv.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  } else {
    void* scratch = nullptr;
    cudaMemPool_t pool = nullptr;
    CK(handle_pool(lp->device, &pool));
    CK(cudaMallocFromPoolAsync(&scratch, transpose_scratch_bytes(int(n), nnz), pool, st));
    cudaError_t te = transpose_device(int(m), int(n), nnz, lp->a_rowptr, lp->a_cols, lp->a_vals64, lp->t_rowptr,
                                      lp->t_cols, lp->t_vals64, scratch, st);
    cudaFreeAsync(scratch, st);  // back to the pool once the transpose is done
    tp.resize(size_t(n) + 1);
    if (te == cudaSuccess) te = cudaMemcpyAsync(tp.data(), lp->t_rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st);
    if (te == cudaSuccess) te = cudaStreamSynchronize(st);
    CK(te);
  }
  // tiles of the transpose, and the grids that depend on their counts
  {
    const std::vector<int2> tt = build_tiles(tp);
    lp->t_ntiles = int(tt.size()) - 1;
    CK(cudaMemcpyAsync(lp->t_tiles, tt.data(), sizeof(int2) * tt.size(), cudaMemcpyHostToDevice, st));
    std::vector<int2> ttw;
    if (wide_p) {
      ttw = build_tiles(tp, kWideRows);
      CK(cudaMemcpyAsync(lp->t_tiles_w, ttw.data(), sizeof(int2) * ttw.size(), cudaMemcpyHostToDevice, st));
    }
    lp->t_ntiles_w = wide_p ? int(ttw.size()) - 1 : lp->t_ntiles;
    lp->grid_p = grid_of(0, lp->form_p,
                         (lp->form_p == kFormWide || lp->form_p == kFormStaged) ? lp->t_ntiles_w : lp->t_ntiles);
    lp->grid_c1 = grid_of(2, 0, lp->t_ntiles);
    CK(cudaStreamSynchronize(st));  // tt and ttw leave scope
  }
  CK(cudaMemcpyAsync(lp->c_un, cP, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->l_un, lP, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->u_un, uP, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (m > 0) {
    CK(cudaMemcpyAsync(lp->lo_un, loP, sizeof(double) * m, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lp->hi_un, hiP, sizeof(double) * m, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(lp->int_mask, imP, n, cudaMemcpyHostToDevice, st));
  // the original columns are the first n0 of the iterated LP's
  CK(cudaMemcpyAsync(lp->c_orig, lp->c_un, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(lp->l_orig, lp->l_un, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(lp->u_orig, lp->u_un, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  // column kinds (0 continuous, 1 integer, 2 general integer with an auxiliary
  // column) and auxiliary indices: from the integrality mask when there are no
  // auxiliary columns
  std::vector<int> kind, aux_of;
  if (na == 0) {
    CK(column_kinds(n0, lp->int_mask, lp->kind_d, lp->aux_of_d, st));
  } else {
    kind.assign(size_t(n0), 0);
    aux_of.assign(size_t(n0), -1);
    for (int64_t j = 0; j < n0; ++j) kind[size_t(j)] = is_int[j] ? 1 : 0;
    for (int64_t t = 0; t < na; ++t) {
      kind[size_t(lp->gen_int[size_t(t)])] = 2;
      aux_of[size_t(lp->gen_int[size_t(t)])] = int(t);
    }
    CK(cudaMemcpyAsync(lp->kind_d, kind.data(), sizeof(int) * n0, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lp->aux_of_d, aux_of.data(), sizeof(int) * n0, cudaMemcpyHostToDevice, st));
  }
  {
    // preconditioning (Section 2.1, PDLP's diagonal scaling) and scaled copies
    DevSetup s{};
    s.m = int(m); s.n = int(n); s.n_orig = int(n0); s.m_orig = int(m0); s.nnz = int(nnz);
    s.a_rowptr = lp->a_rowptr; s.a_cols = lp->a_cols; s.t_rowptr = lp->t_rowptr; s.t_cols = lp->t_cols;
    s.a_tiles = lp->a_tiles; s.a_ntiles = lp->a_ntiles; s.t_tiles = lp->t_tiles; s.t_ntiles = lp->t_ntiles;
    s.a_vals64 = lp->a_vals64; s.t_vals64 = lp->t_vals64; s.a_vals32 = lp->a_vals32; s.t_vals32 = lp->t_vals32;
    s.R = lp->R; s.C = lp->C; s.R2 = lp->R2; s.C2 = lp->C2; s.red = lp->red; s.red_blocks = lp->red_blocks;
    CK(launch_precondition(s, lp->p.ruiz_iters, lp->p.pock_chambolle != 0, st));
    CK(launch_scale_values(s, st));
    DevVecs v{};
    v.c = lp->c_un; v.lo = lp->lo_un; v.hi = lp->hi_un; v.l = lp->l_un; v.u = lp->u_un;
    v.c64 = lp->c64; v.lo64 = lp->lo64; v.hi64 = lp->hi64; v.l64 = lp->l64; v.u64 = lp->u64;
    v.c32 = lp->c32; v.lo32 = lp->lo32; v.hi32 = lp->hi32; v.l32 = lp->l32; v.u32 = lp->u32;
    v.R = lp->R; v.C = lp->C; v.invR = lp->invR; v.invC = lp->invC; v.m = int(m); v.n = int(n);
    CK(launch_scale_vectors(v, st));
    SetupNorms nm{};
    CK(setup_norms(s, lp->c64, lp->lo64, lp->hi64, st, &nm));
    // initial step size: 1/max|a~| (adaptive) or f/||A~||_F (fixed); primal weight
    // ||c~|| / ||q~|| on the scaled LP, q~_i the largest finite row bound magnitude
    // (1 when either norm is zero)
    double eta = 1.0;
    if (lp->p.adaptive_step) eta = nm.amax > 0.0 ? 1.0 / nm.amax : 1.0;
    else eta = nm.fro2 > 0.0 ? lp->p.fixed_step_factor / std::sqrt(nm.fro2) : 1.0;
    const double cn = std::sqrt(nm.c2), qn = std::sqrt(nm.q2);
    Control h{};
    h.eta = eta;
    h.omega = (cn > 0.0 && qn > 0.0) ? cn / qn : 1.0;
    lp->eta0 = h.eta;
    lp->omega0 = h.omega;
    h.ix_cur = 0; h.ix_next = 1; h.ix_avg = 2; h.ia_cur = 0; h.ia_avg = 1;
    h.adaptive = lp->p.adaptive_step ? 1 : 0;
    h.restarts_on = lp->p.restarts ? 1 : 0;
    h.pw_update = lp->p.primal_weight_update ? 1 : 0;
    h.beta_s = lp->p.beta_sufficient; h.beta_n = lp->p.beta_necessary; h.beta_a = lp->p.beta_artificial;
    h.theta = lp->p.pw_smoothing; h.exp_red = lp->p.step_reduction_exp; h.exp_grow = lp->p.step_growth_exp;
    h.done = 1;
    h.inf_gap = -kInf;  // no candidate ray tested yet
    *lp->h_ctl = h;
    CK(cudaMemcpyAsync(lp->ctl, lp->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, st));
    // c_hat = c (already in c_un), offset 0; norms of c and of the row bounds
    const DevObjective o = lp->objective_desc();
    CK(launch_objective_norms(o, 0.0, st));
  }
  if (mixed) {
    fill_dev<float>(lp->d32, lp);
    CK(launch_init_point<float>(lp->d32, st));
  } else {
    fill_dev<double>(lp->d64, lp);
    CK(launch_init_point<double>(lp->d64, st));
  }
  CK(cudaStreamSynchronize(st));
  if (lp->tune) {
    const int rc = mixed ? autotune_form<float>(lp) : autotune_form<double>(lp);
    if (rc != SCYLLA_OK) return rc;
  }
  return SCYLLA_OK;
}

namespace {
template <typename T>
void fill_dev(DevLP<T>& d, scylla_lp* lp) {
  const bool mixed = lp->p.precision == SCYLLA_PREC_MIXED;
  d.m = lp->m;
  d.n = lp->n;
  d.a_rowptr = lp->a_rowptr; d.a_cols = lp->a_cols; d.a_tiles = lp->a_tiles; d.a_ntiles = lp->a_ntiles;
  d.t_rowptr = lp->t_rowptr; d.t_cols = lp->t_cols; d.t_tiles = lp->t_tiles; d.t_ntiles = lp->t_ntiles;
  d.a_tiles_w = lp->a_tiles_w; d.a_ntiles_w = lp->a_ntiles_w; d.t_tiles_w = lp->t_tiles_w; d.t_ntiles_w = lp->t_ntiles_w;
  d.a_vals64 = lp->a_vals64;
  d.t_vals64 = lp->t_vals64;
  if (mixed) {
    d.a_vals = reinterpret_cast<const T*>(lp->a_vals32);
    d.t_vals = reinterpret_cast<const T*>(lp->t_vals32);
    d.c = reinterpret_cast<const T*>(lp->c32);
    d.l = reinterpret_cast<const T*>(lp->l32);
    d.u = reinterpret_cast<const T*>(lp->u32);
    d.lo = reinterpret_cast<const T*>(lp->lo32);
    d.hi = reinterpret_cast<const T*>(lp->hi32);
  } else {
    d.a_vals = reinterpret_cast<const T*>(lp->a_vals64);
    d.t_vals = reinterpret_cast<const T*>(lp->t_vals64);
    d.c = reinterpret_cast<const T*>(lp->c64);
    d.l = reinterpret_cast<const T*>(lp->l64);
    d.u = reinterpret_cast<const T*>(lp->u64);
    d.lo = reinterpret_cast<const T*>(lp->lo64);
    d.hi = reinterpret_cast<const T*>(lp->hi64);
  }
  d.c64 = lp->c64; d.l64 = lp->l64; d.u64 = lp->u64; d.lo64 = lp->lo64; d.hi64 = lp->hi64;
  d.R = lp->R;
  d.C = lp->C;
  d.invR = lp->invR;
  d.invC = lp->invC;
  d.int_mask = lp->int_mask;
  for (int k = 0; k < 3; ++k) {
    d.X[k] = reinterpret_cast<T*>(lp->X[k]);
    d.Y[k] = reinterpret_cast<T*>(lp->Y[k]);
    d.AX[k] = reinterpret_cast<T*>(lp->AX[k]);
  }
  for (int k = 0; k < 2; ++k) d.ATY[k] = reinterpret_cast<T*>(lp->ATY[k]);
  d.XLR = reinterpret_cast<T*>(lp->XLR);
  d.YLR = reinterpret_cast<T*>(lp->YLR);
  d.ctl = lp->ctl;
  d.part_p = lp->part_p; d.part_d = lp->part_d; d.part_c1 = lp->part_c1; d.part_c2 = lp->part_c2; d.red_c1 = lp->red_c1;
  d.grid_p = lp->grid_p; d.grid_d = lp->grid_d; d.grid_c1 = lp->grid_c1; d.grid_c2 = lp->grid_c2;
  d.step_fac = lp->step_fac;
  d.pp_part = lp->pp_part;
  d.p_hash = lp->p_hash;
  d.n_check = lp->p.n_check;
  d.pdl = lp->p.pdl ? 1 : 0;
  d.form_p = lp->form_p;
  d.form_d = lp->form_d;
  d.wait_ns = (unsigned long long)(lp->p.device_wait_limit_s * 1e9);
  d.trace_steps = lp->trace_steps;
  d.trace_checks = lp->trace_checks;
  d.trace_cap = lp->p.trace_capacity;
  d.inf_anchor = reinterpret_cast<T*>(lp->inf_anchor);
  d.inf_cand = lp->inf_cand;
  d.inf_part = lp->inf_part;
  d.inf_grid = lp->red_blocks;
}
}  // namespace

DevObjective scylla_lp::objective_desc() {
  DevObjective o{};
  o.n_orig = int(n0); o.m_orig = int(m0); o.n = n; o.m = m;
  o.c_orig = c_orig; o.l_orig = l_orig; o.u_orig = u_orig; o.kind = kind_d; o.aux_of = aux_of_d; o.xhat = xhat_d;
  o.chat = c_un; o.lo_unscaled = lo_un; o.hi_unscaled = hi_un; o.R = R; o.C = C;
  o.c64 = c64; o.lo64 = lo64; o.c32 = c32; o.lo32 = lo32; o.red = red; o.red_blocks = red_blocks; o.ctl = ctl;
  o.l2 = p.distance == 2 ? 1 : 0;
  o.q_un = q_un; o.q64 = q64; o.q32 = q32;
  return o;
}

void scylla_lp::drop_graphs() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  if (chunk_exec) cudaGraphExecDestroy(chunk_exec);
  if (chunk_graph) cudaGraphDestroy(chunk_graph);
  chunk_exec = nullptr;
  chunk_graph = nullptr;
}

void scylla_lp::set_qp_active(bool on) {
  if (on == qp_active) return;
  qp_active = on;
  d64.q = on ? q64 : nullptr;
  d64.q64 = on ? q64 : nullptr;
  d32.q = on ? q32 : nullptr;
  d32.q64 = on ? q64 : nullptr;
  drop_graphs();  // they captured the kernels' parameters
}

void scylla_lp::release() {
  if (prop_mem) cudaFree(prop_mem);
  prop_mem = nullptr;
  if (prop_count_h) cudaFreeHost(prop_count_h);
  prop_count_h = nullptr;
  if (repair_lp) {
    cudaStreamSynchronize(repair_lp->st);
    repair_lp->release();
    delete repair_lp;
    repair_lp = nullptr;
  }
  drop_graphs();
  for (auto& e : ev_chunk) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  h_done = nullptr;  // inside the h_ctl block
  if (arena) cudaFreeAsync(arena, st);  // to the pool, after the stream's work
  arena = nullptr;
  pinned_release(h_ctl);
  h_ctl = nullptr;
  if (ev_user) cudaEventDestroy(ev_user);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  ev_user = ev0 = ev1 = nullptr;
  if (st) cudaStreamDestroy(st);
  st = nullptr;
}

extern "C" int scylla_lp_create(const scylla_csr* A, const double* c, const double* row_lo, const double* row_hi,
                                const double* col_lo, const double* col_hi, const uint8_t* is_integer,
                                const scylla_params* p, void* cuda_stream, scylla_lp** out) {
  if (!out) FAIL(SCYLLA_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  int rc = validate_lp(A, c, row_lo, row_hi, col_lo, col_hi, is_integer);
  if (rc != SCYLLA_OK) return rc;
  scylla_params dp;
  scylla_default_params(&dp);
  scylla_lp* lp = nullptr;
  try {
    lp = new scylla_lp();
    rc = create_impl(A, c, row_lo, row_hi, col_lo, col_hi, is_integer, p ? p : &dp, cuda_stream, lp);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    rc = SCYLLA_ERR_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    rc = SCYLLA_ERR_INVALID_ARG;
  }
  if (rc != SCYLLA_OK) {
    if (lp) {
      lp->release();
      delete lp;
    }
    return rc;
  }
  *out = lp;
  return SCYLLA_OK;
}

extern "C" void scylla_lp_destroy(scylla_lp* lp) {
  if (!lp) return;
  cudaStreamSynchronize(lp->st);
  lp->release();
  delete lp;
}

extern "C" int scylla_lp_dims(const scylla_lp* lp, int64_t* m_total, int64_t* n_total, int64_t* nnz_total,
                              int64_t* n_aux) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  if (m_total) *m_total = lp->m;
  if (n_total) *n_total = lp->n;
  if (nnz_total) *nnz_total = lp->nnz;
  if (n_aux) *n_aux = lp->n_aux;
  return SCYLLA_OK;
}

// -------------------------------------------------------------------- solve ---
int scylla_lp::order_after_user() {
  if (user_st) {
    CK(cudaEventRecord(ev_user, user_st));
    CK(cudaStreamWaitEvent(st, ev_user, 0));
  }
  return SCYLLA_OK;
}

// Both builders leave the handle without a graph of their kind when a step fails
// (the caller's next solve builds it again): the executable is instantiated into a
// local and stored only on success, and a failed build drops what was made.
template <typename T>
static int build_graph_steps(scylla_lp* lp, const DevLP<T>& d) {
  cudaStream_t st = lp->st;
  CK(cudaGraphCreate(&lp->graph, 0));
  CK(cudaGraphConditionalHandleCreate(&lp->cond, lp->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = lp->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, lp->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < lp->p.n_check && e == cudaSuccess; ++s) e = launch_slot<T>(d, st);
  if (e == cudaSuccess) e = launch_check<T>(d, st);
  if (e == cudaSuccess) e = launch_loop_ctl(lp->ctl, lp->cond, st);
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &captured);
  CK(e);
  CK(e2);
  cudaGraphExec_t exec = nullptr;
  CK(cudaGraphInstantiate(&exec, lp->graph, 0));
  lp->exec = exec;
  return SCYLLA_OK;
}

template <typename T>
static int build_graph(scylla_lp* lp, const DevLP<T>& d) {
  const int rc = build_graph_steps<T>(lp, d);
  if (rc != SCYLLA_OK) {
    if (lp->graph) cudaGraphDestroy(lp->graph);
    lp->graph = nullptr;
    lp->exec = nullptr;
  }
  return rc;
}

template <typename T>
static int build_chunk_graph(scylla_lp* lp, const DevLP<T>& d) {
  cudaStream_t st = lp->st;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < lp->p.n_check && e == cudaSuccess; ++s) e = launch_slot<T>(d, st);
  if (e == cudaSuccess) e = launch_check<T>(d, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    CK(e);
    CK(e2);
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e3 = cudaGraphInstantiate(&exec, g, 0);
  if (e3 != cudaSuccess) {
    cudaGraphDestroy(g);
    CK(e3);
  }
  lp->chunk_graph = g;
  lp->chunk_exec = exec;
  return SCYLLA_OK;
}

template <typename T>
static int solve_impl(scylla_lp* lp, const DevLP<T>& d, double tol, int64_t iter_limit, int stall_checks) {
  cudaStream_t st = lp->st;
  const long long nchk = lp->p.n_check;
  const long long max_chunks = (iter_limit + nchk - 1) / nchk + 2;
  CK(cudaEventRecord(lp->ev0, st));
  CK(launch_solve_init<T>(d, tol, (long long)iter_limit, stall_checks, max_chunks, st));
  long long launches = 1;
  // the persistent kernel has no infeasibility detection: with it on, chunk graphs
  if (lp->p.use_graph == 3 && lp->p_grid > 0 && !lp->inf_cand) {
    // one cooperative launch evaluates the start point and runs every attempt
    CK(cudaMemsetAsync(lp->grid_bar, 0, kGridBarBytes, st));
    CK(cudaMemsetAsync(lp->p_hash, 0, 2 * sizeof(unsigned long long), st));
    CK(launch_persistent<T>(d, lp->grid_bar, lp->p_grid, lp->p.device_wait_limit_s, st));
    lp->last_launches = 2;
    CK(cudaEventRecord(lp->ev1, st));
    CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SCYLLA_OK;
  }
  CK(launch_check<T>(d, st));  // evaluates the start point, caches A x and A^T y
  const long long per_chunk = 2LL * nchk + 2;
  launches = 3;
  if (lp->p.use_graph == 2) {
    if (!lp->exec) {
      const int rc = build_graph<T>(lp, d);
      if (rc != SCYLLA_OK) return rc;
    }
    CK(cudaGraphLaunch(lp->exec, st));
    launches = -1;  // counted on the device
  } else if (lp->p.use_graph == 1 || lp->p.use_graph == 3) {
    if (!lp->chunk_exec) {
      const int rc = build_chunk_graph<T>(lp, d);
      if (rc != SCYLLA_OK) return rc;
    }
    // chunk c+1 is queued before the done flag of chunk c is read, so the GPU never
    // waits for the host; the chunk queued after the last one returns at once
    auto enqueue = [&](long long c) -> cudaError_t {
      cudaError_t e = cudaGraphLaunch(lp->chunk_exec, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&lp->h_done[c & 1], &lp->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(lp->ev_chunk[c & 1], st);
      launches += per_chunk;
      return e;
    };
    CK(enqueue(0));
    for (long long c = 0; c < max_chunks; ++c) {
      if (c + 1 < max_chunks) CK(enqueue(c + 1));
      CK(cudaEventSynchronize(lp->ev_chunk[c & 1]));
      if (lp->h_done[c & 1]) break;
    }
  } else {
    for (long long ch = 0; ch < max_chunks; ++ch) {
      CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (lp->h_ctl->done) break;
      for (int s = 0; s < lp->p.n_check; ++s) CK(launch_slot<T>(d, st));
      CK(launch_check<T>(d, st));
      launches += per_chunk;
    }
  }
  lp->last_launches = launches;
  CK(cudaEventRecord(lp->ev1, st));
  CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

int scylla_lp::solve(double tol, int64_t iter_limit, int stall_checks, scylla_pdhg_result* out) {
  int rc = order_after_user();
  if (rc != SCYLLA_OK) return rc;
  rc = (p.precision == SCYLLA_PREC_MIXED) ? solve_impl<float>(this, d32, tol, iter_limit, stall_checks)
                                          : solve_impl<double>(this, d64, tol, iter_limit, stall_checks);
  if (rc != SCYLLA_OK) return rc;
  Control& h = *h_ctl;
  if (!h.done) FAIL(SCYLLA_ERR_CUDA, "solve ended without a final check");
  if (h.status == SCYLLA_DEVICE_TIMEOUT) FAIL(SCYLLA_ERR_TIMEOUT, "a device-side barrier wait ran out of time");
  // a ray the device found is accepted only when the host's compensated test on the
  // original data confirms it (D > 0); with auxiliary distance rows the ray also weighs
  // rows the host copy does not hold, and the device's test stands
  if (h.status == SCYLLA_INFEASIBLE && n_aux == 0 && m0 > 0) {
    const int rh = ensure_host_matrix();
    if (rh != SCYLLA_OK) return rh;
    ensure_columns();
    std::vector<double> ray(static_cast<size_t>(m0));
    if (p.precision == SCYLLA_PREC_MIXED) CK(launch_get_cert<float>(d32, io_y, int(m0), st));
    else CK(launch_get_cert<double>(d64, io_y, int(m0), st));
    CK(cudaMemcpyAsync(ray.data(), io_y, sizeof(double) * m0, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!(scylla::farkas_gap_host(*this, ray.data()) > 0.0)) {
      h.status = SCYLLA_NUMERICAL;
      set_error("the device's dual ray failed the host test of a certificate");
    }
  }
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->status = h.status;
    out->used_average = h.used_avg;
    out->iterations = h.k;
    out->accepted = h.accepted;
    out->rejected = h.rejected;
    out->restarts = h.restarts;
    out->eps_p = h.eps_p;
    out->eps_d = h.eps_d;
    out->eps_g = h.eps_g;
    out->rel_kkt = h.rel_kkt;
    out->pobj = h.pobj;
    out->dobj = h.dobj;
    out->eta = h.eta;
    out->omega = h.omega;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    out->seconds = ms * 1e-3;
    out->launches = last_launches >= 0 ? last_launches : 3 + h.chunks * (2LL * p.n_check + 3);
    out->kernel_form = api_form(form_p);
    out->kernel_form_dual = api_form(form_d);
  }
  return SCYLLA_OK;
}

extern "C" int scylla_pdhg_solve(scylla_lp* lp, double tol, int64_t iter_limit, scylla_pdhg_result* out) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  if (!(tol >= 0.0)) FAIL(SCYLLA_ERR_INVALID_ARG, "tol must be >= 0");
  if (iter_limit < 0) FAIL(SCYLLA_ERR_INVALID_ARG, "iter_limit must be >= 0");
  return lp->solve(tol, iter_limit, lp->p.stall_checks, out);
}

// ---------------------------------------------------------- objective update ---
int scylla_lp::set_objective(const double* xhat, int32_t K) {
  if (!xhat) FAIL(SCYLLA_ERR_INVALID_ARG, "xhat is null");
  if (K < 1) FAIL(SCYLLA_ERR_INVALID_ARG, "round K must be >= 1");
  const int rv = ensure_host_vectors();
  if (rv != SCYLLA_OK) return rv;
  for (int64_t j = 0; j < n0; ++j) {
    if (!std::isfinite(xhat[j])) FAIL(SCYLLA_ERR_INVALID_ARG, "xhat not finite at " + std::to_string(j));
    if (int0[j] && (xhat[j] != std::floor(xhat[j]) || xhat[j] < l0[j] || xhat[j] > u0[j]))
      FAIL(SCYLLA_ERR_INVALID_ARG, "xhat not integral within bounds at integer column " + std::to_string(j));
  }
  int rc = order_after_user();
  if (rc != SCYLLA_OK) return rc;
  CK(cudaMemcpyAsync(xhat_d, xhat, sizeof(double) * n0, cudaMemcpyHostToDevice, st));
  const double aK = std::pow(p.alpha, double(K));
  const double s = c0norm > 0.0 ? std::sqrt(double(n_int)) / c0norm : 0.0;
  CK(launch_objective_update(objective_desc(), aK * s, 1.0 - aK, st));
  CK(cudaStreamSynchronize(st));
  if (p.distance == 2) set_qp_active(true);  // the l2 update writes a Hessian
  return SCYLLA_OK;
}

extern "C" int scylla_set_qp_objective(scylla_lp* lp, const double* c, const double* q, double offset) {
  if (!lp || !c || !q) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (!std::isfinite(offset)) FAIL(SCYLLA_ERR_INVALID_ARG, "offset not finite");
  bool any_q = false;
  for (int64_t j = 0; j < lp->n0; ++j) {
    if (!std::isfinite(c[j])) FAIL(SCYLLA_ERR_INVALID_ARG, "non-finite objective at column " + std::to_string(j));
    if (!(std::isfinite(q[j]) && q[j] >= 0.0))
      FAIL(SCYLLA_ERR_INVALID_ARG, "Hessian diagonal must be finite and >= 0 (column " + std::to_string(j) + ")");
    any_q = any_q || q[j] > 0.0;
  }
  int rc = lp->order_after_user();
  if (rc != SCYLLA_OK) return rc;
  cudaStream_t st = lp->st;
  CK(cudaMemcpyAsync(lp->c_un, c, sizeof(double) * lp->n0, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(lp->q_un, 0, sizeof(double) * lp->n, st));
  CK(cudaMemcpyAsync(lp->q_un, q, sizeof(double) * lp->n0, cudaMemcpyHostToDevice, st));
  CK(scale_objective(lp->n, lp->c_un, lp->q_un, lp->C, lp->c64, lp->c32, lp->q64, lp->q32, st));
  CK(launch_objective_norms(lp->objective_desc(), offset, st));
  CK(cudaStreamSynchronize(st));
  lp->set_qp_active(any_q);
  return SCYLLA_OK;
}

extern "C" int scylla_set_objective(scylla_lp* lp, const double* xhat, int32_t K) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  return lp->set_objective(xhat, K);
}

extern "C" int scylla_get_objective(const scylla_lp* lp, double* c_hat, double* offset) {
  if (!lp || !c_hat) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(c_hat, lp->c_un, sizeof(double) * lp->n, cudaMemcpyDeviceToHost, lp->st));
  CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, lp->st));
  CK(cudaStreamSynchronize(lp->st));
  if (offset) *offset = lp->h_ctl->offset;
  return SCYLLA_OK;
}

// ------------------------------------------------------------- state access ---
int scylla_lp::fetch_x(double* host, int count) {
  if (p.precision == SCYLLA_PREC_MIXED) CK(launch_get_x<float>(d32, io_x, count, st));
  else CK(launch_get_x<double>(d64, io_x, count, st));
  if (host) {
    CK(cudaMemcpyAsync(host, io_x, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return SCYLLA_OK;
}

int scylla_lp::fetch_y(double* host, int count) {
  if (p.precision == SCYLLA_PREC_MIXED) CK(launch_get_y<float>(d32, io_y, count, st));
  else CK(launch_get_y<double>(d64, io_y, count, st));
  CK(cudaMemcpyAsync(host, io_y, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

extern "C" int scylla_get_certificate(const scylla_lp* lp, double* y, double* gap, double* scale) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  if (!lp->inf_cand) FAIL(SCYLLA_ERR_INVALID_ARG, "the handle was created without infeasibility_checks");
  scylla_lp* h = const_cast<scylla_lp*>(lp);
  cudaStream_t st = h->st;
  if (y && lp->m0 > 0) {
    if (lp->p.precision == SCYLLA_PREC_MIXED) CK(launch_get_cert<float>(h->d32, h->io_y, int(lp->m0), st));
    else CK(launch_get_cert<double>(h->d64, h->io_y, int(lp->m0), st));
    CK(cudaMemcpyAsync(y, h->io_y, sizeof(double) * lp->m0, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (gap) *gap = h->h_ctl->inf_gap;
  if (scale) *scale = h->h_ctl->inf_scale;
  return SCYLLA_OK;
}

extern "C" int scylla_get_primal(const scylla_lp* lp, double* x) {
  if (!lp || !x) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  return const_cast<scylla_lp*>(lp)->fetch_x(x, int(lp->n0));
}

extern "C" int scylla_get_dual(const scylla_lp* lp, double* y) {
  if (!lp || (!y && lp->m0 > 0)) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (lp->m0 == 0) return SCYLLA_OK;
  return const_cast<scylla_lp*>(lp)->fetch_y(y, int(lp->m0));
}

extern "C" int scylla_get_primal_device(const scylla_lp* lp, double* x_device) {
  if (!lp || !x_device) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  scylla_lp* h = const_cast<scylla_lp*>(lp);
  int rc = h->fetch_x(nullptr, int(lp->n0));
  if (rc != SCYLLA_OK) return rc;
  CK(cudaMemcpyAsync(x_device, h->io_x, sizeof(double) * lp->n0, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SCYLLA_OK;
}

extern "C" int scylla_get_state(const scylla_lp* lp, double* x, double* y, double* eta, double* omega) {
  if (!lp || !x || (!y && lp->m > 0)) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  scylla_lp* h = const_cast<scylla_lp*>(lp);
  int rc = h->fetch_x(x, lp->n);
  if (rc != SCYLLA_OK) return rc;
  if (lp->m > 0) {
    rc = h->fetch_y(y, lp->m);
    if (rc != SCYLLA_OK) return rc;
  }
  CK(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (eta) *eta = h->h_ctl->eta;
  if (omega) *omega = h->h_ctl->omega;
  return SCYLLA_OK;
}

extern "C" int scylla_set_state(scylla_lp* lp, const double* x, const double* y, double eta, double omega) {
  if (!lp || !x || (!y && lp->m > 0)) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (!(eta > 0.0) || !(omega > 0.0) || !std::isfinite(eta) || !std::isfinite(omega))
    FAIL(SCYLLA_ERR_INVALID_ARG, "eta and omega must be positive and finite");
  for (int j = 0; j < lp->n; ++j)
    if (!std::isfinite(x[j])) FAIL(SCYLLA_ERR_INVALID_ARG, "x not finite");
  for (int i = 0; i < lp->m; ++i)
    if (!std::isfinite(y[i])) FAIL(SCYLLA_ERR_INVALID_ARG, "y not finite");
  cudaStream_t st = lp->st;
  CK(cudaMemcpyAsync(lp->io_x, x, sizeof(double) * lp->n, cudaMemcpyHostToDevice, st));
  if (lp->m > 0) CK(cudaMemcpyAsync(lp->io_y, y, sizeof(double) * lp->m, cudaMemcpyHostToDevice, st));
  if (lp->p.precision == SCYLLA_PREC_MIXED) CK(launch_set_xy<float>(lp->d32, lp->io_x, lp->io_y, st));
  else CK(launch_set_xy<double>(lp->d64, lp->io_x, lp->io_y, st));
  CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  lp->h_ctl->eta = eta;
  lp->h_ctl->omega = omega;
  CK(cudaMemcpyAsync(lp->ctl, lp->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

extern "C" int scylla_get_scaling(const scylla_lp* lp, double* R, double* C) {
  if (!lp || !C || (!R && lp->m > 0)) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (lp->m > 0) CK(cudaMemcpyAsync(R, lp->R, sizeof(double) * lp->m, cudaMemcpyDeviceToHost, lp->st));
  CK(cudaMemcpyAsync(C, lp->C, sizeof(double) * lp->n, cudaMemcpyDeviceToHost, lp->st));
  CK(cudaStreamSynchronize(lp->st));
  return SCYLLA_OK;
}

extern "C" int scylla_get_transpose(const scylla_lp* lp, int64_t* colptr, int32_t* rows, double* vals) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  if (colptr) {
    std::vector<int> tp(size_t(lp->n) + 1);
    CK(cudaMemcpyAsync(tp.data(), lp->t_rowptr, sizeof(int) * tp.size(), cudaMemcpyDeviceToHost, lp->st));
    CK(cudaStreamSynchronize(lp->st));
    for (size_t j = 0; j < tp.size(); ++j) colptr[j] = tp[j];
  }
  if (rows && lp->nnz > 0)
    CK(cudaMemcpyAsync(rows, lp->t_cols, sizeof(int32_t) * lp->nnz, cudaMemcpyDeviceToHost, lp->st));
  if (vals && lp->nnz > 0)
    CK(cudaMemcpyAsync(vals, lp->t_vals64, sizeof(double) * lp->nnz, cudaMemcpyDeviceToHost, lp->st));
  CK(cudaStreamSynchronize(lp->st));
  return SCYLLA_OK;
}

extern "C" int scylla_get_trace(const scylla_lp* lp, double* steps, int64_t* n_steps, double* checks,
                                int64_t* n_checks) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  const int64_t cap = lp->p.trace_capacity;
  scylla_lp* h = const_cast<scylla_lp*>(lp);
  CK(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int64_t ns = std::min<int64_t>(cap, h->h_ctl->k), nc = std::min<int64_t>(cap, h->h_ctl->n_ctrace);
  if (steps && ns > 0) CK(cudaMemcpy(steps, h->trace_steps, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost));
  if (checks && nc > 0) CK(cudaMemcpy(checks, h->trace_checks, sizeof(double) * 5 * nc, cudaMemcpyDeviceToHost));
  if (n_steps) *n_steps = ns;
  if (n_checks) *n_checks = nc;
  return SCYLLA_OK;
}

// ------------------------------------------------------ column bounds, repair ---
int scylla_lp::set_col_bounds(const double* l, const double* u) {
  root_prop.reset();
  int rc = order_after_user();
  if (rc != SCYLLA_OK) return rc;
  CK(cudaMemcpyAsync(l_un, l, sizeof(double) * n0, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(u_un, u, sizeof(double) * n0, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(l_orig, l_un, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(u_orig, u_un, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  CK(scale_col_bounds(n0, l_un, u_un, C, l64, u64, l32, u32, st));
  if (host_vectors_ready) {
    l0.assign(l, l + n0);
    u0.assign(u, u + n0);
  }
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

int scylla_lp::set_row_bounds(const double* lo, const double* hi) {
  root_prop.reset();
  int rc = order_after_user();
  if (rc != SCYLLA_OK) return rc;
  if (m0 > 0) {
    CK(cudaMemcpyAsync(lo_un, lo, sizeof(double) * m0, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(hi_un, hi, sizeof(double) * m0, cudaMemcpyHostToDevice, st));
    CK(scale_row_bounds(m0, lo_un, hi_un, R, lo64, hi64, lo32, hi32, st));
  }
  // ||b|| from the new bounds; c_hat and the offset stay
  CK(cudaMemcpyAsync(h_ctl, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(launch_objective_norms(objective_desc(), h_ctl->offset, st));
  if (host_vectors_ready) {
    lo0.assign(lo, lo + m0);
    hi0.assign(hi, hi + m0);
  }
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

// ------------------------------------------------------------ propagation ---
// rounds of the propagation that screens a repair's fixing (its verdict of
// infeasibility holds at any round)
constexpr int64_t kRepairPropagationRounds = 1000;

// the buffers of the device propagation, allocated and filled on first use: perm over
// the transpose's entries, proposals at A's positions, domains, row states, two
// active-row masks, three counters.  The handle takes them only once every step has
// succeeded, so a failed first call leaves nothing half set up.
static int ensure_prop_buffers(scylla_lp* lp) {
  if (lp->prop_mem) return SCYLLA_OK;
  const int64_t m0 = lp->m0, n0 = lp->n0;
  const size_t nnz = size_t(lp->nnz);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_perm = take(sizeof(int) * (nnz + 1)), o_plb = take(sizeof(double) * (nnz + 1)),
               o_pub = take(sizeof(double) * (nnz + 1)), o_dl = take(sizeof(double) * size_t(n0 + 1)),
               o_du = take(sizeof(double) * size_t(n0 + 1)), o_st = take(size_t(m0 + 1)),
               o_a0 = take(size_t(m0 + 1)), o_a1 = take(size_t(m0 + 1)),
               o_cnt = take(3 * sizeof(unsigned long long));
  void* mem = nullptr;
  unsigned long long* count_h = nullptr;
  cudaError_t e = cudaMalloc(&mem, off);
  if (e == cudaSuccess) e = cudaMallocHost(&count_h, 3 * sizeof(unsigned long long));
  PropDev P{};
  if (e == cudaSuccess) {
    char* b = static_cast<char*>(mem);
    P.m = int(m0);
    P.n = int(n0);
    P.rowptr = lp->a_rowptr;
    P.cols = lp->a_cols;
    P.vals = lp->a_vals0;
    P.t_rowptr = lp->t_rowptr;
    P.t_rows = lp->t_cols;
    int* perm = reinterpret_cast<int*>(b + o_perm);
    P.perm = perm;
    P.is_int = lp->int_mask;
    P.plb = reinterpret_cast<double*>(b + o_plb);
    P.pub = reinterpret_cast<double*>(b + o_pub);
    P.dl = reinterpret_cast<double*>(b + o_dl);
    P.du = reinterpret_cast<double*>(b + o_du);
    P.state = reinterpret_cast<unsigned char*>(b + o_st);
    P.count = reinterpret_cast<unsigned long long*>(b + o_cnt);
    e = propagate_perm(int(n0), lp->t_rowptr, lp->t_cols, lp->a_rowptr, lp->a_cols, perm, lp->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lp->st);
  }
  if (e != cudaSuccess) {
    if (mem) cudaFree(mem);
    if (count_h) cudaFreeHost(count_h);
    set_error(std::string("device propagation buffers: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SCYLLA_ERR_OOM : SCYLLA_ERR_CUDA;
  }
  char* b = static_cast<char*>(mem);
  lp->prop = P;
  lp->prop_active[0] = reinterpret_cast<unsigned char*>(b + o_a0);
  lp->prop_active[1] = reinterpret_cast<unsigned char*>(b + o_a1);
  lp->prop_count_h = count_h;
  lp->prop_mem = mem;
  return SCYLLA_OK;
}

static int propagate_impl(scylla_lp* lp, double* dl, double* du, uint8_t* ignored, int64_t max_rounds,
                          int64_t* rounds_out, int64_t* conflicts_out) {
  const int64_t m0 = lp->m0, n0 = lp->n0;
  cudaStream_t st = lp->st;
  int rc = lp->order_after_user();
  if (rc != SCYLLA_OK) return rc;
  rc = ensure_prop_buffers(lp);
  if (rc != SCYLLA_OK) return rc;
  PropDev& P = lp->prop;
  P.lo = lp->lo_un;  // the current original row bounds come first
  P.hi = lp->hi_un;
  CK(cudaMemcpyAsync(P.dl, dl, sizeof(double) * n0, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P.du, du, sizeof(double) * n0, cudaMemcpyHostToDevice, st));
  if (m0 > 0) {
    CK(cudaMemsetAsync(P.state, 0, size_t(m0), st));
    CK(cudaMemsetAsync(lp->prop_active[0], 1, size_t(m0), st));
  }
  int64_t rounds = 0, conflicts = 0;
  int cur = 0;
  while (m0 > 0 && rounds < max_rounds) {
    ++rounds;
    CK(propagate_round(P, lp->prop_active[cur], lp->prop_active[cur ^ 1], st));
    CK(cudaMemcpyAsync(lp->prop_count_h, P.count, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    conflicts += int64_t(lp->prop_count_h[1]);
    if (lp->prop_count_h[2] == 0) break;  // no row is active next
    cur ^= 1;
  }
  CK(cudaMemcpyAsync(dl, P.dl, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(du, P.du, sizeof(double) * n0, cudaMemcpyDeviceToHost, st));
  std::vector<unsigned char> state(static_cast<size_t>(m0));
  if (ignored && m0 > 0) CK(cudaMemcpyAsync(state.data(), P.state, size_t(m0), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (ignored)
    for (int64_t i = 0; i < m0; ++i) ignored[i] = state[size_t(i)] == 2 ? 1 : 0;
  if (rounds_out) *rounds_out = rounds;
  if (conflicts_out) *conflicts_out = conflicts;
  return SCYLLA_OK;
}

extern "C" int scylla_propagate(scylla_lp* lp, double* dom_lo, double* dom_hi, uint8_t* ignored_rows,
                                int64_t max_rounds, int64_t* rounds, int64_t* conflicts) {
  if (!lp || !dom_lo || !dom_hi) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (max_rounds < 1) FAIL(SCYLLA_ERR_INVALID_ARG, "max_rounds must be >= 1");
  for (int64_t j = 0; j < lp->n0; ++j)
    if (std::isnan(dom_lo[j]) || std::isnan(dom_hi[j]) || dom_lo[j] > dom_hi[j])
      FAIL(SCYLLA_ERR_INVALID_ARG, "invalid domain at column " + std::to_string(j));
  try {
    return propagate_impl(lp, dom_lo, dom_hi, ignored_rows, max_rounds, rounds, conflicts);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
}

extern "C" int scylla_set_row_bounds(scylla_lp* lp, const double* row_lo, const double* row_hi) {
  if (!lp || ((!row_lo || !row_hi) && lp->m0 > 0)) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  for (int64_t i = 0; i < lp->m0; ++i) {
    const double a = row_lo[i], b = row_hi[i];
    if (std::isnan(a) || std::isnan(b) || a > b || a == kInf || b == -kInf)
      FAIL(SCYLLA_ERR_INVALID_ARG, "invalid row bounds at row " + std::to_string(i));
  }
  return lp->set_row_bounds(row_lo, row_hi);
}

extern "C" int scylla_set_col_bounds(scylla_lp* lp, const double* col_lo, const double* col_hi) {
  if (!lp || !col_lo || !col_hi) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  int rc = lp->ensure_host_vectors();
  if (rc != SCYLLA_OK) return rc;
  for (int64_t j = 0; j < lp->n0; ++j) {
    const double a = col_lo[j], b = col_hi[j];
    if (std::isnan(a) || std::isnan(b) || a > b || a == kInf || b == -kInf)
      FAIL(SCYLLA_ERR_INVALID_ARG, "invalid column bounds at column " + std::to_string(j));
    if (lp->int0[size_t(j)] && ((std::isfinite(a) && a != std::floor(a)) || (std::isfinite(b) && b != std::floor(b))))
      FAIL(SCYLLA_ERR_INVALID_ARG, "integer column with a fractional bound: " + std::to_string(j));
  }
  return lp->set_col_bounds(col_lo, col_hi);
}

// The continuous repair: the original MIP's LP with the integer columns fixed at
// xhat, solved on a second handle without auxiliary columns (built on first use
// from the host copy of the original MIP) from its cold start.
int scylla_lp::repair(const double* xhat, double tol, int64_t iter_limit, double* x_out,
                      scylla_repair_result* out) {
  int rc = ensure_host_matrix();
  if (rc != SCYLLA_OK) return rc;
  for (int64_t j = 0; j < n0; ++j)
    if (int0[size_t(j)] && !(std::isfinite(xhat[j]) && xhat[j] == std::floor(xhat[j]) && xhat[j] >= l0[size_t(j)] &&
                             xhat[j] <= u0[size_t(j)]))
      FAIL(SCYLLA_ERR_INVALID_ARG, "xhat not integral within bounds at integer column " + std::to_string(j));
  std::vector<double> lf(l0), uf(u0);
  for (int64_t j = 0; j < n0; ++j)
    if (int0[size_t(j)]) lf[size_t(j)] = uf[size_t(j)] = xhat[j];
  // Propagation of the fixing on the GPU: every bound it derives holds for every point
  // of the fixed LP, so a row it has to ignore or a column whose bounds cross proves
  // the fixed LP infeasible, and no solve runs.
  {
    std::vector<double> pl(lf), pu(uf);
    std::vector<uint8_t> ign(static_cast<size_t>(m0 > 0 ? m0 : 1), 0);
    int64_t prounds = 0, pconf = 0;
    rc = propagate_impl(this, pl.data(), pu.data(), ign.data(), kRepairPropagationRounds, &prounds, &pconf);
    if (rc != SCYLLA_OK) return rc;
    bool infeasible = pconf > 0;
    for (int64_t i = 0; i < m0 && !infeasible; ++i) infeasible = ign[size_t(i)] != 0;
    if (infeasible) {
      double obj = 0.0;
      for (int64_t j = 0; j < n0; ++j) {
        x_out[j] = std::min(std::max(xhat[j], lf[size_t(j)]), uf[size_t(j)]);
        obj += c0[size_t(j)] * x_out[j];
      }
      out->status = SCYLLA_NOT_FOUND;
      out->objective = obj;
      return SCYLLA_OK;
    }
  }
  if (!repair_lp) {
    scylla_csr A{m0, n0, nnz0, rowptr0.data(), cols0.data(), vals0.data()};
    scylla_params q = p;
    q.aux_general_integers = 0;
    q.trace_capacity = 0;
    q.repair_iters = 0;
    q.precision = SCYLLA_PREC_FP64;
    q.infeasibility_checks = 0;  // the repair's screen proves infeasible fixings
    scylla_lp* r = new scylla_lp();
    rc = create_impl(&A, c0.data(), lo0.data(), hi0.data(), l0.data(), u0.data(), int0.data(), &q, user_st, r);
    if (rc != SCYLLA_OK) {
      r->release();
      delete r;
      return rc;
    }
    repair_lp = r;
  }
  rc = repair_lp->set_col_bounds(lf.data(), uf.data());
  // working row bounds: the original ones for the first solve
  std::vector<double> lo_w(lo0), hi_w(hi0);
  if (rc == SCYLLA_OK) rc = repair_lp->set_row_bounds(lo_w.data(), hi_w.data());
  if (rc == SCYLLA_OK) rc = scylla_reset_state(repair_lp);
  if (rc != SCYLLA_OK) return rc;
  out->status = SCYLLA_NOT_FOUND;
  for (int t = 0; t < p.repair_rounds; ++t) {
    scylla_pdhg_result res{};
    rc = repair_lp->solve(tol, iter_limit - out->iterations, 0, &res);
    if (rc == SCYLLA_OK) rc = repair_lp->fetch_x(x_out, int(n0));
    if (rc != SCYLLA_OK) return rc;
    out->rounds = t + 1;
    out->iterations += res.iterations;
    out->seconds += res.seconds;
    out->pdhg_status = res.status;
    out->rel_kkt = res.rel_kkt;
    for (int64_t j = 0; j < n0; ++j)
      if (int0[size_t(j)]) x_out[j] = xhat[j];
    if (check_feasible_host(*this, x_out)) {
      out->status = SCYLLA_FOUND;
      break;
    }
    if (t + 1 == p.repair_rounds || out->iterations >= iter_limit) break;
    // move the working bound of every row whose activity exceeds an original bound
    int shifted = 0;
    for (int64_t i = 0; i < m0; ++i) {
      double a = 0.0;
      for (int64_t q = rowptr0[size_t(i)]; q < rowptr0[size_t(i) + 1]; ++q) a += vals0[size_t(q)] * x_out[cols0[size_t(q)]];
      const double lo = lo0[size_t(i)], hi = hi0[size_t(i)];
      bool moved = false;
      if (a > hi) {
        hi_w[size_t(i)] -= (a - hi) + 1e-6 * std::max(1.0, std::fabs(hi));
        moved = true;
      } else if (a < lo) {
        lo_w[size_t(i)] += (lo - a) + 1e-6 * std::max(1.0, std::fabs(lo));
        moved = true;
      }
      if (moved) {
        ++shifted;
        if (lo_w[size_t(i)] > hi_w[size_t(i)]) lo_w[size_t(i)] = hi_w[size_t(i)] = 0.5 * (lo_w[size_t(i)] + hi_w[size_t(i)]);
      }
    }
    out->shifted_rows += shifted;
    rc = repair_lp->set_row_bounds(lo_w.data(), hi_w.data());
    if (rc != SCYLLA_OK) return rc;
  }
  double obj = 0.0;
  for (int64_t j = 0; j < n0; ++j) obj += c0[size_t(j)] * x_out[j];
  out->objective = obj;
  return SCYLLA_OK;
}

extern "C" int scylla_repair(scylla_lp* lp, const double* xhat, double tol, int64_t iter_limit, double* x_out,
                             scylla_repair_result* out) {
  if (!lp || !xhat || !x_out || !out) FAIL(SCYLLA_ERR_INVALID_ARG, "null argument");
  if (!(tol >= 0.0) || iter_limit < 0) FAIL(SCYLLA_ERR_INVALID_ARG, "need tol >= 0 and iter_limit >= 0");
  std::memset(out, 0, sizeof(*out));
  out->status = SCYLLA_NOT_FOUND;
  try {
    return lp->repair(xhat, tol, iter_limit, x_out, out);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
}

extern "C" int scylla_reset_state(scylla_lp* lp) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  int rc = lp->order_after_user();
  if (rc != SCYLLA_OK) return rc;
  cudaStream_t st = lp->st;
  if (lp->p.precision == SCYLLA_PREC_MIXED) CK(launch_init_point<float>(lp->d32, st));
  else CK(launch_init_point<double>(lp->d64, st));
  CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  lp->h_ctl->eta = lp->eta0;
  lp->h_ctl->omega = lp->omega0;
  CK(cudaMemcpyAsync(lp->ctl, lp->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

template <typename T>
static int time_kernels_impl(scylla_lp* lp, const DevLP<T>& d, int attempts, double* ms) {
  cudaStream_t st = lp->st;
  const int nchk = lp->p.n_check;
  const int nev = 4 * (attempts + attempts / nchk + 1);  // two events per timed launch
  std::vector<cudaEvent_t> ev(nev);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double sum[4] = {0, 0, 0, 0};
  int cnt[4] = {0, 0, 0, 0};
  std::vector<int> which;
  int q = 0;
  auto timed = [&](int kind, cudaError_t (*fn)(const DevLP<T>&, cudaStream_t)) -> cudaError_t {
    cudaError_t e = cudaEventRecord(ev[q], st);
    if (e == cudaSuccess) e = fn(d, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[q + 1], st);
    which.push_back(kind);
    q += 2;
    return e;
  };
  cudaError_t e = launch_solve_init<T>(d, 0.0, (long long)attempts + 1, 0, 1LL << 40, st);
  if (e == cudaSuccess) e = launch_check<T>(d, st);
  for (int a = 0; a < attempts && e == cudaSuccess; ++a) {
    e = timed(0, launch_primal<T>);
    if (e == cudaSuccess) e = timed(1, launch_dual<T>);
    if (e == cudaSuccess && (a + 1) % nchk == 0) {
      e = timed(2, launch_check_cols<T>);
      if (e == cudaSuccess) e = timed(3, launch_check_rows<T>);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    for (size_t i = 0; i < which.size(); ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      sum[which[i]] += t;
      cnt[which[i]]++;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  CK(e);
  for (int k = 0; k < 4; ++k) ms[k] = cnt[k] ? sum[k] / cnt[k] : 0.0;
  return SCYLLA_OK;
}

namespace {

template <typename T>
const DevLP<T>& dev_of(const scylla_lp* lp) {
  if constexpr (std::is_same<T, float>::value) return lp->d32;
  else return lp->d64;
}

// The forms' grids: resident blocks per SM times the SMs, at most one warp per tile.
template <typename T>
void set_forms(scylla_lp* lp, int form_p, int form_d) {
  const bool wp = form_p == kFormWide || form_p == kFormStaged, wd = form_d == kFormWide || form_d == kFormStaged;
  lp->form_p = form_p;
  lp->form_d = form_d;
  lp->grid_p = occupancy_grid<T>(0, form_p, wp ? lp->t_ntiles_w : lp->t_ntiles);
  lp->grid_d = occupancy_grid<T>(1, form_d, wd ? lp->a_ntiles_w : lp->a_ntiles);
  if (std::is_same<T, float>::value) fill_dev<float>(lp->d32, lp);
  else fill_dev<double>(lp->d64, lp);
}

// Create-time autotuner of the per-attempt kernels' forms: the 32-row tiles (plain
// loads) and the wide tiles (up to 128 rows, streaming loads) are each timed for
// kTuneAttempts attempts (CUDA events around separate launches) from the start point
// on the handle's own matrix, and each of the two kernels takes its own form.  The
// other form replaces the L2-size rule's only when it is more than kTuneMargin
// faster, so that forms close in time keep the rule's, reproducible choice.  The
// choice is kept per matrix shape and precision for the process, and the handle goes
// back to its start point.
constexpr int kTuneAttempts = 16;
constexpr double kTuneMargin = 0.03;

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

template <typename T>
int autotune_form(scylla_lp* lp) {
  const auto key = std::make_tuple(lp->device, lp->m, lp->n, lp->nnz, int(sizeof(T)));
  std::pair<int, int> chosen(-1, -1);
  {
    std::lock_guard<std::mutex> g(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) chosen = it->second;
  }
  cudaStream_t st = lp->st;
  if (chosen.first < 0) {
    // the start point's control block, restored after the timed attempts
    CK(cudaMemcpyAsync(lp->h_ctl, lp->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const Control saved = *lp->h_ctl;
    // the 32-row, wide and (FP32) asynchronous-copy forms
    const int forms[3] = {kFormPlain, kFormWide, kFormAsync};
    const int nf = std::is_same<T, float>::value ? 3 : 2;
    for (int q = 0; q < nf; ++q) {
      set_forms<T>(lp, forms[q], forms[q]);
      double ms[4] = {0, 0, 0, 0};
      const int rc = time_kernels_impl<T>(lp, dev_of<T>(lp), kTuneAttempts, ms);
      if (rc != SCYLLA_OK) return rc;
      lp->tune_ms[2 * q] = ms[0];
      lp->tune_ms[2 * q + 1] = ms[1];
    }
    const int rule = lp->form_rule == kFormWide ? 1 : 0;
    auto pick = [&](int side) {
      int best = rule;
      for (int q = 0; q < nf; ++q)
        if (lp->tune_ms[2 * q + side] < lp->tune_ms[2 * best + side]) best = q;
      return forms[lp->tune_ms[2 * best + side] < (1.0 - kTuneMargin) * lp->tune_ms[2 * rule + side] ? best : rule];
    };
    chosen = std::make_pair(pick(0), pick(1));
    {
      std::lock_guard<std::mutex> g(g_tune_mutex);
      g_tune_cache.emplace(key, chosen);
    }
    *lp->h_ctl = saved;
    CK(cudaMemcpyAsync(lp->ctl, lp->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, st));
  }
  set_forms<T>(lp, chosen.first, chosen.second);
  if (std::is_same<T, float>::value) CK(launch_init_point<float>(lp->d32, st));
  else CK(launch_init_point<double>(lp->d64, st));
  CK(cudaStreamSynchronize(st));
  return SCYLLA_OK;
}

}  // namespace

extern "C" int scylla_kernel_form(const scylla_lp* lp, int32_t* form, int32_t* form_dual, int32_t* rule_form,
                                  double* tune_ms) {
  if (!lp) FAIL(SCYLLA_ERR_INVALID_ARG, "null handle");
  if (form) *form = api_form(lp->form_p);
  if (form_dual) *form_dual = api_form(lp->form_d);
  if (rule_form) *rule_form = api_form(lp->form_rule);
  if (tune_ms)
    for (int q = 0; q < 6; ++q) tune_ms[q] = lp->tune_ms[q];
  return SCYLLA_OK;
}

extern "C" int scylla_time_kernels(scylla_lp* lp, int32_t attempts, double* ms) {
  if (!lp || !ms || attempts < 1) FAIL(SCYLLA_ERR_INVALID_ARG, "need a handle, ms[4] and attempts >= 1");
  int rc = lp->order_after_user();
  if (rc != SCYLLA_OK) return rc;
  return lp->p.precision == SCYLLA_PREC_MIXED ? time_kernels_impl<float>(lp, lp->d32, attempts, ms)
                                              : time_kernels_impl<double>(lp, lp->d64, attempts, ms);
}
