// Internal declarations of the GB300 Scylla PDHG library.
//
// Layout in HBM (all in the preconditioned space unless noted):
//   A   : CSR over rows    (rowptr int32[m+1], cols int32[nnz], vals T[nnz] (+FP64 copy))
//   A^T : CSR over columns (same nonzeros, rows ascending within a column)
//   warp tiles: contiguous row ranges with <= kTileNnz nonzeros and <= 32 rows,
//               or a single longer row (processed by one warp); stored as
//               (first row, first nonzero) pairs, ntiles + 1 of them.
//   iterate pools: X[3], Y[3], AX[3] (roles cur/next/avg chosen by indices in the
//   device control block), ATY[2] (cur/avg), XLR, YLR (last restart point).
// Arrays that are read with 16-byte vector loads are padded to a multiple of 4
// elements plus 4, so an aligned vector starting before the end stays in bounds.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "scylla.h"

namespace scylla {

constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kMaxWarps = 32;       // bound of per-warp shared arrays
constexpr int kPWarps = 16;         // warps per block of the persistent solve kernel
constexpr int kPThreads = kPWarps * 32;
constexpr int kMaxNcheckPersistent = 1024;
constexpr int kTileNnz = 256;  // nonzeros per multi-row warp tile
constexpr int kTileRows = 32;  // rows per multi-row warp tile (one lane per row)
constexpr int kWideRows = 128;  // rows per wide tile (DRAM-resident form): rows lane, lane + 32, ...
constexpr int kWideRPL = kWideRows / 32;
// forms of the per-attempt kernels
constexpr int kFormPlain = 0, kFormPrefetch = 1, kFormWide = 2, kFormStaged = 3;
// 32-row tiles whose next tile (indices, values, row pointers, epilogue operands) is
// staged in shared memory by asynchronous copies (FP32 only)
constexpr int kFormAsync = 4;
constexpr int kVec = 4;        // elements per lane per vector load
constexpr int kSmemPerWarp = kTileNnz + kTileNnz / 32 + 8;  // skewed product buffer

// per-block partial sums written by each kernel
constexpr int kNP = 1;    // primal: ||dx||^2
constexpr int kND = 2;    // dual: ||dy||^2, dy.(A x' - A x)
constexpr int kNC1 = 10;  // column check: 5 sums x {current, average}
constexpr int kNC2 = 8;   // row check: 4 sums x {current, average}
// infeasibility detection: a candidate dual ray proves the LP infeasible when
// D > kInfeasMargin * S (D and S as in scylla_get_certificate)
constexpr double kInfeasMargin = 1e-9;
constexpr int kNIR = 2;  // detector row sums: sum of the row terms of D, of their absolute values
constexpr int kNIC = 3;  // detector column sums: column terms, their absolute values, infinite terms

// Device control block: every decision of the solve is taken on the device and
// kept here, so the iteration loop needs no host round trip.
struct Control {
  double eta, omega, eta_used, wsum, avg_w, tol;
  double kkt_lr, kkt_prev;
  double offset, bnorm, cnorm;
  double eps_p, eps_d, eps_g, rel_kkt, pobj, dobj;  // of the reported point
  double beta_s, beta_n, beta_a, theta, exp_red, exp_grow;
  long long k, iter_limit, k_lr, accepted, rejected, restarts, chunks, max_chunks, n_ctrace;
  long long k_fac;  // attempt count when the step-size factor table was filled
  unsigned long long hash_accum, last_hash;
  int same_hash, stall_checks;
  int ix_cur, ix_next, ix_avg, ia_cur, ia_avg;
  int aty_valid, copy_lr, done, status, used_avg, initial;
  int adaptive, restarts_on, pw_update;
  unsigned int cnt_dual, cnt_c2, cnt_misc;
  // Derived by the control logic whenever eta, omega or the averaging weight change,
  // so the bulk kernels load them instead of recomputing them in every thread (FP64
  // division and conversion are slow on this part): 1/omega, and the next attempt's
  // tau = eta/omega, sigma = eta omega and averaging weights (w, 1 - w) in both types.
  double inv_omega;
  double tau_d, sigma_d, w_d, w1_d;
  float tau_f, sigma_f, w_f, w1_f;
  int avg_on;  // w > 0
  // FP32-mixed mode: the step-size state between checks lives in FP32 copies (eta,
  // omega, 1/omega, the step-weight sum and this attempt's two step-size factors);
  // the FP64 fields eta and wsum are brought up to date from them before each check.
  float eta_f, om_f, iom_f, wsum_f, fr_f, fg_f;
  // infeasibility detection: D and S of the candidate ray tested at this check, and
  // whether one was tested (set by the detector kernels, read by the check decision)
  double inf_gap, inf_scale;
  int inf_tested;
  unsigned int cnt_inf;
};

// Pointers of one LP, passed by value to every kernel.  T is the type of the bulk
// iteration (double or float); the FP64 members are used by the checks.
template <typename T>
struct DevLP {
  int m, n;
  const int* a_rowptr;
  const int* a_cols;
  const int2* a_tiles;
  int a_ntiles;
  const T* a_vals;
  const double* a_vals64;
  const int* t_rowptr;
  const int* t_cols;
  const int2* t_tiles;
  int t_ntiles;
  const int2* a_tiles_w;  // wide tiles (up to kWideRows rows) of the plain-load per-attempt kernels
  int a_ntiles_w;
  const int2* t_tiles_w;
  int t_ntiles_w;
  const T* t_vals;
  const double* t_vals64;
  const T *c, *l, *u, *lo, *hi;
  const double *c64, *l64, *u64, *lo64, *hi64, *R, *C;
  const double *invR, *invC;  // 1 / R, 1 / C (the checks multiply instead of dividing)
  const unsigned char* int_mask;
  // diagonal Hessian of a quadratic objective, scaled (q~ = q C^2): bulk type for the
  // primal step, FP64 for the checks; both null for an LP
  const T* q;
  const double* q64;
  T* X[3];
  T* Y[3];
  T* AX[3];
  T* ATY[2];
  T* XLR;
  T* YLR;
  Control* ctl;
  double *part_p, *part_d, *part_c1, *part_c2;
  double* red_c1;  // the column check's reduced sums (kNC1)
  int grid_p, grid_d, grid_c1, grid_c2;
  double* step_fac;      // (1 - kk^-a, 1 + kk^-b) of the next n_check attempts: 2 n_check doubles,
                         // then the same 2 n_check values as floats (3 n_check doubles in all)
  double* pp_part;       // persistent kernel: 24 partial sums per block
  unsigned long long* p_hash;  // persistent kernel: two rounding-hash slots
  int n_check;
  int pdl;               // launch the per-attempt kernels with programmatic dependent launch
  int form_p, form_d;    // form of the primal and dual per-attempt kernels (kForm*)
  unsigned long long wait_ns;  // bound of every device-side wait
  double* trace_steps;   // 4 doubles per attempt, or null
  double* trace_checks;  // 5 doubles per check, or null
  int trace_cap;
  // infeasibility detection (null when off): y at the anchor check, the candidate ray
  // (FP64, scaled), block partials (kNIR then kNIC per block of inf_grid)
  T* inf_anchor;
  double* inf_cand;
  double* inf_part;
  int inf_grid;
};

// Per-LP values of one attempt in a batched solve, written by its control kernels.
template <typename T>
struct BatchSlot {
  T tau, sigma, w, w1;
  int cur, nxt, avg, ia_cur, ia_avg, flags;
};

// A batch of LPs stored as one block-diagonal LP (d) with per-LP control.
template <typename T>
struct DevBatch {
  DevLP<T> d;                 // global arrays over all LPs; d.ctl and d.part_* unused
  int nlp;
  const int* a_tile_lp;       // LP of each tile of A / A^T
  const int* t_tile_lp;
  const int* a_tile_beg;      // first tile of each LP (nlp + 1)
  const int* t_tile_beg;
  Control* ctl;               // nlp control blocks
  BatchSlot<T>* slot;         // nlp
  double *tp_p, *tp_d, *tp_c1, *tp_c2;  // per-tile partial sums
  int* n_done;                // LPs finished in this solve
  unsigned int* lp_cnt;       // per LP: tiles of A done in this attempt's dual step (the last one decides)
  long long* kglob;           // attempts made by the LPs still running
  double exp_red, exp_grow;
  int grid_p, grid_d, grid_c1, grid_c2, grid_ctl;
  int async_p, async_d;       // FP32: the primal / dual attempt kernel stages each warp's next tile by
                              // asynchronous copies
  int grid_pa, grid_da;       // their grids
  // persistent solve over a shared work queue: the LPs still running (rebuilt at
  // every check) and their tiles, as lists of indices, and the chunk counters that
  // warps take tiles from
  int* q_lps;                 // nlp slots; q_cnt[0] in use
  int* q_a;                   // tiles of A of those LPs; q_cnt[1] in use
  int* q_t;                   // tiles of A^T; q_cnt[2] in use
  int* q_pre;                 // 2 (nlp + 1): prefix sums of their A and A^T tile counts
  int* q_cnt;                 // [0] LPs, [1] A tiles, [2] A^T tiles
  unsigned int* q_ctr;        // [4] chunk counters: primal, dual, column check, row check
  int grid_q;                 // co-resident blocks of the persistent kernel (0: it cannot run)
};

// Per-objective values of one attempt of a fan-out, written by its control kernels.
template <typename T>
struct FanSlot {
  T tau, sigma, w, w1;
  int flags;
};

// Pool roles shared by every objective of a fan-out, and the objectives whose
// slices the copy kernels move into the current pool before the next attempt.
struct FanState {
  unsigned long long att;     // attempts since seeding: X[att & 1], Y[.], AX[.] hold the current points
  unsigned char rej[64];      // 1: rejected in the last attempt (next pool -> current), written every attempt
  unsigned char rst[64];      // 1: restarted to or finished with the average (average -> current), every check
};

// K objectives of one LP solved together: K-wide vectors are row-major with 64
// slots per row (n x 64, m x 64); objectives K..63 are carried unchanged.
template <typename T>
struct DevFan {
  DevLP<T> d;  // the base LP: matrices, bounds, scaling (its iterate pools unused)
  int K;
  T* X[3];     // [cur], [1 - cur] with cur = state->att & 1; [2] the running average
  T* Y[3];
  T* AX[3];
  T* ATY[2];   // the checks' A^T y of the current [0] and averaged [1] point
  T* XLR;
  T* YLR;
  const double* c_orig;                // unscaled base objective, n
  const unsigned long long* lo_bits;   // bit k of column j: target k at l_j
  const unsigned long long* up_bits;   // bit k of column j: target k at u_j
  double t, om;                        // alpha^K s and 1 - alpha^K of the update
  Control* ctl;                        // K control blocks
  FanSlot<T>* slot;                    // K
  FanState* state;
  // block partials: part_p, part_d [sum][objective][block]; part_c1, part_c2
  // [block][sum][objective]
  double *part_p, *part_d, *part_c1, *part_c2;
  int* n_done;
  long long* kglob;
  double exp_red, exp_grow;
  int grid_p, grid_d, grid_c1, grid_c2, grid_copy;
  // FP32 objective of the scaled space per column: (t c_j C_j, om C_j)
  const float2* cw;
  // the checks' FP64 objective values of the scaled space per column, for g = 0, +1
  // and -1 (three per column, as fan_cost_col64 forms them)
  const double* cc64;
  // tile shape of the primal and dual SpMM (objectives per lane, slots per sweep):
  // 1 = (4, 64), 2 = (2, 64), 3 = (4, 32), 4 = (2, 32); FP64 takes 2 and 4
  int shape_p, shape_d;
};

// Buffers of the original (unaugmented) columns used by the objective update and
// by setup; all device pointers.
struct DevSetup {
  int m, n;           // augmented sizes
  int n_orig, m_orig; // original sizes
  int nnz;
  const int* a_rowptr;
  const int* a_cols;
  const int* t_rowptr;
  const int* t_cols;
  const int2* a_tiles;  // warp tiles of A and of A^T (as in DevLP)
  const int2* t_tiles;
  int a_ntiles, t_ntiles;
  double* a_vals64;  // in: original values; out: scaled values
  double* t_vals64;
  float* a_vals32;   // may be null
  float* t_vals32;
  double* R;
  double* C;
  double* R2;  // ping-pong scratch
  double* C2;
  double* red;  // reduction scratch
  int red_blocks;
};

// Device side of the round-based bound propagation (propagate.cu) on the original
// rows and columns of a handle.
struct PropDev {
  int m, n;                            // original rows and columns
  const int* rowptr;                   // A: original rows first, unscaled values
  const int* cols;
  const double* vals;
  const int* t_rowptr;                 // A^T (rows ascending in each column)
  const int* t_rows;
  const int* perm;                     // position in A of each entry of A^T
  const double *lo, *hi;               // row bounds (m)
  const unsigned char* is_int;         // n
  double *dl, *du;                     // domains (n), updated in place
  double *plb, *pub;                   // one round's proposals at the rows' CSR positions
  unsigned char* state;                // per row: 0 none, 1 proposals, 2 ignored
  unsigned long long* count;           // columns changed, conflicts, rows marked
};
cudaError_t propagate_perm(int n, const int* t_rowptr, const int* t_rows, const int* a_rowptr, const int* a_cols,
                           int* perm, cudaStream_t st);
// one round: row visits from `active`, then the column merge marking `active_next`
cudaError_t propagate_round(const PropDev& P, const unsigned char* active, unsigned char* active_next,
                            cudaStream_t st);

// ---- set-up launchers (setup.cu) ---------------------------------------------
// R = C = 1, ruiz_iters Ruiz iterations and the Pock-Chambolle step (R2, C2 scratch)
cudaError_t launch_precondition(const DevSetup& s, int ruiz_iters, bool pock_chambolle, cudaStream_t st);
// a~ = diag(R) A diag(C) in both CSR copies (and their FP32 shadows)
cudaError_t launch_scale_values(const DevSetup& s, cudaStream_t st);
cudaError_t fill_f64(double* p, long long count, double v, cudaStream_t st);
// l64 = l / C, u64 = u / C (and the FP32 shadows when given) over n columns
cudaError_t scale_col_bounds(long long n, const double* l, const double* u, const double* C, double* l64,
                             double* u64, float* l32, float* u32, cudaStream_t st);
// c64 = c C and q64 = q C^2 (and the FP32 shadows when given) over n columns
cudaError_t scale_objective(long long n, const double* c, const double* q, const double* C, double* c64,
                            float* c32, double* q64, float* q32, cudaStream_t st);
// q64 = q C^2 (and the FP32 shadow when given) over n columns
cudaError_t scale_hessian(long long n, const double* q, const double* C, double* q64, float* q32, cudaStream_t st);
// lo64 = lo R, hi64 = hi R (and the FP32 shadows when given) over m rows
cudaError_t scale_row_bounds(long long m, const double* lo, const double* hi, const double* R, double* lo64,
                             double* hi64, float* lo32, float* hi32, cudaStream_t st);
// kind = is_int (0/1) and aux_of = -1 over n columns
cudaError_t column_kinds(long long n, const uint8_t* is_int, int* kind, int* aux_of, cudaStream_t st);
struct SetupNorms {
  double amax, fro2;  // max |a~|, sum a~^2
  double c2, q2;      // sum c~^2, sum over rows of max(|lo~|, |hi~|)^2 (finite bounds)
};
// one launch over the scaled values and vectors, 4 * red_blocks partials in s.red -> host
cudaError_t setup_norms(const DevSetup& s, const double* c64, const double* lo64, const double* hi64, cudaStream_t st,
                        SetupNorms* out);

// ---- kernel launchers (kernels.cu) -------------------------------------------

struct DevVecs {
  // unscaled originals (FP64), augmented sizes
  const double *c, *lo, *hi, *l, *u;
  // scaled outputs
  double *c64, *lo64, *hi64, *l64, *u64;
  float *c32, *lo32, *hi32, *l32, *u32;  // null in FP64 mode
  const double *R, *C;
  double *invR, *invC;  // outputs: 1 / R, 1 / C (optional)
  int m, n;
};
cudaError_t launch_scale_vectors(const DevVecs& v, cudaStream_t st);

// Objective update of round K (Section 2.4) on the device.
struct DevObjective {
  int n_orig, m_orig, n, m;
  int l2;                // l2 distance: q_j = 1 - alpha^K and c_hat_j -= (1 - alpha^K) xhat_j on I
  double* q_un;          // unscaled Hessian diagonal (n), written in l2 mode
  double* q64;           // scaled q C^2 (n), written in l2 mode
  float* q32;            // its FP32 shadow (mixed precision), or null
  const double* c_orig;  // original c (n_orig)
  const double* l_orig;
  const double* u_orig;
  const int* kind;       // 0 continuous, 1 integer with u-l = 1, 2 general integer (aux)
  const int* aux_of;     // aux index t of a general integer column, else -1
  const double* xhat;    // n_orig
  double* chat;          // unscaled c_hat (n)
  double* lo_unscaled;   // unscaled row lower bounds (m); aux rows updated
  const double* hi_unscaled;
  const double* R;
  const double* C;
  double* c64;
  double* lo64;
  float* c32;
  float* lo32;
  double* red;
  int red_blocks;
  Control* ctl;
};
cudaError_t launch_objective_update(const DevObjective& o, double t_scale, double one_minus_aK,
                                    cudaStream_t st);
// ||c||, ||b|| (unscaled) and the offset into the control block, without changing c.
cudaError_t launch_objective_norms(const DevObjective& o, double offset, cudaStream_t st);

template <typename T>
cudaError_t launch_solve_init(const DevLP<T>& d, double tol, long long iter_limit, int stall_checks,
                              long long max_chunks, cudaStream_t st);
template <typename T>
cudaError_t launch_check(const DevLP<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_slot(const DevLP<T>& d, cudaStream_t st);
// the two launches of one attempt and of one check, separately (measurement)
template <typename T>
cudaError_t launch_primal(const DevLP<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_dual(const DevLP<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_check_cols(const DevLP<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_check_rows(const DevLP<T>& d, cudaStream_t st);
cudaError_t launch_loop_ctl(Control* ctl, cudaGraphConditionalHandle h, cudaStream_t st);
// persistent cooperative solve: blocks per SM that fit (0 if it cannot run), and the launch
template <typename T>
int persistent_blocks_per_sm();
template <typename T>
cudaError_t launch_persistent(const DevLP<T>& d, void* grid_bar, int grid, double wait_limit_s, cudaStream_t st);
constexpr int kPersistentPartials = 24;  // doubles per block in DevLP::pp_part
constexpr size_t kGridBarBytes = 16;
template <typename T>
cudaError_t launch_get_x(const DevLP<T>& d, double* out, int count, cudaStream_t st);
template <typename T>
cudaError_t launch_get_y(const DevLP<T>& d, double* out, int count, cudaStream_t st);
// infeasibility detection at a check (infeas.cu): the candidate ray and its row
// terms, then its column terms and the decision's inputs in the control block
template <typename T>
cudaError_t launch_infeas(const DevLP<T>& d, cudaStream_t st);
// the last tested ray, unscaled, into out (count rows)
template <typename T>
cudaError_t launch_get_cert(const DevLP<T>& d, double* out, int count, cudaStream_t st);
template <typename T>
cudaError_t launch_set_xy(const DevLP<T>& d, const double* x, const double* y, cudaStream_t st);
template <typename T>
cudaError_t launch_init_point(const DevLP<T>& d, cudaStream_t st);
template <typename T>
int occupancy_grid(int side, int form, int work_tiles);
// stable device transpose of an m x n CSR matrix (rows ascending within each column);
// scratch of transpose_scratch_bytes(n, nnz) bytes; colptr has n + 1 entries
size_t transpose_scratch_bytes(int n, long long nnz);
cudaError_t transpose_device(int m, int n, long long nnz, const int* rowptr, const int* cols, const double* vals,
                             int* colptr, int* rows_out, double* vals_out, void* scratch, cudaStream_t st);  // side: 0 primal, 1 dual, 2 c1, 3 c2

int device_sm_count();

template <typename T>
cudaError_t launch_batch_init(const DevBatch<T>& B, double tol, long long iter_limit, int stall_checks,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_batch_slot(const DevBatch<T>& B, cudaStream_t st);
template <typename T>
cudaError_t launch_batch_check(const DevBatch<T>& B, cudaStream_t st);
template <typename T>
cudaError_t launch_batch_part(const DevBatch<T>& B, int part, cudaStream_t st);
template <typename T>
cudaError_t launch_batch_get_x(const DevBatch<T>& B, int b, int col0, int count, double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_batch_init_point(const DevBatch<T>& B, cudaStream_t st);
template <typename T>
void batch_grids(DevBatch<T>& B);
// the attempts between two checks of the batched solve in one cooperative launch
// over the shared work queue; grid_bar: a zeroed barrier, wait_limit_s bounds every
// barrier wait, iter_limit the attempts of the solve
template <typename T>
cudaError_t launch_batch_persistent(const DevBatch<T>& B, void* grid_bar, long long iter_limit, double wait_limit_s,
                                    cudaStream_t st);
// every LP and every tile in the work lists, counters zeroed (start of a solve)
template <typename T>
cudaError_t launch_batch_queue_reset(const DevBatch<T>& B, cudaStream_t st);
// after a check: the work lists without the LPs that finished, counters rearmed
template <typename T>
cudaError_t launch_batch_compact(const DevBatch<T>& B, cudaStream_t st);
template <typename T>
int batch_persistent_blocks_per_sm();

// bump allocator over one cudaMalloc: pass 1 with base == nullptr sizes, pass 2 carves
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

template <typename T>
cudaError_t launch_fan_init(const DevFan<T>& F, double tol, long long iter_limit, int stall_checks, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_slot(const DevFan<T>& F, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_check(const DevFan<T>& F, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_part(const DevFan<T>& F, int part, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_seed(const DevFan<T>& F, const void* x0, const void* y0, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_cw(const DevFan<T>& F, float2* cw, double* cc64, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_get_x(const DevFan<T>& F, int k, double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_fan_get_y(const DevFan<T>& F, int k, double* out, cudaStream_t st);
template <typename T>
void fan_grids(DevFan<T>& F);
template <typename T>
bool fan_shape_valid(int shape);
constexpr int kFanMaxK = 64;


// shared host helpers (lp.cpp)
std::vector<int2> build_tiles_range(const std::vector<int>& rowptr, int r_begin, int r_end, int max_rows = kTileRows);
int validate_lp(const scylla_csr* A, const double* c, const double* lo, const double* hi, const double* l,
                const double* u, const uint8_t* is_int);
size_t padded_len(size_t nnz);

// ---- host helpers -------------------------------------------------------------
void set_error(const std::string& msg);
const char* get_error();

}  // namespace scylla
