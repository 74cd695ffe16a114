// The LP handle behind the opaque scylla_lp of scylla.h (host-side definition).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <vector>

#include "internal.h"

struct scylla_lp {
  scylla_params p{};
  int device = 0;
  cudaStream_t st = nullptr;       // the handle's own stream (graphs are captured on it)
  cudaStream_t user_st = nullptr;  // caller's stream: its prior work is ordered before each call
  cudaEvent_t ev_user = nullptr, ev0 = nullptr, ev1 = nullptr;

  // original MIP on the host (fix-and-propagate, feasibility test, run loop)
  int64_t m0 = 0, n0 = 0, nnz0 = 0;
  // the original matrix on the host, for the propagation and the feasibility test;
  // downloaded on first use by ensure_host_matrix() (the device keeps the unscaled
  // values in a_vals0)
  mutable std::vector<int64_t> rowptr0;
  mutable std::vector<int32_t> cols0;
  mutable std::vector<double> vals0;
  mutable bool host_matrix_ready = false;
  int ensure_host_matrix() const;  // also fetches the vectors
  // the original vectors on the host (objective, bounds, integrality), downloaded on
  // first use by ensure_host_vectors() from the device's unscaled copies
  mutable std::vector<double> c0, lo0, hi0, l0, u0;
  mutable std::vector<uint8_t> int0;
  mutable bool host_vectors_ready = false;
  int ensure_host_vectors() const;
  // transpose structure of the original rows (rows of each column, ascending), for
  // the host propagation; built on first use by ensure_columns()
  mutable std::vector<int64_t> colptr0;
  mutable std::vector<int32_t> colrows0;
  mutable std::vector<double> colvals0;  // the values in the same order
  mutable bool columns_ready = false;
  void ensure_columns() const;
  // the host propagation's end state after propagating the bounds alone (fixprop.cpp),
  // kept between fix-and-propagate calls; set_col_bounds and set_row_bounds drop it
  mutable std::shared_ptr<const void> root_prop;
  double c0norm = 0.0;
  int64_t n_int = 0;
  std::vector<int32_t> gen_int;  // the general integer columns given auxiliary columns, ascending
  int64_t n_aux = 0;

  // LP iterated on the device (original + auxiliary)
  int m = 0, n = 0, nnz = 0;
  int a_ntiles = 0, t_ntiles = 0;
  int a_ntiles_w = 0, t_ntiles_w = 0;  // wide tiles of the plain-load per-attempt kernels
  int grid_p = 1, grid_d = 1, grid_c1 = 1, grid_c2 = 1, red_blocks = 1;

  void* arena = nullptr;
  size_t arena_bytes = 0;
  int *a_rowptr = nullptr, *a_cols = nullptr;
  int *t_rowptr = nullptr, *t_cols = nullptr;
  int2 *a_tiles = nullptr, *t_tiles = nullptr, *a_tiles_w = nullptr, *t_tiles_w = nullptr;
  double* step_fac = nullptr;
  double* pp_part = nullptr;
  unsigned long long* p_hash = nullptr;
  void* grid_bar = nullptr;
  int p_grid = 0;  // persistent grid (0: that mode is unavailable)
  int form_p = 0, form_d = 0;  // forms of the primal / dual per-attempt kernels (kForm*)
  int form_rule = 0;           // the form the L2-size rule gives
  bool tune = false;           // the create-time autotuner chooses between the 32-row and wide forms
  double tune_ms[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // its ms per launch: primal, dual of the 32-row form,
                                                       // then of the wide, then of the asynchronous-copy form
  double *a_vals64 = nullptr, *t_vals64 = nullptr;
  float *a_vals32 = nullptr, *t_vals32 = nullptr;
  double *c_un = nullptr, *l_un = nullptr, *u_un = nullptr, *lo_un = nullptr, *hi_un = nullptr;
  double *c64 = nullptr, *l64 = nullptr, *u64 = nullptr, *lo64 = nullptr, *hi64 = nullptr;
  float *c32 = nullptr, *l32 = nullptr, *u32 = nullptr, *lo32 = nullptr, *hi32 = nullptr;
  double *R = nullptr, *C = nullptr, *R2 = nullptr, *C2 = nullptr;
  double* a_vals0 = nullptr;  // unscaled values of A (the original rows first)
  double *invR = nullptr, *invC = nullptr;
  // diagonal Hessian of a quadratic objective (n): unscaled, scaled, FP32 shadow;
  // qp_active when the kernels take it (see set_qp_active)
  double *q_un = nullptr, *q64 = nullptr;
  float* q32 = nullptr;
  bool qp_active = false;
  uint8_t* int_mask = nullptr;
  double *c_orig = nullptr, *l_orig = nullptr, *u_orig = nullptr, *xhat_d = nullptr;
  int *kind_d = nullptr, *aux_of_d = nullptr;
  char* X[3] = {nullptr, nullptr, nullptr};
  char* Y[3] = {nullptr, nullptr, nullptr};
  char* AX[3] = {nullptr, nullptr, nullptr};
  char* ATY[2] = {nullptr, nullptr};
  char *XLR = nullptr, *YLR = nullptr;
  double *part_p = nullptr, *part_d = nullptr, *part_c1 = nullptr, *part_c2 = nullptr, *red = nullptr;
  double* red_c1 = nullptr;
  double *io_x = nullptr, *io_y = nullptr;
  // infeasibility detection (scylla_params.infeasibility_checks; null when off): the
  // anchor dual (bulk type), the candidate ray (FP64), the detector's block partials
  char* inf_anchor = nullptr;
  double* inf_cand = nullptr;
  double* inf_part = nullptr;
  double *trace_steps = nullptr, *trace_checks = nullptr;
  scylla::Control* ctl = nullptr;
  scylla::Control* h_ctl = nullptr;  // pinned host mirror
  scylla::DevLP<double> d64{};
  scylla::DevLP<float> d32{};

  double eta0 = 1.0, omega0 = 1.0;  // step size and primal weight chosen at create

  cudaGraph_t graph = nullptr;       // device-side while loop (use_graph = 2)
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaGraph_t chunk_graph = nullptr;  // n_check attempts + one check (use_graph = 1)
  cudaGraphExec_t chunk_exec = nullptr;
  cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
  int* h_done = nullptr;             // pinned, two slots
  int64_t last_launches = 0;

  // the continuous-repair copy of the original MIP (scylla_repair), built on first use
  scylla_lp* repair_lp = nullptr;
  // buffers of the device bound propagation (scylla_propagate), allocated on first use
  void* prop_mem = nullptr;
  scylla::PropDev prop{};
  unsigned char* prop_active[2] = {nullptr, nullptr};
  unsigned long long* prop_count_h = nullptr;  // pinned copy of the three counters

  scylla::DevObjective objective_desc();
  void release();
  int order_after_user();
  int solve(double tol, int64_t iter_limit, int stall_checks, scylla_pdhg_result* out);
  int set_objective(const double* xhat, int32_t K);
  void set_qp_active(bool on);  // point the kernels at the Hessian (or not); drops the captured graphs
  void drop_graphs();
  int set_col_bounds(const double* l, const double* u);    // no validation
  int set_row_bounds(const double* lo, const double* hi);  // no validation
  int repair(const double* xhat, double tol, int64_t iter_limit, double* x_out, scylla_repair_result* out);
  int fetch_x(double* host, int count);
  int fetch_y(double* host, int count);
};

namespace scylla {
// exact MIP-feasibility test of x (length n0) on the handle's original MIP (fixprop.cpp)
bool check_feasible_host(const scylla_lp& lp, const double* x);
// D(y) of a dual ray y (length m0) on the original LP, compensated FP64 (certify.cpp)
double farkas_gap_host(const scylla_lp& lp, const double* y);
}  // namespace scylla
