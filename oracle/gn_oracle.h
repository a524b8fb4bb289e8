/*
 * gn_oracle.h -- plain FP64 CPU oracle for Graph Normalization (GN).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, constant or helper with the CUDA library; its status values are its
 * own and are mapped by name in the tests.
 *
 * Paper: "Graph Normalization: Fast Binarizing Dynamics for Differentiable
 * MWIS" (arXiv 2605.05330).  Every function cites the definition it writes out.
 * Everything is sequential, FP64, in the paper's x-space notation.
 */
#ifndef GN_ORACLE_H_
#define GN_ORACLE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status values (oracle-local) */
#define GNO_OK                    0
#define GNO_WARN_NOT_CONVERGED    1
#define GNO_WARN_NOT_BINARY       2
#define GNO_WARN_NOT_MAXIMAL      3
#define GNO_ERR_ARG              (-1)
#define GNO_ERR_NOT_SIMPLE       (-2)
#define GNO_ERR_WEIGHT           (-3)
#define GNO_ERR_NOT_NORMALIZABLE (-4)
#define GNO_ERR_NOT_INDEPENDENT  (-7)

#define GNO_GAMMA_PURSUIT 0  /* linear ramp gamma0 -> gamma1 over ramp_iters (Sec. 6) */
#define GNO_GAMMA_FIXED   1  /* gamma held at gamma1 */

typedef struct {
  int gamma_mode;
  double gamma0, gamma1;
  int ramp_iters;
  int check_every;
  double theta_bin;
} gno_params;

typedef struct {
  int iters;          /* iterations performed by this call */
  int converged;      /* 1 if the stop test fired */
  int binary;         /* 1 if every x_i <= theta or >= 1-theta at the last check */
  int status;
  double resid_inf;   /* max_i |x_i^{k+1} - x_i^k| at the last iteration */
  double resid_l1;    /* sum_i |x_i^{k+1} - x_i^k| at the last iteration */
  double objective;   /* sum_i w_i x_i of the returned state */
  double energy;      /* E~ of the state that entered the last step, at that step's gamma */
  long long safe_div_hits;
} gno_info;

int    gno_validate(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* w);
double gno_gamma(const gno_params* p, int k);
void   gno_step(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* v,
                double gamma, const double* x, double* x_next, long long* hits);
int    gno_run(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* w,
               const double* x0, int max_iters, double tol, const gno_params* p, int start_iter,
               double* x_out, gno_info* info, double* trace_obj, double* trace_energy,
               int trace_len);
double gno_objective(int n, const double* w, const double* x);
double gno_energy(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* w,
                  double gamma, const double* x);
int    gno_extract_is(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* w,
                      const double* x, uint8_t* mask, int32_t* members, int32_t* count,
                      double* weight);
double gno_stability(int n, const int32_t* row_ptr, const int32_t* col_idx, const double* w,
                     double gamma, const uint8_t* mask);
int    gno_mwis_enumerate(int n, const int32_t* row_ptr, const int32_t* col_idx,
                          const double* w, double rel_tol, int max_out, uint32_t* masks_out,
                          int* n_best, double* best_weight);
double gno_hungarian(int k, const double* cost, int32_t* assign);

#ifdef __cplusplus
}
#endif
#endif
