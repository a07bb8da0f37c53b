/*
 * FP64 CPU oracle of the batched quasi-Newton dwell-time optimisation (gL-BFGS) of
 * "A GPU-based multi-criteria optimization algorithm for HDR brachytherapy".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow, obviously correct restatement
 * of the paper's arithmetic in double precision.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline / reference leg load it; the product path (the CUDA library
 * under paper_1904_01567_b300/) never does, and the two share no code.
 *
 * Layouts (all row-major, plan-major):
 *   A       n_pnt x n_dwell   dose rate of dwell l at point i (Gy/s), Eq. (dose)
 *   sid     n_pnt             structure id of each point, 0 <= sid < n_struct
 *   params  n_struct x 4      (w_min, D_min, D_max, w_max) per structure, Eq. (1);
 *                             D_min = -inf or D_max = +inf makes the penalty one-sided
 *   w       n_struct          hidden weights of one plan, Eq. (obj)
 *   x       n_dwell           dwell weights, t = x*x (Sec. 2.1.2)
 *   T, T0   P x n_dwell       dwell times of P plans (one row per plan)
 *
 * Parity status of each function is stated beside it; every function here is pinned by a
 * test in tests/test_oracle_*.py against something other than itself.
 */
#ifndef GMCO_ORACLE_H
#define GMCO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_CONVERGED = 0, ORACLE_MAXITER = 1, ORACLE_LSFAIL = 2, ORACLE_NONFINITE = 3 };

/* Step (i) of the planning flow (Sec. 2.2.1), the dose rate matrix A of Eq. (dose).  The
 * paper gives no dose-rate model; this is the isotropic point source the workload names:
 *   A_il = lambda * sk * unit * g(r) / r^2,  r = max(|p_i - q_l|, r_min),  g = g0 + g1 r + g2 r^2
 * pts n_pnt x 3, dw n_dwell x 3 (cm), src = {lambda, sk, unit, r_min, g0, g1, g2}.
 * Returns 0, or -1 on invalid arguments or where g(r) <= 0.  Pinned: the rate 0.12575 Gy/s at
 * 1 cm of the workload's constants, the clamp below r_min, the inverse-square ratio. */
int oracle_dose_rate(const double *pts, int64_t n_pnt, const double *dw, int64_t n_dwell,
                     const double *src, double *A);

/* Plan evaluation and selection (Sec. 2.3.1, Sec. 2.4).  dvh is P x 5 (target V100 %, D90 %,
 * urethra D10 %, rectum V75 %, bladder V75 % of the structure's points); crit = {V100 min
 * (RTOG), V100 min (RTOG+), urethra D10 max, V75 max cc, rectum cc, bladder cc}.  cls[i]: 2 RTOG+
 * valid, 1 RTOG valid, 0 invalid.  *selected: among RTOG+ valid plans, else RTOG valid plans,
 * the highest V100; with no valid plan, among plans meeting the target and urethra criteria
 * (else among all) the lowest rectum + bladder V75 in cc; the first index on ties.  Returns 0,
 * or -1 on invalid arguments.  Pinned: hand-made rows at each criterion's boundary. */
int oracle_rtog_select(const double *dvh, int64_t P, const double *crit, int32_t *cls,
                       int32_t *selected);

/* Non-dominated plans of a pool (Sec. 2.2.4): nondom[i] = 1 unless some plan is no worse in
 * all K objectives (minimised) and better in one.  Brute force over all pairs.  Pinned: a
 * hand-made front with duplicates, the one-objective case. */
int oracle_pareto(const double *obj, int64_t P, int32_t K, int32_t *nondom);

/* Eq. (dose): d_i = sum_l A_il t_l.  Pinned: closed-form single source, exact sums. */
void oracle_dose(const double *A, int64_t n_pnt, int64_t n_dwell, const double *t, double *d);

/* Eq. (1): piecewise quadratic penalty of one dose value, and its derivative in d. */
double oracle_point_penalty(double d, const double *prm);
double oracle_point_dpenalty(double d, const double *prm);

/* Eq. (obj) with Eq. (dose) at t = x*x, and the gradient of Eq. (2) summed over points:
 *   F = sum_s w_s / N_s sum_{i in s} f_i(d_i)
 *   dF/dx_l = 2 x_l sum_i A_il (w_s(i) / N_s(i)) f'_i(d_i)
 * Structures without points contribute nothing.  grad_x, dose, f_struct may be NULL;
 * f_struct[s] = (1/N_s) sum_{i in s} f_i (the unweighted per-structure objective).
 * Returns 0, or -1 on invalid arguments. */
int oracle_objective(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                     int32_t n_struct, const double *params, const double *w, const double *x,
                     double *F, double *grad_x, double *dose, double *f_struct);

/* L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4) with H0 = gamma I,
 * gamma = s'y / y'y of the newest pair.  History is a ring of m slots (S, Y: m x n,
 * rho: m) holding `count` pairs, the newest at slot `newest`.  Writes p = -H g.
 * count == 0 gives p = -g. */
void oracle_two_loop(int64_t n, int32_t m, int32_t count, int32_t newest, const double *S,
                     const double *Y, const double *rho, const double *g, double *p);

/* One plan, the whole method (x = sqrt(t0); L-BFGS with backtracking Armijo line search;
 * stop on relative objective change).  t0 may be NULL (uniform 1 s).  The plan stops when
 * stop_window consecutive accepted iterations each change F by at most tol |F_prev|
 * (stop_window = 1: the single-iteration rule).
 * trace (optional, 3 x (max_iters + 1) doubles): for each accepted iteration k the
 * objective F_k, the accepted step alpha_k and the directional derivative g'p; row 0 holds
 * F_0.  n_evals counts objective evaluations (the first one and every line-search trial);
 * max_evals > 0 caps them: the plan stops at its last accepted point, with the max-iteration
 * status, where a further evaluation would exceed the cap (0 = no cap).  Returns 0 or -1 on
 * invalid arguments. */
int oracle_lbfgs(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                 int32_t n_struct, const double *params, const double *w, const double *t0,
                 int32_t max_iters, double tol, int32_t m, double c1, int32_t max_ls,
                 int32_t stop_window, int32_t max_evals, double *t_out, double *F_out,
                 int32_t *iters_out, int32_t *status_out, double *trace, int64_t *n_evals);

/* P independent plans (rows of W and T0), one plan per OpenMP thread.  T0 may be NULL.
 * n_threads <= 0 uses the OpenMP default.  Returns 0 or -1. */
int oracle_lbfgs_batch(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                       int32_t n_struct, const double *params, const double *W, int64_t P,
                       const double *T0, int32_t max_iters, double tol, int32_t m, double c1,
                       int32_t max_ls, int32_t stop_window, int32_t max_evals, double *T_out,
                       double *F_out, int32_t *iters_out, int32_t *status_out, int64_t *n_evals,
                       int32_t n_threads);

/* Output n (0-based) of SplitMix64 seeded with `seed` (Steele, Lea and Flood 2014): the
 * counter-based generator both engines draw the annealing's random numbers from.  Pinned: the
 * generator's published first outputs. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t n);

/* The stochastic engine gSA (Sec. 2.2.1, steps (ii)-(v) repeated) for one plan, index `plan`
 * of its batch.  The paper gives neither the move nor the cooling schedule; read here as:
 *   x = sqrt(t0) (t0 NULL: 1 s); for k = 0 .. iters-1, with f = k / (iters - 1),
 *   delta_k = step0 (step_final / step0)^f,  T_k = T0 (T_final / T0)^f  (0 when step0 / T0 is 0),
 *   x'_l = x_l + delta_k (2 u_kl - 1)   for every dwell l,  u_kl = top 53 bits of draw
 *          (plan, k, l) times 2^-53,
 *   accept x' when F(x') - F(x) <= -T_k F(x_0) ln v_k,  v_k = (top 53 bits + 1) 2^-53 of
 *          draw (plan, k, 2^21 - 1);
 * draw (p, k, l) = oracle_splitmix64(seed, k 2^42 + p 2^21 + l).  Returns the best point seen
 * (t_out = x_best^2, F_out), the number of accepted moves, and min_margin = the smallest
 * |F(x') - F(x) + T_k F_0 ln v_k| / max(|F(x)|, |F(x')|) over the run (how close a decision came
 * to flipping, relative to the objectives whose rounding could flip it).
 * trace (optional, iters + 1) holds F(x) after each iteration, trace[0] = F(x_0).
 * Parity unpinned beyond its invariants (the method's move and schedule are not in the
 * paper).  Returns 0 or -1 on invalid arguments. */
int oracle_sa(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
              int32_t n_struct, const double *params, const double *w, const double *t0,
              int64_t plan, int32_t iters, uint64_t seed, double T0, double T_final, double step0,
              double step_final, double *t_out, double *F_out, int32_t *accepts_out,
              double *min_margin_out, double *trace);

/* P plans of oracle_sa (plan j = row j of W and T0s), one per OpenMP thread. */
int oracle_sa_batch(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                    int32_t n_struct, const double *params, const double *W, int64_t P,
                    const double *T0s, int32_t iters, uint64_t seed, double T0, double T_final,
                    double step0, double step_final, double *T_out, double *F_out,
                    int32_t *accepts_out, double *min_margin_out, int32_t n_threads);

/* DVH indices of one dose vector (Sec. 2.3.1 definitions), rx = prescription (Gy):
 *   out[0] V100 of structure 0 (% of its points with d >= rx)
 *   out[1] D90  of structure 0 (% of rx): k-th largest dose, k = ceil(0.9 N_0)
 *   out[2] D10  of structure 1 (% of rx): k-th largest dose, k = ceil(0.1 N_1)
 *   out[3] V75  of structure 2 (% of its points with d >= 0.75 rx)
 *   out[4] V75  of structure 3 (same)
 * An index whose structure is absent or empty is NaN. */
void oracle_dvh(const double *d, const int32_t *sid, int64_t n_pnt, int32_t n_struct, double rx,
                double *out);

#ifdef __cplusplus
}
#endif
#endif
