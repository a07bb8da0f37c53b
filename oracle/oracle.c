/*
 * FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY (see oracle.h): the product path never loads
 * this file's library.  Plain loops in double precision, written to be checked against the
 * paper by eye.  Citations name the paper's sections and equations.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Eq. (dose) */
void oracle_dose(const double *A, int64_t n_pnt, int64_t n_dwell, const double *t, double *d)
{
    for (int64_t i = 0; i < n_pnt; ++i) {
        double s = 0.0;
        for (int64_t l = 0; l < n_dwell; ++l) s += A[i * n_dwell + l] * t[l];
        d[i] = s;
    }
}

/* ---------------------------------------------------------------- Eq. (1) */
/* prm = (w_min, D_min, D_max, w_max).  Zero on the closed interval [D_min, D_max]. */
double oracle_point_penalty(double d, const double *prm)
{
    if (d < prm[1]) return prm[0] * (prm[1] - d) * (prm[1] - d);
    if (d > prm[2]) return prm[3] * (d - prm[2]) * (d - prm[2]);
    return 0.0;
}

/* d f / d d; with d = sum_l A_il x_l^2 the chain rule gives Eq. (2):
 * d f / d x_l = f'(d) * A_il * 2 x_l = 4 A_il x_l w (d - D). */
double oracle_point_dpenalty(double d, const double *prm)
{
    if (d < prm[1]) return 2.0 * prm[0] * (d - prm[1]);
    if (d > prm[2]) return 2.0 * prm[3] * (d - prm[2]);
    return 0.0;
}

/* ---------------------------------------------------------------- dose rate matrix */
int oracle_dose_rate(const double *pts, int64_t n_pnt, const double *dw, int64_t n_dwell,
                     const double *src, double *A)
{
    if (!pts || !dw || !src || !A || n_pnt < 0 || n_dwell < 0 || !(src[3] > 0.0)) return -1;
    const double K = src[0] * src[1] * src[2];
    for (int64_t i = 0; i < n_pnt; ++i) {
        for (int64_t l = 0; l < n_dwell; ++l) {
            const double dx = pts[3 * i] - dw[3 * l];
            const double dy = pts[3 * i + 1] - dw[3 * l + 1];
            const double dz = pts[3 * i + 2] - dw[3 * l + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < src[3]) r = src[3];
            const double g = src[4] + src[5] * r + src[6] * r * r;
            if (!(g > 0.0)) return -1;
            A[i * n_dwell + l] = K * g / (r * r);
        }
    }
    return 0;
}

/* ---------------------------------------------------------------- plan pool */
int oracle_rtog_select(const double *dvh, int64_t P, const double *crit, int32_t *cls,
                       int32_t *selected)
{
    if (!dvh || !crit || !cls || !selected || P < 1) return -1;
    /* classify every plan */
    for (int64_t i = 0; i < P; ++i) {
        const double *r = dvh + 5 * i;
        const double rect_cc = r[3] * crit[4] / 100.0, blad_cc = r[4] * crit[5] / 100.0;
        const int target = r[0] >= crit[0], urethra = r[2] < crit[2];
        const int oars = rect_cc < crit[3] && blad_cc < crit[3];
        cls[i] = (target && urethra && oars) ? (r[0] >= crit[1] ? 2 : 1) : 0;
    }
    /* RTOG+ valid plans first, then RTOG valid ones: the highest target V100 */
    for (int want = 2; want >= 1; --want) {
        int64_t best = -1;
        for (int64_t i = 0; i < P; ++i)
            if (cls[i] == want && (best < 0 || dvh[5 * i] > dvh[5 * best])) best = i;
        if (best >= 0) {
            *selected = (int32_t)best;
            return 0;
        }
    }
    /* no valid plan: the lowest rectum + bladder V75 (cc), among the plans meeting the target
       and urethra criteria when there are any */
    int any_tu = 0;
    for (int64_t i = 0; i < P; ++i) any_tu = any_tu || (dvh[5 * i] >= crit[0] && dvh[5 * i + 2] < crit[2]);
    int64_t best = -1;
    double best_cc = 0.0;
    for (int64_t i = 0; i < P; ++i) {
        const double *r = dvh + 5 * i;
        if (any_tu && !(r[0] >= crit[0] && r[2] < crit[2])) continue;
        const double cc = r[3] * crit[4] / 100.0 + r[4] * crit[5] / 100.0;
        if (best < 0 || cc < best_cc) {
            best = i;
            best_cc = cc;
        }
    }
    *selected = (int32_t)best;
    return 0;
}

int oracle_pareto(const double *obj, int64_t P, int32_t K, int32_t *nondom)
{
    if (!obj || !nondom || P < 1 || K < 1) return -1;
    for (int64_t i = 0; i < P; ++i) {
        int dominated = 0;
        for (int64_t j = 0; j < P && !dominated; ++j) {
            int no_worse = 1, better = 0;
            for (int32_t k = 0; k < K; ++k) {
                if (obj[j * K + k] > obj[i * K + k]) no_worse = 0;
                if (obj[j * K + k] < obj[i * K + k]) better = 1;
            }
            dominated = no_worse && better;
        }
        nondom[i] = dominated ? 0 : 1;
    }
    return 0;
}

/* ---------------------------------------------------------------- Eq. (obj), Eq. (2) */
int oracle_objective(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                     int32_t n_struct, const double *params, const double *w, const double *x,
                     double *F, double *grad_x, double *dose, double *f_struct)
{
    if (!A || !sid || !params || !w || !x || !F || n_pnt < 0 || n_dwell < 0 || n_struct <= 0)
        return -1;
    int64_t *count = (int64_t *)calloc((size_t)n_struct, sizeof(int64_t));
    double *t = (double *)malloc((size_t)(n_dwell > 0 ? n_dwell : 1) * sizeof(double));
    double *d = (double *)malloc((size_t)(n_pnt > 0 ? n_pnt : 1) * sizeof(double));
    double *fs = (double *)calloc((size_t)n_struct, sizeof(double));
    if (!count || !t || !d || !fs) { free(count); free(t); free(d); free(fs); return -1; }

    for (int64_t i = 0; i < n_pnt; ++i) {
        if (sid[i] < 0 || sid[i] >= n_struct) { free(count); free(t); free(d); free(fs); return -1; }
        count[sid[i]]++;
    }
    /* dwell weights -> dwell times, t_l = x_l^2 (Sec. 2.1.2) */
    for (int64_t l = 0; l < n_dwell; ++l) t[l] = x[l] * x[l];
    oracle_dose(A, n_pnt, n_dwell, t, d);

    /* per-structure sums of Eq. (1) */
    for (int64_t i = 0; i < n_pnt; ++i)
        fs[sid[i]] += oracle_point_penalty(d[i], params + 4 * sid[i]);
    double Fv = 0.0;
    for (int32_t s = 0; s < n_struct; ++s) {
        if (count[s] > 0) {
            fs[s] /= (double)count[s];
            Fv += w[s] * fs[s];
        }
        if (f_struct) f_struct[s] = count[s] > 0 ? fs[s] : 0.0;
    }
    *F = Fv;

    if (grad_x) {
        for (int64_t l = 0; l < n_dwell; ++l) grad_x[l] = 0.0;
        for (int64_t i = 0; i < n_pnt; ++i) {
            int32_t s = sid[i];
            double gi = w[s] / (double)count[s] * oracle_point_dpenalty(d[i], params + 4 * s);
            if (gi == 0.0) continue;
            for (int64_t l = 0; l < n_dwell; ++l) grad_x[l] += A[i * n_dwell + l] * gi;
        }
        for (int64_t l = 0; l < n_dwell; ++l) grad_x[l] *= 2.0 * x[l];
    }
    if (dose) memcpy(dose, d, (size_t)n_pnt * sizeof(double));
    free(count); free(t); free(d); free(fs);
    return 0;
}

/* ---------------------------------------------------------------- L-BFGS (Sec. 2.2.2) */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

static double norm_inf(int64_t n, const double *a)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s = fmax(s, fabs(a[k]));
    return s;
}

static int all_finite(int64_t n, const double *a)
{
    for (int64_t k = 0; k < n; ++k) if (!isfinite(a[k])) return 0;
    return 1;
}

void oracle_two_loop(int64_t n, int32_t m, int32_t count, int32_t newest, const double *S,
                     const double *Y, const double *rho, const double *g, double *p)
{
    double *q = p; /* work in place in p, negate at the end */
    double alpha[64];
    for (int64_t k = 0; k < n; ++k) q[k] = g[k];
    if (count <= 0) {
        for (int64_t k = 0; k < n; ++k) p[k] = -q[k];
        return;
    }
    /* first loop: newest to oldest */
    for (int32_t j = 0; j < count; ++j) {
        int32_t i = (newest - j + m) % m;
        alpha[i] = rho[i] * dot(n, S + (int64_t)i * n, q);
        for (int64_t k = 0; k < n; ++k) q[k] -= alpha[i] * Y[(int64_t)i * n + k];
    }
    /* initial matrix H0 = gamma I from the newest pair */
    const double *sn = S + (int64_t)newest * n, *yn = Y + (int64_t)newest * n;
    double gamma = dot(n, sn, yn) / dot(n, yn, yn);
    for (int64_t k = 0; k < n; ++k) q[k] *= gamma;
    /* second loop: oldest to newest */
    for (int32_t j = count - 1; j >= 0; --j) {
        int32_t i = (newest - j + m) % m;
        double beta = rho[i] * dot(n, Y + (int64_t)i * n, q);
        for (int64_t k = 0; k < n; ++k) q[k] += S[(int64_t)i * n + k] * (alpha[i] - beta);
    }
    for (int64_t k = 0; k < n; ++k) p[k] = -q[k];
}

int oracle_lbfgs(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                 int32_t n_struct, const double *params, const double *w, const double *t0,
                 int32_t max_iters, double tol, int32_t m, double c1, int32_t max_ls,
                 int32_t stop_window, int32_t max_evals, double *t_out, double *F_out,
                 int32_t *iters_out, int32_t *status_out, double *trace, int64_t *n_evals)
{
    if (m < 1 || m > 64 || max_ls < 1 || max_iters < 0 || stop_window < 1 || max_evals < 0 ||
        !t_out || !F_out || !iters_out || !status_out)
        return -1;
    const int64_t n = n_dwell;
    const size_t vb = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *x = malloc(vb), *g = malloc(vb), *p = malloc(vb), *xt = malloc(vb), *gt = malloc(vb);
    double *S = malloc(vb * (size_t)m), *Y = malloc(vb * (size_t)m);
    double rho[64];
    int64_t evals = 0;
    int rc = 0;
    if (!x || !g || !p || !xt || !gt || !S || !Y) { rc = -1; goto done; }

    /* non-negativity by substitution: x = t^(1/2), t = x^2 (Sec. 2.1.2) */
    for (int64_t l = 0; l < n; ++l) x[l] = t0 ? sqrt(t0[l]) : 1.0;

    double F;
    if (oracle_objective(A, n_pnt, n_dwell, sid, n_struct, params, w, x, &F, g, NULL, NULL)) {
        rc = -1; goto done;
    }
    evals++;
    if (trace) { trace[0] = F; trace[1] = 0.0; trace[2] = 0.0; }

    int32_t k = 0, status, n_small = 0;
    int32_t count = 0, newest = m - 1;
    if (!isfinite(F) || !all_finite(n, g)) { status = ORACLE_NONFINITE; goto finish; }
    if (F == 0.0 || norm_inf(n, g) == 0.0) { status = ORACLE_CONVERGED; goto finish; }

    for (;;) {
        if (k >= max_iters) { status = ORACLE_MAXITER; break; }
        double alpha0 = 1.0;
        if (count == 0) alpha0 = fmin(1.0, 1.0 / norm_inf(n, g));
        oracle_two_loop(n, m, count, newest, S, Y, rho, g, p);
        double gtp = dot(n, g, p);
        if (!(gtp < 0.0)) { /* not a descent direction: restart from steepest descent */
            count = 0;
            alpha0 = fmin(1.0, 1.0 / norm_inf(n, g));
            for (int64_t l = 0; l < n; ++l) p[l] = -g[l];
            gtp = dot(n, g, p);
        }
        /* backtracking Armijo line search: F(x + a p) <= F + c1 a g'p, a <- a / 2 */
        double alpha = alpha0, Ft = 0.0;
        int accepted = 0;
        int out_of_evals = 0;
        for (int32_t ls = 0; ls < max_ls; ++ls) {
            /* evaluation budget (first evaluation and every trial), 0 = none: stop at x */
            if (max_evals > 0 && evals >= max_evals) { out_of_evals = 1; break; }
            for (int64_t l = 0; l < n; ++l) xt[l] = x[l] + alpha * p[l];
            oracle_objective(A, n_pnt, n_dwell, sid, n_struct, params, w, xt, &Ft, gt, NULL, NULL);
            evals++;
            if (isfinite(Ft) && Ft <= F + c1 * alpha * gtp) { accepted = 1; break; }
            alpha *= 0.5;
        }
        if (out_of_evals) { status = ORACLE_MAXITER; break; }
        if (!accepted) {
            if (count > 0) { count = 0; continue; } /* retry once with steepest descent */
            status = ORACLE_LSFAIL;
            break;
        }
        /* curvature pair s = x_{k+1} - x_k, y = g_{k+1} - g_k, kept when s'y > 1e-12 y'y */
        double sy = 0.0, yy = 0.0;
        for (int64_t l = 0; l < n; ++l) {
            double s = xt[l] - x[l], y = gt[l] - g[l];
            sy += s * y;
            yy += y * y;
        }
        if (sy > 1e-12 * yy) {
            newest = (newest + 1) % m;
            for (int64_t l = 0; l < n; ++l) {
                S[(int64_t)newest * n + l] = xt[l] - x[l];
                Y[(int64_t)newest * n + l] = gt[l] - g[l];
            }
            rho[newest] = 1.0 / sy;
            if (count < m) count++;
        }
        double Fprev = F;
        memcpy(x, xt, vb);
        memcpy(g, gt, vb);
        F = Ft;
        k++;
        if (trace) { trace[3 * k] = F; trace[3 * k + 1] = alpha; trace[3 * k + 2] = gtp; }
        if (!all_finite(n, g)) { status = ORACLE_NONFINITE; break; }
        /* stop on the relative variation of the objective (Sec. 2.2.3), over stop_window
         * consecutive iterations */
        n_small = fabs(Fprev - F) <= tol * fmax(fabs(Fprev), 1e-300) ? n_small + 1 : 0;
        if (F == 0.0 || norm_inf(n, g) == 0.0 || n_small >= stop_window) {
            status = ORACLE_CONVERGED;
            break;
        }
    }
finish:
    for (int64_t l = 0; l < n; ++l) t_out[l] = x[l] * x[l];
    *F_out = F;
    *iters_out = k;
    *status_out = status;
done:
    if (n_evals) *n_evals = evals;
    free(x); free(g); free(p); free(xt); free(gt); free(S); free(Y);
    return rc;
}

int oracle_lbfgs_batch(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                       int32_t n_struct, const double *params, const double *W, int64_t P,
                       const double *T0, int32_t max_iters, double tol, int32_t m, double c1,
                       int32_t max_ls, int32_t stop_window, int32_t max_evals, double *T_out,
                       double *F_out, int32_t *iters_out, int32_t *status_out, int64_t *n_evals,
                       int32_t n_threads)
{
    int bad = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : bad)
#endif
    for (int64_t j = 0; j < P; ++j) {
        int64_t ev = 0;
        int r = oracle_lbfgs(A, n_pnt, n_dwell, sid, n_struct, params, W + j * n_struct,
                             T0 ? T0 + j * n_dwell : NULL, max_iters, tol, m, c1, max_ls,
                             stop_window, max_evals, T_out + j * n_dwell, F_out + j, iters_out + j,
                             status_out + j, NULL, &ev);
        if (n_evals) n_evals[j] = ev;
        bad |= (r != 0);
    }
    (void)n_threads;
    return bad ? -1 : 0;
}

/* ------------------------------------------------ simulated annealing engine (gSA, Sec. 2.2.1) */
/* Output n of the SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) seeded with
 * `seed`: the state after n + 1 steps of the Weyl sequence seed + k * 0x9E3779B97F4A7C15,
 * passed through the generator's finaliser. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter of the draw for plan p, iteration k and dwell l (l = 2^21 - 1: the acceptance draw) */
static uint64_t sa_counter(int64_t p, int32_t k, int64_t l)
{
    return ((uint64_t)k << 42) | ((uint64_t)p << 21) | (uint64_t)l;
}

/* Geometric interpolation from a to b over the run: a (b / a)^(k / (K - 1)); 0 when a = 0 */
static double sa_schedule(double a, double b, int32_t k, int32_t K)
{
    if (a == 0.0) return 0.0;
    const double f = K > 1 ? (double)k / (double)(K - 1) : 0.0;
    return a * pow(b / a, f);
}

int oracle_sa(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
              int32_t n_struct, const double *params, const double *w, const double *t0,
              int64_t plan, int32_t iters, uint64_t seed, double T0, double T_final, double step0,
              double step_final, double *t_out, double *F_out, int32_t *accepts_out,
              double *min_margin_out, double *trace)
{
    if (!A || !sid || !params || !w || !t_out || !F_out || n_dwell < 1 || n_dwell >= (1 << 21) - 1 ||
        plan < 0 || plan >= (1 << 21) || iters < 0 || iters >= (1 << 22) || !(T0 >= 0.0) ||
        !(T_final >= 0.0) || !(step0 >= 0.0) || !(step_final >= 0.0) || !isfinite(T0) ||
        !isfinite(T_final) || !isfinite(step0) || !isfinite(step_final) ||
        (T0 == 0.0) != (T_final == 0.0) || (step0 == 0.0) != (step_final == 0.0))
        return -1;
    double *x = malloc((size_t)n_dwell * sizeof(double));
    double *xt = malloc((size_t)n_dwell * sizeof(double));
    double *xb = malloc((size_t)n_dwell * sizeof(double));
    for (int64_t l = 0; l < n_dwell; ++l) {
        x[l] = t0 ? sqrt(t0[l]) : 1.0;
        xb[l] = x[l];
    }
    double F0 = 0.0;
    if (oracle_objective(A, n_pnt, n_dwell, sid, n_struct, params, w, x, &F0, NULL, NULL, NULL) != 0) {
        free(x); free(xt); free(xb);
        return -1;
    }
    double F = F0, Fb = F0, min_margin = INFINITY;
    int32_t acc = 0;
    if (trace) trace[0] = F;
    for (int32_t k = 0; k < iters; ++k) {
        /* step (ii): every dwell weight moves by a uniform draw in [-delta_k, delta_k) */
        const double delta = sa_schedule(step0, step_final, k, iters);
        const double temp = sa_schedule(T0, T_final, k, iters);
        for (int64_t l = 0; l < n_dwell; ++l) {
            const uint64_t z = oracle_splitmix64(seed, sa_counter(plan, k, l));
            const double r = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
            xt[l] = x[l] + delta * r;
        }
        /* steps (iii)-(v): dose, penalties and the plan's objective at the moved weights */
        double Ft = 0.0;
        oracle_objective(A, n_pnt, n_dwell, sid, n_struct, params, w, xt, &Ft, NULL, NULL, NULL);
        /* Metropolis: accept when F_t - F <= -T_k F_0 ln v, v uniform in (0, 1] */
        const uint64_t zv = oracle_splitmix64(seed, sa_counter(plan, k, (1 << 21) - 1));
        const double v = ((double)(zv >> 11) + 1.0) * 0x1.0p-53;
        const double theta = -temp * F0 * log(v);
        const double dF = Ft - F;
        const double scale = fmax(fabs(F), fabs(Ft));
        const double margin = fabs(dF - theta) / (scale > 0.0 ? scale : 1.0);
        if (margin < min_margin) min_margin = margin;
        if (dF <= theta) {
            F = Ft;
            memcpy(x, xt, (size_t)n_dwell * sizeof(double));
            ++acc;
            if (Ft < Fb) {
                Fb = Ft;
                memcpy(xb, xt, (size_t)n_dwell * sizeof(double));
            }
        }
        if (trace) trace[k + 1] = F;
    }
    for (int64_t l = 0; l < n_dwell; ++l) t_out[l] = xb[l] * xb[l];
    *F_out = Fb;
    if (accepts_out) *accepts_out = acc;
    if (min_margin_out) *min_margin_out = min_margin;
    free(x); free(xt); free(xb);
    return 0;
}

int oracle_sa_batch(const double *A, int64_t n_pnt, int64_t n_dwell, const int32_t *sid,
                    int32_t n_struct, const double *params, const double *W, int64_t P,
                    const double *T0s, int32_t iters, uint64_t seed, double T0, double T_final,
                    double step0, double step_final, double *T_out, double *F_out,
                    int32_t *accepts_out, double *min_margin_out, int32_t n_threads)
{
    int bad = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : bad)
#endif
    for (int64_t j = 0; j < P; ++j) {
        int r = oracle_sa(A, n_pnt, n_dwell, sid, n_struct, params, W + j * n_struct,
                          T0s ? T0s + j * n_dwell : NULL, j, iters, seed, T0, T_final, step0,
                          step_final, T_out + j * n_dwell, F_out + j,
                          accepts_out ? accepts_out + j : NULL,
                          min_margin_out ? min_margin_out + j : NULL, NULL);
        bad |= (r != 0);
    }
    (void)n_threads;
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------- DVH indices (Sec. 2.3.1) */
static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* k-th largest dose of structure s (1-based k), by sorting */
static double kth_largest(const double *d, const int32_t *sid, int64_t n_pnt, int32_t s,
                          int64_t k)
{
    int64_t n = 0;
    for (int64_t i = 0; i < n_pnt; ++i) n += (sid[i] == s);
    double *v = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int64_t j = 0;
    for (int64_t i = 0; i < n_pnt; ++i) if (sid[i] == s) v[j++] = d[i];
    qsort(v, (size_t)n, sizeof(double), cmp_desc);
    double r = v[k - 1];
    free(v);
    return r;
}

void oracle_dvh(const double *d, const int32_t *sid, int64_t n_pnt, int32_t n_struct, double rx,
                double *out)
{
    int64_t N[4] = {0, 0, 0, 0}, v100 = 0, v75r = 0, v75b = 0;
    for (int64_t i = 0; i < n_pnt; ++i) {
        if (sid[i] >= 0 && sid[i] < 4) N[sid[i]]++;
        if (sid[i] == 0 && d[i] >= rx) v100++;
        if (sid[i] == 2 && d[i] >= 0.75 * rx) v75r++;
        if (sid[i] == 3 && d[i] >= 0.75 * rx) v75b++;
    }
    for (int q = 0; q < 5; ++q) out[q] = NAN;
    if (n_struct > 0 && N[0] > 0) {
        out[0] = 100.0 * (double)v100 / (double)N[0];
        int64_t k90 = (9 * N[0] + 9) / 10; /* ceil(0.9 N) in integers */
        out[1] = 100.0 * kth_largest(d, sid, n_pnt, 0, k90) / rx;
    }
    if (n_struct > 1 && N[1] > 0) {
        int64_t k10 = (N[1] + 9) / 10; /* ceil(0.1 N) */
        out[2] = 100.0 * kth_largest(d, sid, n_pnt, 1, k10) / rx;
    }
    if (n_struct > 2 && N[2] > 0) out[3] = 100.0 * (double)v75r / (double)N[2];
    if (n_struct > 3 && N[3] > 0) out[4] = 100.0 * (double)v75b / (double)N[3];
}
