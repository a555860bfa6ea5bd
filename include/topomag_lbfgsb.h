/*
 * topomag_lbfgsb -- the bound-constrained limited-memory BFGS method (L-BFGS-B)
 * on the GPU, for minimising the topology objective over 0 <= rho <= 1.
 *
 * The paper minimises its objective with a quasi-Newton method that handles the
 * box constraint on the density, SciPy's L-BFGS-B, for every stray-field method
 * it compares (Sec. "Discretization"; Sec. "Validation and Benchmarks", Table I,
 * whose N_iter counts L-BFGS-B iterations). This is
 * that method (Byrd, Lu, Nocedal and Zhu 1995, with the projected subspace step
 * of Morales and Nocedal 2011 and the line search of More and Thuente 1994),
 * with the iterate, gradient, correction pairs and every length-n operation on
 * the device in float64:
 *   generalized Cauchy point   breakpoints sorted on the device (radix sort),
 *                              f' and f'' at every breakpoint by prefix sums,
 *                              first segment that holds the minimiser;
 *   subspace minimisation      direct primal method on the free variables,
 *                              projected onto the box, with the backtracking
 *                              fallback when the projected step is not descent;
 *   line search                More-Thuente (ftol 1e-3, gtol 0.9, xtol 0.1),
 *                              at most maxls evaluations, first trial step 1.
 * Stopping tests as SciPy's: max_i |P(x - g) - x|_i <= pgtol, or
 * (f_k - f_{k+1}) / max(|f_k|, |f_{k+1}|, 1) <= factr * eps_machine.
 * The only difference from the sequential breakpoint loop: the curvature
 * safeguard f'' >= eps * f''_0 is applied at each breakpoint to the exact f''
 * rather than carried through the recursion (identical unless it engages).
 *
 * Reverse communication. The caller owns the objective:
 *   tm_lbfgsb_start(x0) -> task = TM_LB_FG, x_eval = P(x0)
 *   loop: task == TM_LB_FG:    evaluate f and g at x_eval, tm_lbfgsb_iterate(f, g)
 *         task == TM_LB_NEW_X: an iteration finished, x_eval = the new iterate;
 *                              tm_lbfgsb_iterate (f, g ignored) continues
 *         otherwise: stopped (TM_LB_CONV_*, TM_LB_ABNORMAL)
 * x0, x_eval and g are device arrays of n elements, float32 or float64: pass one
 * of the two pointers of each pair (the other NULL); x_eval may name both.
 * Calls synchronise the stream (they read reductions back to the host).
 * Errors: TM_OK or a negative TM_ERR_* code, message in tm_lbfgsb_last_error.
 */
#ifndef TOPOMAG_LBFGSB_H
#define TOPOMAG_LBFGSB_H

#ifdef __cplusplus
extern "C" {
#endif

#define TM_LB_FG 1
#define TM_LB_NEW_X 2
#define TM_LB_CONV_PGTOL 3   /* projected-gradient test met */
#define TM_LB_CONV_REL_F 4   /* relative-reduction test met */
#define TM_LB_ABNORMAL 5     /* line search failed with an empty memory */

typedef struct tm_lbfgsb tm_lbfgsb;

/* n variables with lower <= x_i <= upper; m correction pairs (1..16; SciPy's default 10);
 * factr (SciPy default 1e7), pgtol (1e-5), maxls (20). */
int tm_lbfgsb_create(tm_lbfgsb** out, int device, long long n, int m, double lower, double upper, double factr,
                     double pgtol, int maxls);
void tm_lbfgsb_destroy(tm_lbfgsb* opt);
const char* tm_lbfgsb_last_error(const tm_lbfgsb* opt);

/* Project x0 onto the box; *task = TM_LB_FG with x_eval = the projected point. */
int tm_lbfgsb_start(tm_lbfgsb* opt, const float* x0_f32, const double* x0_f64, float* xeval_f32, double* xeval_f64,
                    int* task, void* stream);

/* Continue after TM_LB_FG (f, g = objective and gradient at x_eval) or TM_LB_NEW_X (f, g unused). */
int tm_lbfgsb_iterate(tm_lbfgsb* opt, double f, const float* g_f32, const double* g_f64, float* xeval_f32,
                      double* xeval_f64, int* task, void* stream);

/* counts[0..4] = iterations, evaluations, pairs in memory, breakpoints of the last Cauchy
 * point, free variables of the last subspace step; values[0..2] = f, projected-gradient
 * infinity norm, theta (the scaling of the limited-memory matrix). */
int tm_lbfgsb_info(const tm_lbfgsb* opt, long long counts[5], double values[3]);

#ifdef __cplusplus
}
#endif

#endif /* TOPOMAG_LBFGSB_H */
