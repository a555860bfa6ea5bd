/*
 * topomag -- C ABI of the GPU (sm_103a) finite-difference magnet topology
 * optimizer: the FFT-accelerated stray-field operator, its adjoint gradient and
 * a projected-gradient update, after Abert et al., "A fast finite-difference
 * algorithm for topology optimization of permanent magnets" (arXiv:1707.09898).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Geometry. The output grid has n_out = (nx, ny, nz) cuboid cells of size
 *   cellsize = (dx, dy, dz) metres. The design box is its bottom slab
 *   z in [0, nzd) with the same nx, ny. The density rho lives on the design box
 *   (rho = 0, hence M = 0, outside it); fields live on the output grid.
 * Layout. Every array is a C-contiguous float32 (or uint8) array:
 *   rho, dJdrho      [nzd][ny][nx]
 *   H, gH, H_target  [3][nz][ny][nx]   (component-major: x, y, z)
 *   mask             [nz][ny][nx]      (uint8, nonzero = target cell)
 *   M0 (varying)     [3][nzd][ny][nx]  (A/m)
 * Units. M0 and H in A/m; J in (A/m)^2 times the weights.
 * Memory. Array pointers are DEVICE pointers on the context's device, owned by
 *   the caller; the library never frees them. 16-byte alignment is recommended
 *   (the update kernel vectorises when both of its arrays are aligned).
 *   The library owns the tensor, twiddle tables and workspace of a context.
 * Streams. `stream` is a cudaStream_t (NULL = legacy default stream). Calls
 *   enqueue their kernels on it and return without synchronising, except where
 *   stated (tm_set_tensor, and tm_objective_and_gradient with J_host != NULL).
 *   A context must not be used from two host threads at once, and calls on one
 *   context must not overlap on the GPU (they share its workspace).
 * Errors. Every int-returning call returns TM_OK (0) or a negative code and then
 *   leaves a message for tm_last_error(). Nothing is thrown across the ABI.
 *   Kernels never spin without a bound: a wait that runs out sets a bit of the
 *   context's device status word, which tm_evaluate / tm_evaluate_step (with
 *   J_host != NULL) and tm_get_objective read and report as TM_ERR_TIMEOUT.
 */
#ifndef TOPOMAG_H
#define TOPOMAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TM_OK 0
#define TM_ERR_ARG (-1)      /* null/invalid argument */
#define TM_ERR_SIZE (-2)     /* grid outside the supported sizes */
#define TM_ERR_STATE (-3)    /* call order: e.g. no grid, no tensor, no M0 */
#define TM_ERR_CUDA (-4)     /* a CUDA call failed (message has the CUDA error) */
#define TM_ERR_NOMEM (-5)    /* device allocation failed */
#define TM_ERR_TIMEOUT (-6)  /* a bounded wait inside a kernel ran out; that call's results are invalid */
#define TM_ERR_INJECTED (-7) /* failure forced by the fault-injection hook (tm_inject_fault) */

typedef struct tm_ctx tm_ctx;

/* Create a context bound to CUDA device `device`. *out receives the handle. */
int tm_create(tm_ctx** out, int device);

/* Release the context and everything it owns (not the caller's arrays). */
void tm_destroy(tm_ctx* ctx);

/* Message of the last failing call on ctx (empty string if none). */
const char* tm_last_error(const tm_ctx* ctx);

/* Library version string. */
const char* tm_version(void);

/*
 * Grid (Sec. "Discretization": regular cuboid grid, Eq. (convolution)).
 * n_out[3] = (nx, ny, nz), each in [4, 288]; 1 <= nzd <= nz; cellsize[3] > 0.
 * Each axis is zero padded to a length L >= 2 n (open boundaries): the smallest
 * supported even 2^a 3^b >= 2 n, except that 288 and 384 are replaced by 512, whose
 * 32 x 16 plan has the fused kernels (any L >= 2 n gives the same linear
 * convolution). Allocates the workspace; discards tensor and M0.
 * TM_ERR_SIZE if an axis is outside the supported range.
 */
int tm_set_grid(tm_ctx* ctx, const int n_out[3], int nzd, const double cellsize[3]);

/*
 * tm_set_grid with chosen padded lengths: L[a] = 0 takes the default of tm_set_grid,
 * otherwise L[a] must be one of the supported lengths (even 2^a 3^b from 8 to 576 with
 * at most two factors 3) and >= 2 n_out[a], else TM_ERR_SIZE and nothing changes.
 * L may be NULL (all defaults). Counts as tm_set_grid for TM_FAULT_INJECT.
 */
int tm_set_grid_lengths(tm_ctx* ctx, const int n_out[3], int nzd, const double cellsize[3], const int L[3]);

/* The padded length tm_set_grid picks for an axis of n cells (1 <= n <= 288), else 0.
 * Needs no context and no GPU. */
int tm_default_fft_length(int n);

/* The padded FFT lengths (Lx, Ly, Lz) chosen by tm_set_grid. */
int tm_get_fft_lengths(const tm_ctx* ctx, int L[3]);

/* Penalty exponent p of M = rho^p M0 (Sec. "Methodology", Eq. 2). Default 3. p >= 1. */
int tm_set_penalty(tm_ctx* ctx, double p);

/*
 * Prescribed magnetization M0 (Sec. "Methodology", Eq. 2): spatially constant
 * (M0_dev == NULL, M0_const[3] in A/m) or varying (M0_dev = device array
 * [3][nzd][ny][nx], copied into the context on `stream`).
 */
int tm_set_M0(tm_ctx* ctx, const float* M0_dev, const double M0_const[3], void* stream);

/*
 * Demagnetization tensor (Sec. "Discretization", Eq. (demag_tensor)) in float64
 * on the device: Newell's closed form for offsets with max(|i|,|j|,|k|) <= 16,
 * a tent-averaged dipole rule beyond; transformed once, scaled by
 * -1/(Lx Ly Lz) and stored as float32. Synchronises `stream`. Setup only.
 */
int tm_set_tensor(tm_ctx* ctx, void* stream);

/*
 * Stray field H = D[M(rho)] = -sum_j N(i - j) rho_j^p M0_j on the output grid
 * (Sec. "Discretization", Eq. (convolution); Sec. "Methodology", Eq. 2).
 * rho [nzd][ny][nx] in [0, 1] -> H [3][nz][ny][nx].
 */
int tm_stray_field(tm_ctx* ctx, const float* rho, float* H, void* stream);

/*
 * Adjoint of tm_stray_field w.r.t. rho for an arbitrary cotangent gH:
 * dJdrho_j = p rho_j^(p-1) M0_j . (D gH)_j, D self-adjoint (Sec. "Methodology",
 * Eqs. (adjoint1)-(adjoint2) and the operator form of the gradient).
 * gH [3][nz][ny][nx] -> dJdrho [nzd][ny][nx].
 */
int tm_stray_field_adjoint(tm_ctx* ctx, const float* rho, const float* gH, float* dJdrho, void* stream);

/*
 * Objective and adjoint gradient (Sec. "Methodology", Eq. (objective_function)
 * and Eqs. (adjoint1)-(adjoint2)) for the least-squares objective
 *   J = sum_{i: mask_i != 0} sum_c w_c (H_{i,c} - Ht_{i,c})^2,
 * with Ht = H_target (device [3][nz][ny][nx]) or, if H_target == NULL, the
 * constant vector Ht_const[3]. w[3] are host floats.
 * Writes dJdrho [nzd][ny][nx]; H_out (device [3][nz][ny][nx]) if not NULL.
 * J (float64) is kept on the device; if J_host != NULL the call synchronises
 * `stream` and stores it there, else read it later with tm_get_objective.
 */
int tm_objective_and_gradient(tm_ctx* ctx, const float* rho, const uint8_t* mask, const float* H_target,
                              const float Ht_const[3], const float w[3], double* J_host, float* dJdrho,
                              float* H_out, void* stream);

/*
 * Prepared objective for an optimisation loop (the same J and dJ/drho as
 * tm_objective_and_gradient). tm_set_target copies mask [nz][ny][nx] and
 * H_target (or the constant Ht_const) and the weights w into the context and
 * finds the z planes that hold target cells (synchronises `stream`, once).
 * tm_evaluate(rho) then returns J (as tm_objective_and_gradient, J_host may be
 * NULL) and writes dJdrho. When the target occupies at most 8 planes, the z
 * part of the convolution is summed directly in (kx, ky, z) space onto those
 * planes (forward) and from them (adjoint), with the tensor transformed along
 * x and y only -- the same discrete convolution (Eq. (convolution)) without the
 * z transforms; otherwise it runs the full pipeline.
 */
int tm_set_target(tm_ctx* ctx, const uint8_t* mask, const float* H_target, const float Ht_const[3], const float w[3],
                  void* stream);
int tm_evaluate(tm_ctx* ctx, const float* rho, double* J_host, float* dJdrho, void* stream);

/*
 * Prepared quadratic stencil objective for tm_evaluate (instead of tm_set_target):
 *   J = sum_k c_k r_k^2,   r_k = sum_{e in row k} a_e H[comp_e][cell_e],
 * a quadratic form in linear combinations of field values. It expresses the
 * field-and-gradient objective of Sec. "Optimization of field and gradient"
 * (rows of one field value with c = -1/2, and rows of a finite-difference normal
 * derivative with c = -beta/2); dJ/dH = 2 S^T diag(c) S H is its exact partial
 * derivative, and dJ/drho follows by the adjoint as for tm_set_target.
 * HOST arrays, copied: row_ptr [K+1] (row k holds entries row_ptr[k] ..
 * row_ptr[k+1]-1, row_ptr[0] = 0), per entry comp (0..2), cell (z*ny*nx + y*nx + x
 * on the output grid) and coefficient a; per row the weight c. A cell may appear
 * in several rows and twice in one row. K = 0 gives J = 0. When the referenced
 * cells lie on at most 8 consecutive z planes, tm_evaluate computes H only there
 * (direct z sums as for tm_set_target); otherwise on the whole grid. Synchronises
 * `stream`. TM_ERR_ARG for indices out of range or non-finite coefficients.
 */
int tm_set_stencil_objective(tm_ctx* ctx, long long K, const long long* row_ptr, const int* comp,
                             const long long* cell, const double* a, const double* c, void* stream);

/* J of the last tm_objective_and_gradient or tm_evaluate (synchronises `stream`). */
int tm_get_objective(tm_ctx* ctx, double* J_host, void* stream);

/*
 * Asynchronous form: enqueue on `stream` a copy of that J (one double) to dst, pinned
 * host or device memory (any address cudaMemcpyAsync accepts with cudaMemcpyDefault).
 * Returns at once; dst holds J once the stream reaches the copy (record an event after
 * the call and wait for it). Lets a loop read each iteration's J without stalling the
 * GPU: queue iteration i + 1, then wait for J(i).
 */
int tm_copy_objective(tm_ctx* ctx, double* dst, void* stream);

/*
 * Projected-gradient step on the box 0 <= rho <= 1 (box constraint of Sec.
 * "Methodology"): rho <- clip(rho - alpha G / max|G|, 0, 1) if normalize != 0
 * (no change when max|G| = 0), else rho <- clip(rho - alpha G, 0, 1).
 * rho [nzd][ny][nx] updated in place; G = dJdrho [nzd][ny][nx].
 * normalize == 2: as 1, but when dJdrho is the array the last evaluation on this
 * context wrote (tm_evaluate, tm_objective_and_gradient, tm_stray_field_adjoint),
 * max|G| is taken from that evaluation instead of being recomputed; the caller
 * promises not to have changed dJdrho since. Any other array: recomputed.
 */
int tm_optimize_step(tm_ctx* ctx, float* rho, const float* dJdrho, float alpha, int normalize, void* stream);

/*
 * One iteration of the projected-gradient loop (Sec. "Methodology") in a single call:
 * the step of tm_optimize_step on the gradient dJdrho holds (normally the one the
 * previous evaluation wrote), then tm_evaluate at the new rho, which overwrites
 * dJdrho with the new gradient. Same results, bit for bit, as
 *   tm_optimize_step(ctx, rho, dJdrho, alpha, normalize, stream);
 *   tm_evaluate(ctx, rho, J_host, dJdrho, stream);
 * A loop starts with one tm_evaluate and then calls this once per iteration.
 * rho [nzd][ny][nx] updated in place; normalize as for tm_optimize_step (2 reuses
 * max|dJdrho| from the evaluation that wrote it). Where the prepared path transforms
 * rho as one spectrum along x with L = 512 (constant M0, target on at most 8 planes),
 * the step is applied inside that first pass, which then writes the new rho; in every
 * other case it runs as its own pass first. Requires tm_set_target. Errors as
 * tm_evaluate; TM_ERR_ARG for null arrays or a non-finite alpha.
 */
int tm_evaluate_step(tm_ctx* ctx, float* rho, float alpha, int normalize, double* J_host, float* dJdrho,
                     void* stream);

/*
 * Allocation-free projected-gradient step (no context needed). For callers that
 * must not allocate device memory when they call in: code running under a
 * framework whose caching allocator has reserved the device memory (a fresh
 * cudaMalloc may then fail), and time-critical loops that cannot absorb the
 * device-wide synchronisation that cudaMalloc/cudaFree imply. The paper has no
 * counterpart; this is an interface convenience around the update of
 * tm_optimize_step and gives the same result.
 *   rho [n] updated in place, dJdrho [n]: device pointers on the CURRENT device.
 *   normalize != 0: rho <- clip(rho - alpha G / max|G|, 0, 1) (no change when
 *   max|G| = 0); else rho <- clip(rho - alpha G, 0, 1).
 * Scratch: a 64 KiB static device array in the library (held by every GPU that
 * loads it until the process exits) stores the max|G| reduction, so at most
 * n = 33,554,432 elements per call; larger n returns TM_ERR_SIZE without
 * launching anything. Every call reuses that one array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) once; make that first call before any stream
 * capture. Returns TM_OK, TM_ERR_ARG, TM_ERR_SIZE or TM_ERR_CUDA; there is no
 * context, so no message is kept for tm_last_error.
 */
int tm_optimize_step_noalloc(float* rho, const float* dJdrho, long long n, float alpha, int normalize,
                             void* stream);

/*
 * Validation of a density (the box constraint 0 <= rho <= 1 of Sec. "Methodology",
 * after Eq. 1): counts the entries of rho [nzd][ny][nx] that are NaN or outside
 * [0, 1] and stores the count in *n_bad (host). Synchronises `stream`. Returns
 * TM_ERR_ARG (with the count in the message) when any entry is bad, else TM_OK.
 * The evaluation calls do not check their input; a loop calls this where it takes
 * rho from outside (a start, a resume).
 */
int tm_check_design(tm_ctx* ctx, const float* rho, long long* n_bad, void* stream);

/*
 * Per-iteration quantities of an optimisation run (the volume fraction is the
 * quantity of Fig. 4, the share of intermediate densities that of Fig. 3, Sec.
 * "Validation and Benchmarks"): out[0] = max_j |dJdrho_j|, out[1] = sum_j rho_j / N,
 * out[2] = #{j : 0.1 < rho_j < 0.9} / N over the N design cells. float64 sums in a
 * fixed order (the same bits on every call). Synchronises `stream`.
 */
int tm_iteration_stats(tm_ctx* ctx, const float* rho, const float* dJdrho, double out[3], void* stream);

/*
 * Fault injection (test support; the paper has no counterpart). After
 * tm_inject_fault(call, nth), the nth following call of the entry point named
 * `call` (e.g. "tm_evaluate") in this process returns TM_ERR_INJECTED before it
 * does anything, so the context is left as it was; later calls run normally.
 * nth <= 0 or call == NULL disarms. The environment variable
 * TM_FAULT_INJECT=<call>[:<nth>] (nth default 1), read when the library loads,
 * arms it the same way. Every int-returning tm_* entry point that takes a context
 * honours it.
 */
int tm_inject_fault(const char* call, long long nth);

/*
 * Self-test of the bounded waits (test support; no counterpart in the paper).
 * The kernels that receive copies from the tensor memory accelerator wait on an
 * mbarrier with a bounded number of polls; when the bound runs out they set a bit
 * of the context's device status word and return instead of hanging, and the host
 * reports TM_ERR_TIMEOUT. This call launches one block that waits, at most `polls`
 * polls (1 <= polls <= 65536, about a microsecond each), on an mbarrier phase that
 * no copy and no thread completes; it synchronises `stream` and returns
 * TM_ERR_TIMEOUT with the status bit seen (the bit is then cleared), or TM_ERR_CUDA
 * if the bit was not set.
 */
int tm_selftest_wait_timeout(tm_ctx* ctx, int polls, void* stream);

/*
 * Prepared path (tm_evaluate): 1 (default) fuses the y transform of the design
 * planes with the direct z sum when one spectrum meets one target plane (constant
 * M0, one weighted field component): forward onto the plane, adjoint from it, so
 * the y spectra of the design planes never reach memory; 0, or any other case,
 * runs the y and z passes separately. Same convolution either way.
 */
int tm_set_fused(tm_ctx* ctx, int on);

/*
 * Per-kernel timing. tm_profile(ctx, 1) starts recording a CUDA event pair on
 * the launch stream around every kernel the context launches (and resets the
 * record); tm_profile(ctx, 0) stops. tm_profile_read synchronises on the
 * recorded events and returns, per kernel kind, the summed event time in ms and
 * the launch count. Kinds: 0 x forward, 1 y forward, 2 z pass (forward z FFT,
 * tensor product, inverse z FFT; or the direct z sum), 3 y inverse, 4 x inverse
 * (+ objective or chain rule), 5 other (reductions, update), 6 fused y forward +
 * direct z sum, 7 fused direct z sum + y inverse (tm_set_fused), 8 the objective
 * on the target rows of the prepared path (x inverse, J, dJ/dH, x forward).
 */
int tm_profile(tm_ctx* ctx, int on);
int tm_profile_read(tm_ctx* ctx, double ms[9], int launches[9]);

/*
 * Inspection (tests): the float64 tensor N at the offsets of the non-negative
 * octant, host array [6][nz][ny][nx] (components xx, yy, zz, xy, xz, yz), and
 * the stored float32 transformed tensor, host array [6][Lz/2+1][Ly/2+1][Lx/2+1]
 * (already multiplied by -1/(Lx Ly Lz)). Both synchronise `stream`.
 */
int tm_debug_tensor_octant(tm_ctx* ctx, double* host_out, void* stream);
int tm_debug_tensor_spectrum(tm_ctx* ctx, float* host_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TOPOMAG_H */
