/*
 * fvns_host.h -- host-only helpers of libfvns, exported so that the host
 * logic of the library can be checked without a GPU.  None of them launches
 * a kernel.
 */
#ifndef FVNS_HOST_H
#define FVNS_HOST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eigenvalues (wr + i wi, unordered) of the m x m row-major upper
 * Hessenberg H by the Francis double-shift QR iteration, the dense step of
 * the Arnoldi method of Section 3.  Returns 0, or 4 if it did not converge. */
int fv_host_hess_eigenvalues(int m, const double* H, double* wr, double* wi);

/* Apply nshift implicit shifted-QR steps to the Hessenberg H (in place) and
 * accumulate them into Q (m x m, row-major): a conjugate pair (sr, +-si)
 * as one Francis double-shift step, a real shift as a Givens bulge chase.
 * These are the implicit restarts of the Arnoldi method. */
int fv_host_shift_steps(int m, double* H, double* Q, int nshift, const double* sr,
                        const double* si);

/* Float-float conversions used by the mixed-precision SIMPLE loop:
 * hi = nearest float to in, lo = nearest float to in - hi, joined = the
 * float64 of hi + lo, rounded = nearest float (any output may be NULL). */
int fv_host_ff_convert(int64_t n, const double* in, float* hi, float* lo, double* joined,
                       float* rounded);

/* The float-float dot product of the mixed and float-float Krylov-basis
 * kernels, run on the host: out = sum a_i b_i, each double split by
 * truncation into two floats (|d - hi - lo| < 2^-46 |d|), products and sums
 * in float-float arithmetic (about 2^-47 per step), the result joined to the
 * nearest double.  Returns FV_EINVAL on NULL pointers or n < 0. */
int fv_host_ff_dot(int64_t n, const double* a, const double* b, double* out);

/* Float-float arithmetic check: out = (a + b) * c, operands as (hi, lo) pairs. */
int fv_host_ff_arith(int64_t n, const float* a, const float* b, const float* c, float* out);

/* The 1-D multigrid hierarchy of fv_pressure_solve_mg along one axis with n
 * cells and stretching map: the axis at coarsening level `level` (n_out
 * cells; faces[n_out + 1] its faces, every other face of the level above and
 * the last one) and the prolongation from the next coarser level to it:
 * fine cell m takes (1 - pw1[m]) x_c[pc0[m]] + pw1[m] x_c[pc0[m] + 1]
 * (pc0, pw1 of n_out entries; any output pointer may be NULL except n_out).
 * An axis of at most 2 cells is not coarsened.  Returns 0 or FV_EINVAL. */
int fv_host_mg_axis(int n, int map, int level, int* n_out, double* faces, int* pc0, double* pw1);

/* Number of grids in the multigrid hierarchy of an nx x ny x nz grid (the
 * finest included): coarsening continues while an axis has more than 4
 * cells.  -1 on a bad size. */
int fv_host_mg_levels(int nx, int ny, int nz);

#ifdef __cplusplus
}
#endif

#endif /* FVNS_HOST_H */
