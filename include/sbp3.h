/*
 * libsbp, 3-D operator -- C-ABI of the GB300 (sm_103a) SBP-SAT elastic operator in three
 * dimensions on one curvilinear block (the paper states the scheme for d dimensions:
 * Sec. 3.2-3.3 with eq. surfj_app_3d for the metric, Sec. 4.3-4.7 for the operator, Sec. 5 for
 * the boundary SATs with the penalty of Theorem 3 at d = 3).
 *
 * Per node the scheme is rho J u_j'' = sum_ik DD_ik(c_ijkl) u_l + J SAT_j with
 * c_ijkl = J F_Ii C_IjKl F_Kk (F = G^-1, G_iI = D_i X_I), DD_ii the narrow operator D_xx^FC(c)
 * along direction i and DD_ik = D_i c D_k for i != k.  Faces carry either the traction SAT
 * (Robin face of eq. sat_traction with U = 0, g = 0) or the displacement SAT (eq.
 * dirichlet_ansatz with g = 0, J^ Z_JL = beta d / h1 c_mJmL, d = 3).  Time stepping is leapfrog,
 * u^{n+1} = 2 u^n - u^{n-1} + dt^2 (rho J)^-1 [ DD(c) u^n + J SAT(u^n) ].
 *
 * Conventions
 *  - Status codes, precisions and sbp_last_error-style messages as in sbp.h; every call returns
 *    SBP_OK or a negative SBP_E_* code and never aborts.  sbp3_last_error describes the last
 *    failure of a handle (or of sbp3_create when passed NULL).
 *  - The block has n1 x n2 x n3 nodes; node (i1, i2, i3) of a host array sits at index
 *    (i3 * n2 + i2) * n1 + i1 (x1 fastest).  Vector fields hold their three components one after
 *    the other (component stride n1 n2 n3).  Faces: 0: x1=0, 1: x1=1, 2: x2=0, 3: x2=1,
 *    4: x3=0, 5: x3=1.
 *  - Host arrays passed in are copied (the caller keeps ownership); host arrays written out are
 *    caller-allocated.  Host values are double precision.  Device memory is owned by the handle.
 *  - Orders 2, 4, 6 need n_i >= 5, 18, 27 nodes per direction; n2, n3 <= 65535 and an x3-plane
 *    (n1 rounded up to 128 bytes, times n2) below 2^27 elements (SBP_E_INVALID_ARG otherwise).
 */
#ifndef SBP3_H
#define SBP3_H

#include "sbp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SBP3_BC_DISPLACEMENT 0   /* u = 0 weakly, SAT of eq. dirichlet_ansatz */
#define SBP3_BC_TRACTION 1       /* traction-free, SAT of eq. sat_traction with U = 0 */

#define SBP3_PROF_FAMILIES 3     /* 0: k3_flux, 1: k3_div_int, 2: k3_div_shell (with the face SATs) */

typedef struct sbp3_handle sbp3_handle;

/* Create the block and compute its metric on the device.  X: 3 * n1*n2*n3 physical node
 * coordinates (X_1, X_2, X_3 one after the other); face_kinds: six SBP3_BC_* values;
 * beta >= 1 the penalty factor.  The material must then be set for every x3-plane
 * (sbp3_set_material) before sbp3_step or sbp3_apply. */
int sbp3_create(int order, int precision, int n1, int n2, int n3, const double* X, const int* face_kinds,
                double beta, sbp3_handle** out);
/* Synchronizes the device and frees every buffer of the handle; h is invalid afterwards. */
int sbp3_destroy(sbp3_handle* h);
/* Message of the last failed call on h (of the last failed sbp3_create when h is NULL); owned by
 * the library, valid until the next call on the same handle. */
const char* sbp3_last_error(const sbp3_handle* h);

/* Device bytes a handle of this order, precision and size holds: 64 words per node (45 coefficients,
 * 1/(rho J), two levels, the increment, 9 fluxes), the FP64 coordinates and the x1 closure
 * matrices of D_xx^FC (2 x NCLOS x NCLOSJ x 6 words per x1 line). */
int sbp3_footprint(int order, int precision, int n1, int n2, int n3, long long* bytes_out);

/* Density and stiffness of the x3-planes i3_begin <= i3 < i3_begin + i3_count (any chunking).
 * rho: i3_count*n2*n1 values; C45: 45 * (i3_count*n2*n1) values, entry t of the upper triangle
 * (row-major) of the 9 x 9 pair matrix M[3I+J][3K+L] = C_IJKL, t = 9p - p(p-1)/2 + (q - p) for
 * p <= q.  The transformed c_ijkl (45 entries per node) and 1/(rho J) are formed on the device.
 * SBP_E_JACOBIAN_NONPOSITIVE if J <= 0 at a node of these planes (Sec. 3.3). */
int sbp3_set_material(sbp3_handle* h, int i3_begin, int i3_count, const double* rho, const double* C45);

/* Leapfrog levels u^{n-1}, u^n (3 * n1*n2*n3 each, host FP64, copied).  In FP32 the handle keeps
 * the increment u^n - u^{n-1}, formed here in double precision, beside u^n.  sbp3_get_state
 * writes the two current levels (after a step: the levels before and after it) into caller
 * arrays; SBP_E_STATE before any sbp3_set_state.  Both synchronize the device. */
int sbp3_set_state(sbp3_handle* h, const double* u_prev, const double* u_cur);
int sbp3_get_state(sbp3_handle* h, double* u_prev, double* u_cur);

/* accel = (rho J)^-1 [ DD(c) u + J SAT(u) ] for the host field u (3 * n1*n2*n3, FP64, rounded to
 * the handle's precision on the device); the state is left untouched; SBP_E_STATE until the
 * material covers every x3-plane.  Synchronizes the device. */
int sbp3_apply(sbp3_handle* h, const double* u, double* accel);

/* nsteps leapfrog steps of size dt on the given CUDA stream (NULL: the default stream); the call
 * returns once the launches are queued (three kernels per step).  SBP_E_STATE without a complete
 * material or a state; SBP_E_INVALID_ARG for nsteps < 0 or dt <= 0.  The caller picks a stable dt
 * (no CFL estimate in 3-D). */
int sbp3_step(sbp3_handle* h, int nsteps, double dt, void* stream);

/* Per-family device time (CUDA events on the launch stream) of the launches made while enabled,
 * and the launch counts since create (always counted).  ms and launches hold
 * SBP3_PROF_FAMILIES entries; sbp3_profile_read synchronizes the device. */
/* Launch shape of the interior divergence kernel (x2 rows per block and the register cap that
 * follows from the minimum resident blocks): variant 0 .. SBP3_TUNING_VARIANTS-1, order 6 only
 * (other orders keep variant 0).  Every variant computes bitwise the same field.
 * sbp3_autotune times each variant on operator applications of the current level (zeros before
 * any state; the state is not changed), selects the fastest and returns it; ms_out (optional,
 * SBP3_TUNING_VARIANTS entries) receives the time of one application per variant (-1: not built
 * for this order). */
#define SBP3_TUNING_VARIANTS 4
int sbp3_set_tuning(sbp3_handle* h, int variant);
int sbp3_autotune(sbp3_handle* h, int* variant_out, double* ms_out);

int sbp3_profile(sbp3_handle* h, int enable);
int sbp3_profile_read(sbp3_handle* h, double* ms, long long* launches);

/* Node count, precision and order of the handle (any output pointer may be NULL). */
int sbp3_get_info(const sbp3_handle* h, long long* nodes_out, int* precision_out, int* order_out);

#ifdef __cplusplus
}
#endif
#endif
