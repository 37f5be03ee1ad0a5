/*
 * libsbp -- C-ABI of the GB300 (sm_103a) SBP-SAT solver for the 2-D anisotropic elastic
 * wave equation on curvilinear multiblock grids (Almquist & Dunham, "Elastic wave propagation
 * in anisotropic solids using energy-stable finite differences with weakly enforced boundary
 * and interface conditions").
 *
 * The semidiscrete scheme per block is (Sec. 5, eq. semidiscrete_general; Theorem 1)
 *     rho u_J'' = J^-1 [ DD_ik(c_iJkL) u_L + J SAT_J ] + f_J
 * with c_ijkl = F_Ii J C_IjKl F_Kk (eq. transf_density_stiffness) and the Robin, displacement
 * (Sec. 5) and interface (Sec. 6) SATs.  Time stepping is the explicit leapfrog scheme
 *     u^{n+1} = 2 u^n - u^{n-1} + dt^2 (rho J)^-1 [ DD(c) u^n + J SAT(u^n, t_n) + J f(t_n) ].
 *
 * Conventions
 *  - Every call returns an int status: SBP_OK (0) or a negative SBP_E_* code.  No call aborts.
 *    Everything is validated before any device work; sbp_last_error() describes the last failure.
 *  - A block has n1 x n2 nodes; node (i1, i2) of a host array sits at index i2*n1 + i1
 *    (x1 fastest).  Faces: 0: x1=0, 1: x1=1, 2: x2=0, 3: x2=1; the tangential index along
 *    faces 0/1 is i2, along faces 2/3 it is i1.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Host arrays written out
 *    are caller-allocated.  All host values are double precision.
 *  - Device memory is owned by the handle (allocated at create / set time, freed by
 *    sbp_destroy).  Fields are stored in the handle's precision (FP64 or FP32).
 *  - Time-dependent data (boundary data, body force) is separable: value(t) =
 *    sum_k coef_k * T_k(t), T_k from sbp_set_time_basis.
 */
#ifndef SBP_H
#define SBP_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SBP_OK 0
#define SBP_E_INVALID_ARG (-1)
#define SBP_E_JACOBIAN_NONPOSITIVE (-2)      /* J <= 0 at some node (Sec. 3.3 stability requirement) */
#define SBP_E_NONCONFORMING_INTERFACE (-3)   /* interface sides differ in node count or pairing */
#define SBP_E_OOM (-4)
#define SBP_E_CUDA (-5)
#define SBP_E_TIMEOUT (-6)                   /* a bounded wait of a kernel ran out (a TMA copy into shared
                                                memory of the interior or strip kernels did not arrive);
                                                reported by the next call that checks the kernels' error
                                                word; the results of the steps since are invalid */
#define SBP_E_UNSTABLE (-7)                  /* non-finite energy */
#define SBP_E_STATE (-8)                     /* call out of order (e.g. step before material) */

/* precision */
#define SBP_FP64 0
#define SBP_FP32 1

/* spatial operator (sbp_grid_desc.stencil) */
#define SBP_STENCIL_NARROW 0     /* fully compatible narrow second derivatives D_xx^FC(c) (Sec. 4.4-4.6) */
#define SBP_STENCIL_WIDE 1       /* every term D_i c D_k (first derivatives applied twice), same SATs
                                    (the narrow/wide comparison of Sec. 7.1) */

/* face kinds */
#define SBP_BC_DISPLACEMENT 0    /* u = g, SAT of eq. dirichlet_ansatz with Z of Theorem 3 */
#define SBP_BC_ROBIN 1           /* T u + U u = g, SAT of eq. sat_traction (traction when U = 0) */
#define SBP_BC_INTERFACE 2       /* welded interface, SATs of eq. scheme_interface (V = Theta = 0) */

/* stiffness layouts of sbp_set_material and sbp_misfit_gradient */
#define SBP_C_PAIR10 0           /* 10 planes: upper triangle of the 4x4 pair matrix (any major-symmetric C) */
#define SBP_C_VOIGT6 1           /* 6 planes: Voigt C11 C12 C13 C22 C23 C33 (1 = xx, 2 = yy, 3 = xy; needs minor symmetry) */

/* fields for sbp_get_field */
#define SBP_FIELD_PREV 0         /* u^{n-1} (after a step: the previous level) */
#define SBP_FIELD_CUR 1          /* u^n (current level) */
#define SBP_FIELD_APPLY 2        /* result of the last sbp_apply */
#define SBP_FIELD_VELOCITY 3     /* v of the RK4 state (sbp_set_state_rk4 / sbp_step_rk4) */

typedef struct sbp_handle sbp_handle;

typedef struct {
    int kind;                    /* SBP_BC_* */
    int nbr_block;               /* interface: neighbour block */
    int nbr_face;                /* interface: neighbour face */
    int reversed;                /* interface: node s meets neighbour node nf-1-s (else s) */
} sbp_face_desc;

typedef struct {
    int n1, n2;                  /* nodes per direction (>= 5 / 18 / 27 for order 2 / 4 / 6) */
    const double* x1;            /* physical coordinates X_1 of the nodes (n1*n2, host) */
    const double* x2;            /* physical coordinates X_2 */
    double h1, h2;               /* reference spacing; <= 0 selects 1/(n-1) */
    sbp_face_desc faces[4];
} sbp_block_desc;

typedef struct {
    int order;                   /* interior order 2q: 2, 4 or 6 (Sec. 4) */
    int precision;               /* SBP_FP64 or SBP_FP32 */
    int nblocks;
    const sbp_block_desc* blocks;
    double beta;                 /* SAT penalty factor beta >= 1 (Sec. 5.2, 6); 0 selects 1 */
    int stencil;                 /* SBP_STENCIL_NARROW (0, the paper's scheme) or SBP_STENCIL_WIDE; the wide
                                    operator is applied in two passes (fluxes, divergence) by generic kernels;
                                    the misfit gradient, the batch and sbp_apply_noalloc take narrow handles */
} sbp_grid_desc;

/* Create a solver for a multiblock curvilinear grid.  Computes the numerical metric on the
 * device (Sec. 3.3: dX/dx by the SBP first derivative, J = det, F = inverse, face scale factor
 * J^ = |a_t|).  Errors: SBP_E_INVALID_ARG, SBP_E_NONCONFORMING_INTERFACE,
 * SBP_E_JACOBIAN_NONPOSITIVE, SBP_E_OOM, SBP_E_CUDA.  On error *out is NULL. */
int sbp_grid_create(const sbp_grid_desc* desc, sbp_handle** out);

/* Release every device and host resource of the handle (NULL is accepted). */
int sbp_destroy(sbp_handle* h);

/* Message of the last failing call on h (h may be NULL: last sbp_grid_create failure). */
const char* sbp_last_error(const sbp_handle* h);

/* Density and stiffness of one block (Sec. 3, eq. transf_density_stiffness; the stiffness
 * symmetries of Sec. 3: major symmetry always, minor symmetry not assumed).
 * rho: n1*n2 values.  C in the layout c_layout, planes of n1*n2 values:
 *   SBP_C_PAIR10: 10 planes, the upper triangle of the symmetric 4x4 pair matrix M[p][q] = C_IJKL,
 *     p = 2I+J, q = 2K+L (I,J,K,L in {0,1}), in the order (0,0) (0,1) (0,2) (0,3) (1,1) (1,2)
 *     (1,3) (2,2) (2,3) (3,3) -- any major-symmetric (Cosserat) stiffness;
 *   SBP_C_VOIGT6: 6 planes C11 C12 C13 C22 C23 C33 of the symmetric 3x3 Voigt matrix (Voigt
 *     index 1 = (1,1), 2 = (2,2), 3 = (1,2) = (2,1)) -- stiffness with minor symmetry; it is
 *     expanded to the pair layout (C_IJKL = Voigt entry of (IJ), (KL)).
 * Forms c_ijkl and 1/(rho J) on the device.  Errors: SBP_E_INVALID_ARG (bad block, layout,
 * non-positive or non-finite density). */
int sbp_set_material(sbp_handle* h, int block, const double* rho, const double* C, int c_layout);

/* Robin matrix U (Sec. 5.1) of a ROBIN face: 3 planes of nf values (U11, U12, U22), physical. */
int sbp_set_robin(sbp_handle* h, int block, int face, const double* U);

/* Dissipative Robin condition (the remark of Sec. 5.1): T u + U u + V du/dt = g on a ROBIN face, V
 * symmetric positive semidefinite: 3 planes of nf values (V11, V12, V22), physical.  The SAT of
 * eq. sat_traction gains -(JH)^-1 e_f J^ H_f V e_f^T du/dt.  Leapfrog takes the centred velocity
 * (u^{n+1} - u^{n-1}) / (2 dt), a 2 x 2 solve per face node, so the leapfrog energy decreases by
 * exactly |u^{n+1} - u^{n-1}|^2 / (4 dt) in the damping's norm each step; RK4 takes the stage
 * velocity.  sbp_apply and sbp_energy leave the term out (it needs a velocity).
 * Errors: SBP_E_INVALID_ARG (not a Robin face, V not PSD or not finite). */
int sbp_set_robin_damping(sbp_handle* h, int block, int face, const double* V);

/* Super-grid layer dissipation (Sec. 7.3: a term E du/dt that is zero outside the absorbing layers
 * and makes H E symmetric negative semidefinite inside; the stretched layer grid itself is part of
 * the block's mapping).  Reading: J E = -H^-1 sum_i Dt_i^T diag(s) Dt_i for each component, Dt_i
 * the undivided second difference along x_i at the nodes 1 .. N-2 of every grid line, s >= 0 the
 * coefficient of the node at the difference's centre (n1*n2 values, host; zero outside the
 * layers; s = eta rho J c h1 h2 / (32 h) damps the grid-scale checkerboard at the rate eta c / h).
 * Leapfrog takes the backward velocity (u^n - u^{n-1}) / dt (explicit; stable while the layer
 * damping rate times dt stays well below one), RK4 the stage velocity; only the nodes the layer
 * reaches are visited (two small kernels around each leapfrog step, one before each RK4 stage).
 * Errors: SBP_E_INVALID_ARG (negative or non-finite s). */
int sbp_set_layer_dissipation(sbp_handle* h, int block, const double* s);

/* Time basis of separable data: T_k(t) = sin(omega_k t) (kind 0) or cos(omega_k t) (kind 1);
 * nbasis <= 8. */
int sbp_set_time_basis(sbp_handle* h, int nbasis, const int* kinds, const double* omegas);

/* Boundary data of a DISPLACEMENT (g_J = prescribed displacement) or ROBIN (g_J = physical
 * traction data) face: g[(J*nbasis + k)*nf + s]. */
int sbp_set_boundary_data(sbp_handle* h, int block, int face, const double* g);

/* Body force f_J of one block (physical, per unit volume): f[(J*nbasis + k)*n1*n2 + node]. */
int sbp_set_forcing(sbp_handle* h, int block, const double* f);

/* Point force f_J = (f1, f2)_J * amplitude * W(t) * delta(X - X0) (Sec. 7.4), W the Ricker
 * wavelet with peak frequency alpha_p centred at t0.  (x1, x2) is the position in the block's
 * reference coordinates [0,1]^2.  The discrete delta uses, per direction, the Lagrange weights
 * of the 2q nodes nearest x (start = clamp(floor(x/h) - q + 1, 0, n - 2q)) divided by H. */
int sbp_add_point_source(sbp_handle* h, int block, double x1, double x2, double f1, double f2,
                         double amplitude, double alpha_p, double t0);

/* Initial state of one block: u_prev = u^{-1}, u_cur = u^0, each 2 planes (u_1, u_2) of
 * n1*n2 values (host).  t is the time of u_cur (same for all blocks; the last call wins). */
int sbp_set_state(sbp_handle* h, int block, const double* u_prev, const double* u_cur, double t);

/* State through caller-owned device buffers (borrowed: read or written by work enqueued on `stream`,
 * so they must stay alive until that work has finished; the caller, e.g. PyTorch, owns them).
 * Layout: 2 planes (u_1, u_2) of n2 rows x `pitch` elements, x1 fastest, elements in the handle's
 * precision (double for SBP_FP64, float for SBP_FP32); plane 1 starts n2*pitch elements after
 * plane 0.  The pointer must be 16-byte aligned and pitch*sizeof(element) a multiple of 16 bytes
 * with pitch >= n1; buffers must live on the handle's device.
 * sbp_set_state_device: u_prev = u^{-1}, u_cur = u^0 of one block, t the time of u_cur (as
 *   sbp_set_state, without the FP64 host round trip).
 * sbp_get_field_device: copy SBP_FIELD_PREV / CUR / APPLY / VELOCITY of one block into dst.
 * Both are stream-ordered (asynchronous).  Errors: SBP_E_INVALID_ARG (pointer, alignment, pitch,
 * device), SBP_E_CUDA. */
int sbp_set_state_device(sbp_handle* h, int block, const void* u_prev, const void* u_cur, long long pitch, double t,
                         void* stream);
int sbp_get_field_device(sbp_handle* h, int block, int which, void* dst, long long pitch, void* stream);

/* Advance all blocks by nsteps leapfrog steps of size dt, asynchronously on `stream`
 * (a cudaStream_t; NULL = default stream). */
int sbp_step(sbp_handle* h, int nsteps, double dt, void* stream);

/* Classical fourth-order Runge-Kutta time stepping (the paper's integrator, Sec. 7.1 and 7.4) of
 * the first-order form u' = v, v' = (rho J)^-1 [DD(c) u + J SAT(u, t) + J f(t)], as an alternative
 * to leapfrog.  The RK4 state of a block is (u, v) (host, 2 planes of n1*n2 values each); t the
 * time.  sbp_set_state_rk4 allocates the block's RK4 buffers (10 planes) on first use.
 * sbp_step_rk4 advances nsteps steps of size dt asynchronously on `stream`: four operator passes
 * per step, each fused with its stage combination (stage input U_{s+1} = u + c h V_s, stage
 * velocity V_{s+1} = v + c h a_s and the running sums of b_s V_s and b_s a_s are formed in the
 * same kernels that apply the operator; c = 1/2, 1/2, 1, b = 1/6, 1/3, 1/3, 1/6).  After the
 * steps, SBP_FIELD_CUR holds u and SBP_FIELD_VELOCITY holds v; the leapfrog level
 * SBP_FIELD_PREV and the operator output SBP_FIELD_APPLY (used as scratch for the point sources)
 * are then meaningless.  Errors: SBP_E_STATE without materials or RK4 state. */
int sbp_set_state_rk4(sbp_handle* h, int block, const double* u, const double* v, double t);
int sbp_step_rk4(sbp_handle* h, int nsteps, double dt, void* stream);

/* The same leapfrog steps as sbp_step, replayed from a CUDA graph: the first call (and any call
 * with a different nsteps or dt) captures nsteps launches of the step kernels into a graph,
 * later calls only update the device-side time and launch the graph on `stream`.  nsteps must
 * be even (the displacement buffers return to the same parity).  Supports point sources; a
 * handle with time-basis data (sbp_set_time_basis) is rejected with SBP_E_STATE.  Results are
 * bitwise identical to sbp_step. */
int sbp_step_graph(sbp_handle* h, int nsteps, double dt, void* stream);

/* Device bytes a handle for `desc` holds after sbp_grid_create, sbp_set_material and
 * sbp_set_state (fields, coefficients, metric, closure matrices of D_xx^FC, face buffers and
 * interface traces, tensor maps), used to admit solves by HBM footprint.  No device work. */
int sbp_grid_footprint(const sbp_grid_desc* desc, long long* bytes_out);

/* Pick the launch tuning for this grid by timing candidates on leapfrog steps from the current
 * state (the overwritten level is saved and restored: the state is left unchanged; device memory
 * for one copy of the state is allocated for the call): the FP32 interior kernel's rows per CTA (written to
 * *rows_out, 0 = the built-in heuristic; FP64 handles: 0), and whether the boundary-strip kernel
 * runs on a second stream concurrently with the interior kernel (*overlap_out, 0 or 1; the
 * default is 0).  The choice is kept by the handle.  Either pointer may be NULL. */
int sbp_autotune(sbp_handle* h, int* rows_out, int* overlap_out);

/* Set the tuning directly (e.g. a choice sbp_autotune made for another handle with the same
 * grid): rows per CTA of the FP32 interior kernel (0 = heuristic) and the strip/interior overlap
 * (0 off, 1 on, -1 unchanged). */
int sbp_set_tuning(sbp_handle* h, int rows_per_cta, int overlap);

/* Apply the spatial operator to the current level of every block (synchronous):
 * r = DD(c) u + J SAT(u) (+ J f(t) + point sources when with_data != 0, SAT data at t).
 * The result is read with sbp_get_field(..., SBP_FIELD_APPLY, ...). */
int sbp_apply(sbp_handle* h, int with_data, double t);

/* Copy a field of one block to host (2 planes of n1*n2 doubles).  Synchronous. */
int sbp_get_field(sbp_handle* h, int block, int which, double* dst);

/* Leapfrog energy E^{n+1/2} = 1/2 |u^{n+1}-u^n|^2_{rho J H}/dt^2 - 1/2 (u^{n+1})^T H A u^n
 * with u^n = PREV, u^{n+1} = CUR and A the homogeneous operator (Sec. 5-6 energies); FP64
 * reductions.  Returns SBP_E_UNSTABLE if the result is not finite. */
int sbp_energy(sbp_handle* h, double dt, double* E_out);

/* Discrete l2 distance of a field (SBP_FIELD_*) from reference arrays, with the norm of the
 * scheme: err2 = sum_blocks sum_J (u_J - ref_J)^T (J H) (u_J - ref_J) and ref2 = sum ref_J^T (J H)
 * ref_J, FP64 reductions on the device (the l2 error of Table 1 is sqrt(err2) with the exact
 * solution as reference; sqrt(err2 / ref2) is the relative l2 distance).  ref[b]: 2 planes of
 * n1*n2 doubles per block (host, x1 fastest).  Synchronous.  Either output may be NULL. */
int sbp_l2_diff(sbp_handle* h, int which, const double* const* ref, double* err2_out, double* ref2_out);

/* dt = cfl * min over nodes of min(h1,h2) / v_max, v_max the largest quasi-P speed from the
 * Christoffel equation in the reference domain (Sec. 7, eq. christoffel), maximised over
 * 720 sampled directions refined by golden-section search.  Needs all materials set. */
int sbp_suggest_dt(sbp_handle* h, double cfl, double* dt_out);

/* Kernel timing for benchmarks.  sbp_profile(h, 1) resets the counters and, until
 * sbp_profile(h, 0), makes every kernel launch record CUDA events (on the launch stream)
 * around its family: [0] interior stencil, [1] boundary strips (closures, and the SAT terms,
 * which the strip kernel forms itself), [2] interface traces (k_face_trace: each interface
 * side's displacement, traction and penalty share, read by the other side's SAT terms), [3] point sources,
 * [4] gradient interior, [5] gradient strips,
 * [6] gradient face terms, receiver recording and adjoint injection, [7] misfit reduction and
 * gradient output.  sbp_profile_read returns the accumulated milliseconds per family
 * (ms[SBP_PROF_FAMILIES], needs profiling on) and the number of kernel launches per family since
 * the last reset (launches[SBP_PROF_FAMILIES], always counted).  Either pointer may be NULL. */
#define SBP_PROF_FAMILIES 8
int sbp_profile(sbp_handle* h, int enable);
int sbp_profile_read(sbp_handle* h, double* ms, long long* launches);

/* Operator application that allocates nothing (no counterpart in the paper; a service for
 * callers that cannot allocate device memory, e.g. code confined to a fixed memory pool or a
 * real-time loop that must not call cudaMalloc).  Computes, for the grid, material, SATs and
 * data of h, r = DD(c) u + J SAT(u) (+ J f(t) + point sources when with_data != 0), exactly the
 * operator of sbp_apply, but on caller-provided device buffers:
 *   u_dev: input displacement, r_dev: output, both in the library's device layout -- for each
 *          block in order, 2 planes (component 1, component 2) of n2 rows x pitch elements,
 *          pitch = n1 rounded up to a multiple of 32, elements in the handle's precision
 *          (double for SBP_FP64, float for SBP_FP32); blocks follow each other without gaps.
 * The per-face SAT terms and the device copies of the block tables live in one
 * fixed 8 MiB file-scope device array shared by every call; grids needing more scratch are
 * rejected with SBP_E_INVALID_ARG before any device work.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, once per device).  Calls that overlap on the
 * GPU (concurrent streams, several handles) race on the shared array: serialise them.  The call
 * is stream-ordered on `stream` and returns after the stream has drained (it synchronises the
 * stream), so it cannot be called while that stream is being captured into a CUDA graph.  The
 * current device must be the one that was current at sbp_grid_create (else SBP_E_STATE).
 * No cudaMalloc/cudaFree or allocating library routine is called. */
int sbp_apply_noalloc(sbp_handle* h, const void* u_dev, void* r_dev, int with_data, double t, void* stream);

/* Synchronise the device and report any error the kernels recorded since the last check
 * (SBP_E_TIMEOUT when a bounded wait ran out; the error word is cleared by the report). */
int sbp_check(sbp_handle* h);

/* Diagnostic of the timeout path (no counterpart in the paper): enqueues, on the default stream,
 * one thread that waits with the kernels' bounded mbarrier wait on a barrier that nothing arrives
 * at, giving up after `polls` polls (1 .. 2^20); no copy is issued, so nothing is left in flight.
 * The next call that checks the error word (sbp_check, sbp_apply, sbp_get_field, sbp_energy, ...)
 * returns SBP_E_TIMEOUT and clears it.  Errors: SBP_E_INVALID_ARG for polls out of range. */
int sbp_debug_wait_probe(sbp_handle* h, int polls);

/* Current simulation time and number of resident nodes. */
int sbp_get_time(const sbp_handle* h, double* t_out);
int sbp_get_info(const sbp_handle* h, long long* nodes_out, int* precision_out, int* order_out);

/* ---- batch of resident shots: the persistent tile-queue step ---------------------------------
 * Serving layer (no counterpart in the paper): many independent forward solves ("shots") kept
 * resident on the device and advanced together.  One step of the batch is ONE launch of a
 * persistent kernel whose CTAs (as many as fit on the GPU at once) pull work items from a single
 * device queue covering every active shot -- interior tiles of the column-marching stencil (128
 * columns x `rows` rows) and boundary-strip tiles (closures, SAT terms, point sources on the
 * strips) -- so small and large shots fill the GPU together; the last CTA to finish adds the
 * point sources off the strips and advances every shot.  sbp_batch_step replays a CUDA graph of
 * K such launches.  Shots are admitted (sbp_batch_add) and retired (sbp_batch_remove) between
 * sbp_batch_step calls; each shot advances by its own step count and stops when it is reached.
 * The arithmetic per node is that of sbp_step, so a shot's result does not depend on the batch
 * it ran in.
 * Shots: single-block FP32 handles of the batch's order without interfaces or time-basis data,
 * with their material and state set.  A handle in a batch must not be stepped or modified by any
 * other call until it is removed; sbp_batch_remove hands the state (level parity, time) back to
 * the handle, after which sbp_get_field and every other call apply to it as usual. */
typedef struct sbp_batch sbp_batch;

/* Create an empty batch for `max_shots` shots (1 .. 4096) of interior order `order`, on the current
 * device.  Errors: SBP_E_INVALID_ARG, SBP_E_OOM, SBP_E_CUDA. */
int sbp_batch_create(int order, int max_shots, sbp_batch** out);
int sbp_batch_destroy(sbp_batch* b);
const char* sbp_batch_last_error(const sbp_batch* b);

/* Admit handle h for nsteps leapfrog steps of size dt from its current state; *slot_out receives
 * its slot.  Takes effect at the next sbp_batch_step.  Errors: SBP_E_INVALID_ARG (not a
 * single-block FP32 handle of the batch's order, interfaces), SBP_E_STATE (batch full, handle
 * already admitted, time-basis data, material missing). */
int sbp_batch_add(sbp_batch* b, sbp_handle* h, int nsteps, double dt, int* slot_out);

/* Enqueue ksteps batch steps on `stream` (asynchronous; a CUDA graph of ksteps persistent
 * launches, captured on the first call with this ksteps).  Admissions and removals since the last
 * call are uploaded first, stream-ordered. */
int sbp_batch_step(sbp_batch* b, int ksteps, void* stream);

/* Synchronise `stream` and write the steps each slot still has to run into remaining[max_shots]
 * (-1 for a free slot).  Returns SBP_E_TIMEOUT (and clears it) if a bounded wait of the batch
 * kernel ran out since the last poll. */
int sbp_batch_poll(sbp_batch* b, int* remaining, void* stream);

/* Retire the shot in `slot` (finished or not) and free the slot: hands its level parity and time
 * back to its handle.  A shot that the last sbp_batch_poll saw finished no longer changes, so its
 * state is taken from that poll without touching the device (later launches may already be queued
 * on `stream`); otherwise `stream` is synchronised and the state read. */
int sbp_batch_remove(sbp_batch* b, int slot, void* stream);

/* Rows of an interior work item (the tile shape; 0 = default 64).  Only while the batch is empty. */
int sbp_batch_set_rows(sbp_batch* b, int rows);

/* Pick the tile shape (rows of an interior work item: 32, 64, 128 or 256) by timing batch steps of
 * a representative shot h alone; h's levels, parity and time are restored afterwards (one copy of
 * its state is allocated for the call).  The batch must be empty; the choice is kept by the batch
 * and written to *rows_out (may be NULL). */
int sbp_batch_autotune(sbp_batch* b, sbp_handle* h, int* rows_out);

/* ---- misfit gradient (adjoint) --------------------------------------------------------------
 * Sec. 5.2 remarks that self-adjointness (Theorems 3 and 5) lets an adjoint solver reuse the
 * forward solver; these calls build that adjoint for the leapfrog scheme.
 *
 * Receivers: `rec` holds nrec triples (block, i1, i2) of node indices (host, copied); nodes must be
 * distinct.  nrec = 0 removes them.  Errors: SBP_E_INVALID_ARG (bad index, duplicate node). */
int sbp_set_receivers(sbp_handle* h, int nrec, const int* rec);

/* Advance nsteps leapfrog steps exactly as sbp_step does and record, after every step, both
 * displacement components at every receiver: traces[(n * nrec + r) * 2 + J] (host, FP64,
 * nsteps * nrec * 2 values; may be null).  Synchronous.  SBP_E_STATE without receivers. */
int sbp_record(sbp_handle* h, int nsteps, double dt, double* traces);

/* Misfit Phi = 1/2 dt sum_n sum_r sum_J (u_{n+1}[J, x_r] - observed[n, r, J])^2 over nsteps
 * leapfrog steps from the current state (the levels sbp_record would record), and its exact
 * discrete gradient with respect to the density and the stiffness of every node:
 *   grad_rho[b]: n1*n2 doubles (x1 fastest), dPhi/drho;
 *   grad_C[b]:   dPhi/dC in the layout c_layout of sbp_set_material: SBP_C_PAIR10, 10 planes of
 *                n1*n2 doubles (plane P = entry P of the upper triangle of M[2I+J][2K+L] =
 *                C_IJKL, which stands for both M[p][q] and M[q][p]); SBP_C_VOIGT6, 6 planes, the
 *                derivative with respect to each Voigt entry C11 C12 C13 C22 C23 C33 (the sum of
 *                the pair entries it sets).
 * Either array pointer (or an entry) may be null to skip that output; `observed` is host FP64
 * [nsteps][nrec][2]; *misfit receives Phi.  Method: a forward pass that stores the state every
 * `checkpoint_every` steps (0: every level, when the forward and adjoint levels of the whole run
 * fit in 60 % of the free device memory, else ceil(sqrt(nsteps))), then, segment by segment from
 * the last, a recomputation of the segment's levels (none with a single segment: the forward pass
 * keeps them) and the adjoint recursion psi_n = 2 psi_{n+1} - psi_{n+2}
 * + dt^2 W L psi_{n+1} + H^-1 W dPhi/du_{n+1} with the forward kernels (psi = H^-1 W lambda, lambda
 * the Lagrange multipliers of the step equations), accumulating
 *   dPhi/dc_p(x) += dt^2 (H psi_n)^T dL/dc_p(x) u_n,  dPhi/drho(x) -= H J psi_n . (u_{n+1} - 2u_n + u_{n-1}),
 * (the terms of a segment are accumulated in registers over its levels and added once), and
 * finally dPhi/dC from dPhi/dc through c_ijkl = J F_Ii C_IjKl F_Kk.  Device workspace: about
 * (3 nsteps / K + 2 K + 5) field levels per block plus 11 accumulator planes, allocated for the call.
 * On return the state is the one after nsteps steps (as sbp_step would leave it).  Synchronous.
 * Errors: SBP_E_STATE without receivers or when a displacement face carries boundary data (the
 * data would then depend on C); SBP_E_OOM when the workspace does not fit. */
int sbp_misfit_gradient(sbp_handle* h, int nsteps, double dt, const double* observed, int checkpoint_every,
                        double* misfit, double* const* grad_rho, double* const* grad_C, int c_layout);

#ifdef __cplusplus
}
#endif
#endif /* SBP_H */
