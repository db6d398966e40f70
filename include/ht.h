/*
 * ht.h -- C ABI of the GB300 hydrothermal finite element step.
 *
 * The library advances the one-way coupled system of the paper (Sun et al.,
 * "An HPC-Based Hydrothermal Finite Element Simulator ...", Section 2):
 *
 *   head  (Eq. 1 in hydraulic-head form, backward Euler as in Eq. 3)
 *         (S_s M + dt K_K) h^{n+1} = S_s M h^n + dt F_h
 *   heat  (Eq. 2 in energy form, backward Euler as in Eq. 4, q from Darcy's
 *         law q = -K grad h^{n+1} of Section 2)
 *         (M_cT + dt L_lambda + dt C(q) + dt D_w) T^{n+1} = M_cT T^n + dt F_T
 *
 * on a structured box of Q1 or Q2 Lagrange hexahedra with per-cell
 * coefficients, matrix-free, on one GPU.  Every entry point returns HT_OK (0)
 * or a negative HT_E* code; the message of the last failure is available from
 * ht_last_error().  Nothing aborts, traps or asserts on the device.
 *
 * Layout.  Cells c = cx + nx*(cy + ny*cz); nodes n = i + Nx*(j + Ny*k) with
 * Nx = order*nx + 1 (x fastest).  Faces: 0 x-min, 1 x-max, 2 y-min, 3 y-max,
 * 4 z-min (bottom), 5 z-max (top).  All arrays are FP64 and SI units.
 *
 * Ownership.  Inputs are copied during the call; the caller keeps its
 * buffers.  Output buffers belong to the caller.  Pointers flagged
 * "on_device" are CUDA device pointers valid on the context's device (for
 * example the data pointer of a torch CUDA tensor); otherwise host pointers.
 * A context owns all device memory it allocates and frees it in
 * ht_destroy().  Work is issued on the stream given to ht_create (or a
 * stream the library creates); calls that return data synchronise it.
 */
#ifndef HT_H
#define HT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HT_OK 0
#define HT_EINVAL (-1)      /* bad argument, size or state */
#define HT_ENOMEM (-2)      /* device or host allocation failed */
#define HT_ECUDA (-3)       /* a CUDA runtime call failed */
#define HT_ENOCONV (-4)     /* Krylov solve hit max_iter before the tolerance */
#define HT_EBREAKDOWN (-5)  /* BiCGStab breakdown that a restart did not cure */
#define HT_ETIMEOUT (-6)    /* a bounded device wait gave up (the grid barrier of the persistent
                               batched CG, ht_batch_set_persistent) */

enum { HT_HEAD = 0, HT_TEMP = 1, HT_QX = 2, HT_QY = 3, HT_QZ = 4 };
enum { HT_BC_NONE = 0, HT_BC_DIRICHLET = 1, HT_BC_FLUX = 2 };
enum { HT_FP64 = 0, HT_MIXED = 1 };
enum { HT_KRYLOV_BICGSTAB = 0, HT_KRYLOV_GMRES = 1 };
enum { HT_PREC_JACOBI = 0, HT_PREC_CHEBYSHEV = 1 };
enum { HT_APPLY_AUTO = 0, HT_APPLY_TILED = 1, HT_APPLY_TWO_PASS = 2, HT_APPLY_SINGLE_PASS = 3 };
enum { HT_GUESS_PREVIOUS = 0, HT_GUESS_EXTRAPOLATE = 1 };

typedef struct ht_ctx ht_ctx;

/* Structured box: nx*ny*nz cells of order 1 (Q1) or 2 (Q2) spanning
 * [x0, x0+Lx] x [y0, y0+Ly] x [z0, z0+Lz]. */
typedef struct {
    int nx, ny, nz, order;
    double x0, y0, z0, Lx, Ly, Lz;
} ht_mesh;

/* Vertical line heat source (energy pile) from z_bot to z_top at (x, y) with
 * strength q_l(t) = mean + amp*sin(2*pi*t/period + phase) in W/m
 * (Section 3.2-3.3 piles, as consistent line loads int q_l N_i dz). */
typedef struct {
    double x, y, z_top, z_bot, mean, amp, period, phase;
} ht_line_src;

/* Horizontal heat source over a rectangle: building heat entering the ground
 * through a footprint or basement floor (the anthropogenic heat of Section 1),
 * applied like the heat-flux boundary term of Eq. 4 (the bottom flux of
 * Section 3.3).  The rectangle [x0, x1] x [y0, y1] on the plane z is snapped
 * to cell faces: each of x0, x1, y0, y1 and z moves to the nearest face
 * x0_mesh + i*Hx (y, z alike; ties upwards), x and y edges clamped to the
 * mesh.  Flux q(t) = mean + amp*sin(2*pi*t/period + phase) in W/m^2 into the
 * domain; heat load F_T,i += q(t) int_R N_i dS over the snapped rectangle R. */
typedef struct {
    double x0, x1, y0, y1, z, mean, amp, period, phase;
} ht_box_src;

/* Vertical well screened from z_bot to z_top at (x, y): volumetric rate Q
 * (m^3/s, > 0 injects) spread uniformly over the screen length L and
 * laterally with profile s(x, y): the axis itself (sigma = 0, a line source)
 * or a normal density of standard deviation sigma (m).  Head load
 * (Q/L) int N_i s dV; injected water carries temperature T_in through the
 * implicit lumped term c_w (Q/L) int N_i s dV (T_in - T); extraction adds no
 * heat term because Eq. 2 is in advective (q . grad T) form.  The lateral
 * integrals use a 10-point Gauss rule per cell within 10 sigma. */
typedef struct {
    double x, y, z_top, z_bot, Q, T_in, sigma;
} ht_well;

/* Solver options.  tol is the relative residual ||b - A x||_2 <= tol ||b||_2
 * on each linear system (head: preconditioned CG; heat: restarted GMRES(restart)
 * with right Jacobi preconditioning (krylov HT_KRYLOV_GMRES, the default) or
 * BiCGStab (HT_KRYLOV_BICGSTAB)).
 * precision HT_MIXED runs operator applies, preconditioner and inner Krylov
 * iterations in FP32 inside an FP64 defect-correction loop whose residuals,
 * dot products and norms are FP64.  precond HT_PREC_CHEBYSHEV uses a
 * Chebyshev polynomial of degree cheb_degree in D^-1 A for the head CG.
 * z_chunks > 0 fixes the number of z chunks of the operator tiles (0: the
 * library picks it from the SM count).  apply_variant selects the operator
 * kernel: HT_APPLY_TILED (one fused owner-computes tile kernel),
 * HT_APPLY_TWO_PASS (cells into an element buffer, then a node gather),
 * HT_APPLY_SINGLE_PASS (on Q1 meshes the FP32 head CG runs one tiled kernel
 * per iteration in the single-reduction form of CG; other operators as AUTO)
 * or HT_APPLY_AUTO (single-pass head CG on Q1 in FP32, otherwise two-pass
 * in FP32 and tiled in FP64).  They change performance, not results beyond
 * rounding order.
 * inner_tol is the smallest relative residual reduction asked of one FP32
 * inner solve of the head system (the solve stops earlier when the outer
 * tolerance needs less); inner_tol_heat is the same for the heat system
 * (0: inner_tol).
 * outer_fp64 != 0 computes the outer residuals b - A x of the mixed form
 * with the operator in FP64; 0 (the default) applies it in float-float
 * arithmetic on the FP32 pipes (about 48 significant bits, relative error of
 * order 1e-14 in A x), with b, x and r kept in FP64.
 * check_every is the first host convergence check interval of the Krylov
 * loops (doubling to 64).  use_graphs != 0 (the default of ht_default_solver)
 * replays the fused Krylov iterations of the two-pass variant from a CUDA
 * graph of 8 iterations, captured on the context's stream the first time a
 * solve runs with a given set of vectors, step size and operator scalars;
 * a stream that the caller is capturing is launched to directly instead.
 * guess selects the initial guess of each step's two solves (the paper does
 * not state one; the solution is the same to the tolerance either way):
 * HT_GUESS_PREVIOUS starts from the field at t^n; HT_GUESS_EXTRAPOLATE (the
 * default) also forms the Lagrange extrapolation to t^{n+1} through the
 * fields of the last two or three completed steps (linear after two,
 * quadratic after three; the step sizes may differ) and starts from
 * whichever of the two has the smaller relative residual b - A x under the
 * FP32 operator.  The extrapolation keeps two past fields of each system
 * (4 vectors of FP64 node values, allocated on the first step that needs
 * them), also across ht_batch_step; ht_set_state, a failed step and a switch
 * to HT_GUESS_PREVIOUS forget them. */
typedef struct {
    double tol;
    int max_iter;
    int krylov;
    int restart;
    int precond;
    int cheb_degree;
    int precision;
    double inner_tol;
    int max_outer;
    int check_every;
    int use_graphs;
    int z_chunks;
    int apply_variant;
    double inner_tol_heat;
    int outer_fp64;
    int guess;
} ht_solver_opts;

/* Per-step statistics: Krylov iterations (inner iterations in mixed mode),
 * outer defect-correction passes, final true relative residuals computed in
 * FP64, simulated time after the step, and phase times in milliseconds. */
typedef struct {
    int iters_head, iters_heat;
    int outer_head, outer_heat;
    double res_head, res_heat;
    double t;
    double ms_loads, ms_head, ms_heat, ms_total;
    int status;
    int guess_head, guess_heat;          /* initial guess of the solve: 0 the field at t^n,
                                            1 the learned guess, 2 the extrapolated one */
    double guess_res_head, guess_res_heat; /* relative residual of the chosen guess (FP32
                                              operator), -1 when no gate ran */
} ht_step_stats;

/* Fill *opts with the defaults (tol 1e-10, max_iter 20000, Jacobi, FP64). */
int ht_default_solver(ht_solver_opts* opts);

/* Create a context for the mesh on CUDA device `device`.  cuda_stream is a
 * cudaStream_t (NULL: the library creates a non-blocking stream it owns).
 * Errors: HT_EINVAL (order not 1/2, non-positive sizes, more than 2e9 nodes
 * or more than INT_MAX / (3 (order+1)^3) cells), HT_ENOMEM, HT_ECUDA. */
int ht_create(ht_ctx** out, const ht_mesh* mesh, int device, void* cuda_stream);

/* Free all device memory and the context.  NULL is ignored. */
void ht_destroy(ht_ctx* ctx);

/* Message of the most recent failure on ctx (or of the last ht_create). */
const char* ht_last_error(const ht_ctx* ctx);

/* Node and cell counts of the context's mesh. */
int ht_sizes(const ht_ctx* ctx, size_t* n_nodes, size_t* n_cells);

/* Per-cell coefficients (Section 2 below Eq. 2): hydraulic conductivity
 * K [cells] (> 0, host), bulk thermal conductivity lambda and heat capacity
 * cT (per-cell host arrays, or NULL to use the uniform lambda_u / cT_u),
 * water heat capacity cw and specific storage Ss = rho_w g / B_poro.
 * Errors: HT_EINVAL for NaN / non-positive values. */
int ht_set_cells(ht_ctx* ctx, const double* K, const double* lambda, const double* cT,
                 double lambda_u, double cT_u, double cw, double Ss);

/* Boundary condition of `field` (HT_HEAD / HT_TEMP) on `face`: Dirichlet
 * value, uniform normal flux into the domain (m/s for head, W/m^2 for heat;
 * the boundary integrals of Eq. 3 / Eq. 4), or none (no-flow / insulated).
 * On edges shared by two Dirichlet faces the higher face index wins. */
int ht_set_bc(ht_ctx* ctx, int field, int face, int type, double value);

/* The same with one value per face node: Dirichlet values, or a normal flux
 * interpolated by the face's shape functions (F_i += int N_i q_h dS).  Used
 * for boundary data that vary along a face, such as the hydrostatic side
 * pressures and the monthly surface temperature of Section 3.3 (re-set
 * between steps for a time-varying record).  values[n] is a host array in
 * ascending node order: of the two axes along the face, the lower one
 * (x before y before z) runs fastest; n must equal the face's node count
 * (ht_face_nodes).  The array is copied.  ht_set_bc on the face drops the
 * per-node values.  Errors: HT_EINVAL for a wrong count, a non-finite value
 * or a type other than HT_BC_DIRICHLET / HT_BC_FLUX. */
int ht_set_bc_values(ht_ctx* ctx, int field, int face, int type, const double* values, size_t n);

/* Graded tensor-product mesh (Fig. 10b: cells refined towards the piles):
 * the cell widths along `axis` (0 x, 1 y, 2 z), widths[n] on the host with n
 * the cells along that axis; the axis then spans [origin, origin + sum of
 * the widths] (the other axes keep their widths: the mesh's uniform ones
 * until set).  Every geometric quantity is taken per cell: the element
 * matrices (the unit-cell constants scaled by the cell's volume and
 * 1/h_d per derivative), the Gauss-point gradients and Darcy velocities, and
 * the line, well, box, face and pile-surface geometry of the loads.  A graded
 * context uses the generic kernels (two-pass or tiled operator, fused or
 * unfused Krylov); the single-pass Q1 kernels, the persistent and shared-
 * launch batch modes and ht_head_apply_dot_noalloc need uniform cells.  Set
 * the spacing before stepping.  Errors: HT_EINVAL for a bad axis, a wrong
 * count or a width that is not positive. */
int ht_set_spacing(ht_ctx* ctx, int axis, const double* widths, int n);

/* Seasonal Dirichlet face (Section 3.3: the surface and sea temperatures
 * over the year): the face becomes a Dirichlet face of `field` whose value
 * at each step's t^{n+1} is mean + amp sin(2 pi t / period + phase).  On an
 * edge shared with another Dirichlet face the face of higher index wins (as
 * for static faces); pile surfaces (below) win over faces.  ht_set_bc or
 * ht_set_bc_values on the face ends the seasonal value.  Errors: HT_EINVAL
 * for a bad field or face, non-finite values or period <= 0. */
int ht_set_seasonal_face(ht_ctx* ctx, int field, int face, double mean, double amp, double period, double phase);

/* Pile surfaces held at a prescribed temperature (Section 3.3: energy piles
 * at 288.55 K +- 13 K switched every six months).  rows[n][9] (host) =
 * x, y, z_top, z_bot, radius, T_mean, T_amp, period, phase; the pile's nodes
 * are Dirichlet rows of the heat system with the square-wave value
 *   T(t) = T_mean + T_amp sign(sin(2 pi t / period + phase)),  sign(0) = +1,
 * at each step's t^{n+1}.  A pile holds the nodes whose lateral distance to
 * (x, y) is at most `radius` (tolerance 1e-9 of the largest extent) and whose
 * z lies in [z_bot, z_top]; when no node is that close, the node column
 * nearest the axis (ties to the lower y index, then the lower x index) over
 * that depth range.  A node held by several piles takes the last one's
 * value.  Nodes off the Dirichlet faces are handled by wrapping the heat
 * operator (columns removed, identity rows), so the heat solves of such a
 * context use the unfused Krylov kernels and FP64 outer residuals, and
 * ht_residual(..., emulated = 1) of the heat field is formed in FP64.
 * n = 0 removes all pile surfaces.  The array is copied.  Errors: HT_EINVAL
 * for non-finite entries, a negative radius, period <= 0 or a depth range
 * outside the mesh. */
int ht_set_pile_temperatures(ht_ctx* ctx, int n, const double* rows);

/* Number of nodes on `face` (0..5) of the mesh. */
int ht_face_nodes(const ht_ctx* ctx, int face, size_t* n);

/* Set the state h, T [nodes] and the time t.  Either pointer may be NULL to
 * keep that field.  on_device selects device vs host pointers. */
int ht_set_state(ht_ctx* ctx, const double* h, const double* T, double t, int on_device);

/* Append sources; they take effect from the next step.  Errors: HT_EINVAL
 * for a source outside the box or with z_top <= z_bot. */
int ht_add_line_sources(ht_ctx* ctx, int n, const ht_line_src* src);
int ht_add_wells(ht_ctx* ctx, int n, const ht_well* wells);

/* Append box heat sources (see ht_box_src); they take effect from the next
 * step.  The array is copied.  Errors: HT_EINVAL for a non-finite field,
 * x1 <= x0 or y1 <= y0, period <= 0, z outside [z0, z0 + Lz], or a
 * rectangle that is empty once snapped (both edges on the same face). */
int ht_add_box_sources(ht_ctx* ctx, int n, const ht_box_src* boxes);

/* Extra nodal load vector added to F of `field` at every step (NULL clears).
 * A test hook for manufactured solutions. */
int ht_set_extra_rhs(ht_ctx* ctx, int field, const double* F, int on_device);

int ht_set_solver(ht_ctx* ctx, const ht_solver_opts* opts);

/* One backward-Euler step of size dt: loads at t+dt, head solve, then heat
 * solve with the Darcy flux of the new head (Section 2 one-way coupling).
 * stats may be NULL.  Errors: HT_ENOCONV / HT_EBREAKDOWN leave the state at
 * the last iterate and report the residual in stats. */
int ht_step(ht_ctx* ctx, double dt, ht_step_stats* stats);

/* Copy a field out: HT_HEAD / HT_TEMP [nodes], HT_QX/QY/QZ Darcy flux
 * -K_c grad h at cell centres [cells].  n must equal the field size. */
int ht_get_field(ht_ctx* ctx, int field, double* dst, size_t n, int dst_on_device);

/* Simulated time of the current state. */
int ht_get_time(const ht_ctx* ctx, double* t);

/* Parity hooks.  ht_apply: y = A0 x with the constrained operator of `field`
 * for step dt (Dirichlet rows identity, Dirichlet columns removed); the heat
 * operator uses the current head as h^{n+1}.  ht_diag: its diagonal.
 * ht_rhs: the lifted right-hand side b of the next step of `field` (heat
 * uses the current head as h^{n+1} and the loads at t+dt). */
int ht_apply(ht_ctx* ctx, int field, double dt, const double* x, double* y, int on_device);
int ht_diag(ht_ctx* ctx, int field, double dt, double* d, int on_device);
int ht_rhs(ht_ctx* ctx, int field, double dt, double* b, int on_device);
/* Relative residual *rel = ||b - A0 x||_2 / ||b||_2 of the head or heat
 * operator (the heat one with q from the current head), with A0 x computed in
 * FP64 (emulated = 0) or in the float-float arithmetic of the mixed form's
 * outer residuals (emulated = 1).  x and b are [nodes], on the device when
 * on_device != 0; nothing is written back.  A parity hook for the emulated
 * outer residual (the residual definition of the stopping test of R4). */
int ht_residual(ht_ctx* ctx, int field, double dt, const double* x, const double* b, int emulated,
                int on_device, double* rel);

/* Batched steps of independent problems (same device, same element order,
 * any mesh sizes; each problem is a context set up as usual and configured
 * with precision HT_MIXED and the Jacobi preconditioner).  ht_batch_step
 * advances every problem by dt: loads, right-hand sides, FP64 defect-
 * correction residuals and heat solves run per problem, while the inner FP32
 * head CG of all problems runs as one kernel launch per phase over a work
 * list of (problem, block) items with per-problem scalars and convergence
 * flags; a chunk of CG iterations is captured once in a CUDA graph (per dt)
 * and replayed until every problem has converged.  stats may be NULL or
 * point to n entries.  The batch does not own the contexts; destroy it
 * before them.  Errors: HT_EINVAL (mixed devices or orders, wrong solver
 * options), HT_ENOMEM, HT_ECUDA, HT_ENOCONV. */
typedef struct ht_batch ht_batch;
int ht_batch_create(ht_batch** out, int n, ht_ctx* const* problems);
void ht_batch_destroy(ht_batch* batch);
int ht_batch_step(ht_batch* batch, double dt, ht_step_stats* stats);
const char* ht_batch_last_error(const ht_batch* batch);
/* Execution of ht_batch_step.  HT_BATCH_CONCURRENT (the default) steps the
 * problems concurrently: host worker threads run each problem's own step
 * (fused Krylov kernels, CUDA-graph replays) on the problem's own stream, so
 * the small problems of a batch overlap on the GPU; problems that share a
 * stream are stepped one after another.  HT_BATCH_SHARED_LAUNCHES runs the
 * inner head CG of all problems in shared launches as described above.  Both
 * give each problem the result of its own ht_step up to rounding order. */
#define HT_BATCH_CONCURRENT 0
#define HT_BATCH_SHARED_LAUNCHES 1
/* HT_BATCH_PERSISTENT (Q1 problems whose options allow the single-pass
 * kernels, HT_APPLY_AUTO or HT_APPLY_SINGLE_PASS): the set-up and the heat
 * solves run concurrently as in HT_BATCH_CONCURRENT; the head solves of all
 * problems run together, their inner FP32 CG (the single-reduction Jacobi
 * CG of the single-pass kernels) as ONE cooperative launch per outer pass.
 * The launch's CTAs take the (problem, tile, z chunk) work items of every
 * unconverged problem round-robin and meet at a grid barrier twice per
 * iteration (partial sums, then per-problem scalars); a problem drops out of
 * the work list when it converges and the launch ends when all have.  Errors
 * as above, plus HT_EINVAL from ht_batch_set_mode when a problem cannot use
 * the single-pass kernels and HT_ETIMEOUT (below). */
#define HT_BATCH_PERSISTENT 2
int ht_batch_set_mode(ht_batch* batch, int mode);
/* Options of HT_BATCH_PERSISTENT.  planes: node planes per z chunk of a work
 * item (0, the default: chosen from the batch's total work and the number of
 * co-resident CTAs).  wait_ms (0 < wait_ms <= 60000, default 2000): bound of
 * every grid-barrier wait, in milliseconds at the device's maximum SM clock
 * (counted in SM clock cycles); a wait that runs out makes every CTA of the
 * launch return, and ht_batch_step returns HT_ETIMEOUT with the problems'
 * times and fields unchanged (the step can be repeated).  drop_cta: -1 (the
 * default) for normal operation; k >= 0 is a failure injection for tests:
 * CTA k of the first launch of each step leaves at its first barrier without
 * arriving, so that the other CTAs' waits run out.  Errors: HT_EINVAL. */
int ht_batch_set_persistent(ht_batch* batch, int planes, double wait_ms, int drop_cta);
/* The work list of the last persistent step: node planes per z chunk, work
 * items, CTAs of the cooperative launch, and the CTA whose barrier wait ran
 * out (-1 when none did).  Any pointer may be NULL. */
int ht_batch_persistent_info(const ht_batch* batch, int* planes, int* items, int* grid, int* err_cta);

/* Learned warm start: a 3D U-Net of four levels (widths 16, 32, 48, 64) with
 * hand-written forward, backward and Adam kernels.  The paper has no learned
 * component; the network predicts step increments that serve as Krylov
 * initial guesses (ht_set_learned_guess).
 *   level 1: L0 cin -> 16, L1 16 -> 16 (e1); level 2 (pool e1): L2 16 -> 32,
 *   L3 32 -> 32 (e2); level 3: L4 32 -> 48, L5 48 -> 48 (e3); level 4: L6
 *   48 -> 64, L7 64 -> 64; up: L8 [up L7, e3] 112 -> 48, L9 48 -> 48, L10
 *   [up L9, e2] 80 -> 32, L11 32 -> 32, L12 [up L11, e1] 48 -> 16, L13
 *   16 -> 16; L14 16 -> cout (1x1).  3x3x3 convolutions with zero padding
 *   and ReLU, 2x2x2 average pooling, nearest upsampling.
 * The 3x3x3 convolutions, their data gradients and their weight gradients
 * run on the tensor cores (BF16 operands, FP32 accumulation).  Weights, the
 * input, stored activations and the gradient signals entering a
 * convolution's backward pass are BF16; biases, the output, the loss and its
 * gradient FP32; FP32 master weights for Adam.
 * Tensors are device FP32 arrays [channel][D][H][W] (W fastest) with D, H, W
 * multiples of 8 (at least 8).  Parameters (host FP32, ht_unet_num_params
 * values): per layer in the order above the weights [taps][cout][cin] (tap
 * 9 (dz+1) + 3 (dy+1) + (dx+1)) then the biases [cout].  1 <= cin <= 16,
 * cout must be 2. */
typedef struct ht_unet ht_unet;
int ht_unet_create(ht_unet** out, int cin, int cout, int device, void* cuda_stream);
void ht_unet_destroy(ht_unet* net);
int ht_unet_num_params(const ht_unet* net);
const char* ht_unet_last_error(const ht_unet* net);
int ht_unet_set_params(ht_unet* net, const float* theta);
int ht_unet_get_params(ht_unet* net, float* theta);
int ht_unet_forward(ht_unet* net, const float* x, int D, int H, int W, float* y);
/* Mean squared error against target and its gradient (host, optional). */
int ht_unet_loss_grad(ht_unet* net, const float* x, const float* target, int D, int H, int W,
                      double* loss, float* grad);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the mean squared error. */
int ht_unet_train_step(ht_unet* net, const float* x, const float* target, int D, int H, int W,
                       float lr, double* loss);

/* Attach a trained U-Net (cin 8, cout 2) as the source of Krylov initial
 * guesses (NULL detaches).  Once two step increments are known, every step
 * builds the features [dT1, dT2, dh1, dh2, F_T, q_x, q_y, q_z]: the last two
 * increments of T and h divided by s_T and s_h (the RMS of the last ones),
 * the heat loads of the step and the nodal Darcy velocity -K grad h^n, each
 * divided by its RMS; the network predicts the next increments
 * (dT / s_T, dh / s_h), and for each field the Krylov solve starts from
 * x^n + s * prediction if its residual (FP32 operator, FP64 right-hand side)
 * is smaller than that of the guess chosen without it (x^n, or the
 * extrapolated field under HT_GUESS_EXTRAPOLATE) (the gate; the solver still
 * converges to the same tolerance).  With record != 0 the features and targets of every step
 * are kept for ht_learned_sample, also without a network.  Grid sizes are
 * the node counts rounded up to multiples of 8. */
int ht_set_learned_guess(ht_ctx* ctx, ht_unet* net, int record);
/* Copy the last step's features [8][D][H][W] and targets [2][D][H][W]
 * (device FP32 buffers of the caller) and report D, H, W; HT_EINVAL when no
 * complete sample exists yet. */
int ht_learned_sample(ht_ctx* ctx, float* features, float* targets, int* dims);

/* Launch accounting and operator timing.  ht_profile(ctx, on) resets the
 * counters; with on != 0 every operator-apply launch is bracketed by CUDA
 * events on the context's stream.  ht_profile_read() synchronises the stream
 * and returns: all kernels launched by the library since the reset, the
 * number of head / heat apply launches that did work (launches that found
 * the solve already converged and returned at once are excluded by duration)
 * and their summed device time in milliseconds.  The fused Krylov
 * iterations of the two-pass variant (both element and node passes of one CG
 * iteration of the head system; all five launches of one BiCGStab iteration
 * of the heat system) are counted and timed as units of their own and not as
 * applies. */
typedef struct {
    long long launches;
    long long head_applies, heat_applies;
    double head_apply_ms, heat_apply_ms;
    long long head_applies_fp32, heat_applies_fp32;
    double head_apply_ms_fp32, heat_apply_ms_fp32;
    long long cg_iters, bicgstab_iters;
    double cg_iter_ms, bicgstab_iter_ms;
} ht_profile_stats;
int ht_profile(ht_ctx* ctx, int on);
int ht_profile_read(ht_ctx* ctx, ht_profile_stats* out);

/* Allocation-free variant of the head-operator apply, for callers that
 * cannot allocate device memory: a host application that has already handed
 * all device memory to its own pool allocator and forbids other
 * allocations, or a latency-critical stepping loop that must not call
 * cudaMalloc because it can synchronise the device and stall.  Such a caller
 * cannot create a context (ht_create allocates), so this entry point needs
 * none.  The paper has no counterpart; it is an addition of this library.
 *
 * Computes y = A0 x for the constrained head operator S_s M + dt K_K of a
 * structured mesh and *xAx = x^T y.  K [cells], x and y [nodes] and xAx [1]
 * are device pointers owned by the caller on `device`; dirichlet_faces is a
 * bit mask of the faces (bit f = face f) whose nodes are Dirichlet rows.
 * Work is queued on cuda_stream (NULL: the legacy default stream); the call
 * does not synchronise it.  On error a message is written into msg (msg_len
 * bytes; msg may be NULL).
 *
 * Scratch: the per-tile partial sums of x^T y live in one static device
 * array of 4096 doubles (32 KiB) that every GPU loading this library keeps
 * until the process exits.  Meshes needing more than 4096 operator tiles are
 * rejected with HT_EINVAL, and so are meshes of more than INT_MAX nodes or
 * cells.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  The kept address does not survive
 * cudaDeviceReset (or any other teardown of the device's primary context),
 * so do not call this entry point after one.  The call makes `device`
 * current while it queues work and restores the caller's current device
 * before it returns, on success and on error.  All calls on a device share the array; every slot a call
 * reads is written earlier by the same call, so nothing needs clearing, but
 * calls whose kernels can run at the same time on one GPU (for example on
 * two streams) race on it and must be serialised by the caller.  The
 * function allocates no device or host memory. */
int ht_head_apply_dot_noalloc(const ht_mesh* mesh, int dirichlet_faces, double Ss, double dt,
                              const double* K, const double* x, double* y, double* xAx,
                              int device, void* cuda_stream, char* msg, size_t msg_len);

/* Measured arithmetic peak of `device` in TFLOP/s: fused multiply-add
 * chains in every thread of a full grid (FP64 if fp64, else FP32), best of
 * five timed launches.  The paper has no counterpart; it is the denominator
 * of the roofline of the operator kernels bound by arithmetic (FP64 runs at
 * a small fraction of the FP32 rate on GB300).  Allocates and frees one
 * word of device memory; runs on the legacy default stream and restores the
 * caller's current device.  Errors: HT_EINVAL (null tflops), HT_ECUDA. */
int ht_fma_peak(int device, int fp64, double* tflops);

/* Bulk coefficients from the mixture rules of Section 2 and the storage of
 * Eq. 1: lambda = (1-phi) lambda_s + phi lambda_w, cT = (1-phi) c_s +
 * phi c_w, Ss = rho_w g / B_poro. */
int ht_mixture(double phi, double lambda_s, double lambda_w, double c_s, double c_w,
               double* lambda, double* cT);
double ht_specific_storage(double B_poro, double rho_w, double g);

#ifdef __cplusplus
}
#endif

#endif /* HT_H */
