/*
 * fraclap -- C ABI of the GB300 (sm_103a) solver for the fractional
 * Laplacian (-Delta)^{alpha/2} with extended (homogeneous) Dirichlet
 * conditions, after Minden & Ying, "A simple solver for the fractional
 * Laplacian in multiple dimensions" (arXiv:1802.03770).
 *
 * The discrete operator M is the paper's singularity-subtracted trapezoidal
 * rule (Sec. 2, eq. linearelliptic): on a box of n_0 x ... x n_{d-1}
 * interior points with spacing h,
 *
 *   (M u)_i = C_{alpha,d} h^d [ A_1 u_i - sum_{j != i} u_j / |y_i - y_j|^{d+alpha}
 *                               + (A_2 + A_3) L_FD u_i ],
 *
 * applied as a zero-padded FFT convolution (Sec. 3.1).  Solves use
 * conjugate gradients preconditioned with the finite-difference part
 * C h^d L of M (Sec. 3.1), applied by discrete sine transforms on the box.
 *
 * Conventions (every entry point):
 *  - Arrays are row-major with the last axis fastest, length N = prod n_i,
 *    one value per interior grid point.  Pointers named *_dev are device
 *    pointers on the plan's device; *_host are host pointers.  The caller
 *    owns every array it passes; the plan owns its tables and workspaces.
 *  - Work is enqueued on the plan's CUDA stream (fl_opts.stream; NULL =
 *    the legacy default stream).  fl_apply* and fl_precond* return without
 *    waiting; the solve and time-step calls wait for their own work (they
 *    read convergence flags back) and fill fl_solve_info before returning.
 *  - Values outside Omega (mask == 0) are ignored on input and written as 0
 *    (the extended Dirichlet condition u = 0 off Omega, eq. fracelliptic).
 *  - Nothing throws across the ABI.  Every call returns an fl_status; on an
 *    error fl_last_error_string() describes it (thread-local).
 */
#ifndef FRACLAP_H
#define FRACLAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FL_OK = 0,
  FL_INVALID_ARG = 1,     /* bad size, alpha, h, pointer or mode          */
  FL_NOT_CONVERGED = 2,   /* iteration cap hit; the iterate is written    */
  FL_BREAKDOWN = 3,       /* p^T A p <= 0 or a NaN in CG                  */
  FL_DEVICE_TIMEOUT = 4,  /* a bounded device wait gave up                */
  FL_CUDA_ERROR = 5,      /* a CUDA runtime call failed                   */
  FL_OOM = 6              /* device allocation failed                     */
} fl_status;

/* Solve modes (argument `mode` of the solve calls): precision in bits 0-3,
 * preconditioner in bits 4-7. */
enum {
  FL_MODE_F64 = 0,        /* plain FP64 CG                                 */
  FL_MODE_MIXED = 1,      /* FP32 inner CG inside FP64 iterative refinement */
  FL_MODE_LEARNED = 2,    /* as MIXED, inner flexible CG with the learned
                             preconditioner of the attached network        */
  FL_PRECOND_FD = 0x00,   /* FD-Laplacian preconditioner (Sec. 3.1, 3.2);
                             on an occluded domain the FD operator on
                             Omega itself (Sec. 4.4), see fl_precond       */
  FL_PRECOND_NONE = 0x10, /* plain CG                                      */
  FL_PRECOND_AUTO = 0x20, /* FD preconditioner for alpha >= 1, none below
                             (Sec. 4.2: for alpha < 1 no preconditioning is
                             needed)                                       */
  FL_PRECOND_SHIFTED = 0x30, /* FD preconditioner with the balanced shift of
                                fl_precond_params (not in the paper)       */
  FL_PRECOND_STENCIL = 0x40, /* the (2d+1)-point stencil part of M itself,
                                the alternative remarked on in Sec. 3.1    */
  FL_PRECOND_BOX = 0x50,     /* occluded domains: the box FD solve restricted
                                to Omega, R B^{-1} R^T (cheaper per
                                application, not the paper's choice)       */
  FL_BATCH_PERSISTENT = 0x100 /* fl_solve_elliptic_batched, FL_MODE_MIXED:
                                 all inner CG iterations of a refinement step
                                 in one persistent launch instead of one
                                 launch per pass and iteration              */
};

typedef struct fl_plan fl_plan;

typedef struct {
  double rho;        /* window radius delta / h; <= 0 selects the paper's 20 */
  void* stream;      /* cudaStream_t the plan enqueues on; NULL = default    */
  double inner_tol;  /* FL_MODE_MIXED: inner relative tolerance; <= 0: 1e-4  */
  int max_outer;     /* FL_MODE_MIXED: refinement steps; <= 0: 20            */
} fl_opts;

typedef struct {
  int iterations;        /* CG iterations (operator applications in the loop) */
  int outer_iterations;  /* FP64 refinement steps (FL_MODE_MIXED), else 0     */
  double rel_residual;   /* ||b - A u||_2 / ||b||_2 at return (FP64 estimate)  */
  int converged;         /* 1 if rel_residual <= tol                          */
  int status;            /* fl_status of the solve                            */
} fl_solve_info;

typedef struct {
  int d;
  int64_t n[3];          /* interior points per axis                       */
  int64_t fft_len[3];    /* padded FFT length L_i >= 2 n_i - 1 (power of 2, <= 8192) */
  double h, alpha, rho;
  double c_alpha_d;      /* C_{alpha,d}                                    */
  double lattice_zeta;   /* Z_d = sum_{m != 0} |m|^{-(d+alpha)}, A_1 = h^{-(d+alpha)} Z_d */
  double window_corr;    /* a = (A_2 + A_3) h^{d+alpha-2} (< 0)             */
  double kernel0;        /* M_ii                                           */
  int64_t workspace_bytes;
} fl_plan_desc;

/* Create a plan for the operator of eq. linearelliptic (Sec. 3.1).
 *   d      : 1, 2 or 3 (d = 1: the interval examples of Sec. 4.1; the line
 *            is stored as the single row of a 2D layout, so in
 *            fl_plan_set_tiles / fl_plan_autotune its strided pass is the
 *            trivial axis 0)
 *   n      : host array of d extents n_i >= 1: n_i <= 4096 for d = 1, 2
 *            (padded FFT lengths up to 8192), n_i <= 1024 for d = 3.  The FD
 *            preconditioner solves along the first axis in columns of at
 *            most 1024 values: with n_0 > 1024 (d = 2) only unpreconditioned
 *            solves are available (FL_PRECOND_NONE)
 *   h      : grid spacing > 0 (the unit box has h = 1/(n+1))
 *   alpha  : order, 0 < alpha < 2
 *   mask   : nullable host array of N bytes, nonzero = point of Omega
 *            (occluded Cartesian grids, Sec. 1.1); NULL = the full box
 *   opts   : nullable; see fl_opts
 *   out    : receives the plan
 * Computes C_{alpha,d}, A_1..A_3 (eq. int1constants, eq. a3), the kernel
 * symbol (FP64 FFT on the device) and the sine-transform tables; allocates
 * every workspace the other calls use.  Errors: FL_INVALID_ARG, FL_OOM,
 * FL_CUDA_ERROR. */
fl_status fl_plan_create(int d, const int64_t* n, double h, double alpha,
                         const uint8_t* mask, const fl_opts* opts, fl_plan** out);

/* Release a plan and its device memory (waits for its stream). */
fl_status fl_plan_destroy(fl_plan* plan);

/* Constants and sizes of a plan (host struct filled). */
fl_status fl_plan_describe(const fl_plan* plan, fl_plan_desc* desc);

/* Column tiles of the strided FFT passes (no counterpart in the paper).
 * A strided pass along axis i transforms tiles of tx consecutive lines in
 * shared memory; tx is a power of two between 16 bytes of line element
 * (2 FP32 / 1 FP64 complex values) and the widest tile a CTA holds
 * (8192 FP32 / 4096 FP64 complex values over the padded length L_i, at most
 * 64).  The tile width changes neither the arithmetic nor any result (each
 * line is transformed the same way), only the launch shape.
 *   tx[6]: FP32 axes 0..2, then FP64 axes 0..2; 0 = the widest tile.
 * fl_plan_set_tiles sets them (FL_INVALID_ARG for a width out of range or
 * not a power of two; entries of axes without a strided pass are ignored).
 * fl_plan_autotune times, for each precision and each axis with a strided
 * pass, every candidate width over a few operator applies and
 * preconditioner solves on the plan's stream (axis by axis, the others
 * kept), keeps the fastest, and writes the choice to tx_out (nullable).
 * For plans whose rows (the last axis) pad to 256 .. 2048 points it then
 * times the FP32 row passes in both CTA shapes (row shape 0: 128 threads x
 * 16 values per line, 1: 256 threads x 8, radix-8 stages) and keeps the
 * faster (fl_plan_row_shape reads the choice).
 * It uses the plan's workspaces, waits for the stream, and invalidates the
 * plan's captured CG graphs; run it before solves, not during one. */
fl_status fl_plan_set_tiles(fl_plan* plan, const int tx[6]);
fl_status fl_plan_autotune(fl_plan* plan, int tx_out[6]);

/* CTA shape of the FP32 row passes (no counterpart in the paper): 0 = 128
 * threads x 16 values per line (the default), 1 = 256 threads x 8 (rows
 * padded to 256 .. 2048 points only, else FL_INVALID_ARG).  Results agree
 * to FP32 rounding (other radix plan), not bit for bit.  Invalidates the
 * plan's captured CG graphs.  fl_plan_row_shape returns the current shape
 * (-1 for a NULL plan).  Lockstep batched solves use shape 1 when every
 * plan of the batch has it, else shape 0; the persistent launch has its own
 * CTA shape. */
fl_status fl_plan_set_row_shape(fl_plan* plan, int shape);
int fl_plan_row_shape(const fl_plan* plan);

/* y = M u (Sec. 3.1, BTTB apply by FFT), FP64 throughout.  u_dev, y_dev:
 * device arrays of N doubles; they may not alias. */
fl_status fl_apply(fl_plan* plan, const double* u_dev, double* y_dev);

/* y = M u in FP32 (FP32 FFTs and symbol). */
fl_status fl_apply_f32(fl_plan* plan, const float* u_dev, float* y_dev);

/* z = (shift I + scale C h^d L)^{-1} r on the full box (Sec. 3.1 with
 * shift = 0, scale = 1; Sec. 3.2 with shift = 1, scale = theta dt).
 * On a masked plan (occluded domain Omega) the paper's preconditioner of
 * Sec. 4.4: z = (shift I + scale C h^d L_Omega)^{-1} r with L_Omega the FD
 * Laplacian on the points of Omega and Dirichlet conditions on every point
 * outside it; r is read and z written inside Omega only (z = 0 outside).
 * The paper factorises it by sparse Cholesky; here it is applied exactly
 * through two box solves and a dense system on Gamma, the points outside
 * Omega with a grid neighbour in Omega (capacitance matrix method): the
 * first call for a (shift, scale) forms and factorises that |Gamma| x
 * |Gamma| matrix from |Gamma| FP64 box solves (plan set-up work, kept until
 * another (shift, scale) is asked for); |Gamma| <= 2048, else
 * FL_INVALID_ARG (FL_PRECOND_BOX solves do not need it).
 * Requires shift >= 0 and scale > 0 and, for d >= 2, n_0 <= 1024
 * (FL_INVALID_ARG otherwise).  r_dev, z_dev: N doubles, may not alias. */
fl_status fl_precond(fl_plan* plan, double shift, double scale, const double* r_dev,
                     double* z_dev);
fl_status fl_precond_f32(fl_plan* plan, double shift, double scale, const float* r_dev,
                         float* z_dev);

/* The preconditioner a solve uses in `mode` for the operator
 * shift I + scale M (shift = 0, scale = 1: the elliptic problem; shift = 1,
 * scale = theta dt: a time step) is z = (pshift I + pscale C h^d L)^{-1} r on
 * the box (on Omega itself on a masked plan), applied like fl_precond:
 *   FL_PRECOND_FD (and AUTO with alpha >= 1): pshift = shift, pscale = scale
 *     (Sec. 3.1; Sec. 3.2 for time steps).
 *   FL_PRECOND_BOX: as FD, but on a masked plan the box solve restricted to
 *     Omega, z = R (pshift I + pscale C h^d L_box)^{-1} R^T r.
 *   FL_PRECOND_STENCIL: shift I + scale M~, M~ = M with the entries off the
 *     (2d+1)-point stencil set to zero (Sec. 3.1 remarks on it): in terms
 *     of c = C h^-alpha, the constant Z of M's diagonal and the stencil
 *     weight a (< 0), pshift = shift + scale c (Z - 2d),
 *     pscale = scale (1 - a) / (-a).
 *   FL_PRECOND_SHIFTED: pscale = scale and pshift = x >= 0 balancing the
 *     ratio (shift + scale mu) / (x + scale lam) between the lowest and the
 *     highest sine modes v_k (k = 1 and k = n_i on every axis, restricted to
 *     Omega), mu the Rayleigh quotient v^T M v / v^T v and lam the
 *     eigenvalue of C h^d L: x = scale (A lam_hi - B lam_lo) / (B - A),
 *     A = shift + scale mu_lo, B = shift + scale mu_hi.  The two quotients
 *     are computed once per plan with FP64 applies (the first call waits
 *     for the plan's stream) and cached.
 *   FL_PRECOND_NONE (and AUTO with alpha < 1): none; *pshift = *pscale = 0.
 * The precision bits of `mode` are ignored.  Requires shift >= 0 and
 * scale > 0.  Returns FL_OK or FL_INVALID_ARG (unknown mode, NULL output). */
fl_status fl_precond_params(fl_plan* plan, int mode, double shift, double scale, double* pshift,
                            double* pscale);

/* Solve M u = f (eq. matelliptic) to ||f - M u|| <= tol ||f||.
 *   f_dev : N doubles (device)
 *   u_dev : N doubles (device); in: initial guess (ignored unless
 *           x0_nonzero), out: solution
 *   mode  : FL_MODE_* | FL_PRECOND_*
 *   maxit : cap on CG iterations (per inner solve in FL_MODE_MIXED)
 *   info  : nullable, filled on return
 * Returns FL_OK, FL_NOT_CONVERGED (u holds the last iterate), FL_BREAKDOWN,
 * FL_INVALID_ARG.  On a masked plan the FD family (FD, AUTO, STENCIL,
 * SHIFTED) is solved on Omega as fl_precond describes; FL_PRECOND_BOX takes
 * the box solve restricted to Omega instead. */
fl_status fl_solve_elliptic(fl_plan* plan, const double* f_dev, double* u_dev, int x0_nonzero,
                            double tol, int maxit, int mode, fl_solve_info* info);

/* The same solve with host arrays: copies f to the device, solves, copies
 * u back (the end-to-end call). */
fl_status fl_solve_elliptic_host(fl_plan* plan, const double* f_host, double* u_host,
                                 double tol, int maxit, int mode, fl_solve_info* info);

/* One implicit theta step of the diffusion problem (eq. timestepping with
 * theta = 1/2; theta = 1 is backward Euler):
 *   (I + theta dt M) u_next = (I - (1-theta) dt M) u_prev
 *                             + dt (theta f_next + (1-theta) f_prev),
 * preconditioned with I + theta dt C h^d L (Sec. 3.2) and warm-started
 * from u_prev (Sec. 4.5).  f_prev_dev / f_next_dev are nullable (= 0).
 * u_next_dev may equal u_prev_dev.
 * In FL_MODE_MIXED / FL_MODE_LEARNED the plan keeps M u_next from the
 * step's last FP64 residual (N doubles, allocated at the first such step)
 * with the array's address and a 64-bit hash of its contents; a following
 * step whose u_prev is that array, unchanged, starts from it instead of
 * applying M to u_prev again (one FP64 apply fewer per step, two for
 * theta < 1).  Any other u_prev (or a changed one) is applied as usual. */
fl_status fl_time_step(fl_plan* plan, double dt, double theta, const double* u_prev_dev,
                       const double* f_prev_dev, const double* f_next_dev, double* u_next_dev,
                       double tol, int maxit, int mode, fl_solve_info* info);

/* Instrumentation (no counterpart in the paper).
 * fl_launch_count: number of kernels the library has launched in this
 * process (all plans, all threads).
 * fl_profile_enable: while enabled, every kernel the plan's calls launch is
 * bracketed by CUDA events on the plan's stream (adds two event records per
 * launch); disabling discards the statistics.
 * fl_profile_read: waits for the stream, then fills up to max_stats entries
 * (per kernel name: launches and summed device time) and returns the number
 * of distinct kernels recorded (0 when profiling is off). */
typedef struct {
  char name[48];
  long long launches;
  double total_ms;
} fl_kernel_stat;

long long fl_launch_count(void);
fl_status fl_profile_enable(fl_plan* plan, int enable);
int fl_profile_read(fl_plan* plan, fl_kernel_stat* stats, int max_stats);

/* Check of the bounded grid barrier of the FL_BATCH_PERSISTENT launch (no
 * counterpart in the paper): one cooperative launch on the current device,
 * one CTA per SM, all arriving at a barrier that waits for `missing` (0 ..
 * 1024) arrivals more than the grid has.  missing = 0: FL_OK.  missing > 0:
 * the barrier never completes; every CTA gives up after its bounded wait
 * (2 s) and the call returns FL_DEVICE_TIMEOUT with the context intact.
 * Synchronous; allocates and frees a 16-byte device buffer. */
fl_status fl_check_grid_barrier(int missing);

/* y = M u in FP32, like fl_apply_f32, but its one scratch buffer (the
 * half-spectrum workspace of the FFT passes) is a fixed, library-owned
 * device array instead of the plan's workspace, and the call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  The
 * paper has no counterpart; this entry exists for callers that cannot call
 * cudaMalloc at the point where they apply the operator -- a host whose
 * device memory is owned by another runtime's allocator or pool, or a
 * service that reserves all of its device memory at start-up and may not
 * allocate while it serves requests -- and who created the plan earlier, at
 * set-up time.
 *   - Limit: the plan's spectrum must fit the array, 2^21 complex floats
 *     (16 MiB): n_0 * (L_1/2 + 1) <= 2^21 in 2D (1024 x 1024 fits),
 *     n_0 * L_1 * (L_2/2 + 1) <= 2^21 in 3D (64^3 fits).  Larger plans get
 *     FL_INVALID_ARG and nothing runs.
 *   - Set-up: fl_plan_create, with the plan's device current, loads the
 *     library's code module on that device (where it was not loaded yet),
 *     which places the 16 MiB array there, and looks up the array's device
 *     address.  The array then stays on that device until the process
 *     exits.  Create the plan before any stream capture.
 *   - The plan's device must be current when this is called
 *     (FL_INVALID_ARG otherwise).
 *   - All calls, on every plan and stream of a device, share the one array
 *     and it keeps the last call's contents: calls that overlap on the GPU
 *     race and give wrong results.  Nothing in it needs to start at zero.
 *   - Arguments, layout and errors are otherwise those of fl_apply_f32; the
 *     result equals fl_apply_f32's bit for bit (same kernels, same launch
 *     shapes). */
fl_status fl_apply_f32_static(fl_plan* plan, const float* u_dev, float* y_dev);

/* Solve count independent problems M_i u_i = f_i (each eq. matelliptic with
 * its own plan: size, h, alpha) to ||f_i - M_i u_i|| <= tol ||f_i||, all at
 * once.  With FL_MODE_MIXED every pass of the FP64 residual, of the FP32 CG
 * start-up and of a CG iteration is one launch over all problems
 * (lockstep), and the CG iterations run as a captured CUDA graph of 8
 * iterations, replayed until every problem is done, on a private stream
 * (ordered after and before the plans' streams).  With FL_BATCH_PERSISTENT
 * added to mode (batches of fewer than 2048 problems) all inner CG
 * iterations of one refinement step, of every problem, instead run in ONE
 * persistent cooperative launch (all its CTAs resident; bounded grid
 * barriers between the passes; it ends when every problem's inner CG is
 * done), captured once into a CUDA graph.  Both give the same iterates up
 * to the order of the partial sums.  FL_MODE_F64 solves the problems one
 * after another with fl_solve_elliptic.
 *   plans : host array of count distinct plans, all of the same d
 *   f_dev : host array of count device pointers (N_i doubles each)
 *   u_dev : host array of count device pointers, out: solutions (x0 = 0)
 *   infos : nullable host array of count entries
 * Mixed batches need padded lengths <= 2048 (n_i <= 1024), and masked plans
 * in them take FL_PRECOND_BOX or no preconditioner.
 * Returns FL_OK when every problem converged, FL_NOT_CONVERGED if one did
 * not (all solutions are written), FL_INVALID_ARG, FL_CUDA_ERROR, and
 * FL_DEVICE_TIMEOUT if a CTA of the persistent launch waited more than 2 s
 * at a grid barrier (the launch then ends; the solutions are not valid). */
fl_status fl_solve_elliptic_batched(fl_plan* const* plans, int count, const double* const* f_dev,
                                    double* const* u_dev, double tol, int maxit, int mode,
                                    fl_solve_info* infos);

/* --- learned preconditioner (not in the paper) ---------------------------
 * A 3-level U-Net (channels 16/32/64, 3 x 3 convolutions, BF16 weights,
 * FP32 accumulation) maps features [r / s_r, z0 / s_z, alpha] of a residual
 * r (z0 = the base preconditioner applied to r, s = root mean square) on an
 * H x W grid to a correction y; the learned preconditioner is
 * z = z0 + s_z y, used inside flexible CG.  Activations and features are
 * device float arrays [channel][y][x].
 *
 * Parameter layout (fl_net_get_params / fl_net_set_params, checkpoints): per
 * layer in the order e0a, e0b, e1a, e1b, ba, bb, d1a, d1b, d0a, d0b, head,
 * the weights W[cout][cin][k][k] then the biases b[cout], as float. */
typedef struct fl_net fl_net;

/* H, W: multiples of 64 (two 2 x 2 poolings on 16 x 16 tiles); seed of the
 * He-normal initialisation; stream: cudaStream_t (NULL = default). */
fl_status fl_net_create(int H, int W, uint64_t seed, void* stream, fl_net** out);
fl_status fl_net_destroy(fl_net* net);
long long fl_net_num_params(const fl_net* net);
/* Copy the FP32 parameters and/or the last gradients to host (nullable). */
fl_status fl_net_get_params(fl_net* net, float* params_host, float* grads_host);
/* Set the parameters from host; resets the Adam state. */
fl_status fl_net_set_params(fl_net* net, const float* params_host);
/* y_dev[H*W] = N(x_dev[3*H*W]). */
fl_status fl_net_forward(fl_net* net, const float* x_dev, float* y_dev);
/* Mean squared error over a batch (xs_dev[batch][3][H][W], ts_dev[batch][H][W])
 * and its gradient (kept in the net, see fl_net_get_params). */
fl_status fl_net_loss_grad(fl_net* net, const float* xs_dev, const float* ts_dev, int batch,
                           double* loss);
/* fl_net_loss_grad followed by one Adam step with learning rate lr. */
fl_status fl_net_train_step(fl_net* net, const float* xs_dev, const float* ts_dev, int batch,
                            float lr, double* loss);
/* Checkpoint file: header (magic, version, parameter count, Adam step),
 * FNV-1a checksum, FP32 parameters. */
fl_status fl_net_save(fl_net* net, const char* path);
fl_status fl_net_load(fl_net* net, const char* path);

/* Copy one of the network's FP32 tensors, as the last call left it, to host
 * (inspection; no counterpart in the paper).  kind 0: activations, kind 1:
 * their loss gradients (of the last sample of the last fl_net_loss_grad /
 * fl_net_train_step batch).  index 0 is the input features (3 channels),
 * index l + 1 the output of layer l in the parameter-layout order (e0a ...
 * head; index 11 = the network's output).  Layout [channel][y][x] at the
 * tensor's level: H x W for e0a, e0b, d0a, d0b and the head, H/2 x W/2 for
 * e1a, e1b, d1a, d1b, H/4 x W/4 for ba, bb.  count must equal the tensor's
 * size (FL_INVALID_ARG otherwise).  Waits for the net's stream. */
fl_status fl_net_get_tensor(fl_net* net, int kind, int index, float* host, long long count);

/* Run the 3 x 3 convolutions on the tcgen05 tensor cores (enable = 1, the
 * default: BF16 activations and weights, FP32 accumulation in TMEM) or on
 * the CUDA cores (enable = 0: FP32 activations, BF16 weights). */
fl_status fl_net_set_tensor_cores(fl_net* net, int enable);
/* Alpha gate: with bands > 0, FL_MODE_LEARNED solves of a plan of order
 * alpha use the network only when alpha lies in [lo, hi) and in an enabled
 * band (the interval split into `bands` equal bands, enabled[b] != 0; host
 * array, copied); otherwise they run the plain FP32 preconditioned CG of
 * FL_MODE_MIXED.  bands = 0 removes the gate (the network serves every
 * alpha, the default).  The gate is chosen from held-out solves where the
 * network lowers the iteration count (learned.py).  FL_INVALID_ARG for a
 * NULL net, lo >= hi, non-finite bounds, bands < 0 or > 4096, or a NULL
 * array with bands > 0. */
fl_status fl_net_set_alpha_gate(fl_net* net, double lo, double hi, int bands, const uint8_t* enabled);

/* FL_DEVICE_TIMEOUT if a bounded tensor-core wait of an earlier call gave up
 * (its outputs were zeroed), else FL_OK; waits for the net's stream. */
fl_status fl_net_check(fl_net* net);

/* One training pair of the network from a plan's solves (no counterpart in
 * the paper): given the right-hand side f, the converged solution u* and an
 * iterate x (N doubles each, device), forms on the plan's stream
 *   r = f - M x (FP64 apply),  z0 = B r (the FD-Laplacian solve of
 *   fl_precond for alpha >= 1, r / M_ii below),
 *   s_r, s_z = max(root mean square of r, z0; 1e-300),
 *   feat_dev[3 N] = [r / s_r, z0 / s_z, alpha],
 *   target_dev[N] = (u* - x - z0) / s_z      (FP32),
 * so that z = z0 + s_z N(feat) approximates M^{-1} r.  Box plans only
 * (FL_INVALID_ARG for a masked plan).  Uses the plan's FP64 work vectors:
 * not concurrently with a solve on the same plan. */
fl_status fl_net_training_pair(fl_plan* plan, const double* f_dev, const double* u_star_dev,
                               const double* x_dev, float* feat_dev, float* target_dev);

/* Attach (net != NULL) or detach a network for FL_MODE_LEARNED solves on a
 * 2D plan without mask; the network's H x W must equal n_0 x n_1.  Allocates
 * the plan's feature buffers on first attach.  The plan does not own the
 * network. */
fl_status fl_plan_attach_net(fl_plan* plan, fl_net* net);

/* Wait for all work on the plan's stream. */
fl_status fl_sync(fl_plan* plan);

/* Description of the last error on this thread ("" if none). */
const char* fl_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* FRACLAP_H */
