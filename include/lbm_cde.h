/*
 * lbm_cde.h - C ABI of the GB300 (sm_103a) modified-MRT lattice Boltzmann
 * solver for the convection-diffusion equation
 *
 *     d_t phi + div(phi u) = div(D grad phi)                          (Eq. 1)
 *
 * of Huang & Wu, "A modified multiple-relaxation-time lattice Boltzmann model
 * for convection-diffusion equation" (arXiv:1404.2363).
 *
 * One time step (lbm_cde_step) is one fused CUDA kernel per cell:
 *   pull-stream f_i(x) <- f'_i(x - e_i)                  (Eq. 5, pull form)
 *   wall rules at the boundary nodes                      (Sec. 3.2; see bc_*)
 *   m = M f                                              (Eq. 11, 12 / A.2)
 *   m' = m - S (m - m^eq(phi, u))  with the modified S   (Eq. 13, 30-31 / A.5)
 *   f' = M^-1 m'                                         (Eq. 14)
 * with m^eq of Eq. 15-16 (D2Q9) or Eq. A.3-A.4 (D3Q15).
 *
 * Conventions common to every entry point
 *   - Lattice units: dx = dt = c = 1.
 *   - Cell index c = x + nx * (y + ny * z); every axis is periodic unless its
 *     two faces carry walls (bc_lo_y / bc_hi_y, bc_lo_x / bc_hi_x, bc_lo_z /
 *     bc_hi_z).
 *   - "dev" pointers are CUDA device pointers on the current device; "host"
 *     pointers are ordinary host memory (pinned memory is faster).
 *   - Per-cell arrays of vectors are SoA: u[a * ncell + c], a = 0 .. dim-1.
 *   - Every call is asynchronous on desc.stream unless documented as
 *     synchronising; the caller keeps borrowed pointers valid until the work
 *     that reads them has finished.
 *   - No entry point throws, aborts or exits. Errors come back as lbm_status;
 *     lbm_cde_last_error() gives a message. Faults detected on the device are
 *     latched in a device status word and reported by the next synchronising
 *     call (lbm_cde_sum_phi, lbm_cde_sync, lbm_cde_run_host).
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef LBM_CDE_H
#define LBM_CDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_cde_s* lbm_cde_t;

typedef enum {
    LBM_OK = 0,
    LBM_E_ARG = 1,         /* invalid argument (null pointer, bad size, bad enum) */
    LBM_E_NOT_SPD = 2,     /* D not symmetric positive definite (Eq. 1)           */
    LBM_E_STATE = 3,       /* call out of order (e.g. step before set_phi)         */
    LBM_E_OOM = 4,         /* allocation failed                                    */
    LBM_E_CUDA = 5,        /* a CUDA runtime call failed                           */
    LBM_E_NONFINITE = 6,   /* phi became NaN/Inf (instability, tau -> 1/2, large u) */
    LBM_E_TIMEOUT = 7,     /* a bounded device wait gave up                        */
    LBM_E_UNSUPPORTED = 8  /* valid but not implemented combination                */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q15 = 15 };

/* Wall kinds of the grid faces. The y faces take any kind; the x faces (and the
 * z faces of D3Q15) take PERIODIC, NOFLUX_NODE or BOUNCEBACK. Where two wall
 * faces meet, a population whose source lies beyond a bounce-back face returns
 * reversed, and one whose source lies beyond Neumann faces copies the
 * population reflected in the axes of those faces. */
enum {
    LBM_BC_PERIODIC = 0,    /* both faces of the axis must then be periodic         */
    LBM_BC_NOFLUX_NODE = 1, /* wall on the boundary node, Neumann d phi/dy = 0 by the
                               mirror rule of Sec. 3.2: at y = 0 f2=f4, f5=f8,
                               f6=f7; at y = ny-1 f4=f2, f7=f6, f8=f5 (D3Q15: every
                               population entering from beyond the wall copies its
                               mirror image in y)                                   */
    LBM_BC_BOUNCEBACK = 2,  /* halfway bounce-back: a population leaving through the
                               wall returns to its node reversed (conserves sum phi) */
    LBM_BC_DIRICHLET = 3    /* wall on the node, phi = phi_w: every population
                               entering from beyond the wall is f^eq_i(phi*, u) with
                               phi* chosen so that sum_i f_i = phi_w (not in the
                               paper)                                               */
};

/* Storage form of the distributions between steps. Collision arithmetic is
 * FP32 in every form. */
enum {
    LBM_STORE_F32 = 0,      /* f'_i in FP32                                          */
    LBM_STORE_F16_NEQ = 1,  /* g_i = f'_i - f^eq_i(phi, u) in FP16, phi in FP32; g is
                               stored times 2^11 (exact), so |g| must stay below 32
                               (phi up to about 100); BF16 has FP32's range            */
    LBM_STORE_BF16_NEQ = 2  /* g_i in BF16, phi in FP32                              */
};

/* Collision models (Sec. 3): MRT-A is the modified model (Eq. 30-31 with the
 * equilibrium of Eq. 15 / 37); the MRT-B models use the unmodified S of Eq. 24
 * with the equilibria of Eq. 38 (B1), Eq. 39 (B2) or Eq. 37 (B3). The MRT-B
 * models exist for D2Q9; B1 and B2 need FP32 storage. */
enum { LBM_MRT_A = 0, LBM_MRT_B1 = 1, LBM_MRT_B2 = 2, LBM_MRT_B3 = 3 };

/* Velocity representations (lbm_cde_set_velocity). */
enum {
    LBM_U_NONE = 0,         /* u = 0                                                 */
    LBM_U_FIELD = 1,        /* u(x, t) = a(x) * s(t), a: [dim][ncell]                */
    LBM_U_ROW_PROFILE = 2   /* u(x, t) = a(y) * s(t), a: [dim][ny]                   */
};

typedef struct {
    int32_t lattice;         /* LBM_D2Q9 or LBM_D3Q15                                */
    int32_t storage;         /* LBM_STORE_*                                          */
    int64_t nx, ny, nz;      /* nz = 1 for D2Q9; nx >= 2, ny >= 3 (walls) or >= 1    */
    int32_t bc_lo_y;         /* LBM_BC_* on the y = 0 face                           */
    int32_t bc_hi_y;         /* LBM_BC_* on the y = ny-1 face                        */
    double phi_w_lo_y;       /* Dirichlet value on y = 0                             */
    double phi_w_hi_y;       /* Dirichlet value on y = ny-1                          */
    double alpha1, alpha2;   /* free equilibrium parameters (Eq. 15b-c / A.3b-c);
                                NaN selects the defaults: D2Q9 -8, 8 (Eq. 37);
                                D3Q15 -6/5, 192 (A.6 factor 1/3)                     */
    double s[15];            /* diagonal relaxation rates s_0 .. s_{q-1}; NaN selects
                                the defaults s1 = s2 = 1.1, s7.. = 1.2, s4 = s6 (= s8)
                                = 1 (Sec. 3.1). Entries of the flux rows (3, 5, 7)
                                are ignored: they come from lbm_cde_set_D.           */
    int32_t tie_q_rates;     /* 1: s4 = sxx, s6 = syy (, s8 = szz) as in Sec. 3.1    */
    /* Optional device allocator (e.g. the caller's caching allocator). When alloc
       is NULL the library calls cudaMalloc / cudaFree. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free_)(void* ptr, void* ctx);
    void* alloc_ctx;
    void* stream;            /* cudaStream_t for every launch (NULL: legacy stream)  */
    int32_t model;           /* LBM_MRT_A (default) / LBM_MRT_B1 / B2 / B3; for the B
                                models alpha1, alpha2 are fixed by their equilibria  */
    int32_t bc_lo_x;         /* LBM_BC_PERIODIC / NOFLUX_NODE / BOUNCEBACK on x = 0;
                                walls need nx >= 3                                   */
    int32_t bc_hi_x;         /* the same on x = nx-1                                 */
    int32_t bc_lo_z;         /* the same on z = 0 (D3Q15; walls need nz >= 3)        */
    int32_t bc_hi_z;         /* the same on z = nz-1                                 */
} lbm_cde_desc;

/* Fills *d with defaults for a periodic grid (F32 storage, default alpha and
 * rates, tie_q_rates = 1, no allocator, NULL stream). */
lbm_status lbm_cde_desc_init(lbm_cde_desc* d, int32_t lattice, int64_t nx, int64_t ny, int64_t nz);

/* Creates a solver. Allocates two state buffers (ping-pong) plus small scratch
 * through desc->alloc. The handle owns that memory until lbm_cde_destroy.
 * Errors: LBM_E_ARG (bad desc), LBM_E_OOM, LBM_E_CUDA. */
lbm_status lbm_cde_create(const lbm_cde_desc* desc, lbm_cde_t* out);

/* Synchronises the stream, frees everything the handle owns. NULL is a no-op. */
lbm_status lbm_cde_destroy(lbm_cde_t h);

/* Sets the diffusion tensor. D is dim x dim, row-major, host memory, lattice
 * units. The relaxation block is A = (D / k + I / 2)^-1 with
 * k = 2/3 + alpha1/8 + alpha2/12 (Eq. 36, MRT-A), 2/3 + alpha1/24 (Eq. 29, the
 * MRT-B models) or 2/3 + 55 alpha1/54 + alpha2/216 (Eq. A.6); A enters S through
 * Eq. 30-31 / 24 / A.5.
 * Errors: LBM_E_ARG (NULL), LBM_E_NOT_SPD (D not symmetric to 1e-12 relative or
 * not positive definite, or k <= 0). */
lbm_status lbm_cde_set_D(lbm_cde_t h, const double* D);

/* Reads back the relaxation block A (dim x dim, host) and the 15 diagonal rates
 * in use (host, may be NULL). */
lbm_status lbm_cde_get_rates(lbm_cde_t h, double* A_out, double* s_out);

/* Sets the velocity u(x, t) = a(x) * s(t) used by the collision at step t
 * (t = 0 for the initial equilibrium).
 *   kind     : LBM_U_NONE / LBM_U_FIELD / LBM_U_ROW_PROFILE
 *   a_dev    : device FP32, [dim][ncell] (FIELD) or [dim][ny] (ROW_PROFILE);
 *              borrowed until the next set_velocity or destroy
 *   sched_dev: device FP32 [sched_len][dim] per-component multipliers s(t),
 *              indexed by t mod sched_len (1 <= sched_len <= 2^26); NULL
 *              means s = 1; borrowed like a_dev
 * Errors: LBM_E_ARG. */
lbm_status lbm_cde_set_velocity(lbm_cde_t h, int32_t kind, const float* a_dev,
                                const float* sched_dev, int64_t sched_len);

/* Initialises f = f^eq(phi, u(x, 0)) from a device FP32 field phi_dev [ncell]
 * and resets the step counter to 0. */
lbm_status lbm_cde_set_phi(lbm_cde_t h, const float* phi_dev);

/* Advances nsteps time steps (asynchronous; one kernel launch per step). */
lbm_status lbm_cde_step(lbm_cde_t h, int64_t nsteps);

/* Sets the launch shape of the step kernel: block threads per CTA along x
 * (a multiple of 32 in [32, 256]) and vec cells per thread (1 or 2); for the
 * 16-bit storage forms of both lattices, 5 selects the node-pair kernel
 * (two adjacent nodes per thread in paired FP32 arithmetic), which needs nx
 * even, (q + 3) ncell < 2^31 and an 8-byte aligned velocity field; for D2Q9
 * with any storage, 6 selects the node-quad kernel: four nodes per thread,
 * 128-bit (FP32) or 64-bit (16-bit) vector loads and stores, which needs
 * nx % 4 == 0, 12 ncell < 2^31 and a 16-byte aligned velocity field; for
 * D2Q9 16-bit storage, vec 7 or 8 with block 128 selects the TMA-staged
 * kernel: source rows arrive in a shared-memory ring through tensor copies,
 * CTAs walking row ranges of 256-column strips (vec 7: two rows per
 * iteration, 256 threads, six stages; vec 8: one row, 128 threads, four
 * stages); needs nx % 256 == 0, 12 ncell < 2^31 and a 16-byte aligned
 * velocity field. For D3Q15 16-bit storage, vec 9 with block 256 or 128
 * selects the z-walk kernel: CTAs own 64 x (block / 32) tiles of the (x, y)
 * plane and walk a range of z planes, with phi and the velocity factors of the
 * planes z - 1 .. z + 1 and the offsets each step pulls staged in shared
 * memory by asynchronous copies; needs nx % 64 == 0, ny a multiple of
 * block / 32, 18 ncell < 2^31 and 16-byte aligned offsets, phi and velocity
 * fields. A shape
 * whose field does not meet these runs the one-node kernel, and so does every
 * shape when the x or z faces carry walls.
 * Results do not depend on the shape beyond FP32 rounding order. Errors:
 * LBM_E_ARG. */
lbm_status lbm_cde_set_launch(lbm_cde_t h, int32_t block, int32_t vec);

/* Bound on each device-side wait of the TMA-staged D2Q9 kernel (launch vec 7 / 8), in SM
 * clock cycles (default 4e9, about 2 s; 0 gives up at once). A wait that runs
 * out latches LBM_E_TIMEOUT, the kernel stops computing, waits (bounded) for
 * its copies in flight and returns; lbm_cde_sum_phi / lbm_cde_sync report the
 * status and clear it, and the handle stays usable. Errors: LBM_E_ARG
 * (cycles < 0). */
lbm_status lbm_cde_set_wait_limit(lbm_cde_t h, int64_t cycles);

/* Planes each CTA of the D3Q15 z-walk kernel (launch vec 9) walks: 0 (the
 * default) lets the launcher choose the z ranges so that the resident CTAs
 * fill whole waves; planes > 0 splits nz into ceil(nz / planes) ranges of
 * nearly equal length. Results do not depend on it. Errors: LBM_E_ARG
 * (planes < 0). */
lbm_status lbm_cde_set_zwalk(lbm_cde_t h, int32_t planes);

/* Autotuner: times every launch shape (block 64/128/256 x vec 1/2, the node-quad
 * kernel for D2Q9, the node-pair and TMA-staged kernels for D2Q9 16-bit
 * storage, the node-pair kernel at 64 .. 256 threads and the z-walk kernel
 * for D3Q15 16-bit storage) over `steps` steps from the
 * current state, keeps the fastest, and restores the state and step count.
 * With LBMCDE_TUNE_CACHE set, the choice is read from / appended to that text
 * file (lines "key block vec"; the key holds lattice, storage, grid, velocity
 * kind, walls and GPU name). Needs set_phi first; synchronising. */
lbm_status lbm_cde_autotune(lbm_cde_t h, int64_t steps, int32_t* block_out, int32_t* vec_out);

/* Number of steps taken since the last set_phi / set_state. */
lbm_status lbm_cde_get_time(lbm_cde_t h, int64_t* t_out);

/* Writes phi = sum_i f_i (Eq. 8) of the current state into phi_dev [ncell]
 * (device FP32, caller-owned). Asynchronous. */
lbm_status lbm_cde_get_phi(lbm_cde_t h, float* phi_dev);

/* Deterministic FP64 sum of phi over all cells (fixed two-pass order).
 * Synchronises the stream; returns LBM_E_NONFINITE if the sum is not finite and
 * any latched device status. */
lbm_status lbm_cde_sum_phi(lbm_cde_t h, double* out_host);

/* Synchronises the stream and returns the latched device status. */
lbm_status lbm_cde_sync(lbm_cde_t h);

/* Size in bytes of the raw state (for checkpoints). */
lbm_status lbm_cde_state_bytes(lbm_cde_t h, size_t* bytes_out);

/* Copies the raw state to / from a caller buffer (device or host memory,
 * cudaMemcpyDefault) together with the step counter. Resuming from a saved
 * state reproduces the uninterrupted run bit for bit. */
lbm_status lbm_cde_get_state(lbm_cde_t h, void* dst, int64_t* t_out);
lbm_status lbm_cde_set_state(lbm_cde_t h, const void* src, int64_t t);

/* End-to-end convenience call with host buffers: copies phi0_host [ncell] to
 * the device, initialises, runs nsteps, and copies phi back to phi_out_host
 * [ncell]. Synchronising. */
lbm_status lbm_cde_run_host(lbm_cde_t h, const float* phi0_host, int64_t nsteps, float* phi_out_host);

/* ---- Differentiation (reverse-time adjoint) --------------------------------
 * Not in the paper: for a fixed velocity one step is linear in f (Eq. 11-15),
 * B_k = C_k P B_{k-1} with B the stored post-collision state, P the pull-stream
 * with walls (Eq. 5, Sec. 3.2) and C_k = M^-1 [I - S (I - m^eq(1, u(k)) e_0^T)] M
 * the collision (Eq. 13, 30-31 / A.5). The adjoint mu_k = dL/dB_k obeys
 * mu_{k-1} = P^T C_k^T mu_k. Supported: FP32 storage, every model (MRT-A and
 * the MRT-B1/B2/B3 of Eq. 37-39, whose u^2 equilibrium terms enter dL/du),
 * periodic / NOFLUX_NODE / BOUNCEBACK walls on any face and DIRICHLET walls on
 * the y faces, where the step is affine and its linear part is transposed
 * (velocity gradients are not formed with DIRICHLET walls); LBM_E_UNSUPPORTED
 * otherwise. */

/* Number of gradient accumulators of one reverse step: 2 dim^2 + q
 * (G_A[dim][dim], G_AC[dim][dim], G_diag[q]; see lbm_cde_grad_rates). */
int32_t lbm_cde_adjoint_ngrad(int32_t lattice);

/* One reverse step k >= 1 (the forward step that collided with u(k)):
 *   mu_k_dev    : dL/dB_k, device FP32 [q][ncell]
 *   mu_prev_dev : receives dL/dB_{k-1} (must not alias mu_k_dev)
 *   f_prev_dev  : the forward state B_{k-1}, device FP32 [q][ncell]
 *   grad_acc_dev: device FP32 [2 x lbm_cde_adjoint_ngrad], 8-byte aligned,
 *                 caller-owned, zeroed by the caller before the first step:
 *                 compensated sums, accumulator j = grad_acc_dev[2j] +
 *                 grad_acc_dev[2j + 1] (add them in FP64 on the host before
 *                 lbm_cde_grad_rates; the GPU does no FP64 arithmetic); the partials
 *                 G_A[a][b] += -sum (M^-T mu)_{j_a} (m - m^eq)_{j_b},
 *                 G_AC[a][b] += -sum (M^-T mu)_{j_a} (m - m^eq)_{q_b},
 *                 G_diag[r] += -sum (M^-T mu)_r (m - m^eq)_r are added
 *                 (j_a = 3 + 2a flux rows, q_b = 4 + 2b energy-flux rows)
 *   dL_da_dev   : NULL or device FP32 [dim][ncell]; += s(k) dL/du(x, k) for a
 *                 LBM_U_FIELD velocity u = a(x) s(t)
 * Asynchronous. Errors: LBM_E_ARG, LBM_E_UNSUPPORTED, LBM_E_STATE, LBM_E_OOM. */
lbm_status lbm_cde_adjoint_step(lbm_cde_t h, int64_t k, const float* mu_k_dev, float* mu_prev_dev,
                                const float* f_prev_dev, float* grad_acc_dev, float* dL_da_dev);

/* Converts accumulated partials g (host, lbm_cde_adjoint_ngrad doubles) into
 * dL/dD (host, dim x dim, every entry an independent variable; includes the
 * tied rates s4 = sxx ... when tie_q_rates = 1) through A = (D/k + I/2)^-1, and
 * dL/ds (host [15], the diagonal rates as independent variables). For the
 * MRT-B models S has no coupling entries (Eq. 24) and G_AC is not used. Either
 * output may be NULL. */
lbm_status lbm_cde_grad_rates(lbm_cde_t h, const double* g, double* dL_dD_host, double* dL_ds_host);

/* Forward run for differentiation: f(0) = f^eq(phi0, u(0)), nsteps steps, keeping
 * the state every `every` steps (0: ceil(sqrt(nsteps))) in handle-owned device
 * memory (ceil(nsteps/every) + every - 1 states), then phi(nsteps) into phiN_dev
 * (device FP32 [ncell], may be NULL). The handle's state afterwards is the one
 * of step nsteps. */
lbm_status lbm_cde_forward_ckpt(lbm_cde_t h, const float* phi0_dev, int64_t nsteps, int64_t every,
                                float* phiN_dev);

/* Reverse sweep of the last lbm_cde_forward_ckpt: recomputes each checkpoint
 * segment, runs the adjoint steps and the initial-state term. Given
 * dL/dphi(nsteps) (device FP32 [ncell]) it writes dL/dphi0 (device FP32
 * [ncell]), dL/dD and dL/ds (host, see lbm_cde_grad_rates; may be NULL) and,
 * if dL_da_dev is not NULL, overwrites it with dL/da (device FP32 [dim][ncell],
 * LBM_U_FIELD velocity only). Synchronising. */
lbm_status lbm_cde_backward(lbm_cde_t h, const float* dL_dphiN_dev, float* dL_dphi0_dev, double* dL_dD_host,
                            double* dL_ds_host, float* dL_da_dev);

/* Per-phase device timing of lbm_cde_backward (measurement aid, not in the
 * paper). With on != 0 every later backward sweep records CUDA events on the
 * handle's stream around each checkpoint segment's recompute and reverse steps;
 * lbm_cde_backward_phases then returns, for the last sweep, ms_out[0] = the
 * recompute time, ms_out[1] = the reverse steps with their gradient reductions,
 * ms_out[2] = the whole sweep from its first to its last device operation
 * (host array of 3 doubles; zeros before the first profiled sweep). The events
 * add a little launch overhead, so profiled and unprofiled sweeps differ
 * slightly. Errors: LBM_E_ARG (NULL argument). */
lbm_status lbm_cde_set_profiling(lbm_cde_t h, int32_t on);
lbm_status lbm_cde_backward_phases(lbm_cde_t h, double* ms_out);

/* ---- Batched channels (Sec. 3.2 set-up, many instances per launch) --------
 * Independent D2Q9 MRT-A instances of uneven size, each with its own D, rates,
 * walls and row velocity profile u(y), advanced together; every step also
 * reduces, per instance, the moments of the cross-section mean
 *     phi-bar(x) = sum_y w_y phi(x, y)   (w = 1/2 on the two wall nodes, 1 else;
 *                                          w = 1 everywhere for periodic y)
 * as M_k = sum_x phi-bar(x) xi^k, k = 0, 1, 2, with xi = x - c(t) wrapped to
 * [-nx/2, nx/2) and c(t) = round(x_ref0 + x_ref_velocity * t): the sums of
 * Eq. 47, from which sigma^2 = M2/M0 - (M1/M0)^2 and alpha_L (Eq. 46). */
typedef struct lbm_cde_batch_s* lbm_cde_batch_t;

enum { LBM_BATCH_AUTO = 0, LBM_BATCH_PERSISTENT = 1, LBM_BATCH_PER_STEP = 2 };

typedef struct {
    int64_t nx, ny;          /* nx periodic columns, ny nodes across (walls on nodes 0, ny-1) */
    int32_t bc_lo_y, bc_hi_y;/* LBM_BC_NOFLUX_NODE, LBM_BC_BOUNCEBACK or LBM_BC_PERIODIC (both) */
    double D[4];             /* diffusion tensor, row-major 2 x 2, symmetric positive definite;
                                A = (3 D + I/2)^-1 (Eq. 36, MRT-A factor 1/3) */
    double s[15];            /* diagonal rates (NaN: s0 = 1, s1 = s2 = 1.1, s7 = s8 = 1.2) */
    int32_t tie_q_rates;     /* 1: s4 = sxx, s6 = syy */
    const float* u_row_dev;  /* device [2][ny] velocity per row (borrowed), or NULL (u = 0) */
    double x_ref0;           /* moment reference centre at t = 0 (node index) */
    double x_ref_velocity;   /* its drift per step */
    int32_t model;           /* LBM_MRT_A / B1 / B2 / B3 */
} lbm_cde_channel_desc;

typedef struct {
    int32_t mode;            /* LBM_BATCH_AUTO (persistent until autotuned) / PERSISTENT (one
                                cooperative launch per graph chunk: blocks or warps take work
                                tiles from a counter, bounded grid barriers separate the step's
                                phases) / PER_STEP (per step: one launch over 32 x 16 cell
                                tiles, two nodes per thread in paired FP32 arithmetic; its two
                                moment passes run on a second, library-owned stream, overlapping
                                the next step's cells, and join the batch's stream at the end
                                of each run) */
    int32_t tile_rows;       /* PERSISTENT work tiles: 0 (default) the 32 x 16 cell tiles of
                                PER_STEP taken by whole blocks, one grid barrier per step, the
                                moment passes of steps k - 1 and k - 2 run ahead of the cells of
                                step k inside the launch; 1 .. 1024: tiles of 32 columns x
                                tile_rows rows, one warp each, one node per thread */
    int32_t graph_steps;     /* steps per captured CUDA graph (ring of moments), 1 .. 4096 */
    int64_t barrier_timeout_cycles; /* clock64 cycles a CTA waits at a grid barrier (and, on
                                cell tiles, at its shared-memory barriers) before the launch
                                gives up with LBM_E_TIMEOUT (default 2e9, about 1 s) */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free_)(void* ptr, void* ctx);
    void* alloc_ctx;
    void* stream;
} lbm_cde_batch_opts;

lbm_status lbm_cde_batch_opts_init(lbm_cde_batch_opts* opts);

/* Creates a batch of n instances. Cells of all instances are concatenated in
 * instance order (x fastest, then y). Errors: LBM_E_ARG, LBM_E_NOT_SPD, LBM_E_OOM. */
lbm_status lbm_cde_batch_create(const lbm_cde_channel_desc* descs, int32_t n, const lbm_cde_batch_opts* opts,
                                lbm_cde_batch_t* out);
lbm_status lbm_cde_batch_destroy(lbm_cde_batch_t b);

/* Total number of cells of all instances. */
lbm_status lbm_cde_batch_cells(lbm_cde_batch_t b, int64_t* ncat);

/* f = f^eq(phi0, u) from a device FP32 field [ncat] (concatenated), step 0. */
lbm_status lbm_cde_batch_set_phi(lbm_cde_batch_t b, const float* phi_dev);

/* phi of the current state into a device FP32 buffer [ncat]. */
lbm_status lbm_cde_batch_get_phi(lbm_cde_batch_t b, float* phi_dev);

/* Runs nsteps steps (full chunks replay one captured CUDA graph) and copies the
 * moments of every step to moments_host ([nsteps][n][3] doubles, or NULL).
 * Synchronising; returns LBM_E_TIMEOUT if a grid barrier gave up (the state is
 * then invalid until the next set_phi). */
lbm_status lbm_cde_batch_run(lbm_cde_batch_t b, int64_t nsteps, double* moments_host);

/* Times PERSISTENT on cell tiles (0) and at tile heights 8, 16, 32 rows, and PER_STEP on `steps` steps,
 * keeps the fastest (restoring the state and step count) and reports it. */
lbm_status lbm_cde_batch_autotune(lbm_cde_batch_t b, int64_t steps, int32_t* mode_out, int32_t* tile_out);

/* Selects an execution mode and tile height explicitly. */
lbm_status lbm_cde_batch_config(lbm_cde_batch_t b, int32_t mode, int32_t tile_rows);

const char* lbm_cde_batch_last_error(lbm_cde_batch_t b);

/* Allocation-free FP64 sum of phi over a raw state (no counterpart in the
 * paper; an addition for callers that cannot allocate device memory, such as
 * code running while a stream is captured into a CUDA graph or under a fixed
 * memory budget). It performs no cudaMalloc/cudaFree or other allocation: the
 * per-block partial sums live in a file-scope __device__ array of
 * LBM_NOALLOC_MAX_PARTIALS doubles (128 KiB, held on every GPU that loads the
 * library until the process exits).
 *   state_dev : device pointer to a state laid out as lbm_cde_get_state writes
 *               it (lattice planes of ncell elements, then for the 16-bit forms
 *               an FP32 phi plane); 4-byte aligned, and for the 16-bit forms
 *               q * ncell must be even so that the phi plane is aligned
 *   lattice, storage : LBM_D2Q9 / LBM_D3Q15 and LBM_STORE_* of that state
 *   ncell     : cells in the state, 1 .. LBM_NOALLOC_MAX_CELLS; larger states
 *               are rejected with LBM_E_ARG
 *   sum_dev   : device pointer to one double, overwritten with the sum
 *   stream    : cudaStream_t (NULL: legacy stream); asynchronous
 * The first call on a device resolves the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call before
 * capturing a stream into a graph. That address is kept for the life of the
 * process: calls made after cudaDeviceReset (or any other teardown of the
 * device's primary context) in the same process are not supported, since the
 * array then lives at a new address. Every call overwrites the partials it uses,
 * so nothing needs clearing, but all calls on a GPU share the one array: calls
 * whose kernels overlap on the GPU (unordered streams) race. Errors: LBM_E_ARG,
 * LBM_E_CUDA; lbm_cde_noalloc_last_error() describes the last failure of the
 * calling thread. */
#define LBM_NOALLOC_MAX_PARTIALS 16384
#define LBM_NOALLOC_CELLS_PER_BLOCK 4096
#define LBM_NOALLOC_MAX_CELLS (16384LL * 4096LL)
lbm_status lbm_cde_sum_state_noalloc(const void* state_dev, int32_t lattice, int32_t storage,
                                     int64_t ncell, double* sum_dev, void* stream);
const char* lbm_cde_noalloc_last_error(void);

/* Message for the last error on this handle (static storage owned by the
 * handle; NULL handle gives the last creation error). */
const char* lbm_cde_last_error(lbm_cde_t h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_CDE_H */
