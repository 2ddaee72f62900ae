/*
 * hproj.h - C ABI of the GB300 (sm_103a) pressure-projection library.
 *
 * The library computes the pressure-projection step of the hybrid
 * CNN + Jacobi incompressible solver of arXiv 2109.09363 on 2D staggered
 * (MAC) grids with a boolean obstacle field:
 *   - corrected velocity  u = u* - (dt / rho0) grad p              (Eq. 2)
 *   - Poisson equation    (dt / rho0) lap p = div u*               (Eq. 3)
 *   - Jacobi iteration    X_{t+1} = D^{-1} (b - (L + U) X_t)       (Sec. 2.2)
 *   - stop test on E_1 = mean |div u| against a user threshold     (Sec. 3.3, Sec. 4.1)
 *
 * Grid conventions (every array is row-major and contiguous, batch first):
 *   cell (i, j): i = column, j = row, row 0 is the top of the image.
 *   u     float [B][ny][nx+1]  face (j, i) between cells (i-1, j) and (i, j)
 *   v     float [B][ny+1][nx]  face (j, i) between cells (i, j-1) and (i, j)
 *   flags uint8 [B][ny][nx]    non-zero = solid cell
 *   p, div, rho float [B][ny][nx]
 *   A face is open when it is not on the domain boundary and both adjacent
 *   cells are fluid; closed faces carry zero velocity (static walls).
 *   phi = (dt / rho0) p is the scaled pressure; the sweeps work on phi.
 *   E_1 divides by all nx * ny cells; solid cells have zero divergence.
 *
 * Memory: every array pointer is caller-owned DEVICE memory unless stated
 * otherwise.  Calls are asynchronous and ordered on the given CUDA stream
 * (passed as void*; NULL = legacy default stream); nothing synchronises the
 * host unless stated.  All calls of one context must be issued from one host
 * thread at a time, on one stream at a time.
 *
 * Errors: argument errors are returned immediately and nothing is launched.
 * HP_ERR_CUDA reports a failed launch or CUDA call; hp_last_cuda_error()
 * gives the CUDA error string.  There is no CPU fallback: a process without a
 * usable sm_103a device gets HP_ERR_CUDA from hp_ctx_create.
 */
#ifndef HPROJ_H
#define HPROJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HP_OK = 0,
    HP_ERR_INVALID_ARG = 1, /* null pointer, bad shape, shape above the context maximum */
    HP_ERR_CUDA = 2,        /* a CUDA call or launch failed */
    HP_ERR_NONFINITE = 3,   /* the input velocity holds NaN or Inf */
    HP_ERR_OOM = 5,         /* device allocation failed */
    HP_ERR_UNSUPPORTED = 6, /* the requested combination is not built */
    HP_ERR_TIMEOUT = 7,     /* a tensor-core completion wait gave up (hp_cnn_check) */
    HP_ERR_IO = 8,          /* a checkpoint file could not be written, or is missing,
                               truncated, corrupted or of another format version */
    HP_ERR_GUARD = 9,       /* a workspace's guard zone was overwritten (hp_ctx_check,
                               hp_cnn_check, hp_trainer_check) */
    /* not an error: the network's guess of some grid was not finite, and the
     * hybrid projection started that grid's sweeps from zero (hp_cnn_check) */
    HP_WARN_CNN_NONFINITE = 100
} hp_status;

/* Shape of a batch of grids.  Every call rejects a shape with a non-positive
 * size, or with batch > HP_MAX_BATCH or ny > HP_MAX_NY, with
 * HP_ERR_INVALID_ARG before it launches anything: the kernels cover rows and
 * grids with one CUDA grid dimension each (65535 blocks at most), some of
 * them with one more (the ny + 1 rows of v faces). */
#define HP_MAX_BATCH 65534
#define HP_MAX_NY 65534
typedef struct {
    int32_t batch; /* number of independent grids B */
    int32_t ny;    /* rows */
    int32_t nx;    /* columns */
} hp_shape;

/* Parameters of one projection (Sec. 2.2 and 3.3).
 *   threshold      E_t: stop at the first k with E_1(phi_k) <= E_t (k = 0 included)
 *   max_iters      cap on the number of sweeps; reaching it gives converged = 0
 *   fixed_iters    > 0: run exactly this many sweeps, no stop test (converged = 1)
 *   dt, rho0       p = phi * rho0 / dt
 *   temporal_block sweeps fused per launch of the blocked kernel, 1..8
 *                  (0 = library default)
 *   use_graph      1 = run the sweep loop as a CUDA-graph conditional WHILE node
 *                  (no host round trip per block); 0 = host-polled loop
 *   sweep_kernel   0 = library choice (4 where it runs, else 2), 1 = streaming
 *                  (one sweep per launch, stop decided one launch later),
 *                  2 = temporally blocked (T
 *                  sweeps per launch, replay to the exact stop; 4 rows per
 *                  thread), 3 = temporally blocked with 2 rows per thread
 *                  (twice the warps), 4 = grid-resident: one thread-block
 *                  cluster (up to 16 CTAs of 128 x 128 cells) keeps a whole
 *                  grid on chip for all sweeps, falling back to 2 when the
 *                  grid is larger than 512 x 512 cells or the cluster does
 *                  not fit on the device.  All give the same iterates bit for
 *                  bit; the FP64 E_k may differ in the last bits between
 *                  kernels (their partial sums are grouped differently).
 *   open_top       1 = the top boundary (the v faces of row 0) is open to an
 *                  exterior at p = 0: the faces of fluid cells of row 0 are
 *                  open (counted in n, in the divergence and corrected from
 *                  the exterior value 0); 0 = a closed wall (the default).
 *   inflow_x0, inflow_x1  bottom-boundary v faces (row ny) of the columns
 *                  [x0, x1) under fluid cells keep the velocity the caller
 *                  gives (a prescribed inflow, e.g. -U_in): they enter the
 *                  divergence of the cells above them, are never corrected
 *                  and stay closed for the pressure; x1 <= x0 = none.
 *   A closed box (both 0, the default) leaves the pressure defined up to a
 *   constant; with an open top it is unique.  Prescribed inflow without an
 *   open top has no solution unless the inflow sums to zero. */
typedef struct {
    double threshold;
    int32_t max_iters;
    int32_t fixed_iters;
    float dt;
    float rho0;
    int32_t temporal_block;
    int32_t use_graph;
    int32_t sweep_kernel;
    int32_t open_top;
    int32_t inflow_x0;
    int32_t inflow_x1;
} hp_project_params;

typedef struct hp_ctx hp_ctx;

/* Create a context on `device` that owns the workspaces for grids up to
 * max_shape (cells = batch * ny * nx).  Allocates device memory once; no later
 * call allocates.  Returns HP_ERR_CUDA when the device is missing or is not
 * sm_103. */
hp_status hp_ctx_create(hp_ctx **ctx, hp_shape max_shape, int device);
void hp_ctx_destroy(hp_ctx *ctx);
/* Memory check of a context (a substitute for a memory checker): every
 * device workspace of a context, a network and a trainer is allocated 256
 * bytes longer and those guard bytes hold a fixed pattern; this call
 * synchronises the device and returns HP_ERR_GUARD if a kernel wrote into a
 * guard zone (past the end of a workspace), HP_ERR_CUDA on a pending CUDA
 * error, else HP_OK. */
hp_status hp_ctx_check(hp_ctx *ctx);

const char *hp_status_string(hp_status s);
const char *hp_last_cuda_error(void);

/* Open-face bits per cell (a geometry step of Sec. 2.2): bit 0 west (u face i),
 * bit 1 east (u face i+1), bit 2 north (v face j), bit 3 south (v face j+1).
 * flags, mask_out: uint8 [B][ny][nx], device. */
hp_status hp_face_mask(const uint8_t *flags, uint8_t *mask_out, hp_shape shape, void *stream);

/* Divergence of u* (right-hand side of Eq. 3), first-order forward difference
 * over the OPEN faces, dx = 1; div = 0 on solid cells.  u, v are read only
 * (closed-face values are ignored).  div_out: float [B][ny][nx], device. */
hp_status hp_divergence(const float *u, const float *v, const uint8_t *flags, float *div_out,
                        hp_shape shape, void *stream);

/* Mean and max of |div u| over all cells per grid (E_1 and E_inf of Sec. 4.1),
 * divergence over open faces as in hp_divergence.  e1_out, einf_out: double
 * [B], device.  Uses the context's workspaces (no allocation). */
hp_status hp_div_norms(hp_ctx *ctx, const float *u, const float *v, const uint8_t *flags,
                       double *e1_out, double *einf_out, hp_shape shape, void *stream);

/* Pressure projection (Eq. 2-3, hybrid rule of Sec. 3.3), in place on (u, v).
 *   1. div = div u*  over open faces;
 *   2. phi_0 = phi0 (the CNN guess of the hybrid method; NULL = 0), set to 0
 *      on cells without an open face;
 *   3. k* = first k with E_1(phi_k) <= threshold, else max_iters; the sweeps
 *      are masked Jacobi on the open-face Laplacian, E_1 is summed in FP64
 *      after every sweep in a fixed order;
 *   4. u = u* - grad phi on open faces, 0 on closed faces; p = phi rho0 / dt.
 * A grid whose E_1 is not finite (NaN or Inf in its input) stops at that k
 * with converged = 0; the other grids of the batch are not affected.
 * Outputs (device): p_out float [B][ny][nx] (may be NULL), iters_out int32 [B],
 * e1_out / einf_out double [B] (norms of the CORRECTED velocity; may be NULL),
 * converged_out uint8 [B] (may be NULL).
 * phi0: float [B][ny][nx] device or NULL.
 * e_hist: optional double [B][hist_len] device; receives E_1(phi_k) for
 * k < hist_len up to the stop (entries after the stop are left untouched).
 * Uses the context's workspaces; calls on one context must not overlap. */
hp_status hp_project(hp_ctx *ctx, float *u, float *v, const uint8_t *flags, hp_shape shape,
                     const hp_project_params *params, const float *phi0, float *p_out,
                     int32_t *iters_out, double *e1_out, double *einf_out,
                     uint8_t *converged_out, double *e_hist, int32_t hist_len, void *stream);

/* Jacobi sweeps only (the inner step of hp_project): phi_out = n sweeps of the
 * masked Jacobi iteration applied to phi_in with right-hand side div (both
 * device float [B][ny][nx]).  e_out (device double [B][n], may be NULL)
 * receives E_1(phi_k) of the input of each sweep.  phi_in and phi_out must not
 * alias.  Uses the context's workspaces. */
hp_status hp_jacobi_sweeps(hp_ctx *ctx, const float *phi_in, const float *div,
                           const uint8_t *flags, float *phi_out, int32_t n, double *e_out,
                           hp_shape shape, void *stream);

/* Pressure target of a training pair from the plain solver (the networks are
 * trained on pairs of divergence and pressure, Sec. 3.2): n masked Jacobi
 * sweeps from phi_0 = 0 on the right-hand side div (n >= 0), then
 *     target_out = (phi_n + phi_{n+1}) / 2,
 * the mean of the last iterate and one more sweep; the mean cancels the
 * period-2 (checkerboard) component that plain Jacobi never damps.  The
 * iterates are those of hp_jacobi_sweeps bit for bit.  div, target_out float
 * [B][ny][nx], flags uint8, device memory; target_out must not alias div.
 * Uses the context's workspaces. */
hp_status hp_jacobi_target(hp_ctx *ctx, const float *div, const uint8_t *flags, int32_t n,
                           float *target_out, hp_shape shape, void *stream);

/* Number of grids of this shape that the grid-resident sweep kernel
 * (sweep_kernel = 4) can hold on the device at once, one thread-block cluster
 * of ceil(nx/128) x ceil(ny/128) CTAs per grid; 0 when that kernel cannot run
 * the shape (grid above 512 x 512 cells, or the cluster does not fit), in
 * which case hp_project falls back to the temporally blocked kernel.  Host
 * query only (no kernel launch); 0 for a NULL context or an invalid shape. */
int32_t hp_resident_clusters(hp_ctx *ctx, hp_shape shape);

/* Parameters of the plume driver step (Sec. 2.2: semi-Lagrangian advection
 * of the density and of the velocity, then the external force by forward
 * Euler, giving u* for the projection).
 *   dt        time step
 *   gravity   g of the Boussinesq force on v: v += dt * g * (rho_face - rho_amb);
 *             row 0 is the top, so g < 0 makes light fluid rise
 *   rho_amb   ambient density
 *   rho_in    density imposed on the inlet cells before the step
 *   inlet_x0, inlet_x1  inlet columns [x0, x1) of the bottom row (x1 <= x0: no inlet)
 *   scheme    0: first-order semi-Lagrangian; 1: MacCormack (the scheme of
 *             Sec. 2.2, after Selle et al. 2008): the forward semi-Lagrangian
 *             value q_f, the forward field sampled backwards at x + dt vel(x)
 *             (q_b), and q_f + (q - q_b) / 2 clamped to the range of the four
 *             samples the forward step interpolated; for rho, u and v alike.
 *             Other values return HP_ERR_INVALID_ARG.
 *   u_in      speed of the injected fluid (Sec. 4.1): the bottom-boundary v
 *             faces of the inlet columns under fluid cells are set to -u_in
 *             (upwards) after the step; 0 = no velocity injection
 *   open_top  1: the top boundary is open (the outflow of the injected
 *             fluid); its v faces keep their advected velocity instead of
 *             being closed; 0 = a closed wall.
 *   Project such a step with open_top and inflow_x0, inflow_x1 of
 *   hp_project_params set to the same values. */
typedef struct {
    float dt;
    float gravity;
    float rho_amb;
    float rho_in;
    int32_t inlet_x0;
    int32_t inlet_x1;
    int32_t scheme;
    float u_in;
    int32_t open_top;
} hp_plume_params;

/* One driver step on B grids, out of place (outputs must not alias inputs):
 *   1. rho = rho_in on the inlet cells;
 *   2. rho (cell centres), u and v (faces) sampled bilinearly at the departure
 *      point x - dt * vel(x), vel = the input velocity interpolated per
 *      component; positions clamped to each quantity's sample span;
 *   3. v += dt * g * (mean of the two advected densities next to the face
 *      - rho_amb) on interior v faces;
 *   4. every closed face set to zero, except the top faces of fluid cells
 *      when open_top (advected like interior faces); the inlet faces of the
 *      bottom boundary set to -u_in (when u_in != 0).
 * u, u_out float [B][ny][nx+1]; v, v_out [B][ny+1][nx]; rho, rho_out, flags
 * [B][ny][nx]; device memory. */
hp_status hp_advect_step(const float *u, const float *v, const float *rho, const uint8_t *flags,
                         float *u_out, float *v_out, float *rho_out, hp_shape shape,
                         const hp_plume_params *params, void *stream);

/* Plume head of the paper's diagnostics (Sec. 4.1: the highest point of the
 * plume, and its horizontal extent on both sides around an obstacle): for
 * each grid, over the cells with |rho - rho_amb| >= contrast (compared in
 * FP32), out[b] = {smallest row index (row 0 is the top), smallest column,
 * largest column}; {ny, nx, -1} when no cell qualifies.  The normalised
 * positions follow on the host: h_y = (ny - row) / ny, left and right extent
 * (nx / 2 - col_min) / nx and (col_max + 1 - nx / 2) / nx.  rho float
 * [B][ny][nx], out int32 [B][3]: device memory; contrast >= 0. */
hp_status hp_plume_head(const float *rho, hp_shape shape, float rho_amb, float contrast,
                        int32_t *out, void *stream);

/* 3 x 3 convolution with replicated borders (the convolutions of the
 * MultiScale network, Sec. 3.1), on the tensor cores: BF16 inputs and weights,
 * FP32 accumulation, y = [relu](conv(x, w) + bias) rounded to BF16.
 *   x     bf16 [batch][height][width][cin]   (NHWC, 16-byte aligned)
 *   w     bf16 [3][3][cout][cin]             (tap (dy, dx) for offsets -1..1)
 *   bias  float [cout]
 *   y     bf16 [batch][height][width][cout]  (16-byte aligned)
 *   err   optional int32 device word set to 1 if a tensor-core completion
 *         wait timed out (the call then leaves y incomplete)
 * (cin, cout) in {32, 64} x {32, 64}; other sizes return HP_ERR_UNSUPPORTED.
 * Device memory, stream-ordered; bf16 values are passed as their 16-bit
 * patterns (uint16_t). */
hp_status hp_conv3x3_bf16(const uint16_t *x, const uint16_t *w, const float *bias, uint16_t *y,
                          int32_t batch, int32_t height, int32_t width, int32_t cin, int32_t cout,
                          int32_t relu, int32_t *err, void *stream);

/* Adjoint of the fixed-count projection (the paper trains its networks through
 * the solver and notes that the gradient of the correction is known,
 * Sec. 3.2).  Forward map (hp_project with fixed_iters = k and a guess phi0):
 * (u*, v*, phi_0) -> (u, v, p).  Given gu = dL/du, gv = dL/dv and gp = dL/dp
 * (may be NULL), returns dL/du*, dL/dv* (0 on closed faces) and dL/dphi_0,
 * using k transposed sweeps (no stored iterates: the map is affine).  The
 * closed box only (open_top = 0, no inflow faces).
 * gu, gu_star float [B][ny][nx+1]; gv, gv_star [B][ny+1][nx]; gp, g_phi0
 * [B][ny][nx]; device memory; outputs must not alias inputs.  Uses the
 * context's workspaces. */
hp_status hp_project_adjoint(hp_ctx *ctx, const float *gu, const float *gv, const float *gp,
                             const uint8_t *flags, hp_shape shape, int32_t k, float dt,
                             float rho0, float *gu_star, float *gv_star, float *g_phi0,
                             void *stream);

/* CNNs of the hybrid method (Sec. 3.1).  The MultiScale: three branches at
 * 1/4, 1/2 and full resolution, 3 x 3 convolutions with replicated borders,
 * ReLU after every convolution of a branch except its last two, 2 x 2 / 4 x 4
 * average pooling down, bilinear x 2 up; input [div / s, flags], s = mean
 * |div| over fluid cells (1 if zero); 372,643 parameters.  The SmallScale and
 * the MonoScale below.  BF16 weights and activations, FP32 accumulation
 * (tensor cores for the 32/64-channel layers).  An hp_cnn owns its device
 * weights and a workspace for grids up to max_shape (ny, nx multiples of 4). */
typedef struct hp_cnn hp_cnn;
/* Architectures (Sec. 3.1).  SmallScale: the MultiScale graph with fewer
 * filters, every 64-channel layer at 32 channels, 123,491 parameters.
 * MonoScale: one feed-forward branch at full resolution on [div / s, flags],
 * 2 -> 32 -> 64 -> 64 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1 (3 x 3, replicated
 * borders, ReLU after all but the last two), 222,497 parameters; its params
 * vector holds its 9 layers in that order.
 * Unet: encoder levels n, n/2, n/4, n/8 ending in 32-channel skip features
 * (2 -> 32 -> 32, then after each 2 x 2 max pooling 32 -> 64 -> 32), bottom
 * n/16 32 -> 64 -> 64 -> 32, decoder levels on [bilinear x 2 of the coarser
 * features, skip features] 64 -> 64 -> 32, the last 64 -> 32 -> 32 and a
 * 1 x 1 32 -> 1 (its weights [1][32][1][1] in params); ReLU after all but
 * the last two; 388,545 parameters; grid sizes multiples of 16 (also for its
 * trainer). */
typedef enum {
    HP_CNN_MULTISCALE = 0,
    HP_CNN_SMALLSCALE = 1,
    HP_CNN_MONOSCALE = 2,
    HP_CNN_UNET = 3
} hp_cnn_arch;
/* Parameter count of the MultiScale; of the architecture arch (-1 if arch is
 * not one of hp_cnn_arch). */
int64_t hp_cnn_param_count(void);
int64_t hp_cnn_arch_param_count(int32_t arch);
/* A MultiScale network (hp_cnn_create) or one of architecture arch;
 * HP_ERR_INVALID_ARG for an unknown arch or a bad shape. */
hp_status hp_cnn_create(hp_cnn **cnn, hp_shape max_shape, int device);
hp_status hp_cnn_create_arch(hp_cnn **cnn, int32_t arch, hp_shape max_shape, int device);
/* The architecture of cnn (-1 for NULL). */
int32_t hp_cnn_get_arch(const hp_cnn *cnn);
void hp_cnn_destroy(hp_cnn *cnn);
/* params: HOST float [hp_cnn_arch_param_count(arch)], layers in network
 * order (MultiScale and SmallScale: scale 1/4 (5 layers), 1/2 (7), 1 (7));
 * per layer weights [cout][cin][k][k] (k = 3, the Unet's output layer 1)
 * then bias [cout].  Weights are rounded to BF16 on upload; synchronous. */
hp_status hp_cnn_set_params(hp_cnn *cnn, const float *params, int64_t n);
/* Device-side status of a network: every wait of its tensor-core kernels on
 * the completion of MMAs or copies is bounded; one that gives up leaves that
 * kernel's output incomplete, sets an error word of the network and lets the
 * kernel return instead of hanging.  hp_project_hybrid also records there
 * that it replaced a non-finite guess.  This call synchronises the device,
 * reads and clears that word: HP_ERR_TIMEOUT if a wait gave up since the last
 * check (in hp_cnn_forward, hp_project_hybrid or a trainer built on the
 * network), else HP_ERR_GUARD if a guard zone of the network's workspaces was
 * overwritten (as hp_ctx_check), else HP_WARN_CNN_NONFINITE if a hybrid
 * projection fell back to a zero guess, else HP_OK. */
hp_status hp_cnn_check(hp_cnn *cnn);
/* Polls of each bounded pipeline wait (copies and MMAs of the warp-
 * specialised convolution and weight-gradient kernels, images from 32 pixels
 * wide) before it gives up; 0 restores the compiled limit (2^22 polls, far
 * above any wait of a healthy kernel).  A small value makes those waits give
 * up on purpose: the kernels then still wait (with the compiled limit) for
 * the MMAs they issued, free their tensor memory and return, and
 * hp_cnn_check reports HP_ERR_TIMEOUT; the outputs of such calls are
 * incomplete.  Host only, no synchronisation; HP_ERR_INVALID_ARG for NULL. */
hp_status hp_cnn_set_wait_limit(hp_cnn *cnn, uint32_t polls);
hp_status hp_cnn_get_params(const hp_cnn *cnn, float *params, int64_t n);
/* Network output phi_hat (float [B][ny][nx], device; the guess is s * phi_hat)
 * and s (float [B], device, may be NULL) for the divergence div (float
 * [B][ny][nx]) and flags. */
hp_status hp_cnn_forward(hp_cnn *cnn, const float *div, const uint8_t *flags, float *phi_hat,
                         float *s_out, hp_shape shape, void *stream);
/* Hybrid projection (Sec. 3.3): phi_0 = s * CNN(div / s, flags) (0 on cells
 * without an open face), then hp_project from phi_0.  Same arguments and
 * outputs as hp_project; the batch and grid must also fit the network (its
 * max_shape, sides multiples of 4, of 16 for the Unet); every argument is
 * checked before anything is launched.  The Jacobi sweeps always follow and
 * check the guess: a grid whose guess is not finite (NaN or Inf on a cell
 * with an open face) starts from phi_0 = 0 instead, i.e. it is the plain
 * projection, while the other grids keep their guesses; hp_cnn_check then
 * returns HP_WARN_CNN_NONFINITE. */
hp_status hp_project_hybrid(hp_ctx *ctx, hp_cnn *cnn, float *u, float *v, const uint8_t *flags,
                            hp_shape shape, const hp_project_params *params, float *p_out,
                            int32_t *iters_out, double *e1_out, double *einf_out,
                            uint8_t *converged_out, double *e_hist, int32_t hist_len,
                            void *stream);

/* Training of the CNNs (Sec. 3.2 trains the networks with a
 * gradient-descent algorithm): FP32 master weights on the device, Adam,
 * BF16 weights of the hp_cnn refreshed after every step.  Loss per grid,
 * averaged over the batch, with t = target / s (target = the scaled pressure
 * phi* of the plain solver), d = div / s and e = phi_hat - t:
 * sum over fluid cells of (e - mean e)^2 / sum over fluid cells of
 * (t - mean t)^2, plus lambda_div * sum r^2 / sum d^2 with r = d - L phi_hat
 * on cells with an open face.  The trainer keeps every activation of a batch
 * up to max_shape (ny, nx multiples of 4). */
typedef struct hp_trainer hp_trainer;
typedef struct {
    float lr, beta1, beta2, eps;
    float lambda_div;
} hp_train_params;
/* Every architecture trains (the Unet's backward routes each pooled gradient
 * to the first maximum of its 2 x 2 window, in the order (0, 0), (0, 1),
 * (1, 0), (1, 1)).  max_shape may not exceed the network's own, and its sides
 * are multiples of 4 (16 for the Unet) (HP_ERR_INVALID_ARG).  *trainer is
 * NULL on every error. */
hp_status hp_trainer_create(hp_trainer **trainer, hp_cnn *cnn, hp_shape max_shape);
void hp_trainer_destroy(hp_trainer *trainer);
/* Loss (double [1], device, may be NULL) and its gradient w.r.t. every
 * parameter (float [the network's parameter count], device, may be NULL; network
 * parameter order) for one batch; div, target float [B][ny][nx], flags u8. */
hp_status hp_trainer_gradient(hp_trainer *trainer, const float *div, const uint8_t *flags,
                              const float *target, hp_shape shape, float lambda_div,
                              float *grad_out, double *loss_out, void *stream);
/* One Adam step on one batch; loss_out as above. */
hp_status hp_trainer_step(hp_trainer *trainer, const float *div, const uint8_t *flags,
                          const float *target, hp_shape shape, const hp_train_params *params,
                          double *loss_out, void *stream);
/* Physics-driven (unsupervised) loss of Sec. 3.2, Eq. 4: no target pressure.
 * During training the network alone solves the Poisson problem: its guess
 * s_b * phi_hat_b corrects the velocity u*_b whose divergence is div (Eq. 2,
 * no Jacobi sweep), and the loss is
 *     sum over grids b of weight[b] / (nx ny) * sum over cells |div u_b|^norm
 * with norm = 1 (the printed Eq. 4) or 2 (the mean squared error the text
 * names).  div u_b equals s_b times the residual of the scaled problem, so
 * only div and flags are needed.  The paper's short- and long-term terms
 * (alpha at t + 1, beta at t + n) are two sets of grids of one batch with
 * weights alpha / B and beta / B.
 * div float [B][ny][nx], flags u8, weight float [B]: device memory.
 * grad_out, loss_out as for hp_trainer_gradient.  norm other than 1 or 2
 * returns HP_ERR_INVALID_ARG. */
hp_status hp_trainer_pdnn_gradient(hp_trainer *trainer, const float *div, const uint8_t *flags,
                                   const float *weight, hp_shape shape, int32_t norm,
                                   float *grad_out, double *loss_out, void *stream);
/* One Adam step on the physics-driven loss (params->lambda_div unused). */
hp_status hp_trainer_pdnn_step(hp_trainer *trainer, const float *div, const uint8_t *flags,
                               const float *weight, hp_shape shape, int32_t norm,
                               const hp_train_params *params, double *loss_out, void *stream);
/* Copy the trained FP32 masters into the hp_cnn (hp_cnn_get_params then
 * returns them); synchronises the device and then reports the network's
 * device status as hp_cnn_check does (the masters are copied either way). */
hp_status hp_trainer_sync_params(hp_trainer *trainer);
/* The guard zones of a trainer's workspaces (as hp_ctx_check), then
 * hp_cnn_check of its network. */
hp_status hp_trainer_check(hp_trainer *trainer);

/* Optimiser state of a trainer, copied to HOST memory (synchronous): the FP32
 * masters, the first and second Adam moments (float [the network's parameter
 * count] each, network parameter order) and the number of Adam steps taken;
 * any pointer may be NULL. */
hp_status hp_trainer_get_state(hp_trainer *trainer, float *master, float *m, float *v,
                               int64_t *step);

/* Checkpoint files (a training run that stops resumes from one; the format
 * is versioned and checksummed; little-endian):
 *   magic "HPCNNCK1", uint32 version 1, int32 arch, int64 n (the
 *   architecture's parameter count), int64 step, uint32 moments (0/1),
 *   uint32 0, float32 parameters[n] (network order, as hp_cnn_set_params),
 *   when moments = 1 float32 m[n] and v[n] (Adam moments), then the FNV-1a
 *   64-bit checksum of all bytes before it.
 * Files are written under path + ".tmp" and renamed; host I/O only, the
 * trainer calls synchronise the device.  Unreadable, truncated, foreign or
 * corrupted files give HP_ERR_IO and change nothing.
 * hp_cnn_save: the network's architecture and parameters (those last set
 * with hp_cnn_set_params or copied back by hp_trainer_sync_params), step 0,
 * no moments.
 * hp_cnn_load: a new network of the file's architecture for grids up to
 * max_shape on `device`, with the file's parameters (as hp_cnn_create_arch
 * followed by hp_cnn_set_params); *cnn is NULL on every error.
 * hp_trainer_save: the trainer's masters, Adam moments and step.
 * hp_trainer_load: restores them into a trainer whose network has the
 * file's architecture (else HP_ERR_IO) and refreshes the network's BF16
 * weights and its host copy of the parameters; a file without moments
 * restarts Adam from step 0 with zero moments. */
hp_status hp_cnn_save(const hp_cnn *cnn, const char *path);
hp_status hp_cnn_load(hp_cnn **cnn, const char *path, hp_shape max_shape, int device);
hp_status hp_trainer_save(hp_trainer *trainer, const char *path);
hp_status hp_trainer_load(hp_trainer *trainer, const char *path);

/* Allocation-free variant of hp_div_norms.  The paper has no counterpart; it
 * exists for callers that cannot call cudaMalloc: a host framework that owns
 * all device memory through its own pool and forbids other allocations, a
 * latency-critical loop where an allocation (and the device synchronisation
 * it may cause) is not acceptable, or a process that has reached its memory
 * budget.  Such a caller cannot create an hp_ctx, so this call takes no
 * context; it computes the same E_1 and E_inf as hp_div_norms, with the same
 * kernel.
 *
 * Its scratch (one 8-byte partial, the FP32 sum and max of |div|, per
 * 256-cell block) is a fixed array inside libhproj.so: every GPU that loads
 * the library holds it (2 MB) until the process exits.  Limits: batch <=
 * HP_NOALLOC_MAX_BATCH and batch * ny * ceil(nx / 256) <= HP_NOALLOC_MAX_BLOCKS
 * (16 grids of 2048 x 2048 fit), and batch, ny within HP_MAX_BATCH,
 * HP_MAX_NY like every call; larger shapes return HP_ERR_INVALID_ARG and
 * launch nothing.  The call works on the device and CUDA context that are
 * current.  The array's device address belongs to the context that loaded
 * the library's kernels: the first call in each context (the device's
 * primary context, again after a cudaDeviceReset, or a context the caller
 * made current through the driver API) looks it up with that context current
 * (cudaGetSymbolAddress) and caches it per context, so make that first call
 * before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and give wrong
 * results.  Each call
 * overwrites every partial it reads before reading it; no cudaMalloc,
 * cudaFree or allocating library routine is called.  u, v, flags, e1_out, einf_out as in hp_div_norms. */
#define HP_NOALLOC_MAX_BATCH 16384
#define HP_NOALLOC_MAX_BLOCKS 262144
hp_status hp_div_norms_noalloc(const float *u, const float *v, const uint8_t *flags,
                               double *e1_out, double *einf_out, hp_shape shape, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HPROJ_H */
