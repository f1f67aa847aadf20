/*
 * libdpsr: spectral Differentiable Poisson Surface Reconstruction (DPSR) on a
 * single GB300 GPU (sm_103a). The layer of "Shape As Points" (Peng et al.,
 * arXiv 2106.03452), Sec. 3.1, derived in supplementary Sec. A:
 *
 *   v    = trilinear splat of the point normals onto an r^3 grid     (Eq. A1-A2)
 *   v~   = FFT(v)                                                     (Eq. A3)
 *   chi~ = g(u) * (i u . v~) / (-2 pi |u|^2),
 *          g(u) = exp(-2 sigma^2 |u|^2 / r^2)                         (Eq. 3, A7)
 *   chi' = IFFT(chi~)                                                 (Eq. A8)
 *   chi  = m / |chi'(0) - mu| * (chi' - mu),  mu = mean_i chi'(c_i),
 *          m = 0.5                                                    (Eq. 4, A9)
 *
 * and its exact reverse-mode derivative (what Eq. 5 backpropagates through).
 *
 * Conventions (all calls):
 *  - The domain is the periodic unit cube [0,1)^3 with grid origin 0 and voxel
 *    size 1/r; vertex (ix,iy,iz) sits at (ix,iy,iz)/r. Coordinates outside
 *    [0,1) wrap around. Frequencies are integer cycles per unit length; the
 *    a-th term of u . v~ is zero at the Nyquist index k_a = r/2 and the DC
 *    term of chi~ is zero. The scale uses the shifted value chi'(0) - mu, so
 *    |chi(0)| = m exactly, with a positive factor (outside positive for
 *    outward normals).
 *  - points, normals, dpoints, dnormals: N x 3 row-major float32.
 *    Normals are NOT normalised: their length weights the point.
 *  - chi_out, dchi: r^3 float32 in C order chi[ix][iy][iz] (iz fastest);
 *    axis 0 is the x coordinate. Both must start on a 16-byte boundary (they
 *    move by bulk copies and vector loads); DPSR_EINVAL otherwise.
 *  - Every pointer argument of dpsr_forward / dpsr_backward is a DEVICE
 *    pointer on the current CUDA device, owned by the caller; the library
 *    never frees it. dpsr_forward_host / dpsr_backward_host take HOST
 *    pointers instead and copy through the plan's stream.
 *  - Device work is asynchronous on the plan's stream. Errors found on the
 *    host (bad arguments, wrong call order) are returned at once and nothing
 *    is launched. Conditions found on the device (a non-finite input, a
 *    vanishing scale chi'(0) - mu) set a status word that dpsr_sync returns;
 *    the outputs of that call are then unspecified.
 *  - A plan is not thread-safe: one host thread at a time per plan.
 */
#ifndef DPSR_H
#define DPSR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DPSR_API __attribute__((visibility("default")))
#else
#define DPSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpsr_plan_s *dpsr_plan;

enum {
    DPSR_OK = 0,
    DPSR_EINVAL = -1,      /* bad argument: r not a power of two in range, N < 1, NULL, ... */
    DPSR_ENOMEM = -2,      /* device allocation failed */
    DPSR_ECUDA = -3,       /* a CUDA runtime call failed */
    DPSR_EDEGENERATE = -4, /* non-finite input or chi'(0) - mu == 0 (no finite scale) */
    DPSR_ESTATE = -5,      /* backward without a forward, or N above the reserved size */
    DPSR_ETIMEOUT = -6,    /* a bounded device wait gave up */
    DPSR_EBUSY = -7,       /* resource busy (serving admission) */
    DPSR_ECANCELED = -8,   /* a serving request cancelled before admission */
    DPSR_EBOUNDS = -9      /* debug builds: a data-dependent index failed its range check */
};

/* Create a plan for grid size r (a power of two, 8 <= r <= 512) and Gaussian
 * bandwidth sigma >= 0 in grid units of Eq. 3 (sigma = 0: no smoothing).
 * Allocates the plan's device workspace on the current device; the plan
 * stays bound to that device. On success *out receives the plan. */
DPSR_API int dpsr_plan_create(int r, float sigma, dpsr_plan *out);

/* The same over a periodic box [0, L0) x [0, L1) x [0, L2) instead of the
 * unit cube: the r^3 grid's voxel size is L_d / r along axis d (Eq. A1 with
 * a per-axis voxel size s, Sec. 3.1). box: 3 side lengths in FP64 (the
 * binning's cell arithmetic uses them unrounded), each finite and > 0, read
 * during the call (NULL: the unit cube). Points are then given in
 * box coordinates (wrapped with period L_d); the spectral operator of Eq. 3
 * uses the physical frequency u_d = f_d / L_d of the integer frequency f_d,
 * and the Gaussian keeps sigma in grid units on every axis,
 * g = exp(-2 sigma^2 sum_d f_d^2 / r^2). dL/dpoints come back in box
 * coordinates. The normalisation of Eq. 4 is unchanged. Errors: DPSR_EINVAL
 * for a bad box, else as dpsr_plan_create. Batches take a box per instance
 * (dpsr_batch_create_box); the serving, static and mesh entry points work on
 * the unit cube. */
DPSR_API int dpsr_plan_create_box(int r, float sigma, const double *box, dpsr_plan *out);

/* Free the plan and its workspace (synchronises its stream first). */
DPSR_API int dpsr_plan_destroy(dpsr_plan plan);

/* Run subsequent work on `stream` (a cudaStream_t; NULL = legacy default). */
DPSR_API int dpsr_plan_set_stream(dpsr_plan plan, void *stream);

/* Grow the point buffers to hold up to n_max points. dpsr_forward grows them
 * on demand; reserving first keeps forward calls free of allocations (needed
 * before capturing them in a CUDA graph). */
DPSR_API int dpsr_plan_reserve(dpsr_plan plan, int64_t n_max);

/* Device bytes a plan of size r uses with n_max points; with_bwd != 0 counts
 * what the backward pass needs as well. Used for admission by memory budget. */
DPSR_API size_t dpsr_plan_workspace_bytes(int r, int64_t n_max, int with_bwd);

/* Forward pass of Eq. 3-4 for N oriented points (device pointers). Writes
 * chi_out (r^3). Keeps, inside the plan, what the backward pass needs: the
 * points sorted by x-plane, the transformed weight field of the points, the
 * scalars mu and s, and the per-point gradient of the trilinear lookup of
 * chi'. The caller must keep points, normals and chi_out unchanged until the
 * matching dpsr_backward has run. */
DPSR_API int dpsr_forward(dpsr_plan plan, const float *points, const float *normals, int64_t N,
                 float *chi_out);

/* Backward pass: the exact adjoint (reverse-mode derivative, what Eq. 5
 * backpropagates through) of Eq. 4 (normalisation, including the mean mu and
 * the scale s), Eq. 3 / A7 (spectral solve: conj(H_a) = -H_a) and Eq. A1-A2
 * (the splat: its transpose is the trilinear gather, plus the derivative of
 * the trilinear weights for dL/dpoints). Given dchi = dL/dchi (r^3, device,
 * 16-byte aligned), overwrite dpoints and dnormals (N x 3, device) with
 * dL/dpoints and dL/dnormals of the last forward pass on this plan. Returns
 * DPSR_ESTATE if no forward pass ran, DPSR_EINVAL for a NULL or misaligned
 * pointer. */
DPSR_API int dpsr_backward(dpsr_plan plan, const float *dchi, float *dpoints, float *dnormals);

/* Host-memory variants: the same computation with host input and output
 * buffers; the host<->device copies run on the plan's stream inside the call,
 * which returns after the results are on the host. */
DPSR_API int dpsr_forward_host(dpsr_plan plan, const float *points, const float *normals, int64_t N,
                      float *chi_out);
DPSR_API int dpsr_backward_host(dpsr_plan plan, const float *dchi, float *dpoints, float *dnormals);

/* Forward and backward of one solve with HOST buffers in one call (the
 * layer of Sec. 3.1 and its adjoint, as dpsr_forward_host followed by
 * dpsr_backward_host with the upstream gradient dchi given up front). The
 * copies that do not feed the next kernel overlap the kernels on a second
 * stream of the plan: dchi goes up during the forward pass and chi comes down
 * during the backward pass; one synchronisation at the end returns the
 * device status. Page-locked host buffers let the copies overlap (pageable
 * ones serialise them). chi_out, dpoints, dnormals are overwritten; the plan
 * keeps the forward context, as after dpsr_forward_host. */
DPSR_API int dpsr_solve_host(dpsr_plan plan, const float *points, const float *normals, int64_t N,
                             const float *dchi, float *chi_out, float *dpoints, float *dnormals);

/* Wait for the plan's stream; return the device status of the work queued so
 * far and clear it: DPSR_ETIMEOUT if a bounded device wait gave up (checked
 * first: the outputs of that call are incomplete), else DPSR_EDEGENERATE for
 * a non-finite input or a vanishing scale of Eq. 4, else DPSR_OK. DPSR_ECUDA
 * if the stream itself failed. */
DPSR_API int dpsr_sync(dpsr_plan plan);

/* Failure-detection check through a plan: queue on the plan's stream one
 * kernel whose bounded wait (the wait every TMA barrier of the library uses)
 * is on a barrier that nothing completes. It gives up after limit_s seconds
 * (0 < limit_s <= 10) and sets the plan's status word, so that the next
 * dpsr_sync returns DPSR_ETIMEOUT; the context and the plan stay usable.
 * Asynchronous; DPSR_EINVAL for a bad limit. The paper has no counterpart. */
DPSR_API int dpsr_plan_check_bounded_wait(dpsr_plan plan, double limit_s);

/* Synchronise, then read the scalars of Eq. 4 of the last forward pass:
 * out[0] = mu (mean of chi' at the points), out[1] = s = chi'(0) - mu,
 * out[2] = m/|s|. chi' is recovered from chi as chi/out[2] + mu. */
DPSR_API int dpsr_get_scalars(dpsr_plan plan, double out[3]);

/* L_DPSR of Eq. 9, the training loss of the learning setting (Sec. 3.3;
 * supplementary Sec. B): the mean squared error between the chi of the last
 * forward pass on this plan and a target grid (for instance the solve of a
 * dense ground-truth sampling: 100 000 points at 128^3 in the paper),
 * loss = (1/n) sum_j (chi_j - target_j)^2, n = r^3 (the paper prints the
 * squared norm; the mean differs by the constant 1/n), and its gradient
 * dchi = (2/n) (chi - target), in one fused pass. target and dchi: r^3
 * float32 device arrays in chi's layout, 16-byte aligned, owned by the
 * caller; dchi is overwritten and can be passed to dpsr_backward as is.
 * Asynchronous on the plan's stream; dpsr_get_loss synchronises and reads
 * the loss (FP64 from deterministic float-float sums). DPSR_ESTATE without a
 * forward pass, DPSR_EINVAL for NULL or misaligned pointers. */
DPSR_API int dpsr_mse_grad(dpsr_plan plan, const float *target, float *dchi);
DPSR_API int dpsr_get_loss(dpsr_plan plan, double *loss);

/* Number of kernel launches the last dpsr_forward / dpsr_backward queued. */
DPSR_API int dpsr_plan_last_launches(dpsr_plan plan);

/* Trilinear lookup of an r^3 grid (device, layout as chi) at M query points
 * q (device, M x 3, periodic as the points of Eq. A1): out[k] = chi(q_k).
 * Its adjoint: grid[j] (+)= sum_k w_kj vals[k], the rasterization of Eq. A2
 * with scalar values; accumulate = 0 zeroes the grid first. Both run on
 * `stream` (a cudaStream_t). They give a loss defined on chi at target
 * points, such as mean_k chi(q_k)^2, and its gradient dL/dchi. */
DPSR_API int dpsr_grid_sample(const float *grid, int r, const float *q, int64_t M, float *out,
                              void *stream);
DPSR_API int dpsr_grid_splat(float *grid, int r, const float *q, const float *vals, int64_t M,
                             int accumulate, void *stream);

/* Mesh extraction for the optimisation setting (Sec. 3.2: the indicator grid
 * becomes a mesh at level 0, where the paper runs Marching Cubes). chi: r^3
 * float32 device grid (layout as dpsr_forward's chi_out, periodic), r a
 * power of two, 2 <= r <= 512. Each cube is split into Kuhn's six
 * tetrahedra (a marching-cubes variant without case tables; neighbouring
 * cubes agree on every shared vertex, so the surface is closed away from
 * the periodic wrap-around) and the level set chi = level is cut from each.
 * Writes up to max_tris triangles: tris[t][3][3] float32 corner coordinates
 * in the unit cube (unwrapped: cube r - 1 reaches 1.0), counter-clockwise
 * about normals[t][3], the unit normal pointing towards increasing chi. The
 * total number of triangles goes to *count (a device uint64, written on
 * `stream`); more than max_tris means the buffers were too small (the
 * triangles beyond max_tris are dropped). Triangle order varies between
 * calls; the set does not. Asynchronous; DPSR_EINVAL for bad arguments. */
DPSR_API int dpsr_mesh_extract(const float *chi, int r, float level, float *tris, float *normals,
                               int64_t max_tris, unsigned long long *count, void *stream);

/* The surrogate gradient of Eq. 6 (d p_mesh / d chi = -n_mesh) for M points
 * on the mesh, p (M x 3, unit cube) with unit normals n (M x 3) and the
 * loss gradient dldp = dL/dp (M x 3), all device float32: each point
 * contributes dL/dp . (-n) to dL/dchi through the adjoint of the trilinear
 * lookup at p (the rasterization of Eq. A2, periodic). dchi: r^3 device
 * grid, zeroed first unless accumulate != 0; float atomics (summation order
 * varies). The result goes to dpsr_backward as its dchi. */
DPSR_API int dpsr_mesh_surrogate_splat(float *dchi, int r, const float *points, const float *normals,
                                       const float *dldp, int64_t M, int accumulate, void *stream);

/* The optimisation setting's other kernels (Sec. 3.2; supplementary Sec. B).
 * All pointers are device pointers, all work is queued on `stream`.
 *
 * Bi-directional L2 Chamfer distance between points a (na x 3) sampled on the
 * mesh and the input cloud b (nb x 3):
 *   loss = mean_a min_b |a - b|^2 + mean_b min_a |a - b|^2
 * (nearest neighbours by brute force, ties to the lowest index), written to
 * *loss (one double), and its gradient with respect to a into grad_a
 * (na x 3, overwritten; float atomics). ws_idx: na + nb ints, ws_d2: na + nb
 * floats of caller-owned scratch. */
DPSR_API int dpsr_chamfer(const float *a, int64_t na, const float *b, int64_t nb, int *ws_idx, float *ws_d2,
                          float *grad_a, double *loss, void *stream);

/* The largest component of the inside region {chi < level} of the periodic
 * grid (voxels joined along the edges of the extraction's tetrahedra: x, y, z
 * and the monotone diagonals), for the resampling step: the surface of that
 * component is the mesh's largest component, without small detached pieces.
 * labels: r^3 ints (out), the component's representative voxel for inside
 * voxels, -1 outside; ws: r^3 ints of scratch; *best (one uint64, out):
 * (voxel count << 32) | (0xffffffff - representative) of the largest
 * component (0: no inside voxel); *err (one unsigned, out) nonzero if a
 * bounded union-find loop ran out (not expected). */
DPSR_API int dpsr_largest_region(const float *chi, int r, float level, int *labels, int *ws,
                                 unsigned long long *best, unsigned *err, void *stream);

/* dpsr_mesh_extract restricted to the component `keep` of labels (the
 * tetrahedra whose inside corners belong to it). */
DPSR_API int dpsr_mesh_extract_region(const float *chi, int r, float level, const int *labels, int keep,
                                      float *tris, float *normals, int64_t max_tris,
                                      unsigned long long *count, void *stream);

/* M points drawn uniformly by area on a triangle soup (tris T x 3 x 3 with
 * normals T x 3, as from dpsr_mesh_extract), each with its triangle's
 * normal: points, pnormals (M x 3, out). The draws come from a counter-based
 * generator (SplitMix64's finaliser of seed and index), so the same seed
 * gives the same points. ws: T + ceil(T / 1024) + 1 doubles of scratch. */
DPSR_API int dpsr_mesh_sample(const float *tris, const float *normals, int64_t T, int64_t M,
                              uint64_t seed, double *ws, float *points, float *pnormals, void *stream);

/* Per-kernel timing. With profiling on, every kernel launch of the plan is
 * bracketed by CUDA events on the plan's stream (a small overhead per launch).
 * dpsr_plan_profile_read synchronises, then returns, per kernel kind (the
 * DPSR_K_* indices below), the summed device milliseconds and the number of
 * launches since profiling was switched on or last read, and resets both.
 * ms and launches must hold DPSR_K_COUNT entries. */
enum {
    DPSR_K_BIN = 0,         /* bucketing of the points (2 small kernels) */
    DPSR_K_PLANE_FWD = 1,   /* splat + R2C(z) + FFT(y), one cluster per x-plane */
    DPSR_K_XPASS_FWD = 2,   /* FFT(x) + spectral solve (Eq. 3) + IFFT(x) */
    DPSR_K_FINAL_FWD = 3,   /* scalars of Eq. 4 */
    DPSR_K_PLANE_INV = 4,   /* IFFT(y) + C2R(z) + normalisation (Eq. 4) */
    DPSR_K_PLANE_BFWD = 5,  /* backward: R2C(z) + FFT(y) of dchi */
    DPSR_K_FINAL_BWD = 6,   /* backward scalars */
    DPSR_K_XPASS_BWD = 7,   /* backward: adjoint spectral solve along x */
    DPSR_K_PLANE_BINV = 8,  /* backward: IFFT(y) + C2R(z) + point adjoint */
    DPSR_K_COMBINE = 9,     /* backward: per-point combine */
    DPSR_K_COUNT = 10
};
DPSR_API int dpsr_plan_profile(dpsr_plan plan, int enable);

/* Plane paths the plan currently uses for its four plane kinds, in the
 * order forward, forward inverse, backward, backward inverse: 0 = two pencil
 * passes of independent CTAs, 1, 2, 4 or 8 = the cluster size (CTAs per
 * x-plane), 3 = the backward inverse as three independent CTAs per x-plane,
 * one per adjoint channel (r = 64 and 128; backward inverse only). An
 * autotuner sets them on the first solve of each grid size in a process
 * (DPSR_TUNE=0 keeps the static choice). The environment can fix them:
 * DPSR_PLANE_PATHS_<r>="a,b,c,d" for grid size r, or DPSR_PLANE_PATH=c for
 * every kind and size (c in 0, 1, 2, 4, 8). At r = 512 only the pencil
 * passes exist (a plane no longer fits a cluster's shared memory). A path
 * that does not exist for a kind and size makes the solve fail with
 * DPSR_ECUDA. */
DPSR_API int dpsr_plan_clusters(dpsr_plan plan, int *C4);
DPSR_API int dpsr_plan_profile_read(dpsr_plan plan, double *ms, int *launches);

/* Forward pass for callers that cannot allocate device memory (code running
 * where cudaMalloc is forbidden or would block, such as host callbacks,
 * driver-level plugins with a fixed memory budget, or real-time loops that
 * must not enter the allocator). The paper has no counterpart: this is a
 * deployment variant of dpsr_forward. points, normals and chi_out are device
 * pointers as in dpsr_forward (chi_out 16-byte aligned, else DPSR_EINVAL);
 * `stream` is a cudaStream_t (NULL = legacy).
 * All scratch memory is one static device array of about 14 MB that every
 * GPU loading the library holds until exit; the call allocates nothing.
 * Limits: r a power of two with 8 <= r <= 64, 1 <= N <= 65536; anything
 * larger returns DPSR_EINVAL. Every call shares the array and sees what the
 * previous call left there, so calls that overlap on the GPU race: the call
 * waits for its own work and returns the device status (DPSR_OK,
 * DPSR_ETIMEOUT or DPSR_EDEGENERATE, as dpsr_sync). Concurrent calls from
 * several host threads are not supported: they overlap on the GPU and
 * corrupt each other's results, whatever streams they use.
 * The call synchronises its stream and reads the status word back, which a
 * stream capture forbids: it returns DPSR_ESTATE, without launching
 * anything, while its stream is capturing or a capture in global mode is
 * active. The first call in a CUDA context of a device (and again after a
 * device reset) looks up the array's device address. */
DPSR_API int dpsr_forward_static(int r, float sigma, const float *points, const float *normals,
                                 int64_t N, float *chi_out, void *stream);

/* ------------------------------------------------------------------------
 * Batched solves. A batch holds `count` independent solves, instance i with
 * grid size r[i], bandwidth sigma[i] and at most n_max[i] points. Every kernel
 * of the forward / backward sequence runs once per distinct grid size for all
 * instances of that size; dpsr_batch_graph_launch captures the whole
 * sequence into one CUDA graph on first use and then replays it with one
 * launch. Instances are numerically identical to solo dpsr_forward /
 * dpsr_backward calls on the same inputs, up to floating-point rounding.
 * ------------------------------------------------------------------------ */
typedef struct dpsr_batch_s *dpsr_batch;
DPSR_API int dpsr_batch_create(int count, const int *r, const float *sigma, const int64_t *n_max,
                               dpsr_batch *out);
/* The same with a periodic box per instance (as dpsr_plan_create_box):
 * box holds 3 side lengths per instance, count x 3 floats (NULL: every
 * instance on the unit cube), FP64 as for dpsr_plan_create_box. Instances of one grid size still share every
 * launch; each keeps its own spectral tables and coordinate scaling. */
DPSR_API int dpsr_batch_create_box(int count, const int *r, const float *sigma, const double *box,
                                   const int64_t *n_max, dpsr_batch *out);
DPSR_API int dpsr_batch_destroy(dpsr_batch batch);
/* A non-default stream is required for dpsr_batch_graph_launch (capture). */
DPSR_API int dpsr_batch_set_stream(dpsr_batch batch, void *stream);
/* Bind instance i to caller-owned device buffers (layouts as for
 * dpsr_forward / dpsr_backward; dchi, dpoints, dnormals may be NULL for a
 * forward-only batch). N <= n_max[i], else DPSR_ESTATE. Rebinding takes effect
 * at the next forward / backward / graph launch. */
DPSR_API int dpsr_batch_bind(dpsr_batch batch, int i, const float *points, const float *normals,
                             int64_t N, float *chi, const float *dchi, float *dpoints,
                             float *dnormals);
/* Forward (and backward) of every instance, launched on the batch stream. */
DPSR_API int dpsr_batch_forward(dpsr_batch batch);
DPSR_API int dpsr_batch_backward(dpsr_batch batch);
/* Forward, and the backward if with_bwd != 0, as one CUDA graph launch. */
DPSR_API int dpsr_batch_graph_launch(dpsr_batch batch, int with_bwd);
/* Training step of the learning setting (Sec. 3.3, Eq. 9) over the whole
 * batch as one CUDA graph launch: the forward pass of every instance, the
 * L_DPSR loss and gradient of each against its target (as dpsr_mse_grad,
 * written into the instance's bound dchi buffer, which must be writable), and
 * the backward pass into its dpoints / dnormals. Targets are bound per
 * instance with dpsr_batch_bind_target (r^3 float32 device array, 16-byte
 * aligned, caller-owned); dpsr_batch_losses synchronises and writes the
 * `count` losses to out. DPSR_EINVAL if an instance lacks a target or a
 * gradient buffer. */
DPSR_API int dpsr_batch_bind_target(dpsr_batch batch, int i, const float *target);
DPSR_API int dpsr_batch_train_step(dpsr_batch batch);
DPSR_API int dpsr_batch_losses(dpsr_batch batch, double *out);
/* Wait; return the worst device status over the instances (and clear them). */
DPSR_API int dpsr_batch_sync(dpsr_batch batch);
/* Kernel launches in one forward (+ backward) of the batch. */
DPSR_API int dpsr_batch_launches(dpsr_batch batch, int with_bwd);
/* Plane paths of the batch's instances of grid size r, in the order of
 * dpsr_plan_clusters (0 = pencil passes, 3 = the backward inverse split by
 * channel, else the cluster size). A batch
 * tunes them on its first eager run (dpsr_batch_forward / _backward, or the
 * first dpsr_batch_graph_launch, which runs the sequence once before it
 * captures it): each plane kind of each grid size is timed over every path on
 * the batch's own instances and the fastest kept. DPSR_EINVAL if the batch
 * has no instance of size r. */
DPSR_API int dpsr_batch_paths(dpsr_batch batch, int r, int *C4);

/* ------------------------------------------------------------------------
 * Serving. A server runs submitted solves concurrently on `slots` CUDA
 * streams, admitting each request when a slot is free and its device bytes
 * (plan workspace + staging) fit `hbm_budget_bytes` next to the requests in
 * flight (FIFO; a request larger than the whole budget fails with
 * DPSR_EBUSY). Plans are pooled per grid size and stay on the device between
 * requests. All buffers of a request are HOST buffers owned by the caller
 * until the ticket completes; page-locked buffers let the copies overlap
 * with other requests' kernels. dchi = NULL asks for the forward pass only.
 * A worker thread inside the server makes every CUDA call. Results equal a
 * solo dpsr_forward_host / dpsr_backward_host of the same request up to
 * floating-point rounding.
 * ------------------------------------------------------------------------ */
typedef struct dpsr_server_s *dpsr_server;
DPSR_API int dpsr_server_create(size_t hbm_budget_bytes, int slots, float sigma,
                                dpsr_server *out);
DPSR_API int dpsr_server_destroy(dpsr_server server);
DPSR_API int dpsr_server_submit(dpsr_server server, int r, const float *points,
                                const float *normals, int64_t N, const float *dchi,
                                float *chi_out, float *dpoints, float *dnormals,
                                int64_t *ticket);
/* *done = 1 once the results are in the host buffers; the return value is
 * then the request's status and the ticket is retired. */
DPSR_API int dpsr_server_poll(dpsr_server server, int64_t ticket, int *done);
/* Block until the ticket completes (or timeout_s passes: DPSR_ETIMEOUT). */
DPSR_API int dpsr_server_wait(dpsr_server server, int64_t ticket, double timeout_s);
/* Block until at least one request has completed (or timeout_s passes:
 * DPSR_ETIMEOUT, *count = 0), then retire up to `max` completed requests in
 * completion order: their tickets and statuses go to tickets[i] and
 * statuses[i], i < *count. Tickets already retired by poll or wait are
 * skipped. One call replaces a poll of every outstanding ticket: a client
 * with many requests in flight retires them without holding the server's
 * lock once per ticket. Errors: DPSR_EINVAL (NULL or max < 1). */
DPSR_API int dpsr_server_wait_any(dpsr_server server, int64_t *tickets, int *statuses, int max,
                                  double timeout_s, int *count);
/* Cancel a request that is still queued: it is taken out of the queue, no
 * work for it reaches the GPU, its output buffers are not written, and its
 * poll/wait returns DPSR_ECANCELED (which retires the ticket). Returns
 * DPSR_OK when cancelled; DPSR_EBUSY when the request was already admitted
 * or has completed (it then finishes normally and its poll/wait returns its
 * own status); DPSR_EINVAL for an unknown or retired ticket. */
DPSR_API int dpsr_server_cancel(dpsr_server server, int64_t ticket);
/* Coalescing: requests of grid size up to 128 that wait in the queue with
 * the same grid size and mode (forward only / forward + backward) are
 * admitted together, up to max_group of them (1..8, default 8), and run as
 * one batched launch per kernel on one slot, each result equal to its solo
 * solve up to floating-point rounding. Grid size 256 always runs solo.
 * max_group = 1 turns coalescing off (a server of one slot is then the
 * per-solve loop). */
DPSR_API int dpsr_server_set_max_group(dpsr_server server, int max_group);
/* out2 = {coalesced launches so far, requests they ran}. */
DPSR_API int dpsr_server_group_stats(dpsr_server server, int64_t *out2);
/* out4 = {admitted, completed, most slots busy at once, bytes in use}. */
DPSR_API int dpsr_server_stats(dpsr_server server, int64_t *out4);

/* Static description of an error code. */
DPSR_API const char *dpsr_strerror(int status);

/* Failure-detection check of the device side: launches one kernel whose
 * bounded wait (the same wait every TMA and DSMEM barrier of the library
 * uses) is on a barrier that nothing ever completes; the wait must give up
 * after limit_s seconds (0 < limit_s <= 10) and report it in a device status
 * word, leaving the GPU and the context usable. Synchronous. Returns
 * DPSR_ETIMEOUT when the wait ran out as designed, DPSR_OK if it did not
 * (a defect), DPSR_EINVAL or DPSR_ECUDA on errors. */
DPSR_API int dpsr_check_bounded_wait(double limit_s);

/* Stage read-back for tests (Sec. 3.1 / Eq. A3, Eq. 3): copies one of the
 * forward pass's intermediate spectra to the host buffer out_host, which
 * receives r * r * (r/2 + 1) complex64 values laid out [x][ky][kz] (kz =
 * 0 .. r/2, the z half spectrum; x a grid coordinate, not transformed):
 *   which = 0: D = i u_y FFT_yz(V_y) + i u_z FFT_yz(V_z) (u in integer
 *              cycles, zero at a Nyquist index);
 *   which = 1: C = FFT_yz(V_x);
 *   which = 2: W~ = FFT_yz(w), w the splat of ones (the weights of Eq. 4);
 *   which = 3: r * FFT_yz(chi'), the unnormalised x-inverse of chi~;
 * after dpsr_backward, the adjoint spectrum of Eq. 3 (G_bar of Eq. 4's
 * adjoint, F = G(k) FFT3(G_bar) / r^3 with G(k) = g(k) / (-2 pi |u|^2)):
 *   which = 4: Q1 = the unnormalised x-inverse of F;
 *   which = 5: Q2 = the unnormalised x-inverse of -i u_x F.
 * FFT_yz: unnormalised DFT over y (length r) and the z half spectrum. 0..3
 * are valid after dpsr_forward until the next dpsr_backward, 4..5 after
 * dpsr_backward until the next dpsr_forward (DPSR_ESTATE otherwise).
 * Synchronises the plan's stream. Errors: DPSR_EINVAL (which outside 0..5,
 * NULL), DPSR_ECUDA. */
DPSR_API int dpsr_debug_read_spectrum(dpsr_plan plan, int which, void *out_host);

/* Debug builds. A library compiled with DPSR_DEBUG_CHECKS (the build
 * script's debug variant; the Python binding loads it when the environment
 * sets DPSR_DEBUG_CHECKS=1) checks every data-dependent index of the point
 * kernels (bin keys, sorted positions, point indices read from the bins)
 * before use: an index out of range skips its access and sets a status bit
 * that dpsr_sync reports as DPSR_EBOUNDS. No check traps or aborts.
 * dpsr_debug_checks returns 1 in such a build, 0 otherwise.
 * dpsr_debug_check_selftest runs one kernel whose single access has an index
 * outside its logical range but inside its allocation: DPSR_EBOUNDS in a
 * debug build, DPSR_OK otherwise (DPSR_ECUDA if CUDA fails). It synchronises
 * the device. */
DPSR_API int dpsr_debug_checks(void);
DPSR_API int dpsr_debug_check_selftest(void);

/* Measurement utility (not part of the method): the FP32 FMA throughput of
 * the current device in FLOP/s (2 per FMA), timed with events over a kernel
 * of `iters` steps of 8 independent FMA chains per thread, 8 CTAs of 256
 * threads per SM, fastest of three runs. Blocks the calling thread; uses
 * its own stream and a small device buffer that it frees. Errors:
 * DPSR_EINVAL (iters < 1 or NULL), DPSR_ECUDA. */
DPSR_API int dpsr_fp32_fma_peak(int iters, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* DPSR_H */
