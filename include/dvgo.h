/*
 * dvgo.h -- C ABI of the GB300 (sm_103a) implementation of the Direct Voxel Grid Optimization
 * render step: differentiable volume rendering of ray batches through a post-activated density
 * voxel grid and a colour grid (coarse stage) or a feature grid with a shallow colour MLP (fine
 * stage), forward, backward and Adam.
 *
 * Paper: C. Sun, M. Sun, H.-T. Chen, "Direct Voxel Grid Optimization: Super-fast Convergence for
 * Radiance Fields Reconstruction", arXiv 2111.11215.  Citations below name its sections and
 * equations.
 *
 * Conventions
 *   - Every pointer argument named *_out, grad_*, or a grid / ray / weight array is a DEVICE
 *     pointer; the structs themselves (dvgo_params, dvgo_grid_desc, dvgo_mlp, dvgo_samples) are
 *     read on the host during the call and may be freed when it returns.
 *   - The caller owns all device memory and the stream.  Apart from the one entry point that
 *     says otherwise, the library never allocates: scratch space is a caller-supplied workspace
 *     of dvgo_workspace_size() bytes (256-byte aligned).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.  Every call
 *     only enqueues work on that stream and returns; nothing synchronises.
 *   - Gradients are ACCUMULATED (+=); clear them first (dvgo_adam_step can clear them).
 *   - Return value: DVGO_OK or a negative dvgo_status.  Argument errors are detected on the host
 *     before anything is enqueued.  Conditions only visible on the device (a ray with a zero or
 *     non-finite direction) make that ray sample-free and set a flag in the workspace that
 *     dvgo_workspace_status() reads back.
 *   - Grids are channel-last on an align-corners lattice: value (ix, iy, iz, ch) of an
 *     nx*ny*nz*C grid is at ((ix*ny + iy)*nz + iz)*C + ch; lattice point (ix, iy, iz) sits at
 *     xyz_min + (ix, iy, iz) * (xyz_max - xyz_min) / (n - 1)   (Sec. 3 Eq. interp).
 *     The render calls read the colour / feature grid with 16-byte loads: its pointer must be
 *     16-byte aligned (DVGO_ERR_INVALID_ARG otherwise).
 */
#ifndef DVGO_H
#define DVGO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DVGO_ABI_VERSION 10

/* Grid memory layouts (dvgo_grid_desc.layout).
 *   CANONICAL: channel-last [nx][ny][nz][C], nx*ny*nz*C elements.
 *   PACKED:    4x4x4-point bricks in row-major brick order (ceil(n/4) bricks per axis) with the
 *              64 points of a brick in Morton order (bits i0 j0 k0 in the low three, i1 j1 k1
 *              above), channel-last inside a point: ceil(nx/4)*ceil(ny/4)*ceil(nz/4)*64*C
 *              elements, padding points included (they stay 0 under training: they get no
 *              gradient).  The eight corners of a cell share a brick unless the cell straddles
 *              one, and are eight consecutive points when the cell's base indices are even.
 *              At most 2048 x 2048 x 1024 points. */
#define DVGO_LAYOUT_CANONICAL 0
#define DVGO_LAYOUT_PACKED 1

/* Interpolation / activation order of the density (dvgo_params.act_order). */
#define DVGO_ACT_POST 0
#define DVGO_ACT_PRE 1
#define DVGO_ACT_IN 2

typedef enum {
    DVGO_OK = 0,
    DVGO_ERR_INVALID_ARG = -1,   /* null pointer, bad size, inconsistent descriptors          */
    DVGO_ERR_WORKSPACE = -2,     /* workspace NULL, misaligned or smaller than required       */
    DVGO_ERR_UNSUPPORTED = -3,   /* a combination this build does not implement               */
    DVGO_ERR_CUDA = -4,          /* a kernel launch failed (cudaGetLastError)                 */
    DVGO_ERR_DEVICE = -5,        /* device-side flag: a ray had a zero / non-finite direction,
                                    or a tensor-core kernel's bounded wait ran out              */
    DVGO_ERR_CAPACITY = -6       /* batch larger than the static scratch of dvgo_render_fwd_noalloc */
} dvgo_status;

enum { DVGO_DTYPE_F32 = 0, DVGO_DTYPE_BF16 = 1 };
enum { DVGO_MODE_COARSE = 0, DVGO_MODE_FINE = 1 };
enum { DVGO_MLP_FP32 = 0, DVGO_MLP_BF16 = 1 };

/* A voxel grid (Sec. 3 Eq. interp): values on an align-corners lattice spanning the box. */
typedef struct {
    int nx, ny, nz;      /* lattice points per axis, each >= 2                                 */
    int channels;        /* 1 (density), 3 (coarse colour), D (fine features, D <= 16)         */
    float xyz_min[3];    /* box corners; the density and colour grids must share the box        */
    float xyz_max[3];
    int dtype;           /* DVGO_DTYPE_F32, or DVGO_DTYPE_BF16 for the fine feature grid only   */
    int layout;          /* DVGO_LAYOUT_CANONICAL or DVGO_LAYOUT_PACKED; a render's density and
                            colour / feature grids share one layout                            */
} dvgo_grid_desc;

/* Number of scalar elements of a grid's storage in its layout (padding points included). */
size_t dvgo_grid_elements(const dvgo_grid_desc *g);

/* Copies a grid into another layout and / or element type on the same lattice (nx, ny, nz,
 * channels and box equal): FP32 <-> BF16 (round to nearest even), canonical <-> packed; padding
 * points of a packed output are set to 0.  in / out are device buffers of dvgo_grid_elements()
 * elements of their descriptors; they must not overlap. */
int dvgo_pack_grid(const dvgo_grid_desc *src, const void *in, const dvgo_grid_desc *dst, void *out, void *stream);

/* Image-fitting toy of Sec. 3 (Fig. exdv_poc): a binary image regressed by a low-resolution 2D grid
 * queried with bilinear interpolation under the pre-, in- or post-activation order of
 * Eq. pre_in_post.  The image covers [0, 1]^2, pixel (i, j) (row i) at ((i + 0.5) / height,
 * (j + 0.5) / width); the grid's grid_h x grid_w points sit on the align-corners lattice of
 * [0, 1]^2; the predicted pixel is alpha = 1 - exp(-sigma delta) with sigma from
 * softplus(v + shift_b) in the given order; the loss is the mean squared error over all pixels. */
typedef struct {
    int height, width;   /* target image, row-major [height][width]                              */
    int grid_h, grid_w;  /* lattice points of the 2D grid (row-major [grid_h][grid_w]), each >= 2  */
    int act_order;       /* DVGO_ACT_POST / DVGO_ACT_PRE / DVGO_ACT_IN                             */
    float shift_b;       /* b of Eq. density_activation                                           */
    float delta;         /* the alpha function's step                                             */
} dvgo_fit2d_desc;

/* One evaluation of the toy on device buffers: image_out [height*width] gets the predicted image
 * (nullable); with a target [height*width], loss_out[0] is set to the mean squared error and
 * grad_grid [grid_h*grid_w] accumulates (+=) its gradient (each nullable).  Pixel cells and
 * fractions come from exact integer arithmetic; the activations run in FP32.  Stream-ordered. */
int dvgo_fit2d(const dvgo_fit2d_desc *d, const float *grid, const float *target, float *image_out, float *grad_grid,
               float *loss_out, void *stream);

/* Progressive scaling (Sec. 4.2): resizes a grid by trilinear interpolation onto another lattice.
 * Point (i, j, k) of the destination sits at x = dst.xyz_min + (i, j, k) (dst.xyz_max -
 * dst.xyz_min) / (n - 1) and takes interp(x, V_src) (Sec. 3 Eq. interp) of the source grid, x
 * first clamped into the source box; positions and weights are formed in FP64, the result is
 * rounded once to FP32.  Both grids FP32 with the same channel count, either layout each (padding
 * points of a packed destination are set to 0); in / out are device buffers of
 * dvgo_grid_elements() elements of their descriptors and must not overlap.  Stream-ordered. */
int dvgo_resize_grid(const dvgo_grid_desc *src, const float *in, const dvgo_grid_desc *dst, float *out,
                     void *stream);

/*
 * Known free space of the fine stage (Sec. 4.2, "Known free space and unknown space" and "Free
 * space skipping"): the optimised coarse-stage density grid with its own lattice and box
 * (desc.channels = 1, FP32), the coarse stage's shift b_c and step delta_c.  A fine-stage query
 * point x is skipped -- alpha := 0, no fine density or colour query, no gradient -- when
 *     alpha_c(x) = 1 - exp(-softplus(interp(x, V_c) + b_c) delta_c) < tau,
 * evaluated in FP32 (trilinear interpolation with the same edge clamping as the fine grid).
 * The struct is read on the host during the call; density is a device pointer.
 */
typedef struct {
    dvgo_grid_desc desc;
    const float *density;    /* [nx*ny*nz] FP32; NULL disables the test                          */
    float shift_b;           /* b_c                                                              */
    float step;              /* delta_c, world units                                             */
    float tau;               /* tau_c (Supp. A: 1e-3)                                            */
} dvgo_freespace;

/* Render parameters. */
typedef struct {
    int mode;            /* DVGO_MODE_COARSE: colour = interp(x, V_rgb) (Sec. 4.1 Eq. coarse_queries)
                            DVGO_MODE_FINE: colour = MLP(interp(x, V_feat), PE(d))
                            (Sec. 4.2 Eq. fine_queries)                                          */
    int rgb_act;         /* coarse: 0 = identity (the paper states no activation), 1 = sigmoid   */
    int mlp_prec;        /* fine: DVGO_MLP_FP32 (SIMT FP32) or DVGO_MLP_BF16 (tensor cores,
                            BF16 operands, FP32 accumulation)                                    */
    int n_freq_dir;      /* fine: positional-encoding frequencies on d (Supp. A: k_d = 4)        */
    int hidden;          /* fine: MLP width; this build supports 128 (Supp. A)                   */
    float step;          /* delta, the sampling step in world units (Supp. A: 0.5 voxel)         */
    float shift_b;       /* b of Eq. density_activation, e.g. from Eq. low_density_init          */
    float tau_f;         /* samples with alpha < tau_f are removed (Sec. 4.2 free space skipping) */
    float t_near, t_far; /* ray clip range before the box intersection                           */
    float bg[3];         /* c_bg of Eq. volume_rendering                                          */
    const dvgo_freespace *freespace;   /* fine stage only, nullable: skip the known free space   */
    /* Auxiliary losses of Supp. A, added when dvgo_render_fwd gets a target (0 disables):
     *   w_pt_rgb: per-point rgb loss L_pt = (1/R) sum_r sum_k w_k ||c_k - C_r||^2 with the
     *             compositing weights w_k held constant (the loss supervises each point's colour);
     *   w_bg:     background entropy L_bg = (1/R) sum_r H(A_r), H the natural-log binary entropy of
     *             the accumulated alpha A = 1 - T_K clamped to [1e-6, 1 - 1e-6].
     * Supp. A: 1e-1 / 1e-2 in the coarse stage, 1e-2 / 1e-3 in the fine stage.                 */
    float w_pt_rgb, w_bg;
    int act_order;       /* Sec. 3 Eq. pre_in_post: DVGO_ACT_POST (the paper's choice),
                            DVGO_ACT_PRE  alpha = interp(x, alpha(softplus(V + b))),
                            DVGO_ACT_IN   alpha = alpha(interp(x, softplus(V + b)))              */
    int n_freq_pos;      /* fine: positional-encoding frequencies on the query point x (Sec. 4.2
                            Eq. fine_queries_rgb, Supp. A: k_x = 5); 0 leaves x out of the MLP
                            input.  This build supports 0 and 5.                                 */
    /* Failure detection of the tensor-core colour kernels (DVGO_MLP_BF16; not part of the method).
     * Every device-side wait of those kernels (an mbarrier phase: the producers' tile, the
     * consumers' release of a buffer, the completion of an MMA batch) gives up after
     * wait_limit_us microseconds (0: the default, 2 s); the kernel then stops its CTA's work, waits
     * (bounded) for MMAs it issued, releases its tensor memory, sets bit 1 of the workspace flag
     * word (dvgo_workspace_status then returns DVGO_ERR_DEVICE until the next forward) and returns;
     * the gradients or colours of that call are incomplete.  Range 0 .. 60,000,000.
     * test_withhold_tile (testing aid, 0 in normal use): k > 0 makes one producer thread of the
     * colour kernels withhold its arrival on tile k - 1, so that the consumers' wait for that tile
     * runs out -- the failure path above, taken on purpose. */
    int wait_limit_us;
    int test_withhold_tile;
    /* cgrid_ready: NULL, or a cudaEvent_t (of the calling device) that dvgo_render_fwd and
     * dvgo_render_bwd make their stream wait on right before their first kernel that reads the
     * colour / feature grid -- for a producer of that grid on another stream (an optimiser step):
     * the ray set-up, the sample scan and the density pass before it are not held back.  Not
     * validated; an event that was never recorded is complete.  Other calls ignore it. */
    void *cgrid_ready;
    /* forward_only: non-zero when no dvgo_render_bwd follows the forward (test-time rendering).
     * The forward then keeps nothing for a backward -- with DVGO_MLP_BF16 in the fine stage, the
     * colour kernels' input panels (16 KiB per 128 samples) -- and dvgo_workspace_size leaves that
     * block out.  A backward on such a workspace gathers its inputs again (same results). */
    int forward_only;
    /* density_ready: NULL, or a cudaEvent_t (of the calling device) that dvgo_render_fwd and
     * dvgo_render_bwd make their stream wait on right before their first kernel that reads the
     * density grid -- for a producer of that grid on another stream: the ray set-up and the sample
     * scan before it are not held back.  Not validated; an event that was never recorded is
     * complete.  Other calls ignore it. */
    void *density_ready;
} dvgo_params;

/* Colour MLP (fine stage), FP32 row-major [in][out]:
 *   in = C + 3 + 6*n_freq_dir (+ 3 + 6*n_freq_pos)  ->  hidden  ->  hidden  ->  3
 *   input row e = [interp(x, V_feat) (C), d (3), sin(2^k d_c) (c-major, k < n_freq_dir),
 *                  cos(2^k d_c) (c-major)] and, with n_freq_pos > 0, the same encoding of the
 *                  world-space query point x appended: [x (3), sin(2^k x_c), cos(2^k x_c)];
 *   ReLU after the hidden layers, sigmoid on the output (Sec. 2 Eq. nerf_mlp output activation,
 *   Sec. 4.2 Eq. fine_queries_rgb, Supp. A: C = 12, k_d = 4, k_x = 5, in = 72). */
typedef struct {
    const float *w1, *b1, *w2, *b2, *w3, *b3;
} dvgo_mlp;

/* Optional explicit samples (the proposal path): ray r uses n_per_ray samples at distances
 * t[r*n_per_ray + j] along its normalised direction with step lengths dt[...]; a ray that
 * misses the box gets none.  NULL selects uniform stepping t_k = t_enter + (k + p) * step. */
typedef struct {
    const float *t;
    const float *dt;
    int n_per_ray;
} dvgo_samples;

/* Bytes of workspace that dvgo_render_fwd / dvgo_render_bwd need for n_rays rays.  The bound
 * covers the longest possible ray: ceil(|xyz_max - xyz_min| / step) + 1 samples.  The fine stage
 * with DVGO_MLP_BF16 adds 16 KiB per 128 samples unless p->forward_only: the tensor-core forward
 * keeps every tile's BF16 MLP input rows there for the backward. */
size_t dvgo_workspace_size(const dvgo_params *p, const dvgo_grid_desc *density, int n_rays,
                           const dvgo_samples *explicit_samples);

/*
 * Forward render of n_rays rays (Sec. 2 Eq. volume_rendering with the post-activated density
 * of Sec. 3 Eq. post_activation and the queries of Sec. 4.1 / 4.2):
 *   1. normalise d and clip the ray to the box and [t_near, t_far] (Sec. 4.2 fine-stage sampling);
 *   2. sample t_k = t_enter + (k + p) step, k = 0.. while t_k < t_exit (Eq. coarse_sample and the
 *      jitter p of Supp. A), or use the explicit samples;
 *   3. sigma_k = softplus(interp(x_k, V_density) + b), alpha_k = 1 - exp(-sigma_k dt_k)
 *      (Eq. density_activation, Eq. density_2_alpha), dropped when alpha_k < tau_f;
 *   4. colour c_k from the colour grid (coarse) or the feature grid and the MLP (fine);
 *   5. C_hat = sum_k T_k alpha_k c_k + T_K bg, T_k = prod_{j<k} (1 - alpha_j).
 * Inputs: density [nx*ny*nz] FP32; cgrid [nx*ny*nz*C] (FP32, or BF16 for fine features);
 *   rays_o, rays_d [n_rays*3] FP32; jitter [n_rays] in [0,1) or NULL (p = 0.5);
 *   target [n_rays*3] or NULL.
 * Outputs: rgb_out [n_rays*3]; tfinal_out [n_rays] (T_K) or NULL; if target is given,
 *   loss_out[0] = (1/R) sum_r ||C_hat_r - C_r||^2 (Eq. photo_loss) + w_pt_rgb L_pt + w_bg L_bg and
 *   dloss_drgb_out [n_rays*3] = 2 (C_hat - C) / R (the photometric part), each nullable; with
 *   non-zero auxiliary weights the workspace keeps the targets for dvgo_render_bwd.
 * The workspace keeps the per-ray and per-sample state that dvgo_render_bwd consumes; it must
 * not be modified between the two calls, which must see the same inputs.
 */
int dvgo_render_fwd(const dvgo_params *p, const dvgo_grid_desc *density_desc, const float *density,
                    const dvgo_grid_desc *cgrid_desc, const void *cgrid, const dvgo_mlp *mlp,
                    int n_rays, const float *rays_o, const float *rays_d, const float *jitter,
                    const dvgo_samples *explicit_samples, const float *target, float *rgb_out,
                    float *tfinal_out, float *loss_out, float *dloss_drgb_out, void *workspace,
                    size_t workspace_bytes, void *stream);

/*
 * Backward of dvgo_render_fwd: accumulates into the gradients the derivative of
 *     sum_r ( grad_rgb_r . C_hat_r + grad_tfinal_r * T_K,r ),
 * plus that of w_pt_rgb L_pt + w_bg L_bg when the forward had a target and non-zero weights
 * with respect to the density grid, the colour / feature grid and the MLP parameters.
 * Compositing state (T_k, the weights and the suffix colour sums) is recomputed from the
 * per-sample values the forward left in the workspace (optical depths and colours); the MLP's
 * activations are recomputed (the BF16 tensor-core backward takes the output colour and the
 * interpolated, encoded MLP input rows from the forward instead of recomputing the last layer
 * and gathering the features again).
 * grad_rgb [n_rays*3] (required), grad_tfinal [n_rays] or NULL.
 * grad_density [nx*ny*nz] FP32; grad_cgrid [nx*ny*nz*C] FP32 (also for a BF16 feature grid);
 * grad_mlp (fine only) FP32, packed w1 | b1 | w2 | b2 | w3 | b3 in the dvgo_mlp layouts.
 */
int dvgo_render_bwd(const dvgo_params *p, const dvgo_grid_desc *density_desc, const float *density,
                    const dvgo_grid_desc *cgrid_desc, const void *cgrid, const dvgo_mlp *mlp,
                    int n_rays, const float *rays_o, const float *rays_d, const float *jitter,
                    const dvgo_samples *explicit_samples, const float *grad_rgb,
                    const float *grad_tfinal, float *grad_density, float *grad_cgrid,
                    float *grad_mlp, void *workspace, size_t workspace_bytes, void *stream);

/* Adam hyper-parameters (Kingma & Ba; Sec. 5.2 / Supp. A use Adam with base rates 0.1 for the
 * grids and 1e-3 for the MLP, decayed by 0.1 over 20k steps). */
typedef struct {
    float lr;            /* already-decayed learning rate for this step                        */
    float beta1, beta2, eps;
    int step;            /* 1-based step count t (bias correction 1 - beta^t)                  */
    int skip_zero_grad;  /* 1: lazy variant -- an element whose gradient is exactly 0 keeps its
                            parameter and moments (reads 4 B instead of 32 B there); this
                            library's option, the paper's Adam is dense (0)                     */
} dvgo_adam_hparams;

/*
 * One Adam step on n FP32 parameters:  m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 *   p -= lr * s_i * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 * with s_i = lr_scale[i] (nullable; the per-voxel rate of Sec. 4.1 Prior 2) or 1.
 * param_bf16_out (nullable): also writes the updated parameters rounded to BF16 (the storage
 * copy of a BF16 feature grid).  zero_grad != 0 clears grad after reading it.
 * All arrays are device pointers of n elements, 16-byte aligned.
 */
int dvgo_adam_step(float *param, float *grad, float *m, float *v, size_t n,
                   const dvgo_adam_hparams *h, const float *lr_scale, uint16_t *param_bf16_out,
                   int zero_grad, void *stream);

/* One tensor of dvgo_adam_step_multi: the arguments of dvgo_adam_step. */
typedef struct {
    float *param, *grad, *m, *v;   /* device, n elements each, 16-byte aligned                     */
    size_t n;
    dvgo_adam_hparams h;           /* this tensor's rate, betas, eps, step count, lazy flag          */
    const float *lr_scale;         /* nullable, as in dvgo_adam_step                                 */
    uint16_t *param_bf16_out;      /* nullable, 8-byte aligned, as in dvgo_adam_step                 */
    int zero_grad;
} dvgo_adam_tensor;

#define DVGO_ADAM_MAX_TENSORS 4

/*
 * The Adam step of dvgo_adam_step on each of n_tensors (0 .. DVGO_ADAM_MAX_TENSORS) tensors, with
 * their own hyper-parameters, in one launch (every element gets exactly the arithmetic of
 * dvgo_adam_step: the results are the same bits).  For the small tensors a training step updates
 * last, whose separate launches would each cost a launch's latency.  The tensors must not overlap.
 * Every tensor is checked as dvgo_adam_step checks it before anything is enqueued
 * (DVGO_ERR_INVALID_ARG).
 */
int dvgo_adam_step_multi(const dvgo_adam_tensor *tensors, int n_tensors, void *stream);

/* Pinhole training views for the view counts below: image size, intrinsics and near distance
 * shared by all views. */
typedef struct {
    int n_views;             /* V >= 0                                                           */
    int height, width;       /* image size in pixels, each >= 1; rows run downward                */
    double fx, fy;           /* focal lengths in pixels, > 0                                      */
    double cx, cy;           /* principal point in pixels (finite)                                */
    double near;             /* a point must lie further than this (>= 0) along the viewing axis  */
} dvgo_view_rig;

/*
 * Sec. 4.1 Prior 2 (view-count-based learning rate): for every point j of the lattice of g
 * (channels 1, FP32), the number n_j of views that see it, and the scale n_j / n_max of its base
 * learning rate (n_max = max_j n_j), for lr_scale of dvgo_adam_step on that grid.
 *   c2w      device, [n_views][3][4] FP64 row-major camera-to-world matrices [R | c], finite:
 *            columns R_0, R_1, R_2 are the camera's x (right), y (up) and z (backward) axes in
 *            world space, c its centre; the camera looks along -z (R need not be orthonormal:
 *            q = R^T (x - c) is used as given).
 *   A point x is seen by a view when q = R^T (x - c) has depth -q_z > near and projects into the
 *   closed image rectangle: 0 <= cx + fx q_x / (-q_z) <= width, 0 <= cy - fy q_y / (-q_z) <= height.
 *   Occlusion is not considered.  The decision equals that of the FP64 arithmetic written in that
 *   order, each operation correctly rounded, the lattice point at xyz_min + i (xyz_max - xyz_min) /
 *   (n - 1) (FP32 box corners taken exactly).
 *   counts   device uint32 [dvgo_grid_elements(g)], overwritten in g's storage layout (packed
 *            padding: 0).
 *   lr_scale device float [dvgo_grid_elements(g)], nullable: counts / n_max correctly rounded, or 1
 *            everywhere when no point is seen (n_max = 0).
 *   n_max    device uint32 [1], overwritten with n_max.
 * Device pointers 4-byte aligned (c2w 8-byte).  Stream-ordered; returns DVGO_ERR_INVALID_ARG on a
 * bad descriptor, rig or pointer before launching anything.
 */
int dvgo_view_counts(const dvgo_grid_desc *g, const dvgo_view_rig *rig, const double *c2w, uint32_t *counts,
                     float *lr_scale, uint32_t *n_max, void *stream);

/* Learning rate of Supp. A at 0-based step t: lr0 * 0.1^(t / decay_steps). */
float dvgo_lr_at(float lr0, int step, float decay_steps);

/* Reads (synchronously, on `stream`) the device-side flag word of the workspace: returns DVGO_OK,
 * or DVGO_ERR_DEVICE when a ray of the last forward had a zero or non-finite direction (bit 0) or
 * a tensor-core colour kernel of the last forward or backward gave up a wait (bit 1, see
 * dvgo_params.wait_limit_us).  Each forward clears the word. */
int dvgo_workspace_status(void *workspace, void *stream);

/* Copies the per-ray sample counts that the last forward computed (step 2 of dvgo_render_fwd)
 * from a workspace into counts_out [n_rays] (device int32), and the batch total into
 * total_out[0] (device, nullable).  n_rays must be the forward's ray count. */
int dvgo_sample_counts(const void *workspace, int n_rays, int *counts_out, int *total_out, void *stream);

/* Lattice points one fine-stage render read (the sizes behind the minimum HBM bytes of a step):
 * bitmaps[0 .. W) marks the density grid's points at the 8 corners of every sample outside the known
 * free space and not removed by early ray termination, bitmaps[W .. 2W) the feature grid's points
 * at the 8 corners of every kept sample
 * (W = ceil(nx*ny*nz / 32) uint32 words, bit p of the canonical index p = (i ny + j) nz + k, whatever
 * the storage layout); counts[0], counts[1] = their populations.  Call after dvgo_render_fwd with the
 * same parameters, grid descriptor, ray count, explicit samples and workspace; bitmaps and counts
 * are device buffers, overwritten.  Fine stage only.  Stream-ordered. */
int dvgo_touched_points(const dvgo_params *p, const dvgo_grid_desc *density, int n_rays,
                        const dvgo_samples *explicit_samples, void *workspace, size_t workspace_bytes,
                        uint32_t *bitmaps, unsigned long long *counts, void *stream);

/*
 * Allocation-free variant of the coarse-stage forward (dvgo_render_fwd with mode
 * DVGO_MODE_COARSE and no MLP or explicit samples), for callers that cannot allocate device
 * memory at all and so cannot provide a workspace: for example a plugin inside a host
 * application whose memory manager owns the whole device, a real-time loop that forbids
 * allocation after start-up, or a language binding with no device allocator.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Scratch memory: instead of a caller workspace it uses one static device array of
 * DVGO_NOALLOC_SCRATCH_BYTES (about 2.6 MB) inside the library, which every GPU that loads the
 * library holds until the process exits.  The caller still passes all inputs and outputs, with the
 * meaning, layout and nullability of dvgo_render_fwd.  The call itself allocates nothing (no
 * cudaMalloc / cudaFree or allocating library routine).
 *   - n_rays may be at most DVGO_NOALLOC_MAX_RAYS; a larger batch returns DVGO_ERR_CAPACITY and
 *     enqueues nothing.  Any mode other than DVGO_MODE_COARSE returns DVGO_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current, and keeps it for the life of the process; make that first call before
 *     any stream capture.  A device reset (cudaDeviceReset) or any other teardown of the device's
 *     primary context unloads the library's device code, after which this entry point must not be
 *     called again in that process.
 *   - Every call, on every stream, shares the one array and overwrites what the previous call left
 *     there.  Calls whose execution overlaps on the GPU (different streams without ordering between
 *     them) race and give undefined results: order them on one stream or with events.
 */
#define DVGO_NOALLOC_MAX_RAYS 16384
#define DVGO_NOALLOC_SCRATCH_BYTES 2621696
int dvgo_render_fwd_noalloc(const dvgo_params *p, const dvgo_grid_desc *density_desc, const float *density,
                            const dvgo_grid_desc *cgrid_desc, const void *cgrid, int n_rays,
                            const float *rays_o, const float *rays_d, const float *jitter,
                            const float *target, float *rgb_out, float *tfinal_out, float *loss_out,
                            float *dloss_drgb_out, void *stream);

/*
 * Fine voxels allocation (Sec. 4.2): the lattice-index box of the coarse grid's cells that can
 * hold unknown space.  A lattice point v is unknown when 1 - exp(-softplus(V_c[v] + b_c) delta_c)
 * >= tau (FP32); interpolation inside a cell is a convex combination of its corners and alpha
 * increases with the raw density, so a cell whose 8 corners are known free is known free
 * everywhere, and the unknown space lies in [min - 1, max + 1] of the unknown lattice points,
 * clamped to [0, n - 1] per axis.  out (device, 7 ints): count of unknown lattice points, then
 * lo[3], hi[3] (undefined when the count is 0).  Three small kernels on `stream`.
 */
int dvgo_unknown_bbox(const dvgo_freespace *fs, int *out, void *stream);

/* ------------------------------------------------------------------------------------------
 * Learned sample proposal.  The paper samples every ray uniformly and leaves hierarchical
 * sampling to future work (Supp. B, step-size ablation); this proposal is the library's
 * addition.  A small MLP predicts, for each ray, a piecewise-constant PDF over n_bins equal bins
 * of the clipped interval [t_enter, t_exit]; it is trained with a softmax cross-entropy on the
 * per-bin compositing weights of a uniform render, and its PDF is sampled by inverse CDF to give
 * the explicit samples (dvgo_samples) of a cheaper render.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int n_bins;          /* bins per ray; this build supports 64                                 */
    int n_freq;          /* PE frequencies on the bin centre x_b; this build supports 6            */
    int width;           /* MLP width; this build supports 64                                     */
    int precision;       /* arithmetic of the forward and the backward: DVGO_MLP_FP32 (SIMT) or
                            DVGO_MLP_BF16 (tcgen05 tensor cores: BF16 operands -- inputs,
                            activations, weights, dlogit and the dZ of each layer -- with FP32
                            accumulation; the encoding and the softmax in FP32)                   */
} dvgo_proposal_desc;

/* Proposal MLP, FP32 row-major [in][out]: in = 3 + 6 n_freq (= 39) -> width -> width -> width -> 1,
 * ReLU after the hidden layers; input row [x, sin(2^k x_c) (c-major), cos(2^k x_c) (c-major)] of the
 * bin centre x_b = o + t_b d, t_b = t_enter + (b + 0.5)(t_exit - t_enter) / n_bins. */
typedef struct {
    const float *w0, *b0, *w1, *b1, *w2, *b2, *w3, *b3;
} dvgo_proposal_mlp;

/* Labels for the proposal: per ray, the compositing weights w_k = T_k alpha_k of a uniform-step
 * fine forward (Eq. volume_rendering) summed into n_bins equal bins of [t_enter, t_exit] and
 * normalised to sum 1 (uniform when their sum is below 1e-4).  `workspace` must hold the state of
 * a dvgo_render_fwd in DVGO_MODE_FINE without explicit samples on the same p, density_desc and
 * n_rays.  labels_out [n_rays * n_bins]; n_bins <= 128. */
int dvgo_weight_bins(const dvgo_params *p, const dvgo_grid_desc *density_desc, int n_rays, int n_bins,
                     const void *workspace, size_t workspace_bytes, float *labels_out, void *stream);

/* Proposal forward: probs_out [n_rays * n_bins] = softmax over the bins of the MLP logits (a ray
 * that misses the box gets the uniform PDF).  With labels [n_rays * n_bins] (nullable),
 * loss_out[0] = -(1/R) sum_r sum_b h_rb log p_rb.  Needs no workspace. */
int dvgo_proposal_fwd(const dvgo_params *p, const dvgo_grid_desc *density_desc, const dvgo_proposal_desc *pd,
                      const dvgo_proposal_mlp *mlp, int n_rays, const float *rays_o, const float *rays_d,
                      const float *labels, float *probs_out, float *loss_out, void *stream);

/* Proposal backward: ACCUMULATES the gradient of the cross-entropy loss above into grad_mlp,
 * packed w0 | b0 | w1 | b1 | w2 | b2 | w3 | b3 (recomputes the forward).  labels is required.
 * With DVGO_MLP_BF16, a tensor-core wait that gives up (~2 s) adds NaN to grad_mlp[0]. */
int dvgo_proposal_bwd(const dvgo_params *p, const dvgo_grid_desc *density_desc, const dvgo_proposal_desc *pd,
                      const dvgo_proposal_mlp *mlp, int n_rays, const float *rays_o, const float *rays_d,
                      const float *labels, float *grad_mlp, void *stream);

/* Inverse-CDF sampling of n_samples sorted samples per ray from probs [n_rays * n_bins]: the PDF
 * is mixed with the uniform one, q_b = (1 - eta) p_b + eta / n_bins; sample j sits at quantile
 * u_j = (j + jit) / n_samples of the CDF (jit = jitter[r], or 0.5 when jitter is NULL) with linear
 * interpolation inside its bin.  t_out, dt_out [n_rays * n_samples]: distances along the
 * normalised direction and step lengths (t_{j+1} - t_j; for the last sample the bin width over
 * n_samples times the bin's normalised probability), ready for dvgo_samples.  Rays that miss the
 * box (FP64 clip, as in the renderer) get zeros.  Precision: the CDF, the quantiles and the sample
 * positions are double-float (two FP32 words, ~48 significant bits), the fraction inside a bin
 * FP32, so t and dt are within about an FP32 ulp of their exact values; a bin choice can differ
 * from the exact one only where a quantile lies within ~1e-14 of a bin edge, where t is
 * continuous.  1 <= n_bins <= 128, 1 <= n_samples <= 2^24 (DVGO_ERR_INVALID_ARG otherwise). */
int dvgo_sample_pdf(const dvgo_params *p, const dvgo_grid_desc *density_desc, int n_rays, const float *rays_o,
                    const float *rays_d, const float *probs, int n_bins, int n_samples, const float *jitter,
                    float eta, float *t_out, float *dt_out, void *stream);

/* Kernel kinds for the optional per-kernel timing below. */
enum {
    DVGO_K_RAY_SETUP = 0, DVGO_K_SCAN = 1, DVGO_K_COARSE_FWD = 2, DVGO_K_COARSE_BWD = 3,
    DVGO_K_FINE_DENSITY = 4, DVGO_K_FINE_COLOUR_FWD = 5, DVGO_K_FINE_COMPOSITE = 6,
    DVGO_K_FINE_COMP_BWD = 7, DVGO_K_FINE_COLOUR_BWD = 8, DVGO_K_ADAM = 9, DVGO_K_AUX = 10,
    DVGO_K_WEIGHT_BINS = 11, DVGO_K_PROPOSAL_FWD = 12, DVGO_K_PROPOSAL_BWD = 13, DVGO_K_SAMPLE_PDF = 14,
    DVGO_K_VIEW_COUNTS = 15, DVGO_K_COUNT = 16
};

/* Benchmarking aid.  While enabled (on != 0), every kernel launch of this library is bracketed
 * by a pair of CUDA events recorded on its stream.  dvgo_profile_read() waits for the recorded
 * events, returns the summed device time (ms) and the launch count of one kernel kind, and
 * forgets that kind's records.  Not for use during stream capture.  Host-thread safe. */
int dvgo_profile_enable(int on);
int dvgo_profile_read(int kind, double *total_ms, long long *launches);

/* Tracing: the launches recorded while profiling was enabled, in the order they were launched
 * (on any stream): kind, and start / end times in ms relative to the start of the first one
 * (CUDA events of different streams on one device are comparable).  Writes up to max_records
 * entries to the host arrays kinds, start_ms, end_ms (each of max_records elements), the number
 * written to *n_out, waits for the events, and forgets every record (also those beyond
 * max_records).  DVGO_ERR_INVALID_ARG for a negative max_records or null arrays. */
int dvgo_profile_trace(int max_records, int *kinds, double *start_ms, double *end_ms, int *n_out);

/* Number of kernels this library has launched in this process (all devices, all streams). */
long long dvgo_launch_counter(void);

/* Shift b of Sec. 4.1 Eq. low_density_init for alpha_init and voxel size s. */
float dvgo_shift_from_alpha_init(float alpha_init, float voxel_size);

const char *dvgo_status_string(int status);
int dvgo_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DVGO_H */
