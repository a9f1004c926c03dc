/*
 * dvgo_oracle.c -- plain, slow FP64 CPU oracle for the DVGO fine/coarse render step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  The CUDA path shares no code with it: nothing here is
 * included, linked or generated into the GPU library, and this file includes none of its headers.
 *
 * It restates, step by step and in double precision, what the method of "Direct Voxel Grid
 * Optimization" (Sun, Sun & Chen, arXiv 2111.11215) computes on one optimisation step:
 *
 *   - ray / bounding-box clipping and stepped sampling      (Sec. 4.1 Eq. coarse_sample, Sec. 4.2
 *                                                             "Fine-stage points sampling", Supp. A jitter)
 *   - trilinear interpolation of a voxel grid              (Sec. 3 Eq. interp)
 *   - shifted softplus and alpha, applied after interp     (Sec. 3 Eq. density_activation,
 *                                                             Eq. post_activation, Eq. density_2_alpha)
 *   - low-density initialisation shift b                   (Sec. 4.1 Eq. low_density_init, Supp. F)
 *   - coarse colour grid / fine feature grid + shallow MLP (Sec. 4.1 Eq. coarse_queries,
 *                                                             Sec. 4.2 Eq. fine_queries, Supp. A)
 *   - volume-rendering quadrature and photometric MSE      (Sec. 2 Eq. volume_rendering, Eq. photo_loss)
 *   - hand-derived reverse-mode gradient of all the above  (chain rule of the same equations)
 *   - Adam with exponential learning-rate decay            (Sec. 5.2 / Supp. A; Kingma & Ba)
 *   - view counts of grid points and the learning-rate scale of Prior 2   (Sec. 4.1 Prior 2)
 *   - the learned sample proposal (64-bin PDF, 48 inverse-CDF samples).  The paper leaves
 *     hierarchical sampling to future work (Supp. B, step-size ablation); the proposal is this
 *     library's addition and is defined here by the readings listed in the design notes.
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled on them):
 *   * ray directions are normalised, so the d/||d||^2 factor of Eq. coarse_sample is 1 and the step
 *     delta is a world-space distance;
 *   * sample k (k = 0, 1, ...) sits at t_k = t_enter + (k + p) * delta with the per-ray jitter p in
 *     [0, 1); the ray keeps every k with t_k < t_exit;
 *   * grid values sit on an align-corners lattice of N points per axis spanning the box;
 *   * a sample whose alpha is below tau_f is removed (alpha := 0, no colour query, no gradient);
 *   * the coarse colour has no activation unless rgb_act = 1 (sigmoid);
 *   * the fine MLP input is [features, d, sin(2^k d_c), cos(2^k d_c)] (c-major blocks, no pi),
 *     followed, when positions are encoded too (Supp. A: k_x = 5), by the same encoding of the
 *     world-space query point x;
 *   * progressive scaling resizes a grid onto the align-corners lattice of the new dimensions over
 *     the same box, each new lattice point taking interp(x, V_old) at its position;
 *   * the loss is (1/R) sum_r sum_ch (C_hat - C)^2;
 *   * a grid point is visible to a view when it lies in front of the camera beyond the near
 *     distance and projects into the closed image rectangle (no occlusion test).
 *
 * The integer decisions (how many samples a ray gets) are taken in FP64 with the operation order
 * written in oracle_ray_bounds(); the file is compiled with -ffp-contract=off so that no fused
 * multiply-add changes a rounding.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* Problem description                                                                          */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int mode;          /* 0 = coarse: colour from a C-channel grid; 1 = fine: feature grid + MLP */
    int rgb_act;       /* coarse only: 0 = identity (literal reading), 1 = sigmoid                */
    int feat_dim;      /* channels C of the colour / feature grid                                */
    int n_freq;        /* fine: positional-encoding frequencies on the view direction           */
    int hidden;        /* fine: MLP width                                                        */
    int nx, ny, nz;    /* lattice points per axis (>= 2)                                         */
    double xyz_min[3], xyz_max[3];
    double shift_b;    /* b of Eq. density_activation                                            */
    double delta;      /* step size (world units)                                                */
    double tau_f;      /* skip threshold on alpha (Sec. 4.2 free space skipping)                 */
    double t_near, t_far;
    double bg[3];      /* background colour c_bg of Eq. volume_rendering                         */
    /* Auxiliary losses (Supp. A weights w_pt_rgb, w_bg; used when a target is given):
     *   per-point rgb loss  L_pt = (1/R) sum_r sum_k w_k ||c_k - C_r||^2 with the compositing
     *                       weights w_k = T_k alpha_k held constant (it supervises the emitted colour
     *                       of every query point, Supp. "Effect of the auxiliary losses");
     *   background entropy  L_bg = (1/R) sum_r H(A_r), H(a) = -a log a - (1 - a) log(1 - a) of the
     *                       accumulated alpha A_r = 1 - T_K,r clamped to [1e-6, 1 - 1e-6]. */
    double w_pt, w_bg;
    /* Order of interpolation and activation (Sec. 3 Eq. pre_in_post):
     *   0 post: alpha = alpha(softplus(interp(x, V) + b))        (the paper's choice)
     *   1 pre:  alpha = interp(x, alpha(softplus(V + b)))
     *   2 in:   alpha = alpha(interp(x, softplus(V + b)))                                    */
    int act_order;
    /* Positional-encoding frequencies on the query point x (Sec. 4.2 Eq. fine_queries_rgb, Supp. A
     * k_x = 5); 0 leaves x out of the MLP input. */
    int n_freq_pos;
    /* Arithmetic of the colour MLP's contractions:
     *   0  exact (FP64 throughout: the definition);
     *   1  BF16 operands -- the chosen form's statement that the colour MLP runs in BF16 with wider
     *      accumulation: every operand of a contraction is rounded to BF16 (round to nearest, ties
     *      to even) -- the input row X, H1 and H2 in the forward; dL/do, dZ2 and dZ1 in the
     *      backward -- and the products are accumulated exactly; the weights are used as given (a
     *      caller passes them rounded), biases b2, b3 and the sum of dL/do into db3 unrounded. */
    int mlp_operands;
} og_params;

/* Known free space (Sec. 4.2): the optimised coarse-stage density grid with its own lattice,
 * shift b_c and step delta_c.  A fine-stage query point x lies in the known free space when
 *     alpha_c(x) = 1 - exp(-softplus(interp(x, V_c) + b_c) delta_c) < tau_c,
 * and is then skipped like a point below tau_f (alpha := 0, no colour, no gradient). */
typedef struct {
    int nx, ny, nz;
    double xyz_min[3], xyz_max[3];
    double shift_b;    /* b_c of the coarse stage                                                */
    double delta;      /* delta_c, the coarse stage's step                                       */
    double tau;        /* tau_c                                                                  */
    const double *density;   /* [nx][ny][nz]                                                    */
} og_freespace;

typedef struct {
    const double *density;      /* [nx][ny][nz]                                               */
    const double *cgrid;        /* [nx][ny][nz][C]                                             */
    /* fine MLP, row-major [in][out]: in_dim = C + 3 + 6*n_freq (+ 3 + 6*n_freq_pos) -> hidden
     * -> hidden -> 3                                                                            */
    const double *w1, *b1, *w2, *b2, *w3, *b3;
    const og_freespace *fs;     /* nullable: no known-free-space test                           */
    /* Optional marks (nullable, [nx*ny*nz], set to 1) of the lattice points a render reads: the
     * 8 corners of every sample that queries the density grid (every sample not in the known free
     * space), and the 8 corners of every kept sample for the colour / feature grid. */
    unsigned char *mark_density, *mark_cgrid;
} og_model;

typedef struct {
    double *density, *cgrid, *w1, *b1, *w2, *b2, *w3, *b3;
} og_grads;

/* ------------------------------------------------------------------------------------------ */
/* Small helpers                                                                                */
/* ------------------------------------------------------------------------------------------ */

static double og_softplus(double z) { return (z > 0 ? z : 0.0) + log1p(exp(-fabs(z))); }

#define OG_BG_EPS 1e-6
/* Background entropy of the accumulated alpha a = 1 - T_K (clamped) and its derivative d/dT_K
 * (zero where the clamp is active): dH/dT = -dH/da = log(a / (1 - a)). */
static double og_bg_entropy(double TK) {
    double a = 1.0 - TK;
    if (a < OG_BG_EPS) a = OG_BG_EPS;
    if (a > 1.0 - OG_BG_EPS) a = 1.0 - OG_BG_EPS;
    return -a * log(a) - (1.0 - a) * log(1.0 - a);
}
static double og_bg_entropy_dT(double TK) {
    double a = 1.0 - TK;
    if (a < OG_BG_EPS || a > 1.0 - OG_BG_EPS) return 0.0;
    return log(a) - log(1.0 - a);
}
static double og_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sec. 4.1 Eq. low_density_init: b = log((1 - alpha_init)^(-1/s) - 1). */
double oracle_shift_from_alpha_init(double alpha_init, double voxel_size) {
    return log(pow(1.0 - alpha_init, -1.0 / voxel_size) - 1.0);
}

/* ------------------------------------------------------------------------------------------ */
/* Ray clipping and sample count (Eq. coarse_sample; Sec. 4.2 fine-stage sampling)             */
/* ------------------------------------------------------------------------------------------ */

/*
 * Normalise d, intersect the ray with the box (slab test), clip to [t_near, t_far], and count
 * the samples t_k = t_enter + (k + p) delta < t_exit.  Every operation is a single rounded FP64
 * operation in the order written; the count is
 *     n = ceil((t_exit - t_enter) / delta - p)   if t_exit > t_enter, else 0,
 * capped at n_cap = ceil(|xyz_max - xyz_min| / delta) + 1.
 * Returns -1 for a zero-length direction, else 0.
 */
int oracle_ray_bounds(const og_params *P, const double o[3], const double d[3], double p,
                      double *t_enter, double *t_exit, double dn[3], int *n) {
    double len2 = d[0] * d[0];
    len2 = len2 + d[1] * d[1];
    len2 = len2 + d[2] * d[2];
    double len = sqrt(len2);
    *n = 0;
    *t_enter = 0.0;
    *t_exit = 0.0;
    if (!(len > 0.0)) return -1;
    double lo = P->t_near, hi = P->t_far;
    for (int a = 0; a < 3; ++a) {
        dn[a] = d[a] / len;
        if (dn[a] != 0.0) {
            double t1 = (P->xyz_min[a] - o[a]) / dn[a];
            double t2 = (P->xyz_max[a] - o[a]) / dn[a];
            double tl = t1 < t2 ? t1 : t2;
            double th = t1 < t2 ? t2 : t1;
            if (tl > lo) lo = tl;
            if (th < hi) hi = th;
        } else if (o[a] < P->xyz_min[a] || o[a] > P->xyz_max[a]) {
            lo = 1.0;
            hi = 0.0; /* parallel to this slab and outside it: no intersection */
        }
    }
    *t_enter = lo;
    *t_exit = hi;
    if (!(hi > lo)) return 0;
    double q = (hi - lo) / P->delta;
    q = q - p;
    double c = ceil(q);
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double L = P->xyz_max[a] - P->xyz_min[a];
        diag2 = diag2 + L * L;
    }
    double cap = ceil(sqrt(diag2) / P->delta) + 1.0;
    if (c > cap) c = cap;
    *n = c > 0.0 ? (int)c : 0;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Trilinear interpolation (Sec. 3 Eq. interp)                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Lattice coordinate of x along each axis, the base corner and the 8 corner weights.
 * Corner c (bits: x = c>>2, y = (c>>1)&1, z = c&1) has flat index idx[c] and weight w[c]. */
static void og_corners(const og_params *P, const double x[3], long idx[8], double w[8]) {
    int N[3] = {P->nx, P->ny, P->nz};
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (x[a] - P->xyz_min[a]) / (P->xyz_max[a] - P->xyz_min[a]) * (double)(N[a] - 1);
        double fl = floor(u);
        if (fl < 0.0) fl = 0.0;
        if (fl > (double)(N[a] - 2)) fl = (double)(N[a] - 2);
        i0[a] = (int)fl;
        f[a] = u - fl;
    }
    for (int c = 0; c < 8; ++c) {
        int bx = (c >> 2) & 1, by = (c >> 1) & 1, bz = c & 1;
        long ix = i0[0] + bx, iy = i0[1] + by, iz = i0[2] + bz;
        idx[c] = (ix * P->ny + iy) * P->nz + iz;
        w[c] = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
    }
}

/* interp(x, V) for a C-channel channel-last grid. */
void oracle_interp(const og_params *P, const double *grid, int C, const double x[3], double *out) {
    long idx[8];
    double w[8];
    og_corners(P, x, idx, w);
    for (int ch = 0; ch < C; ++ch) out[ch] = 0.0;
    for (int c = 0; c < 8; ++c)
        for (int ch = 0; ch < C; ++ch) out[ch] += w[c] * grid[idx[c] * C + ch];
}

/* Progressive scaling (Sec. 4.2): resize a C-channel grid by trilinear interpolation.  The new
 * grid has n2[0] x n2[1] x n2[2] points on the align-corners lattice of the box [dmin, dmax]; its
 * point (i, j, k), at x = dmin + (i, j, k) (dmax - dmin) / (n2 - 1), takes interp(x, V) (Eq. interp)
 * of the source grid (n[3] points on [smin, smax]), with x first clamped into the source box. */
void oracle_resize_grid(const int n[3], const double smin[3], const double smax[3], int C, const double *src,
                        const int n2[3], const double dmin[3], const double dmax[3], double *dst) {
    og_params Q;
    memset(&Q, 0, sizeof(Q));
    Q.nx = n[0];
    Q.ny = n[1];
    Q.nz = n[2];
    for (int a = 0; a < 3; ++a) {
        Q.xyz_min[a] = smin[a];
        Q.xyz_max[a] = smax[a];
    }
    long npts = (long)n2[0] * n2[1] * n2[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < npts; ++p) {
        int ijk[3] = {(int)(p / ((long)n2[1] * n2[2])), (int)((p / n2[2]) % n2[1]), (int)(p % n2[2])};
        double x[3];
        for (int a = 0; a < 3; ++a) {
            x[a] = dmin[a] + (double)ijk[a] * (dmax[a] - dmin[a]) / (double)(n2[a] - 1);
            if (x[a] < smin[a]) x[a] = smin[a];
            if (x[a] > smax[a]) x[a] = smax[a];
        }
        oracle_interp(&Q, src, C, x, dst + p * C);
    }
}

/* Post-activated alpha at a point (Eq. post_activation): alpha(softplus(interp(x, V) + b), delta). */
double oracle_alpha_at(const og_params *P, const double *density, const double x[3], double delta) {
    double s;
    oracle_interp(P, density, 1, x, &s);
    double sigma = og_softplus(s + P->shift_b);
    return -expm1(-sigma * delta);
}

/* Post-activated alpha of the coarse grid at x (the known-free-space test of Sec. 4.2). */
double oracle_coarse_alpha(const og_freespace *F, const double x[3]) {
    og_params Q;
    memset(&Q, 0, sizeof(Q));
    Q.nx = F->nx;
    Q.ny = F->ny;
    Q.nz = F->nz;
    for (int a = 0; a < 3; ++a) {
        Q.xyz_min[a] = F->xyz_min[a];
        Q.xyz_max[a] = F->xyz_max[a];
    }
    Q.shift_b = F->shift_b;
    return oracle_alpha_at(&Q, F->density, x, F->delta);
}

/*
 * Fine voxels allocation (Sec. 4.2): a box enclosing the unknown space of the coarse grid.
 * Lattice point v is "unknown" when alpha(softplus(V_c[v] + b_c), delta_c) >= tau_c.  Inside a cell
 * the interpolated raw density is a convex combination of the 8 corner values and alpha is
 * increasing in it, so a cell whose corners are all known free is known free everywhere; the
 * unknown space therefore lies in the cells touching an unknown lattice point, i.e. in the
 * lattice-index box [min - 1, max + 1] of the unknown points, clamped to [0, N - 1] per axis.
 * Writes lo[3], hi[3] (lattice indices) and returns the number of unknown lattice points (0: the
 * whole grid is known free and lo / hi are left unchanged).
 */
long oracle_unknown_bbox(const og_freespace *F, int lo[3], int hi[3]) {
    int N[3] = {F->nx, F->ny, F->nz};
    int mn[3] = {N[0], N[1], N[2]}, mx[3] = {-1, -1, -1};
    long count = 0;
    for (int i = 0; i < N[0]; ++i)
        for (int j = 0; j < N[1]; ++j)
            for (int k = 0; k < N[2]; ++k) {
                double v = F->density[((long)i * N[1] + j) * N[2] + k];
                double alpha = -expm1(-og_softplus(v + F->shift_b) * F->delta);
                if (alpha < F->tau) continue;
                ++count;
                int ijk[3] = {i, j, k};
                for (int a = 0; a < 3; ++a) {
                    if (ijk[a] < mn[a]) mn[a] = ijk[a];
                    if (ijk[a] > mx[a]) mx[a] = ijk[a];
                }
            }
    if (count == 0) return 0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = mn[a] - 1 < 0 ? 0 : mn[a] - 1;
        hi[a] = mx[a] + 1 > N[a] - 1 ? N[a] - 1 : mx[a] + 1;
    }
    return count;
}

/* ------------------------------------------------------------------------------------------ */
/* Colour model                                                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Positional encoding of a 3-vector v with F frequencies into e:
 * [v (3), sin(2^k v_c) (c-major, k < F), cos(2^k v_c) (c-major)], 3 + 6F values. */
static void og_posenc(const double v[3], int F, double *e) {
    for (int a = 0; a < 3; ++a) e[a] = v[a];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < F; ++k) {
            double arg = ldexp(v[a], k);
            e[3 + a * F + k] = sin(arg);
            e[3 + 3 * F + a * F + k] = cos(arg);
        }
}

/* MLP input row (fine stage, Eq. fine_queries_rgb): [feat (C), PE(d, n_freq)] and, with
 * n_freq_pos > 0, PE(x, n_freq_pos) of the world-space query point appended. */
static void og_mlp_input(const og_params *P, const double *feat, const double dn[3], const double x[3],
                         double *e) {
    int C = P->feat_dim;
    for (int ch = 0; ch < C; ++ch) e[ch] = feat[ch];
    og_posenc(dn, P->n_freq, e + C);
    if (P->n_freq_pos > 0) og_posenc(x, P->n_freq_pos, e + C + 3 + 6 * P->n_freq);
}

int oracle_mlp_in_dim(int feat_dim, int n_freq, int n_freq_pos) {
    return feat_dim + 3 + 6 * n_freq + (n_freq_pos > 0 ? 3 + 6 * n_freq_pos : 0);
}

/* v rounded to BF16 (8 significant bits, round to nearest, ties to even); the exponent range of
 * the values met here is FP32's, so no overflow or subnormal handling is needed. */
double oracle_bf16(double v) {
    if (v == 0.0 || !isfinite(v)) return v;
    int ex;
    frexp(v, &ex);                        /* |v| = m 2^ex, 0.5 <= m < 1 */
    double sc = ldexp(1.0, 8 - ex);       /* v sc in [128, 256): the 8 significant bits */
    return nearbyint(v * sc) / sc;        /* default rounding mode: to nearest, ties to even */
}

/* An MLP operand as the contraction uses it: rounded to BF16 in the BF16-operand arithmetic. */
static double og_op(const og_params *P, double v) { return P->mlp_operands ? oracle_bf16(v) : v; }

/* Forward of the shallow colour MLP, keeping pre-activations for the backward.
 * z1 = e W1 + b1, h1 = relu(z1), z2 = h1 W2 + b2, h2 = relu(z2), o = h2 W3 + b3, c = sigmoid(o).
 * With BF16 operands, e must already be rounded and h1, h2 are stored rounded (as the next
 * contraction and the weight gradients use them); z1, z2 stay exact (they decide the masks). */
static void og_mlp_fwd(const og_params *P, const og_model *M, const double *e, double *z1,
                       double *h1, double *z2, double *h2, double c[3]) {
    int I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos), H = P->hidden;
    for (int j = 0; j < H; ++j) {
        double s = M->b1[j];
        for (int i = 0; i < I; ++i) s += e[i] * M->w1[i * H + j];
        z1[j] = s;
        h1[j] = og_op(P, s > 0 ? s : 0.0);
    }
    for (int j = 0; j < H; ++j) {
        double s = M->b2[j];
        for (int i = 0; i < H; ++i) s += h1[i] * M->w2[i * H + j];
        z2[j] = s;
        h2[j] = og_op(P, s > 0 ? s : 0.0);
    }
    for (int j = 0; j < 3; ++j) {
        double s = M->b3[j];
        for (int i = 0; i < H; ++i) s += h2[i] * M->w3[i * 3 + j];
        c[j] = og_sigmoid(s);
    }
}

/* Public MLP forward on a batch of rows (test of the MLP alone against a matmul chain). */
void oracle_mlp_forward(const og_params *P, const og_model *M, int n, const double *e, double *c) {
    int H = P->hidden, I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos);
    double *buf = (double *)malloc(sizeof(double) * (4 * H + I));
    double *row = buf + 4 * H;
    for (int r = 0; r < n; ++r) {
        for (int i = 0; i < I; ++i) row[i] = og_op(P, e[(long)r * I + i]);
        og_mlp_fwd(P, M, row, buf, buf + H, buf + 2 * H, buf + 3 * H, c + 3 * r);
    }
    free(buf);
}

/* ------------------------------------------------------------------------------------------ */
/* Render one ray forward and (optionally) backward                                            */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    double t, dt;        /* sample position along the ray and its delta                         */
    double x[3];
    long idx[8];
    double cw[8];        /* corner weights                                                      */
    double z;            /* interp(density) + b                                                 */
    double alpha;
    int kept;            /* alpha >= tau_f                                                      */
    double c[3];         /* emitted colour                                                      */
    double craw[3];      /* coarse: interpolated colour before the activation                   */
} og_sample;

/* ------------------------------------------------------------------------------------------ */
/* Running error bound of the fine-stage gradients (test infrastructure)                         */
/* ------------------------------------------------------------------------------------------ */

/*
 * Not part of the method: a first-order bound on how far a finite-precision evaluation of the
 * fine-stage render and its gradient can lie from the exact values computed here, used by the
 * tests as a per-element tolerance.  The arithmetic it describes is the one the north-star
 * precision statement fixes for the colour MLP: each contraction takes its operands rounded to a
 * format of relative rounding u_op (BF16: 2^-8; 0 when the operands are used as they are) and
 * accumulates with unit roundoff u_acc (FP32: 2^-24), as do the per-sample interpolation, the
 * positional encoding and the compositing.
 *
 * The rounded operands are, in the forward, the layer inputs X (the MLP input row), H1 and H2,
 * and, in the backward, dL/do (= dL/dc c (1 - c)), dZ2 and dZ1 (after the ReLU masks).  Each
 * quantity v carries a bound e(v) on |computed - exact|, propagated with absolute values
 * (standard running error analysis): a dot product sum_i a_i b_i with errors e(a_i) in one factor
 * gets sum_i |b_i| e(a_i) + n u_acc sum_i |a_i b_i|, and a rounding to the operand format adds
 * u_op |v|.  A ReLU whose input z satisfies |z| <= e(z) may take either branch in finite
 * precision; the bound then allows both (the output error is at most |z| + e(z), and the masked
 * backward quantity's error at most |dh| + e(dh)).  Gradient bounds add over the samples that
 * contribute to an element.  The density gradient's bound propagates the colour bounds e(c_j)
 * through dC/dtau_k = T_{k+1} c_k - S_k (Eq. volume_rendering) term by term,
 * sum_ch |gC_ch| (T_{k+1} e(c_k) + sum_{j>k} w_j e(c_j)), plus the FP32 compositing itself
 * (prefix sums of the optical depth and the exponential: relative u_acc (k P + k + 6) on T_k, with
 * P the optical depth).  Fine stage only; the summation of contributions into one element is not
 * included (the tests' relative tolerance covers it).
 */
typedef struct {
    double u_op;     /* relative rounding of each MLP operand (see above); 0: none              */
    double u_acc;    /* unit roundoff of accumulation and per-sample arithmetic                  */
    og_grads E;      /* the bounds, accumulated like the gradients (members nullable)            */
} og_bound;

/* Errors of the MLP input row before any rounding to the operand format: the interpolated
 * features (8 weighted corners, FP32 weights), then the positional encodings (sin / cos of 2^k v). */
static void og_input_err(const og_params *P, const og_model *M, const og_sample *s, double u_acc, double *ex) {
    int C = P->feat_dim, F = P->n_freq, Fp = P->n_freq_pos;
    for (int ch = 0; ch < C; ++ch) {
        double a = 0.0;
        for (int c = 0; c < 8; ++c) a += s->cw[c] * fabs(M->cgrid[s->idx[c] * C + ch]);
        ex[ch] = 12.0 * u_acc * a;
    }
    int b = C;
    for (int a = 0; a < 3; ++a) ex[b + a] = 2.0 * u_acc;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < F; ++k) {
            ex[b + 3 + a * F + k] = u_acc * ldexp(4.0, k);
            ex[b + 3 + 3 * F + a * F + k] = u_acc * ldexp(4.0, k);
        }
    if (Fp > 0) {
        b = C + 3 + 6 * F;
        for (int a = 0; a < 3; ++a) {
            double sc = 1.0 + fabs(s->x[a]);
            ex[b + a] = 4.0 * u_acc * sc;
            for (int k = 0; k < Fp; ++k) {
                ex[b + 3 + a * Fp + k] = u_acc * ldexp(4.0, k) * sc;
                ex[b + 3 + 3 * Fp + a * Fp + k] = u_acc * ldexp(4.0, k) * sc;
            }
        }
    }
}

/* Error of a ReLU output given its input z with error ez: both branches allowed when |z| <= ez. */
static double og_relu_err(double z, double ez) {
    if (fabs(z) <= ez) return fabs(z) + ez;
    return z > 0 ? ez : 0.0;
}

/* Error of a masked backward quantity dz = [z > 0] dh given dh's error edh. */
static double og_mask_err(double z, double ez, double dh, double edh) {
    if (fabs(z) <= ez) return fabs(dh) + edh;
    return z > 0 ? edh : 0.0;
}

/* Spacing of BF16 numbers in the binade of |v| (v != 0). */
static double og_bf16_ulp(double v) {
    int ex;
    frexp(v, &ex);
    return ldexp(1.0, ex - 8);
}

/* Error of a BF16 operand rounded from a value v that finite precision computes within ev of its
 * exact value.  Both round to nearest, so the two operands are the same BF16 number unless a
 * rounding midpoint lies within ev of v; then they differ by at most ev plus twice the spacing. */
static double og_bf16_err(double v, double ev) {
    if (ev <= 0.0) return 0.0;
    double a = fabs(v);
    if (a == 0.0) return ev + 2.0 * og_bf16_ulp(ev);
    double sp = og_bf16_ulp(a);
    double lo = floor(a / sp) * sp, hi = ceil(a / sp) * sp;
    int ambiguous;
    if (lo == hi) ambiguous = ev >= 0.25 * sp;                     /* v itself representable */
    else ambiguous = ev >= fabs(a - 0.5 * (lo + hi)) || ev >= (a - lo) + 0.25 * sp || ev >= (hi - a) + 0.5 * sp;
    return ambiguous ? ev + 2.0 * og_bf16_ulp(a + ev) : 0.0;
}

/* Error of an MLP operand formed from a value v with error ev: rounded to BF16 with the same
 * rounding on both sides (BF16-operand arithmetic), or by a format of relative rounding u_op on
 * one side only (exact arithmetic with the rounding as the error's source). */
static double og_operand_err(const og_params *P, double v, double ev, double u_op) {
    return P->mlp_operands ? og_bf16_err(v, ev) : ev + u_op * fabs(v);
}

/* Forward errors of the MLP given the activations of og_mlp_fwd (e: the input row as the
 * contraction uses it; e_pre: before its rounding to the operand format, ex: e_pre's errors). */
static void og_mlp_err_fwd(const og_params *P, const og_model *M, const double *e, const double *e_pre,
                           const double *ex, const double *z1, const double *h1, const double *z2, const double *h2,
                           const double c[3], double u_op, double u_acc, double *exo, double *ez1, double *eh1,
                           double *ez2, double *eh2, double ec[3]) {
    int I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos), H = P->hidden;
    for (int i = 0; i < I; ++i) exo[i] = og_operand_err(P, e_pre[i], ex[i], u_op);
    for (int j = 0; j < H; ++j) {
        double a = fabs(M->b1[j]), pe = 0.0;
        for (int i = 0; i < I; ++i) {
            a += fabs(e[i] * M->w1[i * H + j]);
            pe += fabs(M->w1[i * H + j]) * exo[i];
        }
        ez1[j] = pe + (I + 1) * u_acc * a;
        eh1[j] = og_operand_err(P, z1[j] > 0 ? z1[j] : 0.0, og_relu_err(z1[j], ez1[j]), u_op);
    }
    for (int j = 0; j < H; ++j) {
        double a = fabs(M->b2[j]), pe = 0.0;
        for (int i = 0; i < H; ++i) {
            a += fabs(h1[i] * M->w2[i * H + j]);
            pe += fabs(M->w2[i * H + j]) * eh1[i];
        }
        ez2[j] = pe + (H + 1) * u_acc * a;
        eh2[j] = og_operand_err(P, z2[j] > 0 ? z2[j] : 0.0, og_relu_err(z2[j], ez2[j]), u_op);
    }
    for (int j = 0; j < 3; ++j) {
        double a = fabs(M->b3[j]), pe = 0.0;
        for (int i = 0; i < H; ++i) {
            a += fabs(h2[i] * M->w3[i * 3 + j]);
            pe += fabs(M->w3[i * 3 + j]) * eh2[i];
        }
        double eo = pe + (H + 1) * u_acc * a;
        ec[j] = c[j] * (1.0 - c[j]) * eo + 4.0 * u_acc * c[j];
    }
}

/* Backward errors of one sample's MLP gradient contributions.  dc: dL/dc with relative error
 * rho_dc; dout: dL/do before its rounding to the operand format (db3 sums it unrounded);
 * dout_op, dz2, dz1: the operands of the backward contractions.  Adds the weight-gradient bounds
 * into LE (members nullable) and writes the bound of dL/de into ede[0 .. I) (nullable).
 * exo: the input operand errors of og_mlp_err_fwd.  work: 4H doubles. */
static void og_mlp_err_bwd(const og_params *P, const og_model *M, const double *e, const double *exo,
                           const double *z1, const double *h1, const double *z2, const double *h2,
                           const double *ez1, const double *eh1, const double *ez2, const double *eh2,
                           const double c[3], const double ec[3], const double dc[3], double rho_dc,
                           const double dout[3], const double dout_op[3], const double *dz2, const double *dz1,
                           double u_op, double u_acc, double *work, double *ede, og_grads *LE) {
    int I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos), H = P->hidden;
    double *edz2 = work, *edz1 = work + H;
    double edout[3], edout_op[3];
    for (int j = 0; j < 3; ++j) {
        edout[j] = fabs(dc[j]) * fabs(1.0 - 2.0 * c[j]) * ec[j] + rho_dc * fabs(dc[j]) * c[j] * (1.0 - c[j]) +
                   3.0 * u_acc * fabs(dout[j]);
        edout_op[j] = og_operand_err(P, dout[j], edout[j], u_op);
    }
    for (int i = 0; i < H; ++i) {
        double dh = 0.0, a = 0.0, pe = 0.0;
        for (int j = 0; j < 3; ++j) {
            dh += M->w3[i * 3 + j] * dout_op[j];
            a += fabs(M->w3[i * 3 + j] * dout_op[j]);
            pe += fabs(M->w3[i * 3 + j]) * edout_op[j];
        }
        double edh = pe + 3.0 * u_acc * a;
        edz2[i] = og_operand_err(P, z2[i] > 0 ? dh : 0.0, og_mask_err(z2[i], ez2[i], dh, edh), u_op);
    }
    for (int i = 0; i < H; ++i) {
        double dh = 0.0, a = 0.0, pe = 0.0;
        for (int j = 0; j < H; ++j) {
            dh += M->w2[i * H + j] * dz2[j];
            a += fabs(M->w2[i * H + j] * dz2[j]);
            pe += fabs(M->w2[i * H + j]) * edz2[j];
        }
        double edh = pe + H * u_acc * a;
        edz1[i] = og_operand_err(P, z1[i] > 0 ? dh : 0.0, og_mask_err(z1[i], ez1[i], dh, edh), u_op);
    }
    if (ede)
        for (int i = 0; i < I; ++i) {
            double a = 0.0, pe = 0.0;
            for (int j = 0; j < H; ++j) {
                a += fabs(M->w1[i * H + j] * dz1[j]);
                pe += fabs(M->w1[i * H + j]) * edz1[j];
            }
            ede[i] = pe + H * u_acc * a;
        }
    if (LE->w1)
        for (int i = 0; i < I; ++i)
            for (int j = 0; j < H; ++j) LE->w1[i * H + j] += fabs(e[i]) * edz1[j] + exo[i] * fabs(dz1[j]);
    if (LE->b1)
        for (int j = 0; j < H; ++j) LE->b1[j] += edz1[j];
    if (LE->w2)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < H; ++j) LE->w2[i * H + j] += fabs(h1[i]) * edz2[j] + eh1[i] * fabs(dz2[j]);
    if (LE->b2)
        for (int j = 0; j < H; ++j) LE->b2[j] += edz2[j];
    if (LE->w3)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < 3; ++j) LE->w3[i * 3 + j] += fabs(h2[i]) * edout_op[j] + eh2[i] * fabs(dout_op[j]);
    if (LE->b3)
        for (int j = 0; j < 3; ++j) LE->b3[j] += edout[j];
}

/*
 * The bound of one MLP sample on its own (for the bound's own pins): input row e_in [I] (before
 * any rounding to the operand format) with errors ex [I], upstream dL/dc (relative error rho_dc).
 * Writes c, its bound ec, dL/de and its bound, and ADDS the sample's weight-gradient
 * contributions into G and their bounds into Eb (members nullable).
 */
void oracle_mlp_sample_bound(const og_params *P, const og_model *M, const double *e_in, const double *ex,
                             const double dc[3], double rho_dc, double u_op, double u_acc, double c[3], double ec[3],
                             double *de, double *ede, og_grads *G, og_grads *Eb) {
    int I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos), H = P->hidden;
    double *buf = (double *)calloc((size_t)12 * H + 2 * (size_t)I, sizeof(double));
    double *z1 = buf, *h1 = buf + H, *z2 = buf + 2 * H, *h2 = buf + 3 * H;
    double *ez1 = buf + 4 * H, *eh1 = buf + 5 * H, *ez2 = buf + 6 * H, *eh2 = buf + 7 * H;
    double *dz2 = buf + 8 * H, *dz1 = buf + 9 * H, *work = buf + 10 * H;
    double *e = buf + 12 * H, *exo = e + I;
    for (int i = 0; i < I; ++i) e[i] = og_op(P, e_in[i]);
    og_mlp_fwd(P, M, e, z1, h1, z2, h2, c);
    og_mlp_err_fwd(P, M, e, e_in, ex, z1, h1, z2, h2, c, u_op, u_acc, exo, ez1, eh1, ez2, eh2, ec);
    /* the sample's backward: dout = dc c (1 - c); dZ2 = [z2 > 0] dout W3^T; dZ1 = [z1 > 0] dZ2 W2^T,
     * each operand as the contractions use it */
    double dout[3], dout_op[3];
    for (int j = 0; j < 3; ++j) {
        dout[j] = dc[j] * c[j] * (1.0 - c[j]);
        dout_op[j] = og_op(P, dout[j]);
    }
    for (int i = 0; i < H; ++i) {
        double a = 0.0;
        for (int j = 0; j < 3; ++j) a += M->w3[i * 3 + j] * dout_op[j];
        dz2[i] = og_op(P, z2[i] > 0 ? a : 0.0);
    }
    for (int i = 0; i < H; ++i) {
        double a = 0.0;
        for (int j = 0; j < H; ++j) a += M->w2[i * H + j] * dz2[j];
        dz1[i] = og_op(P, z1[i] > 0 ? a : 0.0);
    }
    for (int i = 0; i < I; ++i) {
        double a = 0.0;
        for (int j = 0; j < H; ++j) a += M->w1[i * H + j] * dz1[j];
        de[i] = a;
    }
    if (G) {
        if (G->w1) for (int i = 0; i < I; ++i) for (int j = 0; j < H; ++j) G->w1[i * H + j] += e[i] * dz1[j];
        if (G->b1) for (int j = 0; j < H; ++j) G->b1[j] += dz1[j];
        if (G->w2) for (int i = 0; i < H; ++i) for (int j = 0; j < H; ++j) G->w2[i * H + j] += h1[i] * dz2[j];
        if (G->b2) for (int j = 0; j < H; ++j) G->b2[j] += dz2[j];
        if (G->w3) for (int i = 0; i < H; ++i) for (int j = 0; j < 3; ++j) G->w3[i * 3 + j] += h2[i] * dout_op[j];
        if (G->b3) for (int j = 0; j < 3; ++j) G->b3[j] += dout[j];
    }
    og_grads none;
    memset(&none, 0, sizeof(none));
    og_mlp_err_bwd(P, M, e, exo, z1, h1, z2, h2, ez1, eh1, ez2, eh2, c, ec, dc, rho_dc, dout, dout_op, dz2, dz1, u_op,
                   u_acc, work, ede, Eb ? Eb : &none);
    free(buf);
}

/*
 * Shared per-ray renderer.  Samples come either from uniform stepping (ts == NULL) or from an
 * explicit list (t, dt) of n_expl samples (the proposal path).  Outputs the composite colour,
 * the final transmittance and, if gC != NULL, accumulates the gradients of
 *     dot(gC, C_hat) + gT * T_final
 * into G (atomically, since rays run in parallel).
 */
static void og_render_ray(const og_params *P, const og_model *M, const double o[3],
                          const double d[3], double p, int n_expl, const double *ts,
                          const double *dts, double rgb[3], double *tfinal, int *nsamp,
                          double *tin, double *tout, const double *gC, double gT, og_grads *G,
                          og_grads *L, double *wbins, int nbins, const double *tgt, double aux_scale,
                          double *aux_loss, const og_bound *B, og_grads *LE) {
    double dn[3], t_enter, t_exit;
    int n;
    oracle_ray_bounds(P, o, d, p, &t_enter, &t_exit, dn, &n);
    if (ts) n = (t_exit > t_enter) ? n_expl : 0;
    if (nsamp) *nsamp = n;
    if (tin) *tin = t_enter;
    if (tout) *tout = t_exit;
    int C = P->feat_dim, H = P->hidden;
    int I = (P->mode == 1) ? oracle_mlp_in_dim(C, P->n_freq, P->n_freq_pos) : 0;
    og_sample *S = (og_sample *)calloc(n > 0 ? n : 1, sizeof(og_sample));
    double *act = NULL; /* per-sample MLP activations: e, z1, h1, z2, h2 */
    int stride = I + 4 * H;
    if (P->mode == 1 && n > 0) act = (double *)malloc(sizeof(double) * (size_t)n * stride);
    double *feat = (double *)malloc(sizeof(double) * (C > 0 ? C : 1));
    /* error bounds (fine stage, with B): per sample the input row before its rounding to the
     * operand format e_pre [I], its errors ex [I], the operand errors exo [I], ez1, eh1, ez2, eh2
     * [H each] and ec [3] */
    int want_bound = B && gC && P->mode == 1 && n > 0;
    int sb = 3 * I + 4 * H + 3;
    double *eb = want_bound ? (double *)malloc(sizeof(double) * (size_t)n * sb) : NULL;

    /* Forward: sample, query, composite (Eq. volume_rendering). */
    double T = 1.0, acc[3] = {0, 0, 0}, pt = 0.0;
    for (int k = 0; k < n; ++k) {
        og_sample *s = &S[k];
        if (ts) {
            s->t = ts[k];
            s->dt = dts[k];
        } else {
            s->t = t_enter + ((double)k + p) * P->delta;
            s->dt = P->delta;
        }
        for (int a = 0; a < 3; ++a) s->x[a] = o[a] + s->t * dn[a];
        if (M->fs && M->fs->density && oracle_coarse_alpha(M->fs, s->x) < M->fs->tau) {
            s->kept = 0;      /* known free space: no fine query, alpha 0, no gradient */
            s->alpha = 0.0;
            continue;
        }
        og_corners(P, s->x, s->idx, s->cw);
        if (M->mark_density)
            for (int c = 0; c < 8; ++c) {
#pragma omp atomic write
                M->mark_density[s->idx[c]] = 1;
            }
        if (P->act_order == 1) {            /* pre: interpolate the corners' alphas */
            s->alpha = 0.0;
            for (int c = 0; c < 8; ++c)
                s->alpha += s->cw[c] * -expm1(-og_softplus(M->density[s->idx[c]] + P->shift_b) * s->dt);
        } else if (P->act_order == 2) {     /* in: interpolate the corners' densities */
            double sigma = 0.0;
            for (int c = 0; c < 8; ++c) sigma += s->cw[c] * og_softplus(M->density[s->idx[c]] + P->shift_b);
            s->alpha = -expm1(-sigma * s->dt);
        } else {                            /* post: activate the interpolated raw density */
            double raw = 0.0;
            for (int c = 0; c < 8; ++c) raw += s->cw[c] * M->density[s->idx[c]];
            s->z = raw + P->shift_b;
            double sigma = og_softplus(s->z);
            s->alpha = -expm1(-sigma * s->dt);
        }
        s->kept = !(s->alpha < P->tau_f);
        if (s->kept && M->mark_cgrid)
            for (int c = 0; c < 8; ++c) {
#pragma omp atomic write
                M->mark_cgrid[s->idx[c]] = 1;
            }
        if (!s->kept) s->alpha = 0.0;
        if (s->kept) {
            for (int ch = 0; ch < C; ++ch) feat[ch] = 0.0;
            for (int c = 0; c < 8; ++c)
                for (int ch = 0; ch < C; ++ch) feat[ch] += s->cw[c] * M->cgrid[s->idx[c] * C + ch];
            if (P->mode == 0) {
                for (int ch = 0; ch < 3; ++ch) {
                    s->craw[ch] = feat[ch];
                    s->c[ch] = P->rgb_act ? og_sigmoid(feat[ch]) : feat[ch];
                }
            } else {
                double *e = act + (size_t)k * stride;
                og_mlp_input(P, feat, dn, s->x, e);
                double *q = want_bound ? eb + (size_t)k * sb : NULL;
                if (want_bound) {
                    memcpy(q, e, sizeof(double) * I);
                    og_input_err(P, M, s, B->u_acc, q + I);
                }
                for (int i = 0; i < I; ++i) e[i] = og_op(P, e[i]);    /* the input row as layer 1 uses it */
                og_mlp_fwd(P, M, e, e + I, e + I + H, e + I + 2 * H, e + I + 3 * H, s->c);
                if (want_bound)
                    og_mlp_err_fwd(P, M, e, q, q + I, e + I, e + I + H, e + I + 2 * H, e + I + 3 * H, s->c, B->u_op,
                                   B->u_acc, q + 2 * I, q + 3 * I, q + 3 * I + H, q + 3 * I + 2 * H,
                                   q + 3 * I + 3 * H, q + 3 * I + 4 * H);
            }
        }
        double w = T * s->alpha;
        for (int ch = 0; ch < 3; ++ch) acc[ch] += w * s->c[ch];
        if (tgt)
            for (int ch = 0; ch < 3; ++ch) pt += w * (s->c[ch] - tgt[ch]) * (s->c[ch] - tgt[ch]);
        T = T * (1.0 - s->alpha);
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = acc[ch] + T * P->bg[ch];
    *tfinal = T;
    if (aux_loss) *aux_loss = tgt ? P->w_pt * pt + P->w_bg * og_bg_entropy(T) : 0.0;

    /* Optional: per-ray histogram of normalised compositing weights over nbins equal bins of
     * [t_enter, t_exit] (labels for the sample proposal). */
    if (wbins) {
        for (int b = 0; b < nbins; ++b) wbins[b] = 0.0;
        double Tw = 1.0, wsum = 0.0;
        for (int k = 0; k < n; ++k) {
            double w = Tw * S[k].alpha;
            Tw *= 1.0 - S[k].alpha;
            int b = (int)floor((S[k].t - t_enter) / (t_exit - t_enter) * nbins);
            if (b < 0) b = 0;
            if (b >= nbins) b = nbins - 1;
            wbins[b] += w;
            wsum += w;
        }
        for (int b = 0; b < nbins; ++b) wbins[b] = (wsum < 1e-4) ? 1.0 / nbins : wbins[b] / wsum;
    }

    if (gC && n > 0) {
        /* Backward.  With tau_k = sigma_k dt_k:  dC/dc_k = w_k,
         * dC/dtau_k = T_{k+1} c_k - S_k,  S_k = sum_{j>k} w_j c_j + T_K bg,  dT_K/dtau_k = -T_K. */
        double *Tk = (double *)malloc(sizeof(double) * (n + 1));
        Tk[0] = 1.0;
        for (int k = 0; k < n; ++k) Tk[k + 1] = Tk[k] * (1.0 - S[k].alpha);
        double Ssuf[3];
        for (int ch = 0; ch < 3; ++ch) Ssuf[ch] = Tk[n] * P->bg[ch];
        double *dh2 = (double *)malloc(sizeof(double) * 3 * (H > 0 ? H : 1));
        double *dz2 = dh2 + H, *dz1 = dh2 + 2 * H;
        /* bound state: suffix sums of w_j e(c_j) and of T_{j+1} (|c_j| + cmax) over later kept
         * samples, the compositing's relative error on T_n, and per-sample scratch */
        double Esuf[3] = {0, 0, 0}, Asuf[3] = {0, 0, 0}, cmax[3], rho_n = 0.0;
        double *bwork = NULL, *ede = NULL;
        if (want_bound) {
            for (int ch = 0; ch < 3; ++ch) cmax[ch] = fabs(P->bg[ch]) > 1.0 ? fabs(P->bg[ch]) : 1.0;
            double Pn = Tk[n] > 0 ? -log(Tk[n]) : 745.0;
            rho_n = B->u_acc * (n * Pn + n + 6.0);
            bwork = (double *)malloc(sizeof(double) * (4 * (size_t)H + I));
            ede = bwork + 4 * H;
        }
        for (int k = n - 1; k >= 0; --k) {
            og_sample *s = &S[k];
            double w = Tk[k] * s->alpha;
            if (s->kept) {
                /* the background entropy enters through T_K like gT */
                double gTe = gT + (tgt ? P->w_bg * aux_scale * og_bg_entropy_dT(Tk[n]) : 0.0);
                double dtau = -gTe * Tk[n];
                for (int ch = 0; ch < 3; ++ch) dtau += gC[ch] * (Tk[k + 1] * s->c[ch] - Ssuf[ch]);
                double edtau = 0.0;
                const double *q = want_bound ? eb + (size_t)k * sb : NULL;
                if (want_bound) {
                    const double *ec = q + 3 * I + 4 * H;
                    for (int ch = 0; ch < 3; ++ch) {
                        Asuf[ch] += Tk[k + 1] * (fabs(s->c[ch]) + cmax[ch]);
                        edtau += fabs(gC[ch]) * (Tk[k + 1] * ec[ch] + Esuf[ch] + rho_n * Asuf[ch]);
                    }
                    edtau += fabs(gTe) * Tk[n] * rho_n;
                    for (int c = 0; c < 8; ++c) {
                        double f;
                        if (P->act_order == 1) {
                            double sp = og_softplus(M->density[s->idx[c]] + P->shift_b);
                            f = 1.0 / (1.0 - s->alpha) * s->cw[c] * exp(-sp * s->dt) * s->dt *
                                og_sigmoid(M->density[s->idx[c]] + P->shift_b);
                        } else if (P->act_order == 2) {
                            f = s->dt * s->cw[c] * og_sigmoid(M->density[s->idx[c]] + P->shift_b);
                        } else {
                            f = s->dt * og_sigmoid(s->z) * s->cw[c];
                        }
                        if (B->E.density) {
#pragma omp atomic
                            B->E.density[s->idx[c]] += edtau * fabs(f);
                        }
                    }
                }
                /* dL/dV_q = dL/dtau dtau/dV_q, tau = -log(1 - alpha) */
                for (int c = 0; c < 8; ++c) {
                    double g;
                    if (P->act_order == 1) {
                        double sp = og_softplus(M->density[s->idx[c]] + P->shift_b);
                        g = dtau / (1.0 - s->alpha) * s->cw[c] * exp(-sp * s->dt) * s->dt *
                            og_sigmoid(M->density[s->idx[c]] + P->shift_b);
                    } else if (P->act_order == 2) {
                        g = dtau * s->dt * s->cw[c] * og_sigmoid(M->density[s->idx[c]] + P->shift_b);
                    } else {
                        g = dtau * s->dt * og_sigmoid(s->z) * s->cw[c];
                    }
#pragma omp atomic
                    G->density[s->idx[c]] += g;
                }
                double dc[3];
                for (int ch = 0; ch < 3; ++ch) {
                    dc[ch] = gC[ch] * w;
                    /* per-point rgb loss: w_k held constant, d/dc_k = 2 w_k (c_k - C) */
                    if (tgt) dc[ch] += P->w_pt * aux_scale * 2.0 * w * (s->c[ch] - tgt[ch]);
                }
                if (P->mode == 0) {
                    for (int ch = 0; ch < 3; ++ch) {
                        double g = dc[ch];
                        if (P->rgb_act) g *= s->c[ch] * (1.0 - s->c[ch]);
                        for (int c = 0; c < 8; ++c) {
#pragma omp atomic
                            G->cgrid[s->idx[c] * C + ch] += g * s->cw[c];
                        }
                    }
                } else {
                    const double *e = act + (size_t)k * stride;
                    const double *z1 = e + I, *h1 = z1 + H, *z2 = h1 + H, *h2 = z2 + H;
                    double dout[3], dout_op[3];
                    for (int j = 0; j < 3; ++j) {
                        dout[j] = dc[j] * s->c[j] * (1.0 - s->c[j]);
                        dout_op[j] = og_op(P, dout[j]);       /* the operand of the contractions */
                    }
                    for (int j = 0; j < 3; ++j) L->b3[j] += dout[j];
                    for (int i = 0; i < H; ++i) {
                        double acc2 = 0.0;
                        for (int j = 0; j < 3; ++j) {
                            L->w3[i * 3 + j] += h2[i] * dout_op[j];
                            acc2 += M->w3[i * 3 + j] * dout_op[j];
                        }
                        dh2[i] = acc2;
                        dz2[i] = og_op(P, z2[i] > 0 ? acc2 : 0.0);
                    }
                    for (int j = 0; j < H; ++j) L->b2[j] += dz2[j];
                    for (int i = 0; i < H; ++i) {
                        double acc1 = 0.0;
                        for (int j = 0; j < H; ++j) {
                            L->w2[i * H + j] += h1[i] * dz2[j];
                            acc1 += M->w2[i * H + j] * dz2[j];
                        }
                        dz1[i] = og_op(P, z1[i] > 0 ? acc1 : 0.0);
                    }
                    for (int j = 0; j < H; ++j) L->b1[j] += dz1[j];
                    for (int i = 0; i < I; ++i) {
                        double de = 0.0;
                        for (int j = 0; j < H; ++j) {
                            L->w1[i * H + j] += e[i] * dz1[j];
                            de += M->w1[i * H + j] * dz1[j];
                        }
                        if (i < C) {
                            for (int c = 0; c < 8; ++c) {
#pragma omp atomic
                                G->cgrid[s->idx[c] * C + i] += de * s->cw[c];
                            }
                        }
                    }
                    if (want_bound) {
                        double Pk = Tk[k] > 0 ? -log(Tk[k]) : 745.0;
                        double rho_dc = B->u_acc * (k * Pk + k + 6.0);
                        og_mlp_err_bwd(P, M, e, q + 2 * I, z1, h1, z2, h2, q + 3 * I, q + 3 * I + H, q + 3 * I + 2 * H,
                                       q + 3 * I + 3 * H, s->c, q + 3 * I + 4 * H, dc, rho_dc, dout, dout_op, dz2, dz1,
                                       B->u_op, B->u_acc, bwork, ede, LE);
                        if (B->E.cgrid)
                            for (int i = 0; i < C; ++i)
                                for (int c = 0; c < 8; ++c) {
#pragma omp atomic
                                    B->E.cgrid[s->idx[c] * C + i] += ede[i] * s->cw[c];
                                }
                    }
                }
                for (int ch = 0; ch < 3; ++ch) Ssuf[ch] += w * s->c[ch];
                if (want_bound)
                    for (int ch = 0; ch < 3; ++ch) Esuf[ch] += w * q[3 * I + 4 * H + ch];
            }
        }
        free(bwork);
        free(dh2);
        free(Tk);
    }
    free(eb);
    free(feat);
    free(act);
    free(S);
}

/*
 * Render R rays.  rays_o, rays_d: [R][3]; jitter: [R] or NULL (then p = 0.5).
 * Explicit-sample mode when ts != NULL: ray r uses n_expl samples ts[r*n_expl + j] with deltas
 * dts[...] (a ray that misses the box still gets none).
 * Outputs rgb [R][3], tfinal [R], nsamp [R], t_enter/t_exit [R] (each nullable except rgb).
 * If target != NULL, *loss = (1/R) sum (C_hat - C)^2 (Eq. photo_loss) + w_pt L_pt + w_bg L_bg
 * (the auxiliary losses of og_params, zero with zero weights).
 * If gC != NULL (per-ray dL/dC_hat, [R][3]) the gradients of sum_r (gC_r . C_hat_r + gT_r T_r),
 * plus those of w_pt L_pt + w_bg L_bg when target != NULL, are ACCUMULATED into G (gT nullable
 * = 0).  wbins (nullable): [R][nbins] weight histograms.
 */
void oracle_render(const og_params *P, const og_model *M, int R, const double *rays_o,
                   const double *rays_d, const double *jitter, int n_expl, const double *ts,
                   const double *dts, const double *target, double *rgb, double *tfinal,
                   int *nsamp, double *t_enter, double *t_exit, double *loss, const double *gC,
                   const double *gT, og_grads *G, double *wbins, int nbins, og_bound *B) {
    int H = P->hidden, I = oracle_mlp_in_dim(P->feat_dim, P->n_freq, P->n_freq_pos);
    /* Sizes of the MLP parameter blocks w1, b1, w2, b2, w3, b3. */
    long nw[6] = {(long)I * H, H, (long)H * H, H, (long)H * 3, 3};
    int want_mlp = (gC != NULL) && (P->mode == 1);
    double *aux = target ? (double *)calloc(R > 0 ? R : 1, sizeof(double)) : NULL;
#pragma omp parallel
    {
        /* Thread-local MLP gradient buffers (summed into G at the end); grid gradients are
         * scattered with atomics. */
        og_grads L, LE;
        double *lbuf = NULL, *lebuf = NULL;
        memset(&L, 0, sizeof(L));
        memset(&LE, 0, sizeof(LE));
        if (want_mlp) {
            long tot = 0;
            for (int i = 0; i < 6; ++i) tot += nw[i];
            lbuf = (double *)calloc((size_t)tot, sizeof(double));
            double *q = lbuf;
            double **dst[6] = {&L.w1, &L.b1, &L.w2, &L.b2, &L.w3, &L.b3};
            for (int i = 0; i < 6; ++i) {
                *dst[i] = q;
                q += nw[i];
            }
            if (B) {      /* thread-local bounds of the MLP gradients, like L */
                lebuf = (double *)calloc((size_t)tot, sizeof(double));
                q = lebuf;
                double **dste[6] = {&LE.w1, &LE.b1, &LE.w2, &LE.b2, &LE.w3, &LE.b3};
                for (int i = 0; i < 6; ++i) {
                    *dste[i] = q;
                    q += nw[i];
                }
            }
        }
        long r;
#pragma omp for schedule(dynamic, 4)
        for (r = 0; r < R; ++r) {
            double p = jitter ? jitter[r] : 0.5;
            double tf;
            og_render_ray(P, M, rays_o + 3 * r, rays_d + 3 * r, p, n_expl,
                          ts ? ts + (size_t)r * n_expl : NULL,
                          dts ? dts + (size_t)r * n_expl : NULL, rgb + 3 * r, &tf,
                          nsamp ? nsamp + r : NULL, t_enter ? t_enter + r : NULL,
                          t_exit ? t_exit + r : NULL, gC ? gC + 3 * r : NULL, gT ? gT[r] : 0.0,
                          G, &L, wbins ? wbins + (size_t)r * nbins : NULL, nbins,
                          target ? target + 3 * r : NULL, R > 0 ? 1.0 / R : 0.0, aux ? aux + r : NULL, B, &LE);
            if (tfinal) tfinal[r] = tf;
        }
        if (want_mlp) {
            double *src[6] = {L.w1, L.b1, L.w2, L.b2, L.w3, L.b3};
            double *dst[6] = {G->w1, G->b1, G->w2, G->b2, G->w3, G->b3};
#pragma omp critical
            for (int i = 0; i < 6; ++i)
                for (long j = 0; j < nw[i]; ++j) dst[i][j] += src[i][j];
            if (B) {
                double *srce[6] = {LE.w1, LE.b1, LE.w2, LE.b2, LE.w3, LE.b3};
                double *dste[6] = {B->E.w1, B->E.b1, B->E.w2, B->E.b2, B->E.w3, B->E.b3};
#pragma omp critical
                for (int i = 0; i < 6; ++i)
                    if (dste[i])
                        for (long j = 0; j < nw[i]; ++j) dste[i][j] += srce[i][j];
            }
        }
        free(lbuf);
        free(lebuf);
    }
    if (target && loss) {
        double Ls = 0.0;
        for (long i = 0; i < 3L * R; ++i) {
            double e = rgb[i] - target[i];
            Ls += e * e;
        }
        for (long r = 0; r < R; ++r) Ls += aux[r];    /* auxiliary losses (zero weights: zero) */
        *loss = R > 0 ? Ls / R : 0.0;
    }
    free(aux);
}

/* ------------------------------------------------------------------------------------------ */
/* Adam (Kingma & Ba) with the exponential decay lr_t = lr0 * 0.1^(t / 20000) (Supp. A)         */
/* ------------------------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------------------------ */
/* Image-fitting toy of Sec. 3 (Fig. exdv_poc)                                                  */
/* ------------------------------------------------------------------------------------------ */

/*
 * A binary image of H x W pixels is regressed by a gh x gw grid V queried with bilinear
 * interpolation under the pre-, in- or post-activation order of Eq. pre_in_post.  Readings: the
 * image covers [0, 1]^2 with pixel (i, j) (row i) at ((i + 0.5) / H, (j + 0.5) / W); the grid's
 * points sit on the align-corners lattice of [0, 1]^2 (u = x (g - 1), i0 = clamp(floor(u), 0,
 * g - 2), f = u - i0); the predicted pixel is the alpha of the order with softplus(v + b) and
 * alpha(sigma) = 1 - exp(-sigma delta); the loss is the mean squared error over all pixels.
 * Writes the predicted image (nullable), adds dL/dV into grad (nullable) and returns L.
 */
double oracle_fit2d(int H, int W, int gh, int gw, int order, double b, double delta, const double *V,
                    const double *target, double *image, double *grad) {
    double loss = 0.0;
    double scale = 1.0 / ((double)H * (double)W);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double u[2] = {(i + 0.5) / H * (gh - 1), (j + 0.5) / W * (gw - 1)};
            int g[2] = {gh, gw}, c0[2];
            double f[2];
            for (int a = 0; a < 2; ++a) {
                double fl = floor(u[a]);
                if (fl < 0.0) fl = 0.0;
                if (fl > (double)(g[a] - 2)) fl = (double)(g[a] - 2);
                c0[a] = (int)fl;
                f[a] = u[a] - fl;
            }
            long idx[4];
            double w[4], v[4];
            for (int q = 0; q < 4; ++q) {
                int bi = (q >> 1) & 1, bj = q & 1;
                idx[q] = (long)(c0[0] + bi) * gw + (c0[1] + bj);
                w[q] = (bi ? f[0] : 1.0 - f[0]) * (bj ? f[1] : 1.0 - f[1]);
                v[q] = V[idx[q]];
            }
            double alpha, dadv[4];
            if (order == 1) {            /* pre: interpolate the corners' alphas */
                alpha = 0.0;
                for (int q = 0; q < 4; ++q) {
                    double e = exp(-og_softplus(v[q] + b) * delta);
                    alpha += w[q] * (1.0 - e);
                    dadv[q] = w[q] * delta * e * og_sigmoid(v[q] + b);
                }
            } else if (order == 2) {     /* in: interpolate the corners' densities */
                double sigma = 0.0;
                for (int q = 0; q < 4; ++q) sigma += w[q] * og_softplus(v[q] + b);
                double e = exp(-sigma * delta);
                alpha = 1.0 - e;
                for (int q = 0; q < 4; ++q) dadv[q] = delta * e * w[q] * og_sigmoid(v[q] + b);
            } else {                     /* post: activate the interpolated raw value */
                double z = b;
                for (int q = 0; q < 4; ++q) z += w[q] * v[q];
                double e = exp(-og_softplus(z) * delta);
                alpha = 1.0 - e;
                for (int q = 0; q < 4; ++q) dadv[q] = delta * e * og_sigmoid(z) * w[q];
            }
            double r = alpha - target[(long)i * W + j];
            loss += r * r * scale;
            if (image) image[(long)i * W + j] = alpha;
            if (grad)
                for (int q = 0; q < 4; ++q) grad[idx[q]] += 2.0 * r * scale * dadv[q];
        }
    return loss;
}

double oracle_lr_decay(double lr0, int step, double decay_steps) {
    return lr0 * pow(0.1, (double)step / decay_steps);
}

/* One Adam step at 1-based step t with learning rate lr (already decayed).  lr_scale nullable
 * (per-element scale, Sec. 4.1 Prior 2).  If zero_grad, g is cleared afterwards. */
/* One Adam step.  skip_zero_grad != 0 selects the lazy variant (this library's option, not the
 * paper's): an element whose gradient is exactly 0 keeps its parameter and both moments. */
void oracle_adam(long n, double *param, double *grad, double *m, double *v, double lr,
                 double beta1, double beta2, double eps, int t, const double *lr_scale,
                 int zero_grad, int skip_zero_grad) {
    double bc1 = 1.0 - pow(beta1, t), bc2 = 1.0 - pow(beta2, t);
    for (long i = 0; i < n; ++i) {
        double g = grad[i];
        if (skip_zero_grad && g == 0.0) continue;
        m[i] = beta1 * m[i] + (1.0 - beta1) * g;
        v[i] = beta2 * v[i] + (1.0 - beta2) * g * g;
        double mhat = m[i] / bc1, vhat = v[i] / bc2;
        double step = lr * (lr_scale ? lr_scale[i] : 1.0);
        param[i] -= step * mhat / (sqrt(vhat) + eps);
        if (zero_grad) grad[i] = 0.0;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Learned sample proposal (the library's addition; the paper defers hierarchical sampling)    */
/* ------------------------------------------------------------------------------------------ */

/*
 * Proposal network on one ray: for each of nb equal bins of [t_enter, t_exit], the bin centre
 * x_b = o + t_b d is encoded as [x, sin(2^k x_c), cos(2^k x_c)] (k < pf, c-major), passed through
 * an MLP  in -> ph -> ph -> ph -> 1  with ReLU, and the logits are normalised by softmax over bins.
 * Weights row-major [in][out]: pw[0..3], pb[0..3].
 */
typedef struct {
    int n_bins, n_freq, width;
    const double *w[4], *b[4];
} og_prop;

typedef struct {
    double *w[4], *b[4];
} og_prop_grads;

int oracle_prop_in_dim(int n_freq) { return 3 + 6 * n_freq; }

static void og_prop_ray(const og_params *P, const og_prop *Q, const double o[3], const double d[3],
                        double p, double *probs, const double *label, double *loss_ray,
                        double gscale, og_prop_grads *G) {
    double dn[3], t0, t1;
    int n;
    oracle_ray_bounds(P, o, d, p, &t0, &t1, dn, &n);
    int B = Q->n_bins, W = Q->width, I = oracle_prop_in_dim(Q->n_freq), F = Q->n_freq;
    double *buf = (double *)malloc(sizeof(double) * (size_t)B * (I + 6 * W + 1));
    double *logit = buf + (size_t)B * (I + 6 * W);
    int hit = t1 > t0;
    if (!hit) {
        /* A ray that misses the box has no bins: uniform PDF, no loss, no gradient. */
        for (int b = 0; b < B; ++b) probs[b] = 1.0 / B;
        *loss_ray = 0.0;
        free(buf);
        return;
    }
    for (int b = 0; b < B; ++b) {
        double *e = buf + (size_t)b * (I + 6 * W);
        double *zz[3], *hh[3];
        for (int l = 0; l < 3; ++l) {
            zz[l] = e + I + 2 * l * W;
            hh[l] = zz[l] + W;
        }
        double tb = t0 + ((double)b + 0.5) * (t1 - t0) / B;
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = o[a] + tb * dn[a];
        for (int a = 0; a < 3; ++a) e[a] = x[a];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < F; ++k) {
                e[3 + a * F + k] = sin(ldexp(x[a], k));
                e[3 + 3 * F + a * F + k] = cos(ldexp(x[a], k));
            }
        const double *in = e;
        int nin = I;
        for (int l = 0; l < 3; ++l) {
            for (int j = 0; j < W; ++j) {
                double s = Q->b[l][j];
                for (int i = 0; i < nin; ++i) s += in[i] * Q->w[l][i * W + j];
                zz[l][j] = s;
                hh[l][j] = s > 0 ? s : 0.0;
            }
            in = hh[l];
            nin = W;
        }
        double s = Q->b[3][0];
        for (int i = 0; i < W; ++i) s += hh[2][i] * Q->w[3][i];
        logit[b] = s;
    }
    double mx = logit[0];
    for (int b = 1; b < B; ++b) mx = logit[b] > mx ? logit[b] : mx;
    double Z = 0.0;
    for (int b = 0; b < B; ++b) Z += exp(logit[b] - mx);
    for (int b = 0; b < B; ++b) probs[b] = exp(logit[b] - mx) / Z;
    if (label) {
        double L = 0.0;
        for (int b = 0; b < B; ++b)
            if (label[b] > 0) L -= label[b] * log(probs[b]);
        *loss_ray = L;
    }
    if (label && G) {
        double *dh = (double *)malloc(sizeof(double) * 2 * W);
        double *dz = dh + W;
        for (int b = 0; b < B; ++b) {
            double *e = buf + (size_t)b * (I + 6 * W);
            double *zz[3], *hh[3];
            for (int l = 0; l < 3; ++l) {
                zz[l] = e + I + 2 * l * W;
                hh[l] = zz[l] + W;
            }
            /* d(-sum h log p)/ds_b = p_b - h_b (softmax + cross-entropy), scaled by 1/R. */
            double ds = (probs[b] - label[b]) * gscale;
            G->b[3][0] += ds;
            for (int i = 0; i < W; ++i) {
                G->w[3][i] += hh[2][i] * ds;
                dh[i] = Q->w[3][i] * ds;
            }
            for (int l = 2; l >= 0; --l) {
                const double *in = l > 0 ? hh[l - 1] : e;
                int nin = l > 0 ? W : I;
                for (int j = 0; j < W; ++j) dz[j] = zz[l][j] > 0 ? dh[j] : 0.0;
                for (int j = 0; j < W; ++j) G->b[l][j] += dz[j];
                for (int i = 0; i < nin; ++i) {
                    double a = 0.0;
                    for (int j = 0; j < W; ++j) {
                        G->w[l][i * W + j] += in[i] * dz[j];
                        a += Q->w[l][i * W + j] * dz[j];
                    }
                    if (l > 0) dh[i] = a;
                }
            }
        }
        free(dh);
    }
    free(buf);
}

/* Proposal forward (and, with labels and G, the accumulated gradient of the mean cross-entropy
 * loss -(1/R) sum_r sum_b h_rb log p_rb).  probs: [R][n_bins]. */
void oracle_proposal(const og_params *P, const og_prop *Q, int R, const double *rays_o,
                     const double *rays_d, const double *labels, double *probs, double *loss,
                     og_prop_grads *G) {
    int W = Q->width, I = oracle_prop_in_dim(Q->n_freq);
    long nw[4] = {(long)I * W, (long)W * W, (long)W * W, W};
    long nb[4] = {W, W, W, 1};
    double L = 0.0;
#pragma omp parallel reduction(+ : L)
    {
        og_prop_grads Lg;
        double *lbuf = NULL;
        memset(&Lg, 0, sizeof(Lg));
        if (G && labels) {
            long tot = 0;
            for (int i = 0; i < 4; ++i) tot += nw[i] + nb[i];
            lbuf = (double *)calloc((size_t)tot, sizeof(double));
            double *q = lbuf;
            for (int i = 0; i < 4; ++i) {
                Lg.w[i] = q;
                q += nw[i];
                Lg.b[i] = q;
                q += nb[i];
            }
        }
        long r;
#pragma omp for schedule(dynamic, 4)
        for (r = 0; r < R; ++r) {
            double lr = 0.0;
            og_prop_ray(P, Q, rays_o + 3 * r, rays_d + 3 * r, 0.5, probs + (size_t)r * Q->n_bins,
                        labels ? labels + (size_t)r * Q->n_bins : NULL, &lr, 1.0 / R,
                        lbuf ? &Lg : NULL);
            L += lr;
        }
        if (lbuf) {
#pragma omp critical
            for (int i = 0; i < 4; ++i) {
                for (long j = 0; j < nw[i]; ++j) G->w[i][j] += Lg.w[i][j];
                for (long j = 0; j < nb[i]; ++j) G->b[i][j] += Lg.b[i][j];
            }
        }
        free(lbuf);
    }
    if (loss) *loss = R > 0 ? L / R : 0.0;
}

/*
 * Inverse-CDF sampling of ns sorted samples from a piecewise-constant PDF over nb equal bins of
 * [t0, t1].  The PDF is mixed with the uniform one: q_b = (1 - eta) p_b + eta / nb.
 * u_j = (j + jit) / ns; sample j lies in bin b with Q_b <= u_j < Q_{b+1} (Q = CDF of q) at
 * t = t0 + (b + (u_j - Q_b) / q_b) * w (w = bin width).  Deltas: t_{j+1} - t_j, and for the last
 * sample w / (ns * q_b) of its bin.
 */
void oracle_sample_pdf(int nb, const double *probs, double t0, double t1, int ns, double jit,
                       double eta, double *t, double *dt) {
    double *q = (double *)malloc(sizeof(double) * (nb + 1) * 2);
    double *Q = q + nb + 1;
    double w = (t1 - t0) / nb;
    Q[0] = 0.0;
    for (int b = 0; b < nb; ++b) {
        q[b] = (1.0 - eta) * probs[b] + eta / nb;
        Q[b + 1] = Q[b] + q[b];
    }
    int b = 0, last_b = 0;
    for (int j = 0; j < ns; ++j) {
        double u = ((double)j + jit) / ns * Q[nb];
        while (b < nb - 1 && Q[b + 1] <= u) ++b;
        t[j] = t0 + ((double)b + (u - Q[b]) / q[b]) * w;
        last_b = b;
    }
    for (int j = 0; j + 1 < ns; ++j) dt[j] = t[j + 1] - t[j];
    if (ns > 0) dt[ns - 1] = w / (ns * q[last_b] / Q[nb]);
    free(q);
}

/* ------------------------------------------------------------------------------------------ */
/* Prior 2: view-count-based learning rate (Sec. 4.1)                                          */
/* ------------------------------------------------------------------------------------------ */

/*
 * Number of training views that see each of n_pts world points x[3 n_pts] (Sec. 4.1 Prior 2: the
 * view count n_j of grid point j).  View v is the pinhole camera c2w[12 v ...], a row-major 3x4
 * camera-to-world matrix [R | c] whose columns R_0, R_1, R_2 are the camera's x (right), y (up) and
 * z (backward) axes in world space (the camera looks along -z), with focal lengths fx, fy and
 * principal point (cx, cy) in pixels of an image W pixels wide and H high (rows run downward).
 *
 * Reading of "visible" (the paper gives no definition): the camera-frame position
 * q = R^T (x - c) lies in front of the camera beyond the near distance (-q_z > near) and projects
 * into the closed image rectangle, 0 <= cx + fx q_x / (-q_z) <= W and 0 <= cy - fy q_y / (-q_z) <= H.
 * Occlusion is not considered (the grid holds no geometry when the counts are taken).  The sums are
 * taken left to right in the order written.
 */
static int og_sees(const double *P, int H, int W, double fx, double fy, double cx, double cy, double near,
                   const double x[3]) {
    double d[3], q[3];
    for (int i = 0; i < 3; ++i) d[i] = x[i] - P[4 * i + 3];
    for (int k = 0; k < 3; ++k) q[k] = P[k] * d[0] + P[4 + k] * d[1] + P[8 + k] * d[2];
    double depth = -q[2];
    if (!(depth > near)) return 0;
    double u = cx + fx * q[0] / depth;
    double v = cy - fy * q[1] / depth;
    return u >= 0.0 && u <= (double)W && v >= 0.0 && v <= (double)H;
}

void oracle_view_counts_points(long n_pts, const double *x, int V, const double *c2w, int H, int W, double fx,
                               double fy, double cx, double cy, double near, unsigned *counts) {
#pragma omp parallel for schedule(static)
    for (long j = 0; j < n_pts; ++j) {
        unsigned n = 0;
        for (int v = 0; v < V; ++v) n += (unsigned)og_sees(c2w + 12 * (long)v, H, W, fx, fy, cx, cy, near, x + 3 * j);
        counts[j] = n;
    }
}

/*
 * View counts of the points of an align-corners lattice of n[0] x n[1] x n[2] points over the box
 * [xmin, xmax] (point (i, j, k), canonical index (i n1 + j) n2 + k, sits at
 * xmin + (i, j, k) (xmax - xmin) / (n - 1)), and the learning-rate scale n_j / n_max of Prior 2
 * (n_max: the largest count; when no point is seen at all the scale is 1, i.e. no prior).
 * scale is nullable.  Returns n_max.
 */
unsigned oracle_view_counts(const int n[3], const double xmin[3], const double xmax[3], int V, const double *c2w,
                            int H, int W, double fx, double fy, double cx, double cy, double near,
                            unsigned *counts, double *scale) {
    long npts = (long)n[0] * n[1] * n[2];
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(npts > 0 ? npts : 1));
    for (long p = 0; p < npts; ++p) {
        long ijk[3] = {p / ((long)n[1] * n[2]), (p / n[2]) % n[1], p % n[2]};
        for (int a = 0; a < 3; ++a) x[3 * p + a] = xmin[a] + (double)ijk[a] * (xmax[a] - xmin[a]) / (double)(n[a] - 1);
    }
    oracle_view_counts_points(npts, x, V, c2w, H, W, fx, fy, cx, cy, near, counts);
    free(x);
    unsigned n_max = 0;
    for (long p = 0; p < npts; ++p)
        if (counts[p] > n_max) n_max = counts[p];
    if (scale)
        for (long p = 0; p < npts; ++p) scale[p] = n_max ? (double)counts[p] / (double)n_max : 1.0;
    return n_max;
}
