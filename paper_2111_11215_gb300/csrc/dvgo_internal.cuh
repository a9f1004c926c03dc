// dvgo_internal.cuh -- shared device-side definitions of the DVGO render kernels (sm_103a).
//
// Data flow of one render (all on the caller's stream, no host synchronisation):
//   ray_setup        per ray, FP64: normalise d, clip to the box, count samples, store the ray
//                    in lattice coordinates (Sec. 4.2 fine-stage sampling, Eq. coarse_sample)
//   scan_counts      exclusive scan of the per-ray counts -> first sample slot of every ray
//   coarse_fwd/bwd   warp per ray: gather, post-activation, warp-scan compositing (Sec. 2/3/4.1)
//   fine_density     warp per ray: density gather + post-activation, per-sample optical depth,
//                    compact list of the kept samples (Sec. 4.2 free space skipping)
//   fine_colour      persistent CTAs over tiles of kept samples: feature gather + PE + MLP
//   fine_composite   warp per ray: transmittance scan, C_hat, loss (Eq. volume_rendering)
//   fine_bwd_*       composite backward + density scatter (warp per ray), then the colour tile
//                    kernel backward (MLP backward + feature scatter)
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "dvgo.h"

namespace dvgo {

constexpr int kWarp = 32;
constexpr int kMaxFeat = 16;
constexpr int kPeStride = 32;                      // floats per ray of the direction encoding
constexpr int kMaxChunks = 64;                    // backward kernels: rays of <= 64 x 32 samples
constexpr int kMaxSamplesPerRay = 32 * kMaxChunks;

// Lattice coordinates of samples are carried in 64-bit fixed point with kFxBits fractional bits
// (resolution 9e-13 lattice units, range +-8.4e6): the per-sample position then needs no FP64
// arithmetic, which this GPU executes at a small fraction of its FP32 / integer rate.
constexpr int kFxBits = 40;

// Per-ray record written by ray_setup (128 bytes).  Lattice coordinate u = (x - xyz_min) (n - 1) /
// (xyz_max - xyz_min) per axis; the FP64 values below are rounded once into fixed point.
struct RayRec {
    long long uefx[3];   // entry point (t = t_enter), fixed point
    double e[3];         // normalised direction in lattice units per unit of t
    long long u0fx[3];   // uniform stepping: sample 0 at t_enter + p * step, fixed point
    long long dfx[3];    // uniform stepping: step * e, fixed point
    double t_enter;      // clipped entry distance
    float dir[3];        // normalised direction (FP32, positional encoding input)
    float p;             // jitter in [0, 1)
    int n;               // number of samples
    int off;             // first sample slot (exclusive scan of n)
};
static_assert(sizeof(RayRec) == 128, "RayRec layout");
static_assert(offsetof(RayRec, off) == offsetof(RayRec, n) + 4 && offsetof(RayRec, n) % 8 == 0, "RayRec (n, off) pair");

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
    int flags;           // bit 0: a ray of the last forward had a zero / non-finite direction
    int total;           // total samples of the batch (sum of n)
    int n_kept;          // fine stage: samples kept after the tau_f test
    unsigned done;       // block-completion counter of the loss reduction
    float loss_acc;      // sum over rays of ||C_hat - C||^2
    int aux;             // 1: the last forward had a target and auxiliary loss weights (rtarget valid)
    int xcache;          // 1: the last forward stored the colour kernels' input panels (xcache valid)
    int pad[57];
};
static_assert(sizeof(WsHeader) == 256, "WsHeader size");

// Workspace layout; every block 256-byte aligned.
struct WsLayout {
    size_t header, rays, rayout, rtarget, pe, texit, samp, sgrad, kept, xcache, total;   // xcache 0: none
    long long max_samples;
};

// Everything a render kernel needs, passed by value.
struct RenderArgs {
    int R;
    int mode, rgb_act, mlp_prec, nfreq, hidden;
    int nfreq_pos;              // fine: PE frequencies on the query point x (0: x is not an input)
    float pos0[3], posh[3];     // world position of lattice coordinate u: pos0 + u posh (FP32)
    float step, shift_b, tau_f;
    float bg[3];
    int nx, ny, nz, C;
    int cdtype;                 // dtype of the colour / feature grid
    const float *density;
    const void *cgrid;
    const float *target;        // nullable
    // explicit samples (nullable)
    const float *ts, *dts;
    int n_expl;
    // workspace views
    WsHeader *hdr;
    RayRec *rays;
    float4 *rayout;             // per ray: C_hat (xyz), T_K (w)
    float4 *rtarget;            // per ray: the forward's target (auxiliary losses)
    float w_pt, w_bg;           // auxiliary loss weights
    int act_order;              // DVGO_ACT_POST / PRE / IN
    int packed;                 // density and colour / feature grids in DVGO_LAYOUT_PACKED
    int fs_packed;              // the known-free-space grid in DVGO_LAYOUT_PACKED
    float *pe;                  // fine: per ray [d (3), sin (12), cos (12), 0 x 5] (kPeStride floats)
    double *texit;              // fine: per ray clipped exit distance
    float4 *samp;               // per sample slot: (tau, r, g, b)
    float4 *sgrad;              // per sample slot: (unused, dL/dc)
    int2 *kept;                 // compact list of kept samples: (slot, ray)
    unsigned char *xcache;      // BF16 tensor-core path: the forward's X panel of every tile (16 KiB
                                // each, swizzled as in shared memory), reloaded by the backward
    long long max_samples;
    // outputs
    float *rgb_out, *tfinal_out, *loss_out, *dloss_out;
    // backward inputs / outputs
    const float *grad_rgb, *grad_tfinal;
    float *grad_density, *grad_cgrid, *grad_mlp;
    // MLP
    const float *w1, *b1, *w2, *b2, *w3, *b3;
    int in_dim;
    // known free space (fine stage, nullable fs_density): the coarse grid and the affine map of
    // fine lattice coordinates onto its lattice, u_c = fs_off + u_f * fs_scale / 2^kFsScaleBits
    // (both fixed point; fs_off with kFxBits fractional bits)
    const float *fs_density;
    int fs_nx, fs_ny, fs_nz;
    float fs_shift_b, fs_step, fs_tau;
    long long fs_scale[3], fs_off[3];
    // failure detection of the tensor-core kernels: bound on every device wait (ns), and the
    // testing aid that withholds one producer arrival on tile withhold_tile - 1 (0: none)
    unsigned long long wait_ns;
    int withhold_tile;
};

constexpr unsigned long long kDefaultWaitNs = 2000000000ull;   // 2 s

constexpr int kFsScaleBits = 48;

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ float softplusf(float z) {
    // log(1 + exp(z)) without overflow (Eq. density_activation)
    return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// Background entropy loss term (Supp. A): natural-log binary entropy of the accumulated alpha
// a = 1 - T_K clamped to [1e-6, 1 - 1e-6], and its derivative with respect to T_K,
// log(a) - log(1 - a), which is 0 where the clamp is active.
constexpr float kBgEps = 1e-6f;
__device__ __forceinline__ float bg_entropy(float TK) {
    const float a = fminf(fmaxf(1.0f - TK, kBgEps), 1.0f - kBgEps);
    return -a * logf(a) - (1.0f - a) * log1pf(-a);
}
__device__ __forceinline__ float bg_entropy_dT(float TK) {
    const float a = 1.0f - TK;
    return (a < kBgEps || a > 1.0f - kBgEps) ? 0.0f : logf(a) - log1pf(-a);
}

// FP64 value -> fixed point (round to nearest).
__device__ __forceinline__ long long to_fx(double v) { return __double2ll_rn(v * 0x1p40); }

// Ray / box clip in FP64 with every operation separately rounded (no FMA contraction), in the
// order the sample count depends on (Sec. 4.2 fine-stage points sampling):
//   len = sqrt((dx*dx + dy*dy) + dz*dz), dn = d / len;
//   per axis with dn != 0: t1 = (min - o) / dn, t2 = (max - o) / dn, lo = max(lo, min(t1, t2)),
//   hi = min(hi, max(t1, t2)), starting from lo = t_near, hi = t_far; an axis with dn == 0 and o
//   outside the slab empties the interval.  ok is false for a zero or non-finite direction.
struct Clip {
    double dn[3];
    double lo, hi;
    bool ok;
};

__device__ __forceinline__ Clip slab_clip(const double o[3], const double d[3], const double mn[3], const double mx[3],
                                          double t_near, double t_far) {
    Clip c;
    double len2 = __dmul_rn(d[0], d[0]);
    len2 = __dadd_rn(len2, __dmul_rn(d[1], d[1]));
    len2 = __dadd_rn(len2, __dmul_rn(d[2], d[2]));
    const double len = __dsqrt_rn(len2);
    c.ok = (len > 0.0) && isfinite(len) && isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2]);
    c.dn[0] = c.dn[1] = c.dn[2] = 0.0;
    c.lo = t_near;
    c.hi = t_far;
    if (c.ok) {
        for (int a = 0; a < 3; ++a) {
            c.dn[a] = __ddiv_rn(d[a], len);
            if (c.dn[a] != 0.0) {
                const double t1 = __ddiv_rn(__dsub_rn(mn[a], o[a]), c.dn[a]);
                const double t2 = __ddiv_rn(__dsub_rn(mx[a], o[a]), c.dn[a]);
                const double tl = t1 < t2 ? t1 : t2;
                const double th = t1 < t2 ? t2 : t1;
                if (tl > c.lo) c.lo = tl;
                if (th < c.hi) c.hi = th;
            } else if (o[a] < mn[a] || o[a] > mx[a]) {
                c.lo = 1.0;
                c.hi = 0.0;
            }
        }
    } else {
        c.lo = 1.0;
        c.hi = 0.0;
    }
    return c;
}

// Base corner (clamped to [0, n-2]) and FP32 fractional offsets of a lattice coordinate.
struct Cell {
    int i0, j0, k0;
    float fx, fy, fz;
};

// One axis of a fixed-point lattice coordinate: i0 = clamp(floor(u), 0, n - 2), f = u - i0.  Inside
// the lattice the 40 fractional bits are converted as two 20-bit halves (each exact in FP32) with
// one final rounding; at the clamped edges f = u - i0 is formed in FP64.
__device__ __forceinline__ void fx_axis(long long ufx, int n, int &i0, float &f) {
    const long long ip = ufx >> kFxBits;
    const long long ic = ip < 0 ? 0LL : (ip > (long long)(n - 2) ? (long long)(n - 2) : ip);
    i0 = (int)ic;
    if (ip == ic) {
        const unsigned long long fr = (unsigned long long)ufx & ((1ULL << kFxBits) - 1ULL);
        f = fmaf(__uint2float_rn((unsigned)(fr >> 20)), 0x1p-20f, __uint2float_rn((unsigned)(fr & 0xFFFFFULL)) * 0x1p-40f);
    } else {
        f = (float)((double)(ufx - (ic << kFxBits)) * 0x1p-40);
    }
}

// Packed grid layout (DVGO_LAYOUT_PACKED): 4x4x4-point bricks in row-major brick order
// (ceil(n/4) bricks per axis), the 64 points of a brick in Morton (bit-interleaved) order, so the
// 2x2x2 corners of a cell with even base indices are 8 consecutive entries and most cells' corners
// share a brick.
__host__ __device__ __forceinline__ long long packed_index(int i, int j, int k, int ny, int nz) {
    const int nby = (ny + 3) >> 2, nbz = (nz + 3) >> 2;
    const long long brick = ((long long)(i >> 2) * nby + (j >> 2)) * nbz + (k >> 2);
    const int m = ((i & 1) << 2) | ((j & 1) << 1) | (k & 1) | ((i & 2) << 4) | ((j & 2) << 3) | ((k & 2) << 2);
    return brick * 64 + m;
}

__host__ __device__ __forceinline__ long long grid_index(int i, int j, int k, int ny, int nz, bool packed) {
    return packed ? packed_index(i, j, k, ny, nz) : ((long long)i * ny + j) * nz + k;
}

// Corner q (bits x = q>>2, y = (q>>1)&1, z = q&1): flat lattice index and trilinear weight.
__device__ __forceinline__ long long corner_index(const Cell &c, int q, int ny, int nz, bool packed) {
    return grid_index(c.i0 + ((q >> 2) & 1), c.j0 + ((q >> 1) & 1), c.k0 + (q & 1), ny, nz, packed);
}

// A cell's base corner as kept in the colour kernels' per-row tables: the canonical flat index, or
// for the packed layout the lattice indices as bit fields i0 << 21 | j0 << 10 | k0 (the packed
// layout is limited to 2048 x 2048 x 1024 points).
__device__ __forceinline__ int cell_base(const Cell &c, int ny, int nz, bool packed) {
    return packed ? (c.i0 << 21) | (c.j0 << 10) | c.k0 : (int)grid_index(c.i0, c.j0, c.k0, ny, nz, false);
}

// Flat index of corner (bx, by, bz) of the cell with base `cb` (cell_base).
__device__ __forceinline__ long long corner_from_base(int cb, int bx, int by, int bz, int ny, int nz, bool packed) {
    if (!packed) return (long long)cb + (long long)bx * ny * nz + (long long)by * nz + bz;
    return packed_index(((unsigned)cb >> 21) + bx, ((cb >> 10) & 2047) + by, (cb & 1023) + bz, ny, nz);
}
__device__ __forceinline__ float corner_weight(const Cell &c, int q) {
    float wx = ((q >> 2) & 1) ? c.fx : 1.0f - c.fx;
    float wy = ((q >> 1) & 1) ? c.fy : 1.0f - c.fy;
    float wz = (q & 1) ? c.fz : 1.0f - c.fz;
    return wx * wy * wz;
}

// Fixed-point lattice coordinate and step length of sample k of a ray: uniform stepping
// (t_k = t_enter + (k + p) step, so u_k = u_0 + k (step e) in integer arithmetic) or the explicit
// list (u = u_entry + (t - t_enter) e, the offset in FP64).
__device__ __forceinline__ void sample_fx(const RenderArgs &A, const RayRec &r, int ray, int k, float &dt,
                                          long long u[3]) {
    if (A.ts) {
        const double t = (double)A.ts[(long long)ray * A.n_expl + k];
        dt = A.dts[(long long)ray * A.n_expl + k];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = r.uefx[a] + to_fx((t - r.t_enter) * r.e[a]);
    } else {
        dt = A.step;
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = r.u0fx[a] + (long long)k * r.dfx[a];
    }
}

__device__ __forceinline__ Cell cell_from_fx(const long long u[3], int nx, int ny, int nz) {
    Cell c;
    fx_axis(u[0], nx, c.i0, c.fx);
    fx_axis(u[1], ny, c.j0, c.fy);
    fx_axis(u[2], nz, c.k0, c.fz);
    return c;
}

// World-space position of a sample from its cell, x = xyz_min + (i0 + f) h per axis, in FP32 (the
// input of the positional encoding of x).
__device__ __forceinline__ void cell_world(const RenderArgs &A, const Cell &c, float x[3]) {
    x[0] = fmaf(c.fx, A.posh[0], fmaf((float)c.i0, A.posh[0], A.pos0[0]));
    x[1] = fmaf(c.fy, A.posh[1], fmaf((float)c.j0, A.posh[1], A.pos0[1]));
    x[2] = fmaf(c.fz, A.posh[2], fmaf((float)c.k0, A.posh[2], A.pos0[2]));
}

// Positional encoding of one coordinate v with F frequencies: s[k] = sin(2^k v), c[k] = cos(2^k v),
// k < F, from one sincosf and the double-angle identities sin 2a = 2 sin a cos a,
// cos 2a = (cos a - sin a)(cos a + sin a).
template <int F>
__device__ __forceinline__ void pe_axis(float v, float *s, float *c) {
    sincosf(v, &s[0], &c[0]);
#pragma unroll
    for (int k = 1; k < F; ++k) {
        s[k] = 2.0f * s[k - 1] * c[k - 1];
        c[k] = (c[k - 1] - s[k - 1]) * (c[k - 1] + s[k - 1]);
    }
}

// Cell and step length of sample k of a ray.
__device__ __forceinline__ Cell sample_cell(const RenderArgs &A, const RayRec &r, int ray, int k, float &dt) {
    long long u[3];
    sample_fx(A, r, ray, k, dt, u);
    return cell_from_fx(u, A.nx, A.ny, A.nz);
}

// Optical depth of a sample under the pre- or in-activation order (Sec. 3 Eq. pre_in_post) from its
// corner raw densities v[8]: in: tau = dt sum_q w_q softplus(v_q + b); pre: alpha = sum_q w_q
// (1 - exp(-softplus(v_q + b) dt)), tau = -log(1 - alpha), formed as -log1p(-alpha) while alpha
// is small and as -log(sum_q w_q exp(-softplus(v_q + b) dt)) otherwise (no cancellation, and no
// alpha rounded above 1 when every corner saturates).  (The post order activates the
// interpolated raw density and is computed inline by the kernels.)
__device__ __forceinline__ float tau_pre_in(int order, const Cell &c, const float v[8], float b, float dt) {
    float s = 0.0f;
    if (order == DVGO_ACT_IN) {
#pragma unroll
        for (int q = 0; q < 8; ++q) s = fmaf(corner_weight(c, q), softplusf(v[q] + b), s);
        return s * dt;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s = fmaf(corner_weight(c, q), -expm1f(-softplusf(v[q] + b) * dt), s);
    if (s < 0.5f) return -log1pf(-s);
    float t = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t = fmaf(corner_weight(c, q), expf(-softplusf(v[q] + b) * dt), t);
    return -logf(t);
}

// dtau / dv_q under the pre- or in-activation order (tau of the sample given; the exp(tau) factor of
// the pre order, 1 / (1 - alpha), is capped so that a saturated sample gives a finite value).
__device__ __forceinline__ float dtau_dv_pre_in(int order, const Cell &c, int q, float vq, float b, float dt,
                                                float tau) {
    const float w = corner_weight(c, q), sg = sigmoidf_(vq + b);
    if (order == DVGO_ACT_IN) return w * dt * sg;
    return w * expf(-softplusf(vq + b) * dt) * dt * sg * expf(fminf(tau, 80.0f));
}

// Known-free-space test of Sec. 4.2 at a sample with fine lattice coordinate u: the coarse grid's
// post-activated alpha, 1 - exp(-softplus(interp(x, V_c) + b_c) delta_c), below tau_c.
__device__ __forceinline__ bool known_free(const RenderArgs &A, const long long u[3]) {
    long long uc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        uc[a] = A.fs_off[a] + (long long)(((__int128)u[a] * (__int128)A.fs_scale[a]) >> kFsScaleBits);
    const Cell c = cell_from_fx(uc, A.fs_nx, A.fs_ny, A.fs_nz);
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        s = fmaf(corner_weight(c, q), __ldg(A.fs_density + corner_index(c, q, A.fs_ny, A.fs_nz, A.fs_packed)), s);
    return -expm1f(-softplusf(s + A.fs_shift_b) * A.fs_step) < A.fs_tau;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Inclusive suffix sum over the lanes of a warp: lane i gets sum_{j >= i} v_j.
__device__ __forceinline__ float warp_suffix_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < 32) v += n;
    }
    return v;
}

// Warp-level segmented reduction for gradient scatter.  Lanes hold consecutive samples; a
// segment is a maximal run of adjacent lanes with the same destination index (consecutive
// samples of one ray share lattice corners).  seg_sum() leaves the run total in the run's last
// lane, which then issues one atomic for the whole run.  All 32 lanes must participate.
struct Seg {
    int first;   // first lane of my run
    bool tail;   // I am the last lane of my run
};

__device__ __forceinline__ Seg make_seg(int key, int lane) {
    int prev = __shfl_up_sync(0xffffffffu, key, 1);
    int next = __shfl_down_sync(0xffffffffu, key, 1);
    bool head = (lane == 0) || (prev != key);
    unsigned heads = __ballot_sync(0xffffffffu, head);
    Seg s;
    s.first = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    s.tail = (lane == 31) || (next != key);
    return s;
}

__device__ __forceinline__ float seg_sum(float v, const Seg &s, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane - o >= s.first) v += n;
    }
    return v;
}

// ---------------------------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------

// xcache: add the block of the BF16 colour kernels' X panels (fine mode), after all others so
// that the other offsets do not depend on it.
WsLayout ws_layout(int R, long long max_samples, int mode, bool xcache = false);
void launch_ray_setup(const RenderArgs &A, const float *rays_o, const float *rays_d, const float *jitter,
                      const dvgo_params &p, const dvgo_grid_desc &g, long long cap, cudaStream_t s);
void launch_coarse_fwd(const RenderArgs &A, cudaStream_t s);
void launch_coarse_bwd(const RenderArgs &A, cudaStream_t s);
void launch_fine_density(const RenderArgs &A, cudaStream_t s);
void launch_fine_colour_fwd(const RenderArgs &A, cudaStream_t s);
void launch_fine_composite_fwd(const RenderArgs &A, cudaStream_t s);
void launch_fine_composite_bwd(const RenderArgs &A, cudaStream_t s);
void launch_fine_colour_bwd(const RenderArgs &A, cudaStream_t s);
void launch_adam(float *param, float *grad, float *m, float *v, size_t n, const dvgo_adam_hparams &h,
                 const float *lr_scale, uint16_t *bf16_out, int zero_grad, cudaStream_t s);
void launch_adam_multi(const dvgo_adam_tensor *t, int nt, cudaStream_t s);

void launch_touched(const RenderArgs &A, uint32_t *bitmaps, unsigned long long *counts, cudaStream_t s);
void launch_view_counts(const dvgo_grid_desc &g, const dvgo_view_rig &rig, const double *c2w, uint32_t *counts,
                        float *lr_scale, uint32_t *n_max, cudaStream_t s);

int num_sms();
void ensure_smem(const void *kernel, int bytes);

// Counts a kernel launch and, when timing is enabled, brackets it with two events on its stream.
class ProfScope {
  public:
    ProfScope(int kind, cudaStream_t s);
    ~ProfScope();

  private:
    int kind_;
    cudaStream_t s_;
    void *a_;
};

}  // namespace dvgo
