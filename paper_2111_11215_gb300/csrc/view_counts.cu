// view_counts.cu -- Prior 2 of Sec. 4.1: for every point of a lattice, the number of training views
// that see it (n_j), and the learning-rate scale n_j / n_max of the coarse density grid.
//
// A point is seen by a pinhole view when its camera-frame position q = R^T (x - c) lies beyond the
// near distance in front of the camera and projects into the closed image rectangle (occlusion is
// not considered).  That is an integer decision per (point, view) pair, taken exactly as the FP64
// definition takes it:
//
//   * with depth = -q_z > 0 the decision is the sign test of five forms, each affine in the point:
//     F1 = fx q_x + cx depth (u >= 0), F2 = (W - cx) depth - fx q_x (u <= W),
//     F3 = cy depth - fy q_y (v >= 0), F4 = fy q_y + (H - cy) depth (v <= H), F5 = depth - near;
//     the point is seen iff all five are >= 0 (F5 > 0).  On the lattice, x = min + (i, j, k) step,
//     so each form is b + i w_i + j w_j + k w_k with per-view coefficients;
//   * fast test, FP32: every coefficient, the evaluation and the step along k round with an error
//     below 40 u M (u = 2^-24, M the sum over the box of the magnitudes of the form's terms,
//     bounded per view).  A value further than the guard G = 2^-15 3 M from zero has the sign of the
//     exact form, and so gives the FP64 decision.  Each form is scaled by the power of two that
//     brings its guard into (1/2, 1] (exact), so one minimum over the five decides: > 1 seen,
//     < -1 not seen;
//   * the rare pair in between is decided again in FP64 with the definition's operations in the
//     definition's order, each correctly rounded (no contraction), which reproduces the FP64
//     decision bit for bit.
//
// Layout: a thread takes 8 consecutive points along k of one lattice row (the forms step by w_k),
// the views' scaled coefficients sit in shared memory (read as broadcasts), built by each block from
// the FP64 camera matrices.  Guard-band pairs are queued in shared memory and decided after the
// block's pass over the views, 32 to a warp: this GPU's FP64 pipe issues a warp instruction at the
// same cost whether one lane or all are active, so deciding them where they arise (one lane of a
// warp at a time) made the few blocks that meet many of them several times slower than the rest.
// ALU-bound: ~14 instructions per (point, view) pair, 4 output bytes per point.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr int kVcThreads = 256;
constexpr int kVcK = 8;             // consecutive lattice points along k per thread
constexpr int kVcChunk = 384;       // views held in shared memory at a time (30 KB)
constexpr int kVcQueue = 1024;      // guard-band pairs a block defers to its FP64 pass per tile
constexpr float kVcGuard = 3.0517578125e-05f;    // 2^-15

struct VcArgs {
    int nx, ny, nz;
    bool packed;
    float fmin[3], fstep[3];        // FP32 lattice: fmin + i fstep (box corners exact, step rounded)
    double dmin[3], dmax[3];        // the box corners (FP64 lattice of the definition)
    float bmax[3];                  // max(|min|, |max|) per axis
    int V, H, W;
    const double *c2w;              // [V][3][4] row-major [R | c]
    double fx, fy, cx, cy, near;
    float f_cx, f_wcx, f_cy, f_hcy, f_near;
    uint32_t *counts;
    uint32_t *n_max;
};

// The FP64 decision, operation for operation: lattice point, camera frame, depth, projection.
__device__ __noinline__ unsigned sees_fp64(const VcArgs &A, int v, int i, int j, int k) {
    const double *P = A.c2w + 12 * (long long)v;
    const int ijk[3] = {i, j, k};
    const int n[3] = {A.nx, A.ny, A.nz};
    double d[3], q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = __dadd_rn(A.dmin[a], __ddiv_rn(__dmul_rn((double)ijk[a], __dsub_rn(A.dmax[a], A.dmin[a])),
                                                        (double)(n[a] - 1)));
        d[a] = __dsub_rn(x, __ldg(P + 4 * a + 3));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        q[c] = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(P + c), d[0]), __dmul_rn(__ldg(P + 4 + c), d[1])),
                         __dmul_rn(__ldg(P + 8 + c), d[2]));
    const double depth = -q[2];
    if (!(depth > A.near)) return 0u;
    const double u = __dadd_rn(A.cx, __ddiv_rn(__dmul_rn(A.fx, q[0]), depth));
    const double w = __dsub_rn(A.cy, __ddiv_rn(__dmul_rn(A.fy, q[1]), depth));
    return (u >= 0.0 && u <= (double)A.W && w >= 0.0 && w <= (double)A.H) ? 1u : 0u;
}

// Scaled FP32 coefficients of views [v0, v0 + nv) into shared memory: 5 float4 (b, w_i, w_j, w_k)
// per view, one per form F1..F5, each multiplied by the power of two that puts its guard in (1/2, 1].
__device__ void load_views(const VcArgs &A, float4 *s, int v0, int nv) {
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const double *P = A.c2w + 12 * (long long)(v0 + t);
        float R[3][3], c[3], amp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) R[a][b] = (float)P[4 * a + b];
            c[a] = (float)P[4 * a + 3];
            amp[a] = A.bmax[a] + fabsf(c[a]);     // bounds |x_a - c_a| over the box
        }
        const float fx = (float)A.fx, fy = (float)A.fy;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            float al[3], mag = m == 4 ? A.f_near : 0.0f;
            float bsum = m == 4 ? -A.f_near : 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float t0, t1;             // the two terms of the form's coefficient on axis a
                switch (m) {
                    case 0: t0 = fx * R[a][0]; t1 = -A.f_cx * R[a][2]; break;
                    case 1: t0 = -fx * R[a][0]; t1 = -A.f_wcx * R[a][2]; break;
                    case 2: t0 = -fy * R[a][1]; t1 = -A.f_cy * R[a][2]; break;
                    case 3: t0 = fy * R[a][1]; t1 = -A.f_hcy * R[a][2]; break;
                    default: t0 = 0.0f; t1 = -R[a][2]; break;
                }
                al[a] = t0 + t1;
                mag += (fabsf(t0) + fabsf(t1)) * amp[a];
                bsum = fmaf(al[a], A.fmin[a] - c[a], bsum);
            }
            int e;
            frexpf(kVcGuard * 3.0f * mag, &e);
            const float sc = ldexpf(1.0f, -e);
            s[5 * t + m] = make_float4(bsum * sc, al[0] * A.fstep[0] * sc, al[1] * A.fstep[1] * sc,
                                       al[2] * A.fstep[2] * sc);
        }
    }
}

// Point (i, j, k0) of work item it: rows of the lattice in canonical order, kb items of kVcK points
// per row.
__device__ __forceinline__ void vc_item(const VcArgs &A, long long it, int kb, long long &row, int &i, int &j,
                                        int &k0) {
    row = it / kb;
    k0 = (int)(it - row * kb) * kVcK;
    i = (int)(row / A.ny);
    j = (int)(row - (long long)i * A.ny);
}

// The smallest of the five scaled forms at point k0 + r of a thread's run.
__device__ __forceinline__ float vc_min_form(const float (&f0)[5], const float (&wk)[5], float r) {
    return fminf(fminf(fminf(fmaf(r, wk[0], f0[0]), fmaf(r, wk[1], f0[1])),
                       fminf(fmaf(r, wk[2], f0[2]), fmaf(r, wk[3], f0[3]))),
                 fmaf(r, wk[4], f0[4]));
}

__global__ void __launch_bounds__(kVcThreads, 4) view_count_kernel(const __grid_constant__ VcArgs A) {
    __shared__ float4 sv[kVcChunk * 5];
    // pairs inside a guard band: the FP64 test runs once per tile with every lane of a warp busy
    // (the FP64 pipe is narrow, so a lone lane costs a whole warp's issue slots)
    __shared__ uint32_t q_view[kVcQueue];
    __shared__ uint16_t q_point[kVcQueue];          // threadIdx.x * kVcK + r
    __shared__ uint32_t q_extra[kVcThreads * kVcK];  // FP64 verdicts per point of the tile
    __shared__ unsigned q_n;
    const int kb = (A.nz + kVcK - 1) / kVcK;
    const long long items = (long long)A.nx * A.ny * kb;
    const bool resident = A.V <= kVcChunk;
    if (resident) load_views(A, sv, 0, A.V);
    const bool vec_store = !A.packed && (A.nz % 4) == 0 && (reinterpret_cast<uintptr_t>(A.counts) & 15u) == 0;
    unsigned local_max = 0;
    // block-granular stride, so every thread of a block runs the same iterations (uniform barriers)
    for (long long base = (long long)blockIdx.x * kVcThreads; base < items; base += (long long)gridDim.x * kVcThreads) {
        const long long it = base + threadIdx.x;
        const bool live = it < items;
        long long row;
        int i, j, k0;
        vc_item(A, live ? it : items - 1, kb, row, i, j, k0);
        const float fi = (float)i, fj = (float)j, fk = (float)k0;
        unsigned cnt[kVcK];
#pragma unroll
        for (int r = 0; r < kVcK; ++r) {
            cnt[r] = 0u;
            q_extra[threadIdx.x * kVcK + r] = 0u;
        }
        if (threadIdx.x == 0) q_n = 0u;
        __syncthreads();
        for (int v0 = 0; v0 < A.V; v0 += kVcChunk) {
            const int nv = min(kVcChunk, A.V - v0);
            if (!resident) {
                __syncthreads();
                load_views(A, sv, v0, nv);
                __syncthreads();
            }
            for (int t = 0; t < nv; ++t) {
                float f0[5], wk[5];
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const float4 q = sv[5 * t + m];
                    f0[m] = fmaf(fk, q.w, fmaf(fj, q.z, fmaf(fi, q.y, q.x)));
                    wk[m] = q.w;
                }
                float amin = INFINITY;    // the smallest |min form| of this view's points
#pragma unroll
                for (int r = 0; r < kVcK; ++r) {
                    const float mn = vc_min_form(f0, wk, (float)r);
                    cnt[r] += mn > 1.0f ? 1u : 0u;
                    amin = fminf(amin, fabsf(mn));
                }
                if (amin <= 1.0f && live) {   // rare: queue for the FP64 pass (decide now if the queue is full)
#pragma unroll
                    for (int r = 0; r < kVcK; ++r) {
                        if (fabsf(vc_min_form(f0, wk, (float)r)) <= 1.0f && k0 + r < A.nz) {
                            const unsigned slot = atomicAdd(&q_n, 1u);
                            if (slot < (unsigned)kVcQueue) {
                                q_view[slot] = (uint32_t)(v0 + t);
                                q_point[slot] = (uint16_t)(threadIdx.x * kVcK + r);
                            } else {
                                cnt[r] += sees_fp64(A, v0 + t, i, j, k0 + r);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        const unsigned nq = min(q_n, (unsigned)kVcQueue);
        for (unsigned e = threadIdx.x; e < nq; e += kVcThreads) {
            const unsigned lp = q_point[e];
            long long orow;
            int oi, oj, ok0;
            vc_item(A, base + lp / kVcK, kb, orow, oi, oj, ok0);
            if (sees_fp64(A, (int)q_view[e], oi, oj, ok0 + (int)(lp % kVcK))) atomicAdd(&q_extra[lp], 1u);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kVcK; ++r) cnt[r] += q_extra[threadIdx.x * kVcK + r];
        if (live) {
            if (vec_store && k0 + kVcK <= A.nz) {
                uint4 *dst = reinterpret_cast<uint4 *>(A.counts + row * A.nz + k0);
                dst[0] = make_uint4(cnt[0], cnt[1], cnt[2], cnt[3]);
                dst[1] = make_uint4(cnt[4], cnt[5], cnt[6], cnt[7]);
            } else {
#pragma unroll
                for (int r = 0; r < kVcK; ++r)
                    if (k0 + r < A.nz) A.counts[grid_index(i, j, k0 + r, A.ny, A.nz, A.packed)] = cnt[r];
            }
#pragma unroll
            for (int r = 0; r < kVcK; ++r)
                if (k0 + r < A.nz) local_max = max(local_max, cnt[r]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0 && local_max) atomicMax(A.n_max, local_max);
}

__global__ void __launch_bounds__(256) view_scale_kernel(const uint32_t *__restrict__ counts, long long n,
                                                         const uint32_t *__restrict__ n_max, float *__restrict__ scale) {
    const uint32_t m = *n_max;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        scale[e] = m ? __fdiv_rn((float)counts[e], (float)m) : 1.0f;
}

}  // namespace

void launch_view_counts(const dvgo_grid_desc &g, const dvgo_view_rig &rig, const double *c2w, uint32_t *counts,
                        float *lr_scale, uint32_t *n_max, cudaStream_t s) {
    VcArgs A;
    A.nx = g.nx;
    A.ny = g.ny;
    A.nz = g.nz;
    A.packed = g.layout == DVGO_LAYOUT_PACKED;
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        A.fmin[a] = g.xyz_min[a];
        A.fstep[a] = (g.xyz_max[a] - g.xyz_min[a]) / (float)(n[a] - 1);
        A.dmin[a] = g.xyz_min[a];
        A.dmax[a] = g.xyz_max[a];
        A.bmax[a] = fmaxf(fabsf(g.xyz_min[a]), fabsf(g.xyz_max[a]));
    }
    A.V = rig.n_views;
    A.H = rig.height;
    A.W = rig.width;
    A.c2w = c2w;
    A.fx = rig.fx;
    A.fy = rig.fy;
    A.cx = rig.cx;
    A.cy = rig.cy;
    A.near = rig.near;
    A.f_cx = (float)rig.cx;
    A.f_wcx = (float)((double)rig.width - rig.cx);
    A.f_cy = (float)rig.cy;
    A.f_hcy = (float)((double)rig.height - rig.cy);
    A.f_near = (float)rig.near;
    A.counts = counts;
    A.n_max = n_max;
    const long long npts = (long long)g.nx * g.ny * g.nz;
    const long long elems = A.packed ? (long long)dvgo_grid_elements(&g) : npts;
    cudaMemsetAsync(n_max, 0, sizeof(uint32_t), s);
    if (A.packed) cudaMemsetAsync(counts, 0, (size_t)elems * sizeof(uint32_t), s);
    const long long items = (long long)g.nx * g.ny * ((g.nz + kVcK - 1) / kVcK);
    {
        ProfScope ps_(DVGO_K_VIEW_COUNTS, s);
        view_count_kernel<<<(unsigned)std::min<long long>((items + kVcThreads - 1) / kVcThreads,
                                                          (long long)num_sms() * 64),
                            kVcThreads, 0, s>>>(A);
    }
    if (lr_scale) {
        ProfScope ps_(DVGO_K_VIEW_COUNTS, s);
        view_scale_kernel<<<(unsigned)std::min<long long>((elems + 255) / 256, (long long)num_sms() * 16), 256, 0, s>>>(
            counts, elems, n_max, lr_scale);
    }
}

}  // namespace dvgo
