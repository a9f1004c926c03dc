// view_counts.cu -- Prior 2 of Sec. 4.1: for every point of a lattice, the number of training views
// that see it (n_j), and the learning-rate scale n_j / n_max of the coarse density grid.
//
// A point is seen by a pinhole view when its camera-frame position q = R^T (x - c) lies beyond the
// near distance in front of the camera and projects into the closed image rectangle (occlusion is
// not considered).  That is an integer decision per (point, view) pair, taken exactly as the FP64
// definition takes it:
//
//   * fast test, FP32: with depth = -q_z > 0 the image conditions are the signs of four linear forms
//     (fx q_x + cx depth, (W - cx) depth - fx q_x, cy depth - fy q_y, fy q_y + (H - cy) depth) and
//     of depth - near.  Each is a short sum whose FP32 rounding error is below 20 u M (u = 2^-24,
//     M the sum of the magnitudes of its terms over the whole box, bounded per view); a value
//     further than the guard 2^-16 M from zero has the sign of the exact value, and so the FP64
//     decision;
//   * the rare pair inside a guard band is decided again in FP64 with the definition's operations
//     in the definition's order, each correctly rounded (no contraction), which reproduces the
//     FP64 decision bit for bit.
//
// Layout: one thread per lattice point (4 points per thread, strided by the block size so that the
// writes coalesce), the views' FP32 constants in shared memory (read as broadcasts), built by each
// block from the FP64 camera matrices.  ALU-bound: ~30 FP32 flops per pair, 4 output bytes per point.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr int kVcThreads = 256;
constexpr int kVcPts = 4;           // lattice points per thread
constexpr int kVcChunk = 512;       // views held in shared memory at a time (32 KB)
constexpr float kVcGuard = 1.52587890625e-05f;   // 2^-16

struct VcArgs {
    int nx, ny, nz;
    bool packed;
    float fmin[3], fstep[3];        // FP32 lattice: fmin + i fstep
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

// FP32 constants of views [v0, v0 + nv) into shared memory, 4 float4 per view:
//   s[0] = (c, guard of the x forms), s[1] = (fx R_:,0, guard of the y forms),
//   s[2] = (fy R_:,1, guard of the depth form), s[3] = (R_:,2, 0).
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
        float mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mx += fx * fabsf(R[a][0]) * amp[a];
            my += fy * fabsf(R[a][1]) * amp[a];
            mz += fabsf(R[a][2]) * amp[a];
        }
        const float gx = kVcGuard * (mx + fmaxf(fabsf(A.f_cx), fabsf(A.f_wcx)) * mz);
        const float gy = kVcGuard * (my + fmaxf(fabsf(A.f_cy), fabsf(A.f_hcy)) * mz);
        const float ga = kVcGuard * (mz + A.f_near);
        s[4 * t + 0] = make_float4(c[0], c[1], c[2], gx);
        s[4 * t + 1] = make_float4(fx * R[0][0], fx * R[1][0], fx * R[2][0], gy);
        s[4 * t + 2] = make_float4(fy * R[0][1], fy * R[1][1], fy * R[2][1], ga);
        s[4 * t + 3] = make_float4(R[0][2], R[1][2], R[2][2], 0.0f);
    }
}

__global__ void __launch_bounds__(kVcThreads) view_count_kernel(const __grid_constant__ VcArgs A) {
    __shared__ float4 sv[kVcChunk * 4];
    const long long npts = (long long)A.nx * A.ny * A.nz;
    const long long tile = (long long)kVcThreads * kVcPts;
    const bool resident = A.V <= kVcChunk;
    if (resident) {
        load_views(A, sv, 0, A.V);
        __syncthreads();
    }
    unsigned local_max = 0;
    for (long long base = (long long)blockIdx.x * tile; base < npts; base += (long long)gridDim.x * tile) {
        float px[kVcPts], py[kVcPts], pz[kVcPts];
        int li[kVcPts], lj[kVcPts], lk[kVcPts];
        unsigned cnt[kVcPts];
#pragma unroll
        for (int r = 0; r < kVcPts; ++r) {
            const long long p = base + r * kVcThreads + threadIdx.x;
            const long long pc = p < npts ? p : npts - 1;
            lk[r] = (int)(pc % A.nz);
            lj[r] = (int)((pc / A.nz) % A.ny);
            li[r] = (int)(pc / ((long long)A.ny * A.nz));
            px[r] = fmaf((float)li[r], A.fstep[0], A.fmin[0]);
            py[r] = fmaf((float)lj[r], A.fstep[1], A.fmin[1]);
            pz[r] = fmaf((float)lk[r], A.fstep[2], A.fmin[2]);
            cnt[r] = 0u;
        }
        for (int v0 = 0; v0 < A.V; v0 += kVcChunk) {
            const int nv = min(kVcChunk, A.V - v0);
            if (!resident) {
                __syncthreads();
                load_views(A, sv, v0, nv);
                __syncthreads();
            }
            for (int t = 0; t < nv; ++t) {
                const float4 s0 = sv[4 * t], s1 = sv[4 * t + 1], s2 = sv[4 * t + 2], s3 = sv[4 * t + 3];
#pragma unroll
                for (int r = 0; r < kVcPts; ++r) {
                    const float dx = px[r] - s0.x, dy = py[r] - s0.y, dz = pz[r] - s0.z;
                    const float qx = fmaf(s1.z, dz, fmaf(s1.y, dy, s1.x * dx));      // fx q_x
                    const float qy = fmaf(s2.z, dz, fmaf(s2.y, dy, s2.x * dx));      // fy q_y
                    const float dep = -fmaf(s3.z, dz, fmaf(s3.y, dy, s3.x * dx));    // -q_z
                    const float mx = fminf(fmaf(A.f_cx, dep, qx), fmaf(A.f_wcx, dep, -qx));
                    const float my = fminf(fmaf(A.f_cy, dep, -qy), fmaf(A.f_hcy, dep, qy));
                    const float a = dep - A.f_near;
                    const bool in = (mx > s0.w) & (my > s1.w) & (a > s2.w);
                    const bool out = (mx < -s0.w) | (my < -s1.w) | (a < -s2.w);
                    if (in) {
                        ++cnt[r];
                    } else if (!out && base + r * kVcThreads + threadIdx.x < npts) {
                        cnt[r] += sees_fp64(A, v0 + t, li[r], lj[r], lk[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kVcPts; ++r) {
            const long long p = base + r * kVcThreads + threadIdx.x;
            if (p < npts) {
                A.counts[grid_index(li[r], lj[r], lk[r], A.ny, A.nz, A.packed)] = cnt[r];
                local_max = max(local_max, cnt[r]);
            }
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
    const long long tiles = (npts + kVcThreads * kVcPts - 1) / (kVcThreads * kVcPts);
    {
        ProfScope ps_(DVGO_K_VIEW_COUNTS, s);
        view_count_kernel<<<(unsigned)std::min<long long>(tiles, (long long)num_sms() * 64), kVcThreads, 0, s>>>(A);
    }
    if (lr_scale) {
        ProfScope ps_(DVGO_K_VIEW_COUNTS, s);
        view_scale_kernel<<<(unsigned)std::min<long long>((elems + 255) / 256, (long long)num_sms() * 16), 256, 0, s>>>(
            counts, elems, n_max, lr_scale);
    }
}

}  // namespace dvgo
