// fit2d.cu -- the image-fitting toy of Sec. 3 (Fig. exdv_poc): a binary image regressed by a 2D
// grid under the pre-, in- or post-activation order of Eq. pre_in_post (forward, MSE, gradient).
//
// Blocks of 256 threads own 32 x 32-pixel tiles; a warp takes one 32-pixel row of the tile at a
// time.  A pixel's cell and fraction come from integer arithmetic, u = (2i + 1)(g - 1) / (2 H):
// i0 = the quotient (clamped to g - 2), f = the remainder / (2 H) rounded once to FP32, so cell
// choices are exact; the tile's 32 rows and 32 columns are resolved once into shared memory.
// Gradients: the derivative of a pixel's alpha with respect to corner q factors into a per-pixel
// term, the row weight (shared by the warp) and a per-corner term (shared by the pixels of a cell),
// so the column weights are summed over runs of lanes with the same column cell by a segmented
// warp scan and the run's last lane adds the four corners' sums -- into a shared-memory patch of
// the grid points the tile touches, added to global memory once per point, or, for grids finer
// than the image, straight to global memory.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr int kTile = 32;
constexpr int kPatch = 34;   // grid points a 32-pixel span can touch when grid_h - 1 <= height

struct Axis {
    int c0;   // base lattice point
    float f;  // fraction in [0, 1]
};

__device__ __forceinline__ Axis pixel_axis(int i, int n_pix, int g) {
    const long long num = (2LL * i + 1) * (g - 1), den = 2LL * n_pix;
    long long q = num / den;
    Axis a;
    if (q > g - 2) {   // the last lattice interval takes the right edge (f = 1 there)
        a.c0 = g - 2;
        a.f = (float)((double)(num - (long long)(g - 2) * den) / (double)den);
    } else {
        a.c0 = (int)q;
        a.f = (float)(num - q * den) / (float)den;
    }
    return a;
}

template <int ORDER, bool PATCH>
__global__ void __launch_bounds__(256) fit2d_kernel(dvgo_fit2d_desc d, const float *__restrict__ V,
                                                    const float *__restrict__ T, float *__restrict__ img,
                                                    float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ float patch[PATCH ? kPatch * kPatch : 1];
    __shared__ float red[8];
    __shared__ Axis rows[kTile], cols[kTile];
    const int ti = blockIdx.y * kTile, tj = blockIdx.x * kTile;
    if (threadIdx.x < kTile)
        rows[threadIdx.x] = pixel_axis(min(ti + (int)threadIdx.x, d.height - 1), d.height, d.grid_h);
    else if (threadIdx.x < 2 * kTile)
        cols[threadIdx.x - kTile] = pixel_axis(min(tj + (int)threadIdx.x - kTile, d.width - 1), d.width, d.grid_w);
    if (PATCH && grad)
        for (int k = threadIdx.x; k < kPatch * kPatch; k += blockDim.x) patch[k] = 0.0f;
    __syncthreads();
    const int pr0 = rows[0].c0, pc0 = cols[0].c0;
    const float gscale = 2.0f / ((float)d.height * (float)d.width);
    const int lane = threadIdx.x & 31;
    float lsum = 0.0f;
    // every lane runs the same iterations (kTile^2 is a multiple of the block size), so the warp
    // scans below see all 32 lanes; pixels outside the image are inactive lanes
    for (int k = threadIdx.x; k < kTile * kTile; k += blockDim.x) {
        const int i = ti + k / kTile, j = tj + k % kTile;
        const bool on = i < d.height && j < d.width;
        const Axis ay = rows[k / kTile], ax = cols[k % kTile];
        const float wy[2] = {1.0f - ay.f, ay.f}, wx[2] = {1.0f - ax.f, ax.f};
        // dalpha / dv_q = L wy[bi] wx[bj] K[q]: L varies per pixel, K[q] only with the corner's value
        float v[4], K[4], L, alpha;
        int idx[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            idx[q] = (ay.c0 + ((q >> 1) & 1)) * d.grid_w + ax.c0 + (q & 1);
            v[q] = __ldg(V + idx[q]);
        }
        if (ORDER == DVGO_ACT_PRE) {
            alpha = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float e = expf(-softplusf(v[q] + d.shift_b) * d.delta);
                alpha = fmaf(wy[(q >> 1) & 1] * wx[q & 1], 1.0f - e, alpha);
                K[q] = d.delta * e * sigmoidf_(v[q] + d.shift_b);
            }
            L = 1.0f;
        } else if (ORDER == DVGO_ACT_IN) {
            float sigma = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                sigma = fmaf(wy[(q >> 1) & 1] * wx[q & 1], softplusf(v[q] + d.shift_b), sigma);
                K[q] = sigmoidf_(v[q] + d.shift_b);
            }
            alpha = -expm1f(-sigma * d.delta);
            L = d.delta * expf(-sigma * d.delta);
        } else {
            float z = d.shift_b;
#pragma unroll
            for (int q = 0; q < 4; ++q) z = fmaf(wy[(q >> 1) & 1] * wx[q & 1], v[q], z);
            // softplus and sigmoid from one exponential: t = exp(-|z|)
            const float t = expf(-fabsf(z));
            const float sigma = fmaxf(z, 0.0f) + log1pf(t), sg = (z >= 0.0f ? 1.0f : t) / (1.0f + t);
            alpha = -expm1f(-sigma * d.delta);
            L = d.delta * expf(-sigma * d.delta) * sg;
#pragma unroll
            for (int q = 0; q < 4; ++q) K[q] = 1.0f;
        }
        if (on && img) img[(long long)i * d.width + j] = alpha;
        if (T) {
            const float r = on ? alpha - __ldg(T + (long long)i * d.width + j) : 0.0f;
            lsum = fmaf(r, r, lsum);
            if (grad) {
                // the warp's lanes share the pixel row (hence wy and the corner rows); runs of lanes
                // with the same column cell share all four corners: sum L wx over each run, one
                // atomic per corner and run (inactive lanes get a key of their own and add nothing)
                const float gl = on ? gscale * r * L : 0.0f;
                const Seg sg = make_seg(on ? ax.c0 : -1 - lane, lane);
                const float a0 = seg_sum(gl * wx[0], sg, lane), a1 = seg_sum(gl * wx[1], sg, lane);
                if (sg.tail) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float val = wy[(q >> 1) & 1] * K[q] * ((q & 1) ? a1 : a0);
                        if (val == 0.0f) continue;
                        if (PATCH) {
                            const int pi = ay.c0 + ((q >> 1) & 1) - pr0, pj = ax.c0 + (q & 1) - pc0;
                            atomicAdd(&patch[pi * kPatch + pj], val);
                        } else {
                            atomicAdd(grad + idx[q], val);
                        }
                    }
                }
            }
        }
    }
    if (T && loss) {
        lsum = warp_sum(lsum);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    }
    if (PATCH || (T && loss)) __syncthreads();
    if (T && loss && threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(loss, t / ((float)d.height * (float)d.width));
    }
    if (PATCH && T && grad) {
        const int nr = min(kPatch, d.grid_h - pr0), nc = min(kPatch, d.grid_w - pc0);
        for (int k = threadIdx.x; k < kPatch * kPatch; k += blockDim.x) {
            const int pi = k / kPatch, pj = k % kPatch;
            if (pi < nr && pj < nc && patch[k] != 0.0f) atomicAdd(grad + (pr0 + pi) * d.grid_w + pc0 + pj, patch[k]);
        }
    }
}

template <int ORDER>
void launch(const dvgo_fit2d_desc &d, const float *V, const float *T, float *img, float *grad, float *loss,
            cudaStream_t s) {
    const dim3 grid((d.width + kTile - 1) / kTile, (d.height + kTile - 1) / kTile);
    // a 32-pixel span touches at most ceil(31 (g - 1) / n) + 2 lattice points per axis
    const bool patch = (long long)(kTile - 1) * (d.grid_h - 1) <= (long long)(kPatch - 2) * d.height &&
                       (long long)(kTile - 1) * (d.grid_w - 1) <= (long long)(kPatch - 2) * d.width;
    if (patch) fit2d_kernel<ORDER, true><<<grid, 256, 0, s>>>(d, V, T, img, grad, loss);
    else fit2d_kernel<ORDER, false><<<grid, 256, 0, s>>>(d, V, T, img, grad, loss);
}

}  // namespace

}  // namespace dvgo

using namespace dvgo;

extern "C" int dvgo_fit2d(const dvgo_fit2d_desc *d, const float *grid, const float *target, float *image_out,
                          float *grad_grid, float *loss_out, void *stream) {
    if (!d || !grid || d->height < 1 || d->width < 1 || d->grid_h < 2 || d->grid_w < 2) return DVGO_ERR_INVALID_ARG;
    if (d->act_order != DVGO_ACT_POST && d->act_order != DVGO_ACT_PRE && d->act_order != DVGO_ACT_IN)
        return DVGO_ERR_INVALID_ARG;
    if (!isfinite(d->shift_b) || !isfinite(d->delta) || !(d->delta > 0.0f)) return DVGO_ERR_INVALID_ARG;
    if ((long long)d->height * d->width >= (1LL << 31) || (long long)d->grid_h * d->grid_w >= (1LL << 31) ||
        d->height > 65535 * kTile)
        return DVGO_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        ProfScope ps_(DVGO_K_AUX, s);
        if (target && loss_out) cudaMemsetAsync(loss_out, 0, sizeof(float), s);
        if (d->act_order == DVGO_ACT_PRE) launch<DVGO_ACT_PRE>(*d, grid, target, image_out, grad_grid, loss_out, s);
        else if (d->act_order == DVGO_ACT_IN) launch<DVGO_ACT_IN>(*d, grid, target, image_out, grad_grid, loss_out, s);
        else launch<DVGO_ACT_POST>(*d, grid, target, image_out, grad_grid, loss_out, s);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}
