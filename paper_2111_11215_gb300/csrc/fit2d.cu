// fit2d.cu -- the image-fitting toy of Sec. 3 (Fig. exdv_poc): a binary image regressed by a 2D
// grid under the pre-, in- or post-activation order of Eq. pre_in_post (forward, MSE, gradient).
//
// Blocks of 256 threads own 32 x 32-pixel tiles.  A pixel's cell and fraction come from integer
// arithmetic, u = (2i + 1)(g - 1) / (2 H): i0 = the quotient (clamped to g - 2), f = the remainder /
// (2 H) rounded once to FP32, so cell choices are exact.  The gradient of a tile's pixels is summed
// in a shared-memory patch of the grid points the tile touches and added to global memory once per
// point; tiles wider than the patch (grids finer than the image) add straight to global memory.

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
    const int ti = blockIdx.y * kTile, tj = blockIdx.x * kTile;
    const int pr0 = pixel_axis(ti, d.height, d.grid_h).c0, pc0 = pixel_axis(tj, d.width, d.grid_w).c0;
    if (PATCH && grad)
        for (int k = threadIdx.x; k < kPatch * kPatch; k += blockDim.x) patch[k] = 0.0f;
    if (PATCH) __syncthreads();
    const float gscale = 2.0f / ((float)d.height * (float)d.width);
    float lsum = 0.0f;
    for (int k = threadIdx.x; k < kTile * kTile; k += blockDim.x) {
        const int i = ti + k / kTile, j = tj + k % kTile;
        if (i >= d.height || j >= d.width) continue;
        const Axis ay = pixel_axis(i, d.height, d.grid_h), ax = pixel_axis(j, d.width, d.grid_w);
        float w[4], v[4], dadv[4], alpha;
        int idx[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int bi = (q >> 1) & 1, bj = q & 1;
            idx[q] = (ay.c0 + bi) * d.grid_w + ax.c0 + bj;
            w[q] = (bi ? ay.f : 1.0f - ay.f) * (bj ? ax.f : 1.0f - ax.f);
            v[q] = __ldg(V + idx[q]);
        }
        if (ORDER == DVGO_ACT_PRE) {
            alpha = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float e = expf(-softplusf(v[q] + d.shift_b) * d.delta);
                alpha = fmaf(w[q], 1.0f - e, alpha);
                dadv[q] = w[q] * d.delta * e * sigmoidf_(v[q] + d.shift_b);
            }
        } else if (ORDER == DVGO_ACT_IN) {
            float sigma = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) sigma = fmaf(w[q], softplusf(v[q] + d.shift_b), sigma);
            const float e = expf(-sigma * d.delta);
            alpha = -expm1f(-sigma * d.delta);
#pragma unroll
            for (int q = 0; q < 4; ++q) dadv[q] = d.delta * e * w[q] * sigmoidf_(v[q] + d.shift_b);
        } else {
            float z = d.shift_b;
#pragma unroll
            for (int q = 0; q < 4; ++q) z = fmaf(w[q], v[q], z);
            const float sigma = softplusf(z), e = expf(-sigma * d.delta);
            alpha = -expm1f(-sigma * d.delta);
            const float s = d.delta * e * sigmoidf_(z);
#pragma unroll
            for (int q = 0; q < 4; ++q) dadv[q] = s * w[q];
        }
        if (img) img[(long long)i * d.width + j] = alpha;
        if (T) {
            const float r = alpha - __ldg(T + (long long)i * d.width + j);
            lsum = fmaf(r, r, lsum);
            if (grad) {
                const float g = gscale * r;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (dadv[q] == 0.0f) continue;
                    if (PATCH) {
                        const int pi = ay.c0 + ((q >> 1) & 1) - pr0, pj = ax.c0 + (q & 1) - pc0;
                        atomicAdd(&patch[pi * kPatch + pj], g * dadv[q]);
                    } else {
                        atomicAdd(grad + idx[q], g * dadv[q]);
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
