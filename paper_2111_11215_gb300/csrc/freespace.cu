// freespace.cu -- fine voxels allocation of Sec. 4.2: the box of the coarse grid's cells that can
// hold unknown space (alpha_c >= tau_c).
//
// One pass over the coarse lattice: each thread tests its lattice points (FP32 activation, the
// same expression as the per-sample test of the fine density kernel), reduces its count and
// index extremes over the warp, and one lane per warp updates the 7-int result with atomics; a
// final single-thread kernel widens the extremes by one cell and clamps them to the lattice.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

__global__ void bbox_init_kernel(int *out) {
    if (threadIdx.x == 0) {
        out[0] = 0;
        for (int a = 0; a < 3; ++a) {
            out[1 + a] = INT_MAX;
            out[4 + a] = -1;
        }
    }
}

__global__ void __launch_bounds__(256) bbox_scan_kernel(const float *__restrict__ v, int nx, int ny, int nz, float b,
                                                        float step, float tau, int packed, int *out) {
    const long long n = (long long)nx * ny * nz;
    int cnt = 0, lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % nz), j = (int)((i / nz) % ny), ii = (int)(i / ((long long)ny * nz));
        const float alpha = -expm1f(-softplusf(__ldg(v + grid_index(ii, j, k, ny, nz, packed != 0)) + b) * step);
        if (alpha < tau) continue;   // known free
        const int ijk[3] = {ii, j, k};
        ++cnt;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], ijk[a]);
            hi[a] = max(hi[a], ijk[a]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0) {
        atomicAdd(out, cnt);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(out + 1 + a, lo[a]);
            atomicMax(out + 4 + a, hi[a]);
        }
    }
}

__global__ void bbox_finish_kernel(int nx, int ny, int nz, int *out) {
    if (threadIdx.x != 0 || out[0] == 0) return;
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        out[1 + a] = max(out[1 + a] - 1, 0);
        out[4 + a] = min(out[4 + a] + 1, n[a] - 1);
    }
}

}  // namespace

}  // namespace dvgo

using namespace dvgo;

extern "C" int dvgo_unknown_bbox(const dvgo_freespace *fs, int *out, void *stream) {
    if (!fs || !fs->density || !out) return DVGO_ERR_INVALID_ARG;
    const dvgo_grid_desc &g = fs->desc;
    if (g.nx < 2 || g.ny < 2 || g.nz < 2 || g.channels != 1 || g.dtype != DVGO_DTYPE_F32) return DVGO_ERR_INVALID_ARG;
    if (g.layout != DVGO_LAYOUT_CANONICAL && g.layout != DVGO_LAYOUT_PACKED) return DVGO_ERR_INVALID_ARG;
    if (!(fs->step > 0.0f) || !isfinite(fs->step) || !isfinite(fs->shift_b) || !isfinite(fs->tau))
        return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = (long long)g.nx * g.ny * g.nz;
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)num_sms() * 8) blocks = (long long)num_sms() * 8;
    {
        ProfScope ps_(DVGO_K_AUX, s);
        bbox_init_kernel<<<1, 32, 0, s>>>(out);
        bbox_scan_kernel<<<(unsigned)blocks, 256, 0, s>>>(fs->density, g.nx, g.ny, g.nz, fs->shift_b, fs->step, fs->tau,
                                                         g.layout == DVGO_LAYOUT_PACKED, out);
        bbox_finish_kernel<<<1, 32, 0, s>>>(g.nx, g.ny, g.nz, out);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}
