// layout.cu -- grid storage layouts: element counts and the copy between the canonical channel-last
// layout and the packed one (4x4x4 bricks, Morton order inside a brick), with FP32 / BF16
// conversion.  One thread per (lattice point, channel) of the source lattice.

#include <cuda_bf16.h>

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

long long lattice_points(const dvgo_grid_desc &g) {
    if (g.layout == DVGO_LAYOUT_PACKED)
        return (long long)((g.nx + 3) / 4) * ((g.ny + 3) / 4) * ((g.nz + 3) / 4) * 64;
    return (long long)g.nx * g.ny * g.nz;
}

template <typename TIn, typename TOut>
__device__ __forceinline__ TOut convert(TIn v);
template <> __device__ __forceinline__ float convert<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 convert<float, __nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float convert<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ __nv_bfloat16 convert<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 v) { return v; }

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(256) pack_kernel(const TIn *__restrict__ in, TOut *__restrict__ out, int nx, int ny,
                                                   int nz, int C, int src_packed, int dst_packed) {
    const long long n = (long long)nx * ny * nz * C;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(t % C);
        const long long p = t / C;
        const int k = (int)(p % nz), j = (int)((p / nz) % ny), i = (int)(p / ((long long)ny * nz));
        const long long si = grid_index(i, j, k, ny, nz, src_packed != 0) * C + ch;
        const long long di = grid_index(i, j, k, ny, nz, dst_packed != 0) * C + ch;
        out[di] = convert<TIn, TOut>(in[si]);
    }
}

template <typename TIn, typename TOut>
void launch_pack(const dvgo_grid_desc &s, const void *in, const dvgo_grid_desc &d, void *out, cudaStream_t st) {
    const long long n = (long long)s.nx * s.ny * s.nz * s.channels;
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)num_sms() * 16) blocks = (long long)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    pack_kernel<TIn, TOut><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const TIn *>(in), static_cast<TOut *>(out),
                                                             s.nx, s.ny, s.nz, s.channels,
                                                             s.layout == DVGO_LAYOUT_PACKED, d.layout == DVGO_LAYOUT_PACKED);
}

bool desc_ok(const dvgo_grid_desc *g) {
    return g && g->nx >= 2 && g->ny >= 2 && g->nz >= 2 && g->channels >= 1 &&
           (g->layout == DVGO_LAYOUT_CANONICAL || g->layout == DVGO_LAYOUT_PACKED) &&
           (g->dtype == DVGO_DTYPE_F32 || g->dtype == DVGO_DTYPE_BF16);
}

}  // namespace

}  // namespace dvgo

using namespace dvgo;

extern "C" {

size_t dvgo_grid_elements(const dvgo_grid_desc *g) {
    if (!desc_ok(g)) return 0;
    return (size_t)lattice_points(*g) * (size_t)g->channels;
}

int dvgo_pack_grid(const dvgo_grid_desc *src, const void *in, const dvgo_grid_desc *dst, void *out, void *stream) {
    if (!desc_ok(src) || !desc_ok(dst) || !in || !out) return DVGO_ERR_INVALID_ARG;
    if (src->nx != dst->nx || src->ny != dst->ny || src->nz != dst->nz || src->channels != dst->channels)
        return DVGO_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (src->xyz_min[a] != dst->xyz_min[a] || src->xyz_max[a] != dst->xyz_max[a]) return DVGO_ERR_INVALID_ARG;
    if (in == out) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t out_bytes = dvgo_grid_elements(dst) * (dst->dtype == DVGO_DTYPE_BF16 ? 2 : 4);
    {
        ProfScope ps_(DVGO_K_AUX, s);
        if (dst->layout == DVGO_LAYOUT_PACKED) cudaMemsetAsync(out, 0, out_bytes, s);   // padding points
        const bool sb = src->dtype == DVGO_DTYPE_BF16, db = dst->dtype == DVGO_DTYPE_BF16;
        if (!sb && !db) launch_pack<float, float>(*src, in, *dst, out, s);
        else if (!sb && db) launch_pack<float, __nv_bfloat16>(*src, in, *dst, out, s);
        else if (sb && !db) launch_pack<__nv_bfloat16, float>(*src, in, *dst, out, s);
        else launch_pack<__nv_bfloat16, __nv_bfloat16>(*src, in, *dst, out, s);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // extern "C"
