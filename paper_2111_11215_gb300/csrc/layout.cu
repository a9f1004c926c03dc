// layout.cu -- grid storage: element counts, the copy between the canonical channel-last layout and
// the packed one (4x4x4 bricks, Morton order inside a brick) with FP32 / BF16 conversion (one
// thread per (lattice point, channel) of the source lattice), and the trilinear resize of
// progressive scaling (Sec. 4.2; one thread per destination lattice point).

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

struct Axis3 {
    double v[3];
};

// Destination point p -> world position on the destination lattice, clamped into the source box,
// -> trilinear interpolation of the source grid (positions and weights in FP64, the same
// expressions as the interpolation of Sec. 3 Eq. interp: u = (x - min) / (max - min) (n - 1),
// i0 = clamp(floor(u), 0, n - 2), f = u - i0).
__global__ void __launch_bounds__(256) resize_kernel(const float *__restrict__ in, float *__restrict__ out, int C,
                                                     int snx, int sny, int snz, int s_packed, int dnx, int dny,
                                                     int dnz, int d_packed, Axis3 dmin, Axis3 dmax, Axis3 smin,
                                                     Axis3 smax) {
    const long long n = (long long)dnx * dny * dnz;
    const int sn[3] = {snx, sny, snz}, dn[3] = {dnx, dny, dnz};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int ijk[3] = {(int)(p / ((long long)dny * dnz)), (int)((p / dnz) % dny), (int)(p % dnz)};
        int i0[3];
        double f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = dmin.v[a] + (double)ijk[a] * (dmax.v[a] - dmin.v[a]) / (double)(dn[a] - 1);
            x = fmin(fmax(x, smin.v[a]), smax.v[a]);
            const double u = (x - smin.v[a]) / (smax.v[a] - smin.v[a]) * (double)(sn[a] - 1);
            const double fl = fmin(fmax(floor(u), 0.0), (double)(sn[a] - 2));
            i0[a] = (int)fl;
            f[a] = u - fl;
        }
        const long long di = grid_index(ijk[0], ijk[1], ijk[2], dny, dnz, d_packed != 0) * C;
        long long si[8];
        double w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int bx = (q >> 2) & 1, by = (q >> 1) & 1, bz = q & 1;
            si[q] = grid_index(i0[0] + bx, i0[1] + by, i0[2] + bz, sny, snz, s_packed != 0) * C;
            w[q] = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
        }
        for (int ch = 0; ch < C; ++ch) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) acc += w[q] * (double)__ldg(in + si[q] + ch);
            out[di + ch] = (float)acc;
        }
    }
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

int dvgo_resize_grid(const dvgo_grid_desc *src, const float *in, const dvgo_grid_desc *dst, float *out, void *stream) {
    if (!desc_ok(src) || !desc_ok(dst) || !in || !out || in == out) return DVGO_ERR_INVALID_ARG;
    if (src->dtype != DVGO_DTYPE_F32 || dst->dtype != DVGO_DTYPE_F32 || src->channels != dst->channels)
        return DVGO_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(src->xyz_min[a]) || !isfinite(src->xyz_max[a]) || !(src->xyz_max[a] > src->xyz_min[a]) ||
            !isfinite(dst->xyz_min[a]) || !isfinite(dst->xyz_max[a]) || !(dst->xyz_max[a] > dst->xyz_min[a]))
            return DVGO_ERR_INVALID_ARG;
    if (dvgo_grid_elements(src) >= (1ull << 31) || dvgo_grid_elements(dst) >= (1ull << 31)) return DVGO_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Axis3 dmin, dmax, smin, smax;
    for (int a = 0; a < 3; ++a) {
        dmin.v[a] = dst->xyz_min[a];
        dmax.v[a] = dst->xyz_max[a];
        smin.v[a] = src->xyz_min[a];
        smax.v[a] = src->xyz_max[a];
    }
    const long long n = (long long)dst->nx * dst->ny * dst->nz;
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)num_sms() * 16) blocks = (long long)num_sms() * 16;
    {
        ProfScope ps_(DVGO_K_AUX, s);
        if (dst->layout == DVGO_LAYOUT_PACKED) cudaMemsetAsync(out, 0, dvgo_grid_elements(dst) * sizeof(float), s);
        resize_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, src->channels, src->nx, src->ny, src->nz,
                                                       src->layout == DVGO_LAYOUT_PACKED, dst->nx, dst->ny, dst->nz,
                                                       dst->layout == DVGO_LAYOUT_PACKED, dmin, dmax, smin, smax);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // extern "C"
