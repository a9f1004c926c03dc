// touched.cu -- exact counts of the lattice points one fine-stage render reads: the density grid's
// points at the corners of every sample outside the known free space that the density pass did
// not terminate (a terminated sample's slot holds tau = +inf), and the feature grid's points at
// the corners of every kept sample (the sizes behind the minimum HBM bytes of a step).
//
// Runs after a forward on its workspace: the per-ray records give every sample's fixed-point
// position (uniform or explicit), the compact list gives the kept samples.  One bit per lattice
// point (canonical index, whatever the storage layout), set with atomicOr; then a population
// count.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

__device__ __forceinline__ void mark_cell(uint32_t *bm, const Cell &c, int ny, int nz) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long long p = corner_index(c, q, ny, nz, false);
        atomicOr(bm + (p >> 5), 1u << (unsigned)(p & 31));
    }
}

// Warp per ray, lanes over its samples.
__global__ void __launch_bounds__(256) touched_density_kernel(RenderArgs A, uint32_t *bm) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int ray = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ray < A.R; ray += nwarps) {
        const RayRec &rr = A.rays[ray];
        for (int k = lane; k < rr.n; k += 32) {
            long long u[3];
            float dt;
            if (isinf(A.samp[rr.off + k].x)) break;   // terminated: this and every later sample
            sample_fx(A, rr, ray, k, dt, u);
            if (A.fs_density && known_free(A, u)) continue;
            mark_cell(bm, cell_from_fx(u, A.nx, A.ny, A.nz), A.ny, A.nz);
        }
    }
}

// Thread per kept sample.
__global__ void __launch_bounds__(256) touched_feat_kernel(RenderArgs A, uint32_t *bm) {
    const int n_kept = A.hdr->n_kept;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_kept; e += gridDim.x * blockDim.x) {
        const int2 kv = A.kept[e];
        const RayRec &rr = A.rays[kv.y];
        float dt;
        mark_cell(bm, sample_cell(A, rr, kv.y, kv.x - rr.off, dt), A.ny, A.nz);
    }
}

__global__ void __launch_bounds__(256) popcount_kernel(const uint32_t *__restrict__ bm, long long words,
                                                       unsigned long long *count) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (long long)gridDim.x * blockDim.x)
        c += __popc(bm[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

void launch_touched(const RenderArgs &A, uint32_t *bitmaps, unsigned long long *counts, cudaStream_t s) {
    const long long words = ((long long)A.nx * A.ny * A.nz + 31) / 32;
    ProfScope ps_(DVGO_K_AUX, s);
    cudaMemsetAsync(bitmaps, 0, (size_t)(2 * words) * sizeof(uint32_t), s);
    cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    const int blocks = num_sms() * 8;
    touched_density_kernel<<<blocks, 256, 0, s>>>(A, bitmaps);
    touched_feat_kernel<<<blocks, 256, 0, s>>>(A, bitmaps + words);
    popcount_kernel<<<blocks, 256, 0, s>>>(bitmaps, words, counts);
    popcount_kernel<<<blocks, 256, 0, s>>>(bitmaps + words, words, counts + 1);
}

}  // namespace dvgo
