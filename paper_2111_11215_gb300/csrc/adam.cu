// adam.cu -- elementwise Adam step (Kingma & Ba) used for the grids and the MLP (Sec. 5.2,
// Supp. A: Adam, base learning rates 0.1 for the voxel grids and 1e-3 for the MLP, decayed
// exponentially by 0.1 over 20k iterations; Sec. 4.1 Prior 2: a per-voxel rate scale).
//
// HBM-bound: per element it reads p, g, m, v (16 B) and writes p, m, v and, with zero_grad, g where
// it is not already zero (12-16 B), plus 2 B for the optional BF16 copy.  16-byte vector loads/stores, grid-stride
// loop over a grid sized to fill every SM.  The lazy variant reads the gradient first and leaves
// a 4-element vector whose gradients are all zero untouched (4 B of traffic per element there);
// inside a vector it updates only the elements with a nonzero gradient.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

struct AdamK {
    float lr, b1, b2, eps, inv_bc1, inv_bc2;
};

__device__ __forceinline__ void adam_one(float &p, float &m, float &v, float g, float s, const AdamK &k) {
    m = fmaf(k.b1, m, (1.0f - k.b1) * g);
    v = fmaf(k.b2, v, (1.0f - k.b2) * g * g);
    float mhat = m * k.inv_bc1, vhat = v * k.inv_bc2;
    p -= k.lr * s * mhat / (sqrtf(vhat) + k.eps);
}

__device__ __forceinline__ void adam_lazy(float &p, float &m, float &v, float g, float s, const AdamK &k) {
    if (g != 0.0f) adam_one(p, m, v, g, s, k);
}

// Launch shape: blocks of 256 threads, at most DVGO_ADAM_BLOCKS_PER_SM per SM in the grid, and
// DVGO_ADAM_UNROLL 4-element vectors per thread in flight per iteration of the dense variant.  Three
// blocks per SM is one wave (the kernel's registers allow four) that keeps the copy-rate bound and
// leaves a quarter of each SM's threads and a third of its registers to kernels of other streams.
// DVGO_ADAM_CARVEOUT (percent, -1 = the driver's choice) is the kernel's preferred shared-memory
// carveout.  The driver's choice gives the loads in flight the whole L1: a carveout of 100 %
// (room for concurrent kernels that use shared memory) costs the kernel 15 % of its rate.
#ifndef DVGO_ADAM_BLOCKS_PER_SM
#define DVGO_ADAM_BLOCKS_PER_SM 3
#endif
#ifndef DVGO_ADAM_UNROLL
#define DVGO_ADAM_UNROLL 1
#endif
#ifndef DVGO_ADAM_CARVEOUT
#define DVGO_ADAM_CARVEOUT -1
#endif
// A tensor of at most DVGO_ADAM_SMALL_VECS 4-vectors (the density grid, the MLP) runs with nothing
// beside it at the end of a step, so it takes the larger grid of DVGO_ADAM_SMALL_BLOCKS_PER_SM
// blocks per SM (of which the registers let 4 be resident) and DVGO_ADAM_SMALL_UNROLL vectors per
// thread per iteration: 8 / 1 measured 2 us per step faster than the big sweep's 3 / 1, and 4 or 2
// vectors per thread (116-118 registers) no faster.
#ifndef DVGO_ADAM_SMALL_VECS
#define DVGO_ADAM_SMALL_VECS (1 << 21)
#endif
#ifndef DVGO_ADAM_SMALL_UNROLL
#define DVGO_ADAM_SMALL_UNROLL 1
#endif
#ifndef DVGO_ADAM_SMALL_BLOCKS_PER_SM
#define DVGO_ADAM_SMALL_BLOCKS_PER_SM 8
#endif

// DVGO_ADAM_BF16_EVICT_LAST: the BF16 copy of the features (read by the colour kernels' gathers right
// after the step's Adam) is stored with an L2 evict-last policy, so that the parameters' and moments'
// traffic of the same sweep evicts it last (proposal-step colour forward 58 -> 55 us, the sweep a few
// us slower, the step 0.5 % faster).
#ifndef DVGO_ADAM_BF16_EVICT_LAST
#define DVGO_ADAM_BF16_EVICT_LAST 1
#endif

__device__ __forceinline__ void st_bf16x4(uint2 *a, uint2 o) {
#if DVGO_ADAM_BF16_EVICT_LAST
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;" ::"l"(a), "r"(o.x), "r"(o.y), "l"(pol)
                 : "memory");
#else
    *a = o;
#endif
}

// zero_grad: the gradient vector G read for this update is cleared; a vector that is already zero
// (a lattice point no sample touched) is not written again.
__device__ __forceinline__ void adam_store(float4 *p4, float4 *m4, float4 *v4, float4 *g4, uint2 *pb4, size_t i,
                                           const float4 &P, const float4 &M, const float4 &V, const float4 &G,
                                           int zero_grad) {
    p4[i] = P;
    m4[i] = M;
    v4[i] = V;
    if (zero_grad && (G.x != 0.0f || G.y != 0.0f || G.z != 0.0f || G.w != 0.0f))
        g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pb4) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
        uint2 o;
        o.x = *reinterpret_cast<unsigned *>(&lo);
        o.y = *reinterpret_cast<unsigned *>(&hi);
        st_bf16x4(pb4 + i, o);
    }
}

// Dense variant with U vectors per thread per iteration: all loads of an iteration are issued
// before the first update.
template <int U>
__device__ __forceinline__ void adam_dense_vec(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                                               float *__restrict__ v, size_t n4, const AdamK &k,
                                               const float *__restrict__ scale, uint16_t *__restrict__ pb,
                                               int zero_grad) {
    float4 *p4 = reinterpret_cast<float4 *>(p), *g4 = reinterpret_cast<float4 *>(g);
    float4 *m4 = reinterpret_cast<float4 *>(m), *v4 = reinterpret_cast<float4 *>(v);
    const float4 *s4 = reinterpret_cast<const float4 *>(scale);
    uint2 *pb4 = reinterpret_cast<uint2 *>(pb);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n4; i0 += stride * U) {
        float4 G[U], P[U], M[U], V[U], S[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            if (i < n4) {
                G[u] = g4[i];
                P[u] = p4[i];
                M[u] = m4[i];
                V[u] = v4[i];
                S[u] = s4 ? s4[i] : make_float4(1.f, 1.f, 1.f, 1.f);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            if (i < n4) {
                adam_one(P[u].x, M[u].x, V[u].x, G[u].x, S[u].x, k);
                adam_one(P[u].y, M[u].y, V[u].y, G[u].y, S[u].y, k);
                adam_one(P[u].z, M[u].z, V[u].z, G[u].z, S[u].z, k);
                adam_one(P[u].w, M[u].w, V[u].w, G[u].w, S[u].w, k);
                adam_store(p4, m4, v4, g4, pb4, i, P[u], M[u], V[u], G[u], zero_grad);
            }
        }
    }
}

template <bool LAZY, int U>
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                                                    float *__restrict__ v, size_t n, AdamK k,
                                                    const float *__restrict__ scale, uint16_t *__restrict__ pb,
                                                    int zero_grad) {
    size_t n4 = n / 4;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    if constexpr (!LAZY) {
        adam_dense_vec<U>(p, g, m, v, n4, k, scale, pb, zero_grad);
    } else {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 G = reinterpret_cast<const float4 *>(g)[i];
            if (G.x == 0.0f && G.y == 0.0f && G.z == 0.0f && G.w == 0.0f) continue;
            float4 P = reinterpret_cast<float4 *>(p)[i];
            float4 M = reinterpret_cast<float4 *>(m)[i];
            float4 V = reinterpret_cast<float4 *>(v)[i];
            const float4 S = scale ? reinterpret_cast<const float4 *>(scale)[i] : make_float4(1.f, 1.f, 1.f, 1.f);
            adam_lazy(P.x, M.x, V.x, G.x, S.x, k);
            adam_lazy(P.y, M.y, V.y, G.y, S.y, k);
            adam_lazy(P.z, M.z, V.z, G.z, S.z, k);
            adam_lazy(P.w, M.w, V.w, G.w, S.w, k);
            adam_store(reinterpret_cast<float4 *>(p), reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v),
                       reinterpret_cast<float4 *>(g), reinterpret_cast<uint2 *>(pb), i, P, M, V, G, zero_grad);
        }
    }
    // scalar tail
    for (size_t i = n4 * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (LAZY && g[i] == 0.0f) continue;
        float P = p[i], M = m[i], V = v[i];
        adam_one(P, M, V, g[i], scale ? scale[i] : 1.0f, k);
        p[i] = P;
        m[i] = M;
        v[i] = V;
        if (zero_grad && g[i] != 0.0f) g[i] = 0.0f;
        if (pb) {
            __nv_bfloat16 b = __float2bfloat16_rn(P);
            pb[i] = *reinterpret_cast<uint16_t *>(&b);
        }
    }
}


// Several tensors in one launch: the vectors of all tensors form one index range (tensor j owns
// [off[j], off[j + 1])), swept grid-stride one vector per thread per iteration; then the scalar
// tails.  Every element goes through adam_one / adam_lazy and adam_store as in adam_kernel.
struct AdamTensorK {
    float *p, *g, *m, *v;
    const float *scale;
    uint16_t *pb;
    size_t n;
    AdamK k;
    int zero_grad, lazy;
};
struct AdamMultiK {
    AdamTensorK t[DVGO_ADAM_MAX_TENSORS];
    size_t off[DVGO_ADAM_MAX_TENSORS + 1];   // vector offsets
    int nt;
};

__global__ void __launch_bounds__(256) adam_multi_kernel(AdamMultiK a) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t total = a.off[a.nt];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        int j = 0;
#pragma unroll
        for (int q = 1; q < DVGO_ADAM_MAX_TENSORS; ++q) j += (q < a.nt && i >= a.off[q]) ? 1 : 0;
        const AdamTensorK &t = a.t[j];
        const size_t li = i - a.off[j];
        float4 *p4 = reinterpret_cast<float4 *>(t.p), *g4 = reinterpret_cast<float4 *>(t.g);
        float4 *m4 = reinterpret_cast<float4 *>(t.m), *v4 = reinterpret_cast<float4 *>(t.v);
        const float4 G = g4[li];
        if (t.lazy && G.x == 0.0f && G.y == 0.0f && G.z == 0.0f && G.w == 0.0f) continue;
        float4 P = p4[li], M = m4[li], V = v4[li];
        const float4 S = t.scale ? reinterpret_cast<const float4 *>(t.scale)[li] : make_float4(1.f, 1.f, 1.f, 1.f);
        if (t.lazy) {
            adam_lazy(P.x, M.x, V.x, G.x, S.x, t.k);
            adam_lazy(P.y, M.y, V.y, G.y, S.y, t.k);
            adam_lazy(P.z, M.z, V.z, G.z, S.z, t.k);
            adam_lazy(P.w, M.w, V.w, G.w, S.w, t.k);
        } else {
            adam_one(P.x, M.x, V.x, G.x, S.x, t.k);
            adam_one(P.y, M.y, V.y, G.y, S.y, t.k);
            adam_one(P.z, M.z, V.z, G.z, S.z, t.k);
            adam_one(P.w, M.w, V.w, G.w, S.w, t.k);
        }
        adam_store(p4, m4, v4, g4, reinterpret_cast<uint2 *>(t.pb), li, P, M, V, G, t.zero_grad);
    }
    // scalar tails (n % 4 elements of each tensor)
    for (int j = 0; j < a.nt; ++j) {
        const AdamTensorK &t = a.t[j];
        for (size_t i = (t.n / 4) * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < t.n; i += stride) {
            if (t.lazy && t.g[i] == 0.0f) continue;
            float P = t.p[i], M = t.m[i], V = t.v[i];
            adam_one(P, M, V, t.g[i], t.scale ? t.scale[i] : 1.0f, t.k);
            t.p[i] = P;
            t.m[i] = M;
            t.v[i] = V;
            if (t.zero_grad && t.g[i] != 0.0f) t.g[i] = 0.0f;
            if (t.pb) {
                __nv_bfloat16 b = __float2bfloat16_rn(P);
                t.pb[i] = *reinterpret_cast<uint16_t *>(&b);
            }
        }
    }
}

AdamK adam_constants(const dvgo_adam_hparams &h) {
    AdamK k;
    k.lr = h.lr;
    k.b1 = h.beta1;
    k.b2 = h.beta2;
    k.eps = h.eps;
    k.inv_bc1 = (float)(1.0 / (1.0 - pow((double)h.beta1, (double)h.step)));
    k.inv_bc2 = (float)(1.0 / (1.0 - pow((double)h.beta2, (double)h.step)));
    return k;
}

}  // namespace

void launch_adam(float *param, float *grad, float *m, float *v, size_t n, const dvgo_adam_hparams &h,
                 const float *lr_scale, uint16_t *bf16_out, int zero_grad, cudaStream_t s) {
    const AdamK k = adam_constants(h);
    size_t n4 = (n + 3) / 4;
    const bool small = n4 <= (size_t)DVGO_ADAM_SMALL_VECS;
    size_t blocks = (n4 + 255) / 256;
    size_t cap = (size_t)num_sms() * (small ? DVGO_ADAM_SMALL_BLOCKS_PER_SM : DVGO_ADAM_BLOCKS_PER_SM);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (DVGO_ADAM_CARVEOUT >= 0) {
        static bool once = [] {
            cudaFuncSetAttribute(reinterpret_cast<const void *>(adam_kernel<false, DVGO_ADAM_UNROLL>),
                                 cudaFuncAttributePreferredSharedMemoryCarveout, DVGO_ADAM_CARVEOUT);
            cudaFuncSetAttribute(reinterpret_cast<const void *>(adam_kernel<true, 1>),
                                 cudaFuncAttributePreferredSharedMemoryCarveout, DVGO_ADAM_CARVEOUT);
            return true;
        }();
        (void)once;
    }
    {
        ProfScope ps_(DVGO_K_ADAM, s);
        if (h.skip_zero_grad)
            adam_kernel<true, 1><<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, k, lr_scale, bf16_out, zero_grad);
        else if (small)
            adam_kernel<false, DVGO_ADAM_SMALL_UNROLL><<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, k,
                                                                                        lr_scale, bf16_out, zero_grad);
        else
            adam_kernel<false, DVGO_ADAM_UNROLL><<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, k, lr_scale,
                                                                                  bf16_out, zero_grad);
    }
}

void launch_adam_multi(const dvgo_adam_tensor *t, int nt, cudaStream_t s) {
    AdamMultiK a{};
    a.nt = nt;
    a.off[0] = 0;
    for (int j = 0; j < nt; ++j) {
        a.t[j] = AdamTensorK{t[j].param, t[j].grad, t[j].m, t[j].v, t[j].lr_scale, t[j].param_bf16_out,
                             t[j].n, adam_constants(t[j].h), t[j].zero_grad, t[j].h.skip_zero_grad};
        a.off[j + 1] = a.off[j] + t[j].n / 4;
    }
    const size_t total = a.off[nt];
    const bool small = total <= (size_t)DVGO_ADAM_SMALL_VECS;
    size_t blocks = (total + 255) / 256;
    const size_t cap = (size_t)num_sms() * (small ? DVGO_ADAM_SMALL_BLOCKS_PER_SM : DVGO_ADAM_BLOCKS_PER_SM);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    ProfScope ps_(DVGO_K_ADAM, s);
    adam_multi_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
}

}  // namespace dvgo
