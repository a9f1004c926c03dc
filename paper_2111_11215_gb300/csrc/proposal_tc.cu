// proposal_tc.cu -- forward of the sample-proposal MLP with BF16 operands on the tensor cores.
//
// Same function as the FP32 proposal forward in proposal.cu (bin-centre encoding, 39 -> 64 -> 64
// -> 64 -> 1 with ReLU, softmax over the 64 bins of a ray, optional cross-entropy against labels),
// for sampling at training speed: the three 64-wide layers are tcgen05 MMAs (M = 128 rows = 2 rays x
// 64 bins, N = 64, BF16 operands in 128-byte-swizzled shared-memory panels, FP32 accumulators in
// TMEM); the 64 -> 1 output layer, the softmax and the loss run on the CUDA cores.  The encoding
// evaluates sin / cos of the FP32 bin centre once per axis and doubles the angle with the identities
// sin 2a = 2 sin a cos a, cos 2a = 1 - 2 sin^2 a for the higher frequencies.
//
// CTA: 128 threads, thread r owns row r of the tile (TMEM lane r); 256 TMEM columns and ~100 KB
// of shared memory, so two CTAs share an SM.

#include <math.h>

#include "dvgo_internal.cuh"
#include "tc_helpers.cuh"

namespace dvgo {

namespace {

using namespace tc;

constexpr int NB = 64, NFQ = 6, PIN = 3 + 6 * NFQ, PW = 64, TT = 128;
constexpr uint32_t COL_Z0 = 0, COL_Z1 = 64, COL_Z2 = 128;

struct alignas(1024) SmallP {
    float b1[PW], b2[PW], w3[PW];
    float b3[4];
    float red[2][2][2];       // per ray: partial max / sum of the two warps
    double t0[2], t1[2], dn[2][3];
    int hit[2];
    uint64_t mbar;
    uint32_t tmem_base;
};

struct SmemP {
    unsigned char w0t[kPanelBytes];   // rows = 64 outputs, 64 input columns (bias in column 39)
    unsigned char w1t[kPanelBytes];
    unsigned char w2t[kPanelBytes];
    unsigned char x[kPanelBytes];
    unsigned char h0[kPanelBytes];
    unsigned char h1[kPanelBytes];
    SmallP sm;
};

struct PropTcArgs {
    int R;
    double mn[3], mx[3], t_near, t_far;
    const float *ro, *rd, *labels;
    const float *w0, *b0, *w1, *b1, *w2, *b2, *w3, *b3;
    float *probs, *loss;
};

__device__ __forceinline__ void sync_fenced() {
    fence_before();
    __syncthreads();
    fence_after();
}

__global__ void __launch_bounds__(TT, 2) proposal_fwd_tc_kernel(PropTcArgs P) {
    extern __shared__ unsigned char smem_raw[];
    SmemP &S = *reinterpret_cast<SmemP *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) mbar_init(&S.sm.mbar, 1);
    if (warp == 0) tmem_alloc(&S.sm.tmem_base, 256);
    if (tid < PW) {
        float v[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = k < PIN ? P.w0[k * PW + tid] : (k == PIN ? P.b0[tid] : 0.0f);
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.w0t, tid, c, v + c);
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = P.w1[k * PW + tid];
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.w1t, tid, c, v + c);
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = P.w2[k * PW + tid];
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.w2t, tid, c, v + c);
        S.sm.b1[tid] = P.b1[tid];
        S.sm.b2[tid] = P.b2[tid];
        S.sm.w3[tid] = P.w3[tid];
    }
    if (tid == 0) S.sm.b3[0] = P.b3[0];
    fence_async_smem();
    sync_fenced();
    const uint32_t tb = S.sm.tmem_base;
    const uint32_t id64 = idesc_bf16(128, 64, 0, 0);
    uint32_t phase = 0;
    bool ok = true;
    const float invR = 1.0f / (float)P.R;
    const int ntiles = (P.R + 1) / 2;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        uint32_t x_ = smem_u32(S.x), w0_ = smem_u32(S.w0t), w1_ = smem_u32(S.w1t), w2_ = smem_u32(S.w2t);
        uint32_t h0_ = smem_u32(S.h0), h1_ = smem_u32(S.h1);
        asm volatile("" : "+r"(x_), "+r"(w0_), "+r"(w1_), "+r"(w2_), "+r"(h0_), "+r"(h1_));
        const int rl = tid >> 6, bin = tid & 63, r = 2 * tile + rl;
        if ((tid & 63) == 0) {
            int hit = 0;
            if (r < P.R) {
                const double o[3] = {(double)P.ro[3 * r], (double)P.ro[3 * r + 1], (double)P.ro[3 * r + 2]};
                const double d[3] = {(double)P.rd[3 * r], (double)P.rd[3 * r + 1], (double)P.rd[3 * r + 2]};
                const Clip c = slab_clip(o, d, P.mn, P.mx, P.t_near, P.t_far);
                hit = c.hi > c.lo;
                S.sm.t0[rl] = c.lo;
                S.sm.t1[rl] = c.hi;
                for (int a = 0; a < 3; ++a) S.sm.dn[rl][a] = c.dn[a];
            }
            S.sm.hit[rl] = hit;
        }
        __syncthreads();
        // ---- encode the bin centre of row tid ----
        {
            float v[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = 0.0f;
            if (S.sm.hit[rl]) {
                const double t0 = S.sm.t0[rl], t1 = S.sm.t1[rl];
                const double tb_ = t0 + ((double)bin + 0.5) * (t1 - t0) / (double)NB;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float x = (float)((double)P.ro[3 * r + a] + tb_ * S.sm.dn[rl][a]);
                    v[a] = x;
                    float s, c;
                    sincosf(x, &s, &c);
#pragma unroll
                    for (int k = 0; k < NFQ; ++k) {
                        v[3 + a * NFQ + k] = s;
                        v[3 + 3 * NFQ + a * NFQ + k] = c;
                        const float s2 = 2.0f * s * c, c2 = 1.0f - 2.0f * s * s;
                        s = s2;
                        c = c2;
                    }
                }
                v[PIN] = 1.0f;
            }
#pragma unroll
            for (int c = 0; c < 64; c += 8) panel_store8(S.x, tid, c, v + c);
        }
        fence_async_smem();
        sync_fenced();
        // ---- layer 0 ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + COL_Z0, desc_kmajor(x_, kk), desc_kmajor(w0_, kk), id64, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z0 + 32 * g), z);
#pragma unroll
            for (int k = 0; k < 32; ++k) z[k] = fmaxf(z[k], 0.0f);
#pragma unroll
            for (int k = 0; k < 32; k += 8) panel_store8(S.h0, tid, 32 * g + k, z + k);
        }
        fence_async_smem();
        sync_fenced();
        // ---- layer 1 ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + COL_Z1, desc_kmajor(h0_, kk), desc_kmajor(w1_, kk), id64, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z1 + 32 * g), z);
#pragma unroll
            for (int k = 0; k < 32; ++k) z[k] = fmaxf(z[k] + S.sm.b1[32 * g + k], 0.0f);
#pragma unroll
            for (int k = 0; k < 32; k += 8) panel_store8(S.h1, tid, 32 * g + k, z + k);
        }
        fence_async_smem();
        sync_fenced();
        // ---- layer 2 and the output logit ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + COL_Z2, desc_kmajor(h1_, kk), desc_kmajor(w2_, kk), id64, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        float lo_a = S.sm.b3[0], lo_b = 0.0f;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z2 + 32 * g), z);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float h = fmaxf(z[k] + S.sm.b2[32 * g + k], 0.0f);
                if (k & 1) lo_b = fmaf(h, S.sm.w3[32 * g + k], lo_b);
                else lo_a = fmaf(h, S.sm.w3[32 * g + k], lo_a);
            }
        }
        const float logit = lo_a + lo_b;
        // ---- softmax over the 64 rows of a ray (two warps) ----
        float m = logit;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) S.sm.red[rl][warp & 1][0] = m;
        __syncthreads();
        m = fmaxf(S.sm.red[rl][0][0], S.sm.red[rl][1][0]);
        const float e = expf(logit - m);
        const float es = warp_sum(e);
        if (lane == 0) S.sm.red[rl][warp & 1][1] = es;
        __syncthreads();
        const float z = S.sm.red[rl][0][1] + S.sm.red[rl][1][1];
        if (r < P.R) {
            const bool hit = S.sm.hit[rl] != 0;
            const float pr = hit ? e / z : 1.0f / NB;
            P.probs[(size_t)r * NB + bin] = pr;
            if (P.labels && P.loss && hit) {
                const float h = P.labels[(size_t)r * NB + bin];
                const float lr = warp_sum(h > 0.0f ? -h * logf(pr) : 0.0f);
                if (lane == 0) atomicAdd(P.loss, lr * invR);
            }
        }
        sync_fenced();
    }
    ok = !__syncthreads_or(!ok);
    if (!ok) mbar_wait(&S.sm.mbar, phase ^ 1);
    sync_fenced();
    if (warp == 0) tmem_dealloc(S.sm.tmem_base, 256);
}

}  // namespace

int launch_proposal_fwd_tc(const dvgo_params &p, const dvgo_grid_desc &g, const dvgo_proposal_mlp &m, int R,
                           const float *ro, const float *rd, const float *labels, float *probs, float *loss,
                           cudaStream_t s) {
    PropTcArgs P;
    P.R = R;
    for (int a = 0; a < 3; ++a) {
        P.mn[a] = g.xyz_min[a];
        P.mx[a] = g.xyz_max[a];
    }
    P.t_near = p.t_near;
    P.t_far = p.t_far;
    P.ro = ro;
    P.rd = rd;
    P.labels = labels;
    P.w0 = m.w0; P.b0 = m.b0; P.w1 = m.w1; P.b1 = m.b1; P.w2 = m.w2; P.b2 = m.b2; P.w3 = m.w3; P.b3 = m.b3;
    P.probs = probs;
    P.loss = loss;
    const int bytes = (int)sizeof(SmemP) + 1024;
    ensure_smem(reinterpret_cast<const void *>(proposal_fwd_tc_kernel), bytes);
    const int ntiles = (R + 1) / 2;
    int blocks = 2 * num_sms();
    if (blocks > ntiles) blocks = ntiles;
    {
        ProfScope ps_(DVGO_K_PROPOSAL_FWD, s);
        proposal_fwd_tc_kernel<<<blocks, TT, bytes, s>>>(P);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // namespace dvgo
