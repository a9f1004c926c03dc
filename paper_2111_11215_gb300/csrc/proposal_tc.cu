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
// Forward CTA: 128 threads, thread r owns row r of the tile (TMEM lane r); one 64-column TMEM
// accumulator used by the three layers in turn and ~57 KB of shared memory (64-row weight panels,
// H1 written over X), so three CTAs share an SM.
//
// The backward recomputes the forward the same way and then runs every contraction of the chain
// rule on the tensor cores: dH1 = dZ2 W2^T and dH0 = dZ1 W1^T (the transposed weight panels of
// the forward read MN-major), and the weight gradients dW_l = H_l^T dZ_{l+1}, reduced over the 128
// rows of the tile, with the H and dZ panels read MN-major.  Those are M = 128 MMAs whose upper 64
// rows of A are a constant panel E (column 0 = 1), so row 64 of each accumulator is the column sum
// of dZ, i.e. the bias gradient.  The gradients accumulate in TMEM over all tiles of the CTA and
// are added to global memory once.  dW3 / db3 come the same way from a panel holding dlogit in
// column 0.  One CTA per SM (512 TMEM columns, ~180 KB of shared memory).

#include <math.h>

#include "df64.cuh"
#include "dvgo_internal.cuh"
#include "tc_helpers.cuh"

namespace dvgo {

namespace {

using namespace tc;

constexpr int NB = 64, NFQ = 6, PIN = 3 + 6 * NFQ, PW = 64, TT = 128;
// Forward TMEM: the three layers use one accumulator (64 columns at COL_Z) in turn; their A operand
// (X, then H0, then H1, BF16 packed two per column: 32 columns at COL_A) is written there too.
constexpr uint32_t COL_Z = 0, COL_A = 64, FWD_COLS = 128;
constexpr int kFwdCtasPerSm = 4;   // 4 x 128 TMEM columns

// Box clip of one ray as the encoding uses it: entry t0, bin width w = (t_exit - t_enter) / 64 and
// direction as double-float values of the FP64 clip, the origin, and whether the ray hits the box.
struct ClipDf {
    Df t0, w, dn[3];
    float o[3];
    int hit;
};

constexpr int kClipTiles = TT / 2;   // tiles per clip pass: one ray per thread

struct alignas(1024) SmallP {
    alignas(16) float b1[PW];
    alignas(16) float b2[PW];
    alignas(16) float w3[PW];
    float b3[4];
    float red[2][2][2];       // per ray: partial max / sum of the two warps
    ClipDf clip[TT];          // rays of the CTA's current 64 tiles
    uint64_t mbar;
    uint32_t tmem_base;
};

constexpr uint32_t kHalfPanelBytes = kPanelBytes / 2;   // 64 rows: a K-major operand of N = 64

// The forward's shared memory: the weights and the small state (the activations stay in TMEM).
struct SmemP {
    unsigned char w0t[kHalfPanelBytes];   // rows = 64 outputs, 64 input columns (bias in column 39)
    unsigned char w1t[kHalfPanelBytes];
    unsigned char w2t[kHalfPanelBytes];
    SmallP sm;
};
// Dynamic shared memory the forward requests: more than it uses, so that exactly kFwdCtasPerSm
// CTAs fit on an SM (228 KB, 1 KB reserved per CTA) and their TMEM columns add up to 512.
constexpr int kFwdSmemBytes = 50 * 1024;
static_assert(sizeof(SmemP) + 1024 <= kFwdSmemBytes, "forward shared memory");
static_assert(kFwdCtasPerSm * (kFwdSmemBytes + 1024) <= 233472 &&
              (kFwdCtasPerSm + 1) * (kFwdSmemBytes + 1024) > 233472, "CTAs per SM");
static_assert(kFwdCtasPerSm * FWD_COLS == 512, "TMEM columns per SM");

struct PropTcArgs {
    int R;
    double mn[3], mx[3], t_near, t_far;
    const float *ro, *rd, *labels;
    const float *w0, *b0, *w1, *b1, *w2, *b2, *w3, *b3;
    float *probs, *loss;
    float *grad;    // backward: w0 | b0 | w1 | b1 | w2 | b2 | w3 | b3
};

__device__ __forceinline__ void sync_fenced() {
    fence_before();
    __syncthreads();
    fence_after();
}

// W0^T | b0 (bias in input column 39), W1^T, W2^T as K-major BF16 panels (rows = outputs) and the
// FP32 vectors b1, b2, w3, b3.
__device__ __forceinline__ void load_weights(const PropTcArgs &P, unsigned char *w0t, unsigned char *w1t,
                                             unsigned char *w2t, float *b1, float *b2, float *w3, float *b3) {
    const int tid = threadIdx.x;
    if (tid < PW) {
        float v[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = k < PIN ? P.w0[k * PW + tid] : (k == PIN ? P.b0[tid] : 0.0f);
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(w0t, tid, c, v + c);
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = P.w1[k * PW + tid];
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(w1t, tid, c, v + c);
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = P.w2[k * PW + tid];
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(w2t, tid, c, v + c);
        b1[tid] = P.b1[tid];
        b2[tid] = P.b2[tid];
        w3[tid] = P.w3[tid];
    }
    if (tid == 0) b3[0] = P.b3[0];
}

// Box clips (FP64, as in the renderer) of the rays of the CTA's tiles k0 .. k0 + 63 (its k-th tile
// is blockIdx.x + k gridDim.x, rays 2 tile and 2 tile + 1), one ray per thread.  Clipping per ray
// instead of per tile keeps the FP64 work (1/64 of the FP32 rate on this GPU) off the tile loop.
__device__ __forceinline__ void clip_pass(const PropTcArgs &P, int k0, ClipDf *cl) {
    const int tid = threadIdx.x;
    const long long tile = blockIdx.x + (long long)(k0 + (tid >> 1)) * gridDim.x, r = 2 * tile + (tid & 1);
    ClipDf c;
    c.t0 = c.w = c.dn[0] = c.dn[1] = c.dn[2] = Df{0.0f, 0.0f};
    c.o[0] = c.o[1] = c.o[2] = 0.0f;
    c.hit = 0;
    if (r < P.R) {
        const double o[3] = {(double)P.ro[3 * r], (double)P.ro[3 * r + 1], (double)P.ro[3 * r + 2]};
        const double d[3] = {(double)P.rd[3 * r], (double)P.rd[3 * r + 1], (double)P.rd[3 * r + 2]};
        const Clip q = slab_clip(o, d, P.mn, P.mx, P.t_near, P.t_far);
        c.hit = q.hi > q.lo;
        if (c.hit) {
            c.t0 = df_from_double(q.lo);
            c.w = df_from_double(__ddiv_rn(__dsub_rn(q.hi, q.lo), (double)NB));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                c.dn[a] = df_from_double(q.dn[a]);
                c.o[a] = P.ro[3 * r + a];
            }
        }
    }
    cl[tid] = c;
}

// Input row of this thread's bin centre (zeros for a ray that misses or does not exist).  The bin
// centre t_b = t0 + (b + 1/2) w and the position x = o + t_b d are double-float, so x is the FP32
// rounding of the exact position (up to ties within ~1e-14).
__device__ __forceinline__ void encode_values(const ClipDf &c, float (&v)[64]) {
    const int tid = threadIdx.x, bin = tid & 63;
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = 0.0f;
    if (c.hit) {
        const Df tb = df_add(c.t0, df_mul_f(c.w, (float)bin + 0.5f));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xa = df_add(Df{c.o[a], 0.0f}, df_mul(tb, c.dn[a])).hi;
            v[a] = xa;
            float sn, cs;
            sincosf(xa, &sn, &cs);
#pragma unroll
            for (int k = 0; k < NFQ; ++k) {
                v[3 + a * NFQ + k] = sn;
                v[3 + 3 * NFQ + a * NFQ + k] = cs;
                const float s2 = 2.0f * sn * cs, c2 = 1.0f - 2.0f * sn * sn;
                sn = s2;
                cs = c2;
            }
        }
        v[PIN] = 1.0f;
    }
}

// ... into the X panel (the backward, whose dW0 reads X as an MN-major operand)
__device__ __forceinline__ void encode_row(const ClipDf &c, unsigned char *x) {
    float v[64];
    encode_values(c, v);
#pragma unroll
    for (int c8 = 0; c8 < 64; c8 += 8) panel_store8(x, threadIdx.x, c8, v + c8);
}

// ... as BF16 into this thread's TMEM lane at column ta (the forward)
__device__ __forceinline__ void encode_row_tmem(const ClipDf &c, uint32_t ta) {
    float v[64];
    encode_values(c, v);
    uint32_t w[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = pack_bf16(v[32 * h + 2 * k], v[32 * h + 2 * k + 1]);
        tmem_st16(ta + 16u * (uint32_t)h, w);
    }
}

// Epilogue: 32-column chunk g of the accumulator (+ bias), ReLU, as BF16 into the A-operand
// columns 16 g .. 16 g + 15 of this thread's TMEM lane.
__device__ __forceinline__ void relu_to_tmem(uint32_t tz, uint32_t ta, const float *bias) {
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        float z[32];
        tmem_ld32(tz + 32u * (uint32_t)g, z);
        uint32_t h[16];
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
            float4 bb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (bias) bb = *reinterpret_cast<const float4 *>(bias + 32 * g + k);
            h[k / 2] = pack_bf16(fmaxf(z[k] + bb.x, 0.0f), fmaxf(z[k + 1] + bb.y, 0.0f));
            h[k / 2 + 1] = pack_bf16(fmaxf(z[k + 2] + bb.z, 0.0f), fmaxf(z[k + 3] + bb.w, 0.0f));
        }
        tmem_st16(ta + 16u * (uint32_t)g, h);
    }
    tmem_wait_st();
}

__global__ void __launch_bounds__(TT, kFwdCtasPerSm) proposal_fwd_tc_kernel(PropTcArgs P) {
    extern __shared__ unsigned char smem_raw[];
    SmemP &S = *reinterpret_cast<SmemP *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) mbar_init(&S.sm.mbar, 1);
    if (warp == 0) tmem_alloc(&S.sm.tmem_base, FWD_COLS);
    load_weights(P, S.w0t, S.w1t, S.w2t, S.sm.b1, S.sm.b2, S.sm.w3, S.sm.b3);
    fence_async_smem();
    sync_fenced();
    const uint32_t tb = S.sm.tmem_base;
    const uint32_t tz = taddr(tb, warp, COL_Z), ta = taddr(tb, warp, COL_A);   // this warp's lanes
    const uint32_t id64 = idesc_bf16(128, 64, 0, 0);
    uint32_t phase = 0;
    bool ok = true;
    const float invR = 1.0f / (float)P.R;
    const int ntiles = (P.R + 1) / 2;
    int k = 0;
    // one layer: D (COL_Z) = A (COL_A, TMEM) x W^T (K = 64: four k-steps of 8 columns), then wait
    auto layer = [&](unsigned char *wt) -> bool {
        if (tid == 0) {
            uint32_t w_ = smem_u32(wt);
            asm volatile("" : "+r"(w_));
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk)
                mma_ts(tb + COL_Z, tb + COL_A + 8u * (uint32_t)kk, desc_kmajor(w_, kk), id64, kk > 0);
            commit(&S.sm.mbar);
        }
        const bool w = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        const bool all = !__syncthreads_or(!w);
        fence_after();
        return all;
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++k) {
        const int rl = tid >> 6, bin = tid & 63, r = 2 * tile + rl;
        if (k % kClipTiles == 0) {
            clip_pass(P, k, S.sm.clip);
            __syncthreads();
        }
        const bool hit = S.sm.clip[2 * (k % kClipTiles) + rl].hit != 0;
        encode_row_tmem(S.sm.clip[2 * (k % kClipTiles) + rl], ta);
        tmem_wait_st();
        sync_fenced();
        // ---- layer 0, H0 = relu(Z) over X ----
        if (!(ok = layer(S.w0t))) break;
        relu_to_tmem(tz, ta, nullptr);
        sync_fenced();
        // ---- layer 1, H1 = relu(Z + b1) over H0 ----
        if (!(ok = layer(S.w1t))) break;
        relu_to_tmem(tz, ta, S.sm.b1);
        sync_fenced();
        // ---- layer 2 and the output logit ----
        if (!(ok = layer(S.w2t))) break;
        float lo_a = S.sm.b3[0], lo_b = 0.0f;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            float z[32];
            tmem_ld32(tz + 32u * (uint32_t)g, z);
#pragma unroll
            for (int k4 = 0; k4 < 32; k4 += 4) {
                const float4 bb = *reinterpret_cast<const float4 *>(S.sm.b2 + 32 * g + k4);
                const float4 ww = *reinterpret_cast<const float4 *>(S.sm.w3 + 32 * g + k4);
                lo_a = fmaf(fmaxf(z[k4] + bb.x, 0.0f), ww.x, lo_a);
                lo_b = fmaf(fmaxf(z[k4 + 1] + bb.y, 0.0f), ww.y, lo_b);
                lo_a = fmaf(fmaxf(z[k4 + 2] + bb.z, 0.0f), ww.z, lo_a);
                lo_b = fmaf(fmaxf(z[k4 + 3] + bb.w, 0.0f), ww.w, lo_b);
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
    if (warp == 0) tmem_dealloc(S.sm.tmem_base, FWD_COLS);
}

// ---------------------------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------------------------

// TMEM columns: the layer accumulator (Z, then dH) and the weight-gradient accumulators.
constexpr uint32_t BCOL_Z = 0, BCOL_DW2 = 64, BCOL_DW1 = 128, BCOL_DW0 = 192, BCOL_DW3 = 256, BCOLS = 512;

struct alignas(1024) SmallB {
    float b1[PW], b2[PW], w3[PW];
    float b3[4];
    float red[2][2][2];
    ClipDf clip[TT];
    uint64_t mbar;
    uint32_t tmem_base;
};

struct SmemB {
    unsigned char w0t[kPanelBytes];
    unsigned char w1t[kPanelBytes];
    unsigned char w2t[kPanelBytes];
    unsigned char x[kPanelBytes];
    unsigned char h0[kPanelBytes];
    unsigned char h1[kPanelBytes];
    unsigned char h2[kPanelBytes];
    unsigned char dza[kPanelBytes];   // dZ2, then dZ0
    unsigned char dzb[kPanelBytes];   // dZ1
    unsigned char dl[kPanelBytes];    // column 0 = dlogit, columns 1..15 = 0
    unsigned char e[kPanelBytes];     // column 0 = 1 (must follow x, h0, h1, h2: it is their second M half)
    SmallB sm;
};

// MN-major A operand of M = 128 whose first 64 rows are panel `base` and last 64 rows the panel
// `lbo` bytes after it; k-step kk = 16 tile rows.
__device__ __forceinline__ uint64_t desc_mn_pair(uint32_t base, int kk, uint32_t lbo) {
    return sdesc(base + (uint32_t)kk * 2u * kGroupBytes, lbo, kGroupBytes);
}

// ReLU epilogue of one 64-column layer accumulator: h = max(z + b, 0) into the panel, the ReLU mask
// into two 32-bit words; with w_out, also returns the output-layer dot product h . w_out.
__device__ __forceinline__ float relu_epilogue(uint32_t tb, int warp, const float *bias, unsigned char *panel,
                                               uint32_t (&mask)[2], const float *w_out) {
    const int tid = threadIdx.x;
    float da = 0.0f, db = 0.0f;
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        float z[32];
        tmem_ld32(taddr(tb, warp, BCOL_Z + 32 * g), z);
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            z[k] = fmaxf(z[k] + (bias ? bias[32 * g + k] : 0.0f), 0.0f);
            m |= (z[k] > 0.0f ? 1u : 0u) << k;
        }
        if (w_out) {
#pragma unroll
            for (int k = 0; k < 32; k += 2) {
                da = fmaf(z[k], w_out[32 * g + k], da);
                db = fmaf(z[k + 1], w_out[32 * g + k + 1], db);
            }
        }
        mask[g] = m;
#pragma unroll
        for (int k = 0; k < 32; k += 8) panel_store8(panel, tid, 32 * g + k, z + k);
    }
    return da + db;
}

// dZ = dH * mask from the layer accumulator into the panel.
__device__ __forceinline__ void mask_epilogue(uint32_t tb, int warp, const uint32_t (&mask)[2], unsigned char *panel) {
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        float z[32];
        tmem_ld32(taddr(tb, warp, BCOL_Z + 32 * g), z);
#pragma unroll
        for (int k = 0; k < 32; ++k) z[k] = (mask[g] >> k) & 1u ? z[k] : 0.0f;
#pragma unroll
        for (int k = 0; k < 32; k += 8) panel_store8(panel, tid, 32 * g + k, z + k);
    }
}

// Adds rows [0, nrows) of a 64-column gradient accumulator (lane = row) to dst[row * 64 + n] and
// row `bias_row` to bias[n], scaled by s.  Every thread of the CTA calls it (TMEM loads are
// warp-collective).
__device__ __forceinline__ void flush_acc(uint32_t tb, int warp, uint32_t col, int nrows, int bias_row, float *dst,
                                          float *bias, float s) {
    const int row = threadIdx.x;
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        float v[32];
        tmem_ld32(taddr(tb, warp, col + 32 * g), v);
        if (row < nrows) {
            for (int k = 0; k < 32; ++k) atomicAdd(dst + row * PW + 32 * g + k, v[k] * s);
        } else if (row == bias_row) {
            for (int k = 0; k < 32; ++k) atomicAdd(bias + 32 * g + k, v[k] * s);
        }
    }
}

__global__ void __launch_bounds__(TT, 1) proposal_bwd_tc_kernel(PropTcArgs P) {
    extern __shared__ unsigned char smem_raw[];
    SmemB &S = *reinterpret_cast<SmemB *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) mbar_init(&S.sm.mbar, 1);
    if (warp == 0) tmem_alloc(&S.sm.tmem_base, BCOLS);
    load_weights(P, S.w0t, S.w1t, S.w2t, S.sm.b1, S.sm.b2, S.sm.w3, S.sm.b3);
    {
        float v[8];
#pragma unroll
        for (int c = 0; c < 64; c += 8) {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = (c == 0 && k == 0) ? 1.0f : 0.0f;
            panel_store8(S.e, tid, c, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = 0.0f;
            panel_store8(S.dl, tid, c, v);
        }
    }
    fence_async_smem();
    sync_fenced();
    const uint32_t tb = S.sm.tmem_base;
    const uint32_t id_fwd = idesc_bf16(128, 64, 0, 0);   // Z = A W: A K-major, W^T panel K-major
    const uint32_t id_dh = idesc_bf16(128, 64, 0, 1);    // dH = dZ W^T: dZ K-major, W^T panel MN-major
    const uint32_t id_dw = idesc_bf16(128, 64, 1, 1);    // [H | E]^T dZ: both MN-major
    const uint32_t id_dw3 = idesc_bf16(128, 16, 1, 1);
    uint32_t phase = 0;
    bool ok = true;
    uint32_t acc = 0;   // 0 until the first tile's weight-gradient MMAs have initialised TMEM
    const int ntiles = (P.R + 1) / 2;
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++k) {
        uint32_t x_ = smem_u32(S.x), w0_ = smem_u32(S.w0t), w1_ = smem_u32(S.w1t), w2_ = smem_u32(S.w2t);
        uint32_t h0_ = smem_u32(S.h0), h1_ = smem_u32(S.h1), h2_ = smem_u32(S.h2), e_ = smem_u32(S.e);
        uint32_t dza_ = smem_u32(S.dza), dzb_ = smem_u32(S.dzb), dl_ = smem_u32(S.dl);
        asm volatile("" : "+r"(x_), "+r"(w0_), "+r"(w1_), "+r"(w2_), "+r"(h0_), "+r"(h1_), "+r"(h2_), "+r"(e_));
        asm volatile("" : "+r"(dza_), "+r"(dzb_), "+r"(dl_));
        const int rl = tid >> 6, bin = tid & 63, r = 2 * tile + rl;
        if (k % kClipTiles == 0) {
            clip_pass(P, k, S.sm.clip);
            __syncthreads();
        }
        const bool hit = S.sm.clip[2 * (k % kClipTiles) + rl].hit != 0;
        encode_row(S.sm.clip[2 * (k % kClipTiles) + rl], S.x);
        fence_async_smem();
        sync_fenced();
        uint32_t m0[2], m1[2], m2[2];
        // ---- forward: three layers ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + BCOL_Z, desc_kmajor(x_, kk), desc_kmajor(w0_, kk), id_fwd, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        relu_epilogue(tb, warp, nullptr, S.h0, m0, nullptr);
        fence_async_smem();
        sync_fenced();
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + BCOL_Z, desc_kmajor(h0_, kk), desc_kmajor(w1_, kk), id_fwd, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        relu_epilogue(tb, warp, S.sm.b1, S.h1, m1, nullptr);
        fence_async_smem();
        sync_fenced();
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + BCOL_Z, desc_kmajor(h1_, kk), desc_kmajor(w2_, kk), id_fwd, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        const float logit = S.sm.b3[0] + relu_epilogue(tb, warp, S.sm.b2, S.h2, m2, S.sm.w3);
        // ---- softmax over the 64 rows of a ray; dlogit = p - h (the 1/R is applied at the flush) ----
        float m = logit;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) S.sm.red[rl][warp & 1][0] = m;
        __syncthreads();
        m = fmaxf(S.sm.red[rl][0][0], S.sm.red[rl][1][0]);
        const float ex = expf(logit - m);
        const float es = warp_sum(ex);
        if (lane == 0) S.sm.red[rl][warp & 1][1] = es;
        __syncthreads();
        const float zs = S.sm.red[rl][0][1] + S.sm.red[rl][1][1];
        float dlog = 0.0f;
        if (r < P.R && hit) dlog = ex / zs - P.labels[(size_t)r * NB + bin];
        {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = k == 0 ? dlog : 0.0f;
            panel_store8(S.dl, tid, 0, v);
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                float z[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) z[k] = (m2[g] >> k) & 1u ? dlog * S.sm.w3[32 * g + k] : 0.0f;
#pragma unroll
                for (int k = 0; k < 32; k += 8) panel_store8(S.dza, tid, 32 * g + k, z + k);
            }
        }
        fence_async_smem();
        sync_fenced();
        // ---- dW2 | db2, dW3 | db3, dH1 ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 8; ++kk)
                mma(tb + BCOL_DW2, desc_mn_pair(h1_, kk, e_ - h1_), desc_mnmajor(dza_, kk), id_dw, acc | (kk > 0));
#pragma unroll 1
            for (int kk = 0; kk < 8; ++kk)
                mma(tb + BCOL_DW3, desc_mn_pair(h2_, kk, e_ - h2_), desc_mnmajor(dl_, kk), id_dw3, acc | (kk > 0));
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + BCOL_Z, desc_kmajor(dza_, kk), desc_mnmajor(w2_, kk), id_dh, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        mask_epilogue(tb, warp, m1, S.dzb);
        fence_async_smem();
        sync_fenced();
        // ---- dW1 | db1, dH0 ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 8; ++kk)
                mma(tb + BCOL_DW1, desc_mn_pair(h0_, kk, e_ - h0_), desc_mnmajor(dzb_, kk), id_dw, acc | (kk > 0));
#pragma unroll 1
            for (int kk = 0; kk < 4; ++kk) mma(tb + BCOL_Z, desc_kmajor(dzb_, kk), desc_mnmajor(w1_, kk), id_dh, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        mask_epilogue(tb, warp, m0, S.dza);
        fence_async_smem();
        sync_fenced();
        // ---- [dW0 | db0] (input column 39 is the constant 1) ----
        if (tid == 0) {
#pragma unroll 1
            for (int kk = 0; kk < 8; ++kk)
                mma(tb + BCOL_DW0, desc_mn_pair(x_, kk, e_ - x_), desc_mnmajor(dza_, kk), id_dw, acc | (kk > 0));
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        acc = 1;
        __syncthreads();
    }
    ok = !__syncthreads_or(!ok);
    if (!ok) {
        mbar_wait(&S.sm.mbar, phase ^ 1);
        if (tid == 0) atomicAdd(P.grad, __int_as_float(0x7fc00000));   // NaN marks the failed launch
    }
    sync_fenced();
    if (ok && acc) {
        const float s = 1.0f / (float)P.R;
        float *G0 = P.grad, *GB0 = G0 + PIN * PW, *G1 = GB0 + PW, *GB1 = G1 + PW * PW, *G2 = GB1 + PW;
        float *GB2 = G2 + PW * PW, *G3 = GB2 + PW, *GB3 = G3 + PW;
        flush_acc(tb, warp, BCOL_DW0, PIN, PIN, G0, GB0, s);
        flush_acc(tb, warp, BCOL_DW1, PW, PW, G1, GB1, s);
        flush_acc(tb, warp, BCOL_DW2, PW, PW, G2, GB2, s);
        float v[16];
        tmem_ld16(taddr(tb, warp, BCOL_DW3), v);
        if (tid < PW) atomicAdd(G3 + tid, v[0] * s);
        else if (tid == PW) atomicAdd(GB3, v[0] * s);
    }
    sync_fenced();
    if (warp == 0) tmem_dealloc(S.sm.tmem_base, BCOLS);
}

}  // namespace

int launch_proposal_fwd_tc(const dvgo_params &p, const dvgo_grid_desc &g, const dvgo_proposal_mlp &m, int R,
                           const float *ro, const float *rd, const float *labels, float *probs, float *loss,
                           cudaStream_t s) {
    PropTcArgs P{};
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
    const int bytes = kFwdSmemBytes;
    ensure_smem(reinterpret_cast<const void *>(proposal_fwd_tc_kernel), bytes);
    const int ntiles = (R + 1) / 2;
    int blocks = kFwdCtasPerSm * num_sms();
    if (blocks > ntiles) blocks = ntiles;
    {
        ProfScope ps_(DVGO_K_PROPOSAL_FWD, s);
        proposal_fwd_tc_kernel<<<blocks, TT, bytes, s>>>(P);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

int launch_proposal_bwd_tc(const dvgo_params &p, const dvgo_grid_desc &g, const dvgo_proposal_mlp &m, int R,
                           const float *ro, const float *rd, const float *labels, float *grad, cudaStream_t s) {
    PropTcArgs P{};
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
    P.grad = grad;
    const int bytes = (int)sizeof(SmemB) + 1024;
    ensure_smem(reinterpret_cast<const void *>(proposal_bwd_tc_kernel), bytes);
    const int ntiles = (R + 1) / 2;
    int blocks = num_sms();
    if (blocks > ntiles) blocks = ntiles;
    {
        ProfScope ps_(DVGO_K_PROPOSAL_BWD, s);
        proposal_bwd_tc_kernel<<<blocks, TT, bytes, s>>>(P);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // namespace dvgo
