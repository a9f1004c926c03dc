// fine_tc.cu -- colour queries of the fine stage with the BF16 tensor-core MLP (tcgen05, sm_103a).
//
// Same function as fine_simt.cu (Sec. 4.2 Eq. fine_queries_rgb, Supp. A: 12 features + PE(d, 4)
// = 39 inputs, or 72 with PE(x, 5) appended; two hidden layers of 128 with ReLU, sigmoid output)
// with the two 128-wide layers
// and all weight-gradient contractions on the 5th-generation tensor cores: BF16 operands in
// shared memory (128-byte swizzled panels, see tc_helpers.cuh), FP32 accumulators in TMEM, MMAs
// issued by one thread, completion signalled through mbarriers.  The 128 -> 3 output layer, the
// sigmoid and the element-wise steps run on the CUDA cores in the epilogues.
//
// Persistent CTAs of 384 threads walk tiles of M = 128 kept samples.  Warps 8-11 (producers)
// gather the next tile -- features at the 8 lattice corners, the ray's direction encoding, the
// bias column -- into one of two X panels, and in the backward also scatter the feature gradients
// of the tile that last used that panel.  The forward stores every finished X panel (16 KiB, as
// swizzled in shared memory) in the workspace (one bulk copy per tile); the backward loads it back
// with one bulk copy instead of gathering again (tile t holds the same kept samples in both: the
// kept list is the forward's), so its producers only form the per-row tables, dL/dc and the PE(x)
// tail.  Warps 0-7 (consumers)
// issue the MMAs (thread 0) and run the epilogues: warp w reads TMEM lanes 32 (w % 4)..+31 and
// handles columns 64 (w / 4)..+63 of those rows, so two warps share each row.  full[b] / empty[b]
// mbarriers hand the X panels over; every wait is bounded.
//
// Inputs beyond the 64 columns of the X panel (PE(x) entries 24-32 of the 72-input row) live in a
// "tail panel" that also holds W3: columns 0-15 W3 (3 used), 16-31 / 32-47 the tail of X buffer 0 /
// 1, 48-63 the tail rows of W1 (transposed).  Layer 1 adds one K = 16 MMA over the tails; the
// backward adds dW1_tail^T += dZ1^T X_tail (an MN-major operand that starts 32 or 64 bytes into
// the swizzled rows).
//
// Forward per tile:  X[128x64] (features, PE(d), [PE(x)], 1) -> Z1 = X W1|b1 -> H1 = relu(Z1) -> Z2 = H1 W2
//                    -> H2 = relu(Z2 + b2) -> O = H2 W3 (N = 16, 3 used) -> c = sigmoid(O + b3).
// Backward per tile (recomputes layers 1 and 2; the colour c is the one the forward stored in the
// sample record, so layer 3 is not recomputed), with dL/dc from the compositing backward:
//   dout = dL/dc c (1 - c)                                        (producers; epilogue, BF16 panel)
//   dH2 = dout W3^T;  dZ2 = dH2 [Z2 + b2 > 0]                      (MMA, epilogue)
//   dH1 = dZ2 W2^T;  [dW2^T | db2] += dZ2^T [H1 | dout];  dW3 += H2^T dout   (MMAs; dout's
//   column 3 is 1, so one N = 144 MMA gives dW2^T and db2)
//   dZ1 = dH1 [Z1 > 0]                                             (epilogue)
//   de = dZ1 W1[0:16]^T;  [dW1 | db1]^T += dZ1^T X                 (MMAs)
//   de[0:12] -> shared memory -> scattered to the feature grid by the producers
// TMEM columns: Z1 / O / dH2 [0,128), Z2 / dH1 [128,256), [dW2^T | db2] [256,400), dW1^T [400,464),
// dW3 [464,480), de [480,496), dW1_tail^T [496,512).  The weight-gradient accumulators live in TMEM for
// the whole launch and are added to global memory once per CTA.

#include <stddef.h>

#include "dvgo_internal.cuh"
#include "tc_helpers.cuh"

namespace dvgo {

namespace {

using namespace tc;

constexpr int TM = 128;
constexpr int NC = 256;        // consumer threads: warp w owns TMEM lanes 32 (w % 4).., columns 64 (w / 4)..
constexpr int NP = 128;        // producer threads of one set (one sample row each)
// producer sets: the backward has one (its consumers are the bound); the forward two, set p filling
// X buffer p for consumer group p, so that two tiles are gathered at once
#ifndef DVGO_FWD_PROD_SETS
#define DVGO_FWD_PROD_SETS 2
#endif
template <bool BWD>
constexpr int kProdSets = BWD ? 1 : DVGO_FWD_PROD_SETS;
template <bool BWD>
constexpr int kThreads = NC + NP * kProdSets<BWD>;   // 384 / 512
constexpr int HID = 128;
constexpr int FEAT = 12;
constexpr int NF = 4;
constexpr int NFX = 5;
constexpr int PX = FEAT + 3 + 6 * NF;   // 39: first input of the PE(x) block

// Input row of the two widths: IN inputs, NMAIN of them in the X panel, the first-layer bias as
// the constant-1 column BIAS of the X panel, NTAIL inputs in the tail panel.
template <bool PEX>
struct TcDims {
    static constexpr int IN = PX + (PEX ? 3 + 6 * NFX : 0);   // 39 or 72
    static constexpr int NMAIN = PEX ? 63 : IN;
    static constexpr int BIAS = NMAIN;
    static constexpr int NTAIL = IN - NMAIN;                  // 0 or 9
};

constexpr uint32_t COL_Z1 = 0, COL_O = 0, COL_Z2 = 128, COL_DW2T = 256, COL_DW1 = 400, COL_DW3 = 464,
                   COL_DE = 480, COL_DW1T = 496;

// Small per-CTA state, padded to a multiple of 1024 bytes so that the panels after it stay
// aligned to the 128-byte-swizzle atom.
struct alignas(1024) SmallTC {
    float b2[HID];
    float b3[4];
    float db3[4];
    // per-row tables of a tile, a ring of 4 (tile i in entry i % 4): the scatter of tile i - 2 reads
    // other rows' entries while a producer that is done with it already fills tile i or i + 1
    int slot[4][TM];          // sample slot per row, -1 for padding rows
    int cbase[4][TM];         // flat index of the base lattice corner
    float frac[4][TM][3];     // fractional offsets
    float dc[2][TM][3];       // dL/dc (backward)
    uint64_t full[2], empty[2], mma, mma1;   // mma1: the forward's second consumer group
    uint64_t xl[2];           // backward: the bulk load of X panel b from the forward's copy
    uint32_t tmem_base;
    int abort;
};

struct SmemTC {
    unsigned char w1t[kPanelBytes];       // W1|b1 transposed: row = hidden unit, 64 input columns
    unsigned char w2t[2 * kPanelBytes];   // W2 transposed: row = output unit, 128 input columns
    unsigned char tp[kPanelBytes];        // tail panel: row = hidden unit / sample; W3 in columns 0-2,
                                          // X tails in 16-31 / 32-47, W1 tail in 48-63
    unsigned char x[2][kPanelBytes];      // X (double-buffered): row = sample
    unsigned char h1[2 * kPanelBytes];    // H1, later dZ1
    // backward: columns 0-15: [dout_r, dout_g, dout_b, 1, ...] (MMA operand); bytes 32-79 and 80-127
    // of every row (16-byte chunks 2-4 and 5-7): de[0:12] in FP32 for X buffer 0 and 1.  It follows
    // H1 directly, so [H1 | dout] is one MN-major operand of N = 144 (panels 16 KiB apart)
    unsigned char dout[kPanelBytes];
    unsigned char h2[2 * kPanelBytes];    // H2
    SmallTC sm;
    // backward only (the forward allocates the struct up to here)
    unsigned char dz2[2 * kPanelBytes];   // dZ2
};
static_assert(offsetof(SmemTC, dout) == offsetof(SmemTC, h1) + 2 * kPanelBytes, "[H1 | dout] must be contiguous");

constexpr size_t smem_bytes(bool bwd) { return (bwd ? sizeof(SmemTC) : offsetof(SmemTC, dz2)) + 1024; }
static_assert(smem_bytes(true) <= 232448, "the backward must fit one CTA per SM (227 KB of shared memory)");

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Barrier among the 256 consumer threads only (the producers run on their own schedule).
__device__ __forceinline__ void consumer_sync() {
    fence_before();
    asm volatile("bar.sync 1, 256;" ::: "memory");
    fence_after();
}

// Operands written by the consumers become visible to the tensor core, then the consumers sync.
__device__ __forceinline__ void consumer_publish() {
    fence_async_smem();
    consumer_sync();
}

// 16-byte chunk k (0-2) of the de[0:12] slot of X buffer b in row r of the dout panel.
__device__ __forceinline__ float4 *de_slot(unsigned char *dout, int b, int r, int k) {
    return reinterpret_cast<float4 *>(dout + panel_offset(r, 8 * (2 + 3 * b + k)));
}

// Producer: add a tile's feature gradients (de rows staged in the dout panel) to the grid.  Rows
// are in kept order, so consecutive samples of a ray sit in consecutive rows; rows whose samples lie
// in one lattice cell share all eight corners, and the last row of such a run adds the whole run's
// weighted de with one set of reductions (the run's other rows add nothing).
template <bool PK>
__device__ __forceinline__ void scatter_row(const RenderArgs &A, SmemTC &S, int b, int t, int row) {
    const int slot = S.sm.slot[t][row];
    if (slot < 0) return;
    const int cb = S.sm.cbase[t][row];
    if (row + 1 < TM && S.sm.slot[t][row + 1] >= 0 && S.sm.cbase[t][row + 1] == cb) return;
    float4 acc[8][3];
    {
        const float4 e0 = *de_slot(S.dout, b, row, 0), e1 = *de_slot(S.dout, b, row, 1),
                     e2 = *de_slot(S.dout, b, row, 2);
        const float fx = S.sm.frac[t][row][0], fy = S.sm.frac[t][row][1], fz = S.sm.frac[t][row][2];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float w = (((q >> 2) & 1) ? fx : 1.0f - fx) * (((q >> 1) & 1) ? fy : 1.0f - fy) *
                            ((q & 1) ? fz : 1.0f - fz);
            acc[q][0] = make_float4(w * e0.x, w * e0.y, w * e0.z, w * e0.w);
            acc[q][1] = make_float4(w * e1.x, w * e1.y, w * e1.z, w * e1.w);
            acc[q][2] = make_float4(w * e2.x, w * e2.y, w * e2.z, w * e2.w);
        }
    }
    for (int j = row - 1; j >= 0 && S.sm.slot[t][j] >= 0 && S.sm.cbase[t][j] == cb; --j) {
        const float4 e0 = *de_slot(S.dout, b, j, 0), e1 = *de_slot(S.dout, b, j, 1), e2 = *de_slot(S.dout, b, j, 2);
        const float fx = S.sm.frac[t][j][0], fy = S.sm.frac[t][j][1], fz = S.sm.frac[t][j][2];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float w = (((q >> 2) & 1) ? fx : 1.0f - fx) * (((q >> 1) & 1) ? fy : 1.0f - fy) *
                            ((q & 1) ? fz : 1.0f - fz);
            acc[q][0] = make_float4(fmaf(w, e0.x, acc[q][0].x), fmaf(w, e0.y, acc[q][0].y),
                                    fmaf(w, e0.z, acc[q][0].z), fmaf(w, e0.w, acc[q][0].w));
            acc[q][1] = make_float4(fmaf(w, e1.x, acc[q][1].x), fmaf(w, e1.y, acc[q][1].y),
                                    fmaf(w, e1.z, acc[q][1].z), fmaf(w, e1.w, acc[q][1].w));
            acc[q][2] = make_float4(fmaf(w, e2.x, acc[q][2].x), fmaf(w, e2.y, acc[q][2].y),
                                    fmaf(w, e2.z, acc[q][2].z), fmaf(w, e2.w, acc[q][2].w));
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long long idx = corner_from_base(cb, (q >> 2) & 1, (q >> 1) & 1, q & 1, A.ny, A.nz, PK);
        float4 *g = reinterpret_cast<float4 *>(A.grad_cgrid + idx * FEAT);
        atomicAdd(g + 0, acc[q][0]);
        atomicAdd(g + 1, acc[q][1]);
        atomicAdd(g + 2, acc[q][2]);
    }
}

// The ray data a producer needs to place a sample, fetched a tile ahead: uniform steps, the first
// sample and the per-step increment (fixed point); explicit samples, the entry point (fixed point),
// the direction in lattice units (FP64 bits) and t_enter; and the ray's first sample slot.
struct RayPre {
    long long f0[3], f1[3];
    double t_enter;
    int off;
};

__device__ __forceinline__ RayPre ray_pre(const RenderArgs &A, int ray) {
    RayPre p;
    const RayRec &r = A.rays[ray];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p.f0[a] = A.ts ? r.uefx[a] : r.u0fx[a];
        p.f1[a] = A.ts ? __double_as_longlong(r.e[a]) : r.dfx[a];
    }
    p.t_enter = A.ts ? r.t_enter : 0.0;
    p.off = r.off;
    return p;
}

// sample_cell() from prefetched ray data (the same arithmetic).
__device__ __forceinline__ Cell cell_pre(const RenderArgs &A, const RayPre &p, int ray, int k, float &dt) {
    long long u[3];
    if (A.ts) {
        const double t = (double)A.ts[(long long)ray * A.n_expl + k];
        dt = A.dts[(long long)ray * A.n_expl + k];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = p.f0[a] + to_fx((t - p.t_enter) * __longlong_as_double(p.f1[a]));
    } else {
        dt = A.step;
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = p.f0[a] + (long long)k * p.f1[a];
    }
    return cell_from_fx(u, A.nx, A.ny, A.nz);
}

// Producer: gather sample row `row` of a tile (kept entry kv, kv.y < 0 for a padding row; its ray's
// prefetched data rp) into X panel b (and its tail) and the per-row tables.
template <typename FeatT, bool BWD, bool PEX, bool PK>
__device__ __forceinline__ void produce_row(const RenderArgs &A, SmemTC &S, int b, int t, int2 kv,
                                            const RayPre &rp, int row, bool cached) {
    // cached (backward): the X panel arrives by bulk copy; only the tables, dL/dc and the tail here
    using D = TcDims<PEX>;
    float v[64], tail[16];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) tail[i] = 0.0f;
    int slot = -1, cbase = 0;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f, d0 = 0.0f, d1 = 0.0f, d2 = 0.0f;
    if (kv.y >= 0) {
        float dt;
        const Cell c = cell_pre(A, rp, kv.y, kv.x - rp.off, dt);
        slot = kv.x;
        cbase = cell_base(c, A.ny, A.nz, PK);
        fx = c.fx;
        fy = c.fy;
        fz = c.fz;
        if (BWD) {
            // dout = dL/dc c (1 - c) with the colour c the forward left in the sample record
            // (the same kernel arithmetic on the same operands, so the layer-3 recompute is skipped)
            const float4 gc = A.sgrad[slot], cv = A.samp[slot];
            d0 = gc.y * cv.y * (1.0f - cv.y);
            d1 = gc.z * cv.z * (1.0f - cv.z);
            d2 = gc.w * cv.w * (1.0f - cv.w);
        }
#pragma unroll
        for (int q = 0; q < (cached ? 0 : 4); ++q) {   // corner pairs (x bit, y bit) with z = 0, 1 adjacent
            const int qa = q << 1;
            const long long idx0 = corner_index(c, qa, A.ny, A.nz, PK);
            const float w0 = corner_weight(c, qa), w1 = corner_weight(c, qa | 1);
            const FeatT *g = static_cast<const FeatT *>(A.cgrid) + idx0 * FEAT;
            // the z + 1 corner: the next point in the canonical layout, located in the packed one
            const FeatT *gz = PK ? static_cast<const FeatT *>(A.cgrid) +
                                             corner_index(c, qa | 1, A.ny, A.nz, true) * FEAT
                                       : g + FEAT;
            if constexpr (sizeof(FeatT) == 4) {
                const float4 *g4 = reinterpret_cast<const float4 *>(g), *gz4 = reinterpret_cast<const float4 *>(gz);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 a = __ldg(g4 + k), bb = __ldg(gz4 + k);
                    v[4 * k + 0] += w0 * a.x + w1 * bb.x;
                    v[4 * k + 1] += w0 * a.y + w1 * bb.y;
                    v[4 * k + 2] += w0 * a.z + w1 * bb.z;
                    v[4 * k + 3] += w0 * a.w + w1 * bb.w;
                }
            } else if constexpr (!PK) {
                // canonical BF16: the pair is 48 contiguous bytes at offset 0 or 8 mod 16 (the grid is
                // 16-byte aligned, a point is 24 bytes): three aligned 16-byte loads from the pair's
                // 16-byte granule and, at offset 8, one 8-byte load for its last word pair -- no byte
                // outside the grid (at offset 8 the first 8 bytes loaded belong to the point before)
                const uintptr_t ad = reinterpret_cast<uintptr_t>(g);
                const uint4 *q = reinterpret_cast<const uint4 *>(ad & ~(uintptr_t)15);
                const bool off8 = (ad & 15u) != 0u;
                const uint4 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2);
                const uint2 q3 = off8 ? __ldg(reinterpret_cast<const uint2 *>(q + 3)) : make_uint2(0u, 0u);
                const uint32_t wd[14] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                                         q2.x, q2.y, q2.z, q2.w, q3.x, q3.y};
#pragma unroll
                for (int m = 0; m < 6; ++m) {   // channels 2m, 2m + 1 of the corners z (word m) and z + 1
                    uint32_t ua = off8 ? wd[m + 2] : wd[m], ub = off8 ? wd[m + 8] : wd[m + 6];
                    const float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&ua));
                    const float2 bz = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&ub));
                    v[2 * m + 0] += w0 * a.x + w1 * bz.x;
                    v[2 * m + 1] += w0 * a.y + w1 * bz.y;
                }
            } else {
                const uint2 *g2 = reinterpret_cast<const uint2 *>(g), *gz2 = reinterpret_cast<const uint2 *>(gz);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    uint2 a = __ldg(g2 + k), bb = __ldg(gz2 + k);
                    const float2 a0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&a.x));
                    const float2 a1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&a.y));
                    const float2 b0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&bb.x));
                    const float2 b1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&bb.y));
                    v[4 * k + 0] += w0 * a0.x + w1 * b0.x;
                    v[4 * k + 1] += w0 * a0.y + w1 * b0.y;
                    v[4 * k + 2] += w0 * a1.x + w1 * b1.x;
                    v[4 * k + 3] += w0 * a1.y + w1 * b1.y;
                }
            }
        }
        const float4 *pe = reinterpret_cast<const float4 *>(A.pe + (size_t)kv.y * kPeStride);
#pragma unroll
        for (int k = 0; k < (cached ? 0 : 7); ++k) {
            const float4 q4 = __ldg(pe + k);
            if (4 * k + 0 < 27) v[FEAT + 4 * k + 0] = q4.x;
            if (4 * k + 1 < 27) v[FEAT + 4 * k + 1] = q4.y;
            if (4 * k + 2 < 27) v[FEAT + 4 * k + 2] = q4.z;
            if (4 * k + 3 < 27) v[FEAT + 4 * k + 3] = q4.w;
        }
        if constexpr (PEX) {
            // PE(x) of the world-space sample position: [x (3), sin(2^k x_c) (15), cos(2^k x_c) (15)]
            float xv[3], pe[3 + 6 * NFX];
            cell_world(A, c, xv);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                pe[a] = xv[a];
                pe_axis<NFX>(xv[a], pe + 3 + a * NFX, pe + 3 + 3 * NFX + a * NFX);
            }
#pragma unroll
            for (int j = 0; j < D::NMAIN - PX; ++j) v[PX + j] = pe[j];
#pragma unroll
            for (int j = 0; j < D::NTAIL; ++j) tail[j] = pe[D::NMAIN - PX + j];
        }
        v[D::BIAS] = 1.0f;
    }
    if (!cached) {
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.x[b], row, c, v + c);
    }
    if constexpr (PEX) {
        panel_store8(S.tp, row, 16 * (1 + b), tail);
        panel_store8(S.tp, row, 16 * (1 + b) + 8, tail + 8);
    }
    S.sm.slot[t][row] = slot;
    S.sm.cbase[t][row] = cbase;
    S.sm.frac[t][row][0] = fx;
    S.sm.frac[t][row][1] = fy;
    S.sm.frac[t][row][2] = fz;
    if (BWD) {
        S.sm.dc[b][row][0] = d0;
        S.sm.dc[b][row][1] = d1;
        S.sm.dc[b][row][2] = d2;
    }
}

template <typename FeatT, bool BWD, bool PEX, bool PK>
__global__ void __launch_bounds__(kThreads<BWD>, 1) fine_colour_tc_kernel(RenderArgs A) {
    using D = TcDims<PEX>;
    extern __shared__ unsigned char smem_raw[];
    SmemTC &S = *reinterpret_cast<SmemTC *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t NCOLS = 512;   // backward: activations + weight gradients; forward: 256 per consumer group

    if (tid == 0) {
        mbar_init(&S.sm.full[0], NP);
        mbar_init(&S.sm.full[1], NP);
        mbar_init(&S.sm.empty[0], 1);
        mbar_init(&S.sm.empty[1], 1);
        mbar_init(&S.sm.mma, 1);
        mbar_init(&S.sm.mma1, 1);
        mbar_init(&S.sm.xl[0], 1);
        mbar_init(&S.sm.xl[1], 1);
        S.sm.abort = 0;
    }
    if (warp == 0) tmem_alloc(&S.sm.tmem_base, NCOLS);
    // barriers initialised and TMEM allocated: the producers start gathering the first tile while
    // consumer warps 0-3 stage the weights (published to the consumers and the tensor core below)
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < TM) {
        // weights: row n = tid of W1^T (64 input columns, bias in column BIAS), of W2^T and of the
        // tail panel (W3, and with PE(x) the tail rows of W1)
        float v[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = k < D::NMAIN ? A.w1[k * HID + tid] : (k == D::BIAS ? A.b1[tid] : 0.0f);
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.w1t, tid, c, v + c);
#pragma unroll
        for (int pnl = 0; pnl < 2; ++pnl) {
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = A.w2[(pnl * 64 + k) * HID + tid];
#pragma unroll
            for (int c = 0; c < 64; c += 8) panel_store8(S.w2t + pnl * kPanelBytes, tid, c, v + c);
        }
#pragma unroll
        for (int k = 0; k < 64; ++k)
            v[k] = k < 3 ? A.w3[3 * tid + k]
                         : ((k >= 48 && k - 48 < D::NTAIL) ? A.w1[(D::NMAIN + k - 48) * HID + tid] : 0.0f);
        // only the weight columns (0-15: W3, 48-63: W1 tail): columns 16-47 hold the X tails, which
        // the producers are already writing
        panel_store8(S.tp, tid, 0, v);
        panel_store8(S.tp, tid, 8, v + 8);
        panel_store8(S.tp, tid, 48, v + 48);
        panel_store8(S.tp, tid, 56, v + 56);
        if (BWD) {
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = 0.0f;
#pragma unroll
            for (int c = 0; c < 64; c += 8) panel_store8(S.dout, tid, c, v + c);
        }
        S.sm.b2[tid] = A.b2[tid];
        if (tid < 3) S.sm.b3[tid] = A.b3[tid];
        if (tid < 4) S.sm.db3[tid] = 0.0f;
    }
    if (tid < NC) consumer_publish();

    const int n_kept = A.hdr->n_kept;
    const int ntiles = (n_kept + TM - 1) / TM;
    // backward: reload the X panels the forward stored (the workspace has room and the forward that
    // filled it stored them); otherwise gather them again
    const bool cached = BWD && A.xcache != nullptr && A.hdr->xcache != 0;
    bool ok = true;
    int ntile_mine = 0;

    if (tid >= NC) {
        // ------------------------------- producers -------------------------------
        // Set pset takes the CTA's tiles i = pset, pset + nsets, ... (X buffer i & 1).  Software-
        // pipelined a tile deep: while producing a tile, a producer already has its set's next tile's
        // kept entry and fetches that tile's ray data and the kept entry of the tile after, so that
        // only the corner-feature loads of a tile wait on memory when it is produced.
        constexpr int nsets = kProdSets<BWD>;
        const int row = (tid - NC) & (NP - 1), pset = (tid - NC) / NP;
        const int stride = nsets * (int)gridDim.x;
        auto kept_at = [&](int t) -> int2 {
            const int e = t * TM + row;
            return (t < ntiles && e < n_kept) ? A.kept[e] : make_int2(-1, -1);
        };
        const int tile0 = (int)blockIdx.x + pset * (int)gridDim.x;
        int2 kv_cur = kept_at(tile0);
        RayPre rp_cur = kv_cur.y >= 0 ? ray_pre(A, kv_cur.y) : RayPre{};
        int2 kv_next = kept_at(tile0 + stride);
        int nload[2] = {0, 0};   // row 0, backward: bulk loads issued into X panel 0 / 1
        int i = pset;
        for (int tile = tile0; tile < ntiles; tile += stride, i += nsets) {
            const int b = i & 1;
            const RayPre rp_next = kv_next.y >= 0 ? ray_pre(A, kv_next.y) : RayPre{};
            const int2 kv_after = kept_at(tile + 2 * stride);
            if (i >= 2 && !mbar_wait(&S.sm.empty[b], ((i >> 1) - 1) & 1, A.wait_ns)) {
                ok = false;
                break;
            }
            if (*(volatile int *)&S.sm.abort) break;
            if (cached && row == 0) {   // X panel b is free: the forward's copy of this tile's panel
                bulk_load(S.x[b], A.xcache + (size_t)tile * kPanelBytes, kPanelBytes, &S.sm.xl[b]);
                ++nload[b];
            }
            if (BWD && i >= 2) scatter_row<PK>(A, S, b, (i - 2) & 3, row);   // feature gradients of tile i - 2
            produce_row<FeatT, BWD, PEX, PK>(A, S, b, i & 3, kv_cur, rp_cur, row, cached);
            fence_async_smem();
            // (testing aid: one arrival withheld on a chosen tile makes the consumers' wait run out)
            if (!(row == 0 && tile + 1 == A.withhold_tile)) mbar_arrive(&S.sm.full[b]);
            kv_cur = kv_next;
            rp_cur = rp_next;
            kv_next = kv_after;
        }
        if (BWD && ok) {
            // the last (up to) two tiles: wait until the consumers are done with them, then scatter
            for (int j = (i >= 2 ? i - 2 : 0); j < i && ok; ++j) {
                if (!mbar_wait(&S.sm.empty[j & 1], (j >> 1) & 1, A.wait_ns)) ok = false;
                else if (!*(volatile int *)&S.sm.abort) scatter_row<PK>(A, S, j & 1, j & 3, row);
            }
        }
        // every bulk load issued has landed before the CTA can exit (bounded)
        for (int bb = 0; bb < 2; ++bb)
            if (nload[bb] > 0) mbar_wait(&S.sm.xl[bb], (nload[bb] - 1) & 1, A.wait_ns);
        if (!ok) atomicExch(&S.sm.abort, 1);
    } else if constexpr (!BWD) {
        // --------------------------- forward consumers: two groups ---------------------------
        // Group grp = warp / 4 takes every other tile of this CTA (the CTA's tiles i = grp, grp + 2,
        // ..., so always X buffer grp), so that one group's epilogues run while the other group's
        // MMAs do.  Thread r = tid % 128 owns row r (its TMEM lane) and all 128 columns; the group
        // has its own 256 TMEM columns, MMA barrier and named barrier (2 + grp, 128 threads).  The
        // hidden activations never go to shared memory: each epilogue writes them back to TMEM as
        // BF16 (two per column) and the next layer reads its A operand from there.  Columns:
        // Z1 at +0, then H1 at +0 (64 columns, over the Z1 values already read) and H2 at +64;
        // Z2 at +128, then O at +128.
        constexpr uint32_t F_H1 = 0, F_H2 = 64, F_Z2 = 128, F_O = 128;
        const int grp = warp >> 2, r = tid & (TM - 1);
        const uint32_t tb = S.sm.tmem_base + 256u * (uint32_t)grp;
        uint64_t *mbar = grp ? &S.sm.mma1 : &S.sm.mma;
        uint32_t mphase = 0;
        auto wait_mma = [&]() -> bool {
            bool w = mbar_wait(mbar, mphase, A.wait_ns);
            mphase ^= 1;
            fence_after();
            return w;
        };
        auto group_sync = [&]() {
            fence_before();
            if (grp) asm volatile("bar.sync 3, 128;" ::: "memory");
            else asm volatile("bar.sync 2, 128;" ::: "memory");
            fence_after();
        };
        int i = grp;
        for (int tile = blockIdx.x + grp * gridDim.x; tile < ntiles; tile += 2 * gridDim.x, i += 2) {
            const int b = grp;
            uint32_t x_ = smem_u32(S.x[b]), w1t_ = smem_u32(S.w1t), w2t_ = smem_u32(S.w2t), w3p_ = smem_u32(S.tp);
            asm volatile("" : "+r"(x_), "+r"(w1t_), "+r"(w2t_), "+r"(w3p_));
            // (no abort-flag test here: two warps of a group could read it on either side of its
            // setting and part at the group barrier; a failed producer instead leaves this wait
            // unsatisfied for every thread of the group alike)
            if (!mbar_wait(&S.sm.full[b], (i >> 1) & 1, A.wait_ns)) ok = false;
            fence_after();
            if (!ok) break;
            const int slot = S.sm.slot[i & 3][r];
            // ---- layer 1: Z1 = X W1 ----
            if (r == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 4; ++kk)
                    mma(tb + COL_Z1, desc_kmajor(x_, kk), desc_kmajor(w1t_, kk), idesc_bf16(128, 128, 0, 0), kk > 0);
                if (PEX)
                    mma(tb + COL_Z1, desc_kmajor(w3p_, 1 + b), desc_kmajor(w3p_, 3), idesc_bf16(128, 128, 0, 0), 1u);
                commit(mbar);
                if (A.xcache) bulk_store(A.xcache + (size_t)tile * kPanelBytes, S.x[b], kPanelBytes);   // for the backward
            }
            if (!wait_mma()) { ok = false; break; }
            if (r == 0) {   // X[b] is free once layer 1 and the copy have read it
                if (A.xcache) bulk_wait_read();
                mbar_arrive(&S.sm.empty[b]);
            }
            // ---- epilogue 1: H1 = relu(Z1), all 128 columns of my row, as BF16 into TMEM (32-column
            //      chunk g of Z1 becomes columns 16 g .. 16 g + 15, which chunks before g held) ----
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
                float z[32];
                tmem_ld32(taddr(tb, warp, COL_Z1 + 32 * g), z);
                uint32_t h[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) h[k] = pack_bf16(fmaxf(z[2 * k], 0.0f), fmaxf(z[2 * k + 1], 0.0f));
                tmem_st16(taddr(tb, warp, F_H1 + 16 * g), h);
            }
            tmem_wait_st();
            group_sync();
            // ---- layer 2: Z2 = H1 W2, A = H1 from TMEM ----
            if (r == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk)
                    mma_ts(tb + F_Z2, tb + F_H1 + 8u * (uint32_t)kk, desc_kmajor(w2t_, kk), idesc_bf16(128, 128, 0, 0),
                           kk > 0);
                commit(mbar);
            }
            if (!wait_mma()) { ok = false; break; }
            // ---- epilogue 2: H2 = relu(Z2 + b2), as BF16 into TMEM ----
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
                float z[32];
                tmem_ld32(taddr(tb, warp, F_Z2 + 32 * g), z);
                uint32_t h[16];
#pragma unroll
                for (int k = 0; k < 32; k += 4) {
                    const float4 bb = *reinterpret_cast<const float4 *>(&S.sm.b2[32 * g + k]);
                    h[k / 2] = pack_bf16(fmaxf(z[k] + bb.x, 0.0f), fmaxf(z[k + 1] + bb.y, 0.0f));
                    h[k / 2 + 1] = pack_bf16(fmaxf(z[k + 2] + bb.z, 0.0f), fmaxf(z[k + 3] + bb.w, 0.0f));
                }
                tmem_st16(taddr(tb, warp, F_H2 + 16 * g), h);
            }
            tmem_wait_st();
            group_sync();
            // ---- layer 3: O = H2 W3 (N = 16, columns 0-2 used), A = H2 from TMEM ----
            if (r == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk)
                    mma_ts(tb + F_O, tb + F_H2 + 8u * (uint32_t)kk, desc_mnmajor(w3p_, kk), idesc_bf16(128, 16, 0, 1),
                           kk > 0);
                commit(mbar);
            }
            if (!wait_mma()) { ok = false; break; }
            float o[16];
            tmem_ld16(taddr(tb, warp, F_O), o);
            if (slot >= 0) {
                float *sp = reinterpret_cast<float *>(A.samp + slot);
                sp[1] = sigmoidf_(o[0] + S.sm.b3[0]);
                sp[2] = sigmoidf_(o[1] + S.sm.b3[1]);
                sp[3] = sigmoidf_(o[2] + S.sm.b3[2]);
            }
            group_sync();   // TMEM reads and panel reads done before this group's next MMAs
        }
        if (r == 0 && A.xcache) bulk_wait_all();   // the copies are complete before the kernel ends
        if (!ok) atomicExch(&S.sm.abort, 1);
    } else {
        // ------------------------------- consumers -------------------------------
        // thread: row r = 32 (warp % 4) + lane (its TMEM lane), column half hc = warp / 4
        const int r = tid & (TM - 1), hc = tid >> 7;
        const uint32_t tb = S.sm.tmem_base;
        uint32_t mphase = 0;
        float db3_part[3] = {0.0f, 0.0f, 0.0f};
        int i = 0;
        // waits for the current MMA batch; on a timeout every consumer leaves the loop
        auto wait_mma = [&]() -> bool {
            bool w = mbar_wait(&S.sm.mma, mphase, A.wait_ns);
            mphase ^= 1;
            fence_after();
            return w;
        };
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            const uint32_t acc_w = i > 0 ? 1u : 0u;   // first tile of this CTA initialises the accumulators
            // opaque copies: keeps the compiler from hoisting every MMA descriptor out of the loop
            uint32_t x_ = smem_u32(S.x[b]), w1t_ = smem_u32(S.w1t), w2t_ = smem_u32(S.w2t), w3p_ = smem_u32(S.tp);
            uint32_t h1_ = smem_u32(S.h1), h2_ = smem_u32(S.h2), dz2_ = smem_u32(S.dz2), dout_ = smem_u32(S.dout);
            asm volatile("" : "+r"(x_), "+r"(w1t_), "+r"(w2t_), "+r"(w3p_), "+r"(h1_), "+r"(h2_), "+r"(dz2_), "+r"(dout_));
            // (no abort-flag test: consumers reading it on either side of its setting would part at
            // their named barrier; a failed producer leaves this wait unsatisfied for all of them)
            if (!mbar_wait(&S.sm.full[b], (i >> 1) & 1, A.wait_ns)) ok = false;
            else if (cached && !mbar_wait(&S.sm.xl[b], (i >> 1) & 1, A.wait_ns)) ok = false;
            fence_after();
            if (!ok) break;
            // per-row tables of buffer b, read before the buffer is handed back to the producers
            const int slot = S.sm.slot[i & 3][r];
            const float d0 = BWD ? S.sm.dc[b][r][0] : 0.0f, d1 = BWD ? S.sm.dc[b][r][1] : 0.0f,
                        d2 = BWD ? S.sm.dc[b][r][2] : 0.0f;
            // ---- layer 1: Z1 = X W1 ----
            if (tid == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 4; ++kk)
                    mma(tb + COL_Z1, desc_kmajor(x_, kk), desc_kmajor(w1t_, kk), idesc_bf16(128, 128, 0, 0), kk > 0);
                if (PEX)   // the X tail (k-step 1 + b of the tail panel) against the W1 tail (k-step 3)
                    mma(tb + COL_Z1, desc_kmajor(w3p_, 1 + b), desc_kmajor(w3p_, 3), idesc_bf16(128, 128, 0, 0), 1u);
                commit(&S.sm.mma);
            }
            if (!wait_mma()) { ok = false; break; }
            if (!BWD && tid == 0) mbar_arrive(&S.sm.empty[b]);   // X[b] is free once layer 1 is done
            // ---- epilogue 1: H1 = relu(Z1), my 64 columns ----
            uint32_t m1lo = 0u, m1hi = 0u;   // ReLU masks of my 64 columns
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                float z[32];
                tmem_ld32(taddr(tb, warp, COL_Z1 + 64 * hc + 32 * g), z);
                uint32_t bits = 0;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    bits |= (z[k] > 0.0f ? 1u : 0u) << k;
                    z[k] = fmaxf(z[k], 0.0f);
                }
                if (g == 0) m1lo = bits;
                else m1hi = bits;
#pragma unroll
                for (int k = 0; k < 32; k += 8) panel_store8(S.h1 + hc * kPanelBytes, r, 32 * g + k, z + k);
            }
            // dout = dL/dc c (1 - c), formed by the producers, into the dout panel: the operand of
            // dH2 (issued with layer 2), of dW3 and, through its constant-1 column, of db2
            if (BWD && hc == 0) {
                db3_part[0] += d0;
                db3_part[1] += d1;
                db3_part[2] += d2;
                uint2 q;
                q.x = pack_bf16(d0, d1);
                q.y = pack_bf16(d2, 1.0f);
                *reinterpret_cast<uint2 *>(S.dout + panel_offset(r, 0)) = q;
            }
            consumer_publish();
            // ---- layer 2: Z2 = H1 W2; in the backward also dH2 = dout W3^T (K = 16: dout's columns
            //      [dL/do, 1, 0 ...] against the tail panel's [W3, 0 ...]) into Z1's columns, which
            //      epilogue 1 has read ----
            if (tid == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk)
                    mma(tb + COL_Z2, desc_kmajor(h1_, kk), desc_kmajor(w2t_, kk), idesc_bf16(128, 128, 0, 0), kk > 0);
                if (BWD)
                    mma(tb + COL_Z1, desc_kmajor(dout_, 0), desc_kmajor(w3p_, 0), idesc_bf16(128, 128, 0, 0), 0u);
                commit(&S.sm.mma);
            }
            if (!wait_mma()) { ok = false; break; }
            // ---- epilogue 2: H2 = relu(Z2 + b2), my 64 columns; in the backward also
            //      dZ2 = dH2 [Z2 + b2 > 0] ----
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                const int col = 64 * hc + 32 * g;
                float z[32], dz[32];
                tmem_ld32(taddr(tb, warp, COL_Z2 + col), z);
                if (BWD) tmem_ld32(taddr(tb, warp, COL_Z1 + col), dz);
#pragma unroll
                for (int k = 0; k < 32; k += 4) {
                    const float4 bb = *reinterpret_cast<const float4 *>(&S.sm.b2[col + k]);
                    const float hb[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float h = z[k + j] + hb[j];
                        z[k + j] = fmaxf(h, 0.0f);
                        if (BWD) dz[k + j] = h > 0.0f ? dz[k + j] : 0.0f;
                    }
                }
#pragma unroll
                for (int k = 0; k < 32; k += 8) panel_store8(S.h2 + hc * kPanelBytes, r, 32 * g + k, z + k);
                if (BWD) {
#pragma unroll
                    for (int k = 0; k < 32; k += 8) panel_store8(S.dz2 + hc * kPanelBytes, r, 32 * g + k, dz + k);
                }
            }
            if (!BWD) {
                consumer_publish();
                // ---- layer 3: O = H2 W3 (N = 16, columns 0-2 used) ----
                if (tid == 0) {
#pragma unroll 1
                    for (int kk = 0; kk < 8; ++kk)
                        mma(tb + COL_O, desc_kmajor(h2_, kk), desc_mnmajor(w3p_, kk), idesc_bf16(128, 16, 0, 1),
                            kk > 0);
                    commit(&S.sm.mma);
                }
                if (!wait_mma()) { ok = false; break; }
                float o[16];
                tmem_ld16(taddr(tb, warp, COL_O), o);
                const float c0 = sigmoidf_(o[0] + S.sm.b3[0]), c1 = sigmoidf_(o[1] + S.sm.b3[1]),
                            c2 = sigmoidf_(o[2] + S.sm.b3[2]);
                if (slot >= 0 && hc == 0) {
                    float *sp = reinterpret_cast<float *>(A.samp + slot);
                    sp[1] = c0;
                    sp[2] = c1;
                    sp[3] = c2;
                }
                consumer_sync();   // TMEM reads done before the next tile's MMAs
                continue;
            }
            // ---- backward: H2 and dZ2 published for batch A ----
            consumer_publish();
            if (tid == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk) {
                    mma(tb + COL_Z2, desc_kmajor(dz2_, kk), desc_mnmajor(w2t_, kk), idesc_bf16(128, 128, 0, 1), kk > 0);  // dH1
                    mma(tb + COL_DW2T, desc_mnmajor(dz2_, kk), desc_mnmajor(h1_, kk), idesc_bf16(128, 144, 1, 1),
                        acc_w | (kk > 0));   // [dW2^T | db2]: B = [H1 | dout]
                    mma(tb + COL_DW3, desc_mnmajor(h2_, kk), desc_mnmajor(dout_, kk), idesc_bf16(128, 16, 1, 1),
                        acc_w | (kk > 0));
                }
                commit(&S.sm.mma);
            }
            if (!wait_mma()) { ok = false; break; }
            // ---- dZ1 = dH1 [Z1 > 0], over H1 ----
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                const uint32_t bits = g == 0 ? m1lo : m1hi;
                float z[32];
                tmem_ld32(taddr(tb, warp, COL_Z2 + 64 * hc + 32 * g), z);
#pragma unroll
                for (int k = 0; k < 32; ++k) z[k] = ((bits >> k) & 1u) ? z[k] : 0.0f;
#pragma unroll
                for (int k = 0; k < 32; k += 8) panel_store8(S.h1 + hc * kPanelBytes, r, 32 * g + k, z + k);
            }
            consumer_publish();
            if (tid == 0) {
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk) {
                    mma(tb + COL_DE, desc_kmajor(h1_, kk), desc_mnmajor(w1t_, kk), idesc_bf16(128, 16, 0, 1), kk > 0);
                    mma(tb + COL_DW1, desc_mnmajor(h1_, kk), desc_mnmajor(x_, kk), idesc_bf16(128, 64, 1, 1),
                        acc_w | (kk > 0));
                    if (PEX)
                        mma(tb + COL_DW1T, desc_mnmajor(h1_, kk), desc_mnmajor(w3p_ + 32u * (1 + b), kk),
                            idesc_bf16(128, 16, 1, 1), acc_w | (kk > 0));
                }
                commit(&S.sm.mma);
            }
            if (!wait_mma()) { ok = false; break; }
            // ---- stage de[0:12] for the producers' scatter, then release X[b] ----
            {
                float de[16];
                tmem_ld16(taddr(tb, warp, COL_DE), de);
                if (hc == 0) {
                    *de_slot(S.dout, b, r, 0) = make_float4(de[0], de[1], de[2], de[3]);
                    *de_slot(S.dout, b, r, 1) = make_float4(de[4], de[5], de[6], de[7]);
                    *de_slot(S.dout, b, r, 2) = make_float4(de[8], de[9], de[10], de[11]);
                }
            }
            consumer_sync();
            if (tid == 0) mbar_arrive(&S.sm.empty[b]);   // X[b] consumed, de staged
        }
        ntile_mine = i;
        if (!ok) atomicExch(&S.sm.abort, 1);
        if (BWD) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float sum = warp_sum(db3_part[ch]);
                if ((tid & 31) == 0) atomicAdd(&S.sm.db3[ch], sum);
            }
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    const bool failed = S.sm.abort != 0;
    if (failed) {
        if (tid == 0) atomicOr(&A.hdr->flags, 2);
        // an MMA batch whose completion timed out may still be running: wait (bounded) once more
        if (tid < NC) mbar_wait((!BWD && tid >= TM) ? &S.sm.mma1 : &S.sm.mma, 0, A.wait_ns);
    }
    if (BWD && !failed && tid < NC && ntile_mine > 0) {
        const uint32_t tb = S.sm.tmem_base;
        const int r = tid & (TM - 1), hc = tid >> 7;
        float *gW1 = A.grad_mlp, *gB1 = gW1 + D::IN * HID, *gW2 = gB1 + HID, *gB2 = gW2 + HID * HID;
        float *gW3 = gB2 + HID, *gB3 = gW3 + HID * 3;
        // dW2^T: lane = output unit r, columns = input units (64 per half); column 128 + 3 = db2
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const int col = 64 * hc + 32 * c;
            float v[32];
            tmem_ld32(taddr(tb, warp, COL_DW2T + col), v);
#pragma unroll
            for (int k = 0; k < 32; ++k) atomicAdd(gW2 + (col + k) * HID + r, v[k]);
        }
        // [dW1 | db1]^T: lane = hidden unit r, columns = X columns (BIAS = bias), 32 per half
        {
            float v[32];
            tmem_ld32(taddr(tb, warp, COL_DW1 + 32 * hc), v);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int kin = 32 * hc + k;
                if (kin < D::NMAIN) atomicAdd(gW1 + kin * HID + r, v[k]);
                else if (kin == D::BIAS) atomicAdd(gB1 + r, v[k]);
            }
        }
        if constexpr (PEX) {   // dW1 tail^T: columns = inputs NMAIN..IN-1
            float v[16];
            tmem_ld16(taddr(tb, warp, COL_DW1T), v);
            if (hc == 0)
#pragma unroll
                for (int t = 0; t < D::NTAIL; ++t) atomicAdd(gW1 + (D::NMAIN + t) * HID + r, v[t]);
        }
        float v[16];
        tmem_ld16(taddr(tb, warp, COL_DW3), v);
        if (hc == 0) {
            atomicAdd(gW3 + r * 3 + 0, v[0]);
            atomicAdd(gW3 + r * 3 + 1, v[1]);
            atomicAdd(gW3 + r * 3 + 2, v[2]);
        }
        tmem_ld16(taddr(tb, warp, COL_DW2T + 128), v);
        if (hc == 0) atomicAdd(gB2 + r, v[3]);
        if (tid < 3) atomicAdd(gB3 + tid, S.sm.db3[tid]);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(S.sm.tmem_base, NCOLS);
}

template <typename FeatT, bool BWD, bool PEX, bool PK>
void launch_tc(const RenderArgs &A, int kind, cudaStream_t s) {
    auto kern = fine_colour_tc_kernel<FeatT, BWD, PEX, PK>;
    const int bytes = (int)smem_bytes(BWD);
    ensure_smem(reinterpret_cast<const void *>(kern), bytes);
    ProfScope ps_(kind, s);
    kern<<<num_sms(), kThreads<BWD>, bytes, s>>>(A);
}

template <bool BWD>
void launch_tc_any(const RenderArgs &A, cudaStream_t s) {
    const int kind = BWD ? DVGO_K_FINE_COLOUR_BWD : DVGO_K_FINE_COLOUR_FWD;
    const bool bf = A.cdtype == DVGO_DTYPE_BF16, pex = A.nfreq_pos > 0;
    if (A.packed) {
        if (bf && pex) launch_tc<__nv_bfloat16, BWD, true, true>(A, kind, s);
        else if (bf) launch_tc<__nv_bfloat16, BWD, false, true>(A, kind, s);
        else if (pex) launch_tc<float, BWD, true, true>(A, kind, s);
        else launch_tc<float, BWD, false, true>(A, kind, s);
    } else {
        if (bf && pex) launch_tc<__nv_bfloat16, BWD, true, false>(A, kind, s);
        else if (bf) launch_tc<__nv_bfloat16, BWD, false, false>(A, kind, s);
        else if (pex) launch_tc<float, BWD, true, false>(A, kind, s);
        else launch_tc<float, BWD, false, false>(A, kind, s);
    }
}

}  // namespace

int launch_fine_colour_fwd_tc(const RenderArgs &A, cudaStream_t s) {
    launch_tc_any<false>(A, s);
    return DVGO_OK;
}

int launch_fine_colour_bwd_tc(const RenderArgs &A, cudaStream_t s) {
    launch_tc_any<true>(A, s);
    return DVGO_OK;
}

}  // namespace dvgo
