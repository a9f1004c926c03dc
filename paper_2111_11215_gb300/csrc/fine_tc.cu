// fine_tc.cu -- colour queries of the fine stage with the BF16 tensor-core MLP (tcgen05, sm_103a).
//
// Same function as fine_simt.cu (Sec. 4.2 Eq. fine_queries_rgb, Supp. A: 12 features + PE(d, 4)
// = 39 inputs, two hidden layers of 128 with ReLU, sigmoid output) with the two 128-wide layers
// and all weight-gradient contractions on the 5th-generation tensor cores: BF16 operands in
// shared memory (128-byte swizzled panels, see tc_helpers.cuh), FP32 accumulators in TMEM, MMAs
// issued by one thread, completion signalled through an mbarrier.  The 128 -> 3 output layer,
// the sigmoid and the element-wise steps run on the CUDA cores in the epilogues.
//
// Persistent CTAs of 128 threads walk tiles of M = 128 kept samples; thread r owns sample row r
// of the tile (and TMEM lane r) for the gather, the epilogues and the feature scatter.
//
// Forward per tile:  X[128x64] (features, PE(d), 1) -> Z1 = X W1|b1 (TMEM) -> H1 = relu (BF16, smem)
//                    -> Z2 = H1 W2 (TMEM) -> h2 = relu(Z2 + b2), c = sigmoid(h2 W3 + b3).
// Backward per tile (recomputes the forward), with dL/dc from the compositing backward:
//   dout = dL/dc c (1 - c); dZ2 = (dout W3^T) [Z2 + b2 > 0]                         (epilogue)
//   dH1 = dZ2 W2^T;  dW2 += H1^T dZ2;  dW3 += H2^T dout;  db2 += dZ2^T 1            (MMAs)
//   dZ1 = dH1 [Z1 > 0]                                                              (epilogue)
//   de = dZ1 W1[0:16]^T;  [dW1 | db1]^T += dZ1^T X                                  (MMAs)
//   de[0:12] scattered to the feature grid with the trilinear weights              (epilogue)
// TMEM columns: Z1 [0,128), Z2 / dH1 [128,256), dW2 [256,384), dW1^T [384,448), dW3 [448,464),
// db2 [464,480), de [480,496).  The weight-gradient accumulators live in TMEM for the whole
// launch and are added to global memory once per CTA.

#include <stddef.h>

#include "dvgo_internal.cuh"
#include "tc_helpers.cuh"

namespace dvgo {

namespace {

using namespace tc;

constexpr int TM = 128;
constexpr int NT = 128;
constexpr int HID = 128;
constexpr int FEAT = 12;
constexpr int NF = 4;
constexpr int IN = FEAT + 3 + 6 * NF;   // 39; column 39 of X carries the first-layer bias

constexpr uint32_t COL_Z1 = 0, COL_Z2 = 128, COL_DW2 = 256, COL_DW1 = 384, COL_DW3 = 448, COL_DB2 = 464,
                   COL_DE = 480;

// Small per-CTA state, padded to a multiple of 1024 bytes so that the panels after it stay
// aligned to the 128-byte-swizzle atom.
struct alignas(1024) SmallTC {
    float w3[HID * 3];
    float b2[HID];
    float b3[4];
    float db3[4];
    uint64_t mbar;
    uint32_t tmem_base;
};

struct SmemTC {
    unsigned char w1t[kPanelBytes];       // W1|b1 transposed: row = hidden unit, 64 input columns
    unsigned char w2t[2 * kPanelBytes];   // W2 transposed: row = output unit, 128 input columns
    unsigned char x[kPanelBytes];         // X: row = sample
    unsigned char h1[2 * kPanelBytes];    // H1, later dZ1
    SmallTC sm;
    // backward only (the forward allocates the struct up to here)
    unsigned char h2[2 * kPanelBytes];    // H2
    unsigned char dz2[2 * kPanelBytes];   // dZ2
    unsigned char dout[kPanelBytes];      // [dout_r, dout_g, dout_b, 1, 0, ...]
};

constexpr size_t smem_bytes(bool bwd) { return (bwd ? sizeof(SmemTC) : offsetof(SmemTC, h2)) + 1024; }

struct RowInfo {
    int slot;           // sample slot, -1 for padding rows
    int cbase;          // flat index of the base corner
    float fx, fy, fz;   // fractional offsets
};

// Gather one sample row into X (features, direction encoding, bias column) and remember where it
// sits in the grid.
template <typename FeatT>
__device__ __forceinline__ RowInfo gather_row(const RenderArgs &A, unsigned char *xp, int e, int n_kept, int row) {
    RowInfo ri;
    ri.slot = -1;
    ri.cbase = 0;
    ri.fx = ri.fy = ri.fz = 0.0f;
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
    if (e < n_kept) {
        int2 kv = A.kept[e];
        const RayRec &rr = A.rays[kv.y];
        double t;
        float dt;
        sample_t(A, rr, kv.y, kv.x - rr.off, t, dt);
        double u[3];
        lattice_coord(rr, t, u);
        Cell c = make_cell(u, A.nx, A.ny, A.nz);
        ri.slot = kv.x;
        ri.cbase = (int)corner_index(c, 0, A.ny, A.nz);
        ri.fx = c.fx;
        ri.fy = c.fy;
        ri.fz = c.fz;
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // corner pairs (x bit, y bit) with z = 0, 1 adjacent
            int qa = q << 1;
            long long idx0 = corner_index(c, qa, A.ny, A.nz);
            float w0 = corner_weight(c, qa), w1 = corner_weight(c, qa | 1);
            const FeatT *g = static_cast<const FeatT *>(A.cgrid) + idx0 * FEAT;
            if constexpr (sizeof(FeatT) == 4) {
                const float4 *g4 = reinterpret_cast<const float4 *>(g);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float4 a = __ldg(g4 + k), b = __ldg(g4 + 3 + k);
                    v[4 * k + 0] += w0 * a.x + w1 * b.x;
                    v[4 * k + 1] += w0 * a.y + w1 * b.y;
                    v[4 * k + 2] += w0 * a.z + w1 * b.z;
                    v[4 * k + 3] += w0 * a.w + w1 * b.w;
                }
            } else {
                const uint2 *g2 = reinterpret_cast<const uint2 *>(g);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    uint2 a = __ldg(g2 + k), b = __ldg(g2 + 3 + k);
                    float2 a0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&a.x));
                    float2 a1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&a.y));
                    float2 b0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&b.x));
                    float2 b1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&b.y));
                    v[4 * k + 0] += w0 * a0.x + w1 * b0.x;
                    v[4 * k + 1] += w0 * a0.y + w1 * b0.y;
                    v[4 * k + 2] += w0 * a1.x + w1 * b1.x;
                    v[4 * k + 3] += w0 * a1.y + w1 * b1.y;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float d = rr.dir[a];
            v[FEAT + a] = d;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                float s, cs;
                sincosf(ldexpf(d, k), &s, &cs);
                v[FEAT + 3 + a * NF + k] = s;
                v[FEAT + 3 + 3 * NF + a * NF + k] = cs;
            }
        }
        v[IN] = 1.0f;
    }
#pragma unroll
    for (int c = 0; c < 64; c += 8) panel_store8(xp, row, c, v + c);
    return ri;
}

__device__ __forceinline__ void sync_all() {
    fence_before();
    __syncthreads();
    fence_after();
}

// Operands written by the CUDA cores become visible to the tensor core, then the block syncs.
__device__ __forceinline__ void publish_smem() {
    fence_async_smem();
    sync_all();
}

template <typename FeatT, bool BWD>
__global__ void __launch_bounds__(NT, BWD ? 1 : 2) fine_colour_tc_kernel(RenderArgs A) {
    extern __shared__ unsigned char smem_raw[];
    SmemTC &S = *reinterpret_cast<SmemTC *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t NCOLS = BWD ? 512 : 256;

    if (tid == 0) mbar_init(&S.sm.mbar, 1);
    if (warp == 0) tmem_alloc(&S.sm.tmem_base, NCOLS);
    // weights: row n = tid of W1^T (64 input columns, bias in column 39) and of W2^T
    {
        float v[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = k < IN ? A.w1[k * HID + tid] : (k == IN ? A.b1[tid] : 0.0f);
#pragma unroll
        for (int c = 0; c < 64; c += 8) panel_store8(S.w1t, tid, c, v + c);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = A.w2[(p * 64 + k) * HID + tid];
#pragma unroll
            for (int c = 0; c < 64; c += 8) panel_store8(S.w2t + p * kPanelBytes, tid, c, v + c);
        }
        if (BWD) {
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = 0.0f;
#pragma unroll
            for (int c = 0; c < 64; c += 8) panel_store8(S.dout, tid, c, v + c);
        }
        for (int i = tid; i < HID * 3; i += NT) S.sm.w3[i] = A.w3[i];
        S.sm.b2[tid] = A.b2[tid];
        if (tid < 3) S.sm.b3[tid] = A.b3[tid];
        if (tid < 4) S.sm.db3[tid] = 0.0f;
    }
    publish_smem();
    const uint32_t tb = S.sm.tmem_base;
    const uint32_t a_w1t = smem_u32(S.w1t), a_w2t = smem_u32(S.w2t), a_x = smem_u32(S.x), a_h1 = smem_u32(S.h1);
    const uint32_t a_h2 = smem_u32(S.h2), a_dz2 = smem_u32(S.dz2), a_dout = smem_u32(S.dout);
    const uint32_t id_128 = idesc_bf16(128, 128, 0, 0);
    uint32_t phase = 0;
    bool ok = true;
    float db3_part[3] = {0.0f, 0.0f, 0.0f};

    const int n_kept = A.hdr->n_kept;
    const int ntiles = (n_kept + TM - 1) / TM;
    bool any = false;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const uint32_t acc_w = any ? 1u : 0u;   // first tile of this CTA initialises the accumulators
        any = true;
        // ---- gather X ----
        RowInfo ri = gather_row<FeatT>(A, S.x, tile * TM + tid, n_kept, tid);
        publish_smem();
        // ---- layer 1: Z1 = X W1 ----
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma(tb + COL_Z1, desc_kmajor(a_x, kk), desc_kmajor(a_w1t, kk), id_128, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        // ---- epilogue 1: H1 = relu(Z1) ----
        uint32_t m1[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z1 + 32 * c), z);
            uint32_t bits = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                bits |= (z[i] > 0.0f ? 1u : 0u) << i;
                z[i] = fmaxf(z[i], 0.0f);
            }
            m1[c] = bits;
#pragma unroll
            for (int i = 0; i < 32; i += 8) panel_store8(S.h1 + (c >> 1) * kPanelBytes, tid, (32 * c + i) & 63, z + i);
        }
        publish_smem();
        // ---- layer 2: Z2 = H1 W2 ----
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma(tb + COL_Z2, desc_kmajor(a_h1, kk), desc_kmajor(a_w2t, kk), id_128, kk > 0);
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        // ---- epilogue 2: h2 = relu(Z2 + b2), c = sigmoid(h2 W3 + b3) ----
        float o0 = S.sm.b3[0], o1 = S.sm.b3[1], o2 = S.sm.b3[2];
        uint32_t m2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z2 + 32 * c), z);
            uint32_t bits = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                int j = 32 * c + i;
                float h = z[i] + S.sm.b2[j];
                bits |= (h > 0.0f ? 1u : 0u) << i;
                h = fmaxf(h, 0.0f);
                z[i] = h;
                o0 = fmaf(h, S.sm.w3[3 * j + 0], o0);
                o1 = fmaf(h, S.sm.w3[3 * j + 1], o1);
                o2 = fmaf(h, S.sm.w3[3 * j + 2], o2);
            }
            m2[c] = bits;
            if (BWD) {
#pragma unroll
                for (int i = 0; i < 32; i += 8) panel_store8(S.h2 + (c >> 1) * kPanelBytes, tid, (32 * c + i) & 63, z + i);
            }
        }
        const float c0 = sigmoidf_(o0), c1 = sigmoidf_(o1), c2 = sigmoidf_(o2);
        if (!BWD) {
            if (ri.slot >= 0) {
                float *sp = reinterpret_cast<float *>(A.samp + ri.slot);
                sp[1] = c0;
                sp[2] = c1;
                sp[3] = c2;
            }
            continue;
        }
        // ---- backward epilogue 2: dout, dZ2 ----
        float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f;
        if (ri.slot >= 0) {
            const float4 gc = A.sgrad[ri.slot];
            d0 = gc.y * c0 * (1.0f - c0);
            d1 = gc.z * c1 * (1.0f - c1);
            d2 = gc.w * c2 * (1.0f - c2);
        }
        db3_part[0] += d0;
        db3_part[1] += d1;
        db3_part[2] += d2;
        {
            uint2 q;
            q.x = pack_bf16(d0, d1);
            q.y = pack_bf16(d2, 1.0f);
            *reinterpret_cast<uint2 *>(S.dout + panel_offset(tid, 0)) = q;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float z[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                int j = 32 * c + i;
                float dh = d0 * S.sm.w3[3 * j] + d1 * S.sm.w3[3 * j + 1] + d2 * S.sm.w3[3 * j + 2];
                z[i] = ((m2[c] >> i) & 1u) ? dh : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 32; i += 8) panel_store8(S.dz2 + (c >> 1) * kPanelBytes, tid, (32 * c + i) & 63, z + i);
        }
        publish_smem();
        if (tid == 0) {
            const uint32_t id_mk = idesc_bf16(128, 128, 0, 1);   // K-major A, MN-major B
            const uint32_t id_mm = idesc_bf16(128, 128, 1, 1);
            const uint32_t id_n16 = idesc_bf16(128, 16, 1, 1);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                mma(tb + COL_Z2, desc_kmajor(a_dz2, kk), desc_mnmajor(a_w2t, kk), id_mk, kk > 0);      // dH1
                mma(tb + COL_DW2, desc_mnmajor(a_h1, kk), desc_mnmajor(a_dz2, kk), id_mm, acc_w | (kk > 0));
                mma(tb + COL_DW3, desc_mnmajor(a_h2, kk), desc_mnmajor(a_dout, kk), id_n16, acc_w | (kk > 0));
                mma(tb + COL_DB2, desc_mnmajor(a_dz2, kk), desc_mnmajor(a_dout, kk), id_n16, acc_w | (kk > 0));
            }
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        // ---- backward epilogue 3: dZ1 = dH1 [Z1 > 0], over H1 ----
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float z[32];
            tmem_ld32(taddr(tb, warp, COL_Z2 + 32 * c), z);
#pragma unroll
            for (int i = 0; i < 32; ++i) z[i] = ((m1[c] >> i) & 1u) ? z[i] : 0.0f;
#pragma unroll
            for (int i = 0; i < 32; i += 8) panel_store8(S.h1 + (c >> 1) * kPanelBytes, tid, (32 * c + i) & 63, z + i);
        }
        publish_smem();
        if (tid == 0) {
            const uint32_t id_de = idesc_bf16(128, 16, 0, 1);
            const uint32_t id_w1 = idesc_bf16(128, 64, 1, 1);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                mma(tb + COL_DE, desc_kmajor(a_h1, kk), desc_mnmajor(a_w1t, kk), id_de, kk > 0);
                mma(tb + COL_DW1, desc_mnmajor(a_h1, kk), desc_mnmajor(a_x, kk), id_w1, acc_w | (kk > 0));
            }
            commit(&S.sm.mbar);
        }
        ok = mbar_wait(&S.sm.mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        fence_after();
        // ---- backward epilogue 4: scatter de[0:12] to the feature grid ----
        {
            float de[16];
            tmem_ld16(taddr(tb, warp, COL_DE), de);
            if (ri.slot >= 0) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    int bx = (q >> 2) & 1, by = (q >> 1) & 1, bz = q & 1;
                    float w = (bx ? ri.fx : 1.0f - ri.fx) * (by ? ri.fy : 1.0f - ri.fy) * (bz ? ri.fz : 1.0f - ri.fz);
                    long long idx = (long long)ri.cbase + (long long)bx * A.ny * A.nz + (long long)by * A.nz + bz;
                    float4 *g = reinterpret_cast<float4 *>(A.grad_cgrid + idx * FEAT);
                    atomicAdd(g + 0, make_float4(w * de[0], w * de[1], w * de[2], w * de[3]));
                    atomicAdd(g + 1, make_float4(w * de[4], w * de[5], w * de[6], w * de[7]));
                    atomicAdd(g + 2, make_float4(w * de[8], w * de[9], w * de[10], w * de[11]));
                }
            }
        }
        sync_all();
    }

    ok = !__syncthreads_or(!ok);   // block-uniform from here on
    if (!ok) {
        if (tid == 0) atomicOr(&A.hdr->flags, 2);
        mbar_wait(&S.sm.mbar, phase ^ 1);   // let the MMA that timed out finish (bounded)
    }
    sync_all();
    if (BWD && ok && any) {
        float *gW1 = A.grad_mlp, *gB1 = gW1 + IN * HID, *gW2 = gB1 + HID, *gB2 = gW2 + HID * HID;
        float *gW3 = gB2 + HID, *gB3 = gW3 + HID * 3;
        // dW2: lane = input unit (tid), columns = output units
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(taddr(tb, warp, COL_DW2 + 32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) atomicAdd(gW2 + tid * HID + 32 * c + i, v[i]);
        }
        // [dW1 | db1]^T: lane = hidden unit, columns = inputs (39 = bias)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float v[32];
            tmem_ld32(taddr(tb, warp, COL_DW1 + 32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                int k = 32 * c + i;
                if (k < IN) atomicAdd(gW1 + k * HID + tid, v[i]);
                else if (k == IN) atomicAdd(gB1 + tid, v[i]);
            }
        }
        {
            float v[16];
            tmem_ld16(taddr(tb, warp, COL_DW3), v);
            atomicAdd(gW3 + tid * 3 + 0, v[0]);
            atomicAdd(gW3 + tid * 3 + 1, v[1]);
            atomicAdd(gW3 + tid * 3 + 2, v[2]);
            tmem_ld16(taddr(tb, warp, COL_DB2), v);
            atomicAdd(gB2 + tid, v[3]);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = warp_sum(db3_part[ch]);
            if ((tid & 31) == 0) atomicAdd(&S.sm.db3[ch], s);
        }
        __syncthreads();
        if (tid < 3) atomicAdd(gB3 + tid, S.sm.db3[tid]);
    }
    sync_all();
    if (warp == 0) tmem_dealloc(tb, NCOLS);
}

// The forward holds 256 TMEM columns and ~100 KB of shared memory, so two CTAs share an SM; the
// backward holds all 512 columns, one CTA per SM.
template <typename FeatT, bool BWD>
void launch_tc(const RenderArgs &A, int kind, cudaStream_t s) {
    auto kern = fine_colour_tc_kernel<FeatT, BWD>;
    const int bytes = (int)smem_bytes(BWD);
    ensure_smem(reinterpret_cast<const void *>(kern), bytes);
    ProfScope ps_(kind, s);
    kern<<<num_sms() * (BWD ? 1 : 2), NT, bytes, s>>>(A);
}

}  // namespace

int launch_fine_colour_fwd_tc(const RenderArgs &A, cudaStream_t s) {
    if (A.cdtype == DVGO_DTYPE_BF16)
        launch_tc<__nv_bfloat16, false>(A, DVGO_K_FINE_COLOUR_FWD, s);
    else
        launch_tc<float, false>(A, DVGO_K_FINE_COLOUR_FWD, s);
    return DVGO_OK;
}

int launch_fine_colour_bwd_tc(const RenderArgs &A, cudaStream_t s) {
    if (A.cdtype == DVGO_DTYPE_BF16)
        launch_tc<__nv_bfloat16, true>(A, DVGO_K_FINE_COLOUR_BWD, s);
    else
        launch_tc<float, true>(A, DVGO_K_FINE_COLOUR_BWD, s);
    return DVGO_OK;
}

}  // namespace dvgo
