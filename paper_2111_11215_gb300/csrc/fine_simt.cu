// fine_simt.cu -- colour queries of the fine stage with the FP32 (SIMT) shallow MLP.
//
// Sec. 4.2 Eq. fine_queries_rgb and Supp. A: c = MLP(interp(x, V_feat), PE(d)[, PE(x)]) with D = 12
// feature channels, k_d = 4 direction frequencies, optionally k_x = 5 frequencies on the query
// point, two hidden layers of 128 and ReLU, sigmoid output.  Input row e = [feat (12), d (3),
// sin(2^k d_c) (12, c-major), cos(2^k d_c) (12)] (39 inputs), with PE(x) [x (3), sin(2^k x_c)
// (15), cos(2^k x_c) (15)] appended (72 inputs), and a constant 1 in the next column that carries
// the first-layer bias (W1 row IN = b1).
//
// Persistent CTAs (one per SM, 256 threads) walk tiles of 64 kept samples from the compact
// list.  Weights stay in shared memory for the whole launch.  Activations are stored
// feature-major ([feature][sample], row stride 68) so that the sample dimension of every GEMM
// is read with 16-byte vector loads; W1/W2 rows have stride 132 (a multiple of 4 that is not a
// multiple of 32) to spread the transposed reads of the backward over banks.
//
// Backward per tile: recompute gather + forward, then
//   dout = dL/dc * c (1 - c)                        (sigmoid)
//   dW3 += H2^T dout, db3 += sum dout
//   dZ2 = (dout W3^T) * [Z2 > 0],  dW2 += H1^T dZ2,  db2 += sum dZ2
//   dZ1 = (dZ2 W2^T) * [Z1 > 0],   dW1|b1 += X^T dZ1
//   de  = dZ1 W1[0:12]^T  -> scattered to the feature grid with the trilinear weights.
// Weight gradients accumulate in registers across tiles and are added to global memory once
// per CTA.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr int TM = 64;            // samples per tile
constexpr int NT = 256;           // threads per CTA
constexpr int HID = 128;
constexpr int FEAT = 12;
constexpr int NF = 4;
constexpr int NFX = 5;
constexpr int LDA = TM + 4;             // 68: activation row stride
constexpr int LDW = HID + 4;            // 132: weight row stride
constexpr int PX = FEAT + 3 + 6 * NF;   // 39: first input of the PE(x) block

// Input widths: 39 (features + PE(d)) or 72 (+ PE(x)); K1 adds the bias column; the backward
// splits the K1 (padded to 2 KH) rows of dW1|b1 between two thread halves.
template <bool PEX>
struct Dims {
    static constexpr int IN = PX + (PEX ? 3 + 6 * NFX : 0);
    static constexpr int K1 = IN + 1;
    static constexpr int KH = (K1 + 1) / 2;
};

template <bool PEX>
struct Smem {
    static constexpr int K1 = Dims<PEX>::K1, KP = 2 * Dims<PEX>::KH;
    float w1[K1 * LDW];
    float w2[HID * LDW];
    float b2[HID];
    float w3[HID * 3];
    float b3[4];
    float xt[KP * LDA];        // X^T (a zero padding row when K1 is odd)
    float h1[HID * LDA];       // H1^T, later dZ1^T
    float h2[HID * LDA];       // H2^T, later dZ2^T
    float dout[TM * 3];        // dL/do (pre-sigmoid) per sample
    float de[TM * FEAT];       // dL/dfeat per sample
    int cbase[TM];             // base corner flat index
    float frac[TM * 3];        // fractional offsets
    int slot[TM];              // sample slot, -1 for padding rows
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// Load weights into shared memory (FP32 master weights, row-major [in][out]).
template <bool PEX>
__device__ void load_weights(Smem<PEX> &S, const RenderArgs &A) {
    constexpr int IN = Dims<PEX>::IN, K1 = Dims<PEX>::K1;
    for (int i = threadIdx.x; i < (Smem<PEX>::KP - K1) * LDA; i += NT) S.xt[K1 * LDA + i] = 0.0f;
    for (int i = threadIdx.x; i < K1 * HID; i += NT) {
        int k = i / HID, j = i % HID;
        S.w1[k * LDW + j] = (k < IN) ? A.w1[k * HID + j] : A.b1[j];
    }
    for (int i = threadIdx.x; i < HID * HID; i += NT) S.w2[(i / HID) * LDW + (i % HID)] = A.w2[i];
    for (int i = threadIdx.x; i < HID; i += NT) S.b2[i] = A.b2[i];
    for (int i = threadIdx.x; i < HID * 3; i += NT) S.w3[i] = A.w3[i];
    if (threadIdx.x < 3) S.b3[threadIdx.x] = A.b3[threadIdx.x];
}

// Gather the input rows of one tile: 4 threads per sample, thread q handles the corner pair
// (x bit, y bit) = (q >> 1, q & 1) with z = 0, 1 (adjacent in memory).
template <typename FeatT, bool PEX, bool PK>
__device__ void gather_tile(Smem<PEX> &S, const RenderArgs &A, int tile, int n_kept) {
    constexpr int IN = Dims<PEX>::IN;
    int tid = threadIdx.x;
    int i = tid >> 2, q = tid & 3;
    int e = tile * TM + i;
    bool valid = e < n_kept;
    float f[FEAT];
#pragma unroll
    for (int c = 0; c < FEAT; ++c) f[c] = 0.0f;
    const RayRec *rp = nullptr;
    int ray = 0, slot = -1;
    float xw = 0.0f;   // world coordinate of axis q - 1 (PE(x), threads q = 1..3)
    if (valid) {
        int2 kv = A.kept[e];
        slot = kv.x;
        ray = kv.y;
        rp = A.rays + ray;
        const RayRec &rr = *rp;
        int k = slot - rr.off;
        float dt;
        Cell c = sample_cell(A, rr, ray, k, dt);
        if (PEX && q > 0) {
            float xv[3];
            cell_world(A, c, xv);
            xw = xv[q - 1];
        }
        if (q == 0) {
            S.cbase[i] = cell_base(c, A.ny, A.nz, PK);
            S.frac[3 * i] = c.fx;
            S.frac[3 * i + 1] = c.fy;
            S.frac[3 * i + 2] = c.fz;
            S.slot[i] = slot;
        }
        int qa = q << 1;   // corner bits (x, y, 0)
        long long idx0 = corner_index(c, qa, A.ny, A.nz, PK);
        float w0 = corner_weight(c, qa), w1 = corner_weight(c, qa | 1);
        const FeatT *g = static_cast<const FeatT *>(A.cgrid) + idx0 * FEAT;
        // the z + 1 corner: the next point in the canonical layout, located in the packed one
        const FeatT *gz = PK ? static_cast<const FeatT *>(A.cgrid) + corner_index(c, qa | 1, A.ny, A.nz, true) * FEAT
                                   : g + FEAT;
        if constexpr (sizeof(FeatT) == 4) {
            const float4 *g4 = reinterpret_cast<const float4 *>(g), *gz4 = reinterpret_cast<const float4 *>(gz);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                float4 a = __ldg(g4 + v), b = __ldg(gz4 + v);
                f[4 * v + 0] = fmaf(w0, a.x, w1 * b.x);
                f[4 * v + 1] = fmaf(w0, a.y, w1 * b.y);
                f[4 * v + 2] = fmaf(w0, a.z, w1 * b.z);
                f[4 * v + 3] = fmaf(w0, a.w, w1 * b.w);
            }
        } else {
            // BF16 storage: 24 bytes per corner, 8-byte aligned; 48 contiguous bytes for the pair.
            const uint2 *g2 = reinterpret_cast<const uint2 *>(g), *gz2 = reinterpret_cast<const uint2 *>(gz);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                uint2 a = __ldg(g2 + v), b = __ldg(gz2 + v);
                __nv_bfloat162 a0 = *reinterpret_cast<__nv_bfloat162 *>(&a.x), a1 = *reinterpret_cast<__nv_bfloat162 *>(&a.y);
                __nv_bfloat162 b0 = *reinterpret_cast<__nv_bfloat162 *>(&b.x), b1 = *reinterpret_cast<__nv_bfloat162 *>(&b.y);
                float2 fa0 = __bfloat1622float2(a0), fa1 = __bfloat1622float2(a1);
                float2 fb0 = __bfloat1622float2(b0), fb1 = __bfloat1622float2(b1);
                f[4 * v + 0] = fmaf(w0, fa0.x, w1 * fb0.x);
                f[4 * v + 1] = fmaf(w0, fa0.y, w1 * fb0.y);
                f[4 * v + 2] = fmaf(w0, fa1.x, w1 * fb1.x);
                f[4 * v + 3] = fmaf(w0, fa1.y, w1 * fb1.y);
            }
        }
    } else if (q == 0) {
        S.slot[i] = -1;
        S.cbase[i] = 0;
        S.frac[3 * i] = S.frac[3 * i + 1] = S.frac[3 * i + 2] = 0.0f;
    }
    // reduce the 4 corner pairs of a sample (lanes 4i..4i+3)
#pragma unroll
    for (int c = 0; c < FEAT; ++c) {
        f[c] += __shfl_xor_sync(0xffffffffu, f[c], 1);
        f[c] += __shfl_xor_sync(0xffffffffu, f[c], 2);
    }
    // q = 0 writes the features; q = 1..3 write the direction encoding of one axis each
    if (q == 0) {
#pragma unroll
        for (int c = 0; c < FEAT; ++c) S.xt[c * LDA + i] = f[c];
        S.xt[IN * LDA + i] = 1.0f;
    } else {
        int a = q - 1;
        float d = valid ? rp->dir[a] : 0.0f;
        S.xt[(FEAT + a) * LDA + i] = d;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            float s, cs;
            sincosf(ldexpf(d, k), &s, &cs);
            S.xt[(FEAT + 3 + a * NF + k) * LDA + i] = s;
            S.xt[(FEAT + 3 + 3 * NF + a * NF + k) * LDA + i] = cs;
        }
        if constexpr (PEX) {
            float sx[NFX], cx[NFX];
            pe_axis<NFX>(xw, sx, cx);
            S.xt[(PX + a) * LDA + i] = xw;
#pragma unroll
            for (int k = 0; k < NFX; ++k) {
                S.xt[(PX + 3 + a * NFX + k) * LDA + i] = sx[k];
                S.xt[(PX + 3 + 3 * NFX + a * NFX + k) * LDA + i] = cx[k];
            }
        }
    }
}

// OutT[j][s] = act(sum_k InT[k][s] W[k][j] + bias[j]) for a 64 x 128 tile.  Thread (tx, ty):
// samples 4ty..4ty+3, columns 4tx..4tx+3 and 64+4tx..64+4tx+3.
template <int K>
__device__ __forceinline__ void gemm_fwd(const float *InT, const float *W, const float *bias, float *OutT) {
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int s0 = ty * 4, c0 = tx * 4, c1 = 64 + tx * 4;
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float b = bias ? bias[j < 4 ? c0 + j : c1 + j - 4] : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = b;
    }
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        float4 a = ld4(InT + k * LDA + s0);
        float4 b0 = ld4(W + k * LDW + c0), b1 = ld4(W + k * LDW + c1);
        float av[4] = {a.x, a.y, a.z, a.w};
        float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int col = j < 4 ? c0 + j : c1 + j - 4;
        st4(OutT + col * LDA + s0, make_float4(fmaxf(acc[0][j], 0.0f), fmaxf(acc[1][j], 0.0f),
                                               fmaxf(acc[2][j], 0.0f), fmaxf(acc[3][j], 0.0f)));
    }
}

// Output layer for sample s = tid & 63, channel ch = tid >> 6 (< 3): o = h2 . W3[:, ch] + b3.
template <bool PEX>
__device__ __forceinline__ float out_logit(const Smem<PEX> &S, int s, int ch) {
    float o = S.b3[ch];
#pragma unroll 8
    for (int j = 0; j < HID; ++j) o = fmaf(S.h2[j * LDA + s], S.w3[j * 3 + ch], o);
    return o;
}

template <typename FeatT, bool PEX, bool PK>
__global__ void __launch_bounds__(NT, 1) fine_colour_fwd_kernel(RenderArgs A) {
    constexpr int K1 = Dims<PEX>::K1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<PEX> &S = *reinterpret_cast<Smem<PEX> *>(smem_raw);
    load_weights(S, A);
    const int n_kept = A.hdr->n_kept;
    const int ntiles = (n_kept + TM - 1) / TM;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        gather_tile<FeatT, PEX, PK>(S, A, tile, n_kept);
        __syncthreads();
        gemm_fwd<K1>(S.xt, S.w1, nullptr, S.h1);
        __syncthreads();
        gemm_fwd<HID>(S.h1, S.w2, S.b2, S.h2);
        __syncthreads();
        int s = threadIdx.x & 63, ch = threadIdx.x >> 6;
        if (ch < 3 && S.slot[s] >= 0) {
            float c = sigmoidf_(out_logit(S, s, ch));
            reinterpret_cast<float *>(A.samp + S.slot[s])[1 + ch] = c;
        }
    }
}

template <typename FeatT, bool PEX, bool PK>
__global__ void __launch_bounds__(NT, 1) fine_colour_bwd_kernel(RenderArgs A) {
    constexpr int IN = Dims<PEX>::IN, K1 = Dims<PEX>::K1, KH = Dims<PEX>::KH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<PEX> &S = *reinterpret_cast<Smem<PEX> *>(smem_raw);
    load_weights(S, A);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int n_kept = A.hdr->n_kept;
    const int ntiles = (n_kept + TM - 1) / TM;

    float gw2[8][8];       // dW2[tx + 16 i][ty + 16 jj]
    float gw1[KH];         // dW1|b1[kh*KH + kk][j], j = tid & 127, kh = tid >> 7
    float gw3[3];          // dW3[tid][ch] (tid < 128)
    float gb2 = 0.0f;      // db2[tid - 128] (tid >= 128)
    float gb3 = 0.0f;      // db3[tid] (tid < 3)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) gw2[i][j] = 0.0f;
#pragma unroll
    for (int i = 0; i < KH; ++i) gw1[i] = 0.0f;
    gw3[0] = gw3[1] = gw3[2] = 0.0f;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        gather_tile<FeatT, PEX, PK>(S, A, tile, n_kept);
        __syncthreads();
        gemm_fwd<K1>(S.xt, S.w1, nullptr, S.h1);
        __syncthreads();
        gemm_fwd<HID>(S.h1, S.w2, S.b2, S.h2);
        __syncthreads();
        // output layer + sigmoid backward
        {
            int s = tid & 63, ch = tid >> 6;
            if (ch < 3) {
                float d = 0.0f;
                if (S.slot[s] >= 0) {
                    float c = sigmoidf_(out_logit(S, s, ch));
                    float dc = reinterpret_cast<const float *>(A.sgrad + S.slot[s])[1 + ch];
                    d = dc * c * (1.0f - c);
                }
                S.dout[s * 3 + ch] = d;
            }
        }
        __syncthreads();
        // dW3, db3 (need H2 before it is overwritten)
        if (tid < HID) {
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
            for (int s = 0; s < TM; s += 4) {
                float4 h = ld4(S.h2 + tid * LDA + s);
                float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a0 = fmaf(hv[u], S.dout[(s + u) * 3 + 0], a0);
                    a1 = fmaf(hv[u], S.dout[(s + u) * 3 + 1], a1);
                    a2 = fmaf(hv[u], S.dout[(s + u) * 3 + 2], a2);
                }
            }
            gw3[0] += a0;
            gw3[1] += a1;
            gw3[2] += a2;
        }
        if (tid < 3) {
            float a = 0.0f;
            for (int s = 0; s < TM; ++s) a += S.dout[s * 3 + tid];
            gb3 += a;
        }
        __syncthreads();
        // dZ2 = (dout W3^T) * [H2 > 0], in place over H2^T (same thread mapping as gemm_fwd)
        {
            int s0 = ty * 4, c0 = tx * 4, c1 = 64 + tx * 4;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int col = j < 4 ? c0 + j : c1 + j - 4;
                float w30 = S.w3[col * 3], w31 = S.w3[col * 3 + 1], w32 = S.w3[col * 3 + 2];
                float4 h = ld4(S.h2 + col * LDA + s0);
                float hv[4] = {h.x, h.y, h.z, h.w}, out[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float *dd = S.dout + (s0 + i) * 3;
                    float v = dd[0] * w30 + dd[1] * w31 + dd[2] * w32;
                    out[i] = hv[i] > 0.0f ? v : 0.0f;
                }
                st4(S.h2 + col * LDA + s0, make_float4(out[0], out[1], out[2], out[3]));
            }
        }
        __syncthreads();
        // dW2 += H1^T dZ2 ; db2 += sum_s dZ2
        for (int s = 0; s < TM; s += 4) {
            float4 a[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = ld4(S.h1 + (tx + 16 * i) * LDA + s);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                float4 b = ld4(S.h2 + (ty + 16 * jj) * LDA + s);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    gw2[i][jj] = fmaf(a[i].x, b.x, fmaf(a[i].y, b.y, fmaf(a[i].z, b.z, fmaf(a[i].w, b.w, gw2[i][jj]))));
            }
        }
        if (tid >= HID) {
            float a = 0.0f;
            int j = tid - HID;
            for (int s = 0; s < TM; s += 4) {
                float4 v = ld4(S.h2 + j * LDA + s);
                a += (v.x + v.y) + (v.z + v.w);
            }
            gb2 += a;
        }
        // dH1 = dZ2 W2^T (thread: samples 4ty..4ty+3, hidden k = tx + 16 i); keep in registers
        float dh[4][8];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int i = 0; i < 8; ++i) dh[s][i] = 0.0f;
        {
            int s0 = ty * 4;
            for (int j = 0; j < HID; j += 4) {
                float4 a[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) a[jj] = ld4(S.h2 + (j + jj) * LDA + s0);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float4 b = ld4(S.w2 + (tx + 16 * i) * LDW + j);
                    dh[0][i] = fmaf(a[0].x, b.x, fmaf(a[1].x, b.y, fmaf(a[2].x, b.z, fmaf(a[3].x, b.w, dh[0][i]))));
                    dh[1][i] = fmaf(a[0].y, b.x, fmaf(a[1].y, b.y, fmaf(a[2].y, b.z, fmaf(a[3].y, b.w, dh[1][i]))));
                    dh[2][i] = fmaf(a[0].z, b.x, fmaf(a[1].z, b.y, fmaf(a[2].z, b.z, fmaf(a[3].z, b.w, dh[2][i]))));
                    dh[3][i] = fmaf(a[0].w, b.x, fmaf(a[1].w, b.y, fmaf(a[2].w, b.z, fmaf(a[3].w, b.w, dh[3][i]))));
                }
            }
        }
        __syncthreads();   // every thread is done reading H1 (dW2) and dZ2
        // dZ1 = dH1 * [H1 > 0], in place over H1^T
        {
            int s0 = ty * 4;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int k = tx + 16 * i;
                float4 h = ld4(S.h1 + k * LDA + s0);
                st4(S.h1 + k * LDA + s0, make_float4(h.x > 0.0f ? dh[0][i] : 0.0f, h.y > 0.0f ? dh[1][i] : 0.0f,
                                                     h.z > 0.0f ? dh[2][i] : 0.0f, h.w > 0.0f ? dh[3][i] : 0.0f));
            }
        }
        __syncthreads();
        // dW1|b1 += X^T dZ1 : thread j = tid & 127, rows kh*KH .. kh*KH+KH-1
        {
            int j = tid & 127, kh = tid >> 7;
            for (int s = 0; s < TM; s += 4) {
                float4 b = ld4(S.h1 + j * LDA + s);
#pragma unroll
                for (int kk = 0; kk < KH; ++kk) {
                    float4 a = ld4(S.xt + (kh * KH + kk) * LDA + s);
                    gw1[kk] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, gw1[kk]))));
                }
            }
        }
        // de = dZ1 W1[0:12]^T : sample s = tid & 63, channels 3 cg .. 3 cg + 2
        {
            int s = tid & 63, cg = tid >> 6;
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
            const float *wa = S.w1 + (3 * cg) * LDW, *wb = wa + LDW, *wc = wb + LDW;
#pragma unroll 8
            for (int j = 0; j < HID; ++j) {
                float dz = S.h1[j * LDA + s];
                e0 = fmaf(dz, wa[j], e0);
                e1 = fmaf(dz, wb[j], e1);
                e2 = fmaf(dz, wc[j], e2);
            }
            S.de[s * FEAT + 3 * cg] = e0;
            S.de[s * FEAT + 3 * cg + 1] = e1;
            S.de[s * FEAT + 3 * cg + 2] = e2;
        }
        __syncthreads();
        // scatter de to the feature grid: 4 threads per sample, corner pair (q>>1, q&1, z=0/1)
        {
            int i = tid >> 2, q = tid & 3;
            if (S.slot[i] >= 0) {
                float fx = S.frac[3 * i], fy = S.frac[3 * i + 1], fz = S.frac[3 * i + 2];
                float wxy = ((q >> 1) ? fx : 1.0f - fx) * ((q & 1) ? fy : 1.0f - fy);
                float w0 = wxy * (1.0f - fz), w1 = wxy * fz;
                const long long idx0 = corner_from_base(S.cbase[i], q >> 1, q & 1, 0, A.ny, A.nz, PK);
                const long long idx1 = corner_from_base(S.cbase[i], q >> 1, q & 1, 1, A.ny, A.nz, PK);
                float4 *g0 = reinterpret_cast<float4 *>(A.grad_cgrid + idx0 * FEAT);
                float4 *g1 = reinterpret_cast<float4 *>(A.grad_cgrid + idx1 * FEAT);
                const float *d = S.de + i * FEAT;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    float4 dv = make_float4(d[4 * v], d[4 * v + 1], d[4 * v + 2], d[4 * v + 3]);
                    atomicAdd(g0 + v, make_float4(w0 * dv.x, w0 * dv.y, w0 * dv.z, w0 * dv.w));
                    atomicAdd(g1 + v, make_float4(w1 * dv.x, w1 * dv.y, w1 * dv.z, w1 * dv.w));
                }
            }
        }
    }
    // flush the per-CTA weight gradients: grad_mlp = w1 | b1 | w2 | b2 | w3 | b3
    float *gW1 = A.grad_mlp, *gB1 = gW1 + IN * HID, *gW2 = gB1 + HID, *gB2 = gW2 + HID * HID;
    float *gW3 = gB2 + HID, *gB3 = gW3 + HID * 3;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) atomicAdd(gW2 + (tx + 16 * i) * HID + (ty + 16 * jj), gw2[i][jj]);
    {
        int j = tid & 127, kh = tid >> 7;
#pragma unroll
        for (int kk = 0; kk < KH; ++kk) {
            int k = kh * KH + kk;
            if (k < IN) atomicAdd(gW1 + k * HID + j, gw1[kk]);
            else if (k == IN) atomicAdd(gB1 + j, gw1[kk]);
        }
    }
    if (tid < HID) {
        atomicAdd(gW3 + tid * 3 + 0, gw3[0]);
        atomicAdd(gW3 + tid * 3 + 1, gw3[1]);
        atomicAdd(gW3 + tid * 3 + 2, gw3[2]);
    } else {
        atomicAdd(gB2 + (tid - HID), gb2);
    }
    if (tid < 3) atomicAdd(gB3 + tid, gb3);
}

template <bool PEX>
void launch_persistent(void (*kernel)(RenderArgs), int kind, const RenderArgs &A, cudaStream_t s) {
    ensure_smem(reinterpret_cast<const void *>(kernel), (int)sizeof(Smem<PEX>));
    ProfScope ps_(kind, s);
    kernel<<<num_sms(), NT, sizeof(Smem<PEX>), s>>>(A);
}

template <bool BWD, bool PEX, bool PK>
void launch_colour(const RenderArgs &A, cudaStream_t s) {
    const int kind = BWD ? DVGO_K_FINE_COLOUR_BWD : DVGO_K_FINE_COLOUR_FWD;
    if (A.cdtype == DVGO_DTYPE_BF16)
        launch_persistent<PEX>(BWD ? fine_colour_bwd_kernel<__nv_bfloat16, PEX, PK>
                                   : fine_colour_fwd_kernel<__nv_bfloat16, PEX, PK>,
                               kind, A, s);
    else
        launch_persistent<PEX>(BWD ? fine_colour_bwd_kernel<float, PEX, PK> : fine_colour_fwd_kernel<float, PEX, PK>,
                               kind, A, s);
}

template <bool BWD>
void launch_colour_any(const RenderArgs &A, cudaStream_t s) {
    const bool pex = A.nfreq_pos > 0;
    if (A.packed) {
        if (pex) launch_colour<BWD, true, true>(A, s);
        else launch_colour<BWD, false, true>(A, s);
    } else {
        if (pex) launch_colour<BWD, true, false>(A, s);
        else launch_colour<BWD, false, false>(A, s);
    }
}

}  // namespace

void launch_fine_colour_fwd_simt(const RenderArgs &A, cudaStream_t s) { launch_colour_any<false>(A, s); }

void launch_fine_colour_bwd_simt(const RenderArgs &A, cudaStream_t s) { launch_colour_any<true>(A, s); }

}  // namespace dvgo
