// proposal.cu -- learned sample proposal: per-ray weight histograms (labels), the proposal MLP
// forward / backward (softmax cross-entropy), and inverse-CDF sampling of explicit samples.
//
// The paper renders with uniform steps and leaves hierarchical sampling to future work (Supp. B,
// step-size ablation); this proposal is the library's addition.  Definitions:
//   bins:     n_bins equal bins of the clipped interval [t_enter, t_exit] of each ray;
//   labels:   h_b = sum of the compositing weights w_k = T_k alpha_k of the samples whose t_k
//             falls in bin b, divided by sum_k w_k (uniform when that sum is below 1e-4), from a
//             uniform-step fine forward (Eq. volume_rendering);
//   network:  the bin centre x_b = o + t_b d is encoded as [x, sin(2^k x_c), cos(2^k x_c)]
//             (k < 6, c-major), then 39 -> 64 -> 64 -> 64 -> 1 with ReLU gives a logit per bin and
//             p = softmax over the bins; loss = -(1/R) sum_r sum_b h_rb log p_rb (rays that miss
//             the box contribute nothing);
//   sampling: q_b = (1 - eta) p_b + eta / n_bins, Q its CDF; sample j at u_j = (j + jit) / n * Q_nb
//             lies in the bin with Q_b <= u_j < Q_{b+1}, at t = t0 + (b + (u_j - Q_b) / q_b) w;
//             dt_j = t_{j+1} - t_j and, for the last sample, w Q_nb / (n q_b).
// The bin of a quantile (labels) is decided in FP64 with separately rounded operations, in the
// order written above.  Sampling runs in double-float arithmetic (below): its CDF, quantiles and
// sample positions carry ~48 significant bits, so a sample's bin can differ from the exact one
// only where its quantile lies within ~1e-14 of a bin edge -- where t is continuous across the
// edge -- and t, dt come out as the FP32 roundings of the exact values to within an ulp.

#include <math.h>

#include "df64.cuh"
#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr int NB = 64;             // bins
constexpr int NFQ = 6;             // PE frequencies on the bin centre
constexpr int PIN = 3 + 6 * NFQ;   // 39
constexpr int PK0 = PIN + 1;       // 40 with the bias column
constexpr int PW = 64;             // width
constexpr int PTM = 128;           // rows per tile = 2 rays x 64 bins
constexpr int PNT = 256;
constexpr int PLD = PTM + 4;       // activation row stride (feature-major storage)

struct BoxD {
    double mn[3], mx[3];
    double t_near, t_far;
};

BoxD make_box(const dvgo_params &p, const dvgo_grid_desc &g) {
    BoxD b;
    for (int a = 0; a < 3; ++a) {
        b.mn[a] = g.xyz_min[a];
        b.mx[a] = g.xyz_max[a];
    }
    b.t_near = p.t_near;
    b.t_far = p.t_far;
    return b;
}

__device__ __forceinline__ Clip clip_ray(const BoxD &B, const float *ro, const float *rd, int r) {
    const double o[3] = {(double)ro[3 * r], (double)ro[3 * r + 1], (double)ro[3 * r + 2]};
    const double d[3] = {(double)rd[3 * r], (double)rd[3 * r + 1], (double)rd[3 * r + 2]};
    return slab_clip(o, d, B.mn, B.mx, B.t_near, B.t_far);
}

// ---------------------------------------------------------------------------------------------
// Labels: per-ray histogram of compositing weights over n_bins bins (warp per ray)
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) weight_bins_kernel(RenderArgs A, int nbins, float *labels) {
    __shared__ float bins[8][128];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < A.R; r += nwarps) {
        const RayRec rr = A.rays[r];
        const double t0 = rr.t_enter, t1 = A.texit[r];
        // bin of sample k: floor((t_k - t_enter) / (t_exit - t_enter) nbins), t_k - t_enter = (k + p) step
        const double bin_scale = __ddiv_rn(__dmul_rn((double)A.step, (double)nbins), __dsub_rn(t1, t0));
        for (int b = lane; b < nbins; b += 32) bins[wib][b] = 0.0f;
        __syncwarp();
        float carry = 0.0f, wsum = 0.0f;
        for (int base = 0; base < rr.n; base += 32) {
            const int k = base + lane;
            const float tau = k < rr.n ? A.samp[rr.off + k].x : 0.0f;
            const float incl = warp_incl_scan(tau, lane);
            float excl = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane == 0) excl = 0.0f;
            const float w = expf(-(carry + excl)) * -expm1f(-tau);
            if (k < rr.n) {
                int b = (int)floor(__dmul_rn(__dadd_rn((double)k, (double)rr.p), bin_scale));
                b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
                atomicAdd(&bins[wib][b], w);
            }
            wsum += warp_sum(w);
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        const bool uniform = wsum < 1e-4f;
        for (int b = lane; b < nbins; b += 32)
            labels[(size_t)r * nbins + b] = uniform ? 1.0f / nbins : bins[wib][b] / wsum;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// Proposal MLP (FP32 SIMT), tiles of 2 rays x 64 bins
// ---------------------------------------------------------------------------------------------

struct PropArgs {
    int R;
    BoxD box;
    const float *ro, *rd, *labels;
    const float *w0, *b0, *w1, *b1, *w2, *b2, *w3, *b3;
    float *probs, *loss, *grad;
};

struct PropSmem {
    float w0[PK0 * PW];     // rows 0..38 = W0, row 39 = b0
    float w1[PW * PW], w2[PW * PW];
    float w1t[PW * PW], w2t[PW * PW];   // transposed copies for the backward
    float b1[PW], b2[PW], w3[PW];
    float b3[4];              // [0] used; 4 floats keep the following arrays 16-byte aligned
    float xt[PK0 * PLD];    // inputs, feature-major
    float h0[PW * PLD], h1[PW * PLD], h2[PW * PLD];
    float logit[PTM], dlog[PTM];
    double t0[2], t1[2], dn[2][3];
    int hit[2];
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// OutT[n][row] = act(sum_k InT[k][row] W[k][n] + bias[n]) for 128 rows x 64 outputs.
// Thread: rows 4 (t >> 3) .. +3, outputs 8 (t & 7) .. +7.
template <int K>
__device__ __forceinline__ void ptile_gemm(const float *InT, const float *W, const float *bias, float *OutT) {
    const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
    const int r0 = 4 * ty, c0 = 8 * tx;
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b = bias ? bias[c0 + j] : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = b;
    }
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = ld4(InT + k * PLD + r0);
        const float4 x0 = ld4(W + k * PW + c0), x1 = ld4(W + k * PW + c0 + 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
        st4(OutT + (c0 + j) * PLD + r0, make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]));
}

__device__ __forceinline__ void relu_inplace(float *T, int nfeat) {
    for (int i = threadIdx.x; i < nfeat * PTM; i += PNT) {
        const int f = i / PTM, r = i % PTM;
        T[f * PLD + r] = fmaxf(T[f * PLD + r], 0.0f);
    }
}

// sin / cos of an FP64 argument: reduce by 2 pi in FP64, evaluate in FP32.
__device__ __forceinline__ void sincos_reduced(double a, float *s, float *c) {
    const double two_pi = 6.283185307179586;
    const double n = rint(a / two_pi);
    const double red = fma(-n, two_pi, a);
    sincosf((float)red, s, c);
}

template <bool BWD>
__global__ void __launch_bounds__(PNT, 1) proposal_kernel(PropArgs P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PropSmem &S = *reinterpret_cast<PropSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < PK0 * PW; i += PNT) {
        const int k = i / PW, j = i % PW;
        S.w0[i] = k < PIN ? P.w0[k * PW + j] : P.b0[j];
    }
    for (int i = tid; i < PW * PW; i += PNT) {
        const int k = i / PW, j = i % PW;
        S.w1[i] = P.w1[i];
        S.w2[i] = P.w2[i];
        S.w1t[j * PW + k] = P.w1[i];
        S.w2t[j * PW + k] = P.w2[i];
    }
    if (tid < PW) {
        S.b1[tid] = P.b1[tid];
        S.b2[tid] = P.b2[tid];
        S.w3[tid] = P.w3[tid];
    }
    if (tid == 0) S.b3[0] = P.b3[0];
    // weight-gradient accumulators (backward)
    float g1[2][8], g2[2][8], g0[10], g3 = 0.0f, gb1 = 0.0f, gb2 = 0.0f, gb3 = 0.0f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) g1[i][j] = g2[i][j] = 0.0f;
#pragma unroll
    for (int i = 0; i < 10; ++i) g0[i] = 0.0f;
    const float invR = 1.0f / (float)P.R;

    const int ntiles = (P.R + 1) / 2;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (tid < 2) {
            const int r = 2 * tile + tid;
            int hit = 0;
            if (r < P.R) {
                const Clip c = clip_ray(P.box, P.ro, P.rd, r);
                hit = c.hi > c.lo;
                S.t0[tid] = c.lo;
                S.t1[tid] = c.hi;
                for (int a = 0; a < 3; ++a) S.dn[tid][a] = c.dn[a];
            }
            S.hit[tid] = hit;
        }
        __syncthreads();
        // encode the bin centres: 2 threads per row
        {
            const int row = tid >> 1, part = tid & 1, rl = row >> 6, bin = row & 63, r = 2 * tile + rl;
            double x[3] = {0.0, 0.0, 0.0};
            if (S.hit[rl]) {
                const double t0 = S.t0[rl], t1 = S.t1[rl];
                const double tb = __dadd_rn(t0, __ddiv_rn(__dmul_rn((double)bin + 0.5, __dsub_rn(t1, t0)), (double)NB));
                for (int a = 0; a < 3; ++a)
                    x[a] = __dadd_rn((double)P.ro[3 * r + a], __dmul_rn(tb, S.dn[rl][a]));
            }
            if (part == 0) {
                for (int a = 0; a < 3; ++a) S.xt[a * PLD + row] = (float)x[a];
                S.xt[PIN * PLD + row] = 1.0f;
            }
            // part 0: k = 0..2, part 1: k = 3..5 for every axis
            for (int a = 0; a < 3; ++a)
                for (int kk = 0; kk < 3; ++kk) {
                    const int k = 3 * part + kk;
                    float sv, cv;
                    sincos_reduced(ldexp(x[a], k), &sv, &cv);
                    S.xt[(3 + a * NFQ + k) * PLD + row] = sv;
                    S.xt[(3 + 3 * NFQ + a * NFQ + k) * PLD + row] = cv;
                }
        }
        __syncthreads();
        ptile_gemm<PK0>(S.xt, S.w0, nullptr, S.h0);
        __syncthreads();
        relu_inplace(S.h0, PW);
        __syncthreads();
        ptile_gemm<PW>(S.h0, S.w1, S.b1, S.h1);
        __syncthreads();
        relu_inplace(S.h1, PW);
        __syncthreads();
        ptile_gemm<PW>(S.h1, S.w2, S.b2, S.h2);
        __syncthreads();
        relu_inplace(S.h2, PW);
        __syncthreads();
        if (tid < PTM) {
            float o = S.b3[0];
#pragma unroll 8
            for (int j = 0; j < PW; ++j) o = fmaf(S.h2[j * PLD + tid], S.w3[j], o);
            S.logit[tid] = o;
        }
        __syncthreads();
        // softmax per ray (warp 0: ray 0, warp 1: ray 1), loss, dlogit
        if (tid < 64) {
            const int rl = tid >> 5, lane = tid & 31, r = 2 * tile + rl;
            if (r < P.R) {
                const float l0 = S.logit[64 * rl + lane], l1 = S.logit[64 * rl + lane + 32];
                float m = fmaxf(l0, l1);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                const float e0 = expf(l0 - m), e1 = expf(l1 - m);
                const float z = warp_sum(e0 + e1);
                float p0 = e0 / z, p1 = e1 / z;
                const bool hit = S.hit[rl] != 0;
                if (!hit) p0 = p1 = 1.0f / NB;
                if (!BWD && P.probs) {
                    P.probs[(size_t)r * NB + lane] = p0;
                    P.probs[(size_t)r * NB + lane + 32] = p1;
                }
                float d0 = 0.0f, d1 = 0.0f;
                if (P.labels && hit) {
                    const float h0 = P.labels[(size_t)r * NB + lane], h1 = P.labels[(size_t)r * NB + lane + 32];
                    if (!BWD && P.loss) {
                        float lr = 0.0f;
                        if (h0 > 0.0f) lr -= h0 * logf(p0);
                        if (h1 > 0.0f) lr -= h1 * logf(p1);
                        lr = warp_sum(lr);
                        if (lane == 0) atomicAdd(P.loss, lr * invR);
                    }
                    d0 = (p0 - h0) * invR;
                    d1 = (p1 - h1) * invR;
                }
                S.dlog[64 * rl + lane] = d0;
                S.dlog[64 * rl + lane + 32] = d1;
            } else {
                S.dlog[64 * rl + lane] = 0.0f;
                S.dlog[64 * rl + lane + 32] = 0.0f;
            }
        }
        if (!BWD) continue;
        __syncthreads();
        // output layer: dW3, db3; dH2 = dlogit w3^T [H2 > 0] (in place over h2 is not possible: H2
        // is needed for dW3 first)
        if (tid < PW) {
            float a = 0.0f;
            for (int r = 0; r < PTM; r += 4) {
                const float4 h = ld4(S.h2 + tid * PLD + r);
                a = fmaf(h.x, S.dlog[r], fmaf(h.y, S.dlog[r + 1], fmaf(h.z, S.dlog[r + 2], fmaf(h.w, S.dlog[r + 3], a))));
            }
            g3 += a;
        }
        if (tid == PW) {
            float a = 0.0f;
            for (int r = 0; r < PTM; ++r) a += S.dlog[r];
            gb3 += a;
        }
        __syncthreads();
        for (int i = tid; i < PW * PTM; i += PNT) {
            const int f = i / PTM, r = i % PTM;
            const float h = S.h2[f * PLD + r];
            S.h2[f * PLD + r] = h > 0.0f ? S.dlog[r] * S.w3[f] : 0.0f;   // dZ2
        }
        __syncthreads();
        // dW2 += H1^T dZ2, db2 += sum dZ2 ; thread: inputs 2 kq, 2 kq + 1, outputs 8 nq .. +7
        {
            const int kq = tid >> 3, nq = tid & 7;
            for (int r = 0; r < PTM; r += 4) {
                const float4 a0 = ld4(S.h1 + (2 * kq) * PLD + r), a1 = ld4(S.h1 + (2 * kq + 1) * PLD + r);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 d = ld4(S.h2 + (8 * nq + j) * PLD + r);
                    g2[0][j] = fmaf(a0.x, d.x, fmaf(a0.y, d.y, fmaf(a0.z, d.z, fmaf(a0.w, d.w, g2[0][j]))));
                    g2[1][j] = fmaf(a1.x, d.x, fmaf(a1.y, d.y, fmaf(a1.z, d.z, fmaf(a1.w, d.w, g2[1][j]))));
                }
            }
            if (tid < PW) {
                float a = 0.0f;
                for (int r = 0; r < PTM; r += 4) {
                    const float4 d = ld4(S.h2 + tid * PLD + r);
                    a += (d.x + d.y) + (d.z + d.w);
                }
                gb2 += a;
            }
        }
        // dH1 = dZ2 W2^T -> xt is free: use h0's partner buffers carefully: write dZ1 into S.xt? No:
        // xt is still needed for dW0.  dH1 goes to a register tile, then over h1 after a barrier.
        {
            const int ty = tid >> 3, tx = tid & 7, r0 = 4 * ty, c0 = 8 * tx;
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
            for (int k = 0; k < PW; ++k) {
                const float4 a = ld4(S.h2 + k * PLD + r0);
                const float4 x0 = ld4(S.w2t + k * PW + c0), x1 = ld4(S.w2t + k * PW + c0 + 4);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();   // all reads of h1 (dW2) and h2 done
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 h = ld4(S.h1 + (c0 + j) * PLD + r0);
                st4(S.h1 + (c0 + j) * PLD + r0,
                    make_float4(h.x > 0.0f ? acc[0][j] : 0.0f, h.y > 0.0f ? acc[1][j] : 0.0f,
                                h.z > 0.0f ? acc[2][j] : 0.0f, h.w > 0.0f ? acc[3][j] : 0.0f));
            }
        }
        __syncthreads();
        // dW1 += H0^T dZ1, db1 += sum dZ1
        {
            const int kq = tid >> 3, nq = tid & 7;
            for (int r = 0; r < PTM; r += 4) {
                const float4 a0 = ld4(S.h0 + (2 * kq) * PLD + r), a1 = ld4(S.h0 + (2 * kq + 1) * PLD + r);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 d = ld4(S.h1 + (8 * nq + j) * PLD + r);
                    g1[0][j] = fmaf(a0.x, d.x, fmaf(a0.y, d.y, fmaf(a0.z, d.z, fmaf(a0.w, d.w, g1[0][j]))));
                    g1[1][j] = fmaf(a1.x, d.x, fmaf(a1.y, d.y, fmaf(a1.z, d.z, fmaf(a1.w, d.w, g1[1][j]))));
                }
            }
            if (tid < PW) {
                float a = 0.0f;
                for (int r = 0; r < PTM; r += 4) {
                    const float4 d = ld4(S.h1 + tid * PLD + r);
                    a += (d.x + d.y) + (d.z + d.w);
                }
                gb1 += a;
            }
        }
        // dZ0 = (dZ1 W1^T) [H0 > 0], over h2 (free now)
        {
            const int ty = tid >> 3, tx = tid & 7, r0 = 4 * ty, c0 = 8 * tx;
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
            for (int k = 0; k < PW; ++k) {
                const float4 a = ld4(S.h1 + k * PLD + r0);
                const float4 x0 = ld4(S.w1t + k * PW + c0), x1 = ld4(S.w1t + k * PW + c0 + 4);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 h = ld4(S.h0 + (c0 + j) * PLD + r0);
                st4(S.h2 + (c0 + j) * PLD + r0,
                    make_float4(h.x > 0.0f ? acc[0][j] : 0.0f, h.y > 0.0f ? acc[1][j] : 0.0f,
                                h.z > 0.0f ? acc[2][j] : 0.0f, h.w > 0.0f ? acc[3][j] : 0.0f));
            }
        }
        __syncthreads();
        // [dW0 | db0] += X^T dZ0 : thread: output n = t & 63, inputs 10 (t >> 6) .. +9
        {
            const int n = tid & 63, kq = tid >> 6;
            for (int r = 0; r < PTM; r += 4) {
                const float4 d = ld4(S.h2 + n * PLD + r);
#pragma unroll
                for (int i = 0; i < 10; ++i) {
                    const float4 a = ld4(S.xt + (10 * kq + i) * PLD + r);
                    g0[i] = fmaf(a.x, d.x, fmaf(a.y, d.y, fmaf(a.z, d.z, fmaf(a.w, d.w, g0[i]))));
                }
            }
        }
    }
    if (!BWD) return;
    // flush: grad = w0 | b0 | w1 | b1 | w2 | b2 | w3 | b3
    float *G0 = P.grad, *GB0 = G0 + PIN * PW, *G1 = GB0 + PW, *GB1 = G1 + PW * PW, *G2 = GB1 + PW, *GB2 = G2 + PW * PW;
    float *G3 = GB2 + PW, *GB3 = G3 + PW;
    {
        const int kq = tid >> 3, nq = tid & 7;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                atomicAdd(G1 + (2 * kq + i) * PW + 8 * nq + j, g1[i][j]);
                atomicAdd(G2 + (2 * kq + i) * PW + 8 * nq + j, g2[i][j]);
            }
        const int n = tid & 63, k0 = 10 * (tid >> 6);
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            const int k = k0 + i;
            if (k < PIN) atomicAdd(G0 + k * PW + n, g0[i]);
            else if (k == PIN) atomicAdd(GB0 + n, g0[i]);
        }
    }
    if (tid < PW) {
        atomicAdd(G3 + tid, g3);
        atomicAdd(GB1 + tid, gb1);
        atomicAdd(GB2 + tid, gb2);
    }
    if (tid == PW) atomicAdd(GB3, gb3);
}

// ---------------------------------------------------------------------------------------------
// Inverse-CDF sampling.  FP64 runs at 1/64 of the FP32 rate on this GPU, so everything past the
// box clip is double-float arithmetic (df64.cuh).
// ---------------------------------------------------------------------------------------------

constexpr int kPdfThreads = 32;
constexpr int kPdfMaxBins = 128;

// Thread per ray, no shared memory (the kernel runs beside the HBM-bound Adam, whose loads in
// flight need the SM's L1): the CDF of the ray is summed twice in the same order, once for its
// total and once merged with the sorted quantiles, and the probability of the next bin is loaded
// a bin ahead so that the merge does not wait on memory.
__global__ void __launch_bounds__(kPdfThreads) sample_pdf_kernel(int R, BoxD B, const float *ro, const float *rd,
                                                                 const float *probs, int nb, int ns,
                                                                 const float *jitter, float eta, float *t_out,
                                                                 float *dt_out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const Clip c = clip_ray(B, ro, rd, r);
    float *to = t_out + (size_t)r * ns, *dto = dt_out + (size_t)r * ns;
    if (!(c.hi > c.lo)) {
        for (int j = 0; j < ns; ++j) to[j] = dto[j] = 0.0f;
        return;
    }
    const float *p = probs + (size_t)r * nb;
    const Df t0 = df_from_double(c.lo), w = df_from_double(__ddiv_rn(__dsub_rn(c.hi, c.lo), (double)nb));
    const float nbf = (float)nb, nsf = (float)ns;
    const Df one_m_eta = df_two_sum(1.0f, -eta);
    const Df eta_nb = df_div_n(Df{eta, 0.0f}, nbf);
    auto q_of = [&](float pb) { return df_add(df_mul_f(one_m_eta, pb), eta_nb); };
    Df Qtot = {0.0f, 0.0f};
#pragma unroll 8
    for (int b = 0; b < nb; ++b) Qtot = df_add(Qtot, q_of(__ldg(p + b)));
    const float jit = jitter ? jitter[r] : 0.5f;
    int b = 0;
    Df Qb = {0.0f, 0.0f}, qb = q_of(__ldg(p)), tprev = {0.0f, 0.0f};
    float pn = nb > 1 ? __ldg(p + 1) : 0.0f;   // p of bin b + 1
    for (int j = 0; j < ns; ++j) {
        const Df u = df_mul(df_div_n(df_two_sum((float)j, jit), nsf), Qtot);
        while (b < nb - 1) {
            const Df Qn = df_add(Qb, qb);
            if (!df_le(Qn, u)) break;
            Qb = Qn;
            ++b;
            qb = q_of(pn);
            pn = b + 1 < nb ? __ldg(p + b + 1) : 0.0f;
        }
        const float frac = __fdiv_rn(df_add(u, df_neg(Qb)).hi, qb.hi);
        const Df t = df_add(t0, df_mul(df_two_sum((float)b, frac), w));
        to[j] = t.hi;
        if (j > 0) dto[j - 1] = df_add(t, df_neg(tprev)).hi;
        tprev = t;
    }
    // last step: the bin width over n times the bin's normalised probability
    dto[ns - 1] = __fdiv_rn(w.hi, __fdiv_rn(__fmul_rn(nsf, qb.hi), Qtot.hi));
}

}  // namespace

int launch_proposal_fwd_tc(const dvgo_params &p, const dvgo_grid_desc &g, const dvgo_proposal_mlp &m, int R,
                           const float *ro, const float *rd, const float *labels, float *probs, float *loss,
                           cudaStream_t s);
int launch_proposal_bwd_tc(const dvgo_params &p, const dvgo_grid_desc &g, const dvgo_proposal_mlp &m, int R,
                           const float *ro, const float *rd, const float *labels, float *grad, cudaStream_t s);

}  // namespace dvgo

using namespace dvgo;

extern "C" {

int dvgo_weight_bins(const dvgo_params *p, const dvgo_grid_desc *dd, int n_rays, int n_bins, const void *workspace,
                     size_t ws_bytes, float *labels_out, void *stream) {
    if (!p || !dd || n_rays < 0 || n_bins < 1 || n_bins > 128 || !workspace || (n_rays > 0 && !labels_out))
        return DVGO_ERR_INVALID_ARG;
    if (p->mode != DVGO_MODE_FINE || !(p->step > 0.0f)) return DVGO_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return DVGO_ERR_WORKSPACE;
    if (n_rays == 0) return DVGO_OK;
    const size_t need = dvgo_workspace_size(p, dd, n_rays, nullptr);
    if (need == 0) return DVGO_ERR_INVALID_ARG;
    if (ws_bytes < need) return DVGO_ERR_WORKSPACE;
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double L = (double)dd->xyz_max[a] - (double)dd->xyz_min[a];
        diag2 = diag2 + L * L;
    }
    const long long cap = (long long)(ceil(sqrt(diag2) / (double)p->step) + 1.0);
    const WsLayout L = ws_layout(n_rays, cap * n_rays, DVGO_MODE_FINE);
    RenderArgs A;
    memset(&A, 0, sizeof(A));
    char *b = static_cast<char *>(const_cast<void *>(workspace));
    A.R = n_rays;
    A.step = p->step;
    A.rays = reinterpret_cast<RayRec *>(b + L.rays);
    A.samp = reinterpret_cast<float4 *>(b + L.samp);
    A.texit = reinterpret_cast<double *>(b + L.texit);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int blocks = (n_rays + 7) / 8;
    if (blocks > num_sms() * 16) blocks = num_sms() * 16;
    {
        ProfScope ps_(DVGO_K_WEIGHT_BINS, s);
        weight_bins_kernel<<<blocks, 256, 0, s>>>(A, n_bins, labels_out);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

static int proposal_launch(bool bwd, const dvgo_params *p, const dvgo_grid_desc *dd, const dvgo_proposal_desc *pd,
                           const dvgo_proposal_mlp *m, int n_rays, const float *rays_o, const float *rays_d,
                           const float *labels, float *probs_out, float *loss_out, float *grad, void *stream) {
    if (!p || !dd || !pd || !m || n_rays < 0) return DVGO_ERR_INVALID_ARG;
    if (!m->w0 || !m->b0 || !m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->w3 || !m->b3) return DVGO_ERR_INVALID_ARG;
    if (pd->n_bins != NB || pd->n_freq != NFQ || pd->width != PW) return DVGO_ERR_UNSUPPORTED;
    if (pd->precision != DVGO_MLP_FP32 && pd->precision != DVGO_MLP_BF16) return DVGO_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d)) return DVGO_ERR_INVALID_ARG;
    if (bwd && (!labels || !grad)) return DVGO_ERR_INVALID_ARG;
    if (!bwd && n_rays > 0 && !probs_out) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (loss_out && !bwd) cudaMemsetAsync(loss_out, 0, sizeof(float), s);
    if (n_rays == 0) return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
    if (!bwd && pd->precision == DVGO_MLP_BF16)
        return launch_proposal_fwd_tc(*p, *dd, *m, n_rays, rays_o, rays_d, labels, probs_out,
                                      labels ? loss_out : nullptr, s);
    if (bwd && pd->precision == DVGO_MLP_BF16)
        return launch_proposal_bwd_tc(*p, *dd, *m, n_rays, rays_o, rays_d, labels, grad, s);
    PropArgs P;
    P.R = n_rays;
    P.box = make_box(*p, *dd);
    P.ro = rays_o;
    P.rd = rays_d;
    P.labels = labels;
    P.w0 = m->w0; P.b0 = m->b0; P.w1 = m->w1; P.b1 = m->b1; P.w2 = m->w2; P.b2 = m->b2; P.w3 = m->w3; P.b3 = m->b3;
    P.probs = probs_out;
    P.loss = bwd ? nullptr : (labels ? loss_out : nullptr);
    P.grad = grad;
    void (*kern)(PropArgs) = bwd ? proposal_kernel<true> : proposal_kernel<false>;
    ensure_smem(reinterpret_cast<const void *>(kern), (int)sizeof(PropSmem));
    int ntiles = (n_rays + 1) / 2;
    int blocks = ntiles < num_sms() ? ntiles : num_sms();
    {
        ProfScope ps_(bwd ? DVGO_K_PROPOSAL_BWD : DVGO_K_PROPOSAL_FWD, s);
        kern<<<blocks, PNT, sizeof(PropSmem), s>>>(P);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

int dvgo_proposal_fwd(const dvgo_params *p, const dvgo_grid_desc *dd, const dvgo_proposal_desc *pd,
                      const dvgo_proposal_mlp *m, int n_rays, const float *rays_o, const float *rays_d,
                      const float *labels, float *probs_out, float *loss_out, void *stream) {
    return proposal_launch(false, p, dd, pd, m, n_rays, rays_o, rays_d, labels, probs_out, loss_out, nullptr, stream);
}

int dvgo_proposal_bwd(const dvgo_params *p, const dvgo_grid_desc *dd, const dvgo_proposal_desc *pd,
                      const dvgo_proposal_mlp *m, int n_rays, const float *rays_o, const float *rays_d,
                      const float *labels, float *grad_mlp, void *stream) {
    return proposal_launch(true, p, dd, pd, m, n_rays, rays_o, rays_d, labels, nullptr, nullptr, grad_mlp, stream);
}

int dvgo_sample_pdf(const dvgo_params *p, const dvgo_grid_desc *dd, int n_rays, const float *rays_o,
                    const float *rays_d, const float *probs, int n_bins, int n_samples, const float *jitter,
                    float eta, float *t_out, float *dt_out, void *stream) {
    if (!p || !dd || n_rays < 0 || n_bins < 1 || n_bins > kPdfMaxBins || n_samples < 1 ||
        n_samples > (1 << 24) || !(eta >= 0.0f && eta <= 1.0f))
        return DVGO_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d || !probs || !t_out || !dt_out)) return DVGO_ERR_INVALID_ARG;
    if (n_rays == 0) return DVGO_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        ProfScope ps_(DVGO_K_SAMPLE_PDF, s);
        sample_pdf_kernel<<<(n_rays + kPdfThreads - 1) / kPdfThreads, kPdfThreads, 0, s>>>(
            n_rays, make_box(*p, *dd), rays_o, rays_d, probs, n_bins, n_samples, jitter, eta, t_out, dt_out);
    }
    return cudaGetLastError() == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // extern "C"
