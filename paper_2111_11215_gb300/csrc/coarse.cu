// coarse.cu -- coarse-stage render (Sec. 4.1): density grid + view-invariant colour grid.
//
// One warp per ray, 32 consecutive samples per iteration.  Per sample:
//   sigma_ddot = interp(x, V_density)                      (Eq. coarse_queries_densities)
//   sigma = softplus(sigma_ddot + b), tau = sigma * dt       (Eq. density_activation, post-activation)
//   alpha = 1 - exp(-tau); removed when alpha < tau_f        (Eq. density_2_alpha, Sec. 4.2 skipping)
//   c = interp(x, V_rgb) (optionally sigmoid)                (Eq. coarse_queries)
// Compositing keeps the optical depth prefix sum: T_k = exp(-sum_{j<k} tau_j), w_k = T_k alpha_k,
// C_hat = sum w_k c_k + T_K bg (Eq. volume_rendering).  The prefix is a warp scan per chunk plus a
// running carry, which keeps T exact to FP32 rounding of the sum even over hundreds of samples.
//
// Backward (recomputes the forward chunk by chunk, stores nothing per sample):
//   dC/dc_k = w_k,  dC/dtau_k = T_{k+1} c_k - S_k,  S_k = sum_{j>k} w_j c_j + T_K bg,
//   dT_K/dtau_k = -T_K,  dtau_k/dsigma_ddot = dt * sigmoid(sigma_ddot + b);
// gradients are scattered to the 8 lattice corners with weights equal to the trilinear weights,
// summed first over runs of lanes that hit the same corner.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct CoarseSample {
    Cell cell;
    float z;      // sigma_ddot + b
    float tau;    // optical depth (0 when removed)
    float dt;
    float c[3];   // emitted colour
    bool kept;
};

__device__ __forceinline__ CoarseSample coarse_sample(const RenderArgs &A, const RayRec &rr, int ray, int k) {
    CoarseSample S;
    S.cell = sample_cell(A, rr, ray, k, S.dt);
    const float *rgb = static_cast<const float *>(A.cgrid);
    float s = 0.0f, col[3] = {0.0f, 0.0f, 0.0f}, v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        long long idx = corner_index(S.cell, q, A.ny, A.nz, A.packed);
        float w = corner_weight(S.cell, q);
        v[q] = __ldg(A.density + idx);
        s = fmaf(w, v[q], s);
        const float *cp = rgb + idx * 3;
        col[0] = fmaf(w, __ldg(cp + 0), col[0]);
        col[1] = fmaf(w, __ldg(cp + 1), col[1]);
        col[2] = fmaf(w, __ldg(cp + 2), col[2]);
    }
    S.z = s + A.shift_b;
    S.tau = A.act_order == DVGO_ACT_POST ? softplusf(S.z) * S.dt : tau_pre_in(A.act_order, S.cell, v, A.shift_b, S.dt);
    float alpha = -expm1f(-S.tau);
    S.kept = !(alpha < A.tau_f);
    if (!S.kept) S.tau = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) S.c[ch] = A.rgb_act ? sigmoidf_(col[ch]) : col[ch];
    return S;
}

// Block-level loss reduction: every block adds its partial sum; the last block to finish
// writes loss_out = sum / R.
__device__ void finish_loss(const RenderArgs &A, float part) {
    __shared__ float red[32];
    __shared__ bool last;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    part = warp_sum(part);
    if (lane == 0) red[wid] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        atomicAdd(&A.hdr->loss_acc, s);
        __threadfence();
        unsigned prev = atomicAdd(&A.hdr->done, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0 && A.loss_out) {
        __threadfence();
        float tot = atomicAdd(&A.hdr->loss_acc, 0.0f);
        A.loss_out[0] = A.R > 0 ? tot / (float)A.R : 0.0f;
    }
}

__global__ void __launch_bounds__(256) coarse_fwd_kernel(RenderArgs A) {
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    float loss_part = 0.0f;
    const bool aux = A.target && (A.w_pt != 0.0f || A.w_bg != 0.0f);
    for (int r = warp; r < A.R; r += nwarps) {
        const RayRec rr = A.rays[r];
        float tg[3] = {0.0f, 0.0f, 0.0f};
        if (aux)
            for (int ch = 0; ch < 3; ++ch) tg[ch] = A.target[3 * r + ch];
        float carry = 0.0f, acc[3] = {0.0f, 0.0f, 0.0f}, pt = 0.0f;
        for (int base = 0; base < rr.n; base += 32) {
            int k = base + lane;
            CoarseSample S;
            S.tau = 0.0f;
            S.c[0] = S.c[1] = S.c[2] = 0.0f;
            if (k < rr.n) S = coarse_sample(A, rr, r, k);
            float incl = warp_incl_scan(S.tau, lane);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            float T = expf(-(carry + excl));
            float w = T * -expm1f(-S.tau);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                acc[ch] = fmaf(w, S.c[ch], acc[ch]);
                const float e = S.c[ch] - tg[ch];
                pt = fmaf(w * e, e, pt);          // per-point rgb loss
            }
            carry += __shfl_sync(FULL, incl, 31);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) acc[ch] = warp_sum(acc[ch]);
        if (aux) pt = warp_sum(pt);
        if (lane == 0) {
            float TK = expf(-carry);
            float rgb[3];
            for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(TK, A.bg[ch], acc[ch]);
            for (int ch = 0; ch < 3; ++ch) A.rgb_out[3 * r + ch] = rgb[ch];
            if (A.tfinal_out) A.tfinal_out[r] = TK;
            A.rayout[r] = make_float4(rgb[0], rgb[1], rgb[2], TK);
            if (A.target) {
                for (int ch = 0; ch < 3; ++ch) {
                    float e = rgb[ch] - A.target[3 * r + ch];
                    loss_part = fmaf(e, e, loss_part);
                    if (A.dloss_out) A.dloss_out[3 * r + ch] = 2.0f * e / (float)A.R;
                }
            }
            if (aux) {
                loss_part += A.w_pt * pt + A.w_bg * bg_entropy(TK);
                A.rtarget[r] = make_float4(tg[0], tg[1], tg[2], 0.0f);
            }
        }
    }
    if (A.target) finish_loss(A, loss_part);
}

// Optical depth of one sample (density gather only), with the removal rule.
__device__ __forceinline__ float coarse_tau(const RenderArgs &A, const RayRec &rr, int ray, int k) {
    float dt;
    Cell c = sample_cell(A, rr, ray, k, dt);
    float s = 0.0f, v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        v[q] = __ldg(A.density + corner_index(c, q, A.ny, A.nz, A.packed));
        s = fmaf(corner_weight(c, q), v[q], s);
    }
    float tau = A.act_order == DVGO_ACT_POST ? softplusf(s + A.shift_b) * dt : tau_pre_in(A.act_order, c, v, A.shift_b, dt);
    return (-expm1f(-tau) < A.tau_f) ? 0.0f : tau;
}

// Backward: pass 1 (front to back) recomputes the optical depth at the start of every chunk;
// pass 2 (back to front) recomputes the samples and evaluates dC/dtau_k as the suffix sum
// D_k = sum_{j>=k} T_{j+1} (c_j - c_{j+1}) with c_K = bg (from D_k - D_{k+1} = T_{k+1}(c_k - c_{k+1})
// and D_{K-1} = T_K (c_{K-1} - bg)), which avoids the cancellation of T_{k+1} c_k - S_k.
__global__ void __launch_bounds__(256) coarse_bwd_kernel(RenderArgs A) {
    __shared__ float s_pre[8][kMaxChunks];
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < A.R; r += nwarps) {
        const RayRec rr = A.rays[r];
        if (rr.n == 0) continue;
        const int nch = (rr.n + 31) >> 5;
        const float TK = A.rayout[r].w;
        const float g[3] = {A.grad_rgb[3 * r], A.grad_rgb[3 * r + 1], A.grad_rgb[3 * r + 2]};
        // auxiliary losses of the forward: the background entropy enters through T_K, the
        // per-point rgb loss adds 2 w_pt w_k (c_k - C) / R to dL/dc_k
        const bool aux = A.hdr->aux != 0;
        float4 tg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (aux) tg = A.rtarget[r];
        const float tgc[3] = {tg.x, tg.y, tg.z};
        const float gT = (A.grad_tfinal ? A.grad_tfinal[r] : 0.0f) +
                         (aux ? A.w_bg * bg_entropy_dT(TK) / (float)A.R : 0.0f);
        const float kpt = aux ? 2.0f * A.w_pt / (float)A.R : 0.0f;
        float carry = 0.0f;
        for (int ci = 0; ci < nch; ++ci) {
            int k = ci * 32 + lane;
            float tau = k < rr.n ? coarse_tau(A, rr, r, k) : 0.0f;
            float incl = warp_incl_scan(tau, lane);
            if (lane == 0) s_pre[wib][ci] = carry;
            carry += __shfl_sync(FULL, incl, 31);
        }
        __syncwarp();
        float Dc[3] = {0.0f, 0.0f, 0.0f};
        float cnext[3] = {A.bg[0], A.bg[1], A.bg[2]};
        for (int ci = nch - 1; ci >= 0; --ci) {
            int k = ci * 32 + lane;
            bool valid = k < rr.n;
            CoarseSample S;
            S.tau = 0.0f;
            S.kept = false;
            S.z = 0.0f;
            S.dt = 0.0f;
            S.c[0] = S.c[1] = S.c[2] = 0.0f;
            S.cell.i0 = S.cell.j0 = S.cell.k0 = 0;
            S.cell.fx = S.cell.fy = S.cell.fz = 0.0f;
            if (valid) S = coarse_sample(A, rr, r, k);
            float pre = s_pre[wib][ci];
            float incl = warp_incl_scan(S.tau, lane);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            float T = expf(-(pre + excl));
            float T1 = expf(-(pre + incl));
            float w = T * -expm1f(-S.tau);
            float D[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float cn = __shfl_down_sync(FULL, S.c[ch], 1);
                if (lane == 31 || k + 1 >= rr.n) cn = (k + 1 >= rr.n) ? A.bg[ch] : cnext[ch];
                float X = valid ? T1 * (S.c[ch] - cn) : 0.0f;
                float sx = warp_suffix_scan(X, lane);
                D[ch] = Dc[ch] + sx;
                Dc[ch] += __shfl_sync(FULL, sx, 0);
                cnext[ch] = __shfl_sync(FULL, S.c[ch], 0);
            }
            float dtau = -gT * TK;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) dtau = fmaf(g[ch], D[ch], dtau);
            bool act = valid && S.kept;
            float dz = act ? dtau * S.dt * sigmoidf_(S.z) : 0.0f;
            float dc[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float gc = g[ch] * w + kpt * w * (S.c[ch] - tgc[ch]);
                if (A.rgb_act) gc *= S.c[ch] * (1.0f - S.c[ch]);
                dc[ch] = act ? gc : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int idx = (int)corner_index(S.cell, q, A.ny, A.nz, A.packed);
                float cw = corner_weight(S.cell, q);
                Seg sg = make_seg(act ? idx : -1 - lane, lane);
                float gq = dz * cw;
                if (A.act_order != DVGO_ACT_POST)
                    gq = act ? dtau * dtau_dv_pre_in(A.act_order, S.cell, q, __ldg(A.density + idx), A.shift_b, S.dt,
                                                     S.tau)
                             : 0.0f;
                float v = seg_sum(gq, sg, lane);
                if (act && sg.tail) atomicAdd(A.grad_density + idx, v);
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float vc = seg_sum(dc[ch] * cw, sg, lane);
                    if (act && sg.tail) atomicAdd(A.grad_cgrid + (long long)idx * 3 + ch, vc);
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace

static int warp_grid(int R, int warps_per_block) {
    int want = (R + warps_per_block - 1) / warps_per_block;
    int cap = num_sms() * 16;
    if (want > cap) want = cap;
    return want < 1 ? 1 : want;
}

void launch_coarse_fwd(const RenderArgs &A, cudaStream_t s) {
    {
        ProfScope ps_(DVGO_K_COARSE_FWD, s);
        coarse_fwd_kernel<<<warp_grid(A.R, 8), 256, 0, s>>>(A);
    }
}

void launch_coarse_bwd(const RenderArgs &A, cudaStream_t s) {
    {
        ProfScope ps_(DVGO_K_COARSE_BWD, s);
        coarse_bwd_kernel<<<warp_grid(A.R, 8), 256, 0, s>>>(A);
    }
}

}  // namespace dvgo
