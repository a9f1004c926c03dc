// fine_ray.cu -- the per-ray kernels of the fine-stage render (Sec. 4.2).
//
// fine_density:   warp per ray.  For each sample k of the ray: position; optionally the
//                 known-free-space test on the coarse grid (Sec. 4.2), which removes the sample
//                 before any fine query; density gather, sigma_ddot = interp(x, V_density)
//                 (Eq. fine_queries_densities), tau_k = softplus(sigma_ddot + b) * dt_k
//                 (Eq. density_activation, post-activation), removed when
//                 alpha_k = 1 - exp(-tau_k) < tau_f (Sec. 4.2 free space skipping).
//                 Writes tau_k to the sample slot and appends kept samples to a compact list
//                 (one atomic per warp chunk, lane order kept) for the colour kernel.
//                 Early ray termination, exact: the compositing pass forms T_k = exp(-(sum_{j<k}
//                 tau_j)) with the same chunked warp scan; a sample where that is exactly 0 in
//                 FP32 has weight 0 and no gradient through it, so it is not kept, its slot gets
//                 tau = +inf (alpha 1, every later T and T_K stay exactly 0), and the rest of the
//                 ray is written the same way without density queries.
// fine_composite: warp per ray.  T_k = exp(-sum_{j<k} tau_j), w_k = T_k alpha_k,
//                 C_hat = sum w_k c_k + T_K bg (Eq. volume_rendering), loss (Eq. photo_loss).
// fine_comp_bwd:  warp per ray.  dC/dc_k = w_k -> stored for the colour backward;
//                 dC/dtau_k = T_{k+1} c_k - S_k with S_k = sum_{j>k} w_j c_j + T_K bg, evaluated as
//                 D_k = sum_{j>=k} T_{j+1} (c_j - c_{j+1}) (c_K = bg), which follows from
//                 D_k - D_{k+1} = T_{k+1} (c_k - c_{k+1}) and D_{K-1} = T_K (c_{K-1} - bg); the sum
//                 is taken from the back of the ray, so no large terms cancel when the colour in
//                 front of a surface matches the colour behind it.  dT_K/dtau_k = -T_K;
//                 dtau/dsigma_ddot = dt sigmoid(sigma_ddot + b) = dt (1 - exp(-tau/dt));
//                 the density gradient is scattered to the 8 corners (runs of lanes that share a
//                 corner are summed before one atomic).

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Specialised on the known-free-space test and the activation order (uniform per launch), so the
// default configuration carries neither.  A warp walks its ray two 32-sample chunks at a time: the
// optical depths of both chunks are formed first (their density loads in flight together), then
// the chunks are composited in order, and one atomic reserves the kept-list slots of both.
template <bool kFreeSpace, int kOrder, bool kExpl>
__device__ __forceinline__ float sample_tau(const RenderArgs &A, const RayRec &rr, int r, int k, bool &kept) {
    float dt;
    long long u[3];
    if (kExpl) {   // sample_fx's explicit branch, without the run-time test
        const double t = (double)A.ts[(long long)r * A.n_expl + k];
        dt = A.dts[(long long)r * A.n_expl + k];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = rr.uefx[a] + to_fx((t - rr.t_enter) * rr.e[a]);
    } else {
        dt = A.step;
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = rr.u0fx[a] + (long long)k * rr.dfx[a];
    }
    kept = false;
    if (kFreeSpace && known_free(A, u)) return 0.0f;   // known free space: no fine query
    const Cell c = cell_from_fx(u, A.nx, A.ny, A.nz);
    float tau;
    if (kOrder == DVGO_ACT_POST) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            s = fmaf(corner_weight(c, q), __ldg(A.density + corner_index(c, q, A.ny, A.nz, A.packed)), s);
        tau = softplusf(s + A.shift_b) * dt;
    } else {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(A.density + corner_index(c, q, A.ny, A.nz, A.packed));
        tau = tau_pre_in(kOrder, c, v, A.shift_b, dt);
    }
    kept = !(-expm1f(-tau) < A.tau_f);
    return kept ? tau : 0.0f;
}

// 128-thread blocks: the pass runs beside the feature-grid Adam of the other stream (3 x 256
// threads x 56 registers per SM), next to which three of them fit per SM where one 256-thread
// block does.
constexpr int kDensityThreads = 128;
#ifndef DVGO_DENSITY_MIN_BLOCKS
#define DVGO_DENSITY_MIN_BLOCKS 1
#endif
template <bool kFreeSpace, int kOrder, bool kExpl>
__global__ void __launch_bounds__(kDensityThreads, DVGO_DENSITY_MIN_BLOCKS) fine_density_kernel(RenderArgs A) {
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < A.R; r += nwarps) {
        const RayRec rr = A.rays[r];
        float carry = 0.0f;          // optical depth before this chunk, as the compositing pass forms it
        for (int base = 0; base < rr.n; base += 64) {
            if (isinf(carry)) {      // terminated: T = 0 from here on
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (base + 32 * h + lane < rr.n)
                        A.samp[rr.off + base + 32 * h + lane] = make_float4(INFINITY, 0.0f, 0.0f, 0.0f);
                continue;
            }
            float tau[2];
            bool kept[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = base + 32 * h + lane;
                tau[h] = 0.0f;
                kept[h] = false;
                if (k < rr.n) tau[h] = sample_tau<kFreeSpace, kOrder, kExpl>(A, rr, r, k, kept[h]);
            }
            unsigned m[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = base + 32 * h + lane;
                if (isinf(carry)) {  // the first chunk terminated the ray
                    kept[h] = false;
                    tau[h] = INFINITY;
                } else {
                    // T_k of the compositing pass; exactly 0 -> terminated (the scan sees tau of lanes below only)
                    const float incl = warp_incl_scan(tau[h], lane);
                    float excl = __shfl_up_sync(FULL, incl, 1);
                    if (lane == 0) excl = 0.0f;
                    if (expf(-(carry + excl)) == 0.0f) {
                        kept[h] = false;
                        tau[h] = INFINITY;
                    }
                    const bool any_dead = __any_sync(FULL, isinf(tau[h]));
                    carry = any_dead ? INFINITY : carry + __shfl_sync(FULL, incl, 31);
                }
                if (k < rr.n) A.samp[rr.off + k] = make_float4(tau[h], 0.0f, 0.0f, 0.0f);
                m[h] = __ballot_sync(FULL, kept[h]);
            }
            const int cnt0 = __popc(m[0]), cnt = cnt0 + __popc(m[1]);
            int base_slot = 0;
            if (lane == 0 && cnt) base_slot = atomicAdd(&A.hdr->n_kept, cnt);
            base_slot = __shfl_sync(FULL, base_slot, 0);
            const unsigned below = (1u << lane) - 1u;
            if (kept[0]) A.kept[base_slot + __popc(m[0] & below)] = make_int2(rr.off + base + lane, r);
            if (kept[1]) A.kept[base_slot + cnt0 + __popc(m[1] & below)] = make_int2(rr.off + base + 32 + lane, r);
        }
    }
}

__device__ void finish_loss_fine(const RenderArgs &A, float part) {
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

__global__ void __launch_bounds__(256) fine_composite_kernel(RenderArgs A) {
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    float loss_part = 0.0f;
    const bool aux = A.target && (A.w_pt != 0.0f || A.w_bg != 0.0f);
    for (int r = warp; r < A.R; r += nwarps) {
        const int n = A.rays[r].n, off = A.rays[r].off;
        float tg[3] = {0.0f, 0.0f, 0.0f};
        if (aux)
            for (int ch = 0; ch < 3; ++ch) tg[ch] = A.target[3 * r + ch];
        float carry = 0.0f, acc[3] = {0.0f, 0.0f, 0.0f}, pt = 0.0f;
        for (int base = 0; base < n; base += 32) {
            int k = base + lane;
            float4 sv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (k < n) sv = A.samp[off + k];
            float incl = warp_incl_scan(sv.x, lane);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            float w = expf(-(carry + excl)) * -expm1f(-sv.x);
            acc[0] = fmaf(w, sv.y, acc[0]);
            acc[1] = fmaf(w, sv.z, acc[1]);
            acc[2] = fmaf(w, sv.w, acc[2]);
            const float e0 = sv.y - tg[0], e1 = sv.z - tg[1], e2 = sv.w - tg[2];
            pt = fmaf(w, fmaf(e0, e0, fmaf(e1, e1, e2 * e2)), pt);   // per-point rgb loss
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
    if (A.target) finish_loss_fine(A, loss_part);
}

template <int kOrder>
__global__ void __launch_bounds__(256) fine_comp_bwd_kernel(RenderArgs A) {
    __shared__ float s_pre[8][kMaxChunks];   // optical depth before each chunk, per warp
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
        const float gT = (A.grad_tfinal ? A.grad_tfinal[r] : 0.0f) +
                         (aux ? A.w_bg * bg_entropy_dT(TK) / (float)A.R : 0.0f);
        const float kpt = aux ? 2.0f * A.w_pt / (float)A.R : 0.0f;
        // pass 1 (front to back): optical depth at the start of every chunk, as in the forward
        float carry = 0.0f;
        for (int ci = 0; ci < nch; ++ci) {
            int k = ci * 32 + lane;
            float tau = k < rr.n ? A.samp[rr.off + k].x : 0.0f;
            float incl = warp_incl_scan(tau, lane);
            if (lane == 0) s_pre[wib][ci] = carry;
            carry += __shfl_sync(FULL, incl, 31);
        }
        __syncwarp();
        // pass 2 (back to front): D_k = dC/dtau_k as a suffix sum of T_{j+1} (c_j - c_{j+1})
        float Dc[3] = {0.0f, 0.0f, 0.0f};
        float cnext[3] = {A.bg[0], A.bg[1], A.bg[2]};   // colour after the chunk's last sample
        for (int ci = nch - 1; ci >= 0; --ci) {
            int k = ci * 32 + lane;
            bool valid = k < rr.n;
            float4 sv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (valid) sv = A.samp[rr.off + k];
            const float cc[3] = {sv.y, sv.z, sv.w};
            float pre = s_pre[wib][ci];
            float incl = warp_incl_scan(sv.x, lane);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0.0f;
            float T = expf(-(pre + excl));
            float T1 = expf(-(pre + incl));
            float w = T * -expm1f(-sv.x);
            float D[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float cn = __shfl_down_sync(FULL, cc[ch], 1);
                if (lane == 31 || k + 1 >= rr.n) cn = (k + 1 >= rr.n) ? A.bg[ch] : cnext[ch];
                float X = valid ? T1 * (cc[ch] - cn) : 0.0f;
                float sx = warp_suffix_scan(X, lane);
                D[ch] = Dc[ch] + sx;
                Dc[ch] += __shfl_sync(FULL, sx, 0);
                cnext[ch] = __shfl_sync(FULL, cc[ch], 0);
            }
            float dtau = -gT * TK;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) dtau = fmaf(g[ch], D[ch], dtau);
            // kept samples have tau > 0 or an exactly-zero sigmoid factor; removed ones have tau = 0
            bool act = valid && sv.x > 0.0f;
            Cell c;
            c.i0 = c.j0 = c.k0 = 0;
            c.fx = c.fy = c.fz = 0.0f;
            float dz = 0.0f, dt = 0.0f;
            if (valid) {
                c = sample_cell(A, rr, r, k, dt);
                dz = act ? dtau * dt * -expm1f(-sv.x / dt) : 0.0f;   // post: dt sigmoid(z) = dt (1 - e^{-tau/dt})
                // dL/dc_k for the colour backward (only kept samples are read back)
                A.sgrad[rr.off + k] = make_float4(0.0f, fmaf(kpt * w, cc[0] - tg.x, g[0] * w),
                                                  fmaf(kpt * w, cc[1] - tg.y, g[1] * w),
                                                  fmaf(kpt * w, cc[2] - tg.z, g[2] * w));
            }
            // Runs of lanes in the same cell share all 8 corners (corner q of two samples is the
            // same point exactly when their cells are), so one segmentation serves every corner;
            // the 8 segmented sums run side by side and stop after the warp's longest run.
            const Seg sg = make_seg(act ? cell_base(c, A.ny, A.nz, A.packed) : -1 - lane, lane);
            int run = lane - sg.first + 1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) run = max(run, __shfl_xor_sync(FULL, run, o));
            int idx[8];
            float gq[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                idx[q] = (int)corner_index(c, q, A.ny, A.nz, A.packed);
                if (kOrder == DVGO_ACT_POST) {
                    gq[q] = dz * corner_weight(c, q);
                } else {
                    gq[q] = act ? dtau * dtau_dv_pre_in(kOrder, c, q, __ldg(A.density + idx[q]), A.shift_b, dt, sv.x)
                                : 0.0f;
                }
            }
            for (int o = 1; o < run; o <<= 1) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float n = __shfl_up_sync(FULL, gq[q], o);
                    if (lane - o >= sg.first) gq[q] += n;
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)   // the run's last lane adds its total; terminated samples add 0
                if (act && sg.tail && gq[q] != 0.0f) atomicAdd(A.grad_density + idx[q], gq[q]);
        }
        __syncwarp();
    }
}

int warp_grid(int R, int warps_per_block) {
    int want = (R + warps_per_block - 1) / warps_per_block;
    int cap = num_sms() * 16;
    if (want > cap) want = cap;
    return want < 1 ? 1 : want;
}

}  // namespace

void launch_fine_density(const RenderArgs &A, cudaStream_t s) {
    {
        ProfScope ps_(DVGO_K_FINE_DENSITY, s);
        const dim3 g(warp_grid(A.R, kDensityThreads / 32));
        const bool fs = A.fs_density != nullptr;
        const bool ex = A.ts != nullptr;
        switch (A.act_order * 4 + (fs ? 2 : 0) + (ex ? 1 : 0)) {
            case 0: fine_density_kernel<false, DVGO_ACT_POST, false><<<g, kDensityThreads, 0, s>>>(A); break;
            case 1: fine_density_kernel<false, DVGO_ACT_POST, true><<<g, kDensityThreads, 0, s>>>(A); break;
            case 2: fine_density_kernel<true, DVGO_ACT_POST, false><<<g, kDensityThreads, 0, s>>>(A); break;
            case 3: fine_density_kernel<true, DVGO_ACT_POST, true><<<g, kDensityThreads, 0, s>>>(A); break;
            case 4: fine_density_kernel<false, DVGO_ACT_PRE, false><<<g, kDensityThreads, 0, s>>>(A); break;
            case 5: fine_density_kernel<false, DVGO_ACT_PRE, true><<<g, kDensityThreads, 0, s>>>(A); break;
            case 6: fine_density_kernel<true, DVGO_ACT_PRE, false><<<g, kDensityThreads, 0, s>>>(A); break;
            case 7: fine_density_kernel<true, DVGO_ACT_PRE, true><<<g, kDensityThreads, 0, s>>>(A); break;
            case 8: fine_density_kernel<false, DVGO_ACT_IN, false><<<g, kDensityThreads, 0, s>>>(A); break;
            case 9: fine_density_kernel<false, DVGO_ACT_IN, true><<<g, kDensityThreads, 0, s>>>(A); break;
            case 10: fine_density_kernel<true, DVGO_ACT_IN, false><<<g, kDensityThreads, 0, s>>>(A); break;
            default: fine_density_kernel<true, DVGO_ACT_IN, true><<<g, kDensityThreads, 0, s>>>(A); break;
        }
    }
}
void launch_fine_composite_fwd(const RenderArgs &A, cudaStream_t s) {
    {
        ProfScope ps_(DVGO_K_FINE_COMPOSITE, s);
        fine_composite_kernel<<<warp_grid(A.R, 8), 256, 0, s>>>(A);
    }
}
void launch_fine_composite_bwd(const RenderArgs &A, cudaStream_t s) {
    {
        ProfScope ps_(DVGO_K_FINE_COMP_BWD, s);
        const dim3 g(warp_grid(A.R, 8));
        if (A.act_order == DVGO_ACT_PRE) fine_comp_bwd_kernel<DVGO_ACT_PRE><<<g, 256, 0, s>>>(A);
        else if (A.act_order == DVGO_ACT_IN) fine_comp_bwd_kernel<DVGO_ACT_IN><<<g, 256, 0, s>>>(A);
        else fine_comp_bwd_kernel<DVGO_ACT_POST><<<g, 256, 0, s>>>(A);
    }
}

}  // namespace dvgo
