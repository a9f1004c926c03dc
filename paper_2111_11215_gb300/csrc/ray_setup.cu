// ray_setup.cu -- per-ray clipping and sample counting, and the exclusive scan of the counts.
//
// Sec. 4.2 (fine-stage points sampling): the near and far bounds of every ray become the two
// ends of its intersection with the grid's bounding box (the near bound stays put when the
// origin is inside).  Eq. coarse_sample / Supp. A: samples are equally spaced by the step and
// shifted by the per-ray jitter p.  With a normalised direction the count is the number of k >= 0
// with t_enter + (k + p) * step < t_exit.
//
// The count is an integer decided by floating point, so it is computed in FP64 with every
// operation a separately rounded IEEE operation (__dadd_rn & co. keep nvcc from contracting
// them into FMAs):
//   len   = sqrt((dx*dx + dy*dy) + dz*dz),   dn = d / len
//   per axis with dn != 0: t1 = (min - o) / dn, t2 = (max - o) / dn, lo = max(lo, min(t1, t2)),
//                          hi = min(hi, max(t1, t2));  starting from lo = t_near, hi = t_far
//   per axis with dn == 0 and o outside the slab: empty
//   n = ceil((hi - lo) / step - p) when hi > lo, capped at ceil(|max - min| / step) + 1.

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

__global__ void __launch_bounds__(64) ray_setup_kernel(RenderArgs A, const float *__restrict__ rays_o,
                                                        const float *__restrict__ rays_d,
                                                        const float *__restrict__ jitter, double3 bmin,
                                                        double3 bmax, double3 scale, double t_near,
                                                        double t_far, double step, double cap,
                                                        int n_expl) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        A.hdr->total = 0;
        A.hdr->n_kept = 0;
        A.hdr->done = 0u;
        A.hdr->loss_acc = 0.0f;
        A.hdr->aux = (A.target && (A.w_pt != 0.0f || A.w_bg != 0.0f)) ? 1 : 0;
        A.hdr->xcache = A.xcache != nullptr ? 1 : 0;
    }
    if (r >= A.R) return;
    double o[3] = {(double)rays_o[3 * r], (double)rays_o[3 * r + 1], (double)rays_o[3 * r + 2]};
    double d[3] = {(double)rays_d[3 * r], (double)rays_d[3 * r + 1], (double)rays_d[3 * r + 2]};
    double mn[3] = {bmin.x, bmin.y, bmin.z}, mx[3] = {bmax.x, bmax.y, bmax.z};
    double sc[3] = {scale.x, scale.y, scale.z};
    double p = jitter ? (double)jitter[r] : 0.5;

    const Clip cl = slab_clip(o, d, mn, mx, t_near, t_far);
    const bool ok = cl.ok;
    const double lo = cl.lo, hi = cl.hi;
    const double *dn = cl.dn;
    RayRec rec;
    int n = 0;
    if (hi > lo) {
        double q = __ddiv_rn(__dsub_rn(hi, lo), step);
        q = __dsub_rn(q, p);
        double c = ceil(q);
        if (c > cap) c = cap;
        n = c > 0.0 ? (int)c : 0;
        if (n_expl >= 0) n = n_expl;   // explicit samples: all or nothing
    }
    const bool uniform = n > 0 && n_expl < 0;
    const double t_first = uniform ? fma(p, step, lo) : 0.0;   // t of sample 0 of the uniform stepping
    for (int a = 0; a < 3; ++a) {
        const double uo = __dmul_rn(__dsub_rn(o[a], mn[a]), sc[a]);
        rec.e[a] = __dmul_rn(dn[a], sc[a]);
        rec.dir[a] = (float)dn[a];
        // fixed-point values only where they are used: in range for any sample inside the box
        rec.uefx[a] = n > 0 ? to_fx(fma(lo, rec.e[a], uo)) : 0;
        rec.u0fx[a] = uniform ? to_fx(fma(t_first, rec.e[a], uo)) : 0;
        rec.dfx[a] = uniform ? to_fx(step * rec.e[a]) : 0;
    }
    rec.t_enter = lo;
    rec.p = (float)p;
    if (A.texit) A.texit[r] = hi;
    if (A.pe) {
        // positional encoding of the normalised direction (fine-stage MLP input, Supp. A, k_d = 4):
        // [d, sin(2^k d_c) (c-major), cos(2^k d_c) (c-major)]
        float *pe = A.pe + (size_t)r * kPeStride;
        for (int a = 0; a < 3; ++a) {
            float dv = rec.dir[a];
            pe[a] = dv;
            for (int k = 0; k < 4; ++k) {
                float sv, cv;
                sincosf(ldexpf(dv, k), &sv, &cv);
                pe[3 + a * 4 + k] = sv;
                pe[15 + a * 4 + k] = cv;
            }
        }
        for (int k = 27; k < kPeStride; ++k) pe[k] = 0.0f;
    }
    rec.n = n;
    rec.off = ok ? 0 : -1;   // -1 marks a ray with a zero / non-finite direction for the scan
    A.rays[r] = rec;
}

// Exclusive scan of RayRec::n into RayRec::off by one block; the total and the flag word (a ray
// with a zero / non-finite direction) go to the header.  The block is small (256 threads) so that
// it fits on an SM beside the HBM-bound Adam step of another stream; a 1024-thread block does not,
// and would wait for the whole Adam.  It works in rounds of 256 x kScanPer rays: thread t takes
// the contiguous run of kScanPer rays at base + kScanPer t and issues all their (n, off) loads at
// once (one load latency per round, not one per ray), the run sums are scanned across the block
// with warp shuffles, and the offsets are written from registers.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;

__global__ void __launch_bounds__(kScanThreads) scan_counts_kernel(RenderArgs A) {
    constexpr int NW = kScanThreads / 32;
    __shared__ int warp_tot[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int carry = 0, bad = 0;
    for (int base = 0; base < A.R; base += kScanThreads * kScanPer) {
        const int beg = base + tid * kScanPer;
        int n[kScanPer], local = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            n[k] = 0;
            if (beg + k < A.R) {
                const int2 no = *reinterpret_cast<const int2 *>(&A.rays[beg + k].n);   // (n, off)
                n[k] = no.x;
                bad |= no.y < 0;
            }
            local += n[k];
        }
        // inclusive warp scan of the run sums, then the warp totals
        int v = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int t = warp_tot[w];
            before += w < wid ? t : 0;
            total += t;
        }
        __syncthreads();   // warp_tot is rewritten by the next round
        int run = carry + before + v - local;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            if (beg + k < A.R) A.rays[beg + k].off = run;
            run += n[k];
        }
        carry += total;
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        A.hdr->total = carry;
        A.hdr->flags = bad ? 1 : 0;
    }
}

}  // namespace

void launch_ray_setup(const RenderArgs &A, const float *rays_o, const float *rays_d, const float *jitter,
                      const dvgo_params &p, const dvgo_grid_desc &g, long long cap, cudaStream_t s) {
    double3 bmin = make_double3(g.xyz_min[0], g.xyz_min[1], g.xyz_min[2]);
    double3 bmax = make_double3(g.xyz_max[0], g.xyz_max[1], g.xyz_max[2]);
    double3 sc = make_double3((double)(g.nx - 1) / (bmax.x - bmin.x), (double)(g.ny - 1) / (bmax.y - bmin.y),
                              (double)(g.nz - 1) / (bmax.z - bmin.z));
    int blocks = (A.R + 63) / 64;
    if (blocks < 1) blocks = 1;
    {
        ProfScope ps_(DVGO_K_RAY_SETUP, s);
        ray_setup_kernel<<<blocks, 64, 0, s>>>(A, rays_o, rays_d, jitter, bmin, bmax, sc, (double)p.t_near,
                                           (double)p.t_far, (double)p.step, (double)cap,
                                           A.ts ? A.n_expl : -1);
    }
    {
        ProfScope ps_(DVGO_K_SCAN, s);
        scan_counts_kernel<<<1, kScanThreads, 0, s>>>(A);
    }
}

WsLayout ws_layout(int R, long long max_samples, int mode, bool xcache) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    WsLayout L;
    size_t o = 0;
    L.header = o; o += up(sizeof(WsHeader));
    L.rays = o; o += up(sizeof(RayRec) * (size_t)(R > 0 ? R : 1));
    L.rayout = o; o += up(sizeof(float4) * (size_t)(R > 0 ? R : 1));
    size_t S = (size_t)(max_samples > 0 ? max_samples : 1);
    L.pe = L.texit = 0;
    if (mode == DVGO_MODE_FINE) {
        L.pe = o; o += up(sizeof(float) * kPeStride * (size_t)(R > 0 ? R : 1));
        L.texit = o; o += up(sizeof(double) * (size_t)(R > 0 ? R : 1));
        L.samp = o; o += up(sizeof(float4) * S);
        L.sgrad = o; o += up(sizeof(float4) * S);
        L.kept = o; o += up(sizeof(int2) * S);
    } else {
        L.samp = L.sgrad = L.kept = 0;
    }
    // last; counted in total, so the allocation-free forward's static scratch includes it even
    // though that forward (no auxiliary losses) never writes it
    L.rtarget = o; o += up(sizeof(float4) * (size_t)(R > 0 ? R : 1));
    L.xcache = 0;
    if (xcache && mode == DVGO_MODE_FINE) {   // 128 kept samples per tile, a 16 KiB panel each
        o = (o + 1023) & ~(size_t)1023;
        L.xcache = o;
        o += (size_t)16384 * ((S + 127) / 128);
    }
    L.total = o;
    L.max_samples = max_samples;
    return L;
}

}  // namespace dvgo
