// dvgo_api.cu -- the extern "C" entry points of libdvgo: argument validation, workspace
// layout and the launch sequence of each call (see dvgo.h for the contract).

#include <math.h>
#include <mutex>
#include <set>
#include <utility>

#include "dvgo_internal.cuh"

namespace dvgo {

void launch_fine_colour_fwd_simt(const RenderArgs &A, cudaStream_t s);
void launch_fine_colour_bwd_simt(const RenderArgs &A, cudaStream_t s);
int launch_fine_colour_fwd_tc(const RenderArgs &A, cudaStream_t s);
int launch_fine_colour_bwd_tc(const RenderArgs &A, cudaStream_t s);

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

void ensure_smem(const void *kernel, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, kernel})) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.insert({dev, kernel});
}

namespace {

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

bool grid_ok(const dvgo_grid_desc *g) {
    if (!g) return false;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || g->channels < 1) return false;
    if (g->layout != DVGO_LAYOUT_CANONICAL && g->layout != DVGO_LAYOUT_PACKED) return false;
    if (g->layout == DVGO_LAYOUT_PACKED && (g->nx > 2048 || g->ny > 2048 || g->nz > 1024)) return false;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(g->xyz_min[a]) || !isfinite(g->xyz_max[a]) || !(g->xyz_max[a] > g->xyz_min[a])) return false;
    long long n = (long long)((g->nx + 3) / 4 * 4) * ((g->ny + 3) / 4 * 4) * ((g->nz + 3) / 4 * 4) * g->channels;
    return n < (1LL << 31);
}

bool same_lattice(const dvgo_grid_desc *a, const dvgo_grid_desc *b) {
    if (a->nx != b->nx || a->ny != b->ny || a->nz != b->nz || a->layout != b->layout) return false;
    for (int i = 0; i < 3; ++i)
        if (a->xyz_min[i] != b->xyz_min[i] || a->xyz_max[i] != b->xyz_max[i]) return false;
    return true;
}

// Longest possible ray, computed exactly like the count cap of the ray setup.
long long sample_cap(const dvgo_params *p, const dvgo_grid_desc *g) {
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double L = (double)g->xyz_max[a] - (double)g->xyz_min[a];
        diag2 = diag2 + L * L;
    }
    return (long long)(ceil(sqrt(diag2) / (double)p->step) + 1.0);
}

long long max_samples(const dvgo_params *p, const dvgo_grid_desc *g, int R, const dvgo_samples *ex) {
    long long per = ex ? (long long)ex->n_per_ray : sample_cap(p, g);
    return per * (long long)R;
}

int check_common(const dvgo_params *p, const dvgo_grid_desc *dd, const float *density, const dvgo_grid_desc *cd,
                 const void *cgrid, const dvgo_mlp *mlp, int R, const float *ro, const float *rd,
                 const dvgo_samples *ex) {
    if (!p || !dd || !cd || !density || !cgrid || R < 0) return DVGO_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(cgrid) & 15u) != 0) return DVGO_ERR_INVALID_ARG;   // 16-byte loads
    if (R > 0 && (!ro || !rd)) return DVGO_ERR_INVALID_ARG;
    if (!grid_ok(dd) || !grid_ok(cd) || dd->channels != 1 || dd->dtype != DVGO_DTYPE_F32) return DVGO_ERR_INVALID_ARG;
    if (!same_lattice(dd, cd)) return DVGO_ERR_INVALID_ARG;
    if (!finite_pos(p->step) || !isfinite(p->shift_b) || !isfinite(p->tau_f) || isnan(p->t_near) || isnan(p->t_far))
        return DVGO_ERR_INVALID_ARG;
    if (!isfinite(p->w_pt_rgb) || !isfinite(p->w_bg)) return DVGO_ERR_INVALID_ARG;
    if (p->act_order != DVGO_ACT_POST && p->act_order != DVGO_ACT_PRE && p->act_order != DVGO_ACT_IN)
        return DVGO_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c)
        if (!isfinite(p->bg[c])) return DVGO_ERR_INVALID_ARG;
    if (p->wait_limit_us < 0 || p->wait_limit_us > 60000000 || p->test_withhold_tile < 0) return DVGO_ERR_INVALID_ARG;
    if (p->mode == DVGO_MODE_COARSE) {
        if (cd->channels != 3 || cd->dtype != DVGO_DTYPE_F32) return DVGO_ERR_INVALID_ARG;
        if (p->rgb_act != 0 && p->rgb_act != 1) return DVGO_ERR_INVALID_ARG;
    } else if (p->mode == DVGO_MODE_FINE) {
        if (!mlp || !mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2 || !mlp->w3 || !mlp->b3) return DVGO_ERR_INVALID_ARG;
        if (cd->dtype != DVGO_DTYPE_F32 && cd->dtype != DVGO_DTYPE_BF16) return DVGO_ERR_INVALID_ARG;
        if (p->mlp_prec != DVGO_MLP_FP32 && p->mlp_prec != DVGO_MLP_BF16) return DVGO_ERR_INVALID_ARG;
        if (cd->channels != 12 || p->n_freq_dir != 4 || p->hidden != 128) return DVGO_ERR_UNSUPPORTED;
        if (p->n_freq_pos != 0 && p->n_freq_pos != 5) return DVGO_ERR_UNSUPPORTED;
    } else {
        return DVGO_ERR_INVALID_ARG;
    }
    if (ex) {
        if (!ex->t || !ex->dt || ex->n_per_ray < 1) return DVGO_ERR_INVALID_ARG;
    }
    if (p->freespace && p->freespace->density) {
        const dvgo_freespace &f = *p->freespace;
        if (p->mode != DVGO_MODE_FINE) return DVGO_ERR_INVALID_ARG;
        if (!grid_ok(&f.desc) || f.desc.channels != 1 || f.desc.dtype != DVGO_DTYPE_F32) return DVGO_ERR_INVALID_ARG;
        if (!finite_pos(f.step) || !isfinite(f.shift_b) || !isfinite(f.tau)) return DVGO_ERR_INVALID_ARG;
        // the fixed-point map onto the coarse lattice: its scale must fit kFsScaleBits fractional bits
        for (int a = 0; a < 3; ++a) {
            const int nf[3] = {dd->nx, dd->ny, dd->nz}, nc[3] = {f.desc.nx, f.desc.ny, f.desc.nz};
            const double sf = (nf[a] - 1) / ((double)dd->xyz_max[a] - dd->xyz_min[a]);
            const double sc = (nc[a] - 1) / ((double)f.desc.xyz_max[a] - f.desc.xyz_min[a]);
            if (!(sc / sf < 32768.0)) return DVGO_ERR_UNSUPPORTED;
        }
    }
    if (max_samples(p, dd, R, ex) >= (1LL << 31) - 1) return DVGO_ERR_UNSUPPORTED;
    // the backward keeps one optical-depth value per 32-sample chunk of a ray in shared memory
    if ((ex ? (long long)ex->n_per_ray : sample_cap(p, dd)) > kMaxSamplesPerRay) return DVGO_ERR_UNSUPPORTED;
    return DVGO_OK;
}

RenderArgs make_args(const dvgo_params *p, const dvgo_grid_desc *dd, const float *density,
                     const dvgo_grid_desc *cd, const void *cgrid, const dvgo_mlp *mlp, int R,
                     const dvgo_samples *ex, void *ws, const WsLayout &L) {
    RenderArgs A;
    memset(&A, 0, sizeof(A));
    A.R = R;
    A.mode = p->mode;
    A.rgb_act = p->rgb_act;
    A.mlp_prec = p->mlp_prec;
    A.nfreq = p->n_freq_dir;
    A.hidden = p->hidden;
    A.step = p->step;
    A.shift_b = p->shift_b;
    A.tau_f = p->tau_f;
    for (int c = 0; c < 3; ++c) A.bg[c] = p->bg[c];
    A.nx = dd->nx;
    A.ny = dd->ny;
    A.nz = dd->nz;
    A.C = cd->channels;
    A.cdtype = cd->dtype;
    A.density = density;
    A.cgrid = cgrid;
    if (ex) {
        A.ts = ex->t;
        A.dts = ex->dt;
        A.n_expl = ex->n_per_ray;
    }
    char *b = static_cast<char *>(ws);
    A.hdr = reinterpret_cast<WsHeader *>(b + L.header);
    A.rays = reinterpret_cast<RayRec *>(b + L.rays);
    A.rayout = reinterpret_cast<float4 *>(b + L.rayout);
    A.rtarget = reinterpret_cast<float4 *>(b + L.rtarget);
    A.w_pt = p->w_pt_rgb;
    A.w_bg = p->w_bg;
    A.act_order = p->act_order;
    A.packed = dd->layout == DVGO_LAYOUT_PACKED;
    A.wait_ns = p->wait_limit_us > 0 ? 1000ull * (unsigned long long)p->wait_limit_us : kDefaultWaitNs;
    A.withhold_tile = p->test_withhold_tile;
    if (p->mode == DVGO_MODE_FINE) {
        A.pe = reinterpret_cast<float *>(b + L.pe);
        A.texit = reinterpret_cast<double *>(b + L.texit);
        A.samp = reinterpret_cast<float4 *>(b + L.samp);
        A.sgrad = reinterpret_cast<float4 *>(b + L.sgrad);
        A.kept = reinterpret_cast<int2 *>(b + L.kept);
        A.xcache = L.xcache ? reinterpret_cast<unsigned char *>(b + L.xcache) : nullptr;
    }
    A.max_samples = L.max_samples;
    if (p->mode == DVGO_MODE_FINE && p->freespace && p->freespace->density) {
        const dvgo_freespace &f = *p->freespace;
        A.fs_density = f.density;
        A.fs_nx = f.desc.nx;
        A.fs_ny = f.desc.ny;
        A.fs_nz = f.desc.nz;
        A.fs_shift_b = f.shift_b;
        A.fs_step = f.step;
        A.fs_tau = f.tau;
        A.fs_packed = f.desc.layout == DVGO_LAYOUT_PACKED;
        const int nf[3] = {dd->nx, dd->ny, dd->nz}, nc[3] = {f.desc.nx, f.desc.ny, f.desc.nz};
        for (int a = 0; a < 3; ++a) {
            // u_c = (x - min_c) sc_c with x = min_f + u_f / sf:  u_c = (min_f - min_c) sc_c + u_f sc_c / sf
            const double sf = (nf[a] - 1) / ((double)dd->xyz_max[a] - dd->xyz_min[a]);
            const double sc = (nc[a] - 1) / ((double)f.desc.xyz_max[a] - f.desc.xyz_min[a]);
            A.fs_scale[a] = llrint(sc / sf * 0x1p48);
            A.fs_off[a] = llrint(((double)dd->xyz_min[a] - f.desc.xyz_min[a]) * sc * 0x1p40);
        }
    }
    if (mlp) {
        A.w1 = mlp->w1;
        A.b1 = mlp->b1;
        A.w2 = mlp->w2;
        A.b2 = mlp->b2;
        A.w3 = mlp->w3;
        A.b3 = mlp->b3;
        A.in_dim = cd->channels + 3 + 6 * p->n_freq_dir + (p->n_freq_pos > 0 ? 3 + 6 * p->n_freq_pos : 0);
    }
    if (p->mode == DVGO_MODE_FINE) {
        A.nfreq_pos = p->n_freq_pos;
        const int n[3] = {dd->nx, dd->ny, dd->nz};
        for (int a = 0; a < 3; ++a) {
            A.pos0[a] = dd->xyz_min[a];
            A.posh[a] = (float)(((double)dd->xyz_max[a] - dd->xyz_min[a]) / (n[a] - 1));
        }
    }
    return A;
}

int check_ws(const WsLayout &L, void *ws, size_t bytes) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || bytes < L.total) return DVGO_ERR_WORKSPACE;
    return DVGO_OK;
}

__global__ void sample_counts_kernel(const RayRec *rays, const WsHeader *hdr, int R, int *counts, int *total) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) counts[i] = rays[i].n;
    if (i == 0 && total) *total = hdr->total;
}

int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DVGO_OK : DVGO_ERR_CUDA;
}

}  // namespace
}  // namespace dvgo

using namespace dvgo;

extern "C" {

int dvgo_abi_version(void) { return DVGO_ABI_VERSION; }

const char *dvgo_status_string(int s) {
    switch (s) {
        case DVGO_OK: return "ok";
        case DVGO_ERR_INVALID_ARG: return "invalid argument";
        case DVGO_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case DVGO_ERR_UNSUPPORTED: return "unsupported configuration";
        case DVGO_ERR_CUDA: return "CUDA launch error";
        case DVGO_ERR_DEVICE: return "a ray had a zero or non-finite direction";
        case DVGO_ERR_CAPACITY: return "batch exceeds the static scratch capacity of dvgo_render_fwd_noalloc";
        default: return "unknown status";
    }
}

float dvgo_shift_from_alpha_init(float alpha_init, float voxel_size) {
    return (float)log(pow(1.0 - (double)alpha_init, -1.0 / (double)voxel_size) - 1.0);
}

float dvgo_lr_at(float lr0, int step, float decay_steps) {
    return (float)((double)lr0 * pow(0.1, (double)step / (double)decay_steps));
}

// The BF16 tensor-core colour kernels keep the forward's input panels for the backward (not when
// no backward follows).
static bool xcache_on(const dvgo_params *p) {
    return p->mode == DVGO_MODE_FINE && p->mlp_prec == DVGO_MLP_BF16 && !p->forward_only;
}

size_t dvgo_workspace_size(const dvgo_params *p, const dvgo_grid_desc *density, int n_rays,
                           const dvgo_samples *ex) {
    if (!p || !density || n_rays < 0 || !grid_ok(density) || !(p->step > 0.0f)) return 0;
    long long S = max_samples(p, density, n_rays, ex);
    return ws_layout(n_rays, S, p->mode, xcache_on(p)).total;
}

// The stream waits for the caller's event (if any) before the first kernel that reads cgrid.
static void wait_cgrid(const dvgo_params *p, cudaStream_t s) {
    if (p->cgrid_ready) cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(p->cgrid_ready), 0);
}
// ... and before the first kernel that reads the density grid.
static void wait_density(const dvgo_params *p, cudaStream_t s) {
    if (p->density_ready) cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(p->density_ready), 0);
}

int dvgo_render_fwd(const dvgo_params *p, const dvgo_grid_desc *dd, const float *density, const dvgo_grid_desc *cd,
                    const void *cgrid, const dvgo_mlp *mlp, int R, const float *rays_o, const float *rays_d,
                    const float *jitter, const dvgo_samples *ex, const float *target, float *rgb_out,
                    float *tfinal_out, float *loss_out, float *dloss_out, void *ws, size_t ws_bytes,
                    void *stream) {
    int st = check_common(p, dd, density, cd, cgrid, mlp, R, rays_o, rays_d, ex);
    if (st) return st;
    if (R > 0 && !rgb_out) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsLayout L = ws_layout(R, max_samples(p, dd, R, ex), p->mode, xcache_on(p));
    if ((st = check_ws(L, ws, ws_bytes))) return st;
    if (R == 0) {
        if (loss_out) cudaMemsetAsync(loss_out, 0, sizeof(float), s);
        return launch_status();
    }
    RenderArgs A = make_args(p, dd, density, cd, cgrid, mlp, R, ex, ws, L);
    A.target = target;
    A.rgb_out = rgb_out;
    A.tfinal_out = tfinal_out;
    A.loss_out = target ? loss_out : nullptr;
    A.dloss_out = target ? dloss_out : nullptr;
    launch_ray_setup(A, rays_o, rays_d, jitter, *p, *dd, sample_cap(p, dd), s);
    wait_density(p, s);
    if (p->mode == DVGO_MODE_COARSE) {
        wait_cgrid(p, s);
        launch_coarse_fwd(A, s);
    } else {
        launch_fine_density(A, s);
        wait_cgrid(p, s);
        if (p->mlp_prec == DVGO_MLP_BF16) {
            if ((st = launch_fine_colour_fwd_tc(A, s))) return st;
        } else {
            launch_fine_colour_fwd_simt(A, s);
        }
        launch_fine_composite_fwd(A, s);
    }
    return launch_status();
}

int dvgo_render_bwd(const dvgo_params *p, const dvgo_grid_desc *dd, const float *density, const dvgo_grid_desc *cd,
                    const void *cgrid, const dvgo_mlp *mlp, int R, const float *rays_o, const float *rays_d,
                    const float *jitter, const dvgo_samples *ex, const float *grad_rgb,
                    const float *grad_tfinal, float *grad_density, float *grad_cgrid, float *grad_mlp, void *ws,
                    size_t ws_bytes, void *stream) {
    int st = check_common(p, dd, density, cd, cgrid, mlp, R, rays_o, rays_d, ex);
    if (st) return st;
    if (R > 0 && (!grad_rgb || !grad_density || !grad_cgrid)) return DVGO_ERR_INVALID_ARG;
    if (p->mode == DVGO_MODE_FINE && !grad_mlp) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsLayout L = ws_layout(R, max_samples(p, dd, R, ex), p->mode, xcache_on(p));
    if ((st = check_ws(L, ws, ws_bytes))) return st;
    if (R == 0) return DVGO_OK;
    RenderArgs A = make_args(p, dd, density, cd, cgrid, mlp, R, ex, ws, L);
    A.grad_rgb = grad_rgb;
    A.grad_tfinal = grad_tfinal;
    A.grad_density = grad_density;
    A.grad_cgrid = grad_cgrid;
    A.grad_mlp = grad_mlp;
    wait_density(p, s);
    if (p->mode == DVGO_MODE_COARSE) {
        wait_cgrid(p, s);
        launch_coarse_bwd(A, s);
    } else {
        launch_fine_composite_bwd(A, s);
        wait_cgrid(p, s);
        if (p->mlp_prec == DVGO_MLP_BF16) {
            if ((st = launch_fine_colour_bwd_tc(A, s))) return st;
        } else {
            launch_fine_colour_bwd_simt(A, s);
        }
    }
    return launch_status();
}

static int check_adam(const float *param, const float *grad, const float *m, const float *v, size_t n,
                      const dvgo_adam_hparams *h, const float *lr_scale, const uint16_t *param_bf16_out) {
    if (!h || (n > 0 && (!param || !grad || !m || !v))) return DVGO_ERR_INVALID_ARG;
    if (h->step < 1 || !isfinite(h->lr) || !(h->beta1 >= 0.0f && h->beta1 < 1.0f) ||
        !(h->beta2 >= 0.0f && h->beta2 < 1.0f) || !(h->eps >= 0.0f) || (h->skip_zero_grad & ~1) != 0)
        return DVGO_ERR_INVALID_ARG;
    const void *ptrs[6] = {param, grad, m, v, lr_scale, param_bf16_out};
    for (int i = 0; i < 6; ++i)
        if (ptrs[i] && (reinterpret_cast<uintptr_t>(ptrs[i]) & (i == 5 ? 7u : 15u)) != 0) return DVGO_ERR_INVALID_ARG;
    return DVGO_OK;
}

int dvgo_adam_step(float *param, float *grad, float *m, float *v, size_t n, const dvgo_adam_hparams *h,
                   const float *lr_scale, uint16_t *param_bf16_out, int zero_grad, void *stream) {
    if (int st = check_adam(param, grad, m, v, n, h, lr_scale, param_bf16_out)) return st;
    if (n == 0) return DVGO_OK;
    launch_adam(param, grad, m, v, n, *h, lr_scale, param_bf16_out, zero_grad, static_cast<cudaStream_t>(stream));
    return launch_status();
}

int dvgo_adam_step_multi(const dvgo_adam_tensor *tensors, int n_tensors, void *stream) {
    if (n_tensors < 0 || n_tensors > DVGO_ADAM_MAX_TENSORS || (n_tensors > 0 && !tensors)) return DVGO_ERR_INVALID_ARG;
    dvgo_adam_tensor t[DVGO_ADAM_MAX_TENSORS];
    int nt = 0;
    for (int j = 0; j < n_tensors; ++j) {
        const dvgo_adam_tensor &x = tensors[j];
        if (int st = check_adam(x.param, x.grad, x.m, x.v, x.n, &x.h, x.lr_scale, x.param_bf16_out)) return st;
        if (x.n > 0) t[nt++] = x;
    }
    if (nt == 0) return DVGO_OK;
    launch_adam_multi(t, nt, static_cast<cudaStream_t>(stream));
    return launch_status();
}

int dvgo_sample_counts(const void *ws, int n_rays, int *counts_out, int *total_out, void *stream) {
    if (!ws || n_rays < 0 || (n_rays > 0 && !counts_out)) return DVGO_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return DVGO_ERR_WORKSPACE;
    if (n_rays == 0 && !total_out) return DVGO_OK;
    WsLayout L = ws_layout(n_rays, 0, DVGO_MODE_COARSE);
    const char *b = static_cast<const char *>(ws);
    int blocks = (n_rays + 255) / 256;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ProfScope ps_(DVGO_K_AUX, s);
    sample_counts_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(
        reinterpret_cast<const RayRec *>(b + L.rays), reinterpret_cast<const WsHeader *>(b + L.header), n_rays,
        counts_out, total_out);
    return launch_status();
}

int dvgo_touched_points(const dvgo_params *p, const dvgo_grid_desc *dd, int R, const dvgo_samples *ex, void *ws,
                        size_t ws_bytes, uint32_t *bitmaps, unsigned long long *counts, void *stream) {
    if (!p || !dd || !bitmaps || !counts || R < 0 || p->mode != DVGO_MODE_FINE || !grid_ok(dd) || dd->channels != 1)
        return DVGO_ERR_INVALID_ARG;
    if (!finite_pos(p->step)) return DVGO_ERR_INVALID_ARG;
    if (ex && (!ex->t || !ex->dt || ex->n_per_ray < 1)) return DVGO_ERR_INVALID_ARG;
    if (p->freespace && p->freespace->density && !grid_ok(&p->freespace->desc)) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsLayout L = ws_layout(R, max_samples(p, dd, R, ex), p->mode, xcache_on(p));
    int st = check_ws(L, ws, ws_bytes);
    if (st) return st;
    RenderArgs A = make_args(p, dd, nullptr, dd, nullptr, nullptr, R, ex, ws, L);
    launch_touched(A, bitmaps, counts, s);
    return launch_status();
}

int dvgo_view_counts(const dvgo_grid_desc *g, const dvgo_view_rig *rig, const double *c2w, uint32_t *counts,
                     float *lr_scale, uint32_t *n_max, void *stream) {
    if (!g || !rig || !counts || !n_max || !grid_ok(g) || g->channels != 1 || g->dtype != DVGO_DTYPE_F32)
        return DVGO_ERR_INVALID_ARG;
    if (rig->n_views < 0 || rig->n_views > (1 << 24) || rig->height < 1 || rig->width < 1) return DVGO_ERR_INVALID_ARG;
    if (!(isfinite(rig->fx) && rig->fx > 0.0) || !(isfinite(rig->fy) && rig->fy > 0.0) || !isfinite(rig->cx) ||
        !isfinite(rig->cy) || !(isfinite(rig->near) && rig->near >= 0.0))
        return DVGO_ERR_INVALID_ARG;
    if (rig->n_views > 0 && (!c2w || reinterpret_cast<uintptr_t>(c2w) % 8)) return DVGO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(counts) % 4 || reinterpret_cast<uintptr_t>(lr_scale) % 4 ||
        reinterpret_cast<uintptr_t>(n_max) % 4)
        return DVGO_ERR_INVALID_ARG;
    launch_view_counts(*g, *rig, c2w, counts, lr_scale, n_max, static_cast<cudaStream_t>(stream));
    return launch_status();
}

int dvgo_workspace_status(void *ws, void *stream) {
    if (!ws) return DVGO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int flags = 0;
    WsHeader *h = static_cast<WsHeader *>(ws);
    if (cudaMemcpyAsync(&flags, &h->flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return DVGO_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DVGO_ERR_CUDA;
    return flags ? DVGO_ERR_DEVICE : DVGO_OK;
}

}  // extern "C"
