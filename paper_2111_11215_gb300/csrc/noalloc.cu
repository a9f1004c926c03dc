// noalloc.cu -- coarse-stage forward render whose scratch memory is a static device array.
//
// For callers that cannot allocate device memory at all (they cannot call cudaMalloc or any
// allocator, so they cannot provide the workspace dvgo_render_fwd needs): a plugin inside a host
// application whose memory manager owns the whole device, a real-time loop that forbids
// allocation after start-up, or a language binding with no device allocator.  The paper has no
// counterpart; this is a deployment convenience of the library.
//
// The scratch is one file-scope __device__ array of kNoallocScratchBytes, which every GPU that
// loads the library holds until the process exits.  Host code cannot use the array's name as a
// device address (it is a host-side stand-in), so the first call on each device looks the address
// up with cudaGetSymbolAddress, with that device current, and caches it; that first call should
// therefore happen before any stream capture.  The render itself is the existing coarse forward
// path (dvgo_render_fwd) pointed at the static array.

#include <mutex>

#include "dvgo_internal.cuh"

namespace dvgo {

namespace {

// Workspace of a coarse forward of up to DVGO_NOALLOC_MAX_RAYS rays, block for block as ws_layout()
// lays it out (each block 256-byte aligned): header, per-ray records, per-ray outputs and the
// per-ray target block.  This forward never writes the target block (it rejects the auxiliary
// losses), but the workspace check counts it, so the array holds it too.
constexpr size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNoallocScratchBytes = up256(sizeof(WsHeader)) + up256(sizeof(RayRec) * DVGO_NOALLOC_MAX_RAYS) +
                                        up256(sizeof(float4) * DVGO_NOALLOC_MAX_RAYS) +
                                        up256(sizeof(float4) * DVGO_NOALLOC_MAX_RAYS);
static_assert(kNoallocScratchBytes == DVGO_NOALLOC_SCRATCH_BYTES, "scratch size in dvgo.h");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the static scratch on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DVGO_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DVGO_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return DVGO_OK;
}

}  // namespace
}  // namespace dvgo

extern "C" int dvgo_render_fwd_noalloc(const dvgo_params *p, const dvgo_grid_desc *density_desc,
                                       const float *density, const dvgo_grid_desc *cgrid_desc, const void *cgrid,
                                       int n_rays, const float *rays_o, const float *rays_d, const float *jitter,
                                       const float *target, float *rgb_out, float *tfinal_out, float *loss_out,
                                       float *dloss_drgb_out, void *stream) {
    if (!p || p->mode != DVGO_MODE_COARSE) return DVGO_ERR_UNSUPPORTED;
    if (p->w_pt_rgb != 0.0f || p->w_bg != 0.0f) return DVGO_ERR_UNSUPPORTED;   // no room for the targets
    if (n_rays > DVGO_NOALLOC_MAX_RAYS) return DVGO_ERR_CAPACITY;
    if (dvgo::ws_layout(n_rays, 0, DVGO_MODE_COARSE).total > dvgo::kNoallocScratchBytes) return DVGO_ERR_CAPACITY;
    void *scratch = nullptr;
    int st = dvgo::scratch_address(&scratch);
    if (st != DVGO_OK) return st;
    return dvgo_render_fwd(p, density_desc, density, cgrid_desc, cgrid, nullptr, n_rays, rays_o, rays_d, jitter,
                           nullptr, target, rgb_out, tfinal_out, loss_out, dloss_drgb_out, scratch,
                           dvgo::kNoallocScratchBytes, stream);
}
