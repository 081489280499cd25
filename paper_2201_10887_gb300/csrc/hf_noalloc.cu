// Allocation-free discretization entry point (see hf_discretize_noalloc in
// include/hf.h).  It runs the same visible-row and discretization kernels as
// hf_discretize_cascades, but their scratch (visible-row spans and texel
// coordinates) lives in the fixed array below instead of a caller buffer.
#include <mutex>

#include "hf_internal.h"

namespace {

// Scratch of the allocation-free path: per cascade N int2 spans, then N FP32
// x and N FP32 y texel coordinates, 16 bytes per texture row.  Every device
// that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current) and cached.
int scratch_on_current_device(char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hfi::set_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return hfi::set_cuda_error(cudaErrorInvalidDevice, "device index");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return hfi::set_cuda_error(e, "cudaGetSymbolAddress of the built-in scratch");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<char*>(g_scratch_ptr[dev]);
    return HF_OK;
}

}  // namespace

extern "C" int hf_discretize_noalloc(hf_ctx* ctx, const hf_camera* cam, float* const* tex_out,
                                     hf_cascade_info* info_out, void* stream) {
    return hfi::guarded("hf_discretize_noalloc", [&]() -> int {
        char* scratch = nullptr;
        int rc = scratch_on_current_device(&scratch);
        if (rc != HF_OK) return rc;
        hfi::PrepParams pp;
        hfi::DiscParams dp;
        hfi::LookupTables lt;
        hfi::ListsView lv;
        hfi::CompactView cv{};
        bool compact = false;
        hfi::DevStatus* status = nullptr;
        rc = hfi::noalloc_discretize_params(ctx, cam, tex_out, scratch, HF_NOALLOC_SCRATCH_BYTES, info_out,
                                            &pp, &dp, &lt, &lv, &cv, &compact, &status);
        if (rc != HF_OK) return rc;
        // every span and coordinate read below is written first on the same
        // stream, so nothing in the scratch needs clearing between calls
        int e = hfi::launch_prep(pp, stream);
        if (e != cudaSuccess) return hfi::set_cuda_error(e, "visible-row kernel launch (allocation-free path)");
        e = compact ? hfi::launch_discretize_f32c(dp, lt, cv, status, stream)
                    : hfi::launch_discretize(dp, lt, lv, status, stream);
        if (e != cudaSuccess) return hfi::set_cuda_error(e, "discretization kernel launch (allocation-free path)");
        return HF_OK;
    });
}
