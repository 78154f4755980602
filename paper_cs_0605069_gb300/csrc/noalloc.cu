// gfbp_decode_noalloc: gfbp_decode for callers that must not allocate device
// memory.  Its scratch is one file-scope __device__ array, so the library
// never calls cudaMalloc/cudaFree (or any allocating routine) on this path.
#include <mutex>
#include <string>

#include "gfbp_internal.cuh"

namespace gfbp {
void set_error(const std::string& msg);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

// Reserved on every device that loads the library, until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[256] = {};  // device address of g_static_scratch, per device

}  // namespace

extern "C" gfbp_status gfbp_decode_noalloc(const gfbp_code* code, int32_t n_frames, const float* obs,
                                           gfbp_channel channel, gfbp_schedule schedule, const gfbp_prior* prior,
                                           int32_t max_iter, uint8_t* x_hat, int32_t* iters, uint8_t* converged,
                                           const gfbp_options* options, void* stream) {
    if (!code) {
        gfbp::set_error("gfbp_decode_noalloc: NULL code");
        return GFBP_EINVAL;
    }
    if (options && options->sus_partials == GFBP_PARTIALS_RUNNING_GLOBAL) {
        gfbp::set_error("gfbp_decode_noalloc: sus_partials RUNNING_GLOBAL allocates device memory");
        return GFBP_EINVAL;
    }
    size_t need = 0;
    gfbp_status st = gfbp_workspace_size(code, n_frames, schedule, prior, 0, &need);
    if (st != GFBP_OK) return st;
    if (need > kStaticScratchBytes) {
        gfbp::set_error("gfbp_decode_noalloc: " + std::to_string(n_frames) + " frames need " + std::to_string(need) +
                        " bytes of scratch, more than the static " + std::to_string(kStaticScratchBytes) +
                        "-byte buffer; decode fewer frames per call");
        return GFBP_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        gfbp::set_error(std::string("gfbp_decode_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    void* base = nullptr;
    {
        // First call on this device (with it current): look up the array's
        // device address.  The host-side name is not a device pointer.
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) {
                gfbp::set_error(std::string("gfbp_decode_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return GFBP_ECUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    // Every scratch region gfbp_decode uses is written before it is read, and
    // its frame counter is cleared with cudaMemsetAsync on `stream`, so the
    // previous call's contents do no harm.
    gfbp_options o{};
    if (options) o = *options;
    o.workspace = base;
    o.workspace_bytes = kStaticScratchBytes;
    return gfbp_decode(code, n_frames, obs, channel, schedule, prior, max_iter, x_hat, iters, converged, &o, stream);
}
