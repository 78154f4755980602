// gfbp_wait_selftest: the bounded device waits of the decoder kernels, run on
// a condition that never comes true, so that a caller can check that each
// wait gives up within its bound, reports it, and leaves the context usable
// (the failure path that the kernels take, without faulting or hanging).
//   which 0: the mbarrier wait of the bulk copies (bulk.cuh): a barrier that
//            expects one arrival, none made;
//   which 1: the watermark wait of the multi-team SUS kernel (sus_wave.cuh):
//            a progress word that never passes the awaited column.
#include <string>

#include "bulk.cuh"
#include "gfbp_internal.cuh"
#include "sus_wave.cuh"

namespace gfbp {
void set_error(const std::string& msg);

namespace {

__global__ void k_wait_probe(int which, int* done) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int prog[1];
    if (threadIdx.x != 0) return;
    int ok = 0;
    if (which == 0) {
        mbar_init(&bar);
        mbar_init_fence();
        ok = mbar_wait(&bar, 0) ? 1 : 0;   // phase 0 never completes
    } else {
        prog[0] = 0;
        ok = wave_wait<1>(prog, 0) ? 1 : 0;   // the watermark stays at column 0
    }
    *done = ok;
}

}  // namespace
}  // namespace gfbp

using namespace gfbp;

extern "C" gfbp_status gfbp_wait_selftest(int32_t which, int32_t* completed, void* stream) {
    if ((which != 0 && which != 1) || !completed) {
        set_error("gfbp_wait_selftest: which must be 0 or 1 and completed a host pointer");
        return GFBP_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, sizeof(int), s);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_wait_selftest: ") + cudaGetErrorString(e));
        return GFBP_ENOMEM;
    }
    k_wait_probe<<<1, 32, 0, s>>>(which, d);
    e = cudaGetLastError();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_wait_selftest: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    *completed = h;
    if (!h) {
        set_error(which == 0 ? "gfbp_wait_selftest: the mbarrier wait ran out (as it must: nothing arrives)"
                             : "gfbp_wait_selftest: the watermark wait ran out (as it must: no column finishes)");
        return GFBP_ETIMEOUT;
    }
    return GFBP_OK;
}
