// Launchers of the level-scheduled SUS kernel with the running partial
// convolutions in shared memory (device code in sus_level_sm.cuh).
#include "sus_level_sm.cuh"

namespace gfbp {

namespace {

int optin_smem() { return device_optin_smem(); }

// Static shared memory of the kernel besides the dynamic part (tables, frame
// index) with a margin.
template <int Q>
constexpr size_t sm_static_bytes() { return 2 * Q * Q + 64; }

template <int Q>
cudaError_t launch_sm_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int T = SmLay<Q>::T;
    const size_t bytes = level_sm_bytes<Q>(A.c);
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_level_sm<Q>, T, bytes, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_level_sm<Q><<<(int)grid, T, bytes, s>>>(A);
    return cudaGetLastError();
}

template <int Q>
bool fits(const DecodeArgs& A) {
    return level_sm_bytes<Q>(A.c) + sm_static_bytes<Q>() <= (size_t)optin_smem();
}

}  // namespace

// RUNNING asks for it; AUTO takes it for at most one frame per SM, where a
// frame's latency sets the decode time (GF(16), N = 1000, 20 iterations: 152
// frames 1.78 ms against 2.39 ms with the folding kernel; from 304 frames on
// the folding kernel, with several frames resident per SM, is faster: 3.21
// against 3.56 ms, and 28.4 against 48.0 ms for 4096 frames).
bool sus_level_sm_eligible(const DecodeArgs& A, int num_sms) {
    if (A.method != kDirect) return false;
    const bool want = A.partials == GFBP_PARTIALS_RUNNING ||
                      (A.partials == GFBP_PARTIALS_AUTO && A.layout == GFBP_LAYOUT_THREAD &&
                       (long long)A.F <= (long long)num_sms);
    if (!want) return false;
    switch (A.c.q) {
    case 2: return fits<2>(A);
    case 4: return fits<4>(A);
    case 8: return fits<8>(A);
    case 16: return fits<16>(A);
    }
    return false;
}

cudaError_t launch_sus_level_sm(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_sm_q<2>(A, num_sms, s);
    case 4: return launch_sm_q<4>(A, num_sms, s);
    case 8: return launch_sm_q<8>(A, num_sms, s);
    case 16: return launch_sm_q<16>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
