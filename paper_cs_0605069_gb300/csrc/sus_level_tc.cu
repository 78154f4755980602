// Launchers of the tensor-core SUS level kernel (device code in sus_level_tc.cuh).
#include "sus_level_tc.cuh"

namespace gfbp {

namespace {

constexpr int kLevelTcThreads = 256;

template <int Q>
cudaError_t launch_level_tc_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int T = kLevelTcThreads;
    constexpr size_t smem = TcLay<Q, T>::total;
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_level_tc<Q, T>, T, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_level_tc<Q, T><<<(int)grid, T, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sus_level_tc(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 16: return launch_level_tc_q<16>(A, num_sms, s);
    case 32: return launch_level_tc_q<32>(A, num_sms, s);
    case 64: return launch_level_tc_q<64>(A, num_sms, s);
    case 128: return launch_level_tc_q<128>(A, num_sms, s);
    case 256: return launch_level_tc_q<256>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
