// Launchers of the level-scheduled transform-route SUS kernel (device code in
// sus_level_tr.cuh).
#include "sus_level_tr.cuh"

namespace gfbp {

namespace {

constexpr int kLevelTrThreads = 256;

template <int Q, int T, int METHOD>
cudaError_t launch_level_tr_qmt(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr size_t smem = level_tr_smem<Q, T>();
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_level_tr<Q, T, METHOD>, T, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_level_tr<Q, T, METHOD><<<(int)grid, T, smem, s>>>(A);
    return cudaGetLastError();
}

// 256 threads per frame; with no more frames than SMs (each frame has an SM to
// itself) 512 for q >= 32, twice the lane groups on every level's pairs: the
// same results (each pair's arithmetic does not depend on which group runs
// it), sooner.
template <int Q, int METHOD>
cudaError_t launch_level_tr_qm(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if constexpr (Q >= 32) {
        if (A.F <= num_sms) return launch_level_tr_qmt<Q, 512, METHOD>(A, num_sms, s);
    }
    return launch_level_tr_qmt<Q, kLevelTrThreads, METHOD>(A, num_sms, s);
}

// The probability route by lane groups is instantiated for q >= 32 (below, the
// register kernels of sus_level.cuh and resident.cuh run it).
template <int Q>
cudaError_t launch_level_tr_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if constexpr (Q >= 32) {
        if (A.method == kDirect) return launch_level_tr_qm<Q, kDirect>(A, num_sms, s);
    }
    return launch_level_tr_qm<Q, kTransform>(A, num_sms, s);
}

}  // namespace

cudaError_t launch_sus_level_tr(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_level_tr_q<2>(A, num_sms, s);
    case 4: return launch_level_tr_q<4>(A, num_sms, s);
    case 8: return launch_level_tr_q<8>(A, num_sms, s);
    case 16: return launch_level_tr_q<16>(A, num_sms, s);
    case 32: return launch_level_tr_q<32>(A, num_sms, s);
    case 64: return launch_level_tr_q<64>(A, num_sms, s);
    case 128: return launch_level_tr_q<128>(A, num_sms, s);
    case 256: return launch_level_tr_q<256>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
