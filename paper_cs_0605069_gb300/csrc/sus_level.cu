// Launchers of the level-scheduled SUS kernel (device code in sus_level.cuh).
#include "sus_level.cuh"

namespace gfbp {

namespace {

template <int Q, int T, bool RUN>
cudaError_t launch_level_qr(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_level<Q, 8, T, RUN>, T, 0, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_level<Q, 8, T, RUN><<<(int)grid, T, 0, s>>>(A);
    return cudaGetLastError();
}

template <int Q, int T>
cudaError_t launch_level_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    return A.sfx ? launch_level_qr<Q, T, true>(A, num_sms, s) : launch_level_qr<Q, T, false>(A, num_sms, s);
}

// Threads per frame: about the mean number of pairs in a piece, halved when
// the frames fill the SMs many times over (twice the frames resident per SM,
// each thread taking up to two pairs of a piece in turn).
template <int Q>
cudaError_t launch_level_t(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    const long long per_piece = A.c.npieces > 0 ? A.c.E / A.c.npieces : 0;
    const bool many = (long long)A.F >= 16LL * num_sms;
    if (per_piece <= 32) return launch_level_q<Q, 32>(A, num_sms, s);
    if (per_piece <= 64 || many) return launch_level_q<Q, 64>(A, num_sms, s);
    return launch_level_q<Q, 128>(A, num_sms, s);
}

}  // namespace

bool sus_level_eligible(const DecodeArgs& A) {
    return A.method == kDirect && A.c.q <= 16;
}

cudaError_t launch_sus_level(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_level_t<2>(A, num_sms, s);
    case 4: return launch_level_t<4>(A, num_sms, s);
    case 8: return launch_level_t<8>(A, num_sms, s);
    case 16: return launch_level_t<16>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
