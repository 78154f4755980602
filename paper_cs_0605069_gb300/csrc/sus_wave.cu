// Launchers of the multi-team SUS kernel (device code in sus_wave.cuh).
#include "sus_wave.cuh"

namespace gfbp {

namespace {

template <int Q, int DC, int W>
cudaError_t launch_wave_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int threads = W * WaveLay<Q>::TEAM;
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_wave<Q, DC, W>, threads, 0, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_wave<Q, DC, W><<<(int)grid, threads, 0, s>>>(A);
    return cudaGetLastError();
}

template <int Q, int W>
cudaError_t launch_wave_dc(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    return A.c.dcmax <= 6 ? launch_wave_q<Q, 6, W>(A, num_sms, s) : launch_wave_q<Q, 8, W>(A, num_sms, s);
}

template <int W>
cudaError_t launch_wave_w(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 4: return launch_wave_dc<4, W>(A, num_sms, s);
    case 8: return launch_wave_dc<8, W>(A, num_sms, s);
    case 16: return launch_wave_dc<16, W>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sus_wave(const DecodeArgs& A, int width, int num_sms, cudaStream_t s) {
    switch (width) {
    case 2: return launch_wave_w<2>(A, num_sms, s);
    case 4: return launch_wave_w<4>(A, num_sms, s);
    case 8: return launch_wave_w<8>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
