// Launchers of the PUS kernels (device code in pus_frame.cuh and pus_regs.cuh).
#include "pus_regs.cuh"

namespace gfbp {

namespace {

template <int Q, int DC, int DV, int METHOD, bool BULK>
cudaError_t launch_qb(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int G = Lay<Q>::G;
    constexpr size_t smem = sizeof(float) * (size_t)(kPusThreads / G) * pus_group_scratch<Q, DC, METHOD, BULK>();
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_pus<Q, DC, DV, METHOD, BULK>, kPusThreads, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    long long grid = (long long)num_sms * occ;
    if (grid > A.F) grid = A.F;
    if (grid < 1) return cudaSuccess;
    k_pus<Q, DC, DV, METHOD, BULK><<<(int)grid, kPusThreads, smem, s>>>(A);
    return cudaGetLastError();
}

// The bulk-staged kernel hides the latency of a check's loads behind the
// previous check (GF(16) N = 1000, 1024 frames: 36.7 ms against 40.0 ms) but
// its second buffer costs a CTA per SM, which loses once the frames fill the
// GPU (4096 frames: 132 ms against 122 ms): it runs for at most 8 frames per SM.
template <int Q, int DC, int DV, int METHOD>
cudaError_t launch_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if constexpr (pus_bulk_ok<Q, METHOD>()) {
        if ((long long)A.F <= 8LL * num_sms) return launch_qb<Q, DC, DV, METHOD, true>(A, num_sms, s);
    }
    return launch_qb<Q, DC, DV, METHOD, false>(A, num_sms, s);
}

template <int Q, int METHOD>
cudaError_t launch_deg(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (A.c.dcmax <= 6 && A.c.dvmax <= 3) return launch_q<Q, 6, 3, METHOD>(A, num_sms, s);
    return launch_q<Q, 16, 8, METHOD>(A, num_sms, s);
}

template <int Q>
cudaError_t launch_method(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (A.method == kDirect) return launch_deg<Q, kDirect>(A, num_sms, s);
    return launch_deg<Q, kTransform>(A, num_sms, s);
}

constexpr int kPusRegsThreads = 128;

template <int Q, int T>
cudaError_t launch_regs_qt(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    const size_t smem = sizeof(float) * (size_t)(pus_regs_rows(A.c.dcmax, A.c.dvmax) + 1) * T * (Q + 1);
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_pus_regs<Q, T>, T, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    long long grid = (long long)num_sms * occ;
    if (grid > A.F) grid = A.F;
    if (grid < 1) return cudaSuccess;
    k_pus_regs<Q, T><<<(int)grid, T, smem, s>>>(A);
    return cudaGetLastError();
}

// 128 threads per frame: at 4096 frames of GF(16), N = 1000, 64 threads per
// frame (twice the frames resident) ran 4% slower.
template <int Q>
cudaError_t launch_regs_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    return launch_regs_qt<Q, kPusRegsThreads>(A, num_sms, s);
}

}  // namespace

bool pus_regs_eligible(const DecodeArgs& A) {
    return A.method == kDirect && A.c.q <= 16;
}

// AUTO takes the thread layout wherever it applies (q <= 16, probability
// route), 20 iterations: GF(16), N = 1000, 4096 frames 22.5 ms against 25.1 ms
// for the lane kernel; GF(8), N = 2000 with a Markov prior, 2048 frames 13.7
// against 16.8; GF(4), N = 96, 8192 frames 0.93 against 2.66.
cudaError_t launch_pus(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (pus_res_eligible(A)) return launch_pus_res(A, num_sms, s);
    const bool thread = A.layout != GFBP_LAYOUT_LANES;
    if (thread && pus_regs_eligible(A)) {
        switch (A.c.q) {
        case 2: return launch_regs_q<2>(A, num_sms, s);
        case 4: return launch_regs_q<4>(A, num_sms, s);
        case 8: return launch_regs_q<8>(A, num_sms, s);
        case 16: return launch_regs_q<16>(A, num_sms, s);
        }
    }
    switch (A.c.q) {
    case 2: return launch_method<2>(A, num_sms, s);
    case 4: return launch_method<4>(A, num_sms, s);
    case 8: return launch_method<8>(A, num_sms, s);
    case 16: return launch_method<16>(A, num_sms, s);
    case 32: return launch_method<32>(A, num_sms, s);
    case 64: return launch_method<64>(A, num_sms, s);
    case 128: return launch_method<128>(A, num_sms, s);
    case 256: return launch_method<256>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
