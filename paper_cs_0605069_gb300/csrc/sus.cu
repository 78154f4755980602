// Launchers of the generic SUS kernels (device code in sus_group.cuh).
#include "sus_group.cuh"

namespace gfbp {

namespace {

template <int Q, int DC, int DV, int METHOD>
cudaError_t launch_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int G = Lay<Q>::G;
    constexpr int groups_per_block = kSusThreads / G;
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus<Q, DC, DV, METHOD>, kSusThreads, 0, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    long long want = ((long long)A.F + groups_per_block - 1) / groups_per_block;
    long long cap = (long long)num_sms * occ;
    long long grid = want < cap ? want : cap;
    if (grid < 1) return cudaSuccess;
    k_sus<Q, DC, DV, METHOD><<<(int)grid, kSusThreads, 0, s>>>(A);
    return cudaGetLastError();
}

template <int Q, int METHOD>
cudaError_t launch_deg(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (A.c.dcmax <= 6 && A.c.dvmax <= 3) return launch_q<Q, 6, 3, METHOD>(A, num_sms, s);
    return launch_q<Q, 16, 8, METHOD>(A, num_sms, s);
}

template <int Q>
cudaError_t launch_method(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if constexpr (Q <= 16) {
        if (A.method == kDirect) return launch_deg<Q, kDirect>(A, num_sms, s);
    }
    return launch_deg<Q, kTransform>(A, num_sms, s);
}

template <int Q>
cudaError_t launch_init_q(const DecodeArgs& A, cudaStream_t s) {
    constexpr int G = Lay<Q>::G;
    const long long total = (long long)A.F * A.c.E;
    long long blocks = (total + (256 / G) - 1) / (256 / G);
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (blocks < 1) return cudaSuccess;
    if (A.method == kDirect) {
        k_init_dev<Q, kDirect><<<(unsigned)blocks, 256, 0, s>>>(A);
        return cudaGetLastError();
    }
    if constexpr (Q >= 16) {
        if (A.method == kTensor) {
            k_init_dev<Q, kTensor><<<(unsigned)blocks, 256, 0, s>>>(A);
            return cudaGetLastError();
        }
    }
    k_init_dev<Q, kTransform><<<(unsigned)blocks, 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

// The column-walking group kernel for every q (the Gauss-Seidel prior chains
// the sweep through the source symbols).
cudaError_t launch_sus_group(const DecodeArgs& A, int num_sms, cudaStream_t s) {
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

cudaError_t launch_sus(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (A.method == kTensor) return launch_sus_level_tc(A, num_sms, s);
    if (A.markov_gs) return launch_sus_group(A, num_sms, s);
    if (sus_res_eligible(A, num_sms)) return launch_sus_res(A, num_sms, s);
    if (sus_l2_eligible(A)) return launch_sus_l2(A, num_sms, s);
    // the probability route for q >= 32 runs by levels with a lane group per
    // pair whatever the layout (no column-walking kernel carries it)
    if (A.method == kDirect && A.c.q > 16) return launch_sus_level_tr(A, num_sms, s);
    if (A.layout != GFBP_LAYOUT_LANES) {
        if (sus_level_sm_eligible(A, num_sms)) return launch_sus_level_sm(A, num_sms, s);
        if (sus_level_eligible(A)) return launch_sus_level(A, num_sms, s);
        if (A.method == kTransform) return launch_sus_level_tr(A, num_sms, s);
    }
    if (sus_team_eligible(A)) {
        const int w = A.width ? A.width : sus_auto_width(A, num_sms);
        return w > 1 ? launch_sus_wave(A, w, num_sms, s) : launch_sus_team(A, num_sms, s);
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

cudaError_t launch_init_dev(const DecodeArgs& A, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_init_q<2>(A, s);
    case 4: return launch_init_q<4>(A, s);
    case 8: return launch_init_q<8>(A, s);
    case 16: return launch_init_q<16>(A, s);
    case 32: return launch_init_q<32>(A, s);
    case 64: return launch_init_q<64>(A, s);
    case 128: return launch_init_q<128>(A, s);
    case 256: return launch_init_q<256>(A, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
