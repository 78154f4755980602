// Launchers of the frame-resident kernels (device code in resident.cuh).
#include "resident.cuh"

namespace gfbp {

namespace {

// Static shared memory beside the dynamic part (tables, frame index), with a margin.
template <int Q>
constexpr size_t res_static_bytes() { return 2 * Q * Q + 64; }

template <int Q>
size_t res_bytes(const CodeDev& c, bool sus) {
    return sus ? res_sus_parts<Q, true>(c.E, c.M, c.N, c.npieces).total : res_parts<Q, false>(c.E, c.M, c.N, 0).total;
}

size_t res_bytes_q(const CodeDev& c, bool sus) {
    switch (c.q) {
    case 2: return res_bytes<2>(c, sus);
    case 4: return res_bytes<4>(c, sus);
    case 8: return res_bytes<8>(c, sus);
    case 16: return res_bytes<16>(c, sus);
    }
    return 0;
}

// The frame's shared memory must fit one CTA, and (PUS) every slot offset
// must fit the 16-bit column-slot table.
bool res_fits(const CodeDev& c, bool sus) {
    const size_t stat = 2 * (size_t)c.q * c.q + 64;
    if (c.q > 16) return false;
    const size_t pad = c.q >= 4 ? 4 : 2;
    if (!sus && ((size_t)c.E * c.q + pad * c.M) / pad > 65535) return false;
    return res_bytes_q(c, sus) + stat <= (size_t)device_optin_smem();
}

template <typename K>
cudaError_t launch_persistent(K kernel, const DecodeArgs& A, int threads, size_t smem, int num_sms, cudaStream_t s) {
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)kernel, threads, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long long cap = (long long)num_sms * occ;
    const long long grid = A.F < cap ? A.F : cap;
    if (grid < 1) return cudaSuccess;
    kernel<<<(int)grid, threads, smem, s>>>(A);
    return cudaGetLastError();
}

// PUS: the horizontal pass has M checks and the vertical one N columns of
// work per iteration; a CTA of up to 256 threads (a thread may then take
// several checks or columns), fewer for small codes so that their frames share
// an SM.
template <int Q>
cudaError_t launch_pus_res_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    const size_t smem = res_bytes<Q>(A.c, false);
    const int work = A.c.M > A.c.N ? A.c.M : A.c.N;
    if (work <= 64) return launch_persistent(k_pus_res<Q, 64, 6, 4>, A, 64, smem, num_sms, s);
    if (work <= 128) return launch_persistent(k_pus_res<Q, 128, 6, 4>, A, 128, smem, num_sms, s);
    return launch_persistent(k_pus_res<Q, 256, 6, 4>, A, 256, smem, num_sms, s);
}

// SUS with the slab in shared memory: a thread per (column, check) pair of a
// piece, one frame per CTA.
template <int Q>
cudaError_t launch_sus_res_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    const size_t smem = res_bytes<Q>(A.c, true);
    return launch_persistent(k_sus_res<Q, true>, A, kLevelPiece, smem, num_sms, s);
}

// L2 budget (bytes) for the slabs of the CTAs decoding at once: 75% of the L2,
// the rest left to likelihoods, code arrays and outputs streaming through.
size_t l2_slab_budget() {
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    return (size_t)(l2 > 0 ? l2 : 50 << 20) * 3 / 4;
}

// SUS with each CTA's slab in the workspace: as many CTAs per SM as keep all
// their slabs within the L2 budget (at least one, at most the occupancy).
template <int Q>
cudaError_t launch_sus_l2_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    const size_t smem = res_sus_parts<Q, false>(A.c.E, A.c.M, A.c.N, A.c.npieces).total;
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_res<Q, false>, kLevelPiece, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const size_t slab = sizeof(float) * (size_t)A.c.E * Q;
    long long per_sm = slab ? (long long)(l2_slab_budget() / ((size_t)num_sms * slab)) : occ;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > occ) per_sm = occ;
    const long long cap = (long long)num_sms * per_sm;
    const long long grid = A.F < cap ? A.F : cap;   // <= F: the slabs fit the F E q message region
    if (grid < 1) return cudaSuccess;
    k_sus_res<Q, false><<<(int)grid, kLevelPiece, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

// The resident kernels run the probability route (q <= 16), whole decodes in
// one launch (not the resumable rounds of serving), with the frame's slab in
// shared memory; PUS keeps a check's inner messages in registers (row degree
// <= 6, column degree <= 4).
bool pus_res_eligible(const DecodeArgs& A) {
    if (A.method != kDirect || A.c.q > 16 || A.fstate) return false;
    if (A.layout != GFBP_LAYOUT_AUTO && A.layout != GFBP_LAYOUT_RESIDENT) return false;
    if (A.c.dcmax > 6 || A.c.dvmax > 4) return false;
    return res_fits(A.c, false);
}

// AUTO takes the shared-memory kernel up to 4 frames per SM (GF(16), N = 1000,
// 20 iterations: 152 frames 1.49 ms against 2.41 ms for the folding level
// kernel, 456 frames 3.40 against 4.00 ms); with more frames per SM the
// folding level kernel, whose many resident frames hide each other's latency,
// is faster (4096 frames: 19.6 against 24.5 ms).
bool sus_res_eligible(const DecodeArgs& A, int num_sms) {
    if (A.method != kDirect || A.c.q > 16 || A.fstate || A.markov_gs) return false;
    if (A.partials != GFBP_PARTIALS_AUTO && A.partials != GFBP_PARTIALS_RUNNING) return false;
    const bool want = A.layout == GFBP_LAYOUT_RESIDENT ||
                      (A.layout == GFBP_LAYOUT_AUTO && A.partials == GFBP_PARTIALS_AUTO &&
                       (long long)A.F <= 4LL * num_sms);
    return want && res_fits(A.c, true);
}

// The L2-resident SUS kernel: the arithmetic of the shared-memory one (the
// same bits), any code size (q <= 16); asked for explicitly.
bool sus_l2_eligible(const DecodeArgs& A) {
    if (A.method != kDirect || A.c.q > 16 || A.fstate || A.markov_gs) return false;
    if (A.layout != GFBP_LAYOUT_L2RESIDENT) return false;
    return A.partials == GFBP_PARTIALS_AUTO || A.partials == GFBP_PARTIALS_RUNNING;
}

cudaError_t launch_pus_res(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_pus_res_q<2>(A, num_sms, s);
    case 4: return launch_pus_res_q<4>(A, num_sms, s);
    case 8: return launch_pus_res_q<8>(A, num_sms, s);
    case 16: return launch_pus_res_q<16>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sus_l2(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_sus_l2_q<2>(A, num_sms, s);
    case 4: return launch_sus_l2_q<4>(A, num_sms, s);
    case 8: return launch_sus_l2_q<8>(A, num_sms, s);
    case 16: return launch_sus_l2_q<16>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sus_res(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_sus_res_q<2>(A, num_sms, s);
    case 4: return launch_sus_res_q<4>(A, num_sms, s);
    case 8: return launch_sus_res_q<8>(A, num_sms, s);
    case 16: return launch_sus_res_q<16>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
