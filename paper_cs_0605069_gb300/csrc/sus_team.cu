// Launchers of the team SUS kernel (device code in sus_team.cuh).
#include "sus_team.cuh"

namespace gfbp {

namespace {

template <int Q, int DC>
cudaError_t launch_team_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int teams_per_block = kTeamThreads / TeamLay<Q>::TEAM;
    int occ = 0;
    cudaError_t e = kernel_prepare((const void*)k_sus_team<Q, DC>, kTeamThreads, 0, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    long long want = ((long long)A.F + teams_per_block - 1) / teams_per_block;
    long long cap = (long long)num_sms * occ;
    long long grid = want < cap ? want : cap;
    if (grid < 1) return cudaSuccess;
    k_sus_team<Q, DC><<<(int)grid, kTeamThreads, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

bool sus_team_eligible(const DecodeArgs& A) {
    return A.method == kDirect && A.c.q <= 16 && A.c.q >= 4 && A.c.dvmax <= kSlots && A.c.dcmax <= 8;
}

// Teams per frame when the caller leaves it open.  A frame's sweep is a chain
// of N dependent column updates, and frames that do not converge run max_iter
// sweeps: with few frames per SM the decode time is that chain's latency, which
// more teams per frame cut (GF(16), N = 1000: 1024 frames 489 ms with one team,
// 106 ms with eight; 4096 frames 652 ms and 382 ms).  Only when the frames fill
// the SMs many times over does one team per frame avoid the waits at no cost.
int sus_auto_width(const DecodeArgs& A, int num_sms) {
    const long long frames_per_sm = ((long long)A.F + num_sms - 1) / (num_sms > 0 ? num_sms : 1);
    if (frames_per_sm <= 64) return 8;
    if (frames_per_sm <= 256) return 4;
    return 2;
}

cudaError_t launch_sus_team(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 4: return A.c.dcmax <= 6 ? launch_team_q<4, 6>(A, num_sms, s) : launch_team_q<4, 8>(A, num_sms, s);
    case 8: return A.c.dcmax <= 6 ? launch_team_q<8, 6>(A, num_sms, s) : launch_team_q<8, 8>(A, num_sms, s);
    case 16: return A.c.dcmax <= 6 ? launch_team_q<16, 6>(A, num_sms, s) : launch_team_q<16, 8>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
