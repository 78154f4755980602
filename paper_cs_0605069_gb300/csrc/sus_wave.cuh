// SUS (Sec. 2, steps 1-4) with several lane teams on one frame, for the codes
// and fields of the team kernel (q <= 16, column degree <= 4, row degree <= 8).
//
// The schedule updates the columns in the order j = 0..N-1, and column j reads
// the stored q of every column that shares a check with it.  Two columns that
// share no check touch disjoint data: column j reads and writes only the
// vectors of its own checks.  So column j may run as soon as every earlier
// column that shares a check with it has finished — pred(j), the last such
// column, is stored with the code — and every column then reads exactly the
// values the strictly sequential order gives it: the same arithmetic on the
// same operands, bit for bit.  (A later column k > j that shares a check with
// j cannot overwrite j's inputs early: it waits for j in turn.)
//
// W teams work on one frame (one CTA); team w takes the columns j = w, w + W,
// w + 2W, ... in order and publishes in shared memory the next column it will
// take.  The minimum over the teams (the watermark) is a column below which
// every column is done; column j starts once the watermark exceeds pred(j).
// The team with the smallest published column never waits (its pred is
// already done), so the sweep always advances; every wait is bounded anyway
// and a frame whose wait ran out reports iters = -1.
//
// The loads of a team's next column are issued before the current column is
// computed, with the watermark read just before them; they are reissued after
// the wait when that watermark did not yet cover pred of the next column.
// The per-iteration test, the trace and the Markov update (Eqs. 6-7) run after
// a barrier of the whole CTA.
#pragma once

#include "sus_team.cuh"

namespace gfbp {

namespace {

constexpr int kWaveSpinLimit = 1 << 22;   // polls of at least ~30 ns each

template <int W>
__device__ __forceinline__ int wave_watermark(const volatile int* prog) {
    int m = prog[0];
#pragma unroll
    for (int w = 1; w < W; w++) m = min(m, prog[w]);
    return m;
}

// Wait until every column <= p is done; false when the bound ran out.
template <int W>
__device__ __forceinline__ bool wave_wait(const volatile int* prog, int p) {
    for (int n = 0; n < kWaveSpinLimit; n++) {
        if (wave_watermark<W>(prog) > p) {
            __threadfence_block();
            return true;
        }
        __nanosleep(32);
    }
    return false;
}

// Lanes per slot of the multi-team kernel (one team per warp for q >= 8).
template <int Q>
using WaveLay = TeamLay<Q>;

// One frame's whole SUS decode by the W teams of the calling CTA.
template <int Q, int DC, int W>
__device__ __forceinline__ void sus_wave_frame(const DecodeArgs& A, int f, const uint8_t* s_mul,
                                               const uint8_t* s_div, float* sa, volatile int* prog, int* s_fail) {
    using TL = WaveLay<Q>;
    constexpr int GS = TL::GS, V = TL::V, TEAM = TL::TEAM, NTH = W * TEAM;
    const int tid = threadIdx.x;
    const int w = tid / TEAM;
    const int tl = tid & (TEAM - 1);
    const int k = tl / GS;
    const int g = tl & (GS - 1);
    const unsigned tmask = lanes_mask<TEAM>();
    const int M = A.c.M, N = A.c.N;
    const long long E = A.c.E;
    float* slab = A.msg + (size_t)f * E * Q;
    const uint8_t* zf = A.syn ? A.syn + (size_t)f * M : nullptr;
    uint8_t* xh = A.xhat + (size_t)f * N;

    int t0 = 0;   // iterations already done (resumable decoding)
    if (A.fstate) {
        const int st = A.fstate[f];
        if (st >> 30) return;
        t0 = st;
    }
    if (tid == 0) *s_fail = 0;
    int t = t0 + 1, ok = 0;
    bool fin = false;
    for (;; t++) {
        if (tl == 0) prog[w] = w;
        __syncthreads();
        int fail = 0;
        int jc = w;
        if (jc < N) {
            SlotBuf<Q, DC, V> cur, nxt;
            int pc = A.c.cpred[jc];
            int wmc = wave_watermark<W>(prog);
            __threadfence_block();
            slot_load<Q, DC, V>(cur, A, slab, f, jc, k, g);
            for (;;) {
                const int jn = jc + W;
                int pn = 0, wmn = 0;
                if (jn < N) {
                    pn = A.c.cpred[jn];
                    wmn = wave_watermark<W>(prog);
                    __threadfence_block();
                    slot_load<Q, DC, V>(nxt, A, slab, f, jn, k, g);
                }
                if (wmc <= pc) {
                    if (!wave_wait<W>(prog, pc)) fail = 1;
                    slot_load<Q, DC, V>(cur, A, slab, f, jc, k, g);
                }
                team_column<Q, DC, GS>(A, f, jc, cur, s_mul, s_div, sa, slab, zf, xh);
                __threadfence_block();
                __syncwarp(tmask);
                if (tl == 0) prog[w] = jn;
                if (jn >= N) break;
                jc = jn;
                cur = nxt;
                pc = pn;
                wmc = wmn;
            }
        }
        if (fail) *s_fail = 1;
        __syncthreads();
        int bad = 0;
        for (int i = tid; i < M; i += NTH) {
            int s = 0;
            const int e1 = A.c.rowptr[i + 1];
            for (int e = A.c.rowptr[i]; e < e1; e++) s ^= s_mul[A.c.eh[e] * Q + xh[A.c.ecol[e]]];
            bad |= (s != (zf ? (zf[i] & (Q - 1)) : 0));
        }
        ok = !__syncthreads_or(bad);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int jj = tid; jj < N; jj += NTH) tr[jj] = xh[jj];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) {
            fin = true;
            break;
        }
        if (A.markov) {
            for (int i = w; i < A.K; i += W) team_prior<Q, TEAM>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, tmask, tl);
            __syncthreads();
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = w; i < A.K; i += W)
            team_prior<Q, TEAM>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, tmask, tl);
    }
    if (A.trace) {
        for (size_t o = (size_t)t * N + tid; o < (size_t)A.max_iter * N; o += NTH)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (tid == 0) {
        const bool bad_wait = *s_fail != 0;
        if (!A.fstate || fin || bad_wait) {
            if (A.iters) A.iters[f] = bad_wait ? -1 : t;
            A.conv[f] = (uint8_t)(ok && !bad_wait);
        }
        if (A.fstate) A.fstate[f] = (fin || bad_wait) ? (t | (1 << 30)) : t;
    }
}

template <int Q, int DC, int W>
__global__ void __launch_bounds__(W * WaveLay<Q>::TEAM) k_sus_wave(const DecodeArgs A) {
    using TL = WaveLay<Q>;
    constexpr int GS = TL::GS, NTH = W * TL::TEAM;
    constexpr int SCR = 2 * Q + 4;   // per slot: two operand vectors (+ bank padding)
    __shared__ uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ __align__(16) float s_scr[(NTH / GS) * SCR];
    __shared__ int s_prog[W];
    __shared__ int s_f, s_fail;
    const int tid = threadIdx.x;
    float* sa = s_scr + (tid / GS) * SCR;
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, NTH);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        sus_wave_frame<Q, DC, W>(A, f, s_mul, s_div, sa, s_prog, &s_fail);
    }
}

}  // namespace
}  // namespace gfbp
