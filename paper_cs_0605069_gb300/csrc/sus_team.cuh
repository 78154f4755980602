// Sequential updating scheme (SUS; Sec. 2, steps 1-4) with the
// probability-domain check node, for q <= 16 and codes with column degree
// <= 4 and row degree <= 8: one lane team per frame (one warp for q = 8, 16;
// half a warp for q = 4).  The team has four slots of GS lanes; slot k
// handles the k-th check of the current column, so step 1 (r_ij for every
// check of column j) runs for all of the column's checks at once, and step 2
// (q_ij, Q_j) exchanges the r_ij between slots with shuffles.
//
// Columns are still visited strictly in order j = 0..N-1 within a sweep; the
// loads of column j+1 are issued before column j is computed and reissued
// after its stores when the two columns share a check (a per-column flag
// built with the code).  Each lane reads and writes only its own slice of the
// stored vectors of its slot, so program order makes its stores visible to
// its later loads; vectors that cross slots (r_ij) move by shuffles.
#pragma once

#include "gfbp_internal.cuh"

namespace gfbp {

namespace {

constexpr int kTeamThreads = 128;
constexpr int kSlots = 4;

// Lanes per slot vector (GS), entries per lane (V) and lanes per team; both
// team kernels use GS = min(q, 8).  Every sum below runs in an order fixed by
// the entry indices alone, so any GS gives the same bits.  (GS = q / 4, four
// entries per lane with 128-bit shared loads, needs fewer instructions per
// column but puts two teams in a warp whose waits diverge, and ran 1.7x
// slower on the GF(16) N = 1000 batch.)
template <int Q, int GS_ = (Q < 8 ? Q : 8)>
struct TeamLay {
    static constexpr int GS = GS_;
    static constexpr int V = Q / GS;
    static constexpr int TEAM = kSlots * GS;
    static_assert(V * GS == Q && V <= 4, "at most four entries per lane");
    static_assert(TEAM == 4 || TEAM == 8 || TEAM == 16 || TEAM == 32, "team must divide a warp");
};

template <int L>
__device__ __forceinline__ unsigned lanes_mask() {
    if constexpr (L == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << L) - 1u) << (lane & ~(unsigned)(L - 1));
    }
}

// out[v] = sum_x sa[x] sb[x XOR y] for y = g*V + v (whole vectors in shared memory),
// one FMA chain per output in increasing x: the same order for any V.
template <int Q, int V>
__device__ __forceinline__ void xconv_team(float (&out)[V], const float* sa, const float* sb, int g) {
#pragma unroll
    for (int v = 0; v < V; v++) out[v] = 0.f;
#pragma unroll
    for (int xb = 0; xb < Q; xb += V) {
        float a[V], b[V];
        ldv<V>(a, sa + xb);
        ldv<V>(b, sb + (xb ^ (g * V)));
#pragma unroll
        for (int xl = 0; xl < V; xl++) {
#pragma unroll
            for (int v = 0; v < V; v++) out[v] = fmaf(a[xl], b[xl ^ v], out[v]);
        }
    }
}

// Sum of the slot's q entries as a pairwise tree over the index bits, lowest
// bit first (inside the lane, then across lanes): the same bits for any GS.
template <int GS, int V>
__device__ __forceinline__ float slot_sum(const float (&x)[V], unsigned smask) {
    float s;
    if constexpr (V == 4) s = __fadd_rn(__fadd_rn(x[0], x[1]), __fadd_rn(x[2], x[3]));
    else if constexpr (V == 2) s = __fadd_rn(x[0], x[1]);
    else s = x[0];
#pragma unroll
    for (int m = 1; m < GS; m <<= 1) s = __fadd_rn(s, __shfl_xor_sync(smask, s, m));
    return s;
}

template <int Q, int GS, int V>
__device__ __forceinline__ void slot_normalise(float (&x)[V], unsigned smask, int* zs = nullptr) {
    const float s = slot_sum<GS, V>(x, smask);
    if (s > 0.f && s <= 3.0e38f) {
        const float r = 1.0f / s;
#pragma unroll
        for (int v = 0; v < V; v++) x[v] *= r;
    } else {
#pragma unroll
        for (int v = 0; v < V; v++) x[v] = 1.0f / Q;
        note_zero_sum<GS>(zs);
    }
}

template <int GS, int V>
__device__ __forceinline__ int slot_argmax(const float (&x)[V], unsigned smask, int g) {
    float bv = x[0];
    int bi = g * V;
#pragma unroll
    for (int i = 1; i < V; i++)
        if (x[i] > bv) { bv = x[i]; bi = g * V + i; }
#pragma unroll
    for (int m = 1; m < GS; m <<= 1) {
        const float ov = __shfl_xor_sync(smask, bv, m);
        const int oi = __shfl_xor_sync(smask, bi, m);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    return bi;
}

template <int Q, int DC, int V>
struct SlotBuf {
    float D[DC][V];
    float L[V];              // channel likelihood of the column's symbol
    int4 info;               // {edge, row start, row degree | h << 8, row}
    int d;                   // column degree
    int dep;                 // column shares a check with the previous one
};

template <int Q, int DC, int V>
__device__ __forceinline__ void slot_load(SlotBuf<Q, DC, V>& b, const DecodeArgs& A, const float* slab, int f, int j,
                                          int k, int g) {
    const int c0 = A.c.colptr[j];
    b.d = A.c.colptr[j + 1] - c0;
    b.dep = A.c.cdep[j];
    ldg_v<V>(b.L, A.L + ((size_t)f * A.c.N + j) * Q + g * V);
    if (k < b.d) {
        b.info = A.c.cinfo[c0 + k];
        const int e0 = b.info.y, dc = b.info.z & 255;
#pragma unroll
        for (int m = 0; m < DC; m++)
            if (m < dc) ldv<V>(b.D[m], slab + (size_t)(e0 + m) * Q + g * V);
    }
}

// Markov block prior of source index i for the team (Eq. 7 form, as in
// markov_prior, with the team's lanes splitting the q entries).
template <int Q, int TEAM>
__device__ __forceinline__ void team_prior(const DecodeArgs& A, int f, int i, float* out, unsigned tmask, int tl) {
    const int K = A.K;
    const float* Qm = (i > 0) ? A.Qsrc + ((size_t)f * K + i - 1) * Q : nullptr;
    const float* Qp = (i < K - 1) ? A.Qsrc + ((size_t)f * K + i + 1) * Q : nullptr;
    float P = 0.f;
    const int b = tl;
    if (b < Q) {
        float left = 0.f, right = 0.f;
        if (Qm) { for (int a = 0; a < Q; a++) left = fmaf(Qm[a], A.Mt[a * Q + b], left); }
        else left = A.pi[b];
        if (Qp) { for (int c = 0; c < Q; c++) right = fmaf(A.Mt[b * Q + c], Qp[c], right); }
        else right = 1.f;
        P = left * right;
    }
    float s = P;
#pragma unroll
    for (int m = 1; m < TEAM; m <<= 1) s += __shfl_xor_sync(tmask, s, m);
    if (b < Q) out[b] = (s > 0.f && s <= 3.0e38f) ? P / s : 1.0f / Q;
}

// Steps 1-2 of SUS for column j by the calling team: the r_ij of every check
// of the column (slot k: the column's k-th check) from the stored vectors in
// `cur`, then Q_j (hard decision, posterior, Markov source posterior) and the
// new stored q_ij.  s_mul / s_div: the field's multiply and divide-by-h
// tables; sa: this slot's shared scratch (2q + 4 floats).
template <int Q, int DC, int GS_>
__device__ __forceinline__ void team_column(const DecodeArgs& A, int f, int j, const SlotBuf<Q, DC, Q / GS_>& cur,
                                            const uint8_t* s_mul, const uint8_t* s_div, float* sa, float* slab,
                                            const uint8_t* zf, uint8_t* xh) {
    using TL = TeamLay<Q, GS_>;
    constexpr int GS = TL::GS, V = TL::V, TEAM = TL::TEAM;
    const int tl = threadIdx.x & (TEAM - 1);
    const int k = tl / GS;
    const int g = tl & (GS - 1);
    const unsigned tmask = lanes_mask<TEAM>();
    const unsigned smask = lanes_mask<GS>();
    const int team_lane0 = (threadIdx.x & 31) & ~(TEAM - 1);
    const int N = A.c.N;
    const long long E = A.c.E;
    const int d = cur.d;
    const bool act = k < d;
    const int4 in = cur.info;
    const int own = act ? in.x - in.y : 0;
    const int dc = act ? (in.z & 255) : 1;
    const int h = act ? ((in.z >> 8) & 255) : 1;
    const int z = (act && zf) ? (zf[in.w] & (Q - 1)) : 0;
    // step 1: distribution of the XOR-sum of the check's other edges,
    // folded in neighbour order (the same instruction stream in every slot)
    const int c = dc - 1;
    float U[V];
#pragma unroll
    for (int v = 0; v < V; v++) U[v] = (g * V + v) == 0 ? 1.f : 0.f;
#pragma unroll
    for (int n = 0; n < DC - 1; n++) {
        if (n < c) {
            float Y[V];
#pragma unroll
            for (int v = 0; v < V; v++) Y[v] = (n >= own) ? cur.D[n + 1][v] : cur.D[n][v];
            if (n == 0) {
#pragma unroll
                for (int v = 0; v < V; v++) U[v] = Y[v];
            } else {
                stv<V>(sa + g * V, U);
                stv<V>(sa + Q + g * V, Y);
                __syncwarp(smask);
                xconv_team<Q, V>(U, sa, sa + Q, g);
                __syncwarp(smask);
            }
        }
    }
    // r_ij[a] = s[z XOR h a], normalised
    stv<V>(sa + g * V, U);
    __syncwarp(smask);
    float R[V];
#pragma unroll
    for (int v = 0; v < V; v++) R[v] = sa[(z ^ s_mul[h * Q + g * V + v]) & (Q - 1)];
    __syncwarp(smask);
    slot_normalise<Q, GS, V>(R, smask, act ? zsum_of(A, f) : nullptr);
    if (!act) {
#pragma unroll
        for (int v = 0; v < V; v++) R[v] = 1.f;
    }
    // step 2: products over the other slots' r at the same entries
    float p[V];
#pragma unroll
    for (int v = 0; v < V; v++) p[v] = cur.L[v];
    if (A.markov) {
        const int si = A.src_index[j];
        if (si >= 0) {
            float P[V];
            ldv<V>(P, A.P + ((size_t)f * A.K + si) * Q + g * V);
#pragma unroll
            for (int v = 0; v < V; v++) p[v] *= P[v];
            slot_normalise<Q, GS, V>(p, smask);
        }
    }
    float other[V], all[V];
#pragma unroll
    for (int v = 0; v < V; v++) { other[v] = p[v]; all[v] = p[v]; }
#pragma unroll
    for (int k2 = 0; k2 < kSlots; k2++) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            const float r2 = __shfl_sync(tmask, R[v], team_lane0 + k2 * GS + g);
            all[v] *= r2;
            if (k2 != k) other[v] *= r2;
        }
    }
    slot_normalise<Q, GS, V>(all, smask, k == 0 ? zsum_of(A, f) : nullptr);
    if (k == 0) {
        const int a = slot_argmax<GS, V>(all, smask, g);
        if (g == 0) xh[j] = (uint8_t)a;
        if (A.post) stv<V>(A.post + ((size_t)f * N + j) * Q + g * V, all);
        if (A.markov) {
            const int si = A.src_index[j];
            if (si >= 0) stv<V>(A.Qsrc + ((size_t)f * A.K + si) * Q + g * V, all);
        }
    }
    slot_normalise<Q, GS, V>(other, smask, act ? zsum_of(A, f) : nullptr);
    if (act && A.step) stv<V>(A.msg_io + ((size_t)f * E + in.x) * Q + g * V, other);
    // stored form: qt[y] = q[h^-1 y]
    stv<V>(sa + g * V, other);
    __syncwarp(smask);
#pragma unroll
    for (int v = 0; v < V; v++) other[v] = sa[s_div[h * Q + g * V + v]];
    __syncwarp(smask);
    if (act) stv<V>(slab + (size_t)in.x * Q + g * V, other);
}

// One frame's whole SUS decode by the calling team (all iterations, the test,
// the Markov update and the outputs).
template <int Q, int DC>
__device__ __forceinline__ void sus_team_frame(const DecodeArgs& A, int f, const uint8_t* s_mul,
                                               const uint8_t* s_div, float* sa) {
    using TL = TeamLay<Q>;
    constexpr int GS = TL::GS, V = TL::V, TEAM = TL::TEAM;
    const int tl = threadIdx.x & (TEAM - 1);
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
    int t = t0 + 1, ok = 0;
    bool fin = false;
    for (;; t++) {
        SlotBuf<Q, DC, V> cur, nxt;
        slot_load<Q, DC, V>(cur, A, slab, f, 0, k, g);
        for (int j = 0; j < N; j++) {
            if (j + 1 < N) slot_load<Q, DC, V>(nxt, A, slab, f, j + 1, k, g);
            team_column<Q, DC, GS>(A, f, j, cur, s_mul, s_div, sa, slab, zf, xh);
            if (j + 1 < N) {
                if (nxt.dep) slot_load<Q, DC, V>(nxt, A, slab, f, j + 1, k, g);
                cur = nxt;
            }
        }
        __syncwarp(tmask);
        int bad = 0;
        for (int i = tl; i < M; i += TEAM) {
            int s = 0;
            const int e1 = A.c.rowptr[i + 1];
            for (int e = A.c.rowptr[i]; e < e1; e++) s ^= s_mul[A.c.eh[e] * Q + xh[A.c.ecol[e]]];
            bad |= (s != (zf ? (zf[i] & (Q - 1)) : 0));
        }
#pragma unroll
        for (int m = 1; m < TEAM; m <<= 1) bad |= __shfl_xor_sync(tmask, bad, m);
        ok = !bad;
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int jj = tl; jj < N; jj += TEAM) tr[jj] = xh[jj];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) {
            fin = true;
            break;
        }
        if (A.markov) {
            for (int i = 0; i < A.K; i++) team_prior<Q, TEAM>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, tmask, tl);
            __syncwarp(tmask);
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = 0; i < A.K; i++)
            team_prior<Q, TEAM>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, tmask, tl);
    }
    if (A.trace) {
        for (size_t o = (size_t)t * N + tl; o < (size_t)A.max_iter * N; o += TEAM)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (tl == 0) {
        if (!A.fstate || fin) {
            if (A.iters) A.iters[f] = t;
            A.conv[f] = (uint8_t)ok;
        }
        if (A.fstate) A.fstate[f] = fin ? (t | (1 << 30)) : t;
    }
}

// Tables of h a and h^-1 b for every h, a of the field (q <= 16).
template <int Q>
__device__ __forceinline__ void team_tables(const uint8_t* gexp, const uint8_t* glog, uint8_t* s_mul, uint8_t* s_div,
                                            int tid, int nthreads) {
    for (int x = tid; x < Q * Q; x += nthreads) {
        const int hh = x / Q, a = x % Q;
        s_mul[x] = (uint8_t)gf_mul(gexp, glog, hh, a);
        s_div[x] = hh ? (uint8_t)gf_div<Q>(gexp, glog, a, hh) : 0;
    }
}

template <int Q, int DC>
__global__ void __launch_bounds__(kTeamThreads) k_sus_team(const DecodeArgs A) {
    using TL = TeamLay<Q>;
    constexpr int GS = TL::GS, TEAM = TL::TEAM;
    constexpr int SCR = 2 * Q + 4;   // per slot: two operand vectors (+ bank padding)
    __shared__ uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ __align__(16) float s_scr[(kTeamThreads / GS) * SCR];
    const int tid = threadIdx.x;
    const int tl = tid & (TEAM - 1);
    const unsigned tmask = lanes_mask<TEAM>();
    const int team_lane0 = (threadIdx.x & 31) & ~(TEAM - 1);
    float* sa = s_scr + (tid / GS) * SCR;
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, blockDim.x);
    __syncthreads();
    for (;;) {
        int f = 0;
        if (tl == 0) f = atomicAdd(A.work, 1);
        f = __shfl_sync(tmask, f, team_lane0);
        if (f >= A.F) break;
        sus_team_frame<Q, DC>(A, f, s_mul, s_div, sa);
        __syncwarp(tmask);
    }
}

}  // namespace
}  // namespace gfbp
