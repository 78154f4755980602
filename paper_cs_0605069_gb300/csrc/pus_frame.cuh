// Parallel updating scheme (PUS, flooding; Sec. 2): one persistent CTA per
// frame.  Each CTA takes frames from a global counter and runs all of a
// frame's iterations: horizontal pass (every r_ij from the previous
// iteration's q, Eq. 3), vertical pass (every q_ij and Q_j, Eqs. 4-5),
// hard decision and the test H x = z, then the block-prior update (Eqs. 6-7)
// for a Markov source.  Passes are separated by __syncthreads; no host round
// trip between iterations.
//
// The frame's edge slab is updated in place: the horizontal pass replaces the
// transforms of q_ij by r_ij (each edge belongs to one check), the vertical
// pass replaces r_ij by the transform of the new q_ij (each edge belongs to
// one column).
#pragma once

#include "bulk.cuh"
#include "gfbp_internal.cuh"

namespace gfbp {

namespace {

constexpr int kPusThreads = 256;

// r_ij for every edge of check i: prefix/suffix combinations of the other
// edges' stored vectors (no division: transforms can be exactly 0).
template <int Q, int DC>
__device__ __forceinline__ void pus_check(const DecodeArgs& A, float* slab, int f, int i, float* sc, unsigned mask,
                                          int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    const int e0 = A.c.rowptr[i];
    const int d = A.c.rowptr[i + 1] - e0;
    const int z = A.syn ? (A.syn[(size_t)f * A.c.M + i] & (Q - 1)) : 0;
    const int lane0 = (threadIdx.x & 31) & ~(G - 1);
    float S[DC][V];
    int Cs[DC];
    float acc[V];
    int cacc = 0;
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0.f;
#pragma unroll
    for (int k = DC - 1; k >= 0; k--) {
        if (k < d) {
#pragma unroll
            for (int v = 0; v < V; v++) S[k][v] = acc[v];
            Cs[k] = cacc;
            float D[V];
            int c;
            ld_dev<V>(D, c, slab + (size_t)(e0 + k) * Q + g * V, g);
            dev_combine<V>(acc, D);
            cacc ^= c;
        }
    }
    float pre[V];
    int cpre = 0;
#pragma unroll
    for (int v = 0; v < V; v++) pre[v] = 0.f;
#pragma unroll
    for (int k = 0; k < DC; k++) {
        if (k < d) {
            float D[V], x[V];
            int c;
            ld_dev<V>(D, c, slab + (size_t)(e0 + k) * Q + g * V, g);
#pragma unroll
            for (int v = 0; v < V; v++) x[v] = fmaf(pre[v], 1.0f - S[k][v], S[k][v]);
            const int C = __shfl_sync(mask, cpre ^ Cs[k], lane0);
            dev_combine<V>(pre, D);
            cpre ^= c;
            dev_finish<Q>(x, C, A.c.eh[e0 + k], z, sc, mask, g, ex, lg, zsum_of(A, f));
            stv<V>(slab + (size_t)(e0 + k) * Q + g * V, x);
        }
    }
}

// r_ij for every edge of check i by the probability-domain route: suffix
// convolutions S_k = qt_{k+1} * ... * qt_{d-1}, a running prefix P, and
// r_k from P * S_k (3(d-2) convolutions for d edges).  The group's scratch
// holds the d stored vectors and two operand slots.
// STAGED: the d stored vectors are already in `sc` (a bulk copy) and the
// operand slots are at `ops`; otherwise they are copied in here and the slots
// follow them.
template <int Q, int DC, bool STAGED = false>
__device__ __forceinline__ void pus_check_direct(const DecodeArgs& A, float* slab, int f, int i, float* sc,
                                                 unsigned mask, int g, const uint8_t* ex, const uint8_t* lg,
                                                 float* ops = nullptr) {
    constexpr int V = Lay<Q>::V;
    const int e0 = A.c.rowptr[i];
    const int d = A.c.rowptr[i + 1] - e0;
    const int z = A.syn ? (A.syn[(size_t)f * A.c.M + i] & (Q - 1)) : 0;
    float* T0 = STAGED ? ops : sc + DC * Q;
    float* T1 = T0 + Q;
    if constexpr (!STAGED) {
#pragma unroll
        for (int k = 0; k < DC; k++) {
            if (k < d) {
                float x[V];
                ldv<V>(x, slab + (size_t)(e0 + k) * Q + g * V);
                stv<V>(sc + k * Q + g * V, x);
            }
        }
        __syncwarp(mask);
    }
    float S[DC][V];  // S[k] = qt_{k+1} * ... * qt_{d-1} for k <= d-2
#pragma unroll
    for (int k = DC - 2; k >= 0; k--) {
        if (k == d - 2) {
            ldv<V>(S[k], sc + (k + 1) * Q + g * V);
        } else if (k < d - 2) {
            stv<V>(T0 + g * V, S[k + 1]);
            __syncwarp(mask);
            xconv_sm<Q>(S[k], T0, sc + (k + 1) * Q, g);
            __syncwarp(mask);
        }
    }
    float P[V];
    bool p_id = true;  // P is the identity (no edge folded in yet)
#pragma unroll
    for (int k = 0; k < DC; k++) {
        if (k < d) {
            float out[1][V];
            if (k == d - 1) {
#pragma unroll
                for (int v = 0; v < V; v++) out[0][v] = p_id ? ((g * V + v) == 0 ? 1.f : 0.f) : P[v];
            } else if (p_id) {
#pragma unroll
                for (int v = 0; v < V; v++) out[0][v] = S[k][v];
                ldv<V>(P, sc + k * Q + g * V);
                p_id = false;
            } else {
                // r_k = P * S_k and the next prefix P * qt_k in one pass over P
                stv<V>(T0 + g * V, P);
                stv<V>(T1 + g * V, S[k]);
                __syncwarp(mask);
                xconv_sm2<Q>(out[0], P, T0, T1, sc + k * Q, g);
                __syncwarp(mask);
            }
            const int hh[1] = {A.c.eh[e0 + k]}, zz[1] = {z};
            direct_finish_n<Q, 1>(out, hh, zz, 1, T1, mask, g, ex, lg, zsum_of(A, f));
            stv<V>(slab + (size_t)(e0 + k) * Q + g * V, out[0]);
        }
    }
}

// q_ij for every edge of column j (Eq. 4), Q_j (Eq. 5) and its hard decision.
template <int Q, int DV, int METHOD>
__device__ __forceinline__ void pus_var(const DecodeArgs& A, float* slab, int f, int j, float* sc, unsigned mask,
                                        int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    const int c0 = A.c.colptr[j];
    const int d = A.c.colptr[j + 1] - c0;
    float p[V];
    prior_vec<Q>(A, f, j, p, mask, g);
    float S[DV][V];
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 1.f;
#pragma unroll
    for (int k = DV - 1; k >= 0; k--) {
        if (k < d) {
#pragma unroll
            for (int v = 0; v < V; v++) S[k][v] = acc[v];
            float R[V];
            ldv<V>(R, slab + (size_t)A.c.cedge[c0 + k] * Q + g * V);
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] *= R[v];
        }
    }
    // pseudo-posterior and hard decision
    {
        float Qj[V];
#pragma unroll
        for (int v = 0; v < V; v++) Qj[v] = p[v] * acc[v];
        gnormalise<Q>(Qj, mask, zsum_of(A, f));
        const int a = gargmax<Q>(Qj, mask, g);
        if (g == 0) A.xhat[(size_t)f * A.c.N + j] = (uint8_t)a;
        if (A.post) stv<V>(A.post + ((size_t)f * A.c.N + j) * Q + g * V, Qj);
        if (A.markov) {
            const int si = A.src_index[j];
            if (si >= 0) stv<V>(A.Qsrc + ((size_t)f * A.K + si) * Q + g * V, Qj);
        }
    }
    float pre[V];
#pragma unroll
    for (int v = 0; v < V; v++) pre[v] = 1.f;
#pragma unroll
    for (int k = 0; k < DV; k++) {
        if (k < d) {
            const int e = A.c.cedge[c0 + k];
            float R[V], x[V];
            ldv<V>(R, slab + (size_t)e * Q + g * V);
#pragma unroll
            for (int v = 0; v < V; v++) {
                x[v] = p[v] * (pre[v] * S[k][v]);
                pre[v] *= R[v];
            }
            gnormalise<Q>(x, mask, zsum_of(A, f));
            if (A.step) stv<V>(A.msg_io + ((size_t)f * A.c.E + e) * Q + g * V, x);
            if constexpr (METHOD == kDirect) to_relabelled<Q>(x, A.c.eh[e], sc, mask, g, ex, lg);
            else to_deviation<Q>(x, A.c.eh[e], sc, mask, g, ex, lg);
            stv<V>(slab + (size_t)e * Q + g * V, x);
        }
    }
}

// Per-group scratch floats: one vector (transform route) or the check's d
// stored vectors plus two operands (probability route; with BULK two buffers
// of d vectors, filled by bulk copies one check ahead); +4 floats of padding
// spread the groups over the shared-memory banks.
template <int Q, int DC, int METHOD, bool BULK = false>
constexpr int pus_group_scratch() {
    return (METHOD == kDirect ? ((BULK ? 2 : 1) * DC + 2) * Q : Q) + 4;
}

// One frame's whole PUS decode by the calling CTA (all its threads).
// BULK (probability route): a group's next check is fetched by a bulk copy
// into its second buffer while the current one is combined; s_bar holds two
// mbarriers per group, `phase` the parity of each (per thread, kept across
// frames), s_fail is set when a wait gave up (the frame then reports -1).
template <int Q, int DC, int DV, int METHOD, bool BULK = false>
__device__ __forceinline__ void pus_frame(const DecodeArgs& A, int f, const uint8_t* s_exp, const uint8_t* s_log,
                                          float* s_scr, uint64_t* s_bar = nullptr, uint32_t* phase = nullptr,
                                          int* s_fail = nullptr) {
    static_assert(!BULK || METHOD == kDirect, "bulk staging is for the probability route");
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    constexpr int SCR = pus_group_scratch<Q, DC, METHOD, BULK>();
    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const int grp = tid / G;
    const int ngrp = blockDim.x / G;
    const unsigned mask = group_mask<G>();
    float* sc = s_scr + grp * SCR;
    const int M = A.c.M, N = A.c.N;
    const long long E = A.c.E;
    float* slab = A.msg + (size_t)f * E * Q;

    int t0 = 0;   // iterations already done (resumable decoding)
    if (A.fstate) {
        const int st = A.fstate[f];
        if (st >> 30) return;
        t0 = st;
    }
    // q_ij <- p_j (Sec. 2) or the caller's state, in stored form
    for (long long e = grp; e < E && t0 == 0; e += ngrp) {
        float x[V];
        if (A.step) {
            ldv<V>(x, A.msg_io + ((size_t)f * E + e) * Q + g * V);
        } else {
            prior_vec<Q>(A, f, A.c.ecol[e], x, mask, g);
        }
        if constexpr (METHOD == kDirect) to_relabelled<Q>(x, A.c.eh[e], sc, mask, g, s_exp, s_log);
        else to_deviation<Q>(x, A.c.eh[e], sc, mask, g, s_exp, s_log);
        stv<V>(slab + (size_t)e * Q + g * V, x);
    }
    if constexpr (BULK) {
        fence_proxy_async();   // the stores above, before the bulk copies that read them
        if (tid == 0) *s_fail = 0;
    }
    __syncthreads();

    int t = t0 + 1, ok = 0;
    bool fin = false;
    for (;; t++) {
        if constexpr (BULK) {
            float* ops = sc;
            float* buf[2] = {sc + 2 * Q, sc + (2 + DC) * Q};
            uint64_t* bar = s_bar + 2 * grp;
            auto issue = [&](int i, int b) {
                if (g == 0) {
                    const int e0 = A.c.rowptr[i];
                    const uint32_t bytes = (uint32_t)(A.c.rowptr[i + 1] - e0) * Q * (uint32_t)sizeof(float);
                    fence_proxy_async();
                    bulk_load(buf[b], slab + (size_t)e0 * Q, bytes, bar + b);
                }
            };
            int r = 0;
            if (grp < M) issue(grp, 0);
            for (int i = grp; i < M; i += ngrp, r++) {
                const int b = r & 1;
                if (i + ngrp < M) {
                    __syncwarp(mask);   // every lane is done with the other buffer
                    issue(i + ngrp, b ^ 1);
                }
                if (!mbar_wait(bar + b, (*phase >> b) & 1u)) *s_fail = 1;
                *phase ^= 1u << b;
                pus_check_direct<Q, DC, true>(A, slab, f, i, buf[b], mask, g, s_exp, s_log, ops);
            }
        } else {
            for (int i = grp; i < M; i += ngrp) {
                if constexpr (METHOD == kDirect) pus_check_direct<Q, DC>(A, slab, f, i, sc, mask, g, s_exp, s_log);
                else pus_check<Q, DC>(A, slab, f, i, sc, mask, g, s_exp, s_log);
            }
        }
        __syncthreads();
        for (int j = grp; j < N; j += ngrp) pus_var<Q, DV, METHOD>(A, slab, f, j, sc, mask, g, s_exp, s_log);
        if constexpr (BULK) fence_proxy_async();   // the q just stored, before the next pass's bulk copies
        __syncthreads();
        int bad = 0;
        for (int i = tid; i < M; i += blockDim.x) {
            int s = 0;
            for (int e = A.c.rowptr[i]; e < A.c.rowptr[i + 1]; e++)
                s ^= gf_mul(s_exp, s_log, A.c.eh[e], A.xhat[(size_t)f * N + A.c.ecol[e]]);
            const int z = A.syn ? (A.syn[(size_t)f * M + i] & (Q - 1)) : 0;
            bad |= (s != z);
        }
        ok = !__syncthreads_or(bad);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int j = tid; j < N; j += blockDim.x) tr[j] = A.xhat[(size_t)f * N + j];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) {
            fin = true;
            break;
        }
        if (A.markov) {
            for (int i = grp; i < A.K; i += ngrp)
                markov_prior<Q>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, mask, g);
            __syncthreads();
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = grp; i < A.K; i += ngrp)
            markov_prior<Q>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, mask, g);
    }
    if (A.trace) {
        for (size_t o = (size_t)t * N + tid; o < (size_t)A.max_iter * N; o += blockDim.x)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (tid == 0) {
        bool bad_wait = false;
        if constexpr (BULK) bad_wait = *s_fail != 0;
        if (!A.fstate || fin || bad_wait) {
            if (A.iters) A.iters[f] = bad_wait ? -1 : t;
            A.conv[f] = (uint8_t)(ok && !bad_wait);
        }
        if (A.fstate) A.fstate[f] = (fin || bad_wait) ? (t | (1 << 30)) : t;
    }
}

// Bulk staging applies to the probability route when a vector is a whole
// number of 16-byte units (q >= 4), so that every check's run of vectors
// starts on a 16-byte boundary as the copy engine requires.
template <int Q, int METHOD>
constexpr bool pus_bulk_ok() { return METHOD == kDirect && Q >= 4; }

template <int Q, int DC, int DV, int METHOD, bool BULK = false>
__global__ void __launch_bounds__(kPusThreads) k_pus(const DecodeArgs A) {
    static_assert(!BULK || pus_bulk_ok<Q, METHOD>(), "bulk staging needs the probability route and q >= 4");
    constexpr int T = kPusThreads;
    constexpr int NB = BULK ? 2 * (T / Lay<Q>::G) : 1;
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ int s_frame, s_fail;
    __shared__ __align__(8) uint64_t s_bar[NB];
    extern __shared__ __align__(16) float s_scr[];
    const int tid = threadIdx.x;
    for (int k = tid; k < 512; k += blockDim.x) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += blockDim.x) s_log[k] = A.c.glog[k];
    if constexpr (BULK) {
        for (int k = tid; k < 2 * ((int)blockDim.x / Lay<Q>::G); k += blockDim.x) mbar_init(&s_bar[k]);
        mbar_init_fence();
    }
    uint32_t phase = 0;   // parity of the next completion of this group's two mbarriers
    for (;;) {
        __syncthreads();
        if (tid == 0) s_frame = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_frame;
        if (f >= A.F) break;
        pus_frame<Q, DC, DV, METHOD, BULK>(A, f, s_exp, s_log, s_scr, s_bar, &phase, &s_fail);
    }
}

}  // namespace
}  // namespace gfbp
