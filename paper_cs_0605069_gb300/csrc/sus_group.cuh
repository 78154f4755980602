// Sequential updating scheme (SUS; Sec. 2, steps 1-4): one lane group per
// frame, persistent over a frame counter.  For j = 0..N-1 strictly in order:
// step 1, r_ij for every check i of column j from the current q of the
// check's other edges (Eq. 3); step 2, q_ij for column j (Eq. 4), and Q_j
// (Eq. 5) from the same r_ij.  After the sweep: the test H x = z and the
// block-prior update (Eqs. 6-7).  Parallelism inside a frame comes only from
// a column's d_v checks (processed together) and the q entries of a vector
// (the group's lanes); frames run side by side.
//
// Latency: a frame's sweep is a chain of N dependent column steps, so the
// loads of column j+1 are issued before column j is computed.  They are only
// stale if column j+1 shares a check with column j (a per-column flag built
// with the code); then they are issued again after column j's stores.  Each
// lane only touches its own slice of every stored vector, so program order
// makes its own stores visible to its later loads.
#pragma once

#include "gfbp_internal.cuh"

namespace gfbp {

namespace {

constexpr int kSusThreads = 128;

template <int Q, int DC, int DV>
struct ColBuf {
    float D[DV][DC][Lay<Q>::V];
    int4 info[DV];
    int d;
};

template <int Q, int DC, int DV>
__device__ __forceinline__ void load_col(ColBuf<Q, DC, DV>& b, const DecodeArgs& A, const float* slab, int j, int g) {
    constexpr int V = Lay<Q>::V;
    const int c0 = A.c.colptr[j];
    b.d = A.c.colptr[j + 1] - c0;
#pragma unroll
    for (int k = 0; k < DV; k++)
        if (k < b.d) b.info[k] = A.c.cinfo[c0 + k];
#pragma unroll
    for (int k = 0; k < DV; k++) {
        if (k < b.d) {
            const int e0 = b.info[k].y, dc = b.info[k].z & 255;
#pragma unroll
            for (int m = 0; m < DC; m++)
                if (m < dc) ldv<V>(b.D[k][m], slab + (size_t)(e0 + m) * Q + g * V);
        }
    }
}

// Steps 1-2 for column j once E (the combined other-edge vectors) and C (the
// XOR of their shifts) are known for each of the column's d checks.
template <int Q, int DV, int METHOD>
__device__ __forceinline__ void sus_column_tail(const DecodeArgs& A, float* slab, int f, int j, int d,
                                                float (&E)[DV][Lay<Q>::V], const int (&C)[DV], const int (&eid)[DV],
                                                const int (&h)[DV], const int (&z)[DV], uint8_t* xh, float* sc,
                                                unsigned mask, int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    const int N = A.c.N;
    // E: transform route, the combined deviations; probability route, the
    // distribution of the other edges' sum.  Afterwards E holds r_ij.
    int* zs = zsum_of(A, f);
    if constexpr (METHOD == kDirect) direct_finish_n<Q, DV>(E, h, z, d, sc, mask, g, ex, lg, zs);
    else dev_finish_n<Q, DV>(E, C, h, z, d, sc, mask, g, ex, lg, zs);
    float p[V];
    prior_vec<Q>(A, f, j, p, mask, g);
    float S[DV][V], acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 1.f;
#pragma unroll
    for (int k = DV - 1; k >= 0; k--) {
        if (k < d) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                S[k][v] = acc[v];
                acc[v] *= E[k][v];
            }
        }
    }
    {
        float Qj[V];
#pragma unroll
        for (int v = 0; v < V; v++) Qj[v] = p[v] * acc[v];
        gnormalise<Q>(Qj, mask, zs);
        const int a = gargmax<Q>(Qj, mask, g);
        if (g == 0) xh[j] = (uint8_t)a;
        if (A.post) stv<V>(A.post + ((size_t)f * N + j) * Q + g * V, Qj);
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
#pragma unroll
            for (int v = 0; v < V; v++) {
                const float r = E[k][v];
                E[k][v] = p[v] * (pre[v] * S[k][v]);
                pre[v] *= r;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DV; k++) {
        if (k < d) {
            gnormalise<Q>(E[k], mask, zs);
            if (A.step) stv<V>(A.msg_io + ((size_t)f * A.c.E + eid[k]) * Q + g * V, E[k]);
        }
    }
    if constexpr (METHOD == kDirect) to_relabelled_n<Q, DV>(E, h, d, sc, mask, g, ex, lg);
    else to_deviation_n<Q, DV>(E, h, d, sc, mask, g, ex, lg);
#pragma unroll
    for (int k = 0; k < DV; k++)
        if (k < d) stv<V>(slab + (size_t)eid[k] * Q + g * V, E[k]);
}

// Fold the stored vector y of one more neighbour into check k's accumulator:
// transform route, E <- E + y (1 - E) and the shift XOR; probability route,
// U <- U * y (convolution) in shared memory, batched over the column's checks.
template <int Q, int DV, int METHOD>
__device__ __forceinline__ void fold_round(float (&U)[DV][Lay<Q>::V], int (&C)[DV], bool (&started)[DV],
                                           float (&Y)[DV][Lay<Q>::V], const bool (&take)[DV], float* sc,
                                           unsigned mask, int g) {
    constexpr int V = Lay<Q>::V;
    if constexpr (METHOD == kTransform) {
#pragma unroll
        for (int k = 0; k < DV; k++) {
            if (take[k]) {
                if (g == 0) {
                    C[k] ^= (int)Y[k][0];
                    Y[k][0] = 0.f;
                }
                dev_combine<V>(U[k], Y[k]);
                started[k] = true;
            }
        }
    } else {
        bool conv[DV];
        bool any = false;
#pragma unroll
        for (int k = 0; k < DV; k++) {
            conv[k] = take[k] && started[k];
            if (take[k] && !started[k]) {
#pragma unroll
                for (int v = 0; v < V; v++) U[k][v] = Y[k][v];
                started[k] = true;
            }
            any |= conv[k];
        }
        if (any) {
#pragma unroll
            for (int k = 0; k < DV; k++) {
                if (conv[k]) {
                    stv<V>(sc + (2 * k) * Q + g * V, U[k]);
                    stv<V>(sc + (2 * k + 1) * Q + g * V, Y[k]);
                }
            }
            __syncwarp(mask);
#pragma unroll
            for (int k = 0; k < DV; k++)
                if (conv[k]) xconv_sm<Q>(U[k], sc + (2 * k) * Q, sc + (2 * k + 1) * Q, g);
            __syncwarp(mask);
        }
    }
}

// Per-group shared scratch of the generic SUS routine: one (transform) or two
// (probability route) vector slots per check, + bank padding.
template <int Q, int DV, int METHOD>
constexpr int sus_group_scratch() {
    return (METHOD == kDirect ? 2 : 1) * DV * Q + 4;
}

// One frame's whole SUS decode by the calling lane group (G lanes).
template <int Q, int DC, int DV, int METHOD>
__device__ __forceinline__ void sus_group_frame(const DecodeArgs& A, int f, const uint8_t* s_exp,
                                                const uint8_t* s_log, float* sc) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    // keep both column buffers in registers only while they are small
    constexpr bool PF = (2 * DV * DC * V <= 160);
    const int g = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int lane0 = (threadIdx.x & 31) & ~(G - 1);
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
    if (A.markov_gs && t0 == 0) {
        // Gauss-Seidel priors: before its first visit a source symbol's
        // pseudo-posterior is its initial belief p_j (channel times pi)
        for (int i = 0; i < A.K; i++) {
            float x[V];
            prior_vec<Q>(A, f, A.src_pos[i], x, mask, g);
            stv<V>(A.Qsrc + ((size_t)f * A.K + i) * Q + g * V, x);
        }
        __syncwarp(mask);
    }
    for (;; t++) {
        ColBuf<Q, PF ? DC : 1, PF ? DV : 1> cur, nxt;
        if constexpr (PF) load_col<Q, DC, DV>(cur, A, slab, 0, g);
        for (int j = 0; j < N; j++) {
            if constexpr (PF) {
                if (j + 1 < N) load_col<Q, DC, DV>(nxt, A, slab, j + 1, g);
            }
            if (A.markov_gs) {
                // the block prior of a source symbol, re-estimated (Eq. 6) as the
                // sweep reaches it from its neighbours' current pseudo-posteriors
                const int si = A.src_index[j];
                if (si >= 0) {
                    __syncwarp(mask);   // every lane's part of the latest Q is stored
                    markov_prior<Q>(A, f, si, A.P + ((size_t)f * A.K + si) * Q, mask, g);
                    __syncwarp(mask);
                }
            }
            const int c0 = A.c.colptr[j];
            const int d = A.c.colptr[j + 1] - c0;
            int4 info[DV];
            float U[DV][V];
            int C[DV], eid[DV], h[DV], z[DV], own[DV], dc[DV];
            bool started[DV];
#pragma unroll
            for (int k = 0; k < DV; k++) {
                C[k] = 0;
                started[k] = false;
#pragma unroll
                for (int v = 0; v < V; v++) U[k][v] = 0.f;
                if constexpr (PF) info[k] = cur.info[k];
                else info[k] = (k < d) ? A.c.cinfo[c0 + k] : make_int4(0, 0, 0, 0);
                if (k < d) {
                    eid[k] = info[k].x;
                    h[k] = (info[k].z >> 8) & 255;
                    z[k] = zf ? (zf[info[k].w] & (Q - 1)) : 0;
                    own[k] = info[k].x - info[k].y;
                    dc[k] = info[k].z & 255;
                } else {
                    eid[k] = 0; h[k] = 1; z[k] = 0; own[k] = -1; dc[k] = 0;
                }
            }
            // step 1: fold every other edge of each check of column j
#pragma unroll
            for (int m = 0; m < DC; m++) {
                float Y[DV][V];
                bool take[DV];
#pragma unroll
                for (int k = 0; k < DV; k++) {
                    take[k] = (k < d) && (m < dc[k]) && (m != own[k]);
                    if (take[k]) {
                        if constexpr (PF) {
#pragma unroll
                            for (int v = 0; v < V; v++) Y[k][v] = cur.D[k][m][v];
                        } else {
                            ldv<V>(Y[k], slab + (size_t)(info[k].y + m) * Q + g * V);
                        }
                    }
                }
                fold_round<Q, DV, METHOD>(U, C, started, Y, take, sc, mask, g);
            }
#pragma unroll
            for (int k = 0; k < DV; k++) {
                if constexpr (METHOD == kDirect) {
                    if (k < d && !started[k]) {   // no other edge: y = 0 with certainty
#pragma unroll
                        for (int v = 0; v < V; v++) U[k][v] = (g * V + v) == 0 ? 1.f : 0.f;
                    }
                } else {
                    C[k] = __shfl_sync(mask, C[k], lane0);
                }
            }
            // step 2: q_ij for column j, and Q_j
            sus_column_tail<Q, DV, METHOD>(A, slab, f, j, d, U, C, eid, h, z, xh, sc, mask, g, s_exp, s_log);
            if constexpr (PF) {
                if (j + 1 < N) {
                    if (A.c.cdep[j + 1]) load_col<Q, DC, DV>(nxt, A, slab, j + 1, g);
                    cur = nxt;
                }
            }
        }
        __syncwarp(mask);
        // the hard decisions of the sweep are in xh: test H x = z
        int bad = 0;
        for (int i = g; i < M; i += G) {
            int s = 0;
            for (int e = A.c.rowptr[i]; e < A.c.rowptr[i + 1]; e++)
                s ^= gf_mul(s_exp, s_log, A.c.eh[e], xh[A.c.ecol[e]]);
            bad |= (s != (zf ? (zf[i] & (Q - 1)) : 0));
        }
#pragma unroll
        for (int m = 1; m < G; m <<= 1) bad |= __shfl_xor_sync(mask, bad, m);
        ok = !bad;
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int j = g; j < N; j += G) tr[j] = xh[j];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) {
            fin = true;
            break;
        }
        if (A.markov && !A.markov_gs) {
            for (int i = 0; i < A.K; i++) markov_prior<Q>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, mask, g);
            __syncwarp(mask);
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = 0; i < A.K; i++) markov_prior<Q>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, mask, g);
    }
    if (A.trace) {
        for (size_t o = (size_t)t * N + g; o < (size_t)A.max_iter * N; o += G)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (g == 0) {
        if (!A.fstate || fin) {
            if (A.iters) A.iters[f] = t;
            A.conv[f] = (uint8_t)ok;
        }
        if (A.fstate) A.fstate[f] = fin ? (t | (1 << 30)) : t;
    }
}

template <int Q, int DC, int DV, int METHOD>
__global__ void __launch_bounds__(kSusThreads) k_sus(const DecodeArgs A) {
    constexpr int G = Lay<Q>::G;
    constexpr int SCR = sus_group_scratch<Q, DV, METHOD>();
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ __align__(16) float s_scr[(kSusThreads / G) * SCR];
    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const unsigned mask = group_mask<G>();
    const int lane0 = (threadIdx.x & 31) & ~(G - 1);
    float* sc = s_scr + (tid / G) * SCR;
    for (int k = tid; k < 512; k += blockDim.x) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += blockDim.x) s_log[k] = A.c.glog[k];
    __syncthreads();
    for (;;) {
        int f = 0;
        if (g == 0) f = atomicAdd(A.work, 1);
        f = __shfl_sync(mask, f, lane0);
        if (f >= A.F) break;
        sus_group_frame<Q, DC, DV, METHOD>(A, f, s_exp, s_log, sc);
        __syncwarp(mask);
    }
}

// q_ij <- p_j (Sec. 2 initialisation) or the caller's state, in stored form,
// one lane group per (frame, edge).
template <int Q, int METHOD>
__global__ void __launch_bounds__(256) k_init_dev(const DecodeArgs A) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ __align__(16) float s_scr[256 * V];
    for (int k = threadIdx.x; k < 512; k += blockDim.x) s_exp[k] = A.c.gexp[k];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_log[k] = A.c.glog[k];
    __syncthreads();
    const int g = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    const unsigned mask = group_mask<G>();
    float* sc = s_scr + grp * Q;
    const long long E = A.c.E;
    const long long total = (long long)A.F * E;
    const long long stride = (long long)gridDim.x * (blockDim.x / G);
    for (long long it = (long long)blockIdx.x * (blockDim.x / G) + grp; it < total; it += stride) {
        const int f = (int)(it / E);
        const long long e = it % E;
        float x[V];
        if (A.step) ldv<V>(x, A.msg_io + (size_t)it * Q + g * V);
        else prior_vec<Q>(A, f, A.c.ecol[e], x, mask, g);
        if constexpr (METHOD == kDirect) {
            to_relabelled<Q>(x, A.c.eh[e], sc, mask, g, s_exp, s_log);
        } else if constexpr (METHOD == kTensor) {
            // the plain transform of the relabelled q (FP32 butterflies)
            to_relabelled<Q>(x, A.c.eh[e], sc, mask, g, s_exp, s_log);
            wht<Q>(x, mask, g);
        } else {
            to_deviation<Q>(x, A.c.eh[e], sc, mask, g, s_exp, s_log);
        }
        stv<V>(A.msg + (size_t)it * Q + g * V, x);
    }
}

}  // namespace
}  // namespace gfbp
