// PUS (flooding; Sec. 2) with the probability-domain check node for q <= 16,
// one thread per check in the horizontal pass and one thread per column in
// the vertical pass, whole q-vectors in registers.
//
// A CTA decodes one frame (frames from a global counter) with the frame's
// edge slab updated in place, as the group kernel in pus_frame.cuh does:
// the horizontal pass replaces the stored q of each check's edges by r (Eq. 3:
// suffix convolutions kept in a per-thread shared row, a running prefix, then
// r_k from prefix * suffix), the vertical pass replaces them by the new stored
// q (Eq. 4) and writes Q_j and the hard decision (Eq. 5).  Every convolution
// is q^2 FMAs on registers, with no shared-memory staging of operands; shared
// memory holds only the suffixes and the rows used for the GF relabelling
// gathers.  Each sum and product runs in the group kernel's order, so the two
// kernels give the same bits.
#pragma once

#include "pus_frame.cuh"
#include "sus_level.cuh"

namespace gfbp {

namespace {

// sum of x in the order of gsum<Q>: each lane group's V entries in sequence,
// then a pairwise tree over the G groups.
template <int Q>
__device__ __forceinline__ float gsum_regs(const float (&x)[Q]) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    float s[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < V; i++) a = __fadd_rn(a, x[g * V + i]);
        s[g] = a;
    }
#pragma unroll
    for (int m = 1; m < G; m <<= 1)
#pragma unroll
        for (int g = 0; g < G; g += 2 * m) s[g] = __fadd_rn(s[g], s[g + m]);
    return s[0];
}

template <int Q>
__device__ __forceinline__ void gnormalise_regs(float (&x)[Q], int* zs = nullptr) {
    const float s = gsum_regs<Q>(x);
    if (s > 0.f && s <= 3.0e38f) {
        const float r = 1.0f / s;
#pragma unroll
        for (int i = 0; i < Q; i++) x[i] *= r;
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) x[i] = 1.0f / Q;
        note_zero_sum<1>(zs);
    }
}

// out[y] = sum_x a[x] b[x XOR y], one FMA chain per output in increasing x
// (the order of xconv_sm).
template <int Q>
__device__ __forceinline__ void xconv_chain(float (&out)[Q], const float (&a)[Q], const float (&b)[Q]) {
    xconv_pk<Q>(out, a, b);   // two outputs per packed FMA, each the same chain
}

template <int Q>
__device__ __forceinline__ void ld_row(float (&x)[Q], const float* r) {
#pragma unroll
    for (int i = 0; i < Q; i++) x[i] = r[i];
}

template <int Q>
__device__ __forceinline__ void st_row(float* r, const float (&x)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; i++) r[i] = x[i];
}

// Horizontal pass for check i.  suf: this thread's first suffix row, rows
// `rstride` floats apart; row: this thread's gather row.
template <int Q>
__device__ __forceinline__ void pus_check_regs(const DecodeArgs& A, float* slab, int f, int i, const uint8_t* s_mul,
                                               float* suf, int rstride, float* row) {
    const int e0 = A.c.rowptr[i];
    const int d = A.c.rowptr[i + 1] - e0;
    const int z = A.syn ? (A.syn[(size_t)f * A.c.M + i] & (Q - 1)) : 0;
    const float* D = slab + (size_t)e0 * Q;
    prefetch_l1(D, d * Q * (int)sizeof(float));   // the check's vectors are contiguous
    // S_k = qt_{k+1} * ... * qt_{d-1} for k = d-2 .. 0
    if (d >= 2) {
        float S[Q];
        ldq_g<Q>(S, D + (size_t)(d - 1) * Q);
        st_row<Q>(suf + (d - 2) * rstride, S);
#pragma unroll 1
        for (int k = d - 3; k >= 0; k--) {
            float X[Q], S2[Q];
            ldq_g<Q>(X, D + (size_t)(k + 1) * Q);
            xconv_chain<Q>(S2, S, X);
#pragma unroll
            for (int y = 0; y < Q; y++) S[y] = S2[y];
            st_row<Q>(suf + k * rstride, S);
        }
    }
    float P[Q];
    bool p_id = true;   // P is the identity (no edge folded in yet)
#pragma unroll 1
    for (int k = 0; k < d; k++) {
        float out[Q];
        if (k == d - 1) {
#pragma unroll
            for (int y = 0; y < Q; y++) out[y] = p_id ? (y == 0 ? 1.f : 0.f) : P[y];
        } else if (p_id) {
            ld_row<Q>(out, suf + k * rstride);
        } else {
            float Sk[Q];
            ld_row<Q>(Sk, suf + k * rstride);
            xconv_chain<Q>(out, P, Sk);
        }
        if (k < d - 1) {
            float X[Q];
            ldq_g<Q>(X, D + (size_t)k * Q);   // qt_k, read before r_k replaces it below
            if (p_id) {
#pragma unroll
                for (int y = 0; y < Q; y++) P[y] = X[y];
                p_id = false;
            } else {
                float P2[Q];
                xconv_chain<Q>(P2, P, X);
#pragma unroll
                for (int y = 0; y < Q; y++) P[y] = P2[y];
            }
        }
        // r[a] = s[z XOR h a], normalised
        const int h = A.c.eh[e0 + k];
        st_row<Q>(row, out);
        float R[Q];
#pragma unroll
        for (int a = 0; a < Q; a++) R[a] = row[z ^ s_mul[h * Q + a]];   // both below Q
        gnormalise_regs<Q>(R, zsum_of(A, f));
        stq_g<Q>(slab + (size_t)(e0 + k) * Q, R);
    }
}

// Vertical pass for column j.  rr: this thread's rows for the column's r
// (rows `rstride` floats apart); row: its gather row.
template <int Q>
__device__ __forceinline__ void pus_var_regs(const DecodeArgs& A, float* slab, int f, int j, const uint8_t* s_div,
                                             float* rr, int rstride, float* row) {
    const int c0 = A.c.colptr[j];
    const int d = A.c.colptr[j + 1] - c0;
    const int N = A.c.N;
    for (int k = 0; k < d; k++) prefetch_l1(slab + (size_t)A.c.cedge[c0 + k] * Q, Q * (int)sizeof(float));
    float p[Q];
    ldq_g<Q, true>(p, A.L + ((size_t)f * N + j) * Q);
    int si = -1;
    if (A.markov) {
        si = A.src_index[j];
        if (si >= 0) {
            float P[Q];
            ldq<Q>(P, A.P + ((size_t)f * A.K + si) * Q);
#pragma unroll
            for (int i = 0; i < Q; i++) p[i] *= P[i];
            gnormalise_regs<Q>(p);
        }
    }
    // the column's r (all read before any is overwritten), and their product
    // taken from the last edge to the first
    float acc[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) acc[i] = 1.f;
#pragma unroll 1
    for (int k = d - 1; k >= 0; k--) {
        float R[Q];
        ldq_g<Q>(R, slab + (size_t)A.c.cedge[c0 + k] * Q);
        st_row<Q>(rr + k * rstride, R);
#pragma unroll
        for (int i = 0; i < Q; i++) acc[i] *= R[i];
    }
    {
        float Qj[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) Qj[i] = p[i] * acc[i];
        gnormalise_regs<Q>(Qj, zsum_of(A, f));
        int bi = 0;
        float bv = Qj[0];
#pragma unroll
        for (int i = 1; i < Q; i++)
            if (Qj[i] > bv) { bv = Qj[i]; bi = i; }
        A.xhat[(size_t)f * N + j] = (uint8_t)bi;
        if (A.post) stq<Q>(A.post + ((size_t)f * N + j) * Q, Qj);
        if (si >= 0) stq<Q>(A.Qsrc + ((size_t)f * A.K + si) * Q, Qj);
    }
    float pre[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) pre[i] = 1.f;
#pragma unroll 1
    for (int k = 0; k < d; k++) {
        // S_k = r_{d-1} r_{d-2} ... r_{k+1}, multiplied in that order from 1
        float S[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) S[i] = 1.f;
#pragma unroll 1
        for (int k2 = d - 1; k2 > k; k2--) {
            const float* r = rr + k2 * rstride;
#pragma unroll
            for (int i = 0; i < Q; i++) S[i] *= r[i];
        }
        float x[Q];
        const float* rk = rr + k * rstride;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            x[i] = p[i] * (pre[i] * S[i]);
            pre[i] *= rk[i];
        }
        gnormalise_regs<Q>(x, zsum_of(A, f));
        const int e = A.c.cedge[c0 + k];
        if (A.step) stq<Q>(A.msg_io + ((size_t)f * A.c.E + e) * Q, x);
        // stored form: qt[y] = q[h^-1 y]
        const int h = A.c.eh[e];
        st_row<Q>(row, x);
        float qt[Q];
#pragma unroll
        for (int y = 0; y < Q; y++) qt[y] = row[s_div[h * Q + y]];
        stq_g<Q>(slab + (size_t)e * Q, qt);
    }
}

// Shared rows per thread beside the gather row: the check's suffixes or the
// column's r.
__host__ __device__ constexpr int pus_regs_rows(int dcmax, int dvmax) {
    return (dcmax - 1 > dvmax ? dcmax - 1 : dvmax) > 1 ? (dcmax - 1 > dvmax ? dcmax - 1 : dvmax) : 1;
}

template <int Q, int T>
__device__ __forceinline__ void pus_regs_frame(const DecodeArgs& A, int f, const uint8_t* s_exp, const uint8_t* s_log,
                                               const uint8_t* s_mul, const uint8_t* s_div, float* s_rows,
                                               float* s_gather) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    constexpr int RS = Q + 1;   // row stride: threads' rows on distinct banks
    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const int grp = tid / G;
    constexpr int ngrp = T / G;
    const unsigned mask = group_mask<G>();
    const int M = A.c.M, N = A.c.N;
    const long long E = A.c.E;
    float* slab = A.msg + (size_t)f * E * Q;
    float* rows = s_rows + tid * RS;   // row k of this thread at rows + k * T * RS
    float* grow = s_gather + tid * RS;

    int t0 = 0;   // iterations already done (resumable decoding)
    if (A.fstate) {
        const int st = A.fstate[f];
        if (st >> 30) return;
        t0 = st;
    }
    // q_ij <- p_j (Sec. 2) or the caller's state, in stored form (lane groups,
    // each with Q floats of the gather rows as scratch)
    for (long long e = grp; e < E && t0 == 0; e += ngrp) {
        float x[V];
        if (A.step) {
            ldv<V>(x, A.msg_io + ((size_t)f * E + e) * Q + g * V);
        } else {
            prior_vec<Q>(A, f, A.c.ecol[e], x, mask, g);
        }
        to_relabelled<Q>(x, A.c.eh[e], s_gather + grp * Q, mask, g, s_exp, s_log);
        stv<V>(slab + (size_t)e * Q + g * V, x);
    }
    __syncthreads();

    int t = t0 + 1, ok = 0;
    bool fin = false;
    for (;; t++) {
        for (int i = tid; i < M; i += T) pus_check_regs<Q>(A, slab, f, i, s_mul, rows, T * RS, grow);
        __syncthreads();
        for (int j = tid; j < N; j += T) pus_var_regs<Q>(A, slab, f, j, s_div, rows, T * RS, grow);
        __syncthreads();
        int bad = 0;
        for (int i = tid; i < M; i += T) {
            int s = 0;
            for (int e = A.c.rowptr[i]; e < A.c.rowptr[i + 1]; e++)
                s ^= s_mul[A.c.eh[e] * Q + A.xhat[(size_t)f * N + A.c.ecol[e]]];
            const int z = A.syn ? (A.syn[(size_t)f * M + i] & (Q - 1)) : 0;
            bad |= (s != z);
        }
        ok = !__syncthreads_or(bad);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int j = tid; j < N; j += T) tr[j] = A.xhat[(size_t)f * N + j];
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
        for (size_t o = (size_t)t * N + tid; o < (size_t)A.max_iter * N; o += T)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (tid == 0) {
        if (!A.fstate || fin) {
            if (A.iters) A.iters[f] = t;
            A.conv[f] = (uint8_t)ok;
        }
        if (A.fstate) A.fstate[f] = fin ? (t | (1 << 30)) : t;
    }
}

// Dynamic shared memory: pus_regs_rows(dcmax, dvmax) rows per thread, then
// one gather row per thread.
template <int Q, int T>
__global__ void __launch_bounds__(T) k_pus_regs(const DecodeArgs A) {
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ int s_frame;
    extern __shared__ __align__(16) float s_dyn[];
    const int tid = threadIdx.x;
    const int nrows = pus_regs_rows(A.c.dcmax, A.c.dvmax);
    float* s_rows = s_dyn;
    float* s_gather = s_dyn + (size_t)nrows * T * (Q + 1);
    for (int k = tid; k < 512; k += T) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += T) s_log[k] = A.c.glog[k];
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, T);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_frame = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_frame;
        if (f >= A.F) break;
        pus_regs_frame<Q, T>(A, f, s_exp, s_log, s_mul, s_div, s_rows, s_gather);
    }
}

}  // namespace
}  // namespace gfbp
