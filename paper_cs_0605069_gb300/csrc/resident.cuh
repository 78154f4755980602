// Frame-resident decoders (q <= 16, probability route of Eq. 3): a CTA holds
// one frame's whole edge slab in shared memory from its first iteration to its
// last, so the messages never travel to global memory; per sweep the frame
// reads only its channel likelihoods (and block priors) from global memory.
// A GF(16) code with N = 1000 symbols and degrees (3,6) needs 192 KB, one
// frame per SM; smaller frames share an SM.
//
// Both kernels compute, operation for operation, what the global-memory
// kernels with the same arithmetic compute, so their results are the same
// bits:
//   k_pus_res  the flooding schedule of pus_regs.cuh (a thread per check in
//              the horizontal pass, a thread per column in the vertical one);
//   k_sus_res  the sequential schedule by levels with running partial
//              convolutions (sus_level.cuh with RUNNING partials).
//
// Every XOR-convolution (U (*) Y)[y] = sum_x U[x] Y[x XOR y] is the same FMA
// chain per output, in increasing x, as xconv_regs; the outputs are formed in
// pairs (y, y XOR 1) by packed FP32 FMAs (two independent round-to-nearest
// FMAs per instruction), which halves the instruction count of the q^2 FMAs
// without changing a bit.
//
// Shared-memory layout.  The slots of check i (its d edge vectors, in edge
// order) are contiguous and followed by res_pad<Q>() floats of padding, so
// that the slot of edge e of row i starts res_slot(e, i) = e q + pad i floats
// into the slab: with a (3,6) code every check would otherwise start at a
// multiple of 384 bytes, and the threads that work on consecutive checks would
// all meet in the same shared-memory banks (8-way conflicts on every 16-byte
// access); with the padding eight consecutive checks start in distinct bank
// groups.
//
// In-place storage.  PUS: the horizontal pass of check i keeps the inner
// messages of the check in registers and overwrites the check's slots first
// with the prefix convolutions, then with r; the vertical pass of column j
// reads its r into registers and overwrites them with the new stored q.
// SUS: at the start of a sweep, slot m (1 <= m <= d-2) of check i becomes the
// suffix convolution S[m] of the sweep-start messages of positions m..d-1 and
// slot 0 the running prefix P; the visit of position t reads P and S[t+1]
// (the last message itself when t+1 = d-1) and afterwards stores the new
// message in slot t, whose suffix is no longer needed.  The message of
// position 0 is never read again within a sweep nor by the next sweep's
// suffixes (they start at position 1), so slot 0 can hold P.
#pragma once

#include "pus_regs.cuh"
#include "sus_level.cuh"

namespace gfbp {

namespace {

// ---------------------------------------------------------------- helpers

// A q-vector in shared memory (16-byte aligned for q >= 4).
template <int Q>
__device__ __forceinline__ void lds_q(float (&x)[Q], const float* p) {
    if constexpr (Q == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        x[0] = a.x; x[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < Q; i += 4) {
            const float4 a = *reinterpret_cast<const float4*>(p + i);
            x[i] = a.x; x[i + 1] = a.y; x[i + 2] = a.z; x[i + 3] = a.w;
        }
    }
}

template <int Q>
__device__ __forceinline__ void sts_q(float* p, const float (&x)[Q]) {
    if constexpr (Q == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
    }
}

// Padding (floats) after the slots of every check.
template <int Q>
__host__ __device__ constexpr int res_pad() { return Q >= 4 ? 4 : 2; }

// Offset (floats) of the slot of edge e, which belongs to row i.
template <int Q>
__device__ __forceinline__ int res_slot(int e, int i) { return e * Q + res_pad<Q>() * i; }

// Floats of the padded slab.
template <int Q>
__host__ __device__ constexpr size_t res_slab_floats(long long E, int M) {
    return (size_t)E * Q + (size_t)res_pad<Q>() * M;
}

// r[a] = s[z XOR h a] through the vector's own slot (the calling thread wrote
// s there), normalised in the lane-group order (gsum) as the PUS kernels do,
// written back to the slot.
template <int Q>
__device__ __forceinline__ void res_finish_r_g(float* slot, const float (&s)[Q], int z, int h,
                                               const uint8_t* s_mul, int* zs) {
    sts_q<Q>(slot, s);
    float R[Q];
#pragma unroll
    for (int a = 0; a < Q; a++) R[a] = slot[z ^ s_mul[h * Q + a]];
    gnormalise_regs<Q>(R, zs);
    sts_q<Q>(slot, R);
}

// Stored form qt[y] = x[h^-1 y] of a normalised message, through its slot.
template <int Q>
__device__ __forceinline__ void res_store_relabelled(float* slot, const float (&x)[Q], int h, const uint8_t* s_div) {
    sts_q<Q>(slot, x);
    float qt[Q];
#pragma unroll
    for (int y = 0; y < Q; y++) qt[y] = slot[s_div[h * Q + y]];
    sts_q<Q>(slot, qt);
}

// p_j of a column: channel likelihood times its block prior, normalised in
// the lane-group order of prior_vec (the initialisation kernels' order).
template <int Q>
__device__ __forceinline__ void res_prior_g(const DecodeArgs& A, int f, int j, float (&x)[Q]) {
    if (A.markov) {
        const int si = A.src_index[j];
        if (si >= 0) {
            float P[Q];
            ldq<Q>(P, A.P + ((size_t)f * A.K + si) * Q);
#pragma unroll
            for (int i = 0; i < Q; i++) x[i] *= P[i];
            gnormalise_regs<Q>(x);
        }
    }
}

// q_ij <- p_j (Sec. 2 initialisation) or the caller's state, in stored form,
// for every edge; four edges at a time so that their loads overlap.
template <int Q, int T>
__device__ __forceinline__ void res_init_edges(const DecodeArgs& A, int f, float* X, const uint8_t* s_div) {
    const int E = (int)A.c.E;
    constexpr int B = 4;
    for (int e0 = threadIdx.x; e0 < E; e0 += B * T) {
        int col[B], row[B];
        float x[B][Q];
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            col[b] = (e < E && !A.step) ? A.c.ecol[e] : 0;
            row[b] = e < E ? A.c.erow[e] : 0;
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            if (e < E) {
                if (A.step) ldq<Q>(x[b], A.msg_io + ((size_t)f * E + e) * Q);
                else ldgq<Q>(x[b], A.L + ((size_t)f * A.c.N + col[b]) * Q);
            }
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            if (e < E) {
                if (!A.step) res_prior_g<Q>(A, f, col[b], x[b]);
                res_store_relabelled<Q>(X + res_slot<Q>(e, row[b]), x[b], A.c.eh[e], s_div);
            }
        }
    }
}

// Every check satisfied?  hx[res_slot(e, i) / q] holds h_e x^_j for the
// column j of edge e (contiguous over a row's edges).  Call with all threads;
// ends with a barrier.
template <int Q, int T>
__device__ __forceinline__ bool res_syndrome_ok(int M, const int* s_rowptr, const uint8_t* s_hx,
                                                const uint8_t* s_z) {
    int bad = 0;
    for (int i = threadIdx.x; i < M; i += T) {
        int s = 0;
        const int e0 = s_rowptr[i];
        const int d = s_rowptr[i + 1] - e0;
        const uint8_t* hx = s_hx + res_slot<Q>(e0, i) / Q;
        for (int m = 0; m < d; m++) s ^= hx[m];
        bad |= (s != (s_z ? (s_z[i] & (Q - 1)) : 0));
    }
    return !__syncthreads_or(bad);
}

// Lowest index of the largest entry.
template <int Q>
__device__ __forceinline__ int argmax_regs(const float (&x)[Q]) {
    int bi = 0;
    float bv = x[0];
#pragma unroll
    for (int i = 1; i < Q; i++)
        if (x[i] > bv) { bv = x[i]; bi = i; }
    return bi;
}

// Shared-memory layout of a resident frame, each part 16-byte aligned:
//   X: the padded slab | rows [kLevelPiece][level_rs] (SUS) | rowptr [M+1] |
//   eh [E], colptr [N+1], cslot [E] (uint16), ch [E] (PUS) |
//   lpiece [npieces+1] (SUS) | hx | xh [N] | z [M].
// PUS: cslot and ch list, per column slot (colptr order), the edge's slot
// offset in units of res_pad<Q>() floats and its GF value.
struct ResParts {
    size_t X, rows, rowptr, eh, colptr, cslot, ch, lpiece, hx, xh, z, total;
};

__host__ __device__ constexpr size_t res_align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int Q, bool SUS>
__host__ __device__ constexpr ResParts res_parts(long long E, int M, int N, int npieces) {
    ResParts o{};
    size_t a = 0;
    o.X = a; a += res_align16(sizeof(float) * res_slab_floats<Q>(E, M));
    o.rows = a; if (SUS) a += res_align16(sizeof(float) * (size_t)kLevelPiece * level_rs<Q>());
    o.rowptr = a; a += res_align16(sizeof(int) * (size_t)(M + 1));
    o.eh = a; if (!SUS) a += res_align16((size_t)E);
    o.colptr = a; if (!SUS) a += res_align16(sizeof(int) * (size_t)(N + 1));
    o.cslot = a; if (!SUS) a += res_align16(sizeof(uint16_t) * (size_t)E);
    o.ch = a; if (!SUS) a += res_align16((size_t)E);
    o.lpiece = a; if (SUS) a += res_align16(sizeof(int) * (size_t)(npieces + 1));
    o.hx = a; a += res_align16(res_slab_floats<Q>(E, M) / Q + 1);
    o.xh = a; a += res_align16((size_t)N);
    o.z = a; a += res_align16((size_t)M);
    o.total = a;
    return o;
}

// Shared memory of a SUS frame (each part 16-byte aligned): the padded slab
// (SM only) | rows [kLevelPiece][level_rs] | scratch rows [kLevelPiece][level_rs]
// (global slab only) | rowptr [M+1] | lpiece [npieces+1] | hx | xh [N] | z [M].
struct ResSusParts {
    size_t X, rows, scr, rowptr, lpiece, hx, xh, z, total;
};

template <int Q, bool SM>
__host__ __device__ constexpr ResSusParts res_sus_parts(long long E, int M, int N, int npieces) {
    ResSusParts o{};
    size_t a = 0;
    const size_t rowb = res_align16(sizeof(float) * (size_t)kLevelPiece * level_rs<Q>());
    o.X = a; if (SM) a += res_align16(sizeof(float) * res_slab_floats<Q>(E, M));
    o.rows = a; a += rowb;
    o.scr = a; if (!SM) a += rowb;
    o.rowptr = a; a += res_align16(sizeof(int) * (size_t)(M + 1));
    o.lpiece = a; a += res_align16(sizeof(int) * (size_t)(npieces + 1));
    o.hx = a; a += res_align16((SM ? res_slab_floats<Q>(E, M) / Q : (size_t)E) + 1);
    o.xh = a; a += res_align16((size_t)N);
    o.z = a; a += res_align16((size_t)M);
    o.total = a;
    return o;
}

// Outputs of a finished frame (hard decisions from shared memory, trace
// padding, block priors of gfbp_step, iteration count, flag).
template <int Q, int T, bool SUS>
__device__ __forceinline__ void res_finish_frame(const DecodeArgs& A, int f, int t, int ok, const uint8_t* s_xh) {
    const int N = A.c.N;
    const int tid = threadIdx.x;
    for (int j = tid; j < N; j += T) A.xhat[(size_t)f * N + j] = s_xh[j];
    if (A.step && A.markov && A.prior_out) {
        if constexpr (SUS) {
            const int lane = tid & 31, warp = tid >> 5;
            for (int i = warp; i < A.K; i += T / 32)
                team_prior<Q, 32>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, 0xffffffffu, lane);
        } else {
            constexpr int G = Lay<Q>::G;
            const unsigned mask = group_mask<G>();
            for (int i = tid / G; i < A.K; i += T / G)
                markov_prior<Q>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, mask, tid & (G - 1));
        }
    }
    if (A.trace) {
        for (size_t o = (size_t)t * N + tid; o < (size_t)A.max_iter * N; o += T)
            A.trace[(size_t)f * A.max_iter * N + o] = 255;
    }
    if (tid == 0) {
        if (A.iters) A.iters[f] = t;
        A.conv[f] = (uint8_t)ok;
    }
}

// ------------------------------------------------------------------- PUS

// The code's arrays a PUS frame reads, in shared memory.
struct ResPusCode {
    const int* rowptr;
    const uint8_t* eh;       // [E] GF value of each edge
    const int* colptr;
    const uint16_t* cslot;   // per column slot: the edge's slot offset / res_pad
    const uint8_t* ch;       // per column slot: the edge's GF value
};

// Horizontal pass for check i (Eq. 3), in the arithmetic of pus_check_regs:
// suffixes S_k = S_{k+1} (*) qt_{k+1} from S_{d-2} = qt_{d-1}, prefixes
// P_1 = qt_0, P_{k+1} = P_k (*) qt_k, r_0 = S_0, r_k = P_k (*) S_k,
// r_{d-1} = P_{d-1}.  The inner messages qt_1..qt_{d-2} wait in registers
// while their slots hold the prefixes.
template <int Q, int DC>
__device__ __forceinline__ void res_pus_check(const ResPusCode& C, float* X, int i, const uint8_t* s_z,
                                              const uint8_t* s_mul, int* zs) {
    const int e0 = C.rowptr[i];
    const int d = C.rowptr[i + 1] - e0;
    const int z = s_z ? (s_z[i] & (Q - 1)) : 0;
    float* D = X + res_slot<Q>(e0, i);
    if (d == 0) return;   // an empty row of H
    if (d == 1) {
        float s[Q];
#pragma unroll
        for (int y = 0; y < Q; y++) s[y] = y == 0 ? 1.f : 0.f;
        res_finish_r_g<Q>(D, s, z, C.eh[e0], s_mul, zs);
        return;
    }
    // forward: prefixes into the inner slots
    float inner[DC > 2 ? DC - 2 : 1][Q];
    float P[Q];
    lds_q<Q>(P, D);
#pragma unroll
    for (int k = 1; k < DC - 1; k++) {
        if (k < d - 1) {
            lds_q<Q>(inner[k - 1], D + (size_t)k * Q);
            sts_q<Q>(D + (size_t)k * Q, P);
            float P2[Q];
            xconv_pk<Q>(P2, P, inner[k - 1]);
#pragma unroll
            for (int y = 0; y < Q; y++) P[y] = P2[y];
        }
    }
    // backward: suffixes in registers, r into every slot
    float S[Q];
    lds_q<Q>(S, D + (size_t)(d - 1) * Q);
    res_finish_r_g<Q>(D + (size_t)(d - 1) * Q, P, z, C.eh[e0 + d - 1], s_mul, zs);
#pragma unroll
    for (int k = DC - 2; k >= 1; k--) {
        if (k < d - 1) {
            float Pk[Q], out[Q];
            lds_q<Q>(Pk, D + (size_t)k * Q);
            xconv_pk<Q>(out, Pk, S);
            res_finish_r_g<Q>(D + (size_t)k * Q, out, z, C.eh[e0 + k], s_mul, zs);
            float S2[Q];
            xconv_pk<Q>(S2, S, inner[k - 1]);
#pragma unroll
            for (int y = 0; y < Q; y++) S[y] = S2[y];
        }
    }
    res_finish_r_g<Q>(D, S, z, C.eh[e0], s_mul, zs);
}

// Vertical pass for column j (Eqs. 4-5) in the arithmetic of pus_var_regs; p
// holds the column's channel likelihood (loaded ahead by the caller).  The
// column's r stay in their slots (only this thread touches them) and are read
// again where needed: slot k is overwritten by the new q of edge k after
// every product that uses r_k.
template <int Q, int DV>
__device__ __forceinline__ void res_pus_var(const DecodeArgs& A, const ResPusCode& C, float* X, int f, int j,
                                            float (&p)[Q], uint8_t* s_xh, uint8_t* s_hx, const uint8_t* s_mul,
                                            const uint8_t* s_div) {
    constexpr int PAD = res_pad<Q>();
    const int c0 = C.colptr[j];
    const int d = C.colptr[j + 1] - c0;
    const int N = A.c.N;
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
    int so[DV];   // slot offsets (floats)
#pragma unroll
    for (int k = 0; k < DV; k++) so[k] = k < d ? (int)C.cslot[c0 + k] * PAD : 0;
    float acc[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) acc[i] = 1.f;
#pragma unroll
    for (int k = DV - 1; k >= 0; k--) {
        if (k < d) {
            float R[Q];
            lds_q<Q>(R, X + so[k]);
#pragma unroll
            for (int i = 0; i < Q; i++) acc[i] *= R[i];
        }
    }
    {
        float Qj[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) Qj[i] = p[i] * acc[i];
        gnormalise_regs<Q>(Qj, zsum_of(A, f));
        const int bi = argmax_regs<Q>(Qj);
        s_xh[j] = (uint8_t)bi;
#pragma unroll
        for (int k = 0; k < DV; k++)
            if (k < d) s_hx[so[k] / Q] = s_mul[C.ch[c0 + k] * Q + bi];
        if (A.post) stq<Q>(A.post + ((size_t)f * N + j) * Q, Qj);
        if (si >= 0) stq<Q>(A.Qsrc + ((size_t)f * A.K + si) * Q, Qj);
    }
    float pre[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) pre[i] = 1.f;
#pragma unroll
    for (int k = 0; k < DV; k++) {
        if (k < d) {
            float S[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) S[i] = 1.f;
#pragma unroll
            for (int k2 = DV - 1; k2 > k; k2--) {
                if (k2 < d) {
                    float R[Q];
                    lds_q<Q>(R, X + so[k2]);
#pragma unroll
                    for (int i = 0; i < Q; i++) S[i] *= R[i];
                }
            }
            float R[Q], x[Q];
            lds_q<Q>(R, X + so[k]);
#pragma unroll
            for (int i = 0; i < Q; i++) {
                x[i] = p[i] * (pre[i] * S[i]);
                pre[i] *= R[i];
            }
            gnormalise_regs<Q>(x, zsum_of(A, f));
            if (A.step) stq<Q>(A.msg_io + ((size_t)f * A.c.E + A.c.cedge[c0 + k]) * Q, x);
            res_store_relabelled<Q>(X + so[k], x, C.ch[c0 + k], s_div);
        }
    }
}

// q_ij <- p_j (Sec. 2 initialisation) or the caller's state, a thread per
// column, the likelihood loaded one column ahead.
template <int Q, int T>
__device__ __forceinline__ void res_pus_init(const DecodeArgs& A, const ResPusCode& C, int f, float* X,
                                             const uint8_t* s_div) {
    constexpr int PAD = res_pad<Q>();
    const int N = A.c.N;
    const int tid = threadIdx.x;
    float pn[Q];
    if (tid < N && !A.step) ldgq<Q>(pn, A.L + ((size_t)f * N + tid) * Q);
    for (int j = tid; j < N; j += T) {
        float p[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) p[i] = pn[i];
        if (!A.step) {
            if (j + T < N) ldgq<Q>(pn, A.L + ((size_t)f * N + j + T) * Q);
            res_prior_g<Q>(A, f, j, p);
        }
        for (int c = C.colptr[j]; c < C.colptr[j + 1]; c++) {
            float x[Q];
            if (A.step) {
                ldq<Q>(x, A.msg_io + ((size_t)f * A.c.E + A.c.cedge[c]) * Q);
            } else {
#pragma unroll
                for (int i = 0; i < Q; i++) x[i] = p[i];
            }
            res_store_relabelled<Q>(X + (int)C.cslot[c] * PAD, x, C.ch[c], s_div);
        }
    }
}

template <int Q, int T, int DC, int DV>
__device__ __forceinline__ void res_pus_frame(const DecodeArgs& A, int f, const ResPusCode& C,
                                              const uint8_t* s_mul, const uint8_t* s_div, float* X, uint8_t* s_hx,
                                              uint8_t* s_xh, uint8_t* s_z) {
    constexpr int G = Lay<Q>::G;
    const int tid = threadIdx.x;
    const int M = A.c.M, N = A.c.N;
    const unsigned mask = group_mask<G>();
    if (s_z)
        for (int i = tid; i < M; i += T) s_z[i] = A.syn[(size_t)f * M + i];
    res_pus_init<Q, T>(A, C, f, X, s_div);
    __syncthreads();
    int t = 1, ok = 0;
    for (;; t++) {
        for (int i = tid; i < M; i += T) res_pus_check<Q, DC>(C, X, i, s_z, s_mul, zsum_of(A, f));
        __syncthreads();
        {
            // each column's likelihood is loaded one column ahead
            float p[Q], pn[Q];
            if (tid < N) ldq_g<Q, true>(pn, A.L + ((size_t)f * N + tid) * Q);
            for (int j = tid; j < N; j += T) {
#pragma unroll
                for (int i = 0; i < Q; i++) p[i] = pn[i];
                if (j + T < N) ldq_g<Q, true>(pn, A.L + ((size_t)f * N + j + T) * Q);
                res_pus_var<Q, DV>(A, C, X, f, j, p, s_xh, s_hx, s_mul, s_div);
            }
        }
        __syncthreads();
        ok = res_syndrome_ok<Q, T>(M, C.rowptr, s_hx, s_z);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int j = tid; j < N; j += T) tr[j] = s_xh[j];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) break;
        if (A.markov) {
            for (int i = tid / G; i < A.K; i += T / G)
                markov_prior<Q>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, mask, tid & (G - 1));
            __syncthreads();
        }
    }
    res_finish_frame<Q, T, false>(A, f, t, ok, s_xh);
}

template <int Q, int T, int DC, int DV>
__global__ void __launch_bounds__(T) k_pus_res(const DecodeArgs A) {
    constexpr int PAD = res_pad<Q>();
    __shared__ uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ int s_f;
    extern __shared__ __align__(16) uint8_t s_res[];
    const int tid = threadIdx.x;
    const int M = A.c.M, N = A.c.N, E = (int)A.c.E;
    const ResParts sp = res_parts<Q, false>(E, M, N, 0);
    float* X = reinterpret_cast<float*>(s_res + sp.X);
    int* rowptr = reinterpret_cast<int*>(s_res + sp.rowptr);
    uint8_t* eh = s_res + sp.eh;
    int* colptr = reinterpret_cast<int*>(s_res + sp.colptr);
    uint16_t* cslot = reinterpret_cast<uint16_t*>(s_res + sp.cslot);
    uint8_t* ch = s_res + sp.ch;
    uint8_t* s_hx = s_res + sp.hx;
    uint8_t* s_xh = s_res + sp.xh;
    uint8_t* s_z = A.syn ? s_res + sp.z : nullptr;
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, T);
    for (int i = tid; i <= M; i += T) rowptr[i] = A.c.rowptr[i];
    for (int j = tid; j <= N; j += T) colptr[j] = A.c.colptr[j];
    for (int e = tid; e < E; e += T) {
        eh[e] = A.c.eh[e];
        const int ed = A.c.cedge[e];   // e indexes the column slots here
        cslot[e] = (uint16_t)(res_slot<Q>(ed, A.c.erow[ed]) / PAD);
        ch[e] = A.c.eh[ed];
    }
    const ResPusCode C{rowptr, eh, colptr, cslot, ch};
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        res_pus_frame<Q, T, DC, DV>(A, f, C, s_mul, s_div, X, s_hx, s_xh, s_z);
    }
}

// ------------------------------------------------------------------- SUS
//
// A thread per (column, check) pair of a piece (kLevelPiece threads).  Two
// homes for a frame's slab: shared memory (SM = true: padded slots, one frame
// per CTA, a GF(16) N = 1000 frame fills an SM), or a slab of the workspace
// per CTA (SM = false: unpadded slots; the launcher runs only as many CTAs as
// keep every CTA's slab in L2, several per SM, so that their latencies
// overlap).  Either way the messages stay on chip between sweeps.

// The (padding-aware) slot offset of edge e of row i.
template <int Q, bool SM>
__device__ __forceinline__ int sus_slot(int e, int i) { return SM ? res_slot<Q>(e, i) : e * Q; }

// A q-vector of the slab (shared or global memory, 16-byte aligned for q >= 4).
template <int Q>
__device__ __forceinline__ void ld_slab(float (&x)[Q], const float* p) { lds_q<Q>(x, p); }
template <int Q>
__device__ __forceinline__ void st_slab(float* p, const float (&x)[Q]) { sts_q<Q>(p, x); }

// Step 0 of a sweep: slot m of every check (1 <= m <= d-2) becomes
// S[m] = S[m+1] (*) qt_m from S[d-1] = qt_{d-1} (level_suffixes' order).
template <int Q, bool SM>
__device__ __forceinline__ void res_sus_suffixes(int M, const int* s_rowptr, float* X) {
    for (int i = threadIdx.x; i < M; i += kLevelPiece) {
        const int e0 = s_rowptr[i];
        const int d = s_rowptr[i + 1] - e0;
        if (d < 3) continue;
        float* D = X + sus_slot<Q, SM>(e0, i);
        float U[Q];
        ld_slab<Q>(U, D + (size_t)(d - 1) * Q);
#pragma unroll 1
        for (int m = d - 2; m >= 1; m--) {
            float Y[Q], o[Q];
            ld_slab<Q>(Y, D + (size_t)m * Q);
            xconv_pk<Q>(o, U, Y);
            st_slab<Q>(D + (size_t)m * Q, o);
#pragma unroll
            for (int y = 0; y < Q; y++) U[y] = o[y];
        }
    }
}

// What a thread needs from global memory for its pair of a piece, loaded one
// piece ahead: the pair's records (ra = the slot's cinfo {edge, row start,
// row degree | h << 8, row}; rb = {column, slot | row index << 8, column
// degree, 0}) and the column's channel likelihood.
template <int Q>
struct ResPair {
    int4 ra, rb;
    float L[Q];
};

template <int Q>
__device__ __forceinline__ void res_pair_load(ResPair<Q>& w, const DecodeArgs& A, int f, int idx) {
    w.ra = A.c.lrec[2 * (size_t)idx];
    w.rb = A.c.lrec[2 * (size_t)idx + 1];
    ldq_g<Q, true>(w.L, A.L + ((size_t)f * A.c.N + w.rb.x) * Q);
}

// Step 1 for the pair: r of the column's k-th check into its row
// (level_check_run's arithmetic with the partials in the slab's slots).
template <int Q, bool SM>
__device__ __forceinline__ void res_sus_check(const float* X, const uint8_t* s_z, const ResPair<Q>& w,
                                              const uint8_t* s_mul, float* row, int* zs) {
    if (w.rb.z == 0) return;   // a column without checks
    const int4 in = w.ra;
    const int t = in.x - in.y;
    const int dc = in.z & 255;
    const int h = (in.z >> 8) & 255;
    const int z = s_z ? (s_z[in.w] & (Q - 1)) : 0;
    const float* D = X + sus_slot<Q, SM>(in.y, in.w);
    float U[Q];
    if (dc == 1) {
        // a check of degree 1: the XOR-sum of no other edges is 0
#pragma unroll
        for (int i = 0; i < Q; i++) U[i] = i == 0 ? 1.f : 0.f;
    } else if (t == 0) {
        ld_slab<Q>(U, D + Q);   // S[1] (the last message when d = 2)
    } else {
        ld_slab<Q>(U, D);       // the prefix P
        if (t < dc - 1) {
            float Y[Q], o[Q];
            ld_slab<Q>(Y, D + (size_t)(t + 1) * Q);   // S[t+1], or the last message
            xconv_pk<Q>(o, U, Y);
#pragma unroll
            for (int i = 0; i < Q; i++) U[i] = o[i];
        }
    }
    st_lrow<Q>(row, U);
    float R[Q];
    gather_row<Q>(R, row, s_mul + h * Q, z);   // r[a] = s[z XOR h a]
    normalise_regs<Q>(R, zs);
    st_lrow<Q>(row, R);
}

// Step 2 for the pair: q of (j, k) from p_j and the column's other rows (and
// for slot 0 Q_j, the hard decision, the posterior), stored relabelled in the
// pair's slot; the check's prefix takes in the new message (level_var's
// arithmetic).  Every pair forms the column's hard decision to record
// h x^_j on its edge for the syndrome.  scr: Q floats of scratch for the
// relabelling (the pair's own slot when the slab is in shared memory).
template <int Q, bool SM>
__device__ __forceinline__ void res_sus_var(const DecodeArgs& A, int f, float* X, uint8_t* s_xh, uint8_t* s_hx,
                                            const ResPair<Q>& w, const float* row, const uint8_t* s_mul,
                                            const uint8_t* s_div, float* scr) {
    const int j = w.rb.x, k = w.rb.y & 255, d = w.rb.z;
    const int4 in = w.ra;
    const int h = (in.z >> 8) & 255;
    const int N = A.c.N;
    float p[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) p[i] = w.L[i];
    const int si = A.markov ? A.src_index[j] : -1;   // a Markov source symbol: its block prior
    if (si >= 0) {
        float P[Q];
        ldq<Q>(P, A.P + ((size_t)f * A.K + si) * Q);
#pragma unroll
        for (int i = 0; i < Q; i++) p[i] *= P[i];
        normalise_regs<Q>(p);
    }
    float other[Q], all[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) { other[i] = p[i]; all[i] = p[i]; }
    constexpr int RS = level_rs<Q>();
    const float* r0 = row - (size_t)k * RS;   // row of the column's slot 0
#pragma unroll 1
    for (int k2 = 0; k2 < d; k2++) {
        float r[Q];
        ld_lrow<Q>(r, r0 + (size_t)k2 * RS);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            all[i] *= r[i];
            if (k2 != k) other[i] *= r[i];
        }
    }
    normalise_regs<Q>(all, k == 0 ? zsum_of(A, f) : nullptr);
    const int bi = argmax_regs<Q>(all);
    if (k == 0) {
        s_xh[j] = (uint8_t)bi;
        if (A.post) stq<Q>(A.post + ((size_t)f * N + j) * Q, all);
        if (si >= 0) stq<Q>(A.Qsrc + ((size_t)f * A.K + si) * Q, all);
    }
    if (d == 0) return;
    const int so = sus_slot<Q, SM>(in.x, in.w);
    s_hx[so / Q] = s_mul[h * Q + bi];
    normalise_regs<Q>(other, zsum_of(A, f));
    if (A.step) stq<Q>(A.msg_io + ((size_t)f * A.c.E + in.x) * Q, other);
    // stored form qt[y] = q[h^-1 y]
    st_lrow<Q>(scr, other);
    float qt[Q];
    gather_row<Q>(qt, scr, s_div + h * Q, 0);
    float* slot = X + so;
    st_slab<Q>(slot, qt);
    const int t = in.x - in.y;
    if (t > 0 && t < (in.z & 255) - 1) {   // (t = 0: the slot is the prefix already)
        float* P = X + sus_slot<Q, SM>(in.y, in.w);
        float U[Q], o[Q];
        ld_slab<Q>(U, P);
        xconv_pk<Q>(o, U, qt);
        st_slab<Q>(P, o);
    }
}

// Every check satisfied?  hx[slot / q] holds h_e x^_j for the column j of the
// slot's edge (contiguous over a row's edges).  All threads; ends with a barrier.
template <int Q, bool SM>
__device__ __forceinline__ bool res_sus_syndrome_ok(int M, const int* s_rowptr, const uint8_t* s_hx,
                                                    const uint8_t* s_z) {
    int bad = 0;
    for (int i = threadIdx.x; i < M; i += kLevelPiece) {
        int s = 0;
        const int e0 = s_rowptr[i];
        const int d = s_rowptr[i + 1] - e0;
        const uint8_t* hx = s_hx + sus_slot<Q, SM>(e0, i) / Q;
        for (int m = 0; m < d; m++) s ^= hx[m];
        bad |= (s != (s_z ? (s_z[i] & (Q - 1)) : 0));
    }
    return !__syncthreads_or(bad);
}

// q_ij <- p_j (Sec. 2 initialisation) or the caller's state, in stored form,
// for every edge; four edges at a time so that their loads overlap.  scr: the
// thread's scratch row for the relabelling (global slab), or nullptr to pass
// through each edge's own slot (shared-memory slab).
template <int Q, bool SM>
__device__ __forceinline__ void res_sus_init(const DecodeArgs& A, int f, float* X, const uint8_t* s_div,
                                             float* scr) {
    constexpr int T = kLevelPiece;
    const int E = (int)A.c.E;
    constexpr int B = 4;
    for (int e0 = threadIdx.x; e0 < E; e0 += B * T) {
        int col[B], row[B];
        float x[B][Q];
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            col[b] = (e < E && !A.step) ? A.c.ecol[e] : 0;
            row[b] = (e < E && SM) ? A.c.erow[e] : 0;
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            if (e < E) {
                if (A.step) ldq<Q>(x[b], A.msg_io + ((size_t)f * E + e) * Q);
                else ldgq<Q>(x[b], A.L + ((size_t)f * A.c.N + col[b]) * Q);
            }
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int e = e0 + b * T;
            if (e < E) {
                if (!A.step) res_prior_g<Q>(A, f, col[b], x[b]);
                float* slot = X + sus_slot<Q, SM>(e, row[b]);
                float* sc = SM ? slot : scr;
                st_lrow<Q>(sc, x[b]);
                float qt[Q];
                gather_row<Q>(qt, sc, s_div + A.c.eh[e] * Q, 0);
                st_slab<Q>(slot, qt);
            }
        }
    }
}

// One frame by a CTA of kLevelPiece threads: each takes at most one pair of a
// piece.
template <int Q, bool SM>
__device__ __forceinline__ void res_sus_frame(const DecodeArgs& A, int f, const uint8_t* s_mul,
                                              const uint8_t* s_div, float* X, float* s_rows, float* s_scr,
                                              const int* s_rowptr, const int* s_lp, uint8_t* s_hx, uint8_t* s_xh,
                                              uint8_t* s_z) {
    constexpr int T = kLevelPiece;
    constexpr int RS = level_rs<Q>();
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int M = A.c.M, N = A.c.N;
    const int np = A.c.npieces;
    float* scr = SM ? nullptr : s_scr + (size_t)tid * RS;   // (no scratch rows with the slab in shared memory)
    if (s_z)
        for (int i = tid; i < M; i += T) s_z[i] = A.syn[(size_t)f * M + i];
    res_sus_init<Q, SM>(A, f, X, s_div, scr);
    ResPair<Q> cur;
    cur.rb = make_int4(0, 0, 0, 0);
    if (np > 0 && tid < s_lp[1] - s_lp[0]) res_pair_load<Q>(cur, A, f, s_lp[0] + tid);
    __syncthreads();
    int t = 1, ok = 0;
    for (;; t++) {
        res_sus_suffixes<Q, SM>(M, s_rowptr, X);
        __syncthreads();
#pragma unroll 1
        for (int pc = 0; pc < np; pc++) {
            const int n = s_lp[pc + 1] - s_lp[pc];
            // the next piece's pair (the first piece again after the last),
            // arriving while this one is processed
            const int pn = pc + 1 < np ? pc + 1 : 0;
            ResPair<Q> nxt;
            nxt.rb = make_int4(0, 0, 0, 0);
            if (tid < s_lp[pn + 1] - s_lp[pn]) res_pair_load<Q>(nxt, A, f, s_lp[pn] + tid);
            float* row = s_rows + ((cur.rb.y >> 8) & 255) * RS;
            if (tid < n) res_sus_check<Q, SM>(X, s_z, cur, s_mul, row, zsum_of(A, f));
            __syncthreads();
            if (tid < n) {
                float* sc = SM ? X + sus_slot<Q, SM>(cur.ra.x, cur.ra.w) : scr;
                res_sus_var<Q, SM>(A, f, X, s_xh, s_hx, cur, row, s_mul, s_div, sc);
            }
            __syncthreads();
            cur = nxt;
        }
        ok = res_sus_syndrome_ok<Q, SM>(M, s_rowptr, s_hx, s_z);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int jj = tid; jj < N; jj += T) tr[jj] = s_xh[jj];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) break;
        if (A.markov) {
            for (int i = warp; i < A.K; i += T / 32)
                team_prior<Q, 32>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, 0xffffffffu, lane);
            __syncthreads();
        }
    }
    res_finish_frame<Q, T, true>(A, f, t, ok, s_xh);
}

// SM: the frame's slab in shared memory; else in this CTA's slab of the
// workspace (A.msg + blockIdx.x E q floats; the launcher keeps the grid
// within the F E q floats of the message region).
template <int Q, bool SM>
__global__ void __launch_bounds__(kLevelPiece, SM ? 1 : 3) k_sus_res(const DecodeArgs A) {
    constexpr int T = kLevelPiece;
    __shared__ __align__(16) uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ __align__(16) uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ int s_f;
    extern __shared__ __align__(16) uint8_t s_res[];
    const int tid = threadIdx.x;
    const int M = A.c.M, N = A.c.N;
    const ResSusParts sp = res_sus_parts<Q, SM>(A.c.E, M, N, A.c.npieces);
    float* X = SM ? reinterpret_cast<float*>(s_res + sp.X) : A.msg + (size_t)blockIdx.x * A.c.E * Q;
    float* s_rows = reinterpret_cast<float*>(s_res + sp.rows);
    float* s_scr = reinterpret_cast<float*>(s_res + sp.scr);
    int* s_rowptr = reinterpret_cast<int*>(s_res + sp.rowptr);
    int* s_lp = reinterpret_cast<int*>(s_res + sp.lpiece);
    uint8_t* s_hx = s_res + sp.hx;
    uint8_t* s_xh = s_res + sp.xh;
    uint8_t* s_z = A.syn ? s_res + sp.z : nullptr;
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, T);
    for (int i = tid; i <= M; i += T) s_rowptr[i] = A.c.rowptr[i];
    for (int i = tid; i <= A.c.npieces; i += T) s_lp[i] = A.c.lpiece[i];
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        res_sus_frame<Q, SM>(A, f, s_mul, s_div, X, s_rows, s_scr, s_rowptr, s_lp, s_hx, s_xh, s_z);
    }
}

}  // namespace
}  // namespace gfbp
