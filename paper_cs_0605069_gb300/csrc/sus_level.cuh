// SUS (Sec. 2, steps 1-4) by levels of the column order, with one thread per
// (column, check) pair and whole q-vectors in registers (q <= 16).
//
// Column j reads the stored q of the columns that share a check with it and
// writes its own; two columns that share no check touch disjoint data.  With
// level(j) = 1 + the highest level of the earlier columns sharing a check with
// j, the columns of one level share no check, every earlier neighbour of j
// sits on a lower level and every later one on a higher level.  Updating the
// levels in turn, the columns of a level at once, therefore gives every column
// exactly the operands of the sequential order j = 0..N-1.  A random (3,6)
// code with N = 1000 has about 27 levels of about 37 columns.
//
// A CTA decodes one frame.  Each level is cut (on the host) into pieces of
// whole columns with at most kLevelPiece pairs; per piece:
//   step 1  thread <-> pair (j, k): r_kj of the column's k-th check folded from
//           the check's other stored vectors (direct XOR-convolutions, all q
//           entries of the operands in registers: q^2 FMAs per convolution,
//           no shared-memory traffic), relabelled and normalised into a
//           shared row;
//   step 2  after a barrier, thread <-> pair (j, k): q_kj from the column's
//           other rows (and Q_j, the hard decision and the posterior on slot 0),
//           stored relabelled into the edge slab.
// The arithmetic (each sum's order, each product's order, the normalisation)
// is the single-team kernel's operation for operation, so the two give the
// same bits.  A piece's pairs are taken in the regrouped order of
// CodeDev::lpair_d, each writing the row of its place in the column order.
//
// RUN (running partial convolutions, kept in a second global slab): at the
// start of each sweep every check's suffix convolutions of the sweep-start
// messages are formed (level_suffixes); step 1 then takes r from the check's
// running prefix and one suffix (level_check_run) and step 2 extends the
// prefix by the new message.  sus_level_sm.cuh holds the same arithmetic
// with the partials in shared memory.
#pragma once

#include "sus_team.cuh"

namespace gfbp {

namespace {

template <int Q>
__device__ __forceinline__ void ldq(float (&x)[Q], const float* p) {
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
__device__ __forceinline__ void ldgq(float (&x)[Q], const float* p) {
    if constexpr (Q == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        x[0] = a.x; x[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < Q; i += 4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p + i));
            x[i] = a.x; x[i + 1] = a.y; x[i + 2] = a.z; x[i + 3] = a.w;
        }
    }
}

// A q-vector from global memory by 256-bit loads (one 32-byte sector each;
// p 32-byte aligned) for q >= 8, else as ldq.  NC: through the read-only
// path (data the kernel does not write).
template <int Q, bool NC = false>
__device__ __forceinline__ void ldq_g(float (&x)[Q], const float* p) {
    if constexpr (Q >= 8) {
#pragma unroll
        for (int i = 0; i < Q; i += 8) {
            if constexpr (NC)
                asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=f"(x[i]), "=f"(x[i + 1]), "=f"(x[i + 2]), "=f"(x[i + 3]), "=f"(x[i + 4]),
                               "=f"(x[i + 5]), "=f"(x[i + 6]), "=f"(x[i + 7])
                             : "l"(p + i));
            else
                asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=f"(x[i]), "=f"(x[i + 1]), "=f"(x[i + 2]), "=f"(x[i + 3]), "=f"(x[i + 4]),
                               "=f"(x[i + 5]), "=f"(x[i + 6]), "=f"(x[i + 7])
                             : "l"(p + i)
                             : "memory");
        }
    } else if constexpr (NC) {
        ldgq<Q>(x, p);
    } else {
        ldq<Q>(x, p);
    }
}

// Non-binding L1 prefetch of the 128-byte lines covering [p, p + bytes).
__device__ __forceinline__ void prefetch_l1(const void* p, int bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)127;
    const uintptr_t e = reinterpret_cast<uintptr_t>(p) + (uintptr_t)bytes;
    for (uintptr_t l = a; l < e; l += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
}

template <int Q>
__device__ __forceinline__ void stq(float* p, const float (&x)[Q]) {
    if constexpr (Q == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
    }
}

// A q-vector to global memory by 256-bit stores for q >= 8 (p 32-byte
// aligned), else as stq.
template <int Q>
__device__ __forceinline__ void stq_g(float* p, const float (&x)[Q]) {
    if constexpr (Q >= 8) {
#pragma unroll
        for (int i = 0; i < Q; i += 8)
            asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p + i), "f"(x[i]), "f"(x[i + 1]),
                         "f"(x[i + 2]), "f"(x[i + 3]), "f"(x[i + 4]), "f"(x[i + 5]), "f"(x[i + 6]), "f"(x[i + 7])
                         : "memory");
    } else {
        stq<Q>(p, x);
    }
}

// Stride (floats) of the shared r rows and scratch rows of the level kernel:
// a multiple of 4 floats with (stride / 4) odd for q >= 4, so that eight
// threads' 16-byte accesses to consecutive rows fall on distinct banks; odd
// for q = 2 (scalar accesses).
template <int Q>
__host__ __device__ constexpr int level_rs() { return Q == 2 ? 3 : (Q == 4 ? 4 : Q + 4); }

// A row of Q floats to / from shared memory at a level_rs-aligned address.
template <int Q>
__device__ __forceinline__ void ld_lrow(float (&x)[Q], const float* p) {
    if constexpr (Q == 2) { x[0] = p[0]; x[1] = p[1]; }
    else ldq<Q>(x, p);
}
template <int Q>
__device__ __forceinline__ void st_lrow(float* p, const float (&x)[Q]) {
    if constexpr (Q == 2) { p[0] = x[0]; p[1] = x[1]; }
    else stq<Q>(p, x);
}

// o = U (*) Y: o[y] = fma(U[Q-1], Y[(Q-1)^y], ... fma(U[1], Y[1^y], U[0] Y[y] + 0)),
// outputs y and y^1 in one packed FMA each step.
template <int Q>
__device__ __forceinline__ void xconv_pk(float (&o)[Q], const float (&U)[Q], const float (&Y)[Q]) {
    float2 acc[Q / 2];
    const float2 zero = make_float2(0.f, 0.f);
    {
        const float2 u = make_float2(U[0], U[0]);
#pragma unroll
        for (int k = 0; k < Q / 2; k++) acc[k] = __ffma2_rn(u, make_float2(Y[2 * k], Y[2 * k + 1]), zero);
    }
#pragma unroll
    for (int x = 1; x < Q; x++) {
        const float2 u = make_float2(U[x], U[x]);
#pragma unroll
        for (int k = 0; k < Q / 2; k++) {
            const int i = x ^ (2 * k);
            acc[k] = __ffma2_rn(u, make_float2(Y[i], Y[i ^ 1]), acc[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < Q / 2; k++) {
        o[2 * k] = acc[k].x;
        o[2 * k + 1] = acc[k].y;
    }
}

// U <- U (*) Y, (U (*) Y)[y] = sum_x U[x] Y[x XOR y]: one FMA chain per output
// in increasing x (the q outputs are independent chains), two outputs per
// packed FMA.
template <int Q>
__device__ __forceinline__ void xconv_regs(float (&U)[Q], const float (&Y)[Q]) {
    float o[Q];
    xconv_pk<Q>(o, U, Y);
#pragma unroll
    for (int y = 0; y < Q; y++) U[y] = o[y];
}

// out[a] = src[z XOR tbl[a]] with tbl a 16-byte-aligned row of Q byte indices
// (read in one access for q >= 4).
template <int Q>
__device__ __forceinline__ void gather_row(float (&out)[Q], const float* src, const uint8_t* tbl, int z) {
    if constexpr (Q == 16) {
        const uint4 t = *reinterpret_cast<const uint4*>(tbl);
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int a = 0; a < 16; a++) out[a] = src[z ^ ((w[a >> 2] >> (8 * (a & 3))) & 255)];
    } else if constexpr (Q == 8) {
        const uint2 t = *reinterpret_cast<const uint2*>(tbl);
        const unsigned w[2] = {t.x, t.y};
#pragma unroll
        for (int a = 0; a < 8; a++) out[a] = src[z ^ ((w[a >> 2] >> (8 * (a & 3))) & 255)];
    } else if constexpr (Q == 4) {
        const unsigned w = *reinterpret_cast<const unsigned*>(tbl);
#pragma unroll
        for (int a = 0; a < 4; a++) out[a] = src[z ^ ((w >> (8 * a)) & 255)];
    } else {
#pragma unroll
        for (int a = 0; a < Q; a++) out[a] = src[z ^ tbl[a]];
    }
}

// Pairwise tree over the index bits, lowest bit first (the order of slot_sum).
template <int Q>
__device__ __forceinline__ float tree_sum(const float (&x)[Q]) {
    float s[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) s[i] = x[i];
#pragma unroll
    for (int w = 1; w < Q; w <<= 1)
#pragma unroll
        for (int i = 0; i < Q; i += 2 * w) s[i] = __fadd_rn(s[i], s[i + w]);
    return s[0];
}

template <int Q>
__device__ __forceinline__ void normalise_regs(float (&x)[Q], int* zs = nullptr) {
    const float s = tree_sum<Q>(x);
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

// Step 1 for local pair lp of the piece: r of check k of column j into row.
template <int Q, int DC>
__device__ __forceinline__ void level_check(const DecodeArgs& A, int f, const float* slab, const uint8_t* zf,
                                            int2 pr, const uint8_t* s_mul, float* row) {
    const int j = pr.x, k = pr.y;
    if (A.c.colptr[j + 1] == A.c.colptr[j]) return;   // a column without checks
    const int4 in = A.c.cinfo[A.c.colptr[j] + k];
    const int own = in.x - in.y;
    const int dc = in.z & 255;
    const int h = (in.z >> 8) & 255;
    const int z = zf ? (zf[in.w] & (Q - 1)) : 0;
    const float* D = slab + (size_t)in.y * Q;
    // the check's vectors are contiguous: bring them all towards L1 at once, so
    // that the fold below waits for memory about once
    prefetch_l1(D, dc * Q * (int)sizeof(float));
    if (k == 0) prefetch_l1(A.L + ((size_t)f * A.c.N + j) * Q, Q * (int)sizeof(float));   // for step 2
    float U[Q];
    if (dc > 1) {
        ldq_g<Q>(U, D + (0 < own ? 0 : 1) * Q);
        float Y[Q];
        if (dc > 2) ldq_g<Q>(Y, D + (1 < own ? 1 : 2) * Q);
#pragma unroll 1
        for (int n = 1; n < dc - 1; n++) {
            float Yn[Q];   // next operand, loaded one convolution ahead
            const bool more = n + 1 < dc - 1;
            if (more) ldq_g<Q>(Yn, D + (n + 1 < own ? n + 1 : n + 2) * Q);
            xconv_regs<Q>(U, Y);
            if (more) {
#pragma unroll
                for (int i = 0; i < Q; i++) Y[i] = Yn[i];
            }
        }
    } else {
        // a check of degree 1: the XOR-sum of no other edges is 0
#pragma unroll
        for (int i = 0; i < Q; i++) U[i] = i == 0 ? 1.f : 0.f;
    }
    // r_ij[a] = s[z XOR h a], normalised
    st_lrow<Q>(row, U);
    float R[Q];
    gather_row<Q>(R, row, s_mul + h * Q, z);   // r[a] = s[z XOR h a]
    normalise_regs<Q>(R, zsum_of(A, f));
    st_lrow<Q>(row, R);
}

// Step 1 with the running partial convolutions: the check's other messages
// are the prefix P of those already updated in this sweep (positions before
// t) and the suffix of those still at their sweep-start values (positions
// after t), so r is P (*) S[t+1] (one convolution; none at either end).
template <int Q>
__device__ __forceinline__ void level_check_run(const DecodeArgs& A, int f, const float* slab, const uint8_t* zf,
                                                int2 pr, const uint8_t* s_mul, float* row) {
    const int j = pr.x, k = pr.y;
    if (A.c.colptr[j + 1] == A.c.colptr[j]) return;   // a column without checks
    const int4 in = A.c.cinfo[A.c.colptr[j] + k];
    const int t = in.x - in.y;
    const int dc = in.z & 255;
    const int h = (in.z >> 8) & 255;
    const int z = zf ? (zf[in.w] & (Q - 1)) : 0;
    const float* D = slab + (size_t)in.y * Q;
    const float* S = A.sfx + ((size_t)f * A.c.E + in.y) * Q;
    if (k == 0) prefetch_l1(A.L + ((size_t)f * A.c.N + j) * Q, Q * (int)sizeof(float));   // for step 2
    float U[Q];
    if (dc == 1) {
        // a check of degree 1: the XOR-sum of no other edges is 0
#pragma unroll
        for (int i = 0; i < Q; i++) U[i] = i == 0 ? 1.f : 0.f;
    } else if (t == 0) {
        ldq_g<Q>(U, (dc == 2 ? D : S) + Q);   // S[1]; S[d-1] is the message itself
    } else {
        ldq_g<Q>(U, S);   // the prefix
        if (t < dc - 1) {
            float Y[Q];
            ldq_g<Q>(Y, (t + 1 == dc - 1 ? D : S) + (size_t)(t + 1) * Q);
            xconv_regs<Q>(U, Y);
        }
    }
    st_lrow<Q>(row, U);
    float R[Q];
    gather_row<Q>(R, row, s_mul + h * Q, z);   // r[a] = s[z XOR h a]
    normalise_regs<Q>(R, zsum_of(A, f));
    st_lrow<Q>(row, R);
}

// The suffix convolutions of every check from the sweep-start messages:
// S[d-1] is the last message, S[m] = S[m+1] (*) q~_m down to m = 1; slots
// 1..d-2 are stored (a thread per check).
template <int Q, int T>
__device__ __forceinline__ void level_suffixes(const DecodeArgs& A, int f, const float* slab) {
    float* sf = A.sfx + (size_t)f * A.c.E * Q;
    for (int i = threadIdx.x; i < A.c.M; i += T) {
        const int e0 = A.c.rowptr[i];
        const int d = A.c.rowptr[i + 1] - e0;
        if (d < 3) continue;
        const float* D = slab + (size_t)e0 * Q;
        prefetch_l1(D, d * Q * (int)sizeof(float));
        float U[Q], Y[Q];
        ldq_g<Q>(U, D + (size_t)(d - 1) * Q);
        ldq_g<Q>(Y, D + (size_t)(d - 2) * Q);
#pragma unroll 1
        for (int m = d - 2; m >= 1; m--) {
            float Yn[Q];   // next operand, loaded one convolution ahead
            if (m > 1) ldq_g<Q>(Yn, D + (size_t)(m - 1) * Q);
            xconv_regs<Q>(U, Y);
            stq_g<Q>(sf + (size_t)(e0 + m) * Q, U);
            if (m > 1) {
#pragma unroll
                for (int x = 0; x < Q; x++) Y[x] = Yn[x];
            }
        }
    }
}

// Step 2 for local pair lp: q of (j, k) from the column's other rows, and for
// slot 0 the posterior Q_j and the hard decision.  RUN: the check's running
// prefix then takes in the new message.
template <int Q, bool RUN>
__device__ __forceinline__ void level_var(const DecodeArgs& A, int f, float* slab, uint8_t* xh, int2 pr,
                                          const float* rows0, const uint8_t* s_div, float* orow) {
    const int j = pr.x, k = pr.y;
    const int c0 = A.c.colptr[j];
    const int d = A.c.colptr[j + 1] - c0;
    const int4 in = d > 0 ? A.c.cinfo[c0 + k] : make_int4(0, 0, 0, 0);
    const int h = (in.z >> 8) & 255;
    const int N = A.c.N;
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
            normalise_regs<Q>(p);
        }
    }
    float other[Q], all[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) { other[i] = p[i]; all[i] = p[i]; }
    constexpr int RS = level_rs<Q>();
    const float* r0 = rows0 - (size_t)k * RS;   // row of the column's slot 0
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
    if (k == 0) {
        normalise_regs<Q>(all, zsum_of(A, f));
        int bi = 0;
        float bv = all[0];
#pragma unroll
        for (int i = 1; i < Q; i++)
            if (all[i] > bv) { bv = all[i]; bi = i; }
        xh[j] = (uint8_t)bi;
        if (A.post) stq<Q>(A.post + ((size_t)f * N + j) * Q, all);
        if (si >= 0) stq<Q>(A.Qsrc + ((size_t)f * A.K + si) * Q, all);
    }
    if (d == 0) return;
    normalise_regs<Q>(other, zsum_of(A, f));
    if (A.step) stq<Q>(A.msg_io + ((size_t)f * A.c.E + in.x) * Q, other);
    // stored form: qt[y] = q[h^-1 y]
    st_lrow<Q>(orow, other);
    float qt[Q];
    gather_row<Q>(qt, orow, s_div + h * Q, 0);
    stq_g<Q>(slab + (size_t)in.x * Q, qt);
    if constexpr (RUN) {
        const int t = in.x - in.y;
        if (t < (in.z & 255) - 1) {
            float* P = A.sfx + ((size_t)f * A.c.E + in.y) * Q;
            if (t == 0) {
                stq_g<Q>(P, qt);
            } else {
                float U[Q];
                ldq_g<Q>(U, P);
                xconv_regs<Q>(U, qt);
                stq_g<Q>(P, U);
            }
        }
    }
}

template <int Q, int DC, int T, bool RUN>
__device__ __forceinline__ void sus_level_frame(const DecodeArgs& A, int f, const uint8_t* s_mul,
                                                const uint8_t* s_div, float* s_row, float* s_orow) {
    constexpr int RS = level_rs<Q>();
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int M = A.c.M, N = A.c.N;
    float* slab = A.msg + (size_t)f * A.c.E * Q;
    const uint8_t* zf = A.syn ? A.syn + (size_t)f * M : nullptr;
    uint8_t* xh = A.xhat + (size_t)f * N;
    float* orow = s_orow + tid * RS;

    int t0 = 0;   // iterations already done (resumable decoding)
    if (A.fstate) {
        const int st = A.fstate[f];
        if (st >> 30) return;
        t0 = st;
    }
    int t = t0 + 1, ok = 0;
    bool fin = false;
    for (;; t++) {
        if constexpr (RUN) {
            level_suffixes<Q, T>(A, f, slab);
            __syncthreads();
        }
#pragma unroll 1
        for (int pc = 0; pc < A.c.npieces; pc++) {
            const int pb = A.c.lpiece[pc];
            const int n = A.c.lpiece[pc + 1] - pb;
            for (int lp = tid; lp < n; lp += T) {
                const int2 pr = A.c.lpair_d[pb + lp];
                const int2 jk = make_int2(pr.x, pr.y & 255);
                float* row = s_row + (pr.y >> 8) * RS;
                if constexpr (RUN) level_check_run<Q>(A, f, slab, zf, jk, s_mul, row);
                else level_check<Q, DC>(A, f, slab, zf, jk, s_mul, row);
            }
            __syncthreads();
            for (int lp = tid; lp < n; lp += T) {
                const int2 pr = A.c.lpair_d[pb + lp];
                level_var<Q, RUN>(A, f, slab, xh, make_int2(pr.x, pr.y & 255), s_row + (pr.y >> 8) * RS, s_div,
                                  orow);
            }
            __syncthreads();
        }
        int bad = 0;
        for (int i = tid; i < M; i += T) {
            int s = 0;
            const int e1 = A.c.rowptr[i + 1];
            for (int e = A.c.rowptr[i]; e < e1; e++) s ^= s_mul[A.c.eh[e] * Q + xh[A.c.ecol[e]]];
            bad |= (s != (zf ? (zf[i] & (Q - 1)) : 0));
        }
        ok = !__syncthreads_or(bad);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int jj = tid; jj < N; jj += T) tr[jj] = xh[jj];
        }
        if ((ok && A.early_stop) || t >= A.max_iter) {
            fin = true;
            break;
        }
        if (A.markov) {
            for (int i = warp; i < A.K; i += T / 32)
                team_prior<Q, 32>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, 0xffffffffu, lane);
            __syncthreads();
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = warp; i < A.K; i += T / 32)
            team_prior<Q, 32>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, 0xffffffffu, lane);
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

template <int Q, int DC, int T, bool RUN>
__global__ void __launch_bounds__(T, 640 / T) k_sus_level(const DecodeArgs A) {
    static_assert(T % 32 == 0, "whole warps");
    __shared__ __align__(16) uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ __align__(16) uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ __align__(16) float s_row[kLevelPiece * level_rs<Q>()];
    __shared__ __align__(16) float s_orow[T * level_rs<Q>()];
    __shared__ int s_f;
    const int tid = threadIdx.x;
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, T);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        sus_level_frame<Q, DC, T, RUN>(A, f, s_mul, s_div, s_row, s_orow);
    }
}

}  // namespace
}  // namespace gfbp
