// SUS (Sec. 2) by levels with the running partial convolutions of every
// check held in shared memory (DIRECT check node, q <= 16): a CTA decodes one
// frame with a group of G = q/4 threads per (column, check) pair, each thread
// owning V = 4 entries of the pair's vectors (q = 2: one thread, both entries).
//
// When the sweep reaches column j, check i's messages from columns before j
// hold this sweep's values and those after j the values the sweep started
// with.  So, for check i with edges e0..e0+d-1 (columns increasing), the
// shared array X (one q-vector per edge) holds
//   X[e0 + m], 1 <= m <= d-1:  S[m] = q~_{d-1} (*) q~_{d-2} (*) ... (*) q~_m of
//                              the sweep-start messages (S[d-1] = q~_{d-1});
//   X[e0]:                     P, the convolution of the messages of the
//                              positions already visited in this sweep,
// and the visit of position t needs r from P (*) S[t+1] alone (P at the last
// position, S[1] at the first).  Per sweep:
//   0  one bulk copy (TMA engine) of the frame's stored messages into X, then
//      S[m] = S[m+1] (*) q~_m in place, m = d-2 .. 1, a group per check;
//   per piece of the level schedule (sus_level.cuh):
//   1  group <-> pair (j, k), k-th check of j at position t: r = the check's
//      partial convolution relabelled (z XOR h a) and normalised, into a row;
//   2  after a barrier: q_kj from p_j and the column's other rows (Q_j, the
//      hard decision and the posterior on slot 0), stored relabelled to the
//      frame's edge slab (read back at the next sweep), and P <- P (*) q~.
// Every sum and product runs in the order of the global-memory level kernel
// with running partials (sus_level.cuh), so the two give the same bits.
#pragma once

#include "bulk.cuh"
#include "sus_level.cuh"

namespace gfbp {

namespace {

template <int Q>
struct SmLay {
    static constexpr int G = Q >= 4 ? Q / 4 : 1;    // threads per pair
    static constexpr int V = Q / G;                  // entries per thread
    static constexpr int RS = Q >= 4 ? Q + 4 : 4;    // row stride in floats (16-byte multiple)
    static constexpr int T = kLevelPiece * G;        // a group per pair of a piece
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Dynamic shared memory: mbarrier (16 B) | X [E][Q] | rows [kLevelPiece][RS] |
// group scratch [kLevelPiece][RS] | rowptr [M+1] | lpiece [npieces+1] |
// hard decisions [N] | syndrome [M], each part 16-byte aligned.
struct SmParts {
    size_t X, rows, scr, rowptr, lpiece, xh, z, total;
};

template <int Q>
__host__ __device__ constexpr SmParts level_sm_parts(long long E, int M, int N, int npieces) {
    SmParts o{};
    size_t a = 16;
    o.X = a; a += align16(sizeof(float) * (size_t)E * Q);
    o.rows = a; a += sizeof(float) * (size_t)kLevelPiece * SmLay<Q>::RS;
    o.scr = a; a += sizeof(float) * (size_t)kLevelPiece * SmLay<Q>::RS;
    o.rowptr = a; a += align16(sizeof(int) * (size_t)(M + 1));
    o.lpiece = a; a += align16(sizeof(int) * (size_t)(npieces + 1));
    o.xh = a; a += align16((size_t)N);
    o.z = a; a += align16((size_t)M);
    o.total = a;
    return o;
}

template <int Q>
size_t level_sm_bytes(const CodeDev& c) {
    return level_sm_parts<Q>(c.E, c.M, c.N, c.npieces).total;
}

template <int Q>
__device__ __forceinline__ void lds_v(float (&x)[SmLay<Q>::V], const float* p) {
    if constexpr (SmLay<Q>::V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    } else {
        const float2 a = *reinterpret_cast<const float2*>(p);
        x[0] = a.x; x[1] = a.y;
    }
}

template <int Q>
__device__ __forceinline__ void sts_v(float* p, const float (&x)[SmLay<Q>::V]) {
    if constexpr (SmLay<Q>::V == 4) *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
}

template <int Q>
__device__ __forceinline__ void ldg_vv(float (&x)[SmLay<Q>::V], const float* p) {
    if constexpr (SmLay<Q>::V == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    } else {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        x[0] = a.x; x[1] = a.y;
    }
}

// out[x] = src[x XOR b] for a shared q-vector, b a multiple of 4 (0 at q = 2):
// XOR with b maps aligned blocks of four onto aligned blocks of four.
template <int Q>
__device__ __forceinline__ void lds_perm(float (&out)[Q], const float* src, int b) {
    if constexpr (Q == 2) {
        out[0] = src[0];
        out[1] = src[1];
    } else {
#pragma unroll
        for (int x0 = 0; x0 < Q; x0 += 4) {
            const float4 a = *reinterpret_cast<const float4*>(src + (x0 ^ b));
            out[x0] = a.x; out[x0 + 1] = a.y; out[x0 + 2] = a.z; out[x0 + 3] = a.w;
        }
    }
}

// This thread's entries y = g V + v of U (*) Y (both shared):
// o[v] = sum_x U[x] Y[x XOR y], one FMA chain per output in increasing x, as
// in xconv_regs.  With Yp[x] = Y[x XOR g V], Y[x XOR y] = Yp[x XOR v].
template <int Q>
__device__ __forceinline__ void sm_xconv(float (&o)[SmLay<Q>::V], const float* U_s, const float* Y_s, int g) {
    constexpr int V = SmLay<Q>::V;
    float U[Q], Yp[Q];
    lds_perm<Q>(U, U_s, 0);
    lds_perm<Q>(Yp, Y_s, g * V);
#pragma unroll
    for (int v = 0; v < V; v++) o[v] = fmaf(U[0], Yp[v], 0.f);
#pragma unroll
    for (int x = 1; x < Q; x++)
#pragma unroll
        for (int v = 0; v < V; v++) o[v] = fmaf(U[x], Yp[x ^ v], o[v]);
}

// Sum over the group's q entries in the order of tree_sum (pairwise over the
// index bits, lowest first): the low bits inside the thread, the high bits
// across the group by XOR shuffles (a + b and b + a are the same number).
template <int Q>
__device__ __forceinline__ float sm_sum(const float (&x)[SmLay<Q>::V], unsigned mask) {
    constexpr int V = SmLay<Q>::V, G = SmLay<Q>::G;
    float s[V];
#pragma unroll
    for (int i = 0; i < V; i++) s[i] = x[i];
#pragma unroll
    for (int w = 1; w < V; w <<= 1)
#pragma unroll
        for (int i = 0; i < V; i += 2 * w) s[i] = __fadd_rn(s[i], s[i + w]);
    float t = s[0];
#pragma unroll
    for (int o = 1; o < G; o <<= 1) t = __fadd_rn(t, __shfl_xor_sync(mask, t, o));
    return t;
}

template <int Q>
__device__ __forceinline__ void sm_normalise(float (&x)[SmLay<Q>::V], unsigned mask, int* zs = nullptr) {
    constexpr int V = SmLay<Q>::V;
    const float s = sm_sum<Q>(x, mask);
    if (s > 0.f && s <= 3.0e38f) {
        const float r = 1.0f / s;
#pragma unroll
        for (int i = 0; i < V; i++) x[i] *= r;
    } else {
#pragma unroll
        for (int i = 0; i < V; i++) x[i] = 1.0f / Q;
        note_zero_sum<SmLay<Q>::G>(zs);
    }
}

// Lowest index of the largest entry over the group.
template <int Q>
__device__ __forceinline__ int sm_argmax(const float (&x)[SmLay<Q>::V], unsigned mask, int g) {
    constexpr int V = SmLay<Q>::V, G = SmLay<Q>::G;
    int bi = g * V;
    float bv = x[0];
#pragma unroll
    for (int i = 1; i < V; i++)
        if (x[i] > bv) { bv = x[i]; bi = g * V + i; }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const float ov = __shfl_xor_sync(mask, bv, o);
        const int oi = __shfl_xor_sync(mask, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    return bi;
}

// Step 0b: the suffix convolutions of every check, in place (X holds the
// sweep-start messages).
template <int Q>
__device__ __forceinline__ void sm_suffixes(int M, const int* s_rowptr, float* X, unsigned mask, int g, int grp) {
    constexpr int V = SmLay<Q>::V;
    for (int i = grp; i < M; i += kLevelPiece) {
        const int e0 = s_rowptr[i];
        const int d = s_rowptr[i + 1] - e0;
        float* Xc = X + (size_t)e0 * Q;
#pragma unroll 1
        for (int m = d - 2; m >= 1; m--) {
            float o[V];
            sm_xconv<Q>(o, Xc + (size_t)(m + 1) * Q, Xc + (size_t)m * Q, g);
            __syncwarp(mask);   // the group has read slot m
            sts_v<Q>(Xc + (size_t)m * Q + g * V, o);
            __syncwarp(mask);   // slot m complete before it is read as S[m+1]
        }
    }
}

// Step 1 for the pair of record (ra, rb): r of the column's k-th check into row.
template <int Q>
__device__ __forceinline__ void sm_check(const float* X, const uint8_t* s_z, int4 ra, int4 rb, const uint8_t* s_mul,
                                         float* row, float* scr, unsigned mask, int g, int* zs) {
    constexpr int V = SmLay<Q>::V;
    if (rb.z == 0) return;   // a column without checks
    const int t = ra.x - ra.y;
    const int dc = ra.z & 255;
    const int h = (ra.z >> 8) & 255;
    const int z = s_z ? (s_z[ra.w] & (Q - 1)) : 0;
    const float* Xc = X + (size_t)ra.y * Q;
    float o[V];
    if (dc == 1) {
        // a check of degree 1: the XOR-sum of no other edges is 0
#pragma unroll
        for (int v = 0; v < V; v++) o[v] = g * V + v == 0 ? 1.f : 0.f;
    } else if (t == 0) {
        lds_v<Q>(o, Xc + Q + g * V);   // S[1]
    } else if (t == dc - 1) {
        lds_v<Q>(o, Xc + g * V);       // P
    } else {
        sm_xconv<Q>(o, Xc, Xc + (size_t)(t + 1) * Q, g);
    }
    // r_ij[a] = s[z XOR h a], normalised
    sts_v<Q>(scr + g * V, o);
    __syncwarp(mask);
    float R[V];
#pragma unroll
    for (int v = 0; v < V; v++) R[v] = scr[(z ^ s_mul[h * Q + g * V + v]) & (Q - 1)];
    sm_normalise<Q>(R, mask, zs);
    sts_v<Q>(row + g * V, R);
}

// Step 2 for the pair of record (ra, rb); pl: this thread's entries of the
// column's channel likelihood, Pm of its block prior when si >= 0.
template <int Q>
__device__ __forceinline__ void sm_var(const DecodeArgs& A, int f, float* X, float* slab, uint8_t* s_xh, int4 ra,
                                       int4 rb, const float (&pl)[SmLay<Q>::V], int si,
                                       const float (&Pm)[SmLay<Q>::V], const float* row, const uint8_t* s_div,
                                       float* scr, unsigned mask, int g) {
    constexpr int V = SmLay<Q>::V, RS = SmLay<Q>::RS;
    const int j = rb.x, k = rb.y & 255, d = rb.z;
    const int h = (ra.z >> 8) & 255;
    const int N = A.c.N;
    float p[V];
#pragma unroll
    for (int i = 0; i < V; i++) p[i] = pl[i];
    if (si >= 0) {
#pragma unroll
        for (int i = 0; i < V; i++) p[i] *= Pm[i];
        sm_normalise<Q>(p, mask);
    }
    float other[V], all[V];
#pragma unroll
    for (int i = 0; i < V; i++) { other[i] = p[i]; all[i] = p[i]; }
    const float* r0 = row - (size_t)k * RS;   // row of the column's slot 0
#pragma unroll 1
    for (int k2 = 0; k2 < d; k2++) {
        float r[V];
        lds_v<Q>(r, r0 + (size_t)k2 * RS + g * V);
#pragma unroll
        for (int i = 0; i < V; i++) {
            all[i] *= r[i];
            if (k2 != k) other[i] *= r[i];
        }
    }
    if (k == 0) {
        sm_normalise<Q>(all, mask, zsum_of(A, f));
        const int a = sm_argmax<Q>(all, mask, g);
        if (g == 0) s_xh[j] = (uint8_t)a;
        if (A.post) sts_v<Q>(A.post + ((size_t)f * N + j) * Q + g * V, all);
        if (si >= 0) sts_v<Q>(A.Qsrc + ((size_t)f * A.K + si) * Q + g * V, all);
    }
    if (d == 0) return;
    sm_normalise<Q>(other, mask, zsum_of(A, f));
    if (A.step) sts_v<Q>(A.msg_io + ((size_t)f * A.c.E + ra.x) * Q + g * V, other);
    // stored form: qt[y] = q[h^-1 y]
    sts_v<Q>(scr + g * V, other);
    __syncwarp(mask);
    float qt[V];
#pragma unroll
    for (int v = 0; v < V; v++) qt[v] = scr[s_div[h * Q + g * V + v]];
    sts_v<Q>(slab + (size_t)ra.x * Q + g * V, qt);
    const int t = ra.x - ra.y;
    if (t < (ra.z & 255) - 1) {   // the running prefix takes in the new message
        float* P = X + (size_t)ra.y * Q;
        if (t == 0) {
            sts_v<Q>(P + g * V, qt);
        } else {
            __syncwarp(mask);   // the group has read the scratch
            sts_v<Q>(scr + g * V, qt);
            __syncwarp(mask);
            float o[V];
            sm_xconv<Q>(o, P, scr, g);
            __syncwarp(mask);   // the group has read P
            sts_v<Q>(P + g * V, o);
        }
    }
}

// The frame's stored messages into X: one bulk copy (q >= 4) issued by thread
// 0, completing on bar.  Call after a barrier that follows the last writes of
// the slab and the last reads of X.
template <int Q>
__device__ __forceinline__ void sm_issue_copy(float* X, const float* slab, uint32_t xbytes, uint64_t* bar) {
    if (threadIdx.x == 0) {
        fence_proxy_async();   // the generic accesses before the async copy
        mbar_arrive_expect(bar, xbytes);
        constexpr uint32_t kChunk = 32768;
        for (uint32_t o = 0; o < xbytes; o += kChunk) {
            const uint32_t n = xbytes - o < kChunk ? xbytes - o : kChunk;
            bulk_copy(reinterpret_cast<uint8_t*>(X) + o, reinterpret_cast<const uint8_t*>(slab) + o, n, bar);
        }
    }
}

// Wait for the copy; false (for every thread) when the bounded wait ran out.
__device__ __forceinline__ bool sm_wait_copy(uint64_t* bar, uint32_t& phase) {
    const bool got = mbar_wait(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!got)) {
        mbar_wait(bar, phase ^ 1u);   // let a late copy land before the CTA moves on
        return false;
    }
    return true;
}

// The record of a piece's pair for group grp (n pairs in the piece from pb).
__device__ __forceinline__ void sm_rec(const DecodeArgs& A, int pb, int n, int grp, int4& ra, int4& rb) {
    if (grp < n) {
        ra = A.c.lrec[2 * (size_t)(pb + grp)];
        rb = A.c.lrec[2 * (size_t)(pb + grp) + 1];
    }
}

template <int Q>
__device__ __forceinline__ void sm_lik(const DecodeArgs& A, int f, int n, int grp, int4 rb, int g,
                                       float (&pl)[SmLay<Q>::V]) {
    if (grp < n) ldg_vv<Q>(pl, A.L + ((size_t)f * A.c.N + rb.x) * Q + g * SmLay<Q>::V);
}

// One frame; false when a bounded wait for a bulk copy ran out (the frame is
// then marked failed and the kernel must stop).
template <int Q>
__device__ __forceinline__ bool sus_level_sm_frame(const DecodeArgs& A, int f, const uint8_t* s_mul,
                                                   const uint8_t* s_div, uint8_t* s_dyn, const SmParts& sp,
                                                   uint32_t& phase) {
    using L = SmLay<Q>;
    constexpr int G = L::G, V = L::V, RS = L::RS, T = L::T;
    const int tid = threadIdx.x;
    const int g = tid & (G - 1), grp = tid / G;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned mask = group_mask<G>();
    const int M = A.c.M, N = A.c.N;
    uint64_t* bar = reinterpret_cast<uint64_t*>(s_dyn);
    float* X = reinterpret_cast<float*>(s_dyn + sp.X);
    float* s_rows = reinterpret_cast<float*>(s_dyn + sp.rows);
    float* scr = reinterpret_cast<float*>(s_dyn + sp.scr) + (size_t)grp * RS;
    const int* s_rowptr = reinterpret_cast<const int*>(s_dyn + sp.rowptr);
    const int* s_lp = reinterpret_cast<const int*>(s_dyn + sp.lpiece);
    uint8_t* s_xh = s_dyn + sp.xh;
    uint8_t* s_z = A.syn ? s_dyn + sp.z : nullptr;
    float* slab = A.msg + (size_t)f * A.c.E * Q;
    const uint32_t xbytes = (uint32_t)(sizeof(float) * (size_t)A.c.E * Q);
    const int np = A.c.npieces;

    int t0 = 0;   // iterations already done (resumable decoding)
    if (A.fstate) {
        const int st = A.fstate[f];
        if (st >> 30) return true;
        t0 = st;
    }
    __syncthreads();   // the previous frame is done with X and the staged arrays
    if constexpr (Q >= 4) sm_issue_copy<Q>(X, slab, xbytes, bar);
    if (s_z)
        for (int i = tid; i < M; i += T) s_z[i] = A.syn[(size_t)f * M + i];
    int t = t0 + 1, ok = 0;
    bool fin = false, failed = false;
    for (;; t++) {
        // step 0: the sweep-start messages in X, the suffixes, and the first
        // piece's records
        int4 ra = make_int4(0, 0, 0, 0), rb = make_int4(0, 0, 0, 0);
        float pl[V] = {};
        const int n0 = np > 0 ? s_lp[1] - s_lp[0] : 0;
        sm_rec(A, 0, n0, grp, ra, rb);
        if constexpr (Q >= 4) {
            if (!sm_wait_copy(bar, phase)) { failed = true; break; }
        } else {
            __syncthreads();
            for (int x = tid; x < A.c.E * Q; x += T) X[x] = slab[x];
            __syncthreads();
        }
        sm_lik<Q>(A, f, n0, grp, rb, g, pl);
        sm_suffixes<Q>(M, s_rowptr, X, mask, g, grp);
        __syncthreads();
#pragma unroll 1
        for (int pc = 0; pc < np; pc++) {
            const int n = s_lp[pc + 1] - s_lp[pc];
            // the next piece's records, arriving during this piece
            int4 ra2 = make_int4(0, 0, 0, 0), rb2 = make_int4(0, 0, 0, 0);
            const int n2 = pc + 1 < np ? s_lp[pc + 2] - s_lp[pc + 1] : 0;
            if (pc + 1 < np) sm_rec(A, s_lp[pc + 1], n2, grp, ra2, rb2);
            int si = -1;
            float Pm[V] = {};
            float* row = s_rows + (size_t)((rb.y >> 8) & 255) * RS;
            if (grp < n) {
                if (A.markov) {
                    si = A.src_index[rb.x];
                    if (si >= 0) ldg_vv<Q>(Pm, A.P + ((size_t)f * A.K + si) * Q + g * V);
                }
                sm_check<Q>(X, s_z, ra, rb, s_mul, row, scr, mask, g, zsum_of(A, f));
            }
            __syncthreads();
            float pl2[V] = {};
            if (pc + 1 < np) sm_lik<Q>(A, f, n2, grp, rb2, g, pl2);
            if (grp < n) sm_var<Q>(A, f, X, slab, s_xh, ra, rb, pl, si, Pm, row, s_div, scr, mask, g);
            __syncthreads();
            ra = ra2;
            rb = rb2;
#pragma unroll
            for (int v = 0; v < V; v++) pl[v] = pl2[v];
        }
        // the next sweep's messages start to arrive while the sweep is checked
        if constexpr (Q >= 4) sm_issue_copy<Q>(X, slab, xbytes, bar);
        int bad = 0;
        for (int i = tid; i < M; i += T) {
            int s = 0;
            const int e1 = s_rowptr[i + 1];
            for (int e = s_rowptr[i]; e < e1; e++) s ^= s_mul[A.c.eh[e] * Q + s_xh[A.c.ecol[e]]];
            bad |= (s != (s_z ? (s_z[i] & (Q - 1)) : 0));
        }
        ok = !__syncthreads_or(bad);
        if (A.trace) {
            uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
            for (int jj = tid; jj < N; jj += T) tr[jj] = s_xh[jj];
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
    // a copy issued at the end of the last sweep is still in flight
    if (Q >= 4 && !failed && !sm_wait_copy(bar, phase)) failed = true;
    if (failed) {
        if (tid == 0) {
            if (A.iters) A.iters[f] = -1;
            A.conv[f] = 0;
            if (A.fstate) A.fstate[f] = 1 << 30;
        }
        return false;
    }
    for (int jj = tid; jj < N; jj += T) A.xhat[(size_t)f * N + jj] = s_xh[jj];
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
    return true;
}

template <int Q>
__global__ void __launch_bounds__(SmLay<Q>::T, 1) k_sus_level_sm(const DecodeArgs A) {
    using L = SmLay<Q>;
    __shared__ uint8_t s_mul[Q * Q];   // s_mul[h*Q + a] = h a
    __shared__ uint8_t s_div[Q * Q];   // s_div[h*Q + b] = h^-1 b
    __shared__ int s_f;
    extern __shared__ __align__(16) uint8_t s_dyn[];
    const int tid = threadIdx.x;
    const SmParts sp = level_sm_parts<Q>(A.c.E, A.c.M, A.c.N, A.c.npieces);
    team_tables<Q>(A.c.gexp, A.c.glog, s_mul, s_div, tid, L::T);
    int* s_rowptr = reinterpret_cast<int*>(s_dyn + sp.rowptr);
    int* s_lp = reinterpret_cast<int*>(s_dyn + sp.lpiece);
    for (int i = tid; i <= A.c.M; i += L::T) s_rowptr[i] = A.c.rowptr[i];
    for (int i = tid; i <= A.c.npieces; i += L::T) s_lp[i] = A.c.lpiece[i];
    if (tid == 0) {
        mbar_init(reinterpret_cast<uint64_t*>(s_dyn));
        mbar_init_fence();
    }
    uint32_t phase = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        if (!sus_level_sm_frame<Q>(A, f, s_mul, s_div, s_dyn, sp, phase)) break;
    }
}

}  // namespace
}  // namespace gfbp
