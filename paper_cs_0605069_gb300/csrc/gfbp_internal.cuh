// Internal declarations and device building blocks of the gfbp library.
//
// Message layout.  A probability vector over GF(q) (q = 2^p) is spread over a
// "group" of G consecutive lanes of a warp, V = q / G entries per lane: lane g
// of the group holds entries a = g*V .. g*V+V-1, so a group reads or writes a
// whole vector as G contiguous V-float chunks (float4 for V >= 4).  The
// Walsh-Hadamard butterflies over the low log2(V) index bits run inside a
// lane, those over the high bits with __shfl_xor_sync inside the group.
//
// Edge slabs are [frame][edge][q] float32 with edges in (row, col) order, so
// the d_c vectors of one check are contiguous.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/gfbp.h"

namespace gfbp {

// Lanes per vector (G) and entries per lane (V) for field size Q.
template <int Q>
struct Lay {
    static constexpr int V = (Q <= 4) ? Q : ((Q / 32 > 4) ? Q / 32 : 4);
    static constexpr int G = Q / V;
    static_assert(V * G == Q && G <= 32, "bad layout");
};

// Device view of a code: all arrays live in one allocation owned by gfbp_code.
struct CodeDev {
    int q, p, M, N;
    long long E;
    int dcmax, dvmax;
    const int* rowptr;   // [M+1]
    const int* ecol;     // [E] column of each edge
    const int* erow;     // [E] row of each edge
    const uint8_t* eh;   // [E] GF value of each edge
    const int* colptr;   // [N+1]
    const int* cedge;    // [E] edge ids of each column, rows increasing
    const uint8_t* gexp; // [512] x^i, extended so that i < 2(q-1) needs no reduction
    const uint8_t* glog; // [256] log_x(a) for a != 0
    const int4* cinfo;   // [E] per column slot: {edge, row start, row degree | h << 8, row}
    const uint8_t* cdep; // [N] 1 when column j shares a check with column j-1
    const int* cpred;    // [N] last column k < j sharing a check with column j, -1 if none
    // SUS level schedule: level(j) = 1 + the highest level of the earlier
    // columns that share a check with j.  Columns of one level share no check;
    // updating the levels in turn gives the sequential order's values.
    int nlevels, npieces;
    const int2* lpair;   // (column, slot) pairs by level, columns increasing; a column
                         // without checks has the one pair (j, 0)
    const int* lpiece;   // [npieces+1] pair offsets: whole columns of one level, <= kLevelPiece pairs
    const int2* lpair_d; // the pairs of each piece regrouped for the q <= 16 level kernel:
                         // (column, slot | index in the piece's column order << 8)
    const int4* lrec;    // [2 per lpair_d entry]: the slot's cinfo, then
                         // {column, slot | row index << 8, column degree, 0}
};

constexpr int kLevelPiece = 128;

struct DecodeArgs {
    CodeDev c;
    int F;
    const float* obs;
    int ch_kind;
    float ch_param;
    const float* frame_param;
    const uint8_t* punct;
    const uint8_t* syn;
    int max_iter;
    int early_stop;
    // Markov block priors (Eqs. 6-7)
    int markov;
    int markov_gs;         // Markov priors re-estimated inside the SUS sweep (MARKOV_GS)
    int K;
    const float* Mt;       // [q][q] row-normalised transition matrix
    const float* pi;       // [q] stationary distribution
    const int* src_pos;    // [K]
    const int* src_index;  // [N] position -> source index or -1
    // workspace
    float* L;              // [F][N][q] normalised channel likelihoods
    float* msg;            // [F][E][q] edge slab
    float* Qsrc;           // [F][K][q] posteriors of source symbols (Markov)
    float* P;              // [F][K][q] block priors in use
    int* work;             // frame counter for persistent kernels
    // outputs
    uint8_t* xhat;
    int* iters;
    uint8_t* conv;
    float* post;
    uint8_t* trace;
    // lock-step mode (gfbp_step)
    int step;
    float* msg_io;         // [F][E][q] q_ij in (before) and out (after)
    float* prior_out;      // [F][K][q]
    int method;            // Method
    // resumable decoding (serving): per frame the iterations done so far, with
    // bit 30 set once the frame has stopped; NULL = whole decode in one launch
    int* fstate;
    int round_iters;       // resumable decoding: iterations per launch
    int width;             // SUS team kernels: teams per frame (0 = automatic)
    int layout;            // gfbp_layout
    int partials;          // gfbp_sus_partials as asked
    // SUS running partial convolutions in global memory (q <= 16 level
    // kernel, RUNNING_GLOBAL), else NULL: per frame an [E][q] slab; for check
    // i with edges e0..e0+d-1, slot e0 + m (1 <= m <= d-2) holds the suffix
    // convolution of the sweep-start messages of positions m..d-1 and slot e0
    // the prefix of the messages updated so far
    float* sfx;
    // per frame the normalisations (of r, q and Q) whose sum was zero or not
    // finite and that fell back to the uniform vector, or NULL
    int* zsum;
};

// The frame's zero-sum counter, or NULL when it is not asked for.
__device__ __forceinline__ int* zsum_of(const DecodeArgs& A, int f) { return A.zsum ? A.zsum + f : nullptr; }

// Count one uniform fallback; a lane group of G lanes (aligned in the warp)
// counts it once.
template <int G>
__device__ __forceinline__ void note_zero_sum(int* zs) {
    if (zs && (threadIdx.x & (G - 1)) == 0) atomicAdd(zs, 1);
}

// ---------------------------------------------------------------- helpers
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

template <int V>
__device__ __forceinline__ void ldv(float (&x)[V], const float* p) {
    if constexpr (V == 8) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        const float4 b = *(reinterpret_cast<const float4*>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else if constexpr (V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    } else if constexpr (V == 2) {
        const float2 a = *reinterpret_cast<const float2*>(p);
        x[0] = a.x; x[1] = a.y;
    } else {
        x[0] = p[0];
    }
}

// Load through the read-only path, for inputs no kernel of the decode writes.
template <int V>
__device__ __forceinline__ void ldg_v(float (&x)[V], const float* p) {
    if constexpr (V == 8) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else if constexpr (V == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    } else if constexpr (V == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        x[0] = a.x; x[1] = a.y;
    } else {
        x[0] = __ldg(p);
    }
}

template <int V>
__device__ __forceinline__ void stv(float* p, const float (&x)[V]) {
    if constexpr (V == 8) {
        reinterpret_cast<float4*>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
    } else if constexpr (V == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
    } else {
        p[0] = x[0];
    }
}

// Unnormalised Walsh-Hadamard transform of the group's vector, in place.
template <int Q>
__device__ __forceinline__ void wht(float (&x)[Lay<Q>::V], unsigned mask, int g) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
#pragma unroll
    for (int h = 1; h < V; h <<= 1) {
#pragma unroll
        for (int i = 0; i < V; i++) {
            if (!(i & h)) {
                const float a = x[i], b = x[i + h];
                x[i] = a + b;
                x[i + h] = a - b;
            }
        }
    }
#pragma unroll
    for (int m = 1; m < G; m <<= 1) {
#pragma unroll
        for (int i = 0; i < V; i++) {
            const float o = __shfl_xor_sync(mask, x[i], m);
            x[i] = (g & m) ? (o - x[i]) : (x[i] + o);
        }
    }
}

template <int Q>
__device__ __forceinline__ float gsum(const float (&x)[Lay<Q>::V], unsigned mask) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    // (separately rounded additions throughout, here and in every sum that
    // normalises a message: a product feeding the sum is never fused into it,
    // so every kernel forms the same sums)
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < V; i++) s = __fadd_rn(s, x[i]);
#pragma unroll
    for (int m = 1; m < G; m <<= 1) s = __fadd_rn(s, __shfl_xor_sync(mask, s, m));
    return s;
}

// Scale to sum 1; a zero or non-finite sum gives the uniform vector (counted
// in *zs when zs is not NULL).
template <int Q>
__device__ __forceinline__ void gnormalise(float (&x)[Lay<Q>::V], unsigned mask, int* zs = nullptr) {
    constexpr int V = Lay<Q>::V;
    const float s = gsum<Q>(x, mask);
    if (s > 0.f && s <= 3.0e38f) {
        const float r = 1.0f / s;
#pragma unroll
        for (int i = 0; i < V; i++) x[i] *= r;
    } else {
#pragma unroll
        for (int i = 0; i < V; i++) x[i] = 1.0f / Q;
        note_zero_sum<Lay<Q>::G>(zs);
    }
}

// Index of the largest entry, lowest index among equal maxima.
template <int Q>
__device__ __forceinline__ int gargmax(const float (&x)[Lay<Q>::V], unsigned mask, int g) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    float bv = x[0];
    int bi = g * V;
#pragma unroll
    for (int i = 1; i < V; i++) {
        if (x[i] > bv) { bv = x[i]; bi = g * V + i; }
    }
#pragma unroll
    for (int m = 1; m < G; m <<= 1) {
        const float ov = __shfl_xor_sync(mask, bv, m);
        const int oi = __shfl_xor_sync(mask, bi, m);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    return bi;
}

__device__ __forceinline__ int gf_mul(const uint8_t* ex, const uint8_t* lg, int a, int b) {
    return (a && b) ? ex[lg[a] + lg[b]] : 0;
}

// h^{-1} * b
template <int Q>
__device__ __forceinline__ int gf_div(const uint8_t* ex, const uint8_t* lg, int b, int h) {
    return b ? ex[lg[b] + (Q - 1) - lg[h]] : 0;
}

// ------------------------------------------------------------------------
// Transform-domain representation of a message (the XOR-convolution theorem
// behind Eq. 3, kept accurate in FP32).
//
// For a message q_ij let y = h_ij x_j (the relabelled symbol, distribution
// qt[y] = q[h^-1 y]) and c its most likely value.  The stored vector is
//     D[w] = 1 - WHT(u)[w] = 2 * sum_{b : parity(b & w) = 1} u[b],
// with u[b] = qt[b XOR c] the distribution shifted so that its mode sits at
// 0.  D[0] is always 0, so slot 0 carries c instead.  D is formed with
// additions of non-negative numbers only, so peaked messages (WHT entries
// within 1e-7 of 1, which plain FP32 transforms round away) keep their
// small deviations to relative precision.
//
// The horizontal pass multiplies transforms, prod_m (1 - D_m) = 1 - E with
// E <- E + D (1 - E), XORs the shifts C = XOR_m c_m, and inverts:
//     s[a] = [a = 0] - WHT(E)[a] / q
// is the distribution of sum_m h_m x_m XOR C, so r_ij[a] = s[z XOR C XOR h a].
// ------------------------------------------------------------------------

// Load a stored vector; lane 0 of the group takes the shift out of slot 0.
template <int V>
__device__ __forceinline__ void ld_dev(float (&D)[V], int& c, const float* p, int g) {
    ldv<V>(D, p);
    c = 0;
    if (g == 0) {
        c = (int)D[0];
        D[0] = 0.f;
    }
}

template <int V>
__device__ __forceinline__ void dev_combine(float (&E)[V], const float (&D)[V]) {
#pragma unroll
    for (int v = 0; v < V; v++) E[v] = fmaf(D[v], 1.0f - E[v], E[v]);
}

template <int Q, int NB>
__device__ __forceinline__ void wht_n(float (&x)[NB][Lay<Q>::V], unsigned mask, int g) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
#pragma unroll
    for (int h = 1; h < V; h <<= 1) {
#pragma unroll
        for (int k = 0; k < NB; k++) {
#pragma unroll
            for (int i = 0; i < V; i++) {
                if (!(i & h)) {
                    const float a = x[k][i], b = x[k][i + h];
                    x[k][i] = a + b;
                    x[k][i + h] = a - b;
                }
            }
        }
    }
#pragma unroll
    for (int m = 1; m < G; m <<= 1) {
#pragma unroll
        for (int k = 0; k < NB; k++) {
#pragma unroll
            for (int i = 0; i < V; i++) {
                const float o = __shfl_xor_sync(mask, x[k][i], m);
                x[k][i] = (g & m) ? (o - x[k][i]) : (x[k][i] + o);
            }
        }
    }
}

// Horizontal-pass epilogue for NB vectors at once (n of them in use): from
// E (and the XOR of shifts C, the same in every lane) to r_ij, normalised;
// negatives from rounding are set to 0.  sc holds NB*Q floats.
template <int Q, int NB>
__device__ __forceinline__ void dev_finish_n(float (&x)[NB][Lay<Q>::V], const int (&C)[NB], const int (&h)[NB],
                                             const int (&z)[NB], int n, float* sc, unsigned mask, int g,
                                             const uint8_t* ex, const uint8_t* lg, int* zs = nullptr) {
    constexpr int V = Lay<Q>::V;
    wht_n<Q, NB>(x, mask, g);
#pragma unroll
    for (int k = 0; k < NB; k++) {
        if (k < n) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                const int a = g * V + v;
                const float t = x[k][v] * (1.0f / Q);
                sc[k * Q + a] = fmaxf(a == 0 ? 1.0f - t : -t, 0.0f);
            }
        }
    }
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < NB; k++) {
        if (k < n) {
#pragma unroll
            for (int v = 0; v < V; v++) x[k][v] = sc[k * Q + ((z[k] ^ C[k] ^ gf_mul(ex, lg, h[k], g * V + v)) & (Q - 1))];
        }
    }
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < NB; k++)
        if (k < n) gnormalise<Q>(x[k], mask, zs);
}

// Vertical-pass epilogue for NB normalised messages q (n in use): the stored
// form D (slot 0 = shift) of the distribution of h x.  Two-channel
// butterflies carry the even- and odd-parity masses, additions only.
template <int Q, int NB>
__device__ __forceinline__ void to_deviation_n(float (&x)[NB][Lay<Q>::V], const int (&h)[NB], int n, float* sc,
                                               unsigned mask, int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    int c[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) {
        c[k] = 0;
        if (k < n) {
            const int am = gargmax<Q>(x[k], mask, g);
            c[k] = gf_mul(ex, lg, h[k], am);
#pragma unroll
            for (int v = 0; v < V; v++) sc[k * Q + g * V + v] = x[k][v];
        }
    }
    __syncwarp(mask);
    float ev[NB][V], od[NB][V];
#pragma unroll
    for (int k = 0; k < NB; k++) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            const int b = g * V + v;
            ev[k][v] = (k < n && b != 0) ? sc[k * Q + gf_div<Q>(ex, lg, b ^ c[k], h[k])] : 0.0f;
            od[k][v] = 0.0f;
        }
    }
    __syncwarp(mask);
#pragma unroll
    for (int hb = 1; hb < V; hb <<= 1) {
#pragma unroll
        for (int k = 0; k < NB; k++) {
#pragma unroll
            for (int i = 0; i < V; i++) {
                if (!(i & hb)) {
                    const int j = i + hb;
                    const float e0 = ev[k][i], o0 = od[k][i], e1 = ev[k][j], o1 = od[k][j];
                    ev[k][i] = e0 + e1;
                    od[k][i] = o0 + o1;
                    ev[k][j] = e0 + o1;
                    od[k][j] = o0 + e1;
                }
            }
        }
    }
#pragma unroll
    for (int m = 1; m < G; m <<= 1) {
#pragma unroll
        for (int k = 0; k < NB; k++) {
#pragma unroll
            for (int i = 0; i < V; i++) {
                const float pe = __shfl_xor_sync(mask, ev[k][i], m);
                const float po = __shfl_xor_sync(mask, od[k][i], m);
                if (g & m) {
                    const float ne = pe + od[k][i], no = po + ev[k][i];
                    ev[k][i] = ne;
                    od[k][i] = no;
                } else {
                    ev[k][i] += pe;
                    od[k][i] += po;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NB; k++) {
#pragma unroll
        for (int v = 0; v < V; v++) x[k][v] = 2.0f * od[k][v];
        if (g == 0) x[k][0] = (float)c[k];
    }
}

template <int Q>
__device__ __forceinline__ void to_deviation(float (&x)[Lay<Q>::V], int h, float* sc, unsigned mask, int g,
                                             const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    float xx[1][V];
    const int hh[1] = {h};
#pragma unroll
    for (int v = 0; v < V; v++) xx[0][v] = x[v];
    to_deviation_n<Q, 1>(xx, hh, 1, sc, mask, g, ex, lg);
#pragma unroll
    for (int v = 0; v < V; v++) x[v] = xx[0][v];
}

template <int Q>
__device__ __forceinline__ void dev_finish(float (&x)[Lay<Q>::V], int C, int h, int z, float* sc, unsigned mask,
                                           int g, const uint8_t* ex, const uint8_t* lg, int* zs = nullptr) {
    constexpr int V = Lay<Q>::V;
    float xx[1][V];
    const int cc[1] = {C}, hh[1] = {h}, zz[1] = {z};
#pragma unroll
    for (int v = 0; v < V; v++) xx[0][v] = x[v];
    dev_finish_n<Q, 1>(xx, cc, hh, zz, 1, sc, mask, g, ex, lg, zs);
#pragma unroll
    for (int v = 0; v < V; v++) x[v] = xx[0][v];
}

// ------------------------------------------------------------------------
// Probability-domain route of Eq. 3 (q <= 16): the stored vector of edge ij is
// qt[y] = q_ij[h^-1 y], the distribution of y = h_ij x_j, and the horizontal
// pass convolves the other edges' vectors directly,
//     (a * b)[y] = sum_x a[x] b[x XOR y],
// which adds non-negative products only, so every entry keeps its relative
// precision however small it is.
// ------------------------------------------------------------------------

// Relabel NB normalised messages (n in use) into their stored form qt.
template <int Q, int NB>
__device__ __forceinline__ void to_relabelled_n(float (&x)[NB][Lay<Q>::V], const int (&h)[NB], int n, float* sc,
                                                unsigned mask, int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
#pragma unroll
    for (int k = 0; k < NB; k++)
        if (k < n) stv<V>(sc + k * Q + g * V, x[k]);
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < NB; k++) {
        if (k < n) {
#pragma unroll
            for (int v = 0; v < V; v++) x[k][v] = sc[k * Q + gf_div<Q>(ex, lg, g * V + v, h[k])];
        }
    }
    __syncwarp(mask);
}

template <int Q>
__device__ __forceinline__ void to_relabelled(float (&x)[Lay<Q>::V], int h, float* sc, unsigned mask, int g,
                                              const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    float xx[1][V];
    const int hh[1] = {h};
#pragma unroll
    for (int v = 0; v < V; v++) xx[0][v] = x[v];
    to_relabelled_n<Q, 1>(xx, hh, 1, sc, mask, g, ex, lg);
#pragma unroll
    for (int v = 0; v < V; v++) x[v] = xx[0][v];
}

// out[v] = sum_x sa[x] sb[x XOR y] for this lane's outputs y = g*V + v; sa and
// sb are whole vectors in shared memory (16-byte aligned).  The XOR of a V-block
// of x with the lane's V-block of y is again a V-block, so every read is a
// vector load and the inner index permutation is known at compile time.
template <int Q>
__device__ __forceinline__ void xconv_sm(float (&out)[Lay<Q>::V], const float* sa, const float* sb, int g) {
    constexpr int V = Lay<Q>::V;
    static_assert(V == 2 || V == 4 || V == 8, "direct route needs V in {2, 4, 8}");
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

// out1 = sa (*) sb1 and out2 = sa (*) sb2 (each as xconv_sm) with one read of sa.
template <int Q>
__device__ __forceinline__ void xconv_sm2(float (&out1)[Lay<Q>::V], float (&out2)[Lay<Q>::V], const float* sa,
                                          const float* sb1, const float* sb2, int g) {
    constexpr int V = Lay<Q>::V;
    static_assert(V == 2 || V == 4 || V == 8, "direct route needs V in {2, 4, 8}");
#pragma unroll
    for (int v = 0; v < V; v++) { out1[v] = 0.f; out2[v] = 0.f; }
#pragma unroll
    for (int xb = 0; xb < Q; xb += V) {
        float a[V], b1[V], b2[V];
        ldv<V>(a, sa + xb);
        ldv<V>(b1, sb1 + (xb ^ (g * V)));
        ldv<V>(b2, sb2 + (xb ^ (g * V)));
#pragma unroll
        for (int xl = 0; xl < V; xl++) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                out1[v] = fmaf(a[xl], b1[xl ^ v], out1[v]);
                out2[v] = fmaf(a[xl], b2[xl ^ v], out2[v]);
            }
        }
    }
}

// r[a] = s[z XOR h a] from the distribution s of the other edges' sum, normalised.
template <int Q, int NB>
__device__ __forceinline__ void direct_finish_n(float (&x)[NB][Lay<Q>::V], const int (&h)[NB], const int (&z)[NB],
                                                int n, float* sc, unsigned mask, int g, const uint8_t* ex,
                                                const uint8_t* lg, int* zs = nullptr) {
    constexpr int V = Lay<Q>::V;
#pragma unroll
    for (int k = 0; k < NB; k++)
        if (k < n) stv<V>(sc + k * Q + g * V, x[k]);
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < NB; k++) {
        if (k < n) {
#pragma unroll
            for (int v = 0; v < V; v++) x[k][v] = sc[k * Q + ((z[k] ^ gf_mul(ex, lg, h[k], g * V + v)) & (Q - 1))];
        }
    }
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < NB; k++)
        if (k < n) gnormalise<Q>(x[k], mask, zs);
}

// p_j: normalised channel likelihood times the block prior of a source symbol.
template <int Q>
__device__ __forceinline__ void prior_vec(const DecodeArgs& A, int f, int j, float (&x)[Lay<Q>::V], unsigned mask,
                                          int g) {
    constexpr int V = Lay<Q>::V;
    ldg_v<V>(x, A.L + ((size_t)f * A.c.N + j) * Q + g * V);
    if (A.markov) {
        const int si = A.src_index[j];
        if (si >= 0) {
            float P[V];
            ldv<V>(P, A.P + ((size_t)f * A.K + si) * Q + g * V);
#pragma unroll
            for (int i = 0; i < V; i++) x[i] *= P[i];
            gnormalise<Q>(x, mask);
        }
    }
}

// Eq. 7 for source index i of frame f from the stored posteriors Qsrc:
// P^b = (sum_a Q_{i-1}^a M_ab)(sum_c M_bc Q_{i+1}^c); at the first source
// symbol pi_b replaces the left factor, at the last one 1 replaces the right.
template <int Q>
__device__ __forceinline__ void markov_prior(const DecodeArgs& A, int f, int i, float* out, unsigned mask, int g) {
    constexpr int V = Lay<Q>::V;
    const int K = A.K;
    const float* Qm = (i > 0) ? A.Qsrc + ((size_t)f * K + i - 1) * Q : nullptr;
    const float* Qp = (i < K - 1) ? A.Qsrc + ((size_t)f * K + i + 1) * Q : nullptr;
    float P[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        const int b = g * V + v;
        float left = 0.f, right = 0.f;
        if (Qm) {
            for (int a = 0; a < Q; a++) left = fmaf(Qm[a], A.Mt[a * Q + b], left);
        } else {
            left = A.pi[b];
        }
        if (Qp) {
            for (int c = 0; c < Q; c++) right = fmaf(A.Mt[b * Q + c], Qp[c], right);
        } else {
            right = 1.f;
        }
        P[v] = left * right;
    }
    gnormalise<Q>(P, mask);
    stv<V>(out + g * V, P);
}

// Launchers (one instantiation set per schedule, see pus.cu / sus.cu).
// Check-node arithmetic: probability-domain convolution (q <= 16) or the
// deviation transform (any q).
enum Method { kDirect = 0, kTransform = 1, kTensor = 2 };

// Largest q for which AUTO takes the probability route (q^2 FMAs per
// convolution); above it AUTO takes the transform route (q log q).
constexpr int kAutoDirectMaxQ = 64;

// Per-device launch attributes (launch.cu): raise the kernel's dynamic
// shared-memory limit to smem on the current device if needed and return its
// CTAs per SM for (threads, smem) in *occ; thread-safe.
cudaError_t kernel_prepare(const void* fn, int threads, size_t smem, int* occ);
int device_sms();          // SMs of the current device
int device_optin_smem();   // opt-in shared memory per CTA of the current device

cudaError_t launch_channel(const DecodeArgs& A, cudaStream_t s);
bool sus_team_eligible(const DecodeArgs& A);
cudaError_t launch_sus_team(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus_wave(const DecodeArgs& A, int width, int num_sms, cudaStream_t s);
int sus_auto_width(const DecodeArgs& A, int num_sms);
bool sus_level_eligible(const DecodeArgs& A);
bool sus_level_sm_eligible(const DecodeArgs& A, int num_sms);
cudaError_t launch_sus_level_sm(const DecodeArgs& A, int num_sms, cudaStream_t s);
bool pus_regs_eligible(const DecodeArgs& A);
bool pus_res_eligible(const DecodeArgs& A);
bool sus_res_eligible(const DecodeArgs& A, int num_sms);
bool sus_l2_eligible(const DecodeArgs& A);
cudaError_t launch_sus_l2(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_pus_res(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus_res(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus_level(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus_level_tr(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus_level_tc(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_init_dev(const DecodeArgs& A, cudaStream_t s);
cudaError_t launch_pus(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_sus(const DecodeArgs& A, int num_sms, cudaStream_t s);
cudaError_t launch_init_dev(const DecodeArgs& A, cudaStream_t s);

// One persistent launch over the frames of several items (batch.cu): device
// arrays (items, prefix sums of their frame counts, kernel variants, frame
// counter, field-table owner per q) and the launch shape.
struct MixedLaunch {
    DecodeArgs* d_args = nullptr;
    int* d_prefix = nullptr;
    int* d_variant = nullptr;
    int* d_counter = nullptr;
    int* d_field = nullptr;
    int n_items = 0;
    int total = 0;
    int schedule = 0;
    int grid = 0;
    size_t pus_smem = 0;
    int grid_cta = 0;        // SUS: CTA-family kernel (level schedules)
    size_t cta_smem = 0;     // its dynamic shared memory (largest over the items' variants)
    int cta_threads = 128;   // its threads per CTA
    bool wide = false;       // 512 threads per CTA where 256 would do (frames large enough to use them)
    bool has_cta = false, has_warp = false;
};

void mixed_shape(MixedLaunch& m, const int* variants);
std::vector<int> heavy_first(const std::vector<const CodeDev*>& codes);
cudaError_t mixed_launch(const MixedLaunch& m, cudaStream_t s);
int tuned_variant(const gfbp_code* code, int schedule);
cudaError_t launch_fill_prior(const DecodeArgs& A, cudaStream_t s);
cudaError_t batch_prepare_item(DecodeArgs& A, void* ws, const gfbp_code* code, int32_t F, const float* obs,
                               gfbp_channel ch, gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter,
                               uint8_t* x_hat, int32_t* iters, uint8_t* conv, const gfbp_options* opt, int method,
                               size_t* ws_bytes, cudaStream_t stream);

}  // namespace gfbp

struct gfbp_code {
    gfbp::CodeDev dev;
    void* dmem;      // the single device allocation behind dev's pointers
    uint32_t poly;
    int device;
};
