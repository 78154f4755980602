// SUS (Sec. 2) by levels with the check node evaluated through the
// convolution theorem on plain transforms, each transform of the sweep taken
// on the tensor cores (wht_tc.cuh): the TENSOR check method, q >= 16.
//
// Stored per edge: F = WHT(relabelled q).  Per sub-piece of the level schedule
// (sus_level_tr.cuh has the schedule and why it keeps the sequential order):
//   1  lane group <-> pair (j, k): G = product of the check's other stored F,
//      staged as FP16 hi/lo rows of a power-of-two-scaled vector;
//   2  the CTA's warps: s = WHT(G) / q for every staged row (tensor cores);
//   3  group <-> pair: r[a] = max(s[z XOR h a], 0), normalised;
//   4  group <-> pair: q_kj from p_j and the column's other r (the product order
//      of the lane kernels), Q_j and the hard decision on slot 0, the
//      relabelled q staged as in 1;
//   5  the CTA's warps: F = WHT(relabelled q) for every staged row;
//   6  group <-> pair: F written to the edge slab.
// Barriers separate the steps.  The first stored F (q_ij <- p_j) comes from the
// initialisation kernel's FP32 butterflies.
#pragma once

#include "sus_level_tr.cuh"
#include "wht_tc.cuh"

namespace gfbp {

namespace {

// Shared layout of the kernel (floats / halves), for SUB pairs per sub-piece.
template <int Q, int T>
struct TcLay {
    static constexpr int SUB = level_tr_sub<Q>();
    static constexpr int S = tc_stride<Q>();
    static constexpr int NG = T / Lay<Q>::G;
    static constexpr size_t rows_bytes = sizeof(float) * (size_t)SUB * Q;
    static constexpr size_t stage_bytes = sizeof(__half) * 2 * (size_t)SUB * S;
    static constexpr size_t rs_bytes = sizeof(float) * (size_t)SUB;
    static constexpr size_t sc_bytes = sizeof(float) * (size_t)NG * (Q + 4);
    static constexpr size_t total = rows_bytes + stage_bytes + rs_bytes + sc_bytes;
    static_assert(SUB % 16 == 0, "tensor-core row blocks");
};

// A group's vector (V entries per lane) into staged row `row`: scaled by a
// power of two to a largest magnitude in [1, 2), split into FP16 hi / lo;
// rs receives the inverse scale.
template <int Q>
__device__ __forceinline__ void stage_vec(const float (&x)[Lay<Q>::V], __half* hi_row, __half* lo_row, float* rs,
                                          unsigned mask, int g) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    static_assert(V % 4 == 0, "four entries per lane at least");
    float m = 0.f;
#pragma unroll
    for (int v = 0; v < V; v++) m = fmaxf(m, fabsf(x[v]));
#pragma unroll
    for (int o = 1; o < G; o <<= 1) m = fmaxf(m, __shfl_xor_sync(mask, m, o));
    const float s = pow2_scale(m);
#pragma unroll
    for (int v = 0; v < V; v += 4) {
        __half h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; i++) split_hilo(x[v + i] * s, h[i], l[i]);
        *reinterpret_cast<uint2*>(hi_row + g * V + v) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(lo_row + g * V + v) = *reinterpret_cast<const uint2*>(l);
    }
    if (g == 0) *rs = 1.0f / s;
}

// Step 1: G = product of the other stored transforms of check k of column j.
template <int Q>
__device__ __forceinline__ void level_tc_check(const DecodeArgs& A, const float* slab, int2 pr, __half* hi_row,
                                               __half* lo_row, float* rs, unsigned mask, int g) {
    constexpr int V = Lay<Q>::V;
    if (A.c.colptr[pr.x + 1] == A.c.colptr[pr.x]) {   // a column without checks: a zero row
        const float zero[V] = {};
        stage_vec<Q>(zero, hi_row, lo_row, rs, mask, g);
        return;
    }
    const int4 in = A.c.cinfo[A.c.colptr[pr.x] + pr.y];
    const int own = in.x - in.y;
    const int dc = in.z & 255;
    float Gv[V];
#pragma unroll
    for (int v = 0; v < V; v++) Gv[v] = 1.f;
#pragma unroll 1
    for (int m = 0; m < dc; m++) {
        if (m == own) continue;
        float F[V];
        ldv<V>(F, slab + (size_t)(in.y + m) * Q + g * V);
#pragma unroll
        for (int v = 0; v < V; v++) Gv[v] *= F[v];
    }
    stage_vec<Q>(Gv, hi_row, lo_row, rs, mask, g);
}

// Step 3: r from the check's inverse transform s (row, scaled by 1/q).
template <int Q>
__device__ __forceinline__ void level_tc_finish(const DecodeArgs& A, const uint8_t* zf, int2 pr, float* row,
                                                unsigned mask, int g, const uint8_t* ex, const uint8_t* lg,
                                                int* zs) {
    constexpr int V = Lay<Q>::V;
    if (A.c.colptr[pr.x + 1] == A.c.colptr[pr.x]) return;   // a column without checks
    const int4 in = A.c.cinfo[A.c.colptr[pr.x] + pr.y];
    const int h = (in.z >> 8) & 255;
    const int z = zf ? (zf[in.w] & (Q - 1)) : 0;
    float R[V];
#pragma unroll
    for (int v = 0; v < V; v++) R[v] = fmaxf(row[(z ^ gf_mul(ex, lg, h, g * V + v)) & (Q - 1)], 0.0f);
    __syncwarp(mask);
    gnormalise<Q>(R, mask, zs);
    stv<V>(row + g * V, R);
}

// Step 4: q_kj, Q_j (slot 0), and the relabelled q staged for its transform.
template <int Q>
__device__ __forceinline__ void level_tc_var(const DecodeArgs& A, int f, uint8_t* xh, int2 pr, const float* rows0,
                                             __half* hi_row, __half* lo_row, float* rs, float* sc, unsigned mask,
                                             int g, const uint8_t* ex, const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    const int j = pr.x, k = pr.y;
    const int c0 = A.c.colptr[j];
    const int d = A.c.colptr[j + 1] - c0;
    const int4 in = d > 0 ? A.c.cinfo[c0 + k] : make_int4(0, 0, 0, 0);
    const int N = A.c.N;
    const float* r0 = rows0 - (size_t)k * Q;   // row of the column's slot 0
    float p[V];
    prior_vec<Q>(A, f, j, p, mask, g);
    float S[V], pre[V];
#pragma unroll
    for (int v = 0; v < V; v++) { S[v] = 1.f; pre[v] = 1.f; }
#pragma unroll 1
    for (int k2 = d - 1; k2 > k; k2--) {
        float r[V];
        ldv<V>(r, r0 + (size_t)k2 * Q + g * V);
#pragma unroll
        for (int v = 0; v < V; v++) S[v] *= r[v];
    }
#pragma unroll 1
    for (int k2 = 0; k2 < k; k2++) {
        float r[V];
        ldv<V>(r, r0 + (size_t)k2 * Q + g * V);
#pragma unroll
        for (int v = 0; v < V; v++) pre[v] *= r[v];
    }
    if (k == 0) {
        float r[V], Qj[V];
        if (d > 0) {
            ldv<V>(r, r0 + g * V);
        } else {   // no checks: Q_j = p_j
#pragma unroll
            for (int v = 0; v < V; v++) r[v] = 1.f;
        }
#pragma unroll
        for (int v = 0; v < V; v++) Qj[v] = p[v] * (S[v] * r[v]);
        gnormalise<Q>(Qj, mask, zsum_of(A, f));
        const int a = gargmax<Q>(Qj, mask, g);
        if (g == 0) xh[j] = (uint8_t)a;
        if (A.post) stv<V>(A.post + ((size_t)f * N + j) * Q + g * V, Qj);
        if (A.markov) {
            const int si = A.src_index[j];
            if (si >= 0) stv<V>(A.Qsrc + ((size_t)f * A.K + si) * Q + g * V, Qj);
        }
    }
    if (d == 0) {   // nothing to store; stage a zero row for the warps' transform
        const float zero[V] = {};
        stage_vec<Q>(zero, hi_row, lo_row, rs, mask, g);
        return;
    }
    float x[V];
#pragma unroll
    for (int v = 0; v < V; v++) x[v] = p[v] * (pre[v] * S[v]);
    gnormalise<Q>(x, mask, zsum_of(A, f));
    if (A.step) stv<V>(A.msg_io + ((size_t)f * A.c.E + in.x) * Q + g * V, x);
    // relabelled: qt[b] = q[h^-1 b]
    const int h = (in.z >> 8) & 255;
    stv<V>(sc + g * V, x);
    __syncwarp(mask);
    float y[V];
#pragma unroll
    for (int v = 0; v < V; v++) y[v] = sc[gf_div<Q>(ex, lg, g * V + v, h)];
    __syncwarp(mask);
    stage_vec<Q>(y, hi_row, lo_row, rs, mask, g);
}

template <int Q, int T>
__device__ __forceinline__ void sus_level_tc_frame(const DecodeArgs& A, int f, const uint8_t* s_exp,
                                                   const uint8_t* s_log, uint8_t* dyn) {
    using L = TcLay<Q, T>;
    constexpr int G = Lay<Q>::G, V = Lay<Q>::V, NG = L::NG, SUB = L::SUB, S = L::S;
    float* rows = reinterpret_cast<float*>(dyn);
    __half* hi = reinterpret_cast<__half*>(dyn + L::rows_bytes);
    __half* lo = hi + (size_t)SUB * S;
    float* rs = reinterpret_cast<float*>(dyn + L::rows_bytes + L::stage_bytes);
    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const int grp = tid / G;
    const int warp = tid >> 5;
    float* sc = reinterpret_cast<float*>(dyn + L::rows_bytes + L::stage_bytes + L::rs_bytes) + (size_t)grp * (Q + 4);
    const unsigned mask = group_mask<G>();
    const int M = A.c.M, N = A.c.N;
    float* slab = A.msg + (size_t)f * A.c.E * Q;
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
#pragma unroll 1
        for (int pc = 0; pc < A.c.npieces; pc++) {
            const int pe = A.c.lpiece[pc + 1];
            for (int s = A.c.lpiece[pc]; s < pe;) {
                int e = s + SUB < pe ? s + SUB : pe;
                while (e < pe && A.c.lpair[e].y != 0) e--;
                const int n = e - s;
                for (int lp = grp; lp < n; lp += NG)
                    level_tc_check<Q>(A, slab, A.c.lpair[s + lp], hi + (size_t)lp * S, lo + (size_t)lp * S, rs + lp,
                                      mask, g);
                __syncthreads();
                tc_wht_rows<Q>(hi, lo, rs, n, rows, Q, 1.0f / Q, warp, T / 32);
                __syncthreads();
                for (int lp = grp; lp < n; lp += NG)
                    level_tc_finish<Q>(A, zf, A.c.lpair[s + lp], rows + (size_t)lp * Q, mask, g, s_exp, s_log,
                                       zsum_of(A, f));
                __syncthreads();
                for (int lp = grp; lp < n; lp += NG)
                    level_tc_var<Q>(A, f, xh, A.c.lpair[s + lp], rows + (size_t)lp * Q, hi + (size_t)lp * S,
                                    lo + (size_t)lp * S, rs + lp, sc, mask, g, s_exp, s_log);
                __syncthreads();
                tc_wht_rows<Q>(hi, lo, rs, n, rows, Q, 1.0f, warp, T / 32);
                __syncthreads();
                for (int lp = grp; lp < n; lp += NG) {
                    const int2 pr = A.c.lpair[s + lp];
                    if (A.c.colptr[pr.x + 1] == A.c.colptr[pr.x]) continue;   // no edge to store
                    const int ed = A.c.cinfo[A.c.colptr[pr.x] + pr.y].x;
                    float F[V];
                    ldv<V>(F, rows + (size_t)lp * Q + g * V);
                    stv<V>(slab + (size_t)ed * Q + g * V, F);
                }
                __syncthreads();
                s = e;
            }
        }
        int bad = 0;
        for (int i = tid; i < M; i += T) {
            int sy = 0;
            for (int e = A.c.rowptr[i]; e < A.c.rowptr[i + 1]; e++)
                sy ^= gf_mul(s_exp, s_log, A.c.eh[e], xh[A.c.ecol[e]]);
            bad |= (sy != (zf ? (zf[i] & (Q - 1)) : 0));
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
            for (int i = grp; i < A.K; i += NG) markov_prior<Q>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, mask, g);
            __syncthreads();
        }
        if (A.fstate && t - t0 >= A.round_iters) break;
    }
    if (A.step && A.markov && A.prior_out) {
        for (int i = grp; i < A.K; i += NG)
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

template <int Q, int T>
__global__ void __launch_bounds__(T) k_sus_level_tc(const DecodeArgs A) {
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ int s_f;
    extern __shared__ __align__(16) uint8_t s_dyn8[];
    const int tid = threadIdx.x;
    for (int k = tid; k < 512; k += T) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += T) s_log[k] = A.c.glog[k];
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        sus_level_tc_frame<Q, T>(A, f, s_exp, s_log, s_dyn8);
    }
}

}  // namespace
}  // namespace gfbp
