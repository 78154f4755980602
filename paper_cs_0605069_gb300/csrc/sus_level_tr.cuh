// SUS (Sec. 2) by levels of the column order with a lane group per (column,
// check) pair: the transform route of the check node (any q), or the
// probability route by shared-memory XOR-convolutions (the route AUTO takes
// for q >= 32, where the q <= 16 register kernels do not apply).
//
// The level schedule is the one of sus_level.cuh: the columns of a level share
// no check, so updating a level's columns at once gives every column the
// operands of the sequential order.  A CTA decodes one frame and walks the
// code's pieces (whole columns of one level); a piece is taken in sub-pieces of
// at most SUB pairs so that its r-vectors fit in shared memory:
//   step 1  group <-> pair (j, k): the check's other stored deviation vectors
//           combined (E <- E + D (1 - E)), inverted to r_kj (dev_finish_n) and
//           kept in a shared row; probability route: the check's other stored
//           relabelled messages folded by XOR-convolutions in the order of
//           their positions (the first one is the start), relabelled and
//           normalised (direct_finish_n);
//   step 2  after a barrier, group <-> pair (j, k): q_kj from p_j and the
//           column's other rows, in the product order of sus_column_tail (and
//           on slot 0, Q_j, the hard decision, the posterior), brought to the
//           stored form of the route and written to the slab.
// Each step calls the lane-group kernel's own routines on one vector at a
// time, so the two kernels give the same bits.
#pragma once

#include "sus_group.cuh"

namespace gfbp {

namespace {

// pairs of a sub-piece: r rows of at most 32 KB
template <int Q>
constexpr int level_tr_sub() {
    return (32768 / (Q * 4)) < kLevelPiece ? (32768 / (Q * 4)) : kLevelPiece;
}

template <int Q, int METHOD>
__device__ __forceinline__ void level_tr_check(const DecodeArgs& A, const float* slab, const uint8_t* zf, int2 pr,
                                               float* row, float* sc, unsigned mask, int g, const uint8_t* ex,
                                               const uint8_t* lg, int* zs) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    const int j = pr.x, k = pr.y;
    if (A.c.colptr[j + 1] == A.c.colptr[j]) return;   // a column without checks
    const int4 in = A.c.cinfo[A.c.colptr[j] + k];
    const int own = in.x - in.y;
    const int dc = in.z & 255;
    const int lane0 = (threadIdx.x & 31) & ~(G - 1);
    float E[1][V];
    int C[1] = {0};
    const int h[1] = {(in.z >> 8) & 255};
    const int z[1] = {zf ? (zf[in.w] & (Q - 1)) : 0};
    if constexpr (METHOD == kDirect) {
        bool started = false;
#pragma unroll 1
        for (int m = 0; m < dc; m++) {
            if (m == own) continue;
            const float* Y = slab + (size_t)(in.y + m) * Q;
            if (!started) {
                ldv<V>(E[0], Y + g * V);
                started = true;
            } else {
                stv<V>(sc + g * V, E[0]);
                __syncwarp(mask);
                xconv_sm<Q>(E[0], sc, Y, g);
                __syncwarp(mask);
            }
        }
        if (!started) {   // a check of degree 1: the XOR-sum of no other edges is 0
#pragma unroll
            for (int v = 0; v < V; v++) E[0][v] = (g * V + v) == 0 ? 1.f : 0.f;
        }
        direct_finish_n<Q, 1>(E, h, z, 1, sc, mask, g, ex, lg, zs);
        stv<V>(row + g * V, E[0]);
        return;
    }
#pragma unroll
    for (int v = 0; v < V; v++) E[0][v] = 0.f;
#pragma unroll 1
    for (int m = 0; m < dc; m++) {
        if (m == own) continue;
        float Y[V];
        ldv<V>(Y, slab + (size_t)(in.y + m) * Q + g * V);
        if (g == 0) {
            C[0] ^= (int)Y[0];
            Y[0] = 0.f;
        }
        dev_combine<V>(E[0], Y);
    }
    C[0] = __shfl_sync(mask, C[0], lane0);
    dev_finish_n<Q, 1>(E, C, h, z, 1, sc, mask, g, ex, lg, zs);
    stv<V>(row + g * V, E[0]);
}

template <int Q, int METHOD>
__device__ __forceinline__ void level_tr_var(const DecodeArgs& A, int f, float* slab, uint8_t* xh, int2 pr,
                                             const float* rows0, float* sc, unsigned mask, int g, const uint8_t* ex,
                                             const uint8_t* lg) {
    constexpr int V = Lay<Q>::V;
    const int j = pr.x, k = pr.y;
    const int c0 = A.c.colptr[j];
    const int d = A.c.colptr[j + 1] - c0;
    const int4 in = d > 0 ? A.c.cinfo[c0 + k] : make_int4(0, 0, 0, 0);
    const int N = A.c.N;
    const float* r0 = rows0 - (size_t)k * Q;   // row of the column's slot 0
    float p[V];
    prior_vec<Q>(A, f, j, p, mask, g);
    // S_k: product of the rows after k, taken from the last one down; pre:
    // product of the rows before k, from the first one up
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
        // acc: every row from the last one down (S times row 0, in that order)
        float acc[V], r[V];
        if (d > 0) {
            ldv<V>(r, r0 + g * V);
        } else {   // no checks: Q_j = p_j
#pragma unroll
            for (int v = 0; v < V; v++) r[v] = 1.f;
        }
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = S[v] * r[v];
        float Qj[V];
#pragma unroll
        for (int v = 0; v < V; v++) Qj[v] = p[v] * acc[v];
        gnormalise<Q>(Qj, mask, zsum_of(A, f));
        const int a = gargmax<Q>(Qj, mask, g);
        if (g == 0) xh[j] = (uint8_t)a;
        if (A.post) stv<V>(A.post + ((size_t)f * N + j) * Q + g * V, Qj);
        if (A.markov) {
            const int si = A.src_index[j];
            if (si >= 0) stv<V>(A.Qsrc + ((size_t)f * A.K + si) * Q + g * V, Qj);
        }
    }
    if (d == 0) return;
    float x[1][V];
#pragma unroll
    for (int v = 0; v < V; v++) x[0][v] = p[v] * (pre[v] * S[v]);
    gnormalise<Q>(x[0], mask, zsum_of(A, f));
    if (A.step) stv<V>(A.msg_io + ((size_t)f * A.c.E + in.x) * Q + g * V, x[0]);
    const int h[1] = {(in.z >> 8) & 255};
    if constexpr (METHOD == kDirect) to_relabelled_n<Q, 1>(x, h, 1, sc, mask, g, ex, lg);
    else to_deviation_n<Q, 1>(x, h, 1, sc, mask, g, ex, lg);
    stv<V>(slab + (size_t)in.x * Q + g * V, x[0]);
}

template <int Q, int T, int METHOD = kTransform>
__device__ __forceinline__ void sus_level_tr_frame(const DecodeArgs& A, int f, const uint8_t* s_exp,
                                                   const uint8_t* s_log, float* s_rows, float* sc) {
    constexpr int G = Lay<Q>::G, NG = T / G, SUB = level_tr_sub<Q>();
    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const int grp = tid / G;
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
                // sub-piece [s, e): whole columns, at most SUB pairs
                int e = s + SUB < pe ? s + SUB : pe;
                while (e < pe && A.c.lpair[e].y != 0) e--;
                const int n = e - s;
                for (int lp = grp; lp < n; lp += NG)
                    level_tr_check<Q, METHOD>(A, slab, zf, A.c.lpair[s + lp], s_rows + (size_t)lp * Q, sc, mask, g, s_exp,
                                              s_log, zsum_of(A, f));
                __syncthreads();
                for (int lp = grp; lp < n; lp += NG)
                    level_tr_var<Q, METHOD>(A, f, slab, xh, A.c.lpair[s + lp], s_rows + (size_t)lp * Q, sc, mask, g, s_exp,
                                    s_log);
                __syncthreads();
                s = e;
            }
        }
        int bad = 0;
        for (int i = tid; i < M; i += T) {
            int s = 0;
            for (int e = A.c.rowptr[i]; e < A.c.rowptr[i + 1]; e++)
                s ^= gf_mul(s_exp, s_log, A.c.eh[e], xh[A.c.ecol[e]]);
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

// Dynamic shared memory: SUB rows of Q floats, then one Q-float scratch
// (+ padding) per lane group.
template <int Q, int T, int METHOD>
__global__ void __launch_bounds__(T) k_sus_level_tr(const DecodeArgs A) {
    constexpr int G = Lay<Q>::G, SUB = level_tr_sub<Q>();
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ int s_f;
    extern __shared__ __align__(16) float s_dyn[];
    const int tid = threadIdx.x;
    float* s_rows = s_dyn;
    float* sc = s_dyn + (size_t)SUB * Q + (size_t)(tid / G) * (Q + 4);
    for (int k = tid; k < 512; k += T) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += T) s_log[k] = A.c.glog[k];
    for (;;) {
        __syncthreads();
        if (tid == 0) s_f = atomicAdd(A.work, 1);
        __syncthreads();
        const int f = s_f;
        if (f >= A.F) break;
        sus_level_tr_frame<Q, T, METHOD>(A, f, s_exp, s_log, s_rows, sc);
    }
}

template <int Q, int T>
constexpr size_t level_tr_smem() {
    return sizeof(float) * ((size_t)level_tr_sub<Q>() * Q + (size_t)(T / Lay<Q>::G) * (Q + 4));
}

}  // namespace
}  // namespace gfbp
