// Sequential updating scheme (SUS; Sec. 2, steps 1-4): one lane group per
// frame, persistent over a frame counter.  For j = 0..N-1 strictly in order:
// step 1, r_ij for every check i of column j from the current q of the
// check's other edges (Eq. 3); step 2, q_ij for column j (Eq. 4); Q_j (Eq. 5)
// from the same r_ij.  After the sweep: hard decision test H x = z and the
// block-prior update (Eqs. 6-7).  Parallelism inside a frame comes only from
// the q entries of a vector (the group's lanes); frames run side by side.
//
// The slab holds, per edge, the Walsh-Hadamard transform of the distribution
// of h_ij x_j under q_ij, so step 1 is a product of stored transforms followed
// by one inverse transform.  Each lane only ever touches its own slice of
// every vector in global memory, so no cross-lane memory ordering is needed
// for the slab.
#include "gfbp_internal.cuh"

namespace gfbp {

namespace {

constexpr int kSusThreads = 128;

template <int Q, int DC, int DV>
__global__ void __launch_bounds__(kSusThreads) k_sus(const DecodeArgs A) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    __shared__ uint8_t s_exp[512];
    __shared__ uint8_t s_log[256];
    __shared__ __align__(16) float s_scr[kSusThreads * V];

    const int tid = threadIdx.x;
    const int g = tid & (G - 1);
    const int grp = tid / G;
    const unsigned mask = group_mask<G>();
    float* sc = s_scr + grp * Q;
    for (int k = tid; k < 512; k += blockDim.x) s_exp[k] = A.c.gexp[k];
    for (int k = tid; k < 256; k += blockDim.x) s_log[k] = A.c.glog[k];
    __syncthreads();
    const int M = A.c.M, N = A.c.N;
    const long long E = A.c.E;
    const int* __restrict__ rowptr = A.c.rowptr;
    const int* __restrict__ colptr = A.c.colptr;
    const int* __restrict__ cedge = A.c.cedge;
    const int* __restrict__ erow = A.c.erow;
    const uint8_t* __restrict__ eh = A.c.eh;

    for (;;) {
        int f = 0;
        if (g == 0) f = atomicAdd(A.work, 1);
        f = __shfl_sync(mask, f, threadIdx.x & 31 & ~(G - 1));
        if (f >= A.F) break;
        float* slab = A.msg + (size_t)f * E * Q;
        const uint8_t* zf = A.syn ? A.syn + (size_t)f * M : nullptr;
        uint8_t* xh = A.xhat + (size_t)f * N;

        for (long long e = 0; e < E; e++) {
            float x[V];
            if (A.step) {
                ldv<V>(x, A.msg_io + ((size_t)f * E + e) * Q + g * V);
            } else {
                prior_vec<Q>(A, f, A.c.ecol[e], x, mask, g);
            }
            to_transform<Q>(x, eh[e], sc, mask, g, s_exp, s_log);
            stv<V>(slab + (size_t)e * Q + g * V, x);
        }

        int t = 1, ok = 0;
        for (;; t++) {
            for (int j = 0; j < N; j++) {
                const int c0 = colptr[j];
                const int d = colptr[j + 1] - c0;
                // step 1: r_ij for every check i of column j
                float R[DV][V];
#pragma unroll
                for (int k = 0; k < DV; k++) {
                    if (k < d) {
                        const int e = cedge[c0 + k];
                        const int i = erow[e];
                        const int e0 = rowptr[i];
                        const int dc = rowptr[i + 1] - e0;
                        float x[V];
#pragma unroll
                        for (int v = 0; v < V; v++) x[v] = 1.f;
#pragma unroll
                        for (int m = 0; m < DC; m++) {
                            if (m < dc && e0 + m != e) {
                                float y[V];
                                ldv<V>(y, slab + (size_t)(e0 + m) * Q + g * V);
#pragma unroll
                                for (int v = 0; v < V; v++) x[v] *= y[v];
                            }
                        }
                        check_finish<Q>(x, eh[e], zf ? (zf[i] & (Q - 1)) : 0, sc, mask, g, s_exp, s_log);
#pragma unroll
                        for (int v = 0; v < V; v++) R[k][v] = x[v];
                    }
                }
                // step 2: q_ij for column j, and Q_j
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
                            acc[v] *= R[k][v];
                        }
                    }
                }
                {
                    float Qj[V];
#pragma unroll
                    for (int v = 0; v < V; v++) Qj[v] = p[v] * acc[v];
                    gnormalise<Q>(Qj, mask);
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
                        const int e = cedge[c0 + k];
                        float x[V];
#pragma unroll
                        for (int v = 0; v < V; v++) {
                            x[v] = p[v] * (pre[v] * S[k][v]);
                            pre[v] *= R[k][v];
                        }
                        gnormalise<Q>(x, mask);
                        if (A.step) stv<V>(A.msg_io + ((size_t)f * E + e) * Q + g * V, x);
                        to_transform<Q>(x, eh[e], sc, mask, g, s_exp, s_log);
                        stv<V>(slab + (size_t)e * Q + g * V, x);
                    }
                }
            }
            __syncwarp(mask);
            // hard decisions are in xh; test H x = z over the group's lanes
            int bad = 0;
            for (int i = g; i < M; i += G) {
                int s = 0;
                for (int e = rowptr[i]; e < rowptr[i + 1]; e++) s ^= gf_mul(s_exp, s_log, eh[e], xh[A.c.ecol[e]]);
                bad |= (s != (zf ? (zf[i] & (Q - 1)) : 0));
            }
#pragma unroll
            for (int m = 1; m < G; m <<= 1) bad |= __shfl_xor_sync(mask, bad, m);
            ok = !bad;
            if (A.trace) {
                uint8_t* tr = A.trace + ((size_t)f * A.max_iter + (t - 1)) * N;
                for (int j = g; j < N; j += G) tr[j] = xh[j];
            }
            if ((ok && A.early_stop) || t >= A.max_iter) break;
            if (A.markov) {
                for (int i = 0; i < A.K; i++) markov_prior<Q>(A, f, i, A.P + ((size_t)f * A.K + i) * Q, mask, g);
                __syncwarp(mask);
            }
        }
        if (A.step && A.markov && A.prior_out) {
            for (int i = 0; i < A.K; i++) markov_prior<Q>(A, f, i, A.prior_out + ((size_t)f * A.K + i) * Q, mask, g);
        }
        if (A.trace) {
            for (size_t o = (size_t)t * N + g; o < (size_t)A.max_iter * N; o += G)
                A.trace[(size_t)f * A.max_iter * N + o] = 255;
        }
        if (g == 0) {
            if (A.iters) A.iters[f] = t;
            A.conv[f] = (uint8_t)ok;
        }
        __syncwarp(mask);
    }
}

template <int Q, int DC, int DV>
cudaError_t launch_q(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    constexpr int G = Lay<Q>::G;
    constexpr int groups_per_block = kSusThreads / G;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sus<Q, DC, DV>, kSusThreads, 0);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    long long want = ((long long)A.F + groups_per_block - 1) / groups_per_block;
    long long cap = (long long)num_sms * occ;
    long long grid = want < cap ? want : cap;
    if (grid < 1) return cudaSuccess;
    k_sus<Q, DC, DV><<<(int)grid, kSusThreads, 0, s>>>(A);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_deg(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    if (A.c.dcmax <= 6 && A.c.dvmax <= 3) return launch_q<Q, 6, 3>(A, num_sms, s);
    return launch_q<Q, 16, 8>(A, num_sms, s);
}

}  // namespace

cudaError_t launch_sus(const DecodeArgs& A, int num_sms, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_deg<2>(A, num_sms, s);
    case 4: return launch_deg<4>(A, num_sms, s);
    case 8: return launch_deg<8>(A, num_sms, s);
    case 16: return launch_deg<16>(A, num_sms, s);
    case 32: return launch_deg<32>(A, num_sms, s);
    case 64: return launch_deg<64>(A, num_sms, s);
    case 128: return launch_deg<128>(A, num_sms, s);
    case 256: return launch_deg<256>(A, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gfbp
