// gfbp_decode / gfbp_step: argument checks, workspace layout, the channel
// likelihood kernel and dispatch to the schedule kernels.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gfbp_internal.cuh"

namespace gfbp {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

constexpr int kChanThreads = 256;

// Channel likelihoods (Sec. 2 and its footnote on other channels), one lane
// group per symbol, normalised:
//   BSC:     (1-f)^(p-n) f^n, n = bits where a and the received symbol differ,
//            formed as r^n with r = f/(1-f) (or the mirror for f > 1/2);
//   BEC:     1 when a agrees with every non-erased bit (2 = erased), else 0;
//   BI-AWGN: exp(-sum_k (y_k - s_k(a))^2 / (2 sigma^2)) with BPSK bit 0 -> +1,
//            formed relative to its maximum: exp(-sum over bits whose sign
//            disagrees with y_k of 2|y_k|/sigma^2);
//   LOGLIK:  exp(obs_a - max);
//   punctured symbols: uniform.
template <int Q>
__global__ void __launch_bounds__(kChanThreads) k_channel(const DecodeArgs A) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    constexpr int P = (Q == 2) ? 1 : (Q == 4) ? 2 : (Q == 8) ? 3 : (Q == 16) ? 4 : (Q == 32) ? 5 : (Q == 64) ? 6 : (Q == 128) ? 7 : 8;
    const int g = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const long long groups = (long long)gridDim.x * (blockDim.x / G);
    const long long total = (long long)A.F * A.c.N;
    for (long long it = (long long)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; it < total; it += groups) {
        const int f = (int)(it / A.c.N);
        const int j = (int)(it % A.c.N);
        float x[V];
        const bool punct = A.punct && A.punct[j];
        const float prm = A.frame_param ? A.frame_param[f] : A.ch_param;
        if (punct) {
#pragma unroll
            for (int v = 0; v < V; v++) x[v] = 1.f;
        } else if (A.ch_kind == GFBP_LOGLIK) {
            const float* y = A.obs + (size_t)it * Q;
            float mx = -INFINITY;
#pragma unroll
            for (int v = 0; v < V; v++) { x[v] = y[g * V + v]; mx = fmaxf(mx, x[v]); }
#pragma unroll
            for (int m = 1; m < G; m <<= 1) mx = fmaxf(mx, __shfl_xor_sync(mask, mx, m));
#pragma unroll
            for (int v = 0; v < V; v++) x[v] = expf(x[v] - mx);
        } else {
            const float* y = A.obs + (size_t)it * P;
            int rx = 0, era = 0;
            float wgt[P];
#pragma unroll
            for (int k = 0; k < P; k++) {
                const float yk = y[k];
                if (A.ch_kind == GFBP_BIAWGN) {
                    rx |= (yk < 0.f) << k;   // bit whose BPSK sign agrees with y_k
                    wgt[k] = 2.f * fabsf(yk) / (prm * prm);
                } else {
                    rx |= (yk > 0.5f && yk < 1.5f) << k;
                    era |= (yk > 1.5f) << k;
                    wgt[k] = 0.f;
                }
            }
            if (A.ch_kind == GFBP_BSC) {
                const bool mirror = prm > 0.5f;
                const float r = mirror ? (1.f - prm) / prm : prm / (1.f - prm);
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const int n = __popc((g * V + v) ^ rx);
                    float w = 1.f;
                    for (int k = 0; k < (mirror ? P - n : n); k++) w *= r;
                    x[v] = w;
                }
            } else if (A.ch_kind == GFBP_BEC) {
#pragma unroll
                for (int v = 0; v < V; v++) x[v] = (((g * V + v) ^ rx) & ~era) ? 0.f : 1.f;
            } else {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const int dis = (g * V + v) ^ rx;
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < P; k++)
                        if ((dis >> k) & 1) s += wgt[k];
                    x[v] = expf(-s);
                }
            }
        }
        gnormalise<Q>(x, mask);
        stv<V>(A.L + (size_t)it * Q + g * V, x);
    }
}

template <int Q>
cudaError_t launch_channel_q(const DecodeArgs& A, cudaStream_t s) {
    constexpr int G = Lay<Q>::G;
    const long long total = (long long)A.F * A.c.N;
    long long blocks = (total + (kChanThreads / G) - 1) / (kChanThreads / G);
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (blocks < 1) return cudaSuccess;
    k_channel<Q><<<(unsigned)blocks, kChanThreads, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_channel(const DecodeArgs& A, cudaStream_t s) {
    switch (A.c.q) {
    case 2: return launch_channel_q<2>(A, s);
    case 4: return launch_channel_q<4>(A, s);
    case 8: return launch_channel_q<8>(A, s);
    case 16: return launch_channel_q<16>(A, s);
    case 32: return launch_channel_q<32>(A, s);
    case 64: return launch_channel_q<64>(A, s);
    case 128: return launch_channel_q<128>(A, s);
    case 256: return launch_channel_q<256>(A, s);
    }
    return cudaErrorInvalidValue;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t L, msg, Qsrc, P, Mt, pi, src_index, src_pos, work, total;
};

Layout layout(const CodeDev& c, long long F, bool markov, int K, bool step) {
    Layout l{};
    size_t o = 0;
    const size_t q = (size_t)c.q;
    l.work = o; o += 256;
    l.L = o; o += align256(sizeof(float) * (size_t)F * c.N * q);
    l.msg = o; o += align256(sizeof(float) * (size_t)F * (size_t)c.E * q);
    if (markov) {
        l.Qsrc = o; o += align256(sizeof(float) * (size_t)F * K * q);
        if (!step) { l.P = o; o += align256(sizeof(float) * (size_t)F * K * q); }
        l.Mt = o; o += align256(sizeof(float) * q * q);
        l.pi = o; o += align256(sizeof(float) * q);
        l.src_index = o; o += align256(sizeof(int) * (size_t)c.N);
        l.src_pos = o; o += align256(sizeof(int) * (size_t)K);
    }
    l.total = o;
    return l;
}

// Stationary distribution of a row-stochastic matrix (pi T = pi, sum 1), by
// Gaussian elimination with partial pivoting on (T^T - I) with one row
// replaced by the normalisation.
bool stationary(const std::vector<double>& T, int q, std::vector<double>& pi) {
    std::vector<double> A((size_t)q * (q + 1));
    for (int r = 0; r < q; r++) {
        for (int c = 0; c < q; c++) A[r * (q + 1) + c] = (r == q - 1) ? 1.0 : T[c * q + r] - (r == c ? 1.0 : 0.0);
        A[r * (q + 1) + q] = (r == q - 1) ? 1.0 : 0.0;
    }
    for (int c = 0; c < q; c++) {
        int pv = c;
        for (int r = c + 1; r < q; r++)
            if (std::fabs(A[r * (q + 1) + c]) > std::fabs(A[pv * (q + 1) + c])) pv = r;
        if (std::fabs(A[pv * (q + 1) + c]) < 1e-300) return false;
        if (pv != c)
            for (int k = 0; k <= q; k++) std::swap(A[c * (q + 1) + k], A[pv * (q + 1) + k]);
        for (int r = 0; r < q; r++) {
            if (r == c) continue;
            const double f = A[r * (q + 1) + c] / A[c * (q + 1) + c];
            if (f == 0.0) continue;
            for (int k = c; k <= q; k++) A[r * (q + 1) + k] -= f * A[c * (q + 1) + k];
        }
    }
    pi.assign(q, 0.0);
    for (int r = 0; r < q; r++) pi[r] = A[r * (q + 1) + q] / A[r * (q + 1) + r];
    return true;
}

gfbp_status cuda_fail(const char* where, cudaError_t e) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GFBP_ENOMEM : GFBP_ECUDA;
}

struct Common {
    bool markov = false;
    bool gs = false;
    int K = 0;
    std::vector<float> Mt, pi;
    std::vector<int> src_index, src_pos;
};

gfbp_status check_common(const char* fn, const gfbp_code* code, int32_t F, const float* obs, gfbp_channel ch,
                         gfbp_schedule schedule, const gfbp_prior* prior, Common& C) {
    const std::string w(fn);
    if (!code) { set_error(w + ": NULL code"); return GFBP_EINVAL; }
    if (F < 0) { set_error(w + ": n_frames < 0"); return GFBP_EINVAL; }
    if (F > 0 && !obs) { set_error(w + ": NULL obs"); return GFBP_EINVAL; }
    if (ch.kind < GFBP_BSC || ch.kind > GFBP_LOGLIK) { set_error(w + ": unknown channel kind"); return GFBP_EINVAL; }
    if (!ch.frame_param) {
        if (ch.kind == GFBP_BSC && !(ch.param > 0.f && ch.param < 1.f)) {
            set_error(w + ": BSC flip rate must be in (0, 1)");
            return GFBP_EINVAL;
        }
        if (ch.kind == GFBP_BIAWGN && !(ch.param > 0.f && std::isfinite(ch.param))) {
            set_error(w + ": BI-AWGN sigma must be > 0");
            return GFBP_EINVAL;
        }
    }
    if (schedule != GFBP_PUS && schedule != GFBP_SUS) { set_error(w + ": unknown schedule"); return GFBP_EINVAL; }
    const int q = code->dev.q, N = code->dev.N;
    if (prior && (prior->kind == GFBP_PRIOR_MARKOV || prior->kind == GFBP_PRIOR_MARKOV_GS)) {
        C.gs = prior->kind == GFBP_PRIOR_MARKOV_GS;
        if (!prior->T || prior->K < 1 || prior->K > N) {
            set_error(w + ": Markov prior needs T and 1 <= K <= N");
            return GFBP_EINVAL;
        }
        C.markov = true;
        C.K = prior->K;
        std::vector<double> T((size_t)q * q);
        for (int a = 0; a < q; a++) {
            double s = 0.0;
            for (int b = 0; b < q; b++) {
                const double t = prior->T[a * q + b];
                if (!(t >= 0.0) || !std::isfinite(t)) { set_error(w + ": T entries must be finite and >= 0"); return GFBP_EINVAL; }
                s += t;
            }
            if (!(s > 0.0)) { set_error(w + ": T has a zero row"); return GFBP_EINVAL; }
            for (int b = 0; b < q; b++) T[a * q + b] = prior->T[a * q + b] / s;
        }
        std::vector<double> pi;
        if (!stationary(T, q, pi)) { set_error(w + ": T has no unique stationary distribution"); return GFBP_EINVAL; }
        C.Mt.assign(T.begin(), T.end());
        C.pi.assign(pi.begin(), pi.end());
        C.src_index.assign(N, -1);
        C.src_pos.resize(C.K);
        for (int i = 0; i < C.K; i++) {
            const int j = prior->src_pos ? prior->src_pos[i] : i;
            if (j < 0 || j >= N || C.src_index[j] != -1) {
                set_error(w + ": src_pos must hold distinct positions in [0, N)");
                return GFBP_EINVAL;
            }
            C.src_index[j] = i;
            C.src_pos[i] = j;
        }
    } else if (prior && prior->kind != GFBP_PRIOR_IID) {
        set_error(w + ": unknown prior kind");
        return GFBP_EINVAL;
    }
    return GFBP_OK;
}

// DecodeArgs of one call, without the workspace pointers.
gfbp_status fill_args(DecodeArgs& A, const gfbp_code* code, int32_t F, const float* obs, gfbp_channel ch,
                      const Common& C, int32_t max_iter, bool step, uint8_t* x_hat, int32_t* iters, uint8_t* conv,
                      float* msg_io, float* prior_out, const gfbp_options* opt) {
    const CodeDev& c = code->dev;
    A = DecodeArgs{};
    A.c = c;
    A.F = F;
    A.obs = obs;
    A.ch_kind = ch.kind;
    A.ch_param = ch.param;
    A.frame_param = ch.frame_param;
    A.punct = opt ? opt->punct : nullptr;
    A.syn = opt ? opt->syndrome : nullptr;
    A.max_iter = max_iter;
    A.early_stop = (opt && opt->no_early_stop && !step) ? 0 : 1;
    A.markov = C.markov;
    A.markov_gs = C.gs;
    A.K = C.K;
    A.xhat = x_hat;
    A.iters = iters;
    A.conv = conv;
    A.post = opt ? opt->post : nullptr;
    A.trace = (opt && !step) ? opt->xhat_trace : nullptr;
    A.step = step;
    A.msg_io = msg_io;
    A.prior_out = prior_out;
    A.zsum = opt ? opt->zero_sums : nullptr;
    const int m = opt ? opt->check_method : GFBP_CHECK_AUTO;
    if (m < GFBP_CHECK_AUTO || m > GFBP_CHECK_TENSOR) {
        set_error("unknown check_method");
        return GFBP_EINVAL;
    }
    if (m == GFBP_CHECK_TENSOR && c.q < 16) {
        set_error("check_method TENSOR needs q >= 16");
        return GFBP_EUNSUPPORTED;
    }
    A.method = m == GFBP_CHECK_TENSOR ? kTensor
             : (m == GFBP_CHECK_TRANSFORM || (m == GFBP_CHECK_AUTO && c.q > kAutoDirectMaxQ)) ? kTransform : kDirect;
    A.width = opt ? opt->sus_width : 0;
    A.layout = opt ? opt->layout : GFBP_LAYOUT_AUTO;
    if (A.layout < GFBP_LAYOUT_AUTO || A.layout > GFBP_LAYOUT_L2RESIDENT) {
        set_error("unknown layout");
        return GFBP_EINVAL;
    }
    if (A.width != 0 && A.width != 1 && A.width != 2 && A.width != 4 && A.width != 8) {
        set_error("sus_width must be 0, 1, 2, 4 or 8");
        return GFBP_EINVAL;
    }
    A.partials = opt ? opt->sus_partials : GFBP_PARTIALS_AUTO;
    if (A.partials < GFBP_PARTIALS_AUTO || A.partials > GFBP_PARTIALS_RUNNING_GLOBAL) {
        set_error("unknown sus_partials");
        return GFBP_EINVAL;
    }
    return GFBP_OK;
}

// Point A into the workspace; the Markov constants are copied on `stream`.
cudaError_t place_args(DecodeArgs& A, const Layout& l, void* ws, const Common& C, bool step, const float* prior_in,
                       cudaStream_t stream) {
    uint8_t* base = static_cast<uint8_t*>(ws);
    const CodeDev& c = A.c;
    A.work = reinterpret_cast<int*>(base + l.work);
    A.L = reinterpret_cast<float*>(base + l.L);
    A.msg = reinterpret_cast<float*>(base + l.msg);
    cudaError_t e = cudaSuccess;
    if (C.markov) {
        A.Qsrc = reinterpret_cast<float*>(base + l.Qsrc);
        A.P = step ? const_cast<float*>(prior_in) : reinterpret_cast<float*>(base + l.P);
        float* Mt = reinterpret_cast<float*>(base + l.Mt);
        float* pi = reinterpret_cast<float*>(base + l.pi);
        int* sidx = reinterpret_cast<int*>(base + l.src_index);
        int* spos = reinterpret_cast<int*>(base + l.src_pos);
        A.Mt = Mt;
        A.pi = pi;
        A.src_index = sidx;
        A.src_pos = spos;
        const size_t q = (size_t)c.q;
        e = cudaMemcpyAsync(Mt, C.Mt.data(), sizeof(float) * q * q, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pi, C.pi.data(), sizeof(float) * q, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sidx, C.src_index.data(), sizeof(int) * c.N, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(spos, C.src_pos.data(), sizeof(int) * C.K, cudaMemcpyHostToDevice, stream);
    }
    return e;
}

gfbp_status run(const gfbp_code* code, int32_t F, const float* obs, gfbp_channel ch, gfbp_schedule schedule,
                const Common& C, int32_t max_iter, bool step, uint8_t* x_hat, int32_t* iters, uint8_t* conv,
                float* msg_io, const float* prior_in, float* prior_out, const gfbp_options* opt, void* stream_v) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const CodeDev& c = code->dev;
    const Layout l = layout(c, F, C.markov, C.K, step);
    DecodeArgs A;
    gfbp_status st = fill_args(A, code, F, obs, ch, C, max_iter, step, x_hat, iters, conv, msg_io, prior_out, opt);
    if (st != GFBP_OK) return st;
    if (A.method == kTensor && schedule != GFBP_SUS) {
        set_error("check_method TENSOR is implemented for SUS only");
        return GFBP_EUNSUPPORTED;
    }
    if (C.gs && (schedule != GFBP_SUS || step || (A.method == kDirect && c.q > 16) || A.method == kTensor ||
                 c.dcmax > 16 || c.dvmax > 8)) {
        set_error("prior MARKOV_GS needs SUS with gfbp_decode and, for q >= 32, check_method TRANSFORM");
        return GFBP_EUNSUPPORTED;
    }
    const bool resident = schedule == GFBP_PUS ? pus_res_eligible(A) : (sus_res_eligible(A, device_sms()) || sus_l2_eligible(A));
    if ((A.layout == GFBP_LAYOUT_RESIDENT || A.layout == GFBP_LAYOUT_L2RESIDENT) && !resident) {
        set_error("layouts RESIDENT and L2RESIDENT need the DIRECT check node (q <= 16); RESIDENT a frame whose "
                  "messages fit in one CTA's shared memory and, for PUS, row degree <= 6 and column degree <= 4; "
                  "L2RESIDENT is SUS only; both SUS layouts need AUTO or RUNNING partials and the Jacobi prior");
        return GFBP_EUNSUPPORTED;
    }

    void* ws = opt ? opt->workspace : nullptr;
    bool own = false;
    cudaError_t e = cudaSuccess;
    if (ws) {
        if (opt->workspace_bytes < l.total || (reinterpret_cast<uintptr_t>(ws) & 255)) {
            set_error("workspace too small or not 256-byte aligned");
            return GFBP_EINVAL;
        }
    } else {
        e = cudaMallocAsync(&ws, l.total, stream);
        if (e != cudaSuccess) return cuda_fail("workspace allocation", e);
        own = true;
    }
    if (e == cudaSuccess) e = place_args(A, l, ws, C, step, prior_in, stream);
    // running partials kept in global memory: a second edge slab of this call's own
    void* sfx = nullptr;
    if (e == cudaSuccess && schedule == GFBP_SUS && A.partials == GFBP_PARTIALS_RUNNING_GLOBAL &&
        A.method == kDirect && A.layout != GFBP_LAYOUT_LANES) {
        e = cudaMallocAsync(&sfx, sizeof(float) * (size_t)F * (size_t)c.E * c.q, stream);
        if (e != cudaSuccess) {
            if (own) cudaFreeAsync(ws, stream);
            return cuda_fail("partials allocation", e);
        }
        A.sfx = static_cast<float*>(sfx);
    }
    if (C.markov) {
        const size_t q = (size_t)c.q;
        if (!step) {
            // initial block priors: the stationary distribution (reading of Sec. 2)
            std::vector<float> P0((size_t)F * C.K * q);
            for (size_t k = 0; k < P0.size(); k++) P0[k] = C.pi[k % q];
            if (e == cudaSuccess && !P0.empty())
                e = cudaMemcpyAsync(A.P, P0.data(), sizeof(float) * P0.size(), cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // P0 is pageable and local
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(A.work, 0, sizeof(int), stream);
    if (e == cudaSuccess && A.zsum) e = cudaMemsetAsync(A.zsum, 0, sizeof(int) * (size_t)F, stream);
    if (e == cudaSuccess) e = launch_channel(A, stream);
    // (the resident kernels initialise their messages in shared memory)
    if (e == cudaSuccess && schedule == GFBP_SUS && !resident) e = launch_init_dev(A, stream);
    cudaEvent_t ev0 = opt ? static_cast<cudaEvent_t>(opt->kernel_events[0]) : nullptr;
    cudaEvent_t ev1 = opt ? static_cast<cudaEvent_t>(opt->kernel_events[1]) : nullptr;
    if (e == cudaSuccess && ev0) e = cudaEventRecord(ev0, stream);
    if (e == cudaSuccess) e = (schedule == GFBP_PUS) ? launch_pus(A, device_sms(), stream) : launch_sus(A, device_sms(), stream);
    if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, stream);
    if (sfx) {
        cudaError_t e2 = cudaFreeAsync(sfx, stream);
        if (e == cudaSuccess) e = e2;
    }
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail("decode launch", e);
    return GFBP_OK;
}

__global__ void k_fill_prior(float* P, const float* pi, long long n, int q) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        P[i] = pi[i % q];
}

}  // namespace

// Initial block priors (the stationary distribution) of every frame, on the device.
cudaError_t launch_fill_prior(const DecodeArgs& A, cudaStream_t s) {
    const long long n = (long long)A.F * A.K * A.c.q;
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    k_fill_prior<<<(unsigned)blocks, 256, 0, s>>>(A.P, A.pi, n, A.c.q);
    return cudaGetLastError();
}

// A batch item's DecodeArgs placed in its workspace (Markov constants copied
// synchronously); the batch's runs launch only.
cudaError_t batch_prepare_item(DecodeArgs& A, void* ws, const gfbp_code* code, int32_t F, const float* obs,
                               gfbp_channel ch, gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter,
                               uint8_t* x_hat, int32_t* iters, uint8_t* conv, const gfbp_options* opt, int method,
                               size_t* ws_bytes, cudaStream_t stream) {
    Common C;
    if (check_common("gfbp_batch_create", code, F, obs, ch, schedule, prior, C) != GFBP_OK) return cudaErrorInvalidValue;
    if (C.gs) {
        set_error("gfbp_batch_create: prior MARKOV_GS is decoded by gfbp_decode only");
        return cudaErrorInvalidValue;
    }
    if (fill_args(A, code, F, obs, ch, C, max_iter, false, x_hat, iters, conv, nullptr, nullptr, opt) != GFBP_OK)
        return cudaErrorInvalidValue;
    A.method = method;
    const Layout l = layout(code->dev, F, C.markov, C.K, false);
    if (ws_bytes) *ws_bytes = l.total;
    cudaError_t e = place_args(A, l, ws, C, false, nullptr, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) set_error(std::string("gfbp_batch_create: ") + cudaGetErrorString(e));
    return e;
}

}  // namespace gfbp

using namespace gfbp;

extern "C" const char* gfbp_last_error(void) { return g_last_error.c_str(); }

extern "C" gfbp_status gfbp_workspace_size(const gfbp_code* code, int32_t n_frames, gfbp_schedule schedule,
                                           const gfbp_prior* prior, int32_t step, size_t* bytes) {
    if (!code || !bytes || n_frames < 0) { set_error("gfbp_workspace_size: bad argument"); return GFBP_EINVAL; }
    if (schedule != GFBP_PUS && schedule != GFBP_SUS) { set_error("gfbp_workspace_size: unknown schedule"); return GFBP_EINVAL; }
    const bool markov = prior && (prior->kind == GFBP_PRIOR_MARKOV || prior->kind == GFBP_PRIOR_MARKOV_GS);
    *bytes = layout(code->dev, n_frames, markov, markov ? prior->K : 0, step != 0).total;
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_decode(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                                   gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter, uint8_t* x_hat,
                                   int32_t* iters, uint8_t* converged, const gfbp_options* options, void* stream) {
    Common C;
    gfbp_status st = check_common("gfbp_decode", code, n_frames, obs, channel, schedule, prior, C);
    if (st != GFBP_OK) return st;
    if (max_iter < 1) { set_error("gfbp_decode: max_iter must be >= 1"); return GFBP_EINVAL; }
    if (n_frames > 0 && (!x_hat || !iters || !converged)) { set_error("gfbp_decode: NULL output"); return GFBP_EINVAL; }
    if (n_frames == 0) return GFBP_OK;
    return run(code, n_frames, obs, channel, schedule, C, max_iter, false, x_hat, iters, converged, nullptr,
               nullptr, nullptr, options, stream);
}

extern "C" gfbp_status gfbp_step(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                                 gfbp_schedule schedule, const gfbp_prior* prior, float* msg, const float* prior_in,
                                 float* prior_out, float* post, uint8_t* x_hat, uint8_t* sat,
                                 const gfbp_options* options, void* stream) {
    Common C;
    gfbp_status st = check_common("gfbp_step", code, n_frames, obs, channel, schedule, prior, C);
    if (st != GFBP_OK) return st;
    if (n_frames > 0 && (!msg || !post || !x_hat || !sat)) { set_error("gfbp_step: NULL msg/post/x_hat/sat"); return GFBP_EINVAL; }
    if (C.markov && n_frames > 0 && !prior_in) { set_error("gfbp_step: Markov prior needs prior_in"); return GFBP_EINVAL; }
    if (n_frames == 0) return GFBP_OK;
    gfbp_options o{};
    if (options) o = *options;
    o.post = post;
    o.xhat_trace = nullptr;
    o.no_early_stop = 0;
    return run(code, n_frames, obs, channel, schedule, C, 1, true, x_hat, nullptr, sat, msg, prior_in,
               C.markov ? prior_out : nullptr, &o, stream);
}
