// gfbp_wht: the Walsh-Hadamard transform of a batch of q-vectors, by FP32
// butterflies on the CUDA cores (lane groups, as inside the transform route
// of the decoder) or by the FP16 hi/lo tensor-core contraction of wht_tc.cuh.
#include <string>

#include "gfbp_internal.cuh"
#include "wht_tc.cuh"

namespace gfbp {
void set_error(const std::string& msg);

namespace {

int sm_count() { return device_sms(); }

template <int Q>
__global__ void __launch_bounds__(256) k_wht_simt(const float* __restrict__ x, float* __restrict__ y, long long n) {
    constexpr int V = Lay<Q>::V, G = Lay<Q>::G;
    const int g = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const long long per_block = blockDim.x / G;
    for (long long v = (long long)blockIdx.x * per_block + threadIdx.x / G; v < n; v += (long long)gridDim.x * per_block) {
        float a[V];
        ldv<V>(a, x + (size_t)v * Q + g * V);
        wht<Q>(a, mask, g);
        stv<V>(y + (size_t)v * Q + g * V, a);
    }
}

// The streaming tensor-core transform: a warp task is 16 chunks of 16 entries
// (16 / B vectors, B = q / 16 chunks each); MMA row m of a task is chunk m % B
// of vector task * 16 / B + m / B.  Every lane reads its eight entries of the
// A fragments straight from global memory (rows g and g + 8, columns 2t, 2t+1,
// 2t+8, 2t+9 of the chunk: 32 contiguous bytes per chunk and instruction
// across the four lanes of a row), splits them into FP16 parts in registers
// and writes its outputs at the same positions; the next task's entries are
// loaded before the current one is transformed.
template <int Q>
__device__ __forceinline__ void tc_load(const float* __restrict__ x, long long n, long long task, float (&v)[8]) {
    constexpr int B = Q / 16, RT = 16 / B;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long ra = task * RT + g / B, rb = task * RT + (g + 8) / B;
    const int ia = g % B, ib = (g + 8) % B;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
    if (ra < n) {
        const float2* p = reinterpret_cast<const float2*>(x + (size_t)ra * Q + ia * 16 + 2 * t);
        a0 = __ldcs(p);
        a1 = __ldcs(p + 4);
    }
    if (rb < n) {
        const float2* p = reinterpret_cast<const float2*>(x + (size_t)rb * Q + ib * 16 + 2 * t);
        b0 = __ldcs(p);
        b1 = __ldcs(p + 4);
    }
    v[0] = a0.x; v[1] = a0.y; v[2] = a1.x; v[3] = a1.y;
    v[4] = b0.x; v[5] = b0.y; v[6] = b1.x; v[7] = b1.y;
}

__device__ __forceinline__ uint32_t pack_half2(__half lo_index, __half hi_index) {
    return (uint32_t)__half_as_ushort(lo_index) | ((uint32_t)__half_as_ushort(hi_index) << 16);
}

template <int Q>
__device__ __forceinline__ void tc_transform_store(float* __restrict__ y, long long n, long long task, const float (&v)[8]) {
    constexpr int B = Q / 16, RT = 16 / B;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // largest magnitude of the vector of each of the two rows, over the lanes
    // that hold its chunks (t bits and the g bits below log2 B)
    float ma = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
    float mb = fmaxf(fmaxf(fabsf(v[4]), fabsf(v[5])), fmaxf(fabsf(v[6]), fabsf(v[7])));
    if constexpr (B == 16) ma = mb = fmaxf(ma, mb);   // rows g and g + 8: one vector
#pragma unroll
    for (int m = 1; m <= 2; m <<= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, m));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, m));
    }
#pragma unroll
    for (int bit = 0; bit < 3; bit++) {
        if ((1 << bit) < B) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, 4 << bit));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, 4 << bit));
        }
    }
    const float sa = pow2_scale(ma), sb = pow2_scale(mb);
    __half h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; i++) split_hilo(v[i] * (i < 4 ? sa : sb), h[i], l[i]);
    const uint32_t ah[4] = {pack_half2(h[0], h[1]), pack_half2(h[4], h[5]), pack_half2(h[2], h[3]),
                            pack_half2(h[6], h[7])};
    const uint32_t al[4] = {pack_half2(l[0], l[1]), pack_half2(l[4], l[5]), pack_half2(l[2], l[3]),
                            pack_half2(l[6], l[7])};
    float acc[2][4];
    tc_wht_frag<Q>(ah, al, acc);
    const long long ra = task * RT + g / B, rb = task * RT + (g + 8) / B;
    const int ia = g % B, ib = (g + 8) % B;
    const float ua = 1.0f / sa, ub = 1.0f / sb;   // powers of two: exact
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const int c = nt * 8 + 2 * t;
        if (ra < n) __stcs(reinterpret_cast<float2*>(y + (size_t)ra * Q + ia * 16 + c),
                           make_float2(acc[nt][0] * ua, acc[nt][1] * ua));
        if (rb < n) __stcs(reinterpret_cast<float2*>(y + (size_t)rb * Q + ib * 16 + c),
                           make_float2(acc[nt][2] * ub, acc[nt][3] * ub));
    }
}

template <int Q>
__global__ void __launch_bounds__(256) k_wht_tc(const float* __restrict__ x, float* __restrict__ y, long long n) {
    constexpr int RT = 16 / (Q / 16);
    const long long tasks = (n + RT - 1) / RT;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);   // warp-uniform
    if (task >= tasks) return;
    float cur[8];
    tc_load<Q>(x, n, task, cur);
    for (; task < tasks; task += nw) {
        const bool more = task + nw < tasks;
        float nxt[8];
        if (more) tc_load<Q>(x, n, task + nw, nxt);
        tc_transform_store<Q>(y, n, task, cur);
        if (more) {
#pragma unroll
            for (int i = 0; i < 8; i++) cur[i] = nxt[i];
        }
    }
}

template <int Q>
cudaError_t launch_wht(const float* x, float* y, long long n, int method, cudaStream_t s) {
    if (method == GFBP_WHT_SIMT) {
        constexpr int per_block = 256 / Lay<Q>::G;
        long long blocks = (n + per_block - 1) / per_block;
        const long long cap = (long long)sm_count() * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) return cudaSuccess;
        k_wht_simt<Q><<<(int)blocks, 256, 0, s>>>(x, y, n);
        return cudaGetLastError();
    }
    if constexpr (Q >= 16) {
        int occ = 0;
        cudaError_t e = kernel_prepare((const void*)k_wht_tc<Q>, 256, 0, &occ);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        constexpr int RT = 16 / (Q / 16);
        const long long tasks = (n + RT - 1) / RT;
        long long blocks = (tasks + 7) / 8;
        const long long cap = (long long)sm_count() * occ;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) return cudaSuccess;
        k_wht_tc<Q><<<(int)blocks, 256, 0, s>>>(x, y, n);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace gfbp

using namespace gfbp;

extern "C" gfbp_status gfbp_wht(const float* x, float* y, int64_t n, int32_t q, int32_t method, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) { set_error("gfbp_wht: need n >= 0 and device x, y"); return GFBP_EINVAL; }
    if (method != GFBP_WHT_SIMT && method != GFBP_WHT_TENSOR) { set_error("gfbp_wht: unknown method"); return GFBP_EINVAL; }
    if (method == GFBP_WHT_TENSOR && (q < 16 || q > 256 || (q & (q - 1)))) {
        set_error("gfbp_wht: the tensor-core form needs q in {16, 32, 64, 128, 256}");
        return GFBP_EUNSUPPORTED;
    }
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) {
        set_error("gfbp_wht: x and y must be 16-byte aligned");
        return GFBP_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (q) {
    case 2: e = launch_wht<2>(x, y, n, method, s); break;
    case 4: e = launch_wht<4>(x, y, n, method, s); break;
    case 8: e = launch_wht<8>(x, y, n, method, s); break;
    case 16: e = launch_wht<16>(x, y, n, method, s); break;
    case 32: e = launch_wht<32>(x, y, n, method, s); break;
    case 64: e = launch_wht<64>(x, y, n, method, s); break;
    case 128: e = launch_wht<128>(x, y, n, method, s); break;
    case 256: e = launch_wht<256>(x, y, n, method, s); break;
    default: set_error("gfbp_wht: q must be 2^p with 1 <= p <= 8"); return GFBP_EINVAL;
    }
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_wht: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    return GFBP_OK;
}
