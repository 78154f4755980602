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

constexpr int kTcRows = 64;   // rows staged per block step

template <int Q>
constexpr size_t tc_smem() {
    return sizeof(__half) * 2 * (size_t)kTcRows * tc_stride<Q>() + sizeof(float) * kTcRows;
}

// One warp stages a row: its largest magnitude, the power-of-two scale, the
// FP16 parts of the scaled entries; rs[r] receives the inverse scale.
template <int Q>
__device__ __forceinline__ void stage_row(const float* src, bool valid, __half* hi, __half* lo, float* rs, int lane) {
    constexpr int PER = (Q + 127) / 128;   // float4 chunks per lane
    float4 v[PER];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int k = (i * 32 + lane) * 4;
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid && k < Q) v[i] = *reinterpret_cast<const float4*>(src + k);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v[i].x), fabsf(v[i].y)), fmaxf(fabsf(v[i].z), fabsf(v[i].w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float s = pow2_scale(m);
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int k = (i * 32 + lane) * 4;
        if (k < Q) {
            __half h[4], l[4];
            split_hilo(v[i].x * s, h[0], l[0]);
            split_hilo(v[i].y * s, h[1], l[1]);
            split_hilo(v[i].z * s, h[2], l[2]);
            split_hilo(v[i].w * s, h[3], l[3]);
            *reinterpret_cast<uint2*>(hi + k) = *reinterpret_cast<const uint2*>(h);
            *reinterpret_cast<uint2*>(lo + k) = *reinterpret_cast<const uint2*>(l);
        }
    }
    if (lane == 0) *rs = 1.0f / s;
}

template <int Q>
__global__ void __launch_bounds__(256) k_wht_tc(const float* x, float* y, long long n) {
    constexpr int S = tc_stride<Q>();
    extern __shared__ __align__(16) __half s_stage[];
    __half* hi = s_stage;
    __half* lo = s_stage + (size_t)kTcRows * S;
    float* rs = reinterpret_cast<float*>(s_stage + (size_t)2 * kTcRows * S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (long long base = (long long)blockIdx.x * kTcRows; base < n; base += (long long)gridDim.x * kTcRows) {
        const int nrows = (int)((n - base) < kTcRows ? (n - base) : kTcRows);
        for (int r = warp; r < kTcRows; r += nw)
            stage_row<Q>(x + (size_t)(base + r) * Q, r < nrows, hi + (size_t)r * S, lo + (size_t)r * S, rs + r, lane);
        __syncthreads();
        tc_wht_rows<Q>(hi, lo, rs, nrows, y + (size_t)base * Q, Q, 1.0f, warp, nw);
        __syncthreads();
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
        constexpr size_t smem = tc_smem<Q>();
        int occ = 0;
        cudaError_t e = kernel_prepare((const void*)k_wht_tc<Q>, 256, smem, &occ);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        long long blocks = (n + kTcRows - 1) / kTcRows;
        const long long cap = (long long)sm_count() * occ;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) return cudaSuccess;
        k_wht_tc<Q><<<(int)blocks, 256, smem, s>>>(x, y, n);
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
