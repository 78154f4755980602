// Walsh-Hadamard transform of q-vectors (the convolution theorem of the
// additive group of GF(2^p), used by the transform route of Eq. 3) as a dense
// contraction with the +-1 Hadamard matrix on the tensor cores:
//   Y = X H,   H[k][n] = (-1)^popcount(k AND n),
// each FP32 operand split into an FP16 high part and an FP16 low part
// (x = hi + lo to about 22 bits), both multiplied by H with FP32 accumulation
// (Y = hi H + lo H).  H is exact in FP16 and is not stored: every lane builds
// its B fragments from the indices.  Warp-level mma.sync.m16n8k16 tiles:
// a warp task is 16 rows x 64 columns (eight 16x8 tiles) over the whole K = q.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace gfbp {

namespace {

// H[k][n] and H[k+1][n] as two FP16 values (the lower index in the low half).
__device__ __forceinline__ uint32_t had2(int k, int n) {
    const uint32_t pos = 0x3C00u, neg = 0xBC00u;   // +1.0, -1.0
    const uint32_t a = (__popc(k & n) & 1) ? neg : pos;
    const uint32_t b = (__popc((k + 1) & n) & 1) ? neg : pos;
    return a | (b << 16);
}

__device__ __forceinline__ uint32_t lds32(const __half* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D += A B for one 16x8x16 tile (A row-major FP16, B column-major FP16, D FP32).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// x = hi + lo with both parts in FP16 (|x| < 65504).
__device__ __forceinline__ void split_hilo(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// Power of two that brings a vector's largest magnitude m into [1, 2) (1 for
// m = 0 or not finite): applied before the split (exactly) and undone on the
// output, it keeps small vectors out of FP16's subnormal range.
__device__ __forceinline__ float pow2_scale(float m) {
    if (!(m > 0.f) || !(m <= 3.0e38f)) return 1.0f;
    return ldexpf(1.0f, -ilogbf(m));
}

// Row stride (halves) of a staged operand: q + 8 keeps the fragment loads of
// the eight rows of a tile on distinct banks.
template <int Q>
constexpr int tc_stride() { return Q + 8; }

// out[r][c] = scale * rs[r] * sum_k (hi[r][k] + lo[r][k]) H[k][c] for rows
// r0..r0+15 (those below nrows are written) and columns c0..c0+8*NT-1, by one
// warp.  hi / lo: staged rows of tc_stride<Q>() halves, at least r0 + 16 rows;
// rs: per-row factors (the inverse of the staging scale), or NULL.
template <int Q, int NT>
__device__ __forceinline__ void tc_wht_task(const __half* hi, const __half* lo, const float* rs, int r0, int c0,
                                            float* out, int out_stride, int nrows, float scale) {
    constexpr int S = tc_stride<Q>();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll 4
    for (int k0 = 0; k0 < Q; k0 += 16) {
        const __half* ph = hi + (size_t)(r0 + g) * S + k0 + 2 * t;
        const __half* pl = lo + (size_t)(r0 + g) * S + k0 + 2 * t;
        const uint32_t ah[4] = {lds32(ph), lds32(ph + 8 * S), lds32(ph + 8), lds32(ph + 8 * S + 8)};
        const uint32_t al[4] = {lds32(pl), lds32(pl + 8 * S), lds32(pl + 8), lds32(pl + 8 * S + 8)};
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const int n = c0 + nt * 8 + g;
            const uint32_t b0 = had2(k0 + 2 * t, n), b1 = had2(k0 + 2 * t + 8, n);
            mma16816(acc[nt], ah, b0, b1);
            mma16816(acc[nt], al, b0, b1);
        }
    }
    const int ra = r0 + g, rb = r0 + g + 8;
    const float sa = (rs && ra < nrows) ? scale * rs[ra] : scale;
    const float sb = (rs && rb < nrows) ? scale * rs[rb] : scale;
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int c = c0 + nt * 8 + 2 * t;
        if (ra < nrows) *reinterpret_cast<float2*>(out + (size_t)ra * out_stride + c) =
            make_float2(acc[nt][0] * sa, acc[nt][1] * sa);
        if (rb < nrows) *reinterpret_cast<float2*>(out + (size_t)rb * out_stride + c) =
            make_float2(acc[nt][2] * sb, acc[nt][3] * sb);
    }
}

// All rows 0..nrows-1 of a staged block by the CTA's warps (tasks of 16 rows x
// 64 columns; q >= 16).
template <int Q>
__device__ __forceinline__ void tc_wht_rows(const __half* hi, const __half* lo, const float* rs, int nrows, float* out,
                                            int out_stride, float scale, int warp, int nwarps) {
    constexpr int NT = (Q / 8) < 8 ? (Q / 8) : 8;
    constexpr int CB = Q / (8 * NT);   // column blocks
    const int rblocks = (nrows + 15) / 16;
    for (int task = warp; task < rblocks * CB; task += nwarps) {
        const int rb = task / CB, cb = task % CB;
        tc_wht_task<Q, NT>(hi, lo, rs, rb * 16, cb * 8 * NT, out, out_stride, nrows, scale);
    }
}

}  // namespace
}  // namespace gfbp
