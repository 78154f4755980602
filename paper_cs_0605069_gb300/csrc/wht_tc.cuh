// Walsh-Hadamard transform of q-vectors (the convolution theorem of the
// additive group of GF(2^p), used by the transform route of Eq. 3) with the
// +-1 Hadamard matrix on the tensor cores, factored as a Kronecker product:
// with q = 16 B and index a = 16 i + l,
//   H_q = H_B (x) H_16,   Y[i'][l'] = sum_i H_B[i'][i] sum_l x[i][l] H_16[l][l'],
// so each 16-entry chunk of a vector is contracted with H_16 on the tensor
// cores (Z = X H_16, K = 16: q 16 multiply-adds per vector per part instead of
// q^2 for the dense H_q), and the B-point transforms across chunks run as FP32
// butterflies on the contraction's accumulators (lane shuffles).  Each FP32
// operand is split into an FP16 high part and an FP16 low part (x = hi + lo
// to about 22 bits), both multiplied by H_16 (exact in FP16, built from index
// parity in registers) with FP32 accumulation.  Warp-level mma.sync.m16n8k16:
// a warp task is 16 chunks (16/B vectors) x 16 columns.
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

// The transform of one warp task from its A fragments (the FP16 high and low
// parts of the 16 chunks x 16 entries, in the m16n8k16 row-major layout:
// a[0] row g cols 2t..2t+1, a[1] row g+8, a[2] row g cols 2t+8.., a[3] row
// g+8 cols 2t+8..).  MMA row m is chunk i = m mod B of vector m / B.  The
// chunk transform over l runs on the tensor cores; the transform over i (the
// low log2 B bits of m: row bit 3 inside a thread, bits 0..2 across lane bits
// 2..4) as FP32 butterflies on the accumulators.  acc[nt][0..1]: row g,
// columns nt*8 + 2t, +1; acc[nt][2..3]: row g + 8.
template <int Q>
__device__ __forceinline__ void tc_wht_frag(const uint32_t (&ah)[4], const uint32_t (&al)[4], float (&acc)[2][4]) {
    constexpr int B = Q / 16;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
#pragma unroll
        for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
        const int n = nt * 8 + g;
        const uint32_t b0 = had2(2 * t, n), b1 = had2(2 * t + 8, n);
        mma16816(acc[nt], ah, b0, b1);
        mma16816(acc[nt], al, b0, b1);
    }
    if constexpr (B >= 16) {   // i bit 3: rows g and g + 8 of this thread
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float x0 = acc[nt][c], x1 = acc[nt][2 + c];
                acc[nt][c] = x0 + x1;
                acc[nt][2 + c] = x0 - x1;
            }
    }
#pragma unroll
    for (int bit = 0; bit < 3; bit++) {   // i bits 0..2: g bits, lane bits 2..4
        if ((1 << bit) < B) {
            const int m = 4 << bit;
            const bool up = (lane & m) != 0;
#pragma unroll
            for (int nt = 0; nt < 2; nt++)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float o = __shfl_xor_sync(0xffffffffu, acc[nt][c], m);
                    acc[nt][c] = up ? (o - acc[nt][c]) : (acc[nt][c] + o);
                }
        }
    }
}

// out[r][:] = scale * rs[r] * WHT(hi[r][:] + lo[r][:]) for the 16/B rows of
// task `task` (rows task*16/B ..; those below nrows are written), by one
// warp, from staged FP16 parts (rows of tc_stride<Q>() halves).
template <int Q>
__device__ __forceinline__ void tc_wht_task(const __half* hi, const __half* lo, const float* rs, int task,
                                            float* out, int out_stride, int nrows, float scale) {
    constexpr int S = tc_stride<Q>();
    constexpr int B = Q / 16;            // chunks per vector
    constexpr int RT = 16 / B;           // vectors per task (B <= 16)
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = task * RT;
    // the two MMA rows of this thread: m = g and m = g + 8
    const int ma = g, mb = g + 8;
    const int ra = r0 + ma / B, ia = ma % B, rb = r0 + mb / B, ib = mb % B;
    const __half* pha = hi + (size_t)ra * S + ia * 16 + 2 * t;
    const __half* phb = hi + (size_t)rb * S + ib * 16 + 2 * t;
    const __half* pla = lo + (size_t)ra * S + ia * 16 + 2 * t;
    const __half* plb = lo + (size_t)rb * S + ib * 16 + 2 * t;
    const uint32_t ah[4] = {lds32(pha), lds32(phb), lds32(pha + 8), lds32(phb + 8)};
    const uint32_t al[4] = {lds32(pla), lds32(plb), lds32(pla + 8), lds32(plb + 8)};
    float acc[2][4];
    tc_wht_frag<Q>(ah, al, acc);
    const float sa = (rs && ra < nrows) ? scale * rs[ra] : scale;
    const float sb = (rs && rb < nrows) ? scale * rs[rb] : scale;
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const int c = nt * 8 + 2 * t;
        if (ra < nrows) *reinterpret_cast<float2*>(out + (size_t)ra * out_stride + ia * 16 + c) =
            make_float2(acc[nt][0] * sa, acc[nt][1] * sa);
        if (rb < nrows) *reinterpret_cast<float2*>(out + (size_t)rb * out_stride + ib * 16 + c) =
            make_float2(acc[nt][2] * sb, acc[nt][3] * sb);
    }
}

// All rows 0..nrows-1 of a staged block by the CTA's warps (16 <= q <= 256).
// The staged block must hold whole tasks: rows up to the next multiple of
// 16/B (q / 16 = B), zero-filled beyond nrows.
template <int Q>
__device__ __forceinline__ void tc_wht_rows(const __half* hi, const __half* lo, const float* rs, int nrows, float* out,
                                            int out_stride, float scale, int warp, int nwarps) {
    static_assert(Q >= 16 && Q <= 256, "16 <= q <= 256");
    constexpr int RT = 16 / (Q / 16);
    const int tasks = (nrows + RT - 1) / RT;
    for (int task = warp; task < tasks; task += nwarps)
        tc_wht_task<Q>(hi, lo, rs, task, out, out_stride, nrows, scale);
}

}  // namespace
}  // namespace gfbp
