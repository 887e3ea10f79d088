// Complex matrix products on the 5th-generation tensor cores, at about FP32 accuracy.
//
// C = A B for complex m x m matrices (m <= 112) given in FP32.  Each real part is split into two
// FP16 numbers, x = hi + lo with hi = fp16(x) and lo = fp16(x - hi), and a real product is the sum
// of all four split products lo*lo, hi*lo, lo*hi, hi*hi, accumulated in FP32 in tensor memory in
// that order (small terms first: each addition rounds relative to the running sum).  The complex
// product is four real products into two accumulators: C_r = A_r B_r - A_i B_i (the minus from the
// instruction's negate-A bit), C_i = A_r B_i + A_i B_r.  One CTA of 128 threads owns a product: it
// stages both operands in shared memory in the K-major no-swizzle canonical layout (8 x 16-byte
// core matrices), one thread issues the tcgen05 MMAs (M = 128, N = m rounded up to 16, K = 16 per
// instruction), the commit arrives on an mbarrier, and the four warps read the accumulators back
// row by row (warp w holds rows 32w..).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace qoc {

constexpr int TC_THREADS = 128;
constexpr int TC_MAXM = 112;
constexpr uint32_t TC_TMEM_COLS = 256;  // C_r at column 0, C_i at column 128

// byte offsets of the operand buffers in dynamic shared memory, for padded sizes MP (rows of A,
// 128), NP (rows of B^T) and KP (the K extent): A_r hi/lo, A_i hi/lo (MP x KP), B_r hi/lo, B_i hi/lo
// (NP x KP) as FP16, then the mbarrier and the TMEM address word.
struct TcLayout {
    int NP, KP;
    __host__ __device__ size_t a_bytes() const { return (size_t)128 * KP * 2; }
    __host__ __device__ size_t b_bytes() const { return (size_t)NP * KP * 2; }
    __host__ __device__ size_t a_off(int i) const { return (size_t)i * a_bytes(); }
    __host__ __device__ size_t b_off(int i) const { return 4 * a_bytes() + (size_t)i * b_bytes(); }
    __host__ __device__ size_t bar_off() const { return (4 * a_bytes() + 4 * b_bytes() + 15) / 16 * 16; }
    __host__ __device__ size_t total() const { return bar_off() + 16; }
};

__host__ __device__ inline int tc_pad16(int m) { return (m + 15) / 16 * 16; }

// element (row, k) of a K-major no-swizzle tile with KP columns, in FP16 elements
__device__ __forceinline__ int tc_off(int row, int k, int KP) {
    return (((row >> 3) * (KP >> 3) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

__device__ __forceinline__ void split16(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// Stage A (as the M x K operand) from a complex FP32 m x m row-major matrix; rows >= m and k >= m are 0.
__device__ __forceinline__ void tc_stage_a(unsigned char* sm, const TcLayout& L, const float2* A, int m) {
    __half* Arh = reinterpret_cast<__half*>(sm + L.a_off(0));
    __half* Arl = reinterpret_cast<__half*>(sm + L.a_off(1));
    __half* Aih = reinterpret_cast<__half*>(sm + L.a_off(2));
    __half* Ail = reinterpret_cast<__half*>(sm + L.a_off(3));
    const int KP = L.KP;
    for (int e = threadIdx.x; e < 128 * KP; e += blockDim.x) {
        const int row = e / KP, k = e - row * KP;
        const float2 v = (row < m && k < m) ? A[(size_t)row * m + k] : make_float2(0.f, 0.f);
        const int o = tc_off(row, k, KP);
        split16(v.x, Arh[o], Arl[o]);
        split16(v.y, Aih[o], Ail[o]);
    }
}

// Stage B (as the N x K operand B^T, element (n, k) = B[k][n]); n >= m and k >= m are 0.
__device__ __forceinline__ void tc_stage_b(unsigned char* sm, const TcLayout& L, const float2* B, int m) {
    __half* Brh = reinterpret_cast<__half*>(sm + L.b_off(0));
    __half* Brl = reinterpret_cast<__half*>(sm + L.b_off(1));
    __half* Bih = reinterpret_cast<__half*>(sm + L.b_off(2));
    __half* Bil = reinterpret_cast<__half*>(sm + L.b_off(3));
    const int KP = L.KP, NP = L.NP;
    for (int e = threadIdx.x; e < KP * NP; e += blockDim.x) {
        const int k = e / NP, n = e - k * NP;
        const float2 v = (k < m && n < m) ? B[(size_t)k * m + n] : make_float2(0.f, 0.f);
        const int o = tc_off(n, k, KP);
        split16(v.x, Brh[o], Brl[o]);
        split16(v.y, Bih[o], Bil[o]);
    }
}

// One thread: issue every MMA of the product and commit it to bar.
__device__ __forceinline__ void tc_issue(unsigned char* sm, const TcLayout& L, uint32_t tmem, uint64_t* bar) {
    const uint32_t lbo = 128, sbo = (uint32_t)(L.KP / 8) * 128;
    const uint32_t id_pos = idesc_f16(128, L.NP, false), id_neg = idesc_f16(128, L.NP, true);
    const uint32_t Cr = tmem, Ci = tmem + 128;
    // (lo,lo), (hi,lo), (lo,hi) first and (hi,hi) last: the small terms are summed while the
    // accumulator is small, so only the K/16 large additions round against a large running sum
    const int hiA[4] = {1, 0, 1, 0}, hiB[4] = {1, 1, 0, 0};
    for (int t = 0; t < 4; ++t) {
        for (int kk = 0; kk < L.KP / 16; ++kk) {
            const size_t step = (size_t)kk * 256;  // two cores along K
            const int first = (kk == 0 && t == 0);
            const uint64_t ar = smem_desc(sm + L.a_off(hiA[t]) + step, lbo, sbo);
            const uint64_t ai = smem_desc(sm + L.a_off(2 + hiA[t]) + step, lbo, sbo);
            const uint64_t br = smem_desc(sm + L.b_off(hiB[t]) + step, lbo, sbo);
            const uint64_t bi = smem_desc(sm + L.b_off(2 + hiB[t]) + step, lbo, sbo);
            mma_f16(Cr, ar, br, id_pos, first ? 0 : 1);
            mma_f16(Cr, ai, bi, id_neg, 1);
            mma_f16(Ci, ar, bi, id_pos, first ? 0 : 1);
            mma_f16(Ci, ai, br, id_pos, 1);
        }
    }
    mma_commit(bar);
}

}  // namespace qoc
