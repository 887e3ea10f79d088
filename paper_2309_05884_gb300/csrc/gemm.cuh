// CTA-level complex GEMM on small square matrices, used by the batched matrix exponential.
//
// C = A * B + sum_{l=0}^{nterm-1} coef[l] * P_l, with P_0 = I and P_l (l >= 1) = pw[l] (m x m),
// every matrix m x m, row-major, complex, in global (L2-resident) or shared memory.  256 threads
// own a (16R) x (16R) output tile, each thread an R x R register micro-tile at rows ty+16i and
// columns tx+16j; K is staged through shared memory 16 columns at a time.  The caller must not
// alias C with A, B or any pw[l].
#pragma once

#include "common.cuh"

namespace qoc {

constexpr int GEMM_THREADS = 256;
constexpr int GEMM_TK = 16;

template <class T, int R>
struct GemmSmem {
    cx<T> As[GEMM_TK][16 * R + 1];
    cx<T> Bs[GEMM_TK][16 * R];
};

template <class T, int R>
__device__ void cta_gemm(cx<T>* __restrict__ C, const cx<T>* __restrict__ A, const cx<T>* __restrict__ B,
                         int m, int nterm, const T* coef, const cx<T>* const* pw, GemmSmem<T, R>& sm) {
    constexpr int TM = 16 * R;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    for (int ti = 0; ti < m; ti += TM) {
        for (int tj = 0; tj < m; tj += TM) {
            cx<T> acc[R][R];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = mk<T>(0, 0);
            for (int k0 = 0; k0 < m; k0 += GEMM_TK) {
                // A tile: TM rows x 16 cols, stored transposed As[kk][ii]
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = tid + GEMM_THREADS * r;
                    const int ii = e >> 4, kk = e & 15;
                    const int gi = ti + ii, gk = k0 + kk;
                    sm.As[kk][ii] = (gi < m && gk < m) ? A[(size_t)gi * m + gk] : mk<T>(0, 0);
                }
                // B tile: 16 rows x TM cols
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = tid + GEMM_THREADS * r;
                    const int kk = e / TM, jj = e - kk * TM;
                    const int gk = k0 + kk, gj = tj + jj;
                    sm.Bs[kk][jj] = (gk < m && gj < m) ? B[(size_t)gk * m + gj] : mk<T>(0, 0);
                }
                __syncthreads();
#pragma unroll 4
                for (int kk = 0; kk < GEMM_TK; ++kk) {
                    cx<T> a[R], b[R];
#pragma unroll
                    for (int i = 0; i < R; ++i) a[i] = sm.As[kk][ty + 16 * i];
#pragma unroll
                    for (int j = 0; j < R; ++j) b[j] = sm.Bs[kk][tx + 16 * j];
#pragma unroll
                    for (int i = 0; i < R; ++i)
#pragma unroll
                        for (int j = 0; j < R; ++j) cfma<T>(acc[i][j], a[i], b[j]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int gi = ti + ty + 16 * i;
                if (gi >= m) continue;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const int gj = tj + tx + 16 * j;
                    if (gj >= m) continue;
                    cx<T> v = acc[i][j];
                    const size_t o = (size_t)gi * m + gj;
                    if (nterm > 0 && gi == gj) v.x += coef[0];
                    for (int l = 1; l < nterm; ++l) {
                        const cx<T> p = pw[l][o];
                        v.x = fma(coef[l], p.x, v.x);
                        v.y = fma(coef[l], p.y, v.y);
                    }
                    C[o] = v;
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace qoc
