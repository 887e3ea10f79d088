// Warp-packed matrix exponentials for small blocks (m <= 32; the S_n spin sectors of size n+1).
//
// Same method as expm.cu (Taylor polynomial by Paterson-Stockmeyer after scaling by 2^s, then s
// squarings), laid out for tiny matrices: a warp holds 32/MP matrices (MP = m rounded up to 8, 16 or
// 32), lane l owns row l % MP of matrix l / MP in registers, and the right-hand factors X, X^2, ...
// live in the warp's shared memory, where all lanes of a matrix read the same element at once
// (broadcast).  Products therefore need no block-wide barriers, only __syncwarp over the lanes of
// one matrix; each matrix picks its own degree and squaring count (lane groups of different
// matrices may diverge), so results do not depend on how matrices are packed.  Squarings run in
// the working precision; plans whose squaring chain is FP64 while the polynomial is FP32 use the
// CTA kernel instead.
#include "kernels.h"
#include "../../include/qoc.h"

namespace qoc {
namespace {

// (p, q) of the degrees 2, 4, 6, 9, 12, 16, 20 with p <= 4
__constant__ int c_wp[7] = {2, 2, 3, 3, 4, 4, 4};
__constant__ int c_wq[7] = {1, 2, 2, 3, 3, 4, 5};

template <class T, int MP>
struct WarpSmem {
    cx<T> M[5][MP][MP];  // X^1..X^4, and one product/squaring buffer
};

// row (registers, length MP, entries >= m unused) times matrix Y (shared, MP x MP) -> out row
template <class T, int MP>
__device__ __forceinline__ void row_times(cx<T> (&out)[MP], const cx<T> (&row)[MP], const cx<T> (*Y)[MP], int m) {
#pragma unroll
    for (int j = 0; j < MP; ++j) out[j] = mk<T>(0, 0);
#pragma unroll
    for (int kk = 0; kk < MP; ++kk) {
        if (kk < m) {
            const cx<T> a = row[kk];
#pragma unroll
            for (int j = 0; j < MP; ++j) cfma<T>(out[j], a, Y[kk][j]);
        }
    }
}

template <class T, int MP, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
expm_warp_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks,
                 int n_cls, const int2* __restrict__ cls_items, long long n_cls_items, void* __restrict__ Uout,
                 int per_warp) {
    constexpr int MPW = 32 / MP;  // matrices per warp
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double s_if[24];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto& W = reinterpret_cast<WarpSmem<T, MP>*>(dsm)[warp * MPW + lane / MP];
    const int row = lane % MP;
    if (threadIdx.x < 24) {
        double f = 1.0;
        for (int i = 1; i <= (int)threadIdx.x; ++i) f /= (double)i;
        s_if[threadIdx.x] = f;
    }
    __syncthreads();
    const bool whole = P.nk < 0;
    const long long total = whole ? n_cls_items : (long long)n_cls * P.nk;
    const int mpw = per_warp < MPW ? per_warp : MPW;  // matrices actually packed per warp
    const long long groups = (total + mpw - 1) / mpw;
    const long long gwarp = (long long)blockIdx.x * WARPS + warp;
    const long long nwarps = (long long)gridDim.x * WARPS;

    for (long long g = gwarp; g < groups; g += nwarps) {
        const int slot = lane / MP;
        const long long item = g * mpw + slot;
        const bool valid = slot < mpw && item < total;
        int bi = 0, kw = 0, k = 0;
        if (valid) {
            if (whole) {
                const int2 it = cls_items[item];
                bi = it.x;
                kw = it.y;
                k = it.y;
            } else {
                bi = cls_blocks[item / P.nk];
                kw = (int)(item % P.nk);
                k = P.k0 + kw;
            }
        }
        const DevBlock& B = P.blocks[bi];
        const int m = valid ? B.m : 0;
        const unsigned gmask = MP == 32 ? 0xffffffffu : (((1u << MP) - 1u) << (slot * MP));
        // norm bound, squarings and degree of this lane group's matrix
        double beta = 0.0;
        double uk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) uk[j] = 0.0;
        if (valid) {
            beta = B.h0_norm;
            for (int j = 0; j < P.nc; ++j) {
                const double x = u[(size_t)(B.u_row + k) * P.nc + j];
                const bool fin = isfinite(x);
                if (!fin && row == 0) atomicOr(P.status, ST_NAN_PULSE);
                uk[j] = fin ? x : 0.0;
                beta += fabs(uk[j]) * B.hc_norm[j];
            }
            beta *= B.dt;
        }
        for (int off = MP / 2; off > 0; off >>= 1) beta = fmax(beta, __shfl_xor_sync(gmask, beta, off));
        const double cap = fmin(tabs.theta_cap, tabs.theta[6]);
        int s = 0;
        while (beta > cap && s < P.max_sq) { beta *= 0.5; ++s; }
        if (beta > cap && valid && row == 0) atomicOr(P.status, ST_SQUARING_CAP);
        int di = 0;
        while (di < 6 && tabs.theta[di] < beta) ++di;
        const int p = c_wp[di], q = c_wq[di], d = p * q;
        if (P.stats && valid && row == 0) {
            const unsigned long long m3 = (unsigned long long)m * m * m;
            atomicAdd(P.stats + 0, m3 * (unsigned long long)(p + q - 2));
            atomicAdd(P.stats + 1, m3 * (unsigned long long)s);
            atomicAdd(P.stats + 2, 1ull);
        }
        // X = -i (tau / 2^s)(H0 + sum_j u_j Hc_j), row by row
        cx<T> xr[MP], acc[MP];
        {
            const T sc = valid ? (T)(B.dt / (double)(1LL << s)) : (T)0;
            const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
            const size_t mm = (size_t)m * m;
#pragma unroll
            for (int j = 0; j < MP; ++j) {
                cx<T> h = mk<T>(0, 0);
                if (row < m && j < m) {
                    h = H[(size_t)row * m + j];
                    for (int c = 0; c < P.nc; ++c) {
                        const cx<T> hc = H[(size_t)(1 + c) * mm + (size_t)row * m + j];
                        h.x = fma((T)uk[c], hc.x, h.x);
                        h.y = fma((T)uk[c], hc.y, h.y);
                    }
                }
                xr[j] = cmul_mis<T>(h, sc);
                W.M[0][row][j] = xr[j];
            }
        }
        __syncwarp(gmask);
        // X^2 .. X^p
        for (int l = 2; l <= p; ++l) {
            row_times<T, MP>(acc, xr, W.M[0], m);
#pragma unroll
            for (int j = 0; j < MP; ++j) {
                xr[j] = acc[j];
                W.M[l - 1][row][j] = acc[j];
            }
            __syncwarp(gmask);
        }
        // S = c_d X^p + sum_{l<p} c_{(q-1)p+l} X^l, then S <- S X^p + sum_l c_{kb p + l} X^l
        const int b0 = (q - 1) * p;
        cx<T> S[MP];
#pragma unroll
        for (int j = 0; j < MP; ++j) {
            cx<T> v = cscale<T>(W.M[p - 1][row][j], (T)s_if[d]);
            if (j == row) v.x += (T)s_if[b0];
            for (int l = 1; l < p; ++l) {
                const cx<T> x = W.M[l - 1][row][j];
                const T cf = (T)s_if[b0 + l];
                v.x = fma(cf, x.x, v.x);
                v.y = fma(cf, x.y, v.y);
            }
            S[j] = v;
        }
        for (int kb = q - 2; kb >= 0; --kb) {
            row_times<T, MP>(acc, S, W.M[p - 1], m);
#pragma unroll
            for (int j = 0; j < MP; ++j) {
                cx<T> v = acc[j];
                if (j == row) v.x += (T)s_if[kb * p];
                for (int l = 1; l < p; ++l) {
                    const cx<T> x = W.M[l - 1][row][j];
                    const T cf = (T)s_if[kb * p + l];
                    v.x = fma(cf, x.x, v.x);
                    v.y = fma(cf, x.y, v.y);
                }
                S[j] = v;
            }
        }
        // squarings
        for (int i = 0; i < s; ++i) {
#pragma unroll
            for (int j = 0; j < MP; ++j) W.M[4][row][j] = S[j];
            __syncwarp(gmask);
            row_times<T, MP>(acc, S, W.M[4], m);
            __syncwarp(gmask);
#pragma unroll
            for (int j = 0; j < MP; ++j) S[j] = acc[j];
        }
        if (valid && row < m) {
            cx<T>* Uo = reinterpret_cast<cx<T>*>(Uout) + B.u_off + (size_t)kw * B.mmp + (size_t)row * m;
#pragma unroll
            for (int j = 0; j < MP; ++j)
                if (j < m) Uo[j] = S[j];
        }
        __syncwarp(gmask);
    }
}

template <class T, int MP, int WARPS>
int launch_w(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
             const int2* items, long long n_items, void* Uout, int per_warp, int grid, cudaStream_t st) {
    const size_t sm = sizeof(WarpSmem<T, MP>) * WARPS * (32 / MP);
    cudaFuncSetAttribute(expm_warp_kernel<T, MP, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    expm_warp_kernel<T, MP, WARPS><<<grid, 32 * WARPS, sm, st>>>(P, tabs, u, cls, n_cls, items, n_items, Uout,
                                                                per_warp);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class T, int MP, int WARPS>
int occupancy_w() {
    const size_t sm = sizeof(WarpSmem<T, MP>) * WARPS * (32 / MP);
    int occ = 0;
    cudaFuncSetAttribute(expm_warp_kernel<T, MP, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, expm_warp_kernel<T, MP, WARPS>, 32 * WARPS, sm);
    return occ < 1 ? 1 : occ;
}

}  // namespace

int expm_warp_mp(int prec, int m) {
    if (prec == QOC_PREC_F32) return 0;  // FP64 squaring after an FP32 polynomial: CTA kernel
    const int lim = prec == QOC_PREC_F64 ? 16 : 32;
    if (m > lim) return 0;
    return m <= 8 ? 8 : m <= 16 ? 16 : 32;
}

int expm_warp_grid_limit(int prec, int MP) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 1;
    if (prec == QOC_PREC_F64) occ = MP == 8 ? occupancy_w<double, 8, 4>() : occupancy_w<double, 16, 4>();
    else occ = MP == 8 ? occupancy_w<float, 8, 4>() : MP == 16 ? occupancy_w<float, 16, 4>() : occupancy_w<float, 32, 2>();
    return sms * occ;
}

int launch_expm_warp(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                     const int2* items, long long n_items, int MP, int per_warp, void* Uout, int grid, cudaStream_t st) {
    if (P.prec == QOC_PREC_F64) {
        if (MP == 8) return launch_w<double, 8, 4>(P, tabs, u, cls, n_cls, items, n_items, Uout, per_warp, grid, st);
        return launch_w<double, 16, 4>(P, tabs, u, cls, n_cls, items, n_items, Uout, per_warp, grid, st);
    }
    if (MP == 8) return launch_w<float, 8, 4>(P, tabs, u, cls, n_cls, items, n_items, Uout, per_warp, grid, st);
    if (MP == 16) return launch_w<float, 16, 4>(P, tabs, u, cls, n_cls, items, n_items, Uout, per_warp, grid, st);
    return launch_w<float, 32, 2>(P, tabs, u, cls, n_cls, items, n_items, Uout, per_warp, grid, st);
}

}  // namespace qoc
