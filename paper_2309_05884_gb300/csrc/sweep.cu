// Forward states and backward costates through all slices (Sec. II.A, Eq. exppropagator; the
// costates use U_k^dagger = U_k^{-1}, unitarity as noted in Appendix B), and the FP64 overlap
// o = <psi_f|psi_N> of Eq. probability.
//
// One CTA per (direction, active block) walks the N slices in order; the two directions are
// independent (lam_N = psi_f does not depend on psi_N), so both run concurrently.  When two
// propagators fit in shared memory, U_{k+1} is fetched by a bulk asynchronous copy (TMA) into the
// idle buffer while U_k is applied; waits on the copy are bounded in time.  Each output element
// is reduced by a group of G threads (G = largest power of two with G*m <= blockDim).
#include "kernels.h"
#include "tma.cuh"

namespace qoc {

namespace {

constexpr int SWEEP_THREADS = 256;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

template <class T>
__global__ void __launch_bounds__(SWEEP_THREADS)
sweep_kernel(DevPlan P, const cx<T>* __restrict__ U, const double2* __restrict__ psi0,
             const double2* __restrict__ psif, cx<T>* __restrict__ psi_st, cx<T>* __restrict__ lam_st, int dirs,
             int staged) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar[2];

    const int nfw = (dirs & 1) ? P.nb : 0;
    const bool fwd = (int)blockIdx.x < nfw;
    const int bi = fwd ? (int)blockIdx.x : (int)blockIdx.x - nfw;
    const DevBlock B = P.blocks[bi];
    const int m = B.m, c = B.c, N = P.N;
    const long long mmp = B.mmp;
    const uint32_t ubytes = (uint32_t)(mmp * (long long)sizeof(cx<T>));
    cx<T>* ubuf0 = reinterpret_cast<cx<T>*>(dsm);
    cx<T>* ubuf1 = ubuf0 + (staged ? mmp : 0);
    cx<T>* x = ubuf0 + (staged ? 2 * mmp : 0);
    cx<T>* y = x + (size_t)m * c;
    const int tid = threadIdx.x;

    const long long cb = P.copy_base[bi];
    const double2* src = fwd ? psi0 : psif;
    for (int e = tid; e < m * c; e += blockDim.x) {
        const int r = e / m, a = e - r * m;
        x[e] = ccast<T, double>(src[P.copy_src[cb + r] + a]);
    }
    cx<T>* st = fwd ? psi_st : lam_st;
    const long long s0 = B.s_off;
    __syncthreads();
    {
        const long long kst = fwd ? 0 : N;
        for (int e = tid; e < m * c; e += blockDim.x) st[s0 + kst * c * m + e] = x[e];
    }
    if (staged) {
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            const int k = fwd ? 1 : N;
            mbar_arrive_expect_tx(&bar[0], ubytes);
            bulk_copy_g2s(ubuf0, U + B.u_off + (long long)(k - 1) * mmp, ubytes, &bar[0]);
        }
    }
    int G = 1;
    while (G < 32 && G * 2 * m <= (int)blockDim.x) G *= 2;
    const int outs = blockDim.x / G;
    const int part = tid % G;

    for (int t = 0; t < N; ++t) {
        const int k = fwd ? t + 1 : N - t;
        const cx<T>* Uk;
        if (staged) {
            const int buf = t & 1;
            if (tid == 0 && t + 1 < N) {
                const int kn = fwd ? k + 1 : k - 1;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[buf ^ 1], ubytes);
                bulk_copy_g2s(buf ? ubuf0 : ubuf1, U + B.u_off + (long long)(kn - 1) * mmp, ubytes, &bar[buf ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[buf], (uint32_t)((t >> 1) & 1), WAIT_LIMIT_NS);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(P.status, ST_TIMEOUT);
                    if (t + 1 < N) mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)(((t + 1) >> 1) & 1), WAIT_LIMIT_NS);
                }
                return;
            }
            Uk = buf ? ubuf1 : ubuf0;
        } else {
            Uk = U + B.u_off + (long long)(k - 1) * mmp;
        }
        for (int o0 = 0; o0 < m; o0 += outs) {
            const int o = o0 + tid / G;
            for (int r = 0; r < c; ++r) {
                cx<T> acc = mk<T>(0, 0);
                if (o < m) {
                    const cx<T>* xr = x + (size_t)r * m;
                    if (fwd) {
                        const cx<T>* row = Uk + (size_t)o * m;
                        for (int j = part; j < m; j += G) cfma<T>(acc, row[j], xr[j]);
                    } else {
                        for (int i = part; i < m; i += G) cfma_conj<T>(acc, Uk[(size_t)i * m + o], xr[i]);
                    }
                }
                for (int off = G / 2; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (o < m && part == 0) y[(size_t)r * m + o] = acc;
            }
        }
        __syncthreads();
        const long long ks = fwd ? k : k - 1;
        for (int e = tid; e < m * c; e += blockDim.x) {
            x[e] = y[e];
            st[s0 + ks * c * m + e] = y[e];
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(256)
overlap_kernel(DevPlan P, const cx<T>* __restrict__ psi_st, const double2* __restrict__ psif, double* out3,
               double2* o_ws) {
    __shared__ double sre[256], sim[256];
    double re = 0.0, im = 0.0;
    for (int bi = 0; bi < P.nb; ++bi) {
        const DevBlock& B = P.blocks[bi];
        const int m = B.m, c = B.c;
        const long long cb = P.copy_base[bi];
        const cx<T>* pN = psi_st + B.s_off + (long long)P.N * c * m;
        for (int e = threadIdx.x; e < m * c; e += blockDim.x) {
            const int r = e / m, a = e - r * m;
            const double2 f = psif[P.copy_src[cb + r] + a];
            const double px = (double)pN[e].x, py = (double)pN[e].y;
            re += f.x * px + f.y * py;
            im += f.x * py - f.y * px;
        }
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sre[threadIdx.x] += sre[threadIdx.x + s];
            sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double a = sre[0], b = sim[0];
        out3[0] = a * a + b * b;
        out3[1] = a;
        out3[2] = b;
        o_ws->x = a;
        o_ws->y = b;
    }
}

template <class T>
__global__ void store_final_kernel(DevPlan P, const cx<T>* __restrict__ psi_st, double2* __restrict__ psiN) {
    for (int bi = 0; bi < P.nb; ++bi) {
        const DevBlock& B = P.blocks[bi];
        const int m = B.m, c = B.c;
        const long long cb = P.copy_base[bi];
        const cx<T>* pN = psi_st + B.s_off + (long long)P.N * c * m;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * c; e += gridDim.x * blockDim.x) {
            const int r = e / m, a = e - r * m;
            psiN[P.copy_src[cb + r] + a] = ccast<double, T>(pN[e]);
        }
    }
}

template <class T>
size_t sweep_smem(int m, int c, int staged, long long mmp) {
    return (staged ? 2 * (size_t)mmp * sizeof(cx<T>) : 0) + 2 * (size_t)m * c * sizeof(cx<T>);
}

}  // namespace

int launch_sweeps(const DevPlan& P, const void* U, const double2* psi0, const double2* psif, void* psi_store,
                  void* lam_store, int dirs, int max_m, int max_c, cudaStream_t st) {
    const int nblk = ((dirs & 1) ? P.nb : 0) + ((dirs & 2) ? P.nb : 0);
    if (nblk == 0) return 0;
    const long long mmp = ((long long)max_m * max_m + 3) / 4 * 4;
    const size_t limit = 220 * 1024;
    if (P.prec == 0) {
        int staged = sweep_smem<double>(max_m, max_c, 1, mmp) <= limit;
        size_t sm = sweep_smem<double>(max_m, max_c, staged, mmp);
        if (sm > limit) return -2;
        cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sweep_kernel<double><<<nblk, SWEEP_THREADS, sm, st>>>(P, (const double2*)U, psi0, psif, (double2*)psi_store,
                                                              (double2*)lam_store, dirs, staged);
    } else {
        int staged = sweep_smem<float>(max_m, max_c, 1, mmp) <= limit;
        size_t sm = sweep_smem<float>(max_m, max_c, staged, mmp);
        if (sm > limit) return -2;
        cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sweep_kernel<float><<<nblk, SWEEP_THREADS, sm, st>>>(P, (const float2*)U, psi0, psif, (float2*)psi_store,
                                                             (float2*)lam_store, dirs, staged);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_overlap(const DevPlan& P, const void* psi_store, const double2* psif, double* out3, double2* o_ws,
                   cudaStream_t st) {
    if (P.prec == 0)
        overlap_kernel<double><<<1, 256, 0, st>>>(P, (const double2*)psi_store, psif, out3, o_ws);
    else
        overlap_kernel<float><<<1, 256, 0, st>>>(P, (const float2*)psi_store, psif, out3, o_ws);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_store_final(const DevPlan& P, const void* psi_store, double2* psiN, long long state_len,
                       cudaStream_t st) {
    if (cudaMemsetAsync(psiN, 0, (size_t)state_len * sizeof(double2), st) != cudaSuccess) return -1;
    if (P.prec == 0)
        store_final_kernel<double><<<8, 256, 0, st>>>(P, (const double2*)psi_store, psiN);
    else
        store_final_kernel<float><<<8, 256, 0, st>>>(P, (const float2*)psi_store, psiN);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
