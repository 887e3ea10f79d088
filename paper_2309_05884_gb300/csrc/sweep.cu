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

// Window sweeps: forward from fwd_init (psi at the window start) through the window's nk slices,
// storing psi in window slots 0..nk and psi at the window end in fwd_out; backward from bwd_init
// (lam at the window end) down to the window start, storing lam in slots 0..nk and lam at the window
// start in bwd_out.  Boundary vectors use the [block][copy][m] layout (DevBlock::v_off).
template <class T>
__global__ void __launch_bounds__(SWEEP_THREADS)
sweep_kernel(DevPlan P, const cx<T>* __restrict__ U, const cx<T>* __restrict__ fwd_init, cx<T>* __restrict__ fwd_out,
             const cx<T>* __restrict__ bwd_init, cx<T>* __restrict__ bwd_out, cx<T>* __restrict__ psi_st,
             cx<T>* __restrict__ lam_st, int dirs, int staged) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar[2];

    const int nfw = (dirs & 1) ? P.nb : 0;
    const bool fwd = (int)blockIdx.x < nfw;
    const int bi = fwd ? (int)blockIdx.x : (int)blockIdx.x - nfw;
    const DevBlock B = P.blocks[bi];
    const int m = B.m, c = B.c, NK = P.nk < 0 ? B.N : P.nk;
    const long long mmp = B.mmp;
    const uint32_t ubytes = (uint32_t)(mmp * (long long)sizeof(cx<T>));
    cx<T>* ubuf0 = reinterpret_cast<cx<T>*>(dsm);
    cx<T>* ubuf1 = ubuf0 + (staged ? mmp : 0);
    cx<T>* x = ubuf0 + (staged ? 2 * mmp : 0);
    cx<T>* y = x + (size_t)m * c;
    const int tid = threadIdx.x;

    const cx<T>* init = (fwd ? fwd_init : bwd_init) + B.v_off;
    for (int e = tid; e < m * c; e += blockDim.x) x[e] = init[e];
    cx<T>* st = fwd ? psi_st : lam_st;
    const long long s0 = B.s_off;
    __syncthreads();
    {
        const long long kst = fwd ? 0 : NK;
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
            const int i = fwd ? 0 : NK - 1;
            mbar_arrive_expect_tx(&bar[0], ubytes);
            bulk_copy_g2s(ubuf0, U + B.u_off + (long long)i * mmp, ubytes, &bar[0]);
        }
    }
    int G = 1;
    while (G < 32 && G * 2 * m <= (int)blockDim.x) G *= 2;
    const int outs = blockDim.x / G;
    const int part = tid % G;

    for (int t = 0; t < NK; ++t) {
        const int i = fwd ? t : NK - 1 - t;  // window slot of the propagator applied now
        const cx<T>* Uk;
        if (staged) {
            const int buf = t & 1;
            if (tid == 0 && t + 1 < NK) {
                const int in = fwd ? i + 1 : i - 1;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[buf ^ 1], ubytes);
                bulk_copy_g2s(buf ? ubuf0 : ubuf1, U + B.u_off + (long long)in * mmp, ubytes, &bar[buf ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[buf], (uint32_t)((t >> 1) & 1), WAIT_LIMIT_NS);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(P.status, ST_TIMEOUT);
                    if (t + 1 < NK) mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)(((t + 1) >> 1) & 1), WAIT_LIMIT_NS);
                }
                return;
            }
            Uk = buf ? ubuf1 : ubuf0;
        } else {
            Uk = U + B.u_off + (long long)i * mmp;
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
                        for (int ii = part; ii < m; ii += G) cfma_conj<T>(acc, Uk[(size_t)ii * m + o], xr[ii]);
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
        const long long ks = fwd ? i + 1 : i;
        for (int e = tid; e < m * c; e += blockDim.x) {
            x[e] = y[e];
            st[s0 + ks * c * m + e] = y[e];
        }
        __syncthreads();
    }
    cx<T>* out = (fwd ? fwd_out : bwd_out) + B.v_off;
    for (int e = tid; e < m * c; e += blockDim.x) out[e] = x[e];
}

// dst[v_off_b + r*m + a] = (T) src[copy_src(b, r) + a]: the caller's block state -> boundary layout
template <class T>
__global__ void gather_kernel(DevPlan P, const double2* __restrict__ src, cx<T>* __restrict__ dst) {
    for (int bi = blockIdx.y; bi < P.nb; bi += gridDim.y) {
        const DevBlock& B = P.blocks[bi];
        const int m = B.m, c = B.c;
        const long long cb = P.copy_base[bi];
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * c; e += gridDim.x * blockDim.x) {
            const int r = e / m, a = e - r * m;
            dst[B.v_off + e] = ccast<T, double>(src[P.copy_src[cb + r] + a]);
        }
    }
}

// One CTA per problem: o_p = sum over the problem's active copies <psif|psi_N> in FP64;
// out3[3p..3p+2] = {|o_p|^2, Re o_p, Im o_p}; o_ws[p] = o_p.
template <class T>
__global__ void __launch_bounds__(256)
overlap_kernel(DevPlan P, const cx<T>* __restrict__ fin, const double2* __restrict__ psif, double* out3,
               double2* o_ws) {
    __shared__ double sre[256], sim[256];
    const int p = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int t = P.prob_block_off[p]; t < P.prob_block_off[p + 1]; ++t) {
        const int bi = P.prob_blocks[t];
        const DevBlock& B = P.blocks[bi];
        const int m = B.m, c = B.c;
        const long long cb = P.copy_base[bi];
        const cx<T>* pN = fin + B.v_off;
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
        out3[3 * p + 0] = a * a + b * b;
        out3[3 * p + 1] = a;
        out3[3 * p + 2] = b;
        o_ws[p].x = a;
        o_ws[p].y = b;
    }
}

template <class T>
__global__ void store_final_kernel(DevPlan P, const cx<T>* __restrict__ fin, double2* __restrict__ psiN) {
    for (int bi = 0; bi < P.nb; ++bi) {
        const DevBlock& B = P.blocks[bi];
        const int m = B.m, c = B.c;
        const long long cb = P.copy_base[bi];
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * c; e += gridDim.x * blockDim.x) {
            const int r = e / m, a = e - r * m;
            psiN[P.copy_src[cb + r] + a] = ccast<double, T>(fin[B.v_off + e]);
        }
    }
}

// One CTA per problem: FP64 norms of its initial and target block states (every copy, active or
// not: the caller's whole state); latches ST_NORM if either is off 1 by more than tol (or not finite).
__global__ void __launch_bounds__(256)
norm_check_kernel(const int64_t* __restrict__ prob_state, const double2* __restrict__ a,
                  const double2* __restrict__ b, double tol, int* status) {
    __shared__ double sa[256], sb[256];
    const int p = blockIdx.x;
    const int64_t off = prob_state[2 * p], len = prob_state[2 * p + 1];
    double na = 0.0, nb = 0.0;
    for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
        const double2 x = a[off + e];
        na = fma(x.x, x.x, fma(x.y, x.y, na));
        if (b) {
            const double2 y = b[off + e];
            nb = fma(y.x, y.x, fma(y.y, y.y, nb));
        }
    }
    sa[threadIdx.x] = na;
    sb[threadIdx.x] = nb;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool ok_a = fabs(sqrt(sa[0]) - 1.0) <= tol;
        const bool ok_b = !b || fabs(sqrt(sb[0]) - 1.0) <= tol;
        if (!(ok_a && ok_b)) atomicOr(status, ST_NORM);
    }
}

// Nothing arrives on the barrier, so its phase 0 never completes: the bounded wait gives up.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(status, ST_TIMEOUT);
    }
}

template <class T>
size_t sweep_smem(int m, int c, int staged, long long mmp) {
    return (staged ? 2 * (size_t)mmp * sizeof(cx<T>) : 0) + 2 * (size_t)m * c * sizeof(cx<T>);
}

}  // namespace

int launch_sweeps(const DevPlan& P, const void* U, const void* fwd_init, void* fwd_out, const void* bwd_init,
                  void* bwd_out, void* psi_store, void* lam_store, int dirs, int max_m, int max_c, cudaStream_t st) {
    const int nblk = ((dirs & 1) ? P.nb : 0) + ((dirs & 2) ? P.nb : 0);
    if (nblk == 0) return 0;
    const long long mmp = ((long long)max_m * max_m + 3) / 4 * 4;
    const size_t limit = 220 * 1024;
    if (P.prec == 0) {
        int staged = sweep_smem<double>(max_m, max_c, 1, mmp) <= limit;
        size_t sm = sweep_smem<double>(max_m, max_c, staged, mmp);
        if (sm > limit) return -2;
        cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sweep_kernel<double><<<nblk, SWEEP_THREADS, sm, st>>>(
            P, (const double2*)U, (const double2*)fwd_init, (double2*)fwd_out, (const double2*)bwd_init,
            (double2*)bwd_out, (double2*)psi_store, (double2*)lam_store, dirs, staged);
    } else {
        int staged = sweep_smem<float>(max_m, max_c, 1, mmp) <= limit;
        size_t sm = sweep_smem<float>(max_m, max_c, staged, mmp);
        if (sm > limit) return -2;
        cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sweep_kernel<float><<<nblk, SWEEP_THREADS, sm, st>>>(
            P, (const float2*)U, (const float2*)fwd_init, (float2*)fwd_out, (const float2*)bwd_init,
            (float2*)bwd_out, (float2*)psi_store, (float2*)lam_store, dirs, staged);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_norm_check(const int64_t* prob_state, int n_prob, const double2* a, const double2* b, double tol,
                      int* status, cudaStream_t st) {
    norm_check_kernel<<<n_prob, 256, 0, st>>>(prob_state, a, b, tol, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather(const DevPlan& P, const double2* src, void* dst, cudaStream_t st) {
    dim3 grid(4, P.nb < 1024 ? P.nb : 1024);
    if (P.prec == 0)
        gather_kernel<double><<<grid, 256, 0, st>>>(P, src, (double2*)dst);
    else
        gather_kernel<float><<<grid, 256, 0, st>>>(P, src, (float2*)dst);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_overlap(const DevPlan& P, const void* fin, const double2* psif, double* out3, double2* o_ws,
                   cudaStream_t st) {
    if (P.prec == 0)
        overlap_kernel<double><<<P.n_prob, 256, 0, st>>>(P, (const double2*)fin, psif, out3, o_ws);
    else
        overlap_kernel<float><<<P.n_prob, 256, 0, st>>>(P, (const float2*)fin, psif, out3, o_ws);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_store_final(const DevPlan& P, const void* fin, double2* psiN, long long state_len, cudaStream_t st) {
    if (cudaMemsetAsync(psiN, 0, (size_t)state_len * sizeof(double2), st) != cudaSuccess) return -1;
    if (P.prec == 0)
        store_final_kernel<double><<<8, 256, 0, st>>>(P, (const double2*)fin, psiN);
    else
        store_final_kernel<float><<<8, 256, 0, st>>>(P, (const float2*)fin, psiN);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
