// Forward states and backward costates (Sec. II.A, Eq. exppropagator; costates through U_k^dagger,
// Appendix B) with each chain split over a thread-block cluster.
//
// A sweep is N dependent matrix-vector products; with one CTA per chain (sweep.cu) a step is bounded
// by that CTA's fetch of the whole U_k.  Here a cluster of CL CTAs walks one (direction, block) chain:
// CTA q owns rows [q R, q R + R) of every U_k (R = ceil(m / CL)) and streams them through an
// STAGES-deep cp.async pipeline, so each SM moves only R m elements per step, far ahead of use.
//   forward  psi_k = U_k psi_{k-1}: a CTA computes its rows of psi_k into its exchange buffer; after
//            the cluster barrier every CTA gathers the whole vector from its peers' buffers (DSMEM);
//   backward lam_{k-1} = U_k^dagger lam_k: a CTA forms the partial sums over its rows for every
//            output; after the barrier it adds up its own range over the peers' partials.
// Exchange buffers alternate between steps, so one cluster barrier per step orders both the writes
// before the peers' reads and those reads before the buffer is written again two steps later.  The
// barrier and the cp.async waits are hardware waits: every CTA of a cluster runs the same number of
// steps, and the cluster launch makes its CTAs co-resident.
#include "../../include/qoc.h"
#include "kernels.h"
#include "tma.cuh"

namespace qoc {
namespace {

constexpr int SC_THREADS = 256;

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared variable in CTA 'rank' of the cluster
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t a, float2*) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_cluster(uint32_t a, double2*) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cp_async(void* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(void* dst, const double2* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Dynamic shared memory: U stages [STAGES][R][m], x [c][m] (this CTA's input: the whole vector
// forward, its own rows backward), exchange buffers xb[2][c][m].
template <class T, int STAGES>
__global__ void __launch_bounds__(SC_THREADS)
sweep_cluster_kernel(DevPlan P, const cx<T>* __restrict__ U, const cx<T>* __restrict__ fwd_init,
                     cx<T>* __restrict__ fwd_out, const cx<T>* __restrict__ bwd_init, cx<T>* __restrict__ bwd_out,
                     cx<T>* __restrict__ psi_st, cx<T>* __restrict__ lam_st, int dirs, int CL, int max_m, int max_c) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int chain = (int)(blockIdx.x / (unsigned)CL);
    const int q = (int)cluster_rank();
    const int nfw = (dirs & 1) ? P.nb : 0;
    const bool fwd = chain < nfw;
    const int bi = fwd ? chain : chain - nfw;
    const DevBlock B = P.blocks[bi];
    const int m = B.m, c = B.c, NK = P.nk < 0 ? B.N : P.nk;
    const long long mmp = B.mmp;
    const int R = (m + CL - 1) / CL;
    const int r0 = min(m, q * R), r1 = min(m, r0 + R), nr = r1 - r0;  // nr may be 0
    const int Rmax = (max_m + CL - 1) / CL;
    cx<T>* ust = reinterpret_cast<cx<T>*>(dsm);                  // [STAGES][Rmax * max_m]
    cx<T>* x = ust + (size_t)STAGES * Rmax * max_m;               // [max_c][max_m]
    cx<T>* xb = x + (size_t)max_c * max_m;                        // [2][max_c][max_m]
    const size_t xbs = (size_t)max_c * max_m;
    const int tid = threadIdx.x;
    cx<T>* st = fwd ? psi_st : lam_st;
    const long long s0 = B.s_off;

    // initial vector: forward needs all of it, backward its own rows; slot 0 (fwd) / NK (bwd) holds it
    {
        const cx<T>* init = (fwd ? fwd_init : bwd_init) + B.v_off;
        const long long kst = fwd ? 0 : NK;
        for (int e = tid; e < m * c; e += SC_THREADS) {
            const int r = e / m, o = e - r * m;
            x[(size_t)r * max_m + o] = init[e];
            if (o >= r0 && o < r1) st[s0 + kst * c * m + e] = init[e];
        }
    }
    // prologue of the U pipeline: steps 0 .. STAGES-2
    auto issue = [&](int t) {
        if (t < NK && nr > 0) {
            const int i = fwd ? t : NK - 1 - t;
            const cx<T>* src = U + B.u_off + (long long)i * mmp + (long long)r0 * m;
            cx<T>* dst = ust + (size_t)(t % STAGES) * Rmax * max_m;
            for (int e = tid; e < nr * m; e += SC_THREADS) cp_async(dst + e, src + e);
        }
        cp_commit();
    };
    for (int t = 0; t < STAGES - 1; ++t) issue(t);
    __syncthreads();

    // work split: forward outputs (own rows x copies), G threads each; backward outputs (all m x copies)
    const int nout = fwd ? nr * c : m * c;
    int G = 1;
    while (G < 32 && G * 2 * nout <= SC_THREADS) G *= 2;
    const int part = tid % G, og = tid / G, ngroups = SC_THREADS / G;

    for (int t = 0; t < NK; ++t) {
        issue(t + STAGES - 1);
        cp_wait<STAGES - 1>();
        __syncthreads();
        const cx<T>* Uk = ust + (size_t)(t % STAGES) * Rmax * max_m;  // rows r0.. of U_i, [nr][m]
        cx<T>* out = xb + (size_t)(t & 1) * xbs;
        if (fwd) {
            // rows of psi: out[r][o - r0] = sum_j U[o][j] x[r][j]
            for (int o0 = 0; o0 < nout; o0 += ngroups) {
                const int e = o0 + og;
                cx<T> acc = mk<T>(0, 0);
                int r = 0, ol = 0;
                if (e < nout) {
                    r = e / nr;
                    ol = e - r * nr;
                    const cx<T>* row = Uk + (size_t)ol * m;
                    const cx<T>* xr = x + (size_t)r * max_m;
                    for (int j = part; j < m; j += G) cfma<T>(acc, row[j], xr[j]);
                }
                for (int off = G / 2; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (e < nout && part == 0) out[(size_t)r * max_m + ol] = acc;
            }
        } else {
            // partial sums over this CTA's rows: out[r][o] = sum_{ii in rows} conj(U[ii][o]) x[r][ii]
            for (int o0 = 0; o0 < nout; o0 += ngroups) {
                const int e = o0 + og;
                cx<T> acc = mk<T>(0, 0);
                int r = 0, o = 0;
                if (e < nout) {
                    r = e / m;
                    o = e - r * m;
                    const cx<T>* xr = x + (size_t)r * max_m;
                    for (int ii = part; ii < nr; ii += G) cfma_conj<T>(acc, Uk[(size_t)ii * m + o], xr[r0 + ii]);
                }
                for (int off = G / 2; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (e < nout && part == 0) out[(size_t)r * max_m + o] = acc;
            }
        }
        cluster_sync_all();  // exchange buffers of step t complete in every CTA of the cluster
        const int i = fwd ? t : NK - 1 - t;
        const long long ks = fwd ? i + 1 : i;
        if (fwd) {
            // gather the whole psi_k: element o lives in CTA o / R at local index o - (o / R) R
            for (int e = tid; e < m * c; e += SC_THREADS) {
                const int r = e / m, o = e - r * m;
                const int own = o / R;
                const cx<T> v = ld_cluster(map_rank(out + (size_t)r * max_m + (o - own * R), (uint32_t)own),
                                           (cx<T>*)nullptr);
                x[(size_t)r * max_m + o] = v;
                if (own == q) st[s0 + ks * c * m + e] = v;
            }
        } else {
            // own rows of lam_{k-1}: the sum of every CTA's partial for them
            for (int e = tid; e < nr * c; e += SC_THREADS) {
                const int r = e / nr, o = r0 + (e - r * nr);
                cx<T> v = mk<T>(0, 0);
                for (int p2 = 0; p2 < CL; ++p2) {
                    const cx<T> w = ld_cluster(map_rank(out + (size_t)r * max_m + o, (uint32_t)p2), (cx<T>*)nullptr);
                    v.x += w.x;
                    v.y += w.y;
                }
                x[(size_t)r * max_m + o] = v;
                st[s0 + ks * c * m + (size_t)r * m + o] = v;
            }
        }
        __syncthreads();
    }
    cp_wait<0>();
    // final vector (own range) to the boundary output
    cx<T>* fin = (fwd ? fwd_out : bwd_out) + B.v_off;
    for (int e = tid; e < nr * c; e += SC_THREADS) {
        const int r = e / nr, o = r0 + (e - r * nr);
        fin[(size_t)r * m + o] = x[(size_t)r * max_m + o];
    }
    cluster_sync_all();  // no CTA leaves while a peer may still read its exchange buffers
}

template <class T, int STAGES>
size_t sc_smem(int max_m, int max_c, int CL) {
    const int Rmax = (max_m + CL - 1) / CL;
    return ((size_t)STAGES * Rmax * max_m + 3 * (size_t)max_c * max_m) * sizeof(cx<T>);
}

template <class T, int STAGES>
int sc_launch(const DevPlan& P, const void* U, const void* fi, void* fo, const void* bi, void* bo, void* ps, void* ls,
              int dirs, int CL, int max_m, int max_c, int nchains, cudaStream_t st) {
    const size_t sm = sc_smem<T, STAGES>(max_m, max_c, CL);
    auto kern = sweep_cluster_kernel<T, STAGES>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nchains * CL));
    cfg.blockDim = dim3(SC_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P, (const cx<T>*)U, (const cx<T>*)fi, (cx<T>*)fo,
                                             (const cx<T>*)bi, (cx<T>*)bo, (cx<T>*)ps, (cx<T>*)ls, dirs, CL, max_m,
                                             max_c);
    return e == cudaSuccess ? 0 : -1;
}

constexpr size_t SC_SMEM_LIMIT = 220 * 1024;

}  // namespace

int sweep_cluster_fits(int prec, int max_m, int max_c, int CL) {
    const size_t sm = prec == QOC_PREC_F64 ? sc_smem<double, 8>(max_m, max_c, CL) : sc_smem<float, 8>(max_m, max_c, CL);
    return sm <= SC_SMEM_LIMIT;
}

// Cluster size for the sweeps of a plan with nb active blocks (0: use the one-CTA-per-chain kernel).
// Every chain must find its cluster resident at once: chains x CL CTAs within the GPU's clusters.
int sweep_cluster_size(int prec, int nb, int max_m, int max_c) {
    if (max_m < 24 || nb < 1) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chains = 2 * nb;
    for (int CL = 8; CL >= 2; CL /= 2) {
        if (chains * CL > sms) continue;
        const size_t sm = prec == QOC_PREC_F64 ? sc_smem<double, 8>(max_m, max_c, CL) : sc_smem<float, 8>(max_m, max_c, CL);
        if (sm > SC_SMEM_LIMIT) continue;
        // clusters of this shape that the GPU holds at once
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(chains * CL));
        cfg.blockDim = dim3(SC_THREADS);
        cfg.dynamicSmemBytes = sm;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclu = 0;
        cudaError_t e;
        if (prec == QOC_PREC_F64) {
            cudaFuncSetAttribute(sweep_cluster_kernel<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            e = cudaOccupancyMaxActiveClusters(&nclu, sweep_cluster_kernel<double, 8>, &cfg);
        } else {
            cudaFuncSetAttribute(sweep_cluster_kernel<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            e = cudaOccupancyMaxActiveClusters(&nclu, sweep_cluster_kernel<float, 8>, &cfg);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclu >= chains) return CL;
    }
    return 0;
}

int launch_sweeps_cluster(const DevPlan& P, const void* U, const void* fwd_init, void* fwd_out, const void* bwd_init,
                          void* bwd_out, void* psi_store, void* lam_store, int dirs, int max_m, int max_c, int CL,
                          cudaStream_t st) {
    const int nchains = ((dirs & 1) ? P.nb : 0) + ((dirs & 2) ? P.nb : 0);
    if (nchains == 0) return 0;
    if (P.prec == QOC_PREC_F64)
        return sc_launch<double, 8>(P, U, fwd_init, fwd_out, bwd_init, bwd_out, psi_store, lam_store, dirs, CL, max_m,
                                    max_c, nchains, st);
    return sc_launch<float, 8>(P, U, fwd_init, fwd_out, bwd_init, bwd_out, psi_store, lam_store, dirs, CL, max_m, max_c,
                               nchains, st);
}

}  // namespace qoc
