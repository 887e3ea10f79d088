// Forward states and backward costates (Sec. II.A, Eq. exppropagator; costates through U_k^dagger,
// Appendix B) with each chain split over a thread-block cluster.
//
// A sweep is N dependent matrix-vector products; with one CTA per chain (sweep.cu) a step is bounded
// by that CTA's fetch of the whole U_k.  Here a cluster of CL CTAs walks one (direction, block) chain:
// CTA q owns rows [q R, q R + R) of every U_k (R = ceil(m / CL)) and streams them through an
// STAGES-slot ring of bulk copies (one copy per slot: the rows are contiguous in U_k; an mbarrier per
// slot), so each SM moves only R m elements per step, far ahead of use; when R rows do not fit a slot
// (large blocks) the ring carries sub-blocks of RS rows.
//   forward  psi_k = U_k psi_{k-1}: a CTA computes its rows of psi_k into its exchange buffer; after
//            the cluster barrier every CTA gathers the whole vector from its peers' buffers (DSMEM);
//   backward lam_{k-1} = U_k^dagger lam_k: a CTA forms the partial sums over its rows for every
//            output; after the barrier it adds up its own range over the peers' partials.
// Exchange buffers alternate between steps, so one cluster barrier per step orders both the writes
// before the peers' reads and those reads before the buffer is written again two steps later.  The
// cluster barrier is a hardware wait: every CTA of a cluster runs the same number of steps, and the
// cluster launch makes its CTAs co-resident.  The slot waits are bounded; one that runs out latches
// ST_TIMEOUT and the CTA carries on, so that its cluster still reaches every barrier.
#include <algorithm>

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
constexpr uint64_t SC_WAIT_NS = 2000000000ull;

// elements of one ring slot: RS rows of max_m, one element of lead-in (a bulk copy starts on a 16-byte
// boundary, an FP32 row may start 8 bytes past one) and one of round-up, kept even
template <class T>
__host__ __device__ __forceinline__ size_t sc_slot(int RS, int max_m) {
    return ((size_t)RS * max_m + 2 + 1) / 2 * 2;
}

// Element span of U that one slot copy moves: the first element e0 rounded down to a 16-byte
// boundary (lead = e0 - start, 0 or 1 for FP32 complex), n elements rounded up to 16 bytes.  Both
// ends stay inside the slice's slot of the store: its stride mmp is m^2 rounded up to 4, and a
// misaligned start implies m odd, so m^2 odd and mmp >= m^2 + 1.
template <class T>
__device__ __forceinline__ int sc_lead(long long e0) {
    return sizeof(cx<T>) == 16 ? 0 : (int)(e0 & 1);
}

// Dynamic shared memory: U ring [STAGES][sc_slot], x [c][m] (this CTA's input: the whole vector
// forward, its own rows backward), exchange buffers xb[2][c][m].  SUB = false: a slot holds all of a
// CTA's rows (RS >= R); SUB = true: the rows of a step pass through the ring in sub-blocks of RS.
template <class T, int STAGES, bool SUB>
__global__ void __launch_bounds__(SC_THREADS)
sweep_cluster_kernel(DevPlan P, const cx<T>* __restrict__ U, const cx<T>* __restrict__ fwd_init,
                     cx<T>* __restrict__ fwd_out, const cx<T>* __restrict__ bwd_init, cx<T>* __restrict__ bwd_out,
                     cx<T>* __restrict__ psi_st, cx<T>* __restrict__ lam_st, int dirs, int CL, int max_m, int max_c,
                     int RS) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ cx<T> red[SC_THREADS / 32];
    __shared__ __align__(8) uint64_t full[STAGES];  // slot s filled: one arrival (the issuing thread) + bytes
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
    const size_t SLOT = sc_slot<T>(RS, max_m);
    cx<T>* ust = reinterpret_cast<cx<T>*>(dsm);                  // [STAGES][SLOT]
    cx<T>* x = ust + (size_t)STAGES * SLOT;                       // [max_c][max_m]
    cx<T>* xb = x + (size_t)max_c * max_m;                        // [2][max_c][max_m]
    const size_t xbs = (size_t)max_c * max_m;
    const int tid = threadIdx.x;
    cx<T>* st = fwd ? psi_st : lam_st;
    const long long s0 = B.s_off;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    // one bulk copy of n elements of U starting at element e0 into slot s (thread 0; the slot's
    // previous contents were read before the barrier that precedes this call)
    auto fill = [&](int s, long long e0, long long n) {
        if (tid == 0) {
            const int lead = sc_lead<T>(e0);
            const long long cnt = sizeof(cx<T>) == 16 ? n : (n + lead + 1) / 2 * 2;  // whole 16-byte units
            const uint32_t bytes = (uint32_t)(cnt * sizeof(cx<T>));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_copy_g2s(ust + (size_t)s * SLOT, U + (e0 - lead), bytes, &full[s]);
        }
    };
    // wait for fill number f (slot f % STAGES, phase f / STAGES)
    auto wait_fill = [&](long long f) {
        if (!mbar_wait_bounded(&full[f % STAGES], (uint32_t)((f / STAGES) & 1), SC_WAIT_NS) && tid == 0)
            atomicOr(P.status, ST_TIMEOUT);
    };

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
    // Work split of one pass over staged rows ra .. ra + rn of this CTA's rows of U_i: forward outputs
    // (those rows x copies), backward outputs (all m x copies), 2^lg threads each, nout <= SC_THREADS
    // >> lg; long forward rows (m >= 512, sub-block mode) may span several warps.
    const int lg_max = SUB && fwd && m >= 512 ? 8 : 5;
    auto split = [&](int nout) {
        int lg = 0;
        while (lg < lg_max && (2 << lg) * nout <= SC_THREADS) ++lg;
        return lg;
    };
    // forward: out[r][ra + ol] = sum_j U[r0 + ra + ol][j] x[r][j];
    // backward: out[r][o] (first pass) = or += sum_{ii < rn} conj(U[r0 + ra + ii][o]) x[r][r0 + ra + ii]
    auto compute = [&](const cx<T>* Uk, int ra, int rn, int lg, bool first, cx<T>* out) {
        const int G = 1 << lg, part = tid & (G - 1), og = tid >> lg, ngroups = SC_THREADS >> lg;
        const int nout = fwd ? rn * c : m * c;
        if (SUB && fwd && lg > 5) {
            // one pass: warp sums, then the group's warps through shared memory
            const int e = og;
            const int r = e < nout ? e / rn : 0, ol = e < nout ? e - r * rn : 0;
            cx<T> acc = mk<T>(0, 0);
            if (e < nout) {
                const cx<T>* row = Uk + (size_t)ol * m;
                const cx<T>* xr = x + (size_t)r * max_m;
                for (int j = part; j < m; j += G) cfma<T>(acc, row[j], xr[j]);
            }
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (e < nout && part == 0) {
                for (int w = 1; w < G / 32; ++w) {
                    acc.x += red[(tid >> 5) + w].x;
                    acc.y += red[(tid >> 5) + w].y;
                }
                out[(size_t)r * max_m + ra + ol] = acc;
            }
        } else if (fwd) {
            for (int o0 = 0; o0 < nout; o0 += ngroups) {
                const int e = o0 + og;
                cx<T> acc = mk<T>(0, 0);
                int r = 0, ol = 0;
                if (e < nout) {
                    r = e / rn;
                    ol = e - r * rn;
                    const cx<T>* row = Uk + (size_t)ol * m;
                    const cx<T>* xr = x + (size_t)r * max_m;
                    cx<T> a1 = mk<T>(0, 0);  // two chains, so that loads of successive terms overlap
                    int j = part;
                    for (; j + G < m; j += 2 * G) {
                        cfma<T>(acc, row[j], xr[j]);
                        cfma<T>(a1, row[j + G], xr[j + G]);
                    }
                    if (j < m) cfma<T>(acc, row[j], xr[j]);
                    acc.x += a1.x;
                    acc.y += a1.y;
                }
                for (int off = G / 2; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (e < nout && part == 0) out[(size_t)r * max_m + ra + ol] = acc;
            }
        } else {
            for (int o0 = 0; o0 < nout; o0 += ngroups) {
                const int e = o0 + og;
                cx<T> acc = mk<T>(0, 0);
                int r = 0, o = 0;
                if (e < nout) {
                    r = e / m;
                    o = e - r * m;
                    const cx<T>* xr = x + (size_t)r * max_m + r0 + ra;
                    cx<T> a1 = mk<T>(0, 0);
                    int ii = part;
                    for (; ii + G < rn; ii += 2 * G) {
                        cfma_conj<T>(acc, Uk[(size_t)ii * m + o], xr[ii]);
                        cfma_conj<T>(a1, Uk[(size_t)(ii + G) * m + o], xr[ii + G]);
                    }
                    if (ii < rn) cfma_conj<T>(acc, Uk[(size_t)ii * m + o], xr[ii]);
                    acc.x += a1.x;
                    acc.y += a1.y;
                }
                for (int off = G / 2; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (e < nout && part == 0) {
                    cx<T>& d = out[(size_t)r * max_m + o];
                    if (!SUB || first) d = acc;
                    else {
                        d.x += acc.x;
                        d.y += acc.y;
                    }
                }
            }
        }
    };
    // after step t: the cluster barrier, then the next input vector (and its stored slot) from the
    // exchange buffers out of every CTA of the cluster
    auto exchange = [&](int t, cx<T>* out) {
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
    };

    // first element of step t's rows ra.. of this CTA in U
    auto first = [&](int t, int ra) {
        const int i = fwd ? t : NK - 1 - t;
        return B.u_off + (long long)i * mmp + (long long)(r0 + ra) * m;
    };
    if constexpr (!SUB) {
        // all of a step's rows in one ring slot, issued STAGES - 1 steps ahead of use
        auto issue = [&](int t) {
            if (t < NK && nr > 0) fill(t % STAGES, first(t, 0), (long long)nr * m);
        };
        for (int t = 0; t < STAGES - 1; ++t) issue(t);
        __syncthreads();
        const int lg = split(fwd ? nr * c : m * c);
        for (int t = 0; t < NK; ++t) {
            issue(t + STAGES - 1);
            if (nr > 0) wait_fill(t);
            cx<T>* out = xb + (size_t)(t & 1) * xbs;
            compute(ust + (size_t)(t % STAGES) * SLOT + (nr > 0 ? sc_lead<T>(first(t, 0)) : 0), 0, nr, lg, true, out);
            exchange(t, out);
        }
    } else {
        // sub-blocks of RS rows, issued STAGES - 1 sub-blocks ahead of use
        const int nsb = nr > 0 ? (nr + RS - 1) / RS : 0;
        int it = 0, isb = 0;  // next sub-block to issue: step, index
        long long nfill = 0;  // fills issued (fill f goes to slot f % STAGES)
        auto issue = [&]() {
            if (nsb > 0 && it < NK) {
                const int ra = isb * RS, rn = min(RS, nr - ra);
                fill((int)(nfill % STAGES), first(it, ra), (long long)rn * m);
                ++nfill;
                if (++isb == nsb) {
                    isb = 0;
                    ++it;
                }
            }
        };
        for (int g = 0; g < STAGES - 1; ++g) issue();
        __syncthreads();
        const int rn_last = nr - (nsb - 1) * RS;
        const int lg_full = split(fwd ? RS * c : m * c), lg_last = split(fwd ? rn_last * c : m * c);
        long long cfill = 0;  // the fill in use
        for (int t = 0; t < NK; ++t) {
            cx<T>* out = xb + (size_t)(t & 1) * xbs;
            if (!fwd && nsb == 0)  // no rows: this CTA's partial sums are zero
                for (int e = tid; e < m * c; e += SC_THREADS) out[(size_t)(e / m) * max_m + e % m] = mk<T>(0, 0);
            for (int sb = 0; sb < nsb; ++sb) {
                issue();
                wait_fill(cfill);
                const bool last = sb + 1 == nsb;
                compute(ust + (size_t)(cfill % STAGES) * SLOT + sc_lead<T>(first(t, sb * RS)), sb * RS,
                        last ? rn_last : RS, last ? lg_last : lg_full, sb == 0, out);
                ++cfill;
                // the slot is refilled and out is extended by the next sub-block (after the last one of
                // the step the cluster barrier orders both)
                if (!last) __syncthreads();
            }
            exchange(t, out);
        }
    }
    // final vector (own range) to the boundary output
    cx<T>* fin = (fwd ? fwd_out : bwd_out) + B.v_off;
    for (int e = tid; e < nr * c; e += SC_THREADS) {
        const int r = e / nr, o = r0 + (e - r * nr);
        fin[(size_t)r * m + o] = x[(size_t)r * max_m + o];
    }
    cluster_sync_all();  // no CTA leaves while a peer may still read its exchange buffers
}

template <class T, int STAGES>
size_t sc_smem(int max_m, int max_c, int RS) {
    return ((size_t)STAGES * sc_slot<T>(RS, max_m) + 3 * (size_t)max_c * max_m) * sizeof(cx<T>);
}

constexpr size_t SC_SMEM_LIMIT = 220 * 1024;

// rows per ring slot: all of a CTA's rows when the ring holds them, else as many as fit (0: none)
template <class T, int STAGES>
int sc_rows_per_slot(int max_m, int max_c, int CL) {
    const int Rmax = (max_m + CL - 1) / CL;
    const size_t fixed = (3 * (size_t)max_c * max_m + (size_t)STAGES * 3) * sizeof(cx<T>);  // + slot slack
    if (fixed >= SC_SMEM_LIMIT) return 0;
    const size_t per_row = (size_t)STAGES * max_m * sizeof(cx<T>);
    const long long rs = (long long)((SC_SMEM_LIMIT - fixed) / per_row);
    return (int)std::min<long long>(Rmax, rs);
}

// Ring shape for a cluster of CL: 8 slots of all a CTA's rows when they fit (whole-row mode), else
// (large blocks) 4 slots of as many rows as fit (sub-block mode).  Returns the slots (0: the kernel
// does not fit) and the rows per slot.
template <class T>
int sc_shape(int max_m, int max_c, int CL, int* RS) {
    const int Rmax = (max_m + CL - 1) / CL;
    *RS = sc_rows_per_slot<T, 8>(max_m, max_c, CL);
    if (*RS == Rmax) return 8;
    *RS = sc_rows_per_slot<T, 4>(max_m, max_c, CL);
    return *RS >= 1 ? 4 : 0;
}

template <class T, int STAGES>
cudaLaunchConfig_t sc_config(int CL, int nchains, size_t sm, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nchains * CL));
    cfg.blockDim = dim3(SC_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class T, int STAGES, bool SUB>
int sc_launch(const DevPlan& P, const void* U, const void* fi, void* fo, const void* bi, void* bo, void* ps, void* ls,
              int dirs, int CL, int max_m, int max_c, int RS, int nchains, cudaStream_t st) {
    const size_t sm = sc_smem<T, STAGES>(max_m, max_c, RS);
    auto kern = sweep_cluster_kernel<T, STAGES, SUB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = sc_config<T, STAGES>(CL, nchains, sm, st, attr);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P, (const cx<T>*)U, (const cx<T>*)fi, (cx<T>*)fo,
                                             (const cx<T>*)bi, (cx<T>*)bo, (cx<T>*)ps, (cx<T>*)ls, dirs, CL, max_m,
                                             max_c, RS);
    return e == cudaSuccess ? 0 : -1;
}

// clusters of CL CTAs that the GPU holds at once (0 on error)
template <class T, int STAGES, bool SUB>
int sc_resident(int CL, int nchains, int max_m, int max_c, int RS) {
    const size_t sm = sc_smem<T, STAGES>(max_m, max_c, RS);
    auto kern = sweep_cluster_kernel<T, STAGES, SUB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = sc_config<T, STAGES>(CL, nchains, sm, 0, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class T>
int sc_resident_any(int CL, int nchains, int max_m, int max_c) {
    int RS = 0;
    const int S = sc_shape<T>(max_m, max_c, CL, &RS);
    if (S == 8) return sc_resident<T, 8, false>(CL, nchains, max_m, max_c, RS);
    if (S == 4) return sc_resident<T, 4, true>(CL, nchains, max_m, max_c, RS);
    return 0;
}

template <class T>
int sc_launch_any(const DevPlan& P, const void* U, const void* fi, void* fo, const void* bi, void* bo, void* ps,
                  void* ls, int dirs, int CL, int max_m, int max_c, int nchains, cudaStream_t st) {
    int RS = 0;
    const int S = sc_shape<T>(max_m, max_c, CL, &RS);
    if (S == 8) return sc_launch<T, 8, false>(P, U, fi, fo, bi, bo, ps, ls, dirs, CL, max_m, max_c, RS, nchains, st);
    if (S == 4) return sc_launch<T, 4, true>(P, U, fi, fo, bi, bo, ps, ls, dirs, CL, max_m, max_c, RS, nchains, st);
    return -1;
}

}  // namespace

int sweep_cluster_fits(int prec, int max_m, int max_c, int CL) {
    int RS = 0;
    return (prec == QOC_PREC_F64 ? sc_shape<double>(max_m, max_c, CL, &RS) : sc_shape<float>(max_m, max_c, CL, &RS)) > 0;
}

// Cluster size for the sweeps of a plan with nb active blocks (0: use the one-CTA-per-chain kernel).
// Every chain must find its cluster resident at once: chains x CL CTAs within the GPU's clusters.
// Sizes 8 down to 2 are tried (any size, so that e.g. 20 chains can take clusters of 7).
int sweep_cluster_size(int prec, int nb, int max_m, int max_c) {
    if (max_m < 24 || nb < 1) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chains = 2 * nb;
    for (int CL = 8; CL >= 2; --CL) {
        if (chains * CL > sms) continue;
        const int n = prec == QOC_PREC_F64 ? sc_resident_any<double>(CL, chains, max_m, max_c)
                                           : sc_resident_any<float>(CL, chains, max_m, max_c);
        if (n >= chains) return CL;
    }
    return 0;
}

int launch_sweeps_cluster(const DevPlan& P, const void* U, const void* fwd_init, void* fwd_out, const void* bwd_init,
                          void* bwd_out, void* psi_store, void* lam_store, int dirs, int max_m, int max_c, int CL,
                          cudaStream_t st) {
    const int nchains = ((dirs & 1) ? P.nb : 0) + ((dirs & 2) ? P.nb : 0);
    if (nchains == 0) return 0;
    if (P.prec == QOC_PREC_F64)
        return sc_launch_any<double>(P, U, fwd_init, fwd_out, bwd_init, bwd_out, psi_store, lam_store, dirs, CL, max_m,
                                     max_c, nchains, st);
    return sc_launch_any<float>(P, U, fwd_init, fwd_out, bwd_init, bwd_out, psi_store, lam_store, dirs, CL, max_m,
                                max_c, nchains, st);
}

}  // namespace qoc
