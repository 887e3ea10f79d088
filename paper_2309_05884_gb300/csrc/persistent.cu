// One GRAPE iteration of every problem and block of an FP64 plan in a single persistent launch: F, the
// exact dF/du and the update of u (Sec. II.A, Eqs. exppropagator and probability; Appendix B).
//
// The grid is as large as can be resident at once (a cooperative launch), so CTAs may wait for one
// another: phases are separated by a grid barrier whose waits are bounded (2 s, then the status word
// gets the timeout bit and every CTA returns), and work inside a phase is handed out by an atomic
// queue, largest blocks first:
//   0  norm check of psi0 / psif per problem; boundary vectors gathered from the caller's states;
//   1  propagators U_kb, one (slice, block) item at a time (expm_item.cuh);
//   2  forward states psi_k = U_k psi_{k-1} and costates lam_{k-1} = U_k^dagger lam_k, one chain
//      (block, direction) per CTA, the vectors in shared memory;
//   3  overlap o_p and F_p per problem (FP64);
//   4  slice derivatives lam_k^dagger dU_k/du_kj psi_{k-1}, reverse mode through the computed U_k for
//      every item (rev_item.cuh);
//   5  dF/du = 2 Re(conj(o_p) sum_b ...), the update rule, the F history;
//   6  the iteration counter.
// CTA 0 records the global timer after each barrier, so the phase durations of a call can be read back.
#include "expm_item.cuh"
#include "rev_item.cuh"
#include "tma.cuh"

namespace qoc {
namespace {

constexpr int PK_THREADS = GEMM_THREADS;
constexpr uint64_t PK_WAIT_NS = 2000000000ull;  // 2 s per barrier

struct PkArgs {
    DevPlan P;
    ExpmTables tabs;
    double* u;                 // [rows][nc]: read by the iteration, updated by the rule at the end
    const double2* psi0;       // caller's block states
    const double2* psif;
    const int64_t* prob_state; // [n_prob][2] offset, length of each problem's block state
    double* out3;              // [n_prob][3]
    double2* o_ws;             // [n_prob]
    double2* partial;          // [sum_b N_b][nc]
    double* grad;              // [rows][nc] or null
    UpdateRule rule;
    double2* U;                // propagator store (slot k of block b at u_off + k mmp)
    double2* psi_st;           // [b][slot 0..N][copy][m]
    double2* lam_st;
    double2* fwd0;             // boundary vectors [b][copy][m]: psi_0, then psi_N in fwd1
    double2* fwd1;
    double2* bwd0;             // lam_N = psi_f, then lam_0 in bwd1
    double2* bwd1;
    char* scratch;             // per-CTA slots of slot_bytes
    size_t slot_bytes;
    int m_max;
    int want_grad;
    unsigned* sync;            // [0] barrier arrivals, [1..3] work queues (zero before the launch)
    unsigned long long* ts;    // [8] global timer after each phase (CTA 0)
};

__device__ __forceinline__ int pk_tile(int m) {
    const int r = (m + 15) / 16;
    return r < 1 ? 1 : (r > 4 ? 4 : r);
}

// Grid barrier number idx (1-based): every CTA arrives once, then waits (bounded) for all of them.
__device__ bool pk_barrier(unsigned* arrive, unsigned idx, int* status, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(arrive, 1u);
        const unsigned target = idx * gridDim.x;
        const uint64_t t0 = globaltimer_ns();
        int ok = 1;
        while (atomicAdd(arrive, 0u) < target) {
            if (globaltimer_ns() - t0 > PK_WAIT_NS) {
                ok = 0;
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Next item of a work queue for the whole CTA (total items), or -1.
__device__ long long pk_next(unsigned* head, long long total, long long* s_item) {
    if (threadIdx.x == 0) *s_item = (long long)atomicAdd(head, 1u);
    __syncthreads();
    const long long it = *s_item;
    __syncthreads();
    return it < total ? it : -1;
}

__device__ void pk_stamp(const PkArgs& a, int i) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ts[i] = globaltimer_ns();
}

// y_r = op(U) x_r for the c copies of one block (op = U or U^dagger), vectors in shared memory.  G
// threads share an output element (a power of two with G * m <= blockDim).
__device__ void pk_gemv(const double2* __restrict__ U, const double2* x, double2* y, int m, int c, bool adjoint) {
    int G = 1;
    while (G < 32 && G * 2 * m <= (int)blockDim.x) G *= 2;
    const int outs = blockDim.x / G, part = threadIdx.x % G;
    for (int o0 = 0; o0 < m * c; o0 += outs) {
        const int o = o0 + threadIdx.x / G;
        double2 acc = make_double2(0.0, 0.0);
        const int r = o / m, a = o - r * m;
        if (o < m * c) {
            const double2* xr = x + (size_t)r * m;
            if (!adjoint) {
                const double2* row = U + (size_t)a * m;
                for (int b = part; b < m; b += G) cfma<double>(acc, row[b], xr[b]);
            } else {
                for (int b = part; b < m; b += G) cfma_conj<double>(acc, U[(size_t)b * m + a], xr[b]);
            }
        }
        for (int off = G / 2; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (o < m * c && part == 0) y[o] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PK_THREADS, 1) persistent_kernel(PkArgs a) {
    extern __shared__ __align__(16) unsigned char pk_sm[];
    __shared__ int s_ok;
    __shared__ long long s_item;
    __shared__ double sred[PK_THREADS][2];
    const DevPlan& P = a.P;
    int* status = P.status;
    unsigned bar = 0;
    pk_stamp(a, 0);

    // ---- phase 0: norms and gathers
    for (int p = blockIdx.x; p < P.n_prob; p += gridDim.x) {
        const int64_t off = a.prob_state[2 * p], len = a.prob_state[2 * p + 1];
        double n0 = 0.0, nf = 0.0;
        for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
            const double2 x = a.psi0[off + e], y = a.psif[off + e];
            n0 = fma(x.x, x.x, fma(x.y, x.y, n0));
            nf = fma(y.x, y.x, fma(y.y, y.y, nf));
        }
        sred[threadIdx.x][0] = n0;
        sred[threadIdx.x][1] = nf;
        __syncthreads();
        for (int s = PK_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                sred[threadIdx.x][0] += sred[threadIdx.x + s][0];
                sred[threadIdx.x][1] += sred[threadIdx.x + s][1];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && !(fabs(sqrt(sred[0][0]) - 1.0) <= 1e-8 && fabs(sqrt(sred[0][1]) - 1.0) <= 1e-8))
            atomicOr(status, ST_NORM);
        __syncthreads();
    }
    for (int bi = blockIdx.x; bi < P.nb; bi += gridDim.x) {
        const DevBlock& B = P.blocks[bi];
        const long long cb = P.copy_base[bi];
        for (int e = threadIdx.x; e < B.m * B.c; e += blockDim.x) {
            const int r = e / B.m, i = e - r * B.m;
            a.fwd0[B.v_off + e] = a.psi0[P.copy_src[cb + r] + i];
            a.bwd0[B.v_off + e] = a.psif[P.copy_src[cb + r] + i];
        }
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 1);

    // ---- phase 1: propagators
    {
        const size_t MM = (size_t)a.m_max * a.m_max;
        double2* base = reinterpret_cast<double2*>(a.scratch + (size_t)blockIdx.x * a.slot_bytes);
        for (long long it; (it = pk_next(a.sync + 1, P.n_items, &s_item)) >= 0;) {
            const int2 e = P.items[it];  // (block, slice), largest blocks first
            const int R = pk_tile(P.blocks[e.x].m);
            switch (R) {
                case 1: expm_item<double, 1>(P, a.tabs, a.u, e.x, e.y, e.y, a.U, base, MM, *reinterpret_cast<ExpmShared<double, 1>*>(pk_sm)); break;
                case 2: expm_item<double, 2>(P, a.tabs, a.u, e.x, e.y, e.y, a.U, base, MM, *reinterpret_cast<ExpmShared<double, 2>*>(pk_sm)); break;
                case 3: expm_item<double, 3>(P, a.tabs, a.u, e.x, e.y, e.y, a.U, base, MM, *reinterpret_cast<ExpmShared<double, 3>*>(pk_sm)); break;
                default: expm_item<double, 4>(P, a.tabs, a.u, e.x, e.y, e.y, a.U, base, MM, *reinterpret_cast<ExpmShared<double, 4>*>(pk_sm)); break;
            }
        }
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 2);

    // ---- phase 2: sweeps, one chain (block, direction) at a time
    {
        const int nchains = a.want_grad ? 2 * P.nb : P.nb;
        for (long long ch; (ch = pk_next(a.sync + 2, nchains, &s_item)) >= 0;) {
            const bool fwd = ch < P.nb;
            const int bi = (int)(fwd ? ch : ch - P.nb);
            const DevBlock& B = P.blocks[bi];
            const int m = B.m, c = B.c, n = m * c;
            double2* x = reinterpret_cast<double2*>(pk_sm);
            double2* y = x + n;
            double2* st = fwd ? a.psi_st : a.lam_st;
            const double2* init = fwd ? a.fwd0 : a.bwd0;
            for (int e = threadIdx.x; e < n; e += blockDim.x) {
                x[e] = init[B.v_off + e];
                st[B.s_off + (long long)(fwd ? 0 : B.N) * n + e] = x[e];
            }
            __syncthreads();
            for (int step = 0; step < B.N; ++step) {
                const int k = fwd ? step : B.N - 1 - step;  // slice k (0-based): U at slot k
                pk_gemv(a.U + B.u_off + (size_t)k * B.mmp, x, y, m, c, !fwd);
                const long long slot = fwd ? k + 1 : k;
                for (int e = threadIdx.x; e < n; e += blockDim.x) {
                    x[e] = y[e];
                    st[B.s_off + slot * n + e] = y[e];
                }
                __syncthreads();
            }
            double2* outb = fwd ? a.fwd1 : a.bwd1;
            for (int e = threadIdx.x; e < n; e += blockDim.x) outb[B.v_off + e] = x[e];
            __syncthreads();
        }
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 3);

    // ---- phase 3: overlaps
    for (int p = blockIdx.x; p < P.n_prob; p += gridDim.x) {
        double re = 0.0, im = 0.0;
        for (int t = P.prob_block_off[p]; t < P.prob_block_off[p + 1]; ++t) {
            const int bi = P.prob_blocks[t];
            const DevBlock& B = P.blocks[bi];
            const long long cb = P.copy_base[bi];
            for (int e = threadIdx.x; e < B.m * B.c; e += blockDim.x) {
                const int r = e / B.m, i = e - r * B.m;
                const double2 f = a.psif[P.copy_src[cb + r] + i], pn = a.fwd1[B.v_off + e];
                re += f.x * pn.x + f.y * pn.y;
                im += f.x * pn.y - f.y * pn.x;
            }
        }
        sred[threadIdx.x][0] = re;
        sred[threadIdx.x][1] = im;
        __syncthreads();
        for (int s = PK_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                sred[threadIdx.x][0] += sred[threadIdx.x + s][0];
                sred[threadIdx.x][1] += sred[threadIdx.x + s][1];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double x = sred[0][0], z = sred[0][1];
            a.out3[3 * p + 0] = x * x + z * z;
            a.out3[3 * p + 1] = x;
            a.out3[3 * p + 2] = z;
            a.o_ws[p] = make_double2(x, z);
        }
        __syncthreads();
    }
    if (!a.want_grad) {
        pk_stamp(a, 4);
        pk_stamp(a, 5);
        pk_stamp(a, 6);
        return;
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 4);

    // ---- phase 4: slice derivatives (reverse mode through each computed U_k)
    {
        const size_t MM = (size_t)a.m_max * a.m_max;
        double2* base = reinterpret_cast<double2*>(a.scratch + (size_t)blockIdx.x * a.slot_bytes);
        for (long long it; (it = pk_next(a.sync + 3, P.n_items, &s_item)) >= 0;) {
            const int2 e = P.items[it];
            const int R = pk_tile(P.blocks[e.x].m);
            switch (R) {
                case 1: rev_item<double, 1>(P, a.tabs, a.u, a.psi_st, a.lam_st, a.partial, e.x, e.y, e.y + 1, base, MM, *reinterpret_cast<RevShared<double, 1>*>(pk_sm)); break;
                case 2: rev_item<double, 2>(P, a.tabs, a.u, a.psi_st, a.lam_st, a.partial, e.x, e.y, e.y + 1, base, MM, *reinterpret_cast<RevShared<double, 2>*>(pk_sm)); break;
                case 3: rev_item<double, 3>(P, a.tabs, a.u, a.psi_st, a.lam_st, a.partial, e.x, e.y, e.y + 1, base, MM, *reinterpret_cast<RevShared<double, 3>*>(pk_sm)); break;
                default: rev_item<double, 4>(P, a.tabs, a.u, a.psi_st, a.lam_st, a.partial, e.x, e.y, e.y + 1, base, MM, *reinterpret_cast<RevShared<double, 4>*>(pk_sm)); break;
            }
        }
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 5);

    // ---- phase 5: gradient, update rule, F history (the reduction of grad.cu, grid-stride)
    {
        const UpdateRule& rule = a.rule;
        const int nc = P.nc;
        const int it = rule.iter ? *rule.iter : 0;
        const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
        for (int p = 0; p < P.n_prob; ++p) {
            const int t0 = P.prob_block_off[p], t1 = P.prob_block_off[p + 1];
            const DevBlock& B0 = P.blocks[P.prob_blocks[t0]];
            const double2 o = a.o_ws[p];
            const double Fp = a.out3[3 * p];
            const bool reached_now = Fp >= rule.f_target;
            const bool frozen = rule.freeze && (reached_now || (rule.reached && rule.reached[p] >= 0));
            const double sc = rule.gscale ? rule.gscale[p] : 1.0;
            for (long long e = gt; e < (long long)B0.N * nc; e += gs) {
                const int k = (int)(e / nc), j = (int)(e - (long long)k * nc);
                double sr = 0.0, si = 0.0;
                for (int t = t0; t < t1; ++t) {
                    const DevBlock& B = P.blocks[P.prob_blocks[t]];
                    const double2 d = a.partial[(size_t)(B.part_off + k) * nc + j];
                    sr += d.x;
                    si += d.y;
                }
                const double gv = 2.0 * (o.x * sr + o.y * si) * sc;
                const size_t idx = (size_t)B0.u_row * nc + e;
                if (a.grad) a.grad[idx] = gv;
                if (rule.kind >= 0 && !frozen) {
                    if (rule.kind == 0) {
                        a.u[idx] += rule.step * gv;
                    } else {
                        const double mm1 = rule.beta1 * rule.adam_m[idx] + (1.0 - rule.beta1) * gv;
                        const double vv = rule.beta2 * rule.adam_v[idx] + (1.0 - rule.beta2) * gv * gv;
                        rule.adam_m[idx] = mm1;
                        rule.adam_v[idx] = vv;
                        const double mh = mm1 / (1.0 - pow(rule.beta1, it + 1));
                        const double vh = vv / (1.0 - pow(rule.beta2, it + 1));
                        a.u[idx] += rule.step * mh / (sqrt(vh) + rule.eps);
                    }
                }
            }
            if (gt == 0) {
                if (rule.F_hist) rule.F_hist[(size_t)it * P.n_prob + p] = Fp;
                if (rule.reached && reached_now && rule.reached[p] < 0) rule.reached[p] = it;
            }
        }
    }
    if (!pk_barrier(a.sync, ++bar, status, &s_ok)) return;
    pk_stamp(a, 6);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.rule.iter) *a.rule.iter += 1;
}

}  // namespace

// Grid (CTAs resident at once), per-CTA scratch slot and dynamic shared memory of the persistent
// kernel for blocks up to max_m with up to max_c copies; 0 if it cannot run (shared memory).
int persistent_config(int max_m, int max_c, int* grid, size_t* slot, size_t* smem) {
    size_t sh = sizeof(RevShared<double, 4>);
    sh = sh > sizeof(ExpmShared<double, 4>) ? sh : sizeof(ExpmShared<double, 4>);
    const size_t vec = 2 * (size_t)max_m * max_c * sizeof(double2);
    sh = sh > vec ? sh : vec;
    if (sh > 200 * 1024) return 0;
    if (cudaFuncSetAttribute(persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess)
        return 0;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_kernel, PK_THREADS, sh) != cudaSuccess || occ < 1)
        return 0;
    *grid = sms * occ;
    const size_t mm = (size_t)max_m * max_m;
    const size_t es = 8 * mm * 16 + 2 * mm * 16 + 256, rs = (size_t)REV_MATS * mm * 16 + 256;
    *slot = ((es > rs ? es : rs) + 255) / 256 * 256;
    *smem = sh;
    return 1;
}

int launch_persistent(const DevPlan& P, const ExpmTables& tabs, double* u, const double2* psi0, const double2* psif,
                      const int64_t* prob_state, double* out3, double2* o_ws, double2* partial, double* grad,
                      const UpdateRule& rule, void* U, void* psi_st, void* lam_st, void* fwd0, void* fwd1, void* bwd0,
                      void* bwd1, char* scratch, size_t slot_bytes, int m_max, int want_grad, unsigned* sync,
                      unsigned long long* ts, int grid, size_t smem, cudaStream_t st) {
    if (cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned), st) != cudaSuccess) return -1;
    PkArgs a;
    a.P = P;
    a.tabs = tabs;
    a.u = u;
    a.psi0 = psi0;
    a.psif = psif;
    a.prob_state = prob_state;
    a.out3 = out3;
    a.o_ws = o_ws;
    a.partial = partial;
    a.grad = grad;
    a.rule = rule;
    a.U = reinterpret_cast<double2*>(U);
    a.psi_st = reinterpret_cast<double2*>(psi_st);
    a.lam_st = reinterpret_cast<double2*>(lam_st);
    a.fwd0 = reinterpret_cast<double2*>(fwd0);
    a.fwd1 = reinterpret_cast<double2*>(fwd1);
    a.bwd0 = reinterpret_cast<double2*>(bwd0);
    a.bwd1 = reinterpret_cast<double2*>(bwd1);
    a.scratch = scratch;
    a.slot_bytes = slot_bytes;
    a.m_max = m_max;
    a.want_grad = want_grad;
    a.sync = sync;
    a.ts = ts;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PK_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, persistent_kernel, a) == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
