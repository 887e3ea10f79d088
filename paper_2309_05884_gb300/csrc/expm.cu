// Batched slice propagators U_kb = exp(-i tau (H0_b + sum_j u_kj Hc_jb))   (Sec. II.A, Eq. exppropagator)
//
// Scaling and squaring with a truncated Taylor polynomial of degree d evaluated by the
// Paterson-Stockmeyer scheme (d = p*q: p-1 products for X^2..X^p, then q-1 Horner products in
// X^p).  Per slice and block the norm bound beta = tau (|H0_b|_2 + sum_j |u_kj| |Hc_jb|_2) picks
// the number of squarings s and the smallest degree whose truncation bound
// beta_s^{d+1}/(d+1)! / (1 - beta_s/(d+2)) stays below the working unit roundoff, beta_s = beta/2^s.
// The polynomial runs in the working precision T (FP32 or FP64); the squaring chain always runs in
// FP64.  One CTA owns one (slice, block) item at a time and walks the item list persistently; its
// matrices live in a per-CTA scratch slot in global memory (L2-resident at these sizes).
#include "expm_item.cuh"

namespace qoc {

namespace {

template <class T, int R>
__global__ void __launch_bounds__(GEMM_THREADS)
expm_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks,
            int n_cls, const int2* __restrict__ cls_items, long long n_cls_items, void* __restrict__ Uout,
            char* __restrict__ scratch, size_t slot_bytes, int m_max, int skip_s0) {
    __shared__ ExpmShared<T, R> sh;

    // whole-problem launches walk the class's (block, slice) list; windowed launches (one problem,
    // checkpoint segments) index the window directly
    const bool whole = P.nk < 0;
    const int NK = P.nk;
    const long long total = whole ? n_cls_items : (long long)n_cls * NK;
    char* slot = scratch + (size_t)blockIdx.x * slot_bytes;
    const size_t mm_max = (size_t)m_max * m_max;
    cx<T>* base = reinterpret_cast<cx<T>*>(slot);

    __shared__ int s_list[GEMM_THREADS];
    __shared__ int s_nl;
    __shared__ int s_wc[32];
    // slices this launch owns: all of them, or (skip_s0) those that need squarings
    auto want = [&](long long it) -> bool {
        if (!skip_s0) return true;
        int bi;
        long long k;
        if (whole) {
            const int2 e = cls_items[it];
            bi = e.x;
            k = e.y;
        } else {
            bi = cls_blocks[it / NK];
            k = P.k0 + it % NK;
        }
        return slice_halvings(slice_beta(P, P.blocks[bi], u, k), tabs.theta_cap, P.max_sq) > 0;
    };
    for (long long lb = 0; cta_select(total, lb, want, s_list, &s_nl, s_wc); lb += blockDim.x) {
        const int nl = s_nl;
        for (int li = 0; li < nl; ++li) {
            const long long item = (long long)blockIdx.x + (lb + s_list[li]) * gridDim.x;
            int bi, kw, k;  // block, slot in the window, slice (0-based)
            if (whole) {
                const int2 it = cls_items[item];
                bi = it.x;
                kw = it.y;
                k = it.y;
            } else {
                bi = cls_blocks[item / NK];
                kw = (int)(item % NK);
                k = P.k0 + kw;
            }
            expm_item<T, R>(P, tabs, u, bi, kw, k, Uout, base, mm_max, sh);
        }
    }
}

template <class T, int R>
int launch_one(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
               const int2* items, long long n_items, void* Uout, char* scratch, size_t slot_bytes, int m_max,
               int grid, int skip_s0, cudaStream_t st) {
    expm_kernel<T, R><<<grid, GEMM_THREADS, 0, st>>>(P, tabs, u, cls, n_cls, items, n_items, Uout, scratch,
                                                     slot_bytes, m_max, skip_s0);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class T>
__global__ void export_u_kernel(DevPlan P, const cx<T>* __restrict__ U, double2* __restrict__ out,
                                const long long* __restrict__ a_off) {
    const int bi = blockIdx.y;
    const DevBlock& B = P.blocks[bi];
    const size_t mm = (size_t)B.m * B.m;
    const int nk = P.nk < 0 ? B.N : P.nk;
    const int k0 = P.nk < 0 ? 0 : P.k0;
    for (int k = blockIdx.x; k < nk; k += gridDim.x)
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x)
            out[a_off[bi] + (size_t)(k0 + k) * mm + e] = ccast<double, T>(U[B.u_off + (size_t)k * B.mmp + e]);
}

}  // namespace

int launch_export_u(const DevPlan& P, const void* U, double2* U_out, const long long* a_off, cudaStream_t st) {
    dim3 grid(256, P.nb);
    if (P.prec == 0)
        export_u_kernel<double><<<grid, 256, 0, st>>>(P, (const double2*)U, U_out, a_off);
    else
        export_u_kernel<float><<<grid, 256, 0, st>>>(P, (const float2*)U, U_out, a_off);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t expm_slot_bytes(int prec, int m_max) {
    const size_t mm = (size_t)m_max * m_max;
    const size_t el = prec == 0 ? 16 : 8;
    return 8 * mm * el + 2 * mm * 16 + 256;
}

int expm_r_for(int prec, int m) {
    const int rmax = prec == 0 ? 4 : 7;
    int r = (m + 15) / 16;
    return r < 1 ? 1 : (r > rmax ? rmax : r);
}

int expm_grid_limit(int prec, int R) {
    int dev = 0, sms = 0, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define QOC_OCC(TT, RR) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, expm_kernel<TT, RR>, GEMM_THREADS, 0)
    if (prec == 0) {
        switch (R) { case 1: QOC_OCC(double, 1); break; case 2: QOC_OCC(double, 2); break;
                     case 3: QOC_OCC(double, 3); break; default: QOC_OCC(double, 4); }
    } else {
        switch (R) { case 1: QOC_OCC(float, 1); break; case 2: QOC_OCC(float, 2); break;
                     case 3: QOC_OCC(float, 3); break; case 4: QOC_OCC(float, 4); break;
                     case 5: QOC_OCC(float, 5); break; case 6: QOC_OCC(float, 6); break;
                     default: QOC_OCC(float, 7); }
    }
#undef QOC_OCC
    if (occ < 1) occ = 1;
    return sms * occ;
}

int launch_expm(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                const int2* items, long long n_items, int R, void* Uout, char* scratch, size_t slot_bytes, int m_max,
                int grid, cudaStream_t st, int skip_s0) {
#define QOC_L(TT, RR) \
    launch_one<TT, RR>(P, tabs, u, cls, n_cls, items, n_items, Uout, scratch, slot_bytes, m_max, grid, skip_s0, st)
    if (P.prec == 0) {
        switch (R) {
            case 1: return QOC_L(double, 1);
            case 2: return QOC_L(double, 2);
            case 3: return QOC_L(double, 3);
            default: return QOC_L(double, 4);
        }
    }
    switch (R) {
        case 1: return QOC_L(float, 1);
        case 2: return QOC_L(float, 2);
        case 3: return QOC_L(float, 3);
        case 4: return QOC_L(float, 4);
        case 5: return QOC_L(float, 5);
        case 6: return QOC_L(float, 6);
        default: return QOC_L(float, 7);
    }
#undef QOC_L
}

}  // namespace qoc
