// Slice derivatives of large-norm slices by reverse-mode differentiation of the scaling-and-squaring
// propagator (Appendix B's slice derivative, exact for the computed U_k): one launch per size class,
// one CTA per (slice, block) item at a time; the item itself is rev_item (rev_item.cuh).
#include "rev_item.cuh"

namespace qoc {
namespace {


template <class T, int R>
__global__ void __launch_bounds__(GEMM_THREADS)
grad_rev_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const cx<T>* __restrict__ psi_st,
                const cx<T>* __restrict__ lam_st, double2* __restrict__ partial, char* __restrict__ scratch,
                size_t slot_bytes, int m_max, const int* __restrict__ cls_blocks, int n_cls,
                const int2* __restrict__ cls_items, long long n_cls_items) {
    __shared__ RevShared<T, R> sh;
    const size_t MM = (size_t)m_max * m_max;
    cx<T>* base = reinterpret_cast<cx<T>*>(scratch + (size_t)blockIdx.x * slot_bytes);

    // one launch per size class: the class's (block, slice) list, or its blocks' window slices
    const bool whole = P.nk < 0;
    const long long total = whole ? n_cls_items : (long long)P.nk * n_cls;

    __shared__ int s_list[GEMM_THREADS];
    __shared__ int s_nl;
    __shared__ int s_wc[32];
    // slices this launch owns: those whose exponential needs >= 2^REV_MIN_S squarings (exact mode)
    auto want = [&](long long it) -> bool {
        if (P.grad_mode != 0) return false;
        int bi;
        long long k;
        if (whole) {
            const int2 e = cls_items[it];
            bi = e.x;
            k = e.y;
        } else {
            bi = cls_blocks[it / P.nk];
            k = P.k0 + it % P.nk;
        }
        return slice_halvings(slice_beta(P, P.blocks[bi], u, k), tabs.theta_cap, REV_MAX_S - 1) >= REV_MIN_S;
    };
    for (long long lb = 0; cta_select(total, lb, want, s_list, &s_nl, s_wc); lb += blockDim.x) {
        const int nl = s_nl;
        for (int li = 0; li < nl; ++li) {
            const long long item = (long long)blockIdx.x + (lb + s_list[li]) * gridDim.x;
            int bi, kw, k;
            if (whole) {
                const int2 it = cls_items[item];
                bi = it.x;
                kw = it.y;
                k = it.y + 1;
            } else {
                bi = cls_blocks[item / P.nk];
                kw = (int)(item % P.nk);
                k = P.k0 + kw + 1;
            }
            rev_item<T, R>(P, tabs, u, psi_st, lam_st, partial, bi, kw, k, base, MM, sh);
        }
    }
}

template <class T, int R>
int launch_r(const DevPlan& P, const ExpmTables& tabs, const double* u, const void* psi, const void* lam,
             double2* partial, char* scratch, size_t slot, int m_max, int grid, const int* cls, int n_cls,
             const int2* items, long long n_items, cudaStream_t st) {
    grad_rev_kernel<T, R><<<grid, GEMM_THREADS, 0, st>>>(P, tabs, u, (const cx<T>*)psi, (const cx<T>*)lam, partial,
                                                         scratch, slot, m_max, cls, n_cls, items, n_items);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int grad_rev_min_s() { return REV_MIN_S; }

size_t grad_rev_slot_bytes(int prec, int m_max) {
    return (size_t)REV_MATS * m_max * m_max * (prec == 0 ? 16 : 8) + 256;
}

int grad_rev_tile(int prec, int m_max) {
    const int rmax = prec == 0 ? 4 : 5;
    int r = (m_max + 15) / 16;
    return r < 1 ? 1 : (r > rmax ? rmax : r);
}

int launch_grad_rev(const DevPlan& P, const ExpmTables& tabs, const double* u, const void* psi, const void* lam,
                    double2* partial, char* scratch, size_t slot, int m_max, int grid, const int* cls, int n_cls,
                    const int2* items, long long n_items, int class_m_max, cudaStream_t st) {
    const int R = grad_rev_tile(P.prec == 0 ? 0 : 1, class_m_max);
#define QOC_RL(TT, RR) launch_r<TT, RR>(P, tabs, u, psi, lam, partial, scratch, slot, m_max, grid, cls, n_cls, items, n_items, st)
    if (P.prec == 0) {
        switch (R) {
            case 1: return QOC_RL(double, 1);
            case 2: return QOC_RL(double, 2);
            case 3: return QOC_RL(double, 3);
            default: return QOC_RL(double, 4);
        }
    }
    switch (R) {
        case 1: return QOC_RL(float, 1);
        case 2: return QOC_RL(float, 2);
        case 3: return QOC_RL(float, 3);
        case 4: return QOC_RL(float, 4);
        default: return QOC_RL(float, 5);
    }
#undef QOC_RL
}

}  // namespace qoc
