// Slice derivatives of large-norm slices by reverse-mode differentiation of the scaling-and-squaring
// propagator (Appendix B's slice derivative, exact for the computed U_k).
//
// For a slice whose 1-norm bound needs s >= 3 halvings the series of grad.cu would run 2^s
// sub-slices; here the propagator's own computation is differentiated instead.  With X = A/2^s the
// forward pass recomputes and keeps every intermediate
//     P_1 = X, P_l = P_{l-1} X (l <= p);  S_{q-1} = c_d P_p + sum_{l<p} c_{(q-1)p+l} P_l + c_{(q-1)p} I,
//     S_kb = S_{kb+1} P_p + B_kb(X);  Z_0 = S_0,  Z_{i+1} = Z_i^2,  U = Z_s,
// and the reverse pass carries Gbar = (dF-part / dM)^T from the seed Gbar_U = sum_r psi_r lam_r^dagger
// (psi: state at the slice start, lam: costate at its end; f = lam^dagger U psi is holomorphic in
// U, so the adjoint of C = A B is Gbar_A += B Gbar_C, Gbar_B += Gbar_C A):
//     squarings   Gbar_{Z_i} = Z_i Gbar_{Z_{i+1}} + Gbar_{Z_{i+1}} Z_i
//     Horner      Gbar_{S_{kb+1}} = P_p Gbar_{S_kb},  Gbar_{P_p} += Gbar_{S_kb} S_{kb+1},  Gbar_{P_l} += c Gbar_{S_kb}
//     powers      Gbar_{P_{l-1}} += X Gbar_{P_l},  Gbar_X += Gbar_{P_l} P_{l-1}
// and finally lam^dagger dU/du_j psi = -i (tau/2^s) tr(Gbar_X Hc_j).  One CTA per (slice, block) item,
// matrices in a per-CTA global scratch slot, products by the tiled CTA GEMM; items with s < 3 are
// left to the series kernel.
#include "gemm.cuh"
#include "kernels.h"

namespace qoc {
namespace {

__constant__ int r_deg_p[9] = {2, 2, 3, 3, 4, 4, 5, 5, 5};
__constant__ int r_deg_q[9] = {1, 2, 2, 3, 3, 4, 4, 5, 6};

constexpr int REV_MIN_S = 3;
constexpr int REV_MAX_P = 5, REV_MAX_Q = 6, REV_MAX_S = 16;
// slot: P_1..P_5 | S_1..S_5 (S_0 = Z_0) | Z_0..Z_15 | GP_1..GP_5 | G | T
constexpr int REV_MATS = REV_MAX_P + (REV_MAX_Q - 1) + REV_MAX_S + REV_MAX_P + 2;

template <class T, int R>
__global__ void __launch_bounds__(GEMM_THREADS)
grad_rev_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const cx<T>* __restrict__ psi_st,
                const cx<T>* __restrict__ lam_st, double2* __restrict__ partial, char* __restrict__ scratch,
                size_t slot_bytes, int m_max, const int* __restrict__ cls_blocks, int n_cls,
                const int2* __restrict__ cls_items, long long n_cls_items) {
    __shared__ GemmSmem<T, R> sm;
    __shared__ T coef[8];
    __shared__ const cx<T>* pw[8];
    __shared__ double s_if[32];
    __shared__ double s_uk[8];
    __shared__ int s_s, s_p, s_q;
    __shared__ double red[GEMM_THREADS / 32][8][2];

    const size_t MM = (size_t)m_max * m_max;
    cx<T>* base = reinterpret_cast<cx<T>*>(scratch + (size_t)blockIdx.x * slot_bytes);
    auto Pm = [&](int l) { return base + (size_t)(l - 1) * MM; };                          // P_1..P_5
    auto Sm = [&](int kb) { return base + (size_t)(REV_MAX_P + kb - 1) * MM; };           // S_1..S_5
    auto Zm = [&](int i) { return base + (size_t)(REV_MAX_P + REV_MAX_Q - 1 + i) * MM; }; // Z_0..
    auto GP = [&](int l) { return base + (size_t)(REV_MAX_P + REV_MAX_Q - 1 + REV_MAX_S + l - 1) * MM; };
    cx<T>* G = base + (size_t)(REV_MATS - 2) * MM;
    cx<T>* Tm = base + (size_t)(REV_MATS - 1) * MM;

    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { s_if[i] = f; f /= (double)(i + 1); }
    }
    // one launch per size class: the class's (block, slice) list, or its blocks' window slices
    const bool whole = P.nk < 0;
    const long long total = whole ? n_cls_items : (long long)P.nk * n_cls;
    const int nc = P.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

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
            const DevBlock& B = P.blocks[bi];
            const int m = B.m, c = B.c;
            const size_t mm = (size_t)m * m;
            if (threadIdx.x == 0) {
                double beta = B.h0_norm1;
                for (int j = 0; j < nc; ++j) {
                    const double x = u[(size_t)(B.u_row + k - 1) * nc + j];
                    s_uk[j] = isfinite(x) ? x : 0.0;
                    beta += fabs(s_uk[j]) * B.hc_norm1[j];
                }
                beta *= B.dt;
                int s = 0;
                while (beta > tabs.theta_cap && s < REV_MAX_S - 1) { beta *= 0.5; ++s; }
                int di = 0;
                while (di < tabs.n_deg - 1 && tabs.theta[di] < beta) ++di;
                s_s = s;
                s_p = r_deg_p[di];
                s_q = r_deg_q[di];
            }
            __syncthreads();
            const int s = s_s, p = s_p, q = s_q, d = p * q;
            const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
            const T sc = (T)(B.dt / (double)(1LL << s));
            // ---------------- forward: X, powers, Horner, squarings (all kept)
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                cx<T> h = H[e];
                for (int j = 0; j < nc; ++j) {
                    const cx<T> hc = H[(size_t)(1 + j) * mm + e];
                    const T uj = (T)s_uk[j];
                    h.x = fma(uj, hc.x, h.x);
                    h.y = fma(uj, hc.y, h.y);
                }
                Pm(1)[e] = cmul_mis<T>(h, sc);
            }
            if (threadIdx.x < 8) pw[threadIdx.x] = threadIdx.x >= 1 && threadIdx.x <= REV_MAX_P ? Pm(threadIdx.x) : Pm(1);
            __syncthreads();
            for (int l = 2; l <= p; ++l) cta_gemm<T, R>(Pm(l), Pm(l - 1), Pm(1), m, 0, nullptr, nullptr, sm);
            // S_{q-1} (stored in Z_0 when q == 1, else in S slot q-1)
            cx<T>* Stop = (q == 1) ? Zm(0) : Sm(q - 1);
            {
                const int b0 = (q - 1) * p;
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
                    cx<T> v = cscale<T>(Pm(p)[e], (T)s_if[d]);
                    if (row == col) v.x += (T)s_if[b0];
                    for (int l = 1; l < p; ++l) {
                        const cx<T> x = Pm(l)[e];
                        const T cf = (T)s_if[b0 + l];
                        v.x = fma(cf, x.x, v.x);
                        v.y = fma(cf, x.y, v.y);
                    }
                    Stop[e] = v;
                }
            }
            __syncthreads();
            for (int kb = q - 2; kb >= 0; --kb) {
                if (threadIdx.x < p) coef[threadIdx.x] = (T)s_if[kb * p + threadIdx.x];
                __syncthreads();
                cx<T>* dst = kb == 0 ? Zm(0) : Sm(kb);
                cta_gemm<T, R>(dst, Sm(kb + 1), Pm(p), m, p, coef, pw, sm);
            }
            for (int i = 0; i + 1 < s; ++i) cta_gemm<T, R>(Zm(i + 1), Zm(i), Zm(i), m, 0, nullptr, nullptr, sm);
            // Z_s = U is not needed by the reverse pass
            // ---------------- seed: Gbar_U = sum_r psi_r lam_r^dagger
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                const int a = (int)(e / m), b = (int)(e - (size_t)a * m);
                cx<T> v = mk<T>(0, 0);
                for (int r = 0; r < c; ++r) {
                    const cx<T> ps = psi_st[B.s_off + (long long)kw * c * m + (size_t)r * m + a];
                    const cx<T> la = lam_st[B.s_off + (long long)(kw + 1) * c * m + (size_t)r * m + b];
                    cfma_conj<T>(v, la, ps);  // psi[a] * conj(lam[b])
                }
                G[e] = v;
            }
            __syncthreads();
            // ---------------- reverse squarings: G <- Z_i G + G Z_i
            if (threadIdx.x == 0) { coef[0] = (T)0; coef[1] = (T)1; pw[1] = Tm; }
            __syncthreads();
            for (int i = s - 1; i >= 0; --i) {
                cta_gemm<T, R>(Tm, Zm(i), G, m, 0, nullptr, nullptr, sm);           // T = Z_i G
                cta_gemm<T, R>(i == 0 ? GP(1) : Zm(s), G, Zm(i), m, 2, coef, pw, sm);  // G Z_i + T
                // move the result into G (Zm(s) is free scratch; GP(1) is reused as scratch at i == 0)
                cx<T>* src = i == 0 ? GP(1) : Zm(s);
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) G[e] = src[e];
                __syncthreads();
            }
            // G is now Gbar_{S_0}.  Horner reverse.
            for (int l = 1; l <= p; ++l)
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) GP(l)[e] = mk<T>(0, 0);
            __syncthreads();
            if (threadIdx.x < 8) pw[threadIdx.x] = threadIdx.x >= 1 && threadIdx.x <= REV_MAX_P ? Pm(threadIdx.x) : Pm(1);
            __syncthreads();
            for (int kb = 0; kb <= q - 2; ++kb) {
                // S_kb = S_{kb+1} P_p + B_kb:  GP_l += c_{kb p + l} G (l = 1..p-1);  GP_p += G S_{kb+1};  G <- P_p G
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    const cx<T> g = G[e];
                    for (int l = 1; l < p; ++l) {
                        const T cf = (T)s_if[kb * p + l];
                        cx<T>& dst = GP(l)[e];
                        dst.x = fma(cf, g.x, dst.x);
                        dst.y = fma(cf, g.y, dst.y);
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) { coef[0] = (T)0; coef[1] = (T)1; pw[1] = GP(p); }
                __syncthreads();
                cta_gemm<T, R>(Tm, G, Sm(kb + 1), m, 2, coef, pw, sm);  // GP_p + G S_{kb+1}
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) GP(p)[e] = Tm[e];
                __syncthreads();
                cta_gemm<T, R>(Tm, Pm(p), G, m, 0, nullptr, nullptr, sm);  // P_p G
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) G[e] = Tm[e];
                __syncthreads();
            }
            // top: S_{q-1} = c_d P_p + sum_{l<p} c_{(q-1)p+l} P_l + c I
            {
                const int b0 = (q - 1) * p;
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    const cx<T> g = G[e];
                    for (int l = 1; l <= p; ++l) {
                        const T cf = (T)(l == p ? s_if[d] : s_if[b0 + l]);
                        cx<T>& dst = GP(l)[e];
                        dst.x = fma(cf, g.x, dst.x);
                        dst.y = fma(cf, g.y, dst.y);
                    }
                }
            }
            __syncthreads();
            // powers: P_l = P_{l-1} X, l = p..2:  GP_{l-1} += X GP_l ;  GX += GP_l P_{l-1};  GX accumulates in G
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) G[e] = mk<T>(0, 0);
            __syncthreads();
            for (int l = p; l >= 2; --l) {
                if (threadIdx.x == 0) { coef[0] = (T)0; coef[1] = (T)1; pw[1] = GP(l - 1); }
                __syncthreads();
                cta_gemm<T, R>(Tm, Pm(1), GP(l), m, 2, coef, pw, sm);  // GP_{l-1} + X GP_l
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) GP(l - 1)[e] = Tm[e];
                __syncthreads();
                if (threadIdx.x == 0) { pw[1] = G; }
                __syncthreads();
                cta_gemm<T, R>(Tm, GP(l), Pm(l - 1), m, 2, coef, pw, sm);  // GX + GP_l P_{l-1}
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) G[e] = Tm[e];
                __syncthreads();
            }
            // GX total = G + GP_1 ;  do_j = -i (tau/2^s) sum_{a,b} GX[a][b] Hc_j[b][a]
            T accr[8], acci[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) accr[j] = acci[j] = (T)0;
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                const int a = (int)(e / m), b = (int)(e - (size_t)a * m);
                const cx<T> gx = cadd<T>(G[e], GP(1)[e]);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j < nc) {
                        const cx<T> hc = H[(size_t)(1 + j) * mm + (size_t)b * m + a];
                        accr[j] = fma(gx.x, hc.x, fma(-gx.y, hc.y, accr[j]));
                        acci[j] = fma(gx.x, hc.y, fma(gx.y, hc.x, acci[j]));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= nc) break;
                double xr = (double)accr[j], xi = (double)acci[j];
                for (int off = 16; off > 0; off >>= 1) {
                    xr += __shfl_xor_sync(0xffffffffu, xr, off);
                    xi += __shfl_xor_sync(0xffffffffu, xi, off);
                }
                if (lane == 0) { red[warp][j][0] = xr; red[warp][j][1] = xi; }
            }
            __syncthreads();
            if ((int)threadIdx.x < nc) {
                double xr = 0.0, xi = 0.0;
                for (int w = 0; w < GEMM_THREADS / 32; ++w) { xr += red[w][threadIdx.x][0]; xi += red[w][threadIdx.x][1]; }
                const double ts = B.dt / (double)(1LL << s);
                double2 o;
                o.x = ts * xi;  // (-i ts)(xr + i xi)
                o.y = -ts * xr;
                partial[(size_t)(B.part_off + k - 1) * nc + threadIdx.x] = o;
            }
            __syncthreads();
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
