// One (slice, block) item of the slice derivatives by reverse-mode differentiation of the scaling-and-squaring
// propagator (Appendix B's slice derivative, exact for the computed U_k).
//
// For a slice whose norm bound needs s >= 3 halvings the series of grad.cu would run 2^s
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
// matrices in a per-CTA global scratch slot, products by the tiled CTA GEMM.  The computation is exact
// for the computed U_k at any s; the reverse-mode kernel (grad_rev.cu) takes the items with s >= 3
// (the series kernels take the others), the persistent GRAPE-iteration kernel (persistent.cu) every
// item.
#pragma once

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
struct RevShared {
    GemmSmem<T, R> sm;
    T coef[8];
    const cx<T>* pw[8];
    double s_if[32];
    double s_uk[8];
    int s_s, s_p, s_q;
    double red[GEMM_THREADS / 32][8][2];
};

// partial[(part_off + k - 1) nc + j] = lam_k^dagger dU_k/du_kj psi_{k-1} (summed over copies) for slice k
// (1-based) of block bi, window slot kw (psi_{k-1} in state slot kw, lam_k in slot kw + 1).  base: the
// CTA's scratch slot of REV_MATS m_max^2 matrices.  Every thread of the CTA calls it; it ends with a
// barrier.
template <class T, int R>
__device__ void rev_item(const DevPlan& P, const ExpmTables& tabs, const double* __restrict__ u,
                         const cx<T>* __restrict__ psi_st, const cx<T>* __restrict__ lam_st,
                         double2* __restrict__ partial, int bi, int kw, int k, cx<T>* base, size_t MM,
                         RevShared<T, R>& sh) {
    auto& sm = sh.sm;
    const int nc = P.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto Pm = [&](int l) { return base + (size_t)(l - 1) * MM; };                          // P_1..P_5
    auto Sm = [&](int kb) { return base + (size_t)(REV_MAX_P + kb - 1) * MM; };           // S_1..S_5
    auto Zm = [&](int i) { return base + (size_t)(REV_MAX_P + REV_MAX_Q - 1 + i) * MM; }; // Z_0..
    auto GP = [&](int l) { return base + (size_t)(REV_MAX_P + REV_MAX_Q - 1 + REV_MAX_S + l - 1) * MM; };
    cx<T>* G = base + (size_t)(REV_MATS - 2) * MM;
    cx<T>* Tm = base + (size_t)(REV_MATS - 1) * MM;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { sh.s_if[i] = f; f /= (double)(i + 1); }
    }
    const DevBlock& B = P.blocks[bi];
    const int m = B.m, c = B.c;
    const size_t mm = (size_t)m * m;
    if (threadIdx.x == 0) {
        double beta = B.h0_norm;
        for (int j = 0; j < nc; ++j) {
            const double x = u[(size_t)(B.u_row + k - 1) * nc + j];
            sh.s_uk[j] = isfinite(x) ? x : 0.0;
            beta += fabs(sh.s_uk[j]) * B.hc_norm[j];
        }
        beta *= B.dt;
        int s = 0;
        while (beta > tabs.theta_cap && s < REV_MAX_S - 1) { beta *= 0.5; ++s; }
        int di = 0;
        while (di < tabs.n_deg - 1 && tabs.theta[di] < beta) ++di;
        sh.s_s = s;
        sh.s_p = r_deg_p[di];
        sh.s_q = r_deg_q[di];
    }
    __syncthreads();
    const int s = sh.s_s, p = sh.s_p, q = sh.s_q, d = p * q;
    const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
    const T sc = (T)(B.dt / (double)(1LL << s));
    // ---------------- forward: X, powers, Horner, squarings (all kept)
    for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
        cx<T> h = H[e];
        for (int j = 0; j < nc; ++j) {
            const cx<T> hc = H[(size_t)(1 + j) * mm + e];
            const T uj = (T)sh.s_uk[j];
            h.x = fma(uj, hc.x, h.x);
            h.y = fma(uj, hc.y, h.y);
        }
        Pm(1)[e] = cmul_mis<T>(h, sc);
    }
    if (threadIdx.x < 8) sh.pw[threadIdx.x] = threadIdx.x >= 1 && threadIdx.x <= REV_MAX_P ? Pm(threadIdx.x) : Pm(1);
    __syncthreads();
    for (int l = 2; l <= p; ++l) cta_gemm<T, R>(Pm(l), Pm(l - 1), Pm(1), m, 0, nullptr, nullptr, sm);
    // S_{q-1} (stored in Z_0 when q == 1, else in S slot q-1)
    cx<T>* Stop = (q == 1) ? Zm(0) : Sm(q - 1);
    {
        const int b0 = (q - 1) * p;
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
            cx<T> v = cscale<T>(Pm(p)[e], (T)sh.s_if[d]);
            if (row == col) v.x += (T)sh.s_if[b0];
            for (int l = 1; l < p; ++l) {
                const cx<T> x = Pm(l)[e];
                const T cf = (T)sh.s_if[b0 + l];
                v.x = fma(cf, x.x, v.x);
                v.y = fma(cf, x.y, v.y);
            }
            Stop[e] = v;
        }
    }
    __syncthreads();
    for (int kb = q - 2; kb >= 0; --kb) {
        if (threadIdx.x < p) sh.coef[threadIdx.x] = (T)sh.s_if[kb * p + threadIdx.x];
        __syncthreads();
        cx<T>* dst = kb == 0 ? Zm(0) : Sm(kb);
        cta_gemm<T, R>(dst, Sm(kb + 1), Pm(p), m, p, sh.coef, sh.pw, sm);
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
    if (threadIdx.x == 0) { sh.coef[0] = (T)0; sh.coef[1] = (T)1; sh.pw[1] = Tm; }
    __syncthreads();
    for (int i = s - 1; i >= 0; --i) {
        cta_gemm<T, R>(Tm, Zm(i), G, m, 0, nullptr, nullptr, sm);           // T = Z_i G
        cta_gemm<T, R>(i == 0 ? GP(1) : Zm(s), G, Zm(i), m, 2, sh.coef, sh.pw, sm);  // G Z_i + T
        // move the result into G (Zm(s) is free scratch; GP(1) is reused as scratch at i == 0)
        cx<T>* src = i == 0 ? GP(1) : Zm(s);
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) G[e] = src[e];
        __syncthreads();
    }
    // G is now Gbar_{S_0}.  Horner reverse.
    for (int l = 1; l <= p; ++l)
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) GP(l)[e] = mk<T>(0, 0);
    __syncthreads();
    if (threadIdx.x < 8) sh.pw[threadIdx.x] = threadIdx.x >= 1 && threadIdx.x <= REV_MAX_P ? Pm(threadIdx.x) : Pm(1);
    __syncthreads();
    for (int kb = 0; kb <= q - 2; ++kb) {
        // S_kb = S_{kb+1} P_p + B_kb:  GP_l += c_{kb p + l} G (l = 1..p-1);  GP_p += G S_{kb+1};  G <- P_p G
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            const cx<T> g = G[e];
            for (int l = 1; l < p; ++l) {
                const T cf = (T)sh.s_if[kb * p + l];
                cx<T>& dst = GP(l)[e];
                dst.x = fma(cf, g.x, dst.x);
                dst.y = fma(cf, g.y, dst.y);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) { sh.coef[0] = (T)0; sh.coef[1] = (T)1; sh.pw[1] = GP(p); }
        __syncthreads();
        cta_gemm<T, R>(Tm, G, Sm(kb + 1), m, 2, sh.coef, sh.pw, sm);  // GP_p + G S_{kb+1}
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
                const T cf = (T)(l == p ? sh.s_if[d] : sh.s_if[b0 + l]);
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
        if (threadIdx.x == 0) { sh.coef[0] = (T)0; sh.coef[1] = (T)1; sh.pw[1] = GP(l - 1); }
        __syncthreads();
        cta_gemm<T, R>(Tm, Pm(1), GP(l), m, 2, sh.coef, sh.pw, sm);  // GP_{l-1} + X GP_l
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) GP(l - 1)[e] = Tm[e];
        __syncthreads();
        if (threadIdx.x == 0) { sh.pw[1] = G; }
        __syncthreads();
        cta_gemm<T, R>(Tm, GP(l), Pm(l - 1), m, 2, sh.coef, sh.pw, sm);  // GX + GP_l P_{l-1}
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
        if (lane == 0) { sh.red[warp][j][0] = xr; sh.red[warp][j][1] = xi; }
    }
    __syncthreads();
    if ((int)threadIdx.x < nc) {
        double xr = 0.0, xi = 0.0;
        for (int w = 0; w < GEMM_THREADS / 32; ++w) { xr += sh.red[w][threadIdx.x][0]; xi += sh.red[w][threadIdx.x][1]; }
        const double ts = B.dt / (double)(1LL << s);
        double2 o;
        o.x = ts * xi;  // (-i ts)(xr + i xi)
        o.y = -ts * xr;
        partial[(size_t)(B.part_off + k - 1) * nc + threadIdx.x] = o;
    }
    __syncthreads();
}

}  // namespace
}  // namespace qoc
