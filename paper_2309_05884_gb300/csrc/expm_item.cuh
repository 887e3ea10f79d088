// One (slice, block) item of the batched slice propagators U_kb = exp(-i tau (H0_b + sum_j u_kj Hc_jb))
// (Sec. II.A, Eq. exppropagator), shared by the tiled exponential kernel (expm.cu) and the persistent
// GRAPE-iteration kernel (persistent.cu).
//
// Scaling and squaring with a truncated Taylor polynomial of degree d evaluated by the
// Paterson-Stockmeyer scheme (d = p*q: p-1 products for X^2..X^p, then q-1 Horner products in
// X^p).  The norm bound beta = tau (|H0_b|_2 + sum_j |u_kj| |Hc_jb|_2) picks the number of
// squarings s and the smallest degree whose truncation bound beta_s^{d+1}/(d+1)! / (1 - beta_s/(d+2))
// stays below the working unit roundoff, beta_s = beta/2^s.  The polynomial runs in the working
// precision T (FP32 or FP64); the squaring chain runs in FP64 (or in T when tabs.sq_f64 is 0).  The
// item's matrices live in the calling CTA's scratch slot (expm_slot_bytes).
#pragma once

#include "gemm.cuh"
#include "kernels.h"

namespace qoc {
namespace {

__constant__ int c_deg_p[9] = {2, 2, 3, 3, 4, 4, 5, 5, 5};
__constant__ int c_deg_q[9] = {1, 2, 2, 3, 3, 4, 4, 5, 6};

// The shared-memory state of one item (the caller declares it, once per kernel or in a union).
template <class T, int R>
struct ExpmShared {
    static constexpr int RD = R > 4 ? 4 : R;  // FP64 squaring tile
    static constexpr size_t SMB = sizeof(GemmSmem<T, R>) > sizeof(GemmSmem<double, RD>) ? sizeof(GemmSmem<T, R>)
                                                                                         : sizeof(GemmSmem<double, RD>);
    __align__(16) unsigned char smraw[SMB];
    T coef[8];
    const cx<T>* pw[8];
    double s_if[32];  // 1/i!
    double s_uk[8];
    double s_scale;
    int s_sq, s_p, s_q;
};

// U_b[kw] (slot kw of block bi's propagator store) for slice k (0-based).  base: the CTA's scratch
// slot, laid out as X^1..X^5 at 1..5, Horner ping-pong at 6, 7, the FP64 squaring ping-pong after.
// Every thread of the CTA calls it; it ends with a barrier.
template <class T, int R>
__device__ void expm_item(const DevPlan& P, const ExpmTables& tabs, const double* __restrict__ u, int bi, int kw,
                          int k, void* __restrict__ Uout, cx<T>* base, size_t mm_max, ExpmShared<T, R>& sh) {
    constexpr int RD = ExpmShared<T, R>::RD;
    auto& sm = *reinterpret_cast<GemmSmem<T, R>*>(sh.smraw);
    auto& smd = *reinterpret_cast<GemmSmem<double, RD>*>(sh.smraw);
    cx<T>* S0 = base + 6 * mm_max;
    cx<T>* S1 = base + 7 * mm_max;
    double2* D0 = reinterpret_cast<double2*>(base + 8 * mm_max);
    double2* D1 = D0 + mm_max;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { sh.s_if[i] = f; f /= (double)(i + 1); }
    }
    if (threadIdx.x < 8) sh.pw[threadIdx.x] = base + (size_t)(threadIdx.x < 6 ? threadIdx.x : 0) * mm_max;
    const DevBlock& B = P.blocks[bi];
    const int m = B.m;
    const size_t mm = (size_t)m * m;

    if (threadIdx.x == 0) {
        double beta = B.h0_norm;
        int bad = 0;
        for (int j = 0; j < P.nc; ++j) {
            const double uk = u[(size_t)(B.u_row + k) * P.nc + j];
            const int fin = isfinite(uk);
            bad |= !fin;
            sh.s_uk[j] = fin ? uk : 0.0;
            beta += fabs(sh.s_uk[j]) * B.hc_norm[j];
        }
        if (bad) atomicOr(P.status, ST_NAN_PULSE);
        beta *= B.dt;
        int s = 0;
        while (beta > tabs.theta_cap && s < P.max_sq) { beta *= 0.5; ++s; }
        if (beta > tabs.theta_cap) atomicOr(P.status, ST_SQUARING_CAP);
        int di = 0;
        while (di < tabs.n_deg - 1 && tabs.theta[di] < beta) ++di;
        sh.s_sq = s;
        sh.s_p = c_deg_p[di];
        sh.s_q = c_deg_q[di];
        sh.s_scale = B.dt / (double)(1LL << s);
        if (P.stats) {
            const unsigned long long m3 = (unsigned long long)m * m * m;
            atomicAdd(P.stats + 0, m3 * (unsigned long long)(c_deg_p[di] + c_deg_q[di] - 2));
            atomicAdd(P.stats + 1, m3 * (unsigned long long)s);
            atomicAdd(P.stats + 2, 1ull);
        }
    }
    __syncthreads();
    const int s = sh.s_sq, p = sh.s_p, q = sh.s_q;
    const int d = p * q;

    // X = -i (tau / 2^s) (H0 + sum_j u_j Hc_j)
    {
        const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
        const T sc = (T)sh.s_scale;
        cx<T>* X = base + mm_max;
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            cx<T> h = H[e];
            for (int j = 0; j < P.nc; ++j) {
                const cx<T> hc = H[(size_t)(1 + j) * mm + e];
                const T uj = (T)sh.s_uk[j];
                h.x = fma(uj, hc.x, h.x);
                h.y = fma(uj, hc.y, h.y);
            }
            X[e] = cmul_mis<T>(h, sc);
        }
    }
    __syncthreads();
    // X^2 .. X^p
    for (int i = 2; i <= p; ++i)
        cta_gemm<T, R>(base + i * mm_max, base + (i - 1) * mm_max, base + mm_max, m, 0, nullptr, nullptr, sm);

    // Paterson-Stockmeyer: S = c_d X^p + sum_{l<p} c_{(q-1)p+l} X^l, then
    // S <- S X^p + sum_{l<p} c_{kb p + l} X^l for kb = q-2 .. 0  (c_i = 1/i!)
    cx<T>* S = S0;
    cx<T>* Sn = S1;
    {
        const T cd = (T)sh.s_if[d];
        const cx<T>* Xpp = base + p * mm_max;
        const int b0 = (q - 1) * p;
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
            cx<T> v = cscale<T>(Xpp[e], cd);
            if (row == col) v.x += (T)sh.s_if[b0];
            for (int l = 1; l < p; ++l) {
                const cx<T> xv = sh.pw[l][e];
                const T c = (T)sh.s_if[b0 + l];
                v.x = fma(c, xv.x, v.x);
                v.y = fma(c, xv.y, v.y);
            }
            S[e] = v;
        }
    }
    __syncthreads();
    for (int kb = q - 2; kb >= 0; --kb) {
        if (threadIdx.x < p) sh.coef[threadIdx.x] = (T)sh.s_if[kb * p + threadIdx.x];
        __syncthreads();
        cta_gemm<T, R>(Sn, S, base + p * mm_max, m, p, sh.coef, sh.pw, sm);
        cx<T>* t = S; S = Sn; Sn = t;
    }

    // s squarings in FP64, then store in the working precision
    cx<T>* Uo = reinterpret_cast<cx<T>*>(Uout) + B.u_off + (size_t)kw * B.mmp;
    if (s == 0) {
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Uo[e] = S[e];
    } else if (!tabs.sq_f64 && sizeof(T) == sizeof(float)) {
        // squaring chain in the working precision
        for (int i = 0; i < s; ++i) {
            cta_gemm<T, R>(Sn, S, S, m, 0, nullptr, nullptr, sm);
            cx<T>* t = S; S = Sn; Sn = t;
        }
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Uo[e] = S[e];
    } else {
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) D0[e] = ccast<double, T>(S[e]);
        __syncthreads();
        double2* Da = D0;
        double2* Db = D1;
        for (int i = 0; i < s; ++i) {
            cta_gemm<double, RD>(Db, Da, Da, m, 0, nullptr, nullptr, smd);
            double2* t = Da; Da = Db; Db = t;
        }
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Uo[e] = ccast<T, double>(Da[e]);
    }
    __syncthreads();
}

}  // namespace
}  // namespace qoc
