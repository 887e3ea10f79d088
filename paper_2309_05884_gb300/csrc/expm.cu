// Batched slice propagators U_kb = exp(-i tau (H0_b + sum_j u_kj Hc_jb))   (Sec. II.A, Eq. exppropagator)
//
// Scaling and squaring with a truncated Taylor polynomial of degree d evaluated by the
// Paterson-Stockmeyer scheme (d = p*q: p-1 products for X^2..X^p, then q-1 Horner products in
// X^p).  Per slice and block the 1-norm bound beta = tau (|H0_b|_1 + sum_j |u_kj| |Hc_jb|_1) picks
// the number of squarings s and the smallest degree whose truncation bound
// beta_s^{d+1}/(d+1)! / (1 - beta_s/(d+2)) stays below the working unit roundoff, beta_s = beta/2^s.
// The polynomial runs in the working precision T (FP32 or FP64); the squaring chain always runs in
// FP64.  One CTA owns one (slice, block) item at a time and walks the item list persistently; its
// matrices live in a per-CTA scratch slot in global memory (L2-resident at these sizes).
#include "gemm.cuh"
#include "kernels.h"

namespace qoc {

namespace {

__constant__ int c_deg_p[9] = {2, 2, 3, 3, 4, 4, 5, 5, 5};
__constant__ int c_deg_q[9] = {1, 2, 2, 3, 3, 4, 4, 5, 6};

template <class T, int R>
__global__ void __launch_bounds__(GEMM_THREADS)
expm_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks,
            int n_cls, const int2* __restrict__ cls_items, long long n_cls_items, void* __restrict__ Uout,
            char* __restrict__ scratch, size_t slot_bytes, int m_max, int skip_s0) {
    constexpr int RD = R > 4 ? 4 : R;  // FP64 squaring tile
    constexpr size_t SMB = sizeof(GemmSmem<T, R>) > sizeof(GemmSmem<double, RD>) ? sizeof(GemmSmem<T, R>)
                                                                                   : sizeof(GemmSmem<double, RD>);
    __shared__ __align__(16) unsigned char smraw[SMB];
    auto& sm = *reinterpret_cast<GemmSmem<T, R>*>(smraw);
    auto& smd = *reinterpret_cast<GemmSmem<double, RD>*>(smraw);
    __shared__ T coef[8];
    __shared__ const cx<T>* pw[8];
    __shared__ double s_if[32];   // 1/i!
    __shared__ double s_uk[8];
    __shared__ double s_scale;
    __shared__ int s_sq, s_p, s_q;

    // whole-problem launches walk the class's (block, slice) list; windowed launches (one problem,
    // checkpoint segments) index the window directly
    const bool whole = P.nk < 0;
    const int NK = P.nk;
    const long long total = whole ? n_cls_items : (long long)n_cls * NK;
    char* slot = scratch + (size_t)blockIdx.x * slot_bytes;
    const size_t mm_max = (size_t)m_max * m_max;
    cx<T>* base = reinterpret_cast<cx<T>*>(slot);
    // slot layout: X^1..X^5 at 1..5, Horner ping-pong at 6, 7, FP64 squaring ping-pong after
    cx<T>* S0 = base + 6 * mm_max;
    cx<T>* S1 = base + 7 * mm_max;
    double2* D0 = reinterpret_cast<double2*>(base + 8 * mm_max);
    double2* D1 = D0 + mm_max;

    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { s_if[i] = f; f /= (double)(i + 1); }
    }
    if (threadIdx.x < 8) pw[threadIdx.x] = base + (size_t)(threadIdx.x < 6 ? threadIdx.x : 0) * mm_max;

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
            const DevBlock& B = P.blocks[bi];
            const int m = B.m;
            const size_t mm = (size_t)m * m;

            if (threadIdx.x == 0) {
                double beta = B.h0_norm1;
                int bad = 0;
                for (int j = 0; j < P.nc; ++j) {
                    const double uk = u[(size_t)(B.u_row + k) * P.nc + j];
                    const int fin = isfinite(uk);
                    bad |= !fin;
                    s_uk[j] = fin ? uk : 0.0;
                    beta += fabs(s_uk[j]) * B.hc_norm1[j];
                }
                if (bad) atomicOr(P.status, ST_NAN_PULSE);
                beta *= B.dt;
                int s = 0;
                while (beta > tabs.theta_cap && s < P.max_sq) { beta *= 0.5; ++s; }
                if (beta > tabs.theta_cap) atomicOr(P.status, ST_SQUARING_CAP);
                int di = 0;
                while (di < tabs.n_deg - 1 && tabs.theta[di] < beta) ++di;
                s_sq = s;
                s_p = c_deg_p[di];
                s_q = c_deg_q[di];
                s_scale = B.dt / (double)(1LL << s);
                if (P.stats) {
                    const unsigned long long m3 = (unsigned long long)m * m * m;
                    atomicAdd(P.stats + 0, m3 * (unsigned long long)(c_deg_p[di] + c_deg_q[di] - 2));
                    atomicAdd(P.stats + 1, m3 * (unsigned long long)s);
                    atomicAdd(P.stats + 2, 1ull);
                }
            }
            __syncthreads();
            const int s = s_sq, p = s_p, q = s_q;
            const int d = p * q;

            // X = -i (tau / 2^s) (H0 + sum_j u_j Hc_j)
            {
                const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
                const T sc = (T)s_scale;
                cx<T>* X = base + mm_max;
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    cx<T> h = H[e];
                    for (int j = 0; j < P.nc; ++j) {
                        const cx<T> hc = H[(size_t)(1 + j) * mm + e];
                        const T uj = (T)s_uk[j];
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
                const T cd = (T)s_if[d];
                const cx<T>* Xpp = base + p * mm_max;
                const int b0 = (q - 1) * p;
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
                    cx<T> v = cscale<T>(Xpp[e], cd);
                    if (row == col) v.x += (T)s_if[b0];
                    for (int l = 1; l < p; ++l) {
                        const cx<T> xv = pw[l][e];
                        const T c = (T)s_if[b0 + l];
                        v.x = fma(c, xv.x, v.x);
                        v.y = fma(c, xv.y, v.y);
                    }
                    S[e] = v;
                }
            }
            __syncthreads();
            for (int kb = q - 2; kb >= 0; --kb) {
                if (threadIdx.x < p) coef[threadIdx.x] = (T)s_if[kb * p + threadIdx.x];
                __syncthreads();
                cta_gemm<T, R>(Sn, S, base + p * mm_max, m, p, coef, pw, sm);
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
