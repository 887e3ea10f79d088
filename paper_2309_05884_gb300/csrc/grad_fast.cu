// Exact slice derivatives (Appendix B) for FP32 plans, blocks of size m <= 128, slices that need no
// sub-slicing: the same series and contraction as grad.cu, with the slice matrix held in registers.
//
// For slice k and block b, A = -i tau (H0 + sum_j u_kj Hc_j), v_q = A^q psi_{k-1} and w_p = (-A)^p
// lam_k (A is anti-Hermitian, so (A^dagger)^p = (-A)^p), z_q = sum_{p <= P-q} w_p / (p+q+1)!, and
//     dF-partial_j = -i tau sum_{a,b} Hc_j[a][b] M[a][b],   M[a][b] = sum_{q, copies} conj(z_q[a]) v_q[b].
// grad_mode 1 is the paper's first-order term (Eq. propagator_differentiation): P = 0, z_0 = lam_k,
// v_0 = psi_k.
//
// One CTA of 512 threads owns one (slice, block) item.  Warp w owns rows [w RW, (w+1) RW) of A (RW =
// MT/16); within a warp, the 8 lanes of a group share the group's rows (lane >> 3 selects rows
// rs, rs + 4, ...) and split the columns in pairs: lane part cp = lane & 7 takes columns
// 16 t + 2 cp and 16 t + 2 cp + 1, so that a vector load is one 16-byte access and the 8 lanes of a
// group read 128 contiguous bytes.  Each thread keeps its RPT x CPT tile of A in registers for the
// whole chain: a matrix-vector step reads only the vectors (shared memory), and the 8 partial sums
// of a row are combined by a reduce-scatter over the group's lanes (shuffle rounds) that leaves each
// lane a part of the outputs.  The v and w chains of up to two copies of the block advance in the
// same step (NV = 2 or 4 vectors, fixed at compile time), one barrier per step.  The tile of M uses
// the same layout, and the contraction reads each Hc_j tile once.
#include "../../include/qoc.h"
#include "kernels.h"

namespace qoc {
namespace {

constexpr int GF_THREADS = 512;
constexpr int GF_PM = 24;   // longest series (as the FP32 configuration of grad.cu)
constexpr int GF_CG = 2;    // copies per pass
constexpr int GF_NVM = 2 * GF_CG;
constexpr int GF_VL = 128;  // stride of one vector in shared memory (float2)
constexpr int GF_SUB_MAX = 7;  // sub-slicing decision shared with grad.cu

template <int MT> struct GfShape {
    static constexpr int RW = MT / 16;   // rows per warp
    static constexpr int RPT = RW / 4;   // rows per thread
    static constexpr int CPT = MT / 8;   // columns per thread (CPT / 2 pairs)
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ int gf_col(int cp, int cc) { return 16 * (cc >> 1) + 2 * cp + (cc & 1); }

// Shared vectors (float2): X[q][v] (v < CG: v_q of the copies; CG..2CG-1: w_q), Z[q][r]; each of
// GF_VL entries, entries m.. kept zero.
struct GfSmem {
    float2* X;
    float2* Z;
    __device__ float2* x(int q, int v) const { return X + ((size_t)q * GF_NVM + v) * GF_VL; }
    __device__ float2* z(int q, int r) const { return Z + ((size_t)q * GF_CG + r) * GF_VL; }
};

// The chains, the M tile and the contraction for one copy group (CG = NV / 2 copies) of one item;
// X[0] holds v_0 and w_0, Z[0..Pt] is zero.  Adds each thread's contraction terms into s_acc.
template <int MT, int NV>
__device__ __forceinline__ void gf_group(const GfSmem& S, const float2 (&At)[GfShape<MT>::RPT][GfShape<MT>::CPT],
                                         int m, int Pt, const float* s_if, const float2* H, size_t mm, int nc,
                                         float2 (*s_acc)[GF_THREADS]) {
    using Sh = GfShape<MT>;
    constexpr int RPT = Sh::RPT, CPT = Sh::CPT, RW = Sh::RW;
    constexpr int CG = NV / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cp = lane & 7, rs = lane >> 3;
    for (int p = 0; p <= Pt; ++p) {
        // z_q += w_p / (p+q+1)! for q <= P-p: thread (half, r, a), the two halves split the q range
        {
            const int t = threadIdx.x & 255, half = threadIdx.x >> 8;
            const int r = t / GF_VL, a = t % GF_VL;
            if (r < CG && a < m) {
                const float2 w = S.x(p, CG + r)[a];
                for (int q = half; q <= Pt - p; q += 2) {
                    const float cf = s_if[p + q + 1];
                    float2& z = S.z(q, r)[a];
                    z.x = fmaf(cf, w.x, z.x);
                    z.y = fmaf(cf, w.y, z.y);
                }
            }
        }
        if (p < Pt) {
            // x_{p+1}[v] = A x_p[v] for the v chains (v < CG), -A x_p[v] for the w chains
            float2 acc[RPT][NV];
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[i][v] = f2(0.f, 0.f);
#pragma unroll
            for (int cc = 0; cc < CPT; cc += 2) {
                const int b = gf_col(cp, cc);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float4 x2 = *reinterpret_cast<const float4*>(S.x(p, v) + b);  // columns b, b+1
#pragma unroll
                    for (int i = 0; i < RPT; ++i) {
                        const float2 a0 = At[i][cc], a1 = At[i][cc + 1];
                        acc[i][v].x = fmaf(a0.x, x2.x, fmaf(-a0.y, x2.y, acc[i][v].x));
                        acc[i][v].y = fmaf(a0.x, x2.y, fmaf(a0.y, x2.x, acc[i][v].y));
                        acc[i][v].x = fmaf(a1.x, x2.z, fmaf(-a1.y, x2.w, acc[i][v].x));
                        acc[i][v].y = fmaf(a1.x, x2.w, fmaf(a1.y, x2.z, acc[i][v].y));
                    }
                }
            }
            // reduce-scatter over the 8 lanes of the group.  Float f = 2 (i NV + v) + part; HR halving
            // rounds (offsets 4, 2, 1 while floats remain to split) leave lane cp the floats
            // [fi0, fi0 + F); the remaining rounds are plain sums, after which lanes with the low
            // 3 - HR bits of cp clear write.
            constexpr int NF = 2 * RPT * NV;  // 16, 8 or 4
            constexpr int HR = NF >= 8 ? 3 : 2;
            constexpr int F = NF >= 8 ? NF / 8 : 1;
            float val[NF];
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    val[2 * (i * NV + v)] = acc[i][v].x;
                    val[2 * (i * NV + v) + 1] = acc[i][v].y;
                }
#pragma unroll
            for (int rd = 0; rd < 3; ++rd) {
                const int off = 4 >> rd;
                if (rd < HR) {
                    const int h = NF >> (rd + 1);
                    const bool up = (lane & off) != 0;
#pragma unroll
                    for (int t = 0; t < NF / 2; ++t) {
                        if (t < h) {
                            const float send = up ? val[t] : val[t + h];
                            const float keep = up ? val[t + h] : val[t];
                            val[t] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                        }
                    }
                } else {
                    val[0] += __shfl_xor_sync(0xffffffffu, val[0], off);
                }
            }
            const int fi0 = (cp >> (3 - HR)) * F;
            if ((cp & ((1 << (3 - HR)) - 1)) == 0) {
#pragma unroll
                for (int t = 0; t < F; ++t) {
                    const int fi = fi0 + t;
                    const int ci = fi >> 1, part = fi & 1;
                    const int i = ci / NV, v = ci - i * NV;
                    const int a = warp * RW + rs + 4 * i;  // rows >= m come out exactly 0
                    const float y = v >= CG ? -val[t] : val[t];
                    reinterpret_cast<float*>(S.x(p + 1, v))[2 * a + part] = y;
                }
            }
        }
        __syncthreads();
    }
    // M tile, one row of the thread's tile at a time (bounds the live registers):
    // M[a][b] = sum_{q, r} conj(z_qr[a]) v_qr[b], then the contraction with each Hc_j
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int a = warp * RW + rs + 4 * i;
        float2 Mr[CPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) Mr[cc] = f2(0.f, 0.f);
        for (int q = 0; q <= Pt; ++q) {
#pragma unroll
            for (int r = 0; r < CG; ++r) {
                const float2 za = S.z(q, r)[a];
                const float2* vq = S.x(q, r);
#pragma unroll
                for (int cc = 0; cc < CPT; cc += 2) {  // conj(z) v
                    const float4 vb = *reinterpret_cast<const float4*>(vq + gf_col(cp, cc));
                    Mr[cc].x = fmaf(za.x, vb.x, fmaf(za.y, vb.y, Mr[cc].x));
                    Mr[cc].y = fmaf(za.x, vb.y, fmaf(-za.y, vb.x, Mr[cc].y));
                    Mr[cc + 1].x = fmaf(za.x, vb.z, fmaf(za.y, vb.w, Mr[cc + 1].x));
                    Mr[cc + 1].y = fmaf(za.x, vb.w, fmaf(-za.y, vb.z, Mr[cc + 1].y));
                }
            }
        }
        if (a < m) {
            for (int j = 0; j < nc; ++j) {
                const float2* hrow = H + (size_t)(1 + j) * mm + (size_t)a * m;
                float2 acc = s_acc[j][threadIdx.x];
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    const int bcol = gf_col(cp, cc);
                    if (bcol < m) {
                        const float2 hc = hrow[bcol];
                        acc.x = fmaf(hc.x, Mr[cc].x, fmaf(-hc.y, Mr[cc].y, acc.x));
                        acc.y = fmaf(hc.x, Mr[cc].y, fmaf(hc.y, Mr[cc].x, acc.y));
                    }
                }
                s_acc[j][threadIdx.x] = acc;
            }
        }
    }
}

// One (slice, block) item with tile size MT: for every copy group, the A tile, the chains, the M
// tile and the contraction; each thread's contraction terms accumulate in s_acc.
template <int MT>
__device__ __forceinline__ void gf_item(const GfSmem& S, const DevPlan& P, const DevBlock& B, int m, int c, int kw,
                                        int Pt, const float2* H, size_t mm, float tau, const float* s_uk,
                                        const float* s_if, int nc, const float2* __restrict__ psi_st,
                                        const float2* __restrict__ lam_st, float2 (*s_acc)[GF_THREADS]) {
    using Sh = GfShape<MT>;
    constexpr int RPT = Sh::RPT, CPT = Sh::CPT, RW = Sh::RW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cp = lane & 7, rs = lane >> 3;
    for (int r0 = 0; r0 < c; r0 += GF_CG) {
        const int cg = (c - r0) < GF_CG ? (c - r0) : GF_CG;
        const long long kpsi = P.grad_mode == 0 ? kw : kw + 1;
        // tile of A (grad_mode 0): rows warp RW + rs + 4 i, columns gf_col(cp, cc); assembled per
        // copy group, one pass per matrix so that a tile's loads are in flight together
        float2 At[RPT][CPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) At[i][cc] = f2(0.f, 0.f);
        if (P.grad_mode == 0) {
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int a = warp * RW + rs + 4 * i;
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    const int b = gf_col(cp, cc);
                    if (a < m && b < m) At[i][cc] = H[(size_t)a * m + b];
                }
            }
            for (int j = 0; j < nc; ++j) {
                const float2* Hj = H + (size_t)(1 + j) * mm;
                const float uj = s_uk[j];
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    const int a = warp * RW + rs + 4 * i;
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        const int b = gf_col(cp, cc);
                        if (a < m && b < m) {
                            const float2 hc = Hj[(size_t)a * m + b];
                            At[i][cc].x = fmaf(uj, hc.x, At[i][cc].x);
                            At[i][cc].y = fmaf(uj, hc.y, At[i][cc].y);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) At[i][cc] = f2(tau * At[i][cc].y, -tau * At[i][cc].x);  // -i tau h
        }
        // v_0 = psi, w_0 = lam of the group's copies (full length, zero tail); Z[0..Pt] = 0
        for (int e = threadIdx.x; e < GF_CG * GF_VL; e += GF_THREADS) {
            const int r = e / GF_VL, a = e % GF_VL;
            const bool in = r < cg && a < m;
            S.x(0, r)[a] = in ? psi_st[B.s_off + kpsi * c * m + (size_t)(r0 + r) * m + a] : f2(0.f, 0.f);
            S.x(0, GF_CG + r)[a] = in ? lam_st[B.s_off + (long long)(kw + 1) * c * m + (size_t)(r0 + r) * m + a]
                                      : f2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < (Pt + 1) * GF_CG * GF_VL; e += GF_THREADS) S.Z[e] = f2(0.f, 0.f);
        __syncthreads();
        if (cg == 2) {
            gf_group<MT, 4>(S, At, m, Pt, s_if, H, mm, nc, s_acc);
        } else {
            // one copy: the w vectors live in slot CG = 1 of the NV = 2 layout; move w_0 there
            for (int e = threadIdx.x; e < GF_VL; e += GF_THREADS) S.x(0, 1)[e] = S.x(0, GF_CG)[e];
            __syncthreads();
            gf_group<MT, 2>(S, At, m, Pt, s_if, H, mm, nc, s_acc);
        }
        __syncthreads();  // X, Z are refilled by the next copy group
    }
}

__global__ void __launch_bounds__(GF_THREADS, 1)
grad_fast_kernel(DevPlan P, double tol, double theta, const double* __restrict__ u, const float2* __restrict__ psi_st,
                 const float2* __restrict__ lam_st, double2* __restrict__ partial, int gemm_min_m) {
    extern __shared__ __align__(16) unsigned char dsm[];
    GfSmem S;
    S.X = reinterpret_cast<float2*>(dsm);
    S.Z = S.X + (size_t)(GF_PM + 1) * GF_NVM * GF_VL;
    __shared__ float s_if[GF_PM + 2];
    __shared__ float s_uk[8];
    __shared__ int s_P;
    __shared__ double red[GF_THREADS / 32][8][2];
    // per-thread contraction sums (re, im of each control), kept out of registers during the chains
    __shared__ float2 s_acc[8][GF_THREADS];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = P.nc;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < GF_PM + 2; ++i) {
            s_if[i] = (float)f;
            f /= (double)(i + 1);
        }
    }
    // zero every vector once: entries >= m are never written with anything but zeros afterwards
    for (int e = threadIdx.x; e < (GF_PM + 1) * (GF_NVM + GF_CG) * GF_VL; e += GF_THREADS) S.X[e] = f2(0.f, 0.f);

    const int NK = P.nk;
    const bool whole = P.nk < 0;
    const long long total = whole ? P.n_items : (long long)NK * P.nb;
    __shared__ int s_list[GF_THREADS];
    __shared__ int s_nl;
    __shared__ int s_wc[32];
    // slices this launch owns: blocks of up to 128 states, slices that need no sub-slicing; the norm
    // bound and pulses of each tested slice are kept for the setup below
    __shared__ double s_beta[GF_THREADS];
    __shared__ float s_ul[GF_THREADS][8];
    auto want = [&](long long it) -> bool {
        int bi;
        long long k;
        if (whole) {
            const int2 e = P.items[it];
            bi = e.x;
            k = e.y;
        } else {
            bi = (int)(it / NK);
            k = P.k0 + it % NK;
        }
        const DevBlock& Bw = P.blocks[bi];
        if (Bw.m > 128) return false;
        const double beta = slice_beta(P, Bw, u, k);
        for (int j = 0; j < nc; ++j) {
            const double x = u[(size_t)(Bw.u_row + k) * nc + j];
            s_ul[threadIdx.x][j] = isfinite(x) ? (float)x : 0.f;
        }
        s_beta[threadIdx.x] = beta;
        if (P.grad_mode != 0) return true;
        // unsplit slices of blocks on the GEMM path (grad_gemm.cu) are not this launch's
        return slice_halvings(beta, theta, GF_SUB_MAX) == 0 && !(gemm_min_m > 0 && Bw.m >= gemm_min_m);
    };
    for (long long lb = 0; cta_select(total, lb, want, s_list, &s_nl, s_wc); lb += blockDim.x) {
        const int nl = s_nl;
        for (int li = 0; li < nl; ++li) {
            const long long item = (long long)blockIdx.x + (lb + s_list[li]) * gridDim.x;
            int bi, kw, k;
            if (whole) {
                const int2 it = P.items[item];
                bi = it.x;
                kw = it.y;
                k = it.y + 1;
            } else {
                bi = (int)(item / NK);
                kw = (int)(item % NK);
                k = P.k0 + kw + 1;
            }
            const DevBlock& B = P.blocks[bi];
            const int m = B.m, c = B.c;
            __syncthreads();  // the previous item's readers of s_* are done
            if (threadIdx.x == 0) {
                const int ti = s_list[li];  // the thread that tested this slice
                for (int j = 0; j < nc; ++j) s_uk[j] = s_ul[ti][j];
                double beta = s_beta[ti];
                int Pt = 0, sub = 0;
                if (P.grad_mode == 0) {
                    while (beta > theta && sub < GF_SUB_MAX) { beta *= 0.5; ++sub; }
                    double term = beta;
                    while (Pt < GF_PM && term > tol) { ++Pt; term *= beta / (double)(Pt + 1); }
                    if (sub == 0 && term > tol) atomicOr(P.status, ST_SERIES_CAP);
                }
                s_P = Pt;
                if (P.stats)
                    atomicAdd(P.stats + 3, (unsigned long long)m * m * (unsigned long long)(c * (3 * Pt + 1) + nc));
            }
            __syncthreads();
            const int Pt = s_P;
            const size_t mm = (size_t)m * m;
            const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;
            const float tau = (float)B.dt;
#pragma unroll
            for (int j = 0; j < 8; ++j) s_acc[j][threadIdx.x] = f2(0.f, 0.f);

            if (m <= 64)
                gf_item<64>(S, P, B, m, c, kw, Pt, H, mm, tau, s_uk, s_if, nc, psi_st, lam_st, s_acc);
            else
                gf_item<128>(S, P, B, m, c, kw, Pt, H, mm, tau, s_uk, s_if, nc, psi_st, lam_st, s_acc);
            // block reduction of the nc complex sums in FP64 (the per-thread sums cancel strongly when
            // the gradient is small, so they are added without further FP32 rounding); then -i tau
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= nc) break;
                double xr = (double)s_acc[j][threadIdx.x].x, xi = (double)s_acc[j][threadIdx.x].y;
                for (int off = 16; off > 0; off >>= 1) {
                    xr += __shfl_xor_sync(0xffffffffu, xr, off);
                    xi += __shfl_xor_sync(0xffffffffu, xi, off);
                }
                if (lane == 0) {
                    red[warp][j][0] = xr;
                    red[warp][j][1] = xi;
                }
            }
            __syncthreads();
            if (threadIdx.x < nc) {
                double xr = 0.0, xi = 0.0;
                for (int w = 0; w < GF_THREADS / 32; ++w) {
                    xr += red[w][threadIdx.x][0];
                    xi += red[w][threadIdx.x][1];
                }
                double2 o;
                o.x = B.dt * xi;
                o.y = -B.dt * xr;
                partial[(size_t)(B.part_off + k - 1) * nc + threadIdx.x] = o;
            }
        }
    }
}

size_t gf_smem() { return (size_t)(GF_PM + 1) * (GF_NVM + GF_CG) * GF_VL * sizeof(float2); }

}  // namespace

int grad_fast_max_m(int prec) { return prec == QOC_PREC_F64 ? 0 : 128; }

int launch_grad_fast(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store, double2* partial,
                     int max_m, int grid, cudaStream_t st, int gemm_min_m) {
    if (P.prec == QOC_PREC_F64 || P.nc > 8 || max_m < 1) return 0;
    const size_t sm = gf_smem();
    if (cudaFuncSetAttribute(grad_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return -1;
    grad_fast_kernel<<<grid, GF_THREADS, sm, st>>>(P, GF32_SERIES_TOL, 3.0, u, (const float2*)psi_store, (const float2*)lam_store,
                                                   partial, gemm_min_m);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
