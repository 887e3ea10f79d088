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
// MT/16); within a warp, the 8 lanes of a group (lane & 7 = column part cp) share the group's rows
// (lane >> 3 selects rows rs, rs + 4, ...) and split the columns (col = cp + 8 c).  Each thread
// keeps its RPT x CPT tile of A in registers for the whole chain, so a matrix-vector step reads
// only the vectors (shared memory, broadcast within the 8-lane groups), and the 8 partial sums of a
// row are combined by a reduce-scatter over the group's lanes (3 shuffle rounds) that leaves each
// lane one part of the outputs.  The v and w chains of every copy of the block advance in the same
// step (up to 4 vectors), with one barrier per step.  The tile of M reuses the same layout, and
// the contraction reads each Hc_j tile once.
#include "../../include/qoc.h"
#include "kernels.h"

namespace qoc {
namespace {

constexpr int GF_THREADS = 512;
constexpr int GF_PM = 24;  // longest series (as the FP32 configuration of grad.cu)
constexpr int GF_CG = 2;   // copies per pass: 2 * GF_CG vectors per step
constexpr int GF_NV = 2 * GF_CG;
constexpr int GF_SUB_MAX = 7;  // sub-slicing decision shared with grad.cu

template <int MT> struct GfShape {
    static constexpr int RW = MT / 16;   // rows per warp
    static constexpr int RPT = RW / 4;   // rows per thread
    static constexpr int CPT = MT / 8;   // columns per thread
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// Shared layout (float2 elements): V[(PM+1) * CG][MT], Z[(PM+1) * CG][MT], W[CG][MT], Wn[CG][MT].
// Entries m..MT-1 of every vector stay zero.
template <int MT>
__global__ void __launch_bounds__(GF_THREADS, 1)
grad_fast_kernel(DevPlan P, double tol, double theta, const double* __restrict__ u, const float2* __restrict__ psi_st,
                 const float2* __restrict__ lam_st, double2* __restrict__ partial, int m_lo) {
    using S = GfShape<MT>;
    constexpr int RPT = S::RPT, CPT = S::CPT, RW = S::RW;
    extern __shared__ __align__(16) unsigned char dsm[];
    float2* V = reinterpret_cast<float2*>(dsm);
    float2* Z = V + (size_t)(GF_PM + 1) * GF_CG * MT;
    float2* Wa = Z + (size_t)(GF_PM + 1) * GF_CG * MT;
    float2* Wb = Wa + (size_t)GF_CG * MT;
    __shared__ float s_if[GF_PM + 2];
    __shared__ float s_uk[8];
    __shared__ int s_P, s_skip;
    __shared__ double red[GF_THREADS / 32][8][2];
    // per-thread contraction sums (re, im of each control), kept out of registers during the chains
    __shared__ float2 s_acc[8][GF_THREADS];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cp = lane & 7, rs = lane >> 3;
    const int nc = P.nc;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < GF_PM + 2; ++i) {
            s_if[i] = (float)f;
            f /= (double)(i + 1);
        }
    }
    // zero every vector once (entries >= m must read as 0)
    for (int e = threadIdx.x; e < (2 * (GF_PM + 1) + 2) * GF_CG * MT; e += GF_THREADS) V[e] = f2(0.f, 0.f);

    const int NK = P.nk;
    const bool whole = P.nk < 0;
    const long long total = whole ? P.n_items : (long long)NK * P.nb;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
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
        if (m <= m_lo || m > MT) continue;  // another launch owns this block size
        __syncthreads();                     // the previous item's readers of s_* are done
        if (threadIdx.x == 0) {
            double beta = B.h0_norm1;
            for (int j = 0; j < nc; ++j) {
                const double uk = u[(size_t)(B.u_row + k - 1) * nc + j];
                const double x = isfinite(uk) ? uk : 0.0;
                s_uk[j] = (float)x;
                beta += fabs(x) * B.hc_norm1[j];
            }
            beta *= B.dt;
            int Pt = 0, sub = 0;
            if (P.grad_mode == 0) {
                while (beta > theta && sub < GF_SUB_MAX) { beta *= 0.5; ++sub; }
                double term = beta;
                while (Pt < GF_PM && term > tol) { ++Pt; term *= beta / (double)(Pt + 1); }
                if (sub == 0 && term > tol) atomicOr(P.status, ST_SERIES_CAP);
            }
            s_P = Pt;
            s_skip = sub > 0;  // split slices: grad.cu (sub-slices) or grad_rev.cu (reverse mode)
        }
        __syncthreads();
        if (s_skip) continue;
        const int Pt = s_P;
        const size_t mm = (size_t)m * m;
        const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;
        const float tau = (float)B.dt;

#pragma unroll
        for (int j = 0; j < 8; ++j) s_acc[j][threadIdx.x] = f2(0.f, 0.f);

        for (int r0 = 0; r0 < c; r0 += GF_CG) {
            const int cg = (c - r0) < GF_CG ? (c - r0) : GF_CG;
            const long long kpsi = P.grad_mode == 0 ? kw : kw + 1;
            // tile of A (grad_mode 0 only): rows warp RW + rs + 4 i, columns cp + 8 c; assembled per copy
            // group so that it is dead while the M tile is live
            float2 At[RPT][CPT];
            if (P.grad_mode == 0) {
                // one pass per matrix over the whole tile, so that the tile's loads are in flight together
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    const int a = warp * RW + rs + 4 * i;
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        const int b = cp + 8 * cc;
                        At[i][cc] = (a < m && b < m) ? H[(size_t)a * m + b] : f2(0.f, 0.f);
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
                            const int b = cp + 8 * cc;
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
            // v_0 = psi, w_0 = lam (copies r0 .. r0+cg-1); Z = 0
            for (int e = threadIdx.x; e < cg * MT; e += GF_THREADS) {
                const int r = e / MT, a = e - r * MT;
                const bool in = a < m;
                V[e] = in ? psi_st[B.s_off + kpsi * c * m + (size_t)(r0 + r) * m + a] : f2(0.f, 0.f);
                Wa[e] = in ? lam_st[B.s_off + (long long)(kw + 1) * c * m + (size_t)(r0 + r) * m + a] : f2(0.f, 0.f);
            }
            for (int e = threadIdx.x; e < (Pt + 1) * GF_CG * MT; e += GF_THREADS) Z[e] = f2(0.f, 0.f);
            __syncthreads();
            float2* W = Wa;
            float2* Wn = Wb;
            const int nv = 2 * cg;
            for (int p = 0; p <= Pt; ++p) {
                // z_q += w_p / (p+q+1)!  for q <= P-p  (reads W only)
                for (int e = threadIdx.x; e < (Pt - p + 1) * cg * m; e += GF_THREADS) {
                    const int q = e / (cg * m);
                    const int ra = e - q * cg * m;
                    const int r = ra / m, a = ra - r * m;
                    const float cf = s_if[p + q + 1];
                    float2& z = Z[((size_t)q * GF_CG + r) * MT + a];
                    const float2 w = W[(size_t)r * MT + a];
                    z.x = fmaf(cf, w.x, z.x);
                    z.y = fmaf(cf, w.y, z.y);
                }
                if (p < Pt) {
                    // v_{p+1} = A v_p, w_{p+1} = -A w_p for the cg copies: vectors 0..cg-1 are v, cg..2cg-1
                    // are w; offsets (float2) from V of each vector's input and output
                    const int w_in = (int)(W - V), w_out = (int)(Wn - V);
                    auto in_off = [&](int v) { return v < cg ? (p * GF_CG + v) * MT : w_in + (v - cg) * MT; };
                    auto out_off = [&](int v) { return v < cg ? ((p + 1) * GF_CG + v) * MT : w_out + (v - cg) * MT; };
                    float2 acc[RPT][GF_NV];
#pragma unroll
                    for (int i = 0; i < RPT; ++i)
#pragma unroll
                        for (int v = 0; v < GF_NV; ++v) acc[i][v] = f2(0.f, 0.f);
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        const int b = cp + 8 * cc;
#pragma unroll
                        for (int v = 0; v < GF_NV; ++v) {
                            if (v < nv) {
                                const float2 x = V[in_off(v) + b];
#pragma unroll
                                for (int i = 0; i < RPT; ++i) {
                                    acc[i][v].x = fmaf(At[i][cc].x, x.x, fmaf(-At[i][cc].y, x.y, acc[i][v].x));
                                    acc[i][v].y = fmaf(At[i][cc].x, x.y, fmaf(At[i][cc].y, x.x, acc[i][v].y));
                                }
                            }
                        }
                    }
                    // reduce-scatter over the 8 lanes of the group: float index f = 2 (i GF_NV + v) + part
                    constexpr int NF = 2 * RPT * GF_NV;  // 16 (RPT 2) or 8 (RPT 1)
                    float val[NF];
#pragma unroll
                    for (int i = 0; i < RPT; ++i)
#pragma unroll
                        for (int v = 0; v < GF_NV; ++v) {
                            val[2 * (i * GF_NV + v)] = acc[i][v].x;
                            val[2 * (i * GF_NV + v) + 1] = acc[i][v].y;
                        }
#pragma unroll
                    for (int off = 4, len = NF; off > 0; off >>= 1, len >>= 1) {
                        const int h = len / 2;
                        const bool up = (lane & off) != 0;
#pragma unroll
                        for (int t = 0; t < NF / 2; ++t) {
                            if (t < h) {
                                const float send = up ? val[t] : val[t + h];
                                const float keep = up ? val[t + h] : val[t];
                                val[t] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                            }
                        }
                    }
                    // this lane now holds floats [cp F, cp F + F), F = NF / 8
                    constexpr int F = NF / 8;
#pragma unroll
                    for (int t = 0; t < F; ++t) {
                        const int fi = cp * F + t;
                        const int ci = fi >> 1, part = fi & 1;
                        const int i = ci / GF_NV, v = ci - i * GF_NV;
                        const int a = warp * RW + rs + 4 * i;  // rows >= m come out exactly 0
                        if (v < nv) {
                            const float y = v >= cg ? -val[t] : val[t];
                            reinterpret_cast<float*>(V + out_off(v))[2 * a + part] = y;
                        }
                    }
                }
                __syncthreads();
                if (p < Pt) {
                    float2* t = W;
                    W = Wn;
                    Wn = t;
                }
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
                    for (int r = 0; r < cg; ++r) {
                        const float2* zq = Z + ((size_t)q * GF_CG + r) * MT;
                        const float2* vq = V + ((size_t)q * GF_CG + r) * MT;
                        const float2 za = zq[a];
#pragma unroll
                        for (int cc = 0; cc < CPT; ++cc) {  // conj(z) v
                            const float2 vb = vq[cp + 8 * cc];
                            Mr[cc].x = fmaf(za.x, vb.x, fmaf(za.y, vb.y, Mr[cc].x));
                            Mr[cc].y = fmaf(za.x, vb.y, fmaf(-za.y, vb.x, Mr[cc].y));
                        }
                    }
                }
                if (a < m) {
                    for (int j = 0; j < nc; ++j) {
                        const float2* hrow = H + (size_t)(1 + j) * mm + (size_t)a * m;
                        float2 acc = s_acc[j][threadIdx.x];
#pragma unroll
                        for (int cc = 0; cc < CPT; ++cc) {
                            const int bcol = cp + 8 * cc;
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
            __syncthreads();  // V, Z, W are refilled by the next copy group
        }
        // block reduction of the nc complex sums (FP64 across threads); then multiply by -i tau
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

template <int MT>
size_t gf_smem() {
    return (size_t)(2 * (GF_PM + 1) + 2) * GF_CG * MT * sizeof(float2);
}

template <int MT>
int launch_one(const DevPlan& P, const double* u, const void* psi, const void* lam, double2* partial, int m_lo,
               int grid, cudaStream_t st) {
    const size_t sm = gf_smem<MT>();
    if (cudaFuncSetAttribute(grad_fast_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
        return -1;
    grad_fast_kernel<MT><<<grid, GF_THREADS, sm, st>>>(P, 1e-9, 3.0, u, (const float2*)psi, (const float2*)lam,
                                                        partial, m_lo);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int grad_fast_max_m(int prec) { return prec == QOC_PREC_F64 ? 0 : 128; }

int launch_grad_fast(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store, double2* partial,
                     int max_m, int grid, cudaStream_t st) {
    if (P.prec == QOC_PREC_F64 || P.nc > 8) return 0;
    int rc = 0;
    if (max_m > 0) rc |= launch_one<64>(P, u, psi_store, lam_store, partial, 0, grid, st);
    if (max_m > 64) rc |= launch_one<128>(P, u, psi_store, lam_store, partial, 64, grid, st);
    return rc;
}

}  // namespace qoc
