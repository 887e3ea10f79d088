// Exact slice derivatives of the large blocks (m > 128; FP32 plans, slices without sub-steps) as
// tall GEMMs over all slices of a chunk (Appendix B, Eq. propagator_differentiation, exact form).
//
// With A_k = -i tau (H0 + sum_j u_kj Hc_j), E_j = -i tau Hc_j, psi = psi_{k-1}, lam = lam_k and
//     L(A, E) = sum_{a,b >= 0} A^a E A^b / (a+b+1)!,
// and A^dagger = -A (H Hermitian), the slice derivative is
//     lam^dagger L(A_k, E_j) psi = -i tau sum_{a+b <= P} (-1)^a / (a+b+1)! * z_a^dagger (Hc_j v_b),
//     v_b = A_k^b psi,  z_a = A_k^a lam,
// truncated once beta^{P+1}/(P+1)! is below the FP32 tolerance (beta the slice's norm bound).
// Every chain step needs A_k x = -i tau (H0 x + sum_j u_kj Hc_j x), and H0, Hc_j do not depend on
// the slice: one step for every vector of every slice of the chunk is the product
//     Y = [H0; Hc_1; ...; Hc_nc] X,   X = [v_p and z_p of every (slice, copy)] (m x 2 c S),
// a tall GEMM with (1 + nc) m rows, m deep and 2 c S columns.  The Hc_j v_b it produces are the
// E_j v_b the series contracts with, so nothing else touches the Hamiltonians.  Per chunk:
//   gg_prep      ownership (no sub-steps) and series length of every slice, the largest P;
//   gg_load      X_0 = (psi_{k-1}, lam_k) per copy, Z_0 = lam_k;
//   gg_gemm      step p = 0..P: Y = H_stack X_p (FP32 CUDA-core tiles, 128 x 64 per CTA), or
//   gg_planes +  gg_tc: the same product on the tcgen05 tensor cores with both operands split into FP16
//                hi/lo planes (H_stack once per plan, scale 2^eH; the columns every step, each scaled by
//                2^e with e from the chain bound |x_p| <= beta^p of its slice), FP32 accumulation in TMEM;
//   gg_combine   W_p = (Hc_j v_p)_j, X_{p+1} = -i tau (Y_0 + sum_j u_kj Y_j), Z_{p+1} = z_{p+1};
//   gg_contract  sum over (a, b, copies) in FP32 per thread, FP64 across threads, into the partials.
#include <algorithm>
#include <cmath>

#include "kernels.h"
#include "xl_common.cuh"

namespace qoc {
namespace {

constexpr int GG_THREADS = 256;
constexpr int GG_TILE_R = 128, GG_TILE_C = 64, GG_TK = 16;  // rows x columns per CTA, K chunk
constexpr int GG_MIN_M = 129;                       // default: smaller blocks use the register-tile kernel
constexpr size_t GG_SMEM = 2 * (size_t)GG_TK * (GG_TILE_R + GG_TILE_C) * sizeof(float2);  // 48 KB, two buffers

__constant__ double gg_if[GG_PCAP + 3];  // 1/i!, i = 0..PCAP+2

// Chunk layout: S slice slots per chunk (the last chunk uses the first nv of them).  Columns of a
// block: v columns r * S + kw, then z columns c S + r * S + kw; a family (c S vectors of m) has
// stride c S m.  Slots kw >= nv are never owned and stay zero.

__device__ __forceinline__ int gg_slice_P(double beta, double tol) {
    int Pt = 0;
    double term = beta;  // beta^{P+1}/(P+1)! at P = 0
    while (Pt < GG_PCAP && term > tol) {
        ++Pt;
        term *= beta / (double)(Pt + 1);
    }
    return Pt;
}

// One CTA: ownership and series length of each (block, chunk slice), own = P + 1 (0: not owned),
// and the largest length (the chains run that far; each slice's contraction stops at its own P, so a
// slice's result does not depend on which chunk it falls in).
__global__ void gg_prep_kernel(DevPlan P, const GgBlock* __restrict__ gb, int ngb, int kw0, int S, int nv,
                               double tol, double theta, const double* __restrict__ u, int* __restrict__ own,
                               float* __restrict__ lb, int* __restrict__ Pmax, int min_m) {
    __shared__ int smax;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int best = 0;
    for (int e = threadIdx.x; e < ngb * S; e += blockDim.x) {
        const int g = e / S, kw = e - g * S;
        lb[e] = 0.f;
        if (kw >= nv || gb[g].m < min_m) {
            own[e] = 0;
            continue;
        }
        const DevBlock& B = P.blocks[gb[g].bi];
        const long long k = P.k0 + kw0 + kw;  // 0-based slice
        const double beta = slice_beta(P, B, u, k);
        lb[e] = beta > 1.0 ? (float)log2(beta) : 0.f;  // |x_p| <= beta^p for the slice's chains
        const int o = P.grad_mode == 0 && beta <= theta;
        own[e] = 0;
        if (o) {
            const int Pt = gg_slice_P(beta, tol);
            own[e] = Pt + 1;
            best = Pt > best ? Pt : best;
            if (P.stats) {
                const unsigned long long mm = (unsigned long long)B.m * B.m;
                // chain steps (1 + nc) m^2 per vector, 2c vectors, Pt + 1 steps; the contraction
                atomicAdd(P.stats + 4, (unsigned long long)(1 + P.nc) * mm * 2ull * B.c * (Pt + 1) +
                                           (unsigned long long)B.m * B.c * P.nc * (Pt + 1) * (Pt + 2) / 2);
            }
        }
    }
    atomicMax(&smax, best);
    __syncthreads();
    if (threadIdx.x == 0) *Pmax = smax;
}

// X_0: v columns (r, kw) = psi_{k-1}, z columns = lam_k (zero for slices this path does not own);
// Z_0 = lam_k.  grid (blocks of threads over c*S*m, block g).
__global__ void gg_load_kernel(DevPlan P, const GgBlock* __restrict__ gb, int kw0, int S,
                               const float2* __restrict__ psi_st, const float2* __restrict__ lam_st,
                               const int* __restrict__ own, float2* __restrict__ ws, int min_m) {
    const GgBlock& G = gb[blockIdx.y];
    if (G.m < min_m) return;
    const DevBlock& B = P.blocks[G.bi];
    const int m = B.m, c = B.c;
    const long long n = (long long)c * S * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(e / m), i = (int)(e - (long long)col * m);  // col = r * S + kw
        const int r = col / S, kw = col - r * S;
        const long long slot = kw0 + kw;
        const bool o = own[blockIdx.y * S + kw] != 0;  // false for kw beyond the chunk
        const float2 zero = make_float2(0.f, 0.f);
        const float2 ps = o ? psi_st[B.s_off + slot * c * m + (long long)r * m + i] : zero;
        const float2 la = o ? lam_st[B.s_off + (slot + 1) * c * m + (long long)r * m + i] : zero;
        ws[G.x0 + (long long)col * m + i] = ps;
        ws[G.x0 + (long long)(c * S + col) * m + i] = la;
        ws[G.z + (long long)col * m + i] = la;
    }
}

// 8-byte asynchronous global -> shared copy; pred false writes zeros (nothing is read).
__device__ __forceinline__ void gg_cp8(void* dst, const void* src, bool pred) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void gg_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void gg_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Step p: Y[col][R] = sum_k Hs[R][k] X_p[col][k], Hs the stacked [H0; Hc_1; ...] ((1 + nc) m rows).
// One CTA per (128-row, 64-column) tile of one block; thread (ty, tx) owns rows 8 ty .. + 7 and
// columns 4 tx .. + 3.  K is staged through two shared-memory buffers 16 at a time (cp.async, the next
// chunk in flight while the current one is multiplied), transposed so that each thread reads its
// rows and columns as 16-byte vectors.
__global__ void __launch_bounds__(GG_THREADS, 2)
gg_gemm_kernel(DevPlan P, const GgBlock* __restrict__ gb, const int4* __restrict__ tiles, int p,
               const int* __restrict__ Pmax, float2* __restrict__ ws, int min_m) {
    if (p > *Pmax) return;
    if (gb[tiles[blockIdx.x].x].m < min_m) return;
    extern __shared__ __align__(16) float2 gsm[];
    float2(*As)[GG_TK][GG_TILE_R] = reinterpret_cast<float2(*)[GG_TK][GG_TILE_R]>(gsm);
    float2(*Bs)[GG_TK][GG_TILE_C] = reinterpret_cast<float2(*)[GG_TK][GG_TILE_C]>(gsm + 2 * GG_TK * GG_TILE_R);
    const int4 t = tiles[blockIdx.x];  // (block, row tile, column tile)
    const GgBlock& G = gb[t.x];
    const DevBlock& B = P.blocks[G.bi];
    const int m = B.m;
    const int rows = (1 + P.nc) * m;
    const int row0 = t.y * GG_TILE_R, col0 = t.z * GG_TILE_C;
    const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;  // stacked rows, row-major
    const float2* X = ws + ((p & 1) ? G.x1 : G.x0);
    float2* Y = ws + G.y;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;

    float2 acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);

    // copies: A: thread -> row (tid >> 1), k half (tid & 1) * 8; B: column (tid >> 2), k quarter (tid & 3) * 4
    const int ar = tid >> 1, ak = (tid & 1) * 8;
    const int bcol = tid >> 2, bk = (tid & 3) * 4;
    const int gR = row0 + ar, gC = col0 + bcol;
    const bool rok = gR < rows, cok = gC < G.ncol;
    const float2* hrow = H + (size_t)(rok ? gR : 0) * m;
    const float2* xcol = X + (size_t)(cok ? gC : 0) * m;
    auto stage = [&](int buf, int k0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + ak + q;
            const bool ok = rok && k < m;
            gg_cp8(&As[buf][ak + q][ar], hrow + (ok ? k : 0), ok);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + bk + q;
            const bool ok = cok && k < m;
            gg_cp8(&Bs[buf][bk + q][bcol], xcol + (ok ? k : 0), ok);
        }
        gg_cp_commit();
    };
    const int nch = (m + GG_TK - 1) / GG_TK;
    stage(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nch) {
            stage(buf ^ 1, (ch + 1) * GG_TK);
            gg_cp_wait<1>();
        } else {
            gg_cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GG_TK; ++kk) {
            float2 a[8], b[4];
            const float4* ap = reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
            const float4* bp = reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = ap[q];
                a[2 * q] = make_float2(v.x, v.y);
                a[2 * q + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float4 v = bp[q];
                b[2 * q] = make_float2(v.x, v.y);
                b[2 * q + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma<float>(acc[i][j], a[i], b[j]);
        }
        __syncthreads();  // every reader is done before this buffer is refilled
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = col0 + tx * 4 + j;
        if (col >= G.ncol) continue;
        float2* yc = Y + (size_t)col * rows;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int R = row0 + ty * 8 + i;
            if (R < rows) yc[R] = acc[i][j];
        }
    }
}

// After step p: W_p[j][(r,kw)] = Y_j of the v columns; for p < Pmax, X_{p+1} = -i tau (Y_0 + sum_j
// u_kj Y_j) of every column, and Z_{p+1} for the z columns.  Unowned slices keep zero columns.
__global__ void gg_combine_kernel(DevPlan P, const GgBlock* __restrict__ gb, int kw0, int S, int p,
                                  const int* __restrict__ Pmax, const int* __restrict__ own,
                                  const double* __restrict__ u, float2* __restrict__ ws, int min_m) {
    const int pm = *Pmax;
    if (p > pm) return;
    const GgBlock& G = gb[blockIdx.y];
    if (G.m < min_m) return;
    const DevBlock& B = P.blocks[G.bi];
    const int m = B.m, c = B.c, nc = P.nc;
    const int rows = (1 + nc) * m;
    const float tau = (float)B.dt;
    const float2* Y = ws + G.y;
    float2* Xn = ws + ((p & 1) ? G.x0 : G.x1);
    const long long n = (long long)G.ncol * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(e / m), i = (int)(e - (long long)col * m);
        const bool isz = col >= c * S;
        const int vc = isz ? col - c * S : col;  // (r, kw) index r * S + kw
        const int kw = vc % S;
        const float2* yc = Y + (size_t)col * rows;
        if (!isz) {
            for (int j = 0; j < nc; ++j)
                ws[G.w + (((long long)p * nc + j) * c * S + vc) * m + i] = yc[(size_t)(1 + j) * m + i];
        }
        if (p == pm) continue;
        float2 x = make_float2(0.f, 0.f);
        if (own[blockIdx.y * S + kw]) {
            const long long k = P.k0 + kw0 + kw;  // 0-based slice
            float2 h = yc[i];
            for (int j = 0; j < nc; ++j) {
                const double uu = u[(size_t)(B.u_row + k) * nc + j];
                const float uf = isfinite(uu) ? (float)uu : 0.f;
                const float2 yj = yc[(size_t)(1 + j) * m + i];
                h.x = fmaf(uf, yj.x, h.x);
                h.y = fmaf(uf, yj.y, h.y);
            }
            x = make_float2(h.y * tau, -h.x * tau);  // -i tau h
        }
        Xn[(size_t)col * m + i] = x;
        if (isz) ws[G.z + ((long long)(p + 1) * c * S + vc) * m + i] = x;
    }
}

// One CTA per (block, chunk slice) it owns: d_j = -i tau sum_r sum_{a+b<=P} (-1)^a/(a+b+1)!
// z_a^dagger W_b^j, written to the slice's partials (overwrites: every (block, slice) has one owner).
__global__ void __launch_bounds__(GG_THREADS)
gg_contract_kernel(DevPlan P, const GgBlock* __restrict__ gb, int kw0, int S, const int* __restrict__ Pmax,
                   const int* __restrict__ own, const float2* __restrict__ ws, double2* __restrict__ partial) {
    const int g = blockIdx.y, kw = blockIdx.x;
    if (!own[g * S + kw]) return;
    const GgBlock& G = gb[g];
    const DevBlock& B = P.blocks[G.bi];
    const int m = B.m, c = B.c, nc = P.nc, pm = own[g * S + kw] - 1;  // this slice's series length
    __shared__ double red[GG_THREADS / 32][8][2];
    float accr[8], acci[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) accr[j] = acci[j] = 0.f;
    for (int r = 0; r < c; ++r) {
        const long long vc = (long long)r * S + kw;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            // zeta_b = sum_{a <= P - b} (-1)^a / (a+b+1)! conj(z_a), then sum_b zeta_b W_b^j
            float2 za[GG_PCAP + 1];
            for (int a = 0; a <= pm; ++a) za[a] = ws[G.z + ((long long)a * c * S + vc) * m + i];
            for (int b = 0; b <= pm; ++b) {
                float zr = 0.f, zi = 0.f;
                for (int a = 0; a <= pm - b; ++a) {
                    const float cf = (float)((a & 1) ? -gg_if[a + b + 1] : gg_if[a + b + 1]);
                    zr = fmaf(cf, za[a].x, zr);
                    zi = fmaf(-cf, za[a].y, zi);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j >= nc) break;
                    const float2 w = ws[G.w + (((long long)b * nc + j) * c * S + vc) * m + i];
                    accr[j] = fmaf(zr, w.x, fmaf(-zi, w.y, accr[j]));
                    acci[j] = fmaf(zr, w.y, fmaf(zi, w.x, acci[j]));
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j >= nc) break;
        double xr = accr[j], xi = acci[j];
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
    if ((int)threadIdx.x < nc) {
        double xr = 0.0, xi = 0.0;
        for (int w = 0; w < GG_THREADS / 32; ++w) {
            xr += red[w][threadIdx.x][0];
            xi += red[w][threadIdx.x][1];
        }
        const long long k = P.k0 + kw0 + kw;  // 0-based slice
        double2 o;  // (-i tau) (xr + i xi)
        o.x = B.dt * xi;
        o.y = -B.dt * xr;
        partial[(size_t)(B.part_off + k) * nc + threadIdx.x] = o;
    }
}


// ---------------------------------------------------------------- tensor-core product
constexpr int GT_THREADS = 512;
constexpr uint64_t GT_WAIT_NS = 2000000000ull;

// Byte offset of slab (tile t, K chunk ch) of an operand with kc K chunks per tile row.
__device__ __forceinline__ size_t gt_slab(int t, int ch, int kc) { return ((size_t)t * kc + ch) * XL_SLAB; }

// Scale exponent of the columns at chain step p: |x_p| <= beta^p (lbeta = max(0, log2 beta)), so the
// scaled entries stay below 2^14.
__device__ __forceinline__ int gt_exp(int p, float lbeta) {
    const int e = 14 - (int)ceilf((float)p * lbeta);
    return e < -60 ? -60 : e;
}

// Split-FP16 slabs of the stacked [H0; Hc_1; ...] of block g (one-time, at plan creation): grid
// (groups, block); a group is eight consecutive K entries of one row, rows fastest.
__global__ void gg_hplanes_kernel(const GgBlock* __restrict__ gb, const float2* __restrict__ H, int nc,
                                  const long long* __restrict__ h_off, unsigned char* __restrict__ planes, int* status) {
    const GgBlock& G = gb[blockIdx.y];
    const int m = G.m, rows = (1 + nc) * m;
    const int rp = G.rtc * XL_TM, ng = G.kc * (XL_KC / 8);
    const float2* Hs = H + h_off[blockIdx.y];
    const float sc = ldexpf(1.f, G.eH);
    bool ok = true;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)rp * ng;
         idx += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(idx / rp), r = (int)(idx - (long long)grp * rp);
        float2 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = 8 * grp + c;
            v[c] = (r < rows && k < m) ? Hs[(size_t)r * m + k] : make_float2(0.f, 0.f);
        }
        ok = xl_put8(planes + G.hp + gt_slab(r / XL_TM, (8 * grp) / XL_KC, G.kc), xl_off(r % XL_TM, (8 * grp) % XL_KC),
                     v, sc) && ok;
    }
    if (!ok) atomicOr(status, ST_RANGE);
}

// Column slabs of X_p (FP32 columns in the chunk scratch): grid (groups, block); columns fastest so
// that eight consecutive threads fill a 128-byte core matrix of every plane.  Writes each column's
// scale exponent for the product's epilogue.
__global__ void gg_planes_kernel(DevPlan P, const GgBlock* __restrict__ gb, int S, int p, const int* __restrict__ Pmax,
                                 const float* __restrict__ lb, const float2* __restrict__ ws, unsigned char* __restrict__ xpl,
                                 int* __restrict__ cscale, int min_m) {
    if (p > *Pmax) return;
    const GgBlock& G = gb[blockIdx.y];
    if (G.m < min_m) return;
    const int m = G.m, c = G.c;
    const int cp = G.ctc * XL_TM, ng = G.kc * (XL_KC / 8);
    const float2* X = ws + ((p & 1) ? G.x1 : G.x0);
    bool ok = true;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)cp * ng;
         idx += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(idx / cp), col = (int)(idx - (long long)grp * cp);
        int e = 14;
        if (col < G.ncol) {
            const int vc = col >= c * S ? col - c * S : col;
            e = gt_exp(p, lb[blockIdx.y * S + vc % S]);
        }
        if (grp == 0) cscale[G.cs + col] = e;
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = 8 * grp + q;
            v[q] = (col < G.ncol && k < m) ? X[(size_t)col * m + k] : make_float2(0.f, 0.f);
        }
        ok = xl_put8(xpl + G.xp + gt_slab(col / XL_TM, (8 * grp) / XL_KC, G.kc), xl_off(col % XL_TM, (8 * grp) % XL_KC),
                     v, ldexpf(1.f, e)) && ok;
    }
    if (!ok) atomicOr(P.status, ST_RANGE);
}

// Y = H_stack X_p on the tensor cores: one CTA per (128 x 128 output tile, block): rows of the stacked
// H against columns of X, K in chunks of 32 through a 3-stage ring of bulk copies (A slab + B slab);
// one thread issues the MMAs two chunks behind the copies (without the (lo, lo) products: H and X are
// unrelated matrices); the epilogue writes Y[col][R] in FP32.
__global__ void __launch_bounds__(GT_THREADS, 1)
gg_tc_kernel(DevPlan P, const GgBlock* __restrict__ gb, const int4* __restrict__ tiles, int p,
             const int* __restrict__ Pmax, const unsigned char* __restrict__ hpl, const unsigned char* __restrict__ xpl,
             const int* __restrict__ cscale, float2* __restrict__ ws, int min_m) {
    if (p > *Pmax) return;
    const int4 t = tiles[blockIdx.x];  // (block, row tile, column tile)
    const GgBlock& G = gb[t.x];
    if (G.m < min_m) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[XL_STAGES], empty[XL_STAGES], done;
    __shared__ uint32_t tslot;
    __shared__ int s_fail;
    const int m = G.m, rows = (1 + P.nc) * m;
    const int row0 = t.y * XL_TM, col0 = t.z * XL_TM;
    const unsigned char* Apl = hpl + G.hp;
    const unsigned char* Bpl = xpl + G.xp;
    float2* Y = ws + G.y;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        tmem_alloc(&tslot, XL_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < XL_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const uint32_t hre = tmem, him = tmem + 128, cre = tmem + 256, cim = tmem + 384;
    const uint32_t sbase = smem_u32(sm);

    if (threadIdx.x == 0) {
        const int nch = G.kc;
        auto load = [&](int ch) {
            const int st = ch % XL_STAGES;
            mbar_arrive_expect_tx(&full[st], XL_STAGE);
            bulk_copy_g2s(sm + st * XL_STAGE, Apl + gt_slab(t.y, ch, G.kc), XL_SLAB, &full[st]);
            bulk_copy_g2s(sm + st * XL_STAGE + XL_SLAB, Bpl + gt_slab(t.z, ch, G.kc), XL_SLAB, &full[st]);
        };
        int issued = 0, consumed = 0;
        bool fail = false;
        for (; issued < XL_STAGES && issued < nch; ++issued) load(issued);
        for (int ch = 0; ch < nch; ++ch) {
            const int st = ch % XL_STAGES;
            if (!mbar_wait_bounded(&full[st], (uint32_t)((ch / XL_STAGES) & 1), GT_WAIT_NS)) {
                fail = true;
                break;
            }
            consumed = ch + 1;
            tc_fence_after();
            xl_issue(sbase + st * XL_STAGE, ch == 0, false, false, false, false, hre, him, cre, cim);
            mma_commit(&empty[st]);
            if (ch >= 1 && issued < nch) {
                const int pc = ch - 1;
                if (!mbar_wait_bounded(&empty[pc % XL_STAGES], (uint32_t)((pc / XL_STAGES) & 1), GT_WAIT_NS)) {
                    fail = true;
                    break;
                }
                load(issued++);
            }
        }
        mma_commit(&done);
        if (fail)
            for (int c = consumed; c < issued; ++c)
                mbar_wait_bounded(&full[c % XL_STAGES], (uint32_t)((c / XL_STAGES) & 1), GT_WAIT_NS);
        s_fail = fail;
    }
    __syncthreads();
    const bool fin = mbar_wait_bounded(&done, 0, GT_WAIT_NS);
    if (!__syncthreads_or(!fin || s_fail)) {
        tc_fence_after();
        // warp w drains TMEM lanes 32 (w % 4) .. + 31 (rows), columns 32 (w / 4) .. + 31
        const int quarter = warp & 3, cg = warp >> 2;
        const int lrow = 32 * quarter + lane, R = row0 + lrow;
        const uint32_t lb = (uint32_t)(32 * quarter) << 16;
        for (int g = 0; g < 4; ++g) {
            const int cl = 32 * cg + 8 * g;
            uint32_t a[8], b[8], cc[8], d[8];
            tmem_ld8_nowait(hre + lb + cl, a);
            tmem_ld8_nowait(him + lb + cl, b);
            tmem_ld8_nowait(cre + lb + cl, cc);
            tmem_ld8_nowait(cim + lb + cl, d);
            tmem_wait_ld();
            if (R < rows) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = col0 + cl + c;
                    if (col < G.ncol) {
                        const float us = ldexpf(1.f, -(G.eH + cscale[G.cs + col]));
                        Y[(size_t)col * rows + R] = make_float2((__uint_as_float(a[c]) + __uint_as_float(cc[c])) * us,
                                                                (__uint_as_float(b[c]) + __uint_as_float(d[c])) * us);
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(P.status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, XL_TMEM_COLS);
}

}  // namespace

int grad_gemm_min_m() { return GG_MIN_M; }

int grad_gemm_layout(GgBlock* gb, int ngb, int nc, int S, int tc, int4* tiles, int max_tiles, size_t* elems,
                     size_t* xbytes) {
    size_t off = 0, xb = 0;
    long long cs = 0;
    int nt = 0;
    for (int g = 0; g < ngb; ++g) {
        GgBlock& G = gb[g];
        const size_t vec = (size_t)G.c * S * G.m;
        G.ncol = 2 * G.c * S;
        G.x0 = (long long)off; off += 2 * vec;
        G.x1 = (long long)off; off += 2 * vec;
        G.y = (long long)off; off += 2 * (size_t)(1 + nc) * vec;
        G.z = (long long)off; off += (size_t)(GG_PCAP + 1) * vec;
        G.w = (long long)off; off += (size_t)(GG_PCAP + 1) * nc * vec;
        off = (off + 31) / 32 * 32;
        G.rtc = ((1 + nc) * G.m + XL_TM - 1) / XL_TM;
        G.ctc = (G.ncol + XL_TM - 1) / XL_TM;
        G.kc = (G.m + XL_KC - 1) / XL_KC;
        G.xp = (long long)xb;
        xb += (size_t)G.ctc * G.kc * XL_SLAB;
        G.cs = cs;
        cs += (long long)G.ctc * XL_TM;
        const int rt = tc ? G.rtc : ((1 + nc) * G.m + GG_TILE_R - 1) / GG_TILE_R;
        const int ct = tc ? G.ctc : (G.ncol + GG_TILE_C - 1) / GG_TILE_C;
        for (int a = 0; a < rt; ++a)
            for (int b = 0; b < ct; ++b) {
                if (tiles && nt < max_tiles) tiles[nt] = make_int4(g, a, b, 0);
                ++nt;
            }
    }
    *elems = off;
    if (xbytes) *xbytes = xb;
    return nt;
}

size_t grad_gemm_aux_ints(const GgBlock* gb, int ngb, int S) {
    size_t n = 32 + 2 * (size_t)ngb * S;
    for (int g = 0; g < ngb; ++g) n += (size_t)gb[g].ctc * XL_TM;
    return n;
}

int grad_gemm_hplanes(GgBlock* gb, int ngb, int nc, const double* hmax, size_t* hbytes) {
    size_t off = 0;
    for (int g = 0; g < ngb; ++g) {
        GgBlock& G = gb[g];
        G.rtc = ((1 + nc) * G.m + XL_TM - 1) / XL_TM;
        G.kc = (G.m + XL_KC - 1) / XL_KC;
        G.hp = (long long)off;
        off += (size_t)G.rtc * G.kc * XL_SLAB;
        int e2 = 0;
        std::frexp(hmax[g] > 0.0 ? hmax[g] : 1.0, &e2);  // |entries| < 2^e2
        G.eH = std::max(-60, std::min(60, 14 - e2));
    }
    *hbytes = off;
    return 0;
}

int launch_grad_gemm(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store, double2* partial,
                     const GgBlock* gb, int ngb, const int4* tiles, int ntiles, int S, int* aux, void* scratch,
                     void* xplanes, const void* hplanes, int mode, int min_m, cudaStream_t st) {
    if (P.grad_mode != 0) return 0;
    if (ngb == 0 || mode == GG_OFF) return 0;
    static bool coef_ready = false;
    if (!coef_ready) {
        double f[GG_PCAP + 3];
        double x = 1.0;
        for (int i = 0; i < GG_PCAP + 3; ++i) {
            f[i] = x;
            x /= (double)(i + 1);
        }
        if (cudaMemcpyToSymbol(gg_if, f, sizeof(f)) != cudaSuccess) return -1;
        coef_ready = true;
    }
    const bool tc = mode == GG_TC;
    if (tc && cudaFuncSetAttribute(gg_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(XL_STAGES * XL_STAGE)) != cudaSuccess)
        return -1;
    const int nslices = P.nk < 0 ? P.N : P.nk;
    float2* ws = reinterpret_cast<float2*>(scratch);
    int* Pmax = aux;
    int* own = aux + 32;
    float* lb = reinterpret_cast<float*>(aux + 32 + (size_t)ngb * S);
    int* cscale = aux + 32 + 2 * (size_t)ngb * S;
    unsigned char* xpl = reinterpret_cast<unsigned char*>(xplanes);
    for (int kw0 = 0; kw0 < nslices; kw0 += S) {
        const int nv = std::min(S, nslices - kw0);
        gg_prep_kernel<<<1, 256, 0, st>>>(P, gb, ngb, kw0, S, nv, GF32_SERIES_TOL, 3.0, u, own, lb, Pmax, min_m);
        gg_load_kernel<<<dim3(64, ngb), 256, 0, st>>>(P, gb, kw0, S, reinterpret_cast<const float2*>(psi_store),
                                                      reinterpret_cast<const float2*>(lam_store), own, ws, min_m);
        for (int p = 0; p <= GG_PCAP; ++p) {
            if (tc) {
                gg_planes_kernel<<<dim3(64, ngb), 256, 0, st>>>(P, gb, S, p, Pmax, lb, ws, xpl, cscale, min_m);
                gg_tc_kernel<<<ntiles, GT_THREADS, XL_STAGES * XL_STAGE, st>>>(
                    P, gb, tiles, p, Pmax, reinterpret_cast<const unsigned char*>(hplanes), xpl, cscale, ws, min_m);
            } else {
                gg_gemm_kernel<<<ntiles, GG_THREADS, GG_SMEM, st>>>(P, gb, tiles, p, Pmax, ws, min_m);
            }
            gg_combine_kernel<<<dim3(64, ngb), 256, 0, st>>>(P, gb, kw0, S, p, Pmax, own, u, ws, min_m);
        }
        gg_contract_kernel<<<dim3(nv, ngb), GG_THREADS, 0, st>>>(P, gb, kw0, S, Pmax, own, ws, partial);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

int launch_grad_gemm_hplanes(const GgBlock* gb, int ngb, int nc, const void* H32, const long long* h_off, void* hplanes,
                             int* status, cudaStream_t st) {
    if (ngb == 0) return 0;
    gg_hplanes_kernel<<<dim3(128, ngb), 256, 0, st>>>(gb, reinterpret_cast<const float2*>(H32), nc, h_off,
                                                      reinterpret_cast<unsigned char*>(hplanes), status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
