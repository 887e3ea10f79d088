// Batched slice propagators on the tcgen05 tensor cores (Sec. II.A, Eq. exppropagator).
//
// U = exp(X)^(2^s), X = -i (tau / 2^s) H_k, for blocks of size m <= 112 in FP32 plans.  Every complex
// product runs on the tensor cores through the FP16 hi/lo split of tc_gemm.cuh (all four split
// products per real product, small ones first, FP32 accumulation in tensor memory), and the operands
// stay on chip from one product to the next: the epilogue that drains an accumulator writes the next
// product's operands, already split, straight into shared memory.
//
// Polynomial.  The Taylor polynomial of odd degree 2q-1 is evaluated by Horner's rule in Y = X^2,
//     T(X) = sum_{j<q} (c_{2j} I + c_{2j+1} X) Y^j,   c_k = 1/k!,
// so each step S <- S Y + c_{2j+1} X + c_{2j} I needs only X beside the accumulator, and X stays in
// tensor memory for the whole item: q products for degree 2q-1 (Y, then q-1 Horner steps).  Per
// slice, the norm bound beta = tau (|H0|_2 + sum_j |u_j| |Hc_j|_2) fixes the fewest squarings s that
// bring it under the plan's largest norm, then the lowest odd degree whose truncation bound covers
// beta / 2^s.  With an FP64 squaring chain the squarings run on the CUDA cores.
//
// Layouts.  A product D = A B takes A as an M x K operand (rows of A, K-major) and B as its transpose
// B^T (rows of B^T, K-major), both in 8 x 16-byte core matrices without swizzle.  A transposed copy of
// a result comes from the same product with the operands swapped, (AB)^T = B^T A^T, so every
// epilogue writes rows: Y^T for the Horner steps, (S^2)^T beside S^2 in the squarings; X^T and, before
// the first squaring, S^T come from a product with the identity, so H is read once per slice.
//
// Shared memory: four B^T planes (re hi, re lo, im hi, im lo; NP x NP halves each, NP = m rounded up
// to 16), four A planes, then slack: an MMA with M = 128 reads 128 rows of its A operand, so the rows
// past NP of the last plane read into the slack; the matching accumulator rows are never used.
// Tensor memory: two accumulators of 2 x cs columns (re, im; cs = NP rounded up to a power of two,
// at least 32): R0 at column 0 and R1 at column 2 cs.  R1 holds X during the polynomial.
//
// Scaling.  Each operand is scaled by a power of two 2^e before the split so that its entries stay
// within 2^14 (the FP16 range is 65504): X by its norm bound beta, Y by beta^2, the Horner iterates by
// e^beta, the squaring iterates by 2 (they are unitary up to rounding for Hermitian H).  An entry
// outside the range latches ST_RANGE.  Two FP16 halves hold 22 significant bits; with all four split
// products and the small-first order a product's error is within about 2x that of an FP32 CUDA-core
// product (the accumulator's own rounding is most of the rest).
#include <cuda_fp16.h>

#include "../../include/qoc.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace qoc {
namespace {

constexpr int XT_THREADS = 512;  // 16 warps: warp w drains TMEM lanes 32 (w % 4).., column groups w / 4 + 4 t
constexpr int XT_GSTRIDE = XT_THREADS / 128;  // warps sharing a TMEM lane quarter
constexpr int XT_MAXM = 112;
constexpr uint64_t XT_WAIT_NS = 2000000000ull;

__host__ __device__ inline int xt_pad16(int m) { return (m + 15) / 16 * 16; }
__host__ __device__ inline int xt_cs(int NP) {
    int c = 32;
    while (c < NP) c <<= 1;
    return c;
}
// dynamic shared memory of one CTA for operand size NP: 8 planes + the overread slack
__host__ __device__ inline size_t xt_smem(int NP) { return ((size_t)8 * NP * NP + (size_t)(128 - NP) * NP) * 2; }

// Split 8 values (scaled by sig) into FP16 hi and lo parts, packed two per word in column order; a
// pair converts in one instruction each way.  bad is set if a scaled value leaves the FP16 range.
__device__ __forceinline__ void split8(const float (&v)[8], float sig, uint4& hi, uint4& lo, bool& bad) {
    uint32_t h[4], l[4];
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = v[2 * i] * sig, b = v[2 * i + 1] * sig;
        mx = fmaxf(mx, fmaxf(fabsf(a), fabsf(b)));
        const __half2 hh = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(a - hf.x, b - hf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&hh);
        l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    bad |= !(mx <= 65504.f);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Write row r, columns 8g..8g+7 of a complex matrix into the four planes starting at byte offset grp.
__device__ __forceinline__ void put8(unsigned char* sm, uint32_t grp, uint32_t plane, int NP, int r, int g,
                                     const float (&re)[8], const float (&im)[8], float sig, bool& bad) {
    const uint32_t off = (uint32_t)((((r >> 3) * (NP >> 3) + g) << 6) + ((r & 7) << 3)) * 2u;
    uint4 hi, lo;
    split8(re, sig, hi, lo, bad);
    *reinterpret_cast<uint4*>(sm + grp + off) = hi;
    *reinterpret_cast<uint4*>(sm + grp + plane + off) = lo;
    split8(im, sig, hi, lo, bad);
    *reinterpret_cast<uint4*>(sm + grp + 2 * plane + off) = hi;
    *reinterpret_cast<uint4*>(sm + grp + 3 * plane + off) = lo;
}

// Row r, columns 8g..8g+7 of the identity into one FP16 plane (at byte offset pl).
__device__ __forceinline__ void put_ident8(unsigned char* sm, uint32_t pl, int NP, int r, int g) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t lo16 = (8 * g + 2 * i == r) ? 0x3C00u : 0u;  // FP16 1.0
        const uint32_t hi16 = (8 * g + 2 * i + 1 == r) ? 0x3C00u : 0u;
        w[i] = lo16 | (hi16 << 16);
    }
    const uint32_t off = (uint32_t)((((r >> 3) * (NP >> 3) + g) << 6) + ((r & 7) << 3)) * 2u;
    *reinterpret_cast<uint4*>(sm + pl + off) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Read columns col..col+7 of the re and im planes of an accumulator (one TMEM lane per thread).
__device__ __forceinline__ void ld_acc8(uint32_t t_re, uint32_t t_im, float (&re)[8], float (&im)[8]) {
    uint32_t a[8], b[8];
    tmem_ld8_nowait(t_re, a);
    tmem_ld8_nowait(t_im, b);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        re[i] = __uint_as_float(a[i]);
        im[i] = __uint_as_float(b[i]);
    }
}

// One thread: D(re at d_re, im at d_im) = A B for the complex operands whose plane groups start at
// shared addresses a and b (A as rows, B as rows of B^T), four split products per real product, or
// three (no lo*lo) when LL is false.
template <bool LL = true>
__device__ __forceinline__ void issue_cprod(uint32_t a, uint32_t b, uint32_t plane, int NP, uint32_t d_re,
                                            uint32_t d_im) {
    const uint32_t lbo = 128, sbo = (uint32_t)(NP >> 3) * 128u;
    const uint32_t pos = idesc_f16(128, NP, false), neg = idesc_f16(128, NP, true);
    // descriptors advance by adding byte offsets / 16 to the start-address field (shared addresses
    // stay below 2^18 bytes, so the 14-bit field never carries)
    const uint64_t dA = smem_desc_u32(a, lbo, sbo), dB = smem_desc_u32(b, lbo, sbo);
    const uint64_t pl = plane >> 4;
    // (lo,lo), (hi,lo), (lo,hi) first, (hi,hi) last: the accumulator rounds each addition relative to
    // its running magnitude, so the small terms are summed while it is still small and only the K/16
    // large (hi,hi) additions meet a large accumulator.  Dropping lo*lo would bias products such as
    // X X, whose lo parts are correlated; in a Horner step S Y (unrelated operands) its terms average
    // out like rounding noise and it is left out.
    constexpr int t0 = LL ? 0 : 1;
#pragma unroll 1
    for (int t = t0; t < 4; ++t) {
        const int ha = !(t & 1), hb = t < 2;  // lo parts at plane offset 1: (1,1), (0,1), (1,0), (0,0)
        const uint64_t ar0 = dA + ha * pl, ai0 = dA + (2 + ha) * pl;
        const uint64_t br0 = dB + hb * pl, bi0 = dB + (2 + hb) * pl;
        for (int kk = 0; kk < NP / 16; ++kk) {
            const uint64_t st = (uint64_t)kk * 16u;  // 256 bytes: two core matrices along K
            const int acc = (kk > 0 || t > t0);
            // the two accumulators alternate, so that consecutive MMAs do not chain on one another
            mma_f16(d_re, ar0 + st, br0 + st, pos, acc);
            mma_f16(d_im, ar0 + st, bi0 + st, pos, acc);
            mma_f16(d_re, ai0 + st, bi0 + st, neg, 1);
            mma_f16(d_im, ai0 + st, br0 + st, pos, 1);
        }
    }
}

// One thread: D = I_part B, with the identity (hi plane only) at shared address id and B's planes at
// b: D = B^T, exactly the split sum hi + lo of each entry.
__device__ __forceinline__ void issue_ident(uint32_t id, uint32_t b, uint32_t plane, int NP, uint32_t d_re,
                                            uint32_t d_im) {
    const uint32_t lbo = 128, sbo = (uint32_t)(NP >> 3) * 128u;
    const uint32_t pos = idesc_f16(128, NP, false);
    for (int kk = 0; kk < NP / 16; ++kk) {
        const uint32_t step = (uint32_t)kk * 256u;
        const uint64_t ai = smem_desc_u32(id + step, lbo, sbo);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int acc = (kk > 0 || h > 0);
            mma_f16(d_re, ai, smem_desc_u32(b + h * plane + step, lbo, sbo), pos, acc);
            mma_f16(d_im, ai, smem_desc_u32(b + (2 + h) * plane + step, lbo, sbo), pos, acc);
        }
    }
}

// power-of-two scale exponent for entries bounded by 'bound': 14 - ceil(log2(bound)), clamped
__device__ __forceinline__ int xt_clamp_exp(int e) { return e < -30 ? -30 : (e > 40 ? 40 : e); }
__device__ __forceinline__ int xt_exp_for(double bound) {
    if (!(bound > 0.0)) return 40;
    int ex;
    const double mant = frexp(bound, &ex);  // bound = mant 2^ex, mant in [0.5, 1)
    return xt_clamp_exp(14 - (mant > 0.5 ? ex : ex - 1));
}
// the same from log2(bound)
__device__ __forceinline__ int xt_exp_for_log2(double lg) {
    if (!(lg > -1e300)) return 40;
    return xt_clamp_exp(14 - (int)ceil(lg));
}

// Xs[r LD + c] = -i sc (H0 + sum_j u_j Hc_j)[r][c] for every entry of an m x m block: consecutive
// threads take consecutive entries (coalesced), eight per thread at a time with all 8 (1 + NC) loads
// issued before any is used (NC: controls, -1 = nc_rt at run time).
template <int NC>
__device__ __forceinline__ void stage_x(float2* Xs, const float2* H, const float* uf, size_t mm, int m, int LD, float sc,
                                        int nc_rt = 0) {
    constexpr int NB = 4;
    constexpr int NH = NC > 0 ? NC : 1;
    for (size_t e0 = threadIdx.x; e0 < mm; e0 += (size_t)NB * XT_THREADS) {
        float2 h[NB];
        float2 hc[NH][NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const size_t e = e0 + (size_t)i * XT_THREADS;
            h[i] = e < mm ? H[e] : make_float2(0.f, 0.f);
            if (NC > 0) {
#pragma unroll
                for (int j = 0; j < NH; ++j)
                    hc[j][i] = (e < mm && j < NC) ? H[(size_t)(1 + j) * mm + e] : make_float2(0.f, 0.f);
            }
        }
        if (NC > 0) {
#pragma unroll
            for (int j = 0; j < NH; ++j)
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    h[i].x = fmaf(uf[j], hc[j][i].x, h[i].x);
                    h[i].y = fmaf(uf[j], hc[j][i].y, h[i].y);
                }
        } else if (NC < 0) {
            for (int j = 0; j < nc_rt; ++j)
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const size_t e = e0 + (size_t)i * XT_THREADS;
                    if (e < mm) {
                        const float2 v = H[(size_t)(1 + j) * mm + e];
                        h[i].x = fmaf(uf[j], v.x, h[i].x);
                        h[i].y = fmaf(uf[j], v.y, h[i].y);
                    }
                }
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const size_t e = e0 + (size_t)i * XT_THREADS;
            if (e < mm) {
                const int r = (int)(e / (size_t)m), c = (int)(e - (size_t)r * m);
                Xs[(size_t)r * LD + c] = make_float2(h[i].y * sc, -h[i].x * sc);
            }
        }
    }
}

// Make this thread's shared-memory operand writes visible to the tensor cores and its TMEM reads
// complete, then meet the other threads.
__device__ __forceinline__ void xt_sync() {
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
}

__global__ void __launch_bounds__(XT_THREADS, 1)
expm_tc_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks, int n_cls,
               const int2* __restrict__ cls_items, long long n_cls_items, void* __restrict__ Uout,
               char* __restrict__ scratch, size_t slot_bytes, int m_max, uint32_t tmem_cols, int all_items) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float s_uf[8];
    __shared__ float s_c[36];  // 1/k!
    __shared__ int s_q, s_s, s_eX, s_eY, s_eS;
    __shared__ float s_sc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, gq = warp >> 2;  // gq: this warp's first column group
    const int r = 32 * quarter + lane;  // accumulator row (TMEM lane) this thread drains
    const uint32_t lane_bits = (uint32_t)(32 * quarter) << 16;
    if (warp == 0) {
        tmem_alloc(&tslot, tmem_cols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        double f = 1.0;
        for (int i = 0; i < 36; ++i) {
            s_c[i] = (float)f;
            f /= (double)(i + 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const uint32_t cs = tmem_cols / 4;
    const uint32_t T0re = tmem, T0im = tmem + cs, T1re = tmem + 2 * cs, T1im = tmem + 3 * cs;  // MMA targets
    const uint32_t R0re = T0re + lane_bits, R0im = T0im + lane_bits;  // this warp's lanes
    const uint32_t R1re = T1re + lane_bits, R1im = T1im + lane_bits;
    const uint32_t sm_base = smem_u32(sm);
    uint32_t phase = 0;
    bool failed = false, bad = false;

    const size_t mm_max = (size_t)m_max * m_max;
    double2* D0 = reinterpret_cast<double2*>(scratch + (size_t)blockIdx.x * slot_bytes);
    double2* D1 = D0 + mm_max;

    // wait for the commit of the MMAs just issued; false if it did not arrive in time
    auto mma_wait = [&]() -> bool {
        const bool ok = mbar_wait_bounded(&bar, phase, XT_WAIT_NS);
        if (__syncthreads_or(!ok)) return false;
        phase ^= 1u;
        tc_fence_after();
        return true;
    };

    const bool whole = P.nk < 0;
    const long long total = whole ? n_cls_items : (long long)n_cls * P.nk;
    __shared__ int s_list[XT_THREADS];
    __shared__ int s_nl;
    __shared__ int s_wc[32];
    // slices this launch owns: all of them, or those that need no squaring
    // (the norm bound and the pulses of each tested slice are kept for the setup below)
    __shared__ double s_beta[XT_THREADS];
    __shared__ float s_ul[XT_THREADS][8];
    __shared__ unsigned char s_nan[XT_THREADS];
    auto want = [&](long long it) -> bool {
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
        const DevBlock& Bw = P.blocks[bi];
        const double beta = slice_beta(P, Bw, u, k);
        int nan = 0;
        for (int j = 0; j < P.nc; ++j) {
            const double x = u[(size_t)(Bw.u_row + k) * P.nc + j];
            const int fin = isfinite(x);
            nan |= !fin;
            s_ul[threadIdx.x][j] = fin ? (float)x : 0.f;
        }
        s_beta[threadIdx.x] = beta;
        s_nan[threadIdx.x] = (unsigned char)nan;
        return all_items || slice_halvings(beta, tabs.theta_cap, P.max_sq) == 0;
    };
    for (long long lb = 0; !failed && cta_select(total, lb, want, s_list, &s_nl, s_wc); lb += blockDim.x) {
        const int nl = s_nl;
        for (int li = 0; li < nl && !failed; ++li) {
            const long long item = (long long)blockIdx.x + (lb + s_list[li]) * gridDim.x;
            int bi, kw, k;
            if (whole) {
                const int2 it = cls_items[item];
                bi = it.x;
                kw = it.y;
                k = it.y;
            } else {
                bi = cls_blocks[item / P.nk];
                kw = (int)(item % P.nk);
                k = P.k0 + kw;
            }
            const DevBlock& B = P.blocks[bi];
            const int m = B.m, NP = xt_pad16(m), nkg = NP / 8;
            const size_t mm = (size_t)m * m;
            const uint32_t plane = (uint32_t)NP * NP * 2u;
            const uint32_t oBT = 0, oA = 4 * plane;  // plane groups (byte offsets)
            const uint32_t aBT = sm_base + oBT, aA = sm_base + oA;
            if (threadIdx.x == 0) {
                const int ti = s_list[li];  // the thread that tested this slice
                for (int j = 0; j < P.nc; ++j) s_uf[j] = s_ul[ti][j];
                if (s_nan[ti]) atomicOr(P.status, ST_NAN_PULSE);
                const double beta = s_beta[ti];
                // Fewest squarings: each one doubles the error of what it squares, and a squaring here
                // errs more than an FP32 one, so scaling further than the plan's largest norm loses
                // more than the lower-degree polynomial gains.
                const double cap = tabs.theta_cap;
                int smin = 0;
                double b = beta;
                while (b > cap && smin < P.max_sq) { b *= 0.5; ++smin; }
                if (b > tabs.theta_cap) atomicOr(P.status, ST_SQUARING_CAP);
                // fewest squarings (each one doubles the rounding error of the polynomial), then the
                // lowest odd degree whose truncation bound covers the scaled norm
                const int bs = smin;
                int bq = 1;
                while (bq < 16 && tabs.theta_odd[bq - 1] < ldexp(beta, -bs)) ++bq;
                const double bsn = ldexp(beta, -bs);
                s_q = bq;
                s_s = bs;
                s_sc = (float)ldexp(B.dt, -bs);
                s_eX = xt_exp_for(bsn);
                s_eY = xt_exp_for(bsn * bsn);
                s_eS = xt_exp_for_log2(bsn * 1.4426950408889634);  // e^beta: log2 = beta / ln 2
                if (P.stats) {
                    const unsigned long long m3 = (unsigned long long)m * m * m;
                    atomicAdd(P.stats + 0, m3 * (unsigned long long)(bq >= 2 ? bq : 0));
                    atomicAdd(P.stats + 1, m3 * (unsigned long long)bs);
                    atomicAdd(P.stats + 2, 1ull);
                    if (bq >= 2) atomicAdd(P.stats + 5, m3 * (unsigned long long)(bq - 1));  // Horner: 3 split terms
                }
            }
            __syncthreads();
            const int q = s_q, s = s_s;
            const int eX = s_eX, eY = s_eY, eS = s_eS, eQ = 13;
            const bool sq64 = s > 0 && tabs.sq_f64;
            float2* Uo = reinterpret_cast<float2*>(Uout) + B.u_off + (size_t)kw * B.mmp;

            // ---- X = -i (tau / 2^s)(H0 + sum_j u_j Hc_j), H read once and coalesced into an FP32 buffer
            // in the B^T planes (free until the transpose; odd row stride, so that the column reads
            // below are free of bank conflicts); then every thread moves its rows into the A planes
            // (split) and R1 (FP32)
            {
                const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;
                const float sc = s_sc, sig = ldexpf(1.f, eX);
                float2* Xs = reinterpret_cast<float2*>(sm + oBT);
                const int LD = (m & 1) || m == NP ? m : m + 1;  // LD * m * 8 <= 4 NP^2 * 2 bytes
                switch (P.nc) {
                    case 0: stage_x<0>(Xs, H, s_uf, mm, m, LD, sc); break;
                    case 1: stage_x<1>(Xs, H, s_uf, mm, m, LD, sc); break;
                    case 2: stage_x<2>(Xs, H, s_uf, mm, m, LD, sc); break;
                    case 3: stage_x<3>(Xs, H, s_uf, mm, m, LD, sc); break;
                    case 4: stage_x<4>(Xs, H, s_uf, mm, m, LD, sc); break;
                    default: stage_x<-1>(Xs, H, s_uf, mm, m, LD, sc, P.nc);
                }
                __syncthreads();
                for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                    float xr[8], xi[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int col = 8 * g + c;
                        const float2 x = (r < m && col < m) ? Xs[(size_t)r * LD + col] : make_float2(0.f, 0.f);
                        xr[c] = x.x;
                        xi[c] = x.y;
                    }
                    if (r < NP) put8(sm, oA, plane, NP, r, g, xr, xi, sig, bad);
                    tmem_st8(R1re + 8 * g, xr);
                    tmem_st8(R1im + 8 * g, xi);
                }
                tmem_wait_st();
                __syncthreads();  // the buffer is consumed: the identity may take its place
                if (q >= 2 && r < NP)
                    for (int g = gq; g < nkg; g += XT_GSTRIDE) put_ident8(sm, oBT, NP, r, g);  // for I X
                xt_sync();
            }
            // X^T (rows into the B^T planes), needed by the Horner steps: the product I X on the tensor
            // cores, exactly the split sum of each entry, replaces a second, transposed read of H
            if (q >= 2) {
                if (threadIdx.x == 0) {
                    tc_fence_after();
                    issue_ident(aBT, aA, plane, NP, T0re, T0im);
                    mma_commit(&bar);
                }
                if (!mma_wait()) { failed = true; break; }
                for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                    float dr[8], di[8];
                    ld_acc8(R0re + 8 * g, R0im + 8 * g, dr, di);
                    if (r < NP) put8(sm, oBT, plane, NP, r, g, dr, di, 1.f, bad);
                }
                xt_sync();
            }

            // last polynomial value of row r, columns 8g..: to U, to the FP64 chain, or into the operands
            // of the first squaring (A planes, and the identity into the first B^T plane)
            auto finish8 = [&](int g, const float (&vr)[8], const float (&vi)[8]) {
                if (s == 0) {
                    if (r < m) {
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (8 * g + c < m) Uo[(size_t)r * m + 8 * g + c] = make_float2(vr[c], vi[c]);
                    }
                } else if (sq64) {
                    if (r < m) {
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (8 * g + c < m) D0[(size_t)r * m + 8 * g + c] = make_double2(vr[c], vi[c]);
                    }
                } else if (r < NP) {
                    put8(sm, oA, plane, NP, r, g, vr, vi, ldexpf(1.f, eQ), bad);
                    put_ident8(sm, oBT, NP, r, g);
                }
            };

            // ---- polynomial: Y^T = X^T X^T, then Horner in Y
            if (q >= 2) {
                if (threadIdx.x == 0) {
                    tc_fence_after();
                    issue_cprod(aBT, aA, plane, NP, T0re, T0im);
                    mma_commit(&bar);
                }
                if (!mma_wait()) { failed = true; break; }
                {
                    const float fY = ldexpf(1.f, -2 * eX), sigY = ldexpf(1.f, eY), sigS = ldexpf(1.f, eS);
                    const float c1 = s_c[2 * q - 1], c0 = s_c[2 * q - 2];
                    for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                        float dr[8], di[8], xr[8], xi[8];
                        ld_acc8(R0re + 8 * g, R0im + 8 * g, dr, di);
                        ld_acc8(R1re + 8 * g, R1im + 8 * g, xr, xi);
                        if (r < NP) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                dr[c] *= fY;
                                di[c] *= fY;
                            }
                            put8(sm, oBT, plane, NP, r, g, dr, di, sigY, bad);
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                dr[c] = c1 * xr[c] + ((8 * g + c == r && r < m) ? c0 : 0.f);
                                di[c] = c1 * xi[c];
                            }
                            put8(sm, oA, plane, NP, r, g, dr, di, sigS, bad);
                        }
                    }
                    xt_sync();
                }
                for (int j = q - 2; j >= 0 && !failed; --j) {
                    if (threadIdx.x == 0) {
                        tc_fence_after();
                        issue_cprod<false>(aA, aBT, plane, NP, T0re, T0im);
                        mma_commit(&bar);
                    }
                    if (!mma_wait()) { failed = true; break; }
                    const float f = ldexpf(1.f, -(eS + eY)), sigS = ldexpf(1.f, eS);
                    const float c1 = s_c[2 * j + 1], c0 = s_c[2 * j];
                    // two column groups per TMEM wait: 8 loads in flight, then the arithmetic
                    for (int g = gq; g < nkg; g += 2 * XT_GSTRIDE) {
                        const int gg[2] = {g, g + XT_GSTRIDE};
                        const bool two = gg[1] < nkg;  // warp-uniform
                        uint32_t ld[2][4][8];
                        tmem_ld8_nowait(R0re + 8 * gg[0], ld[0][0]);
                        tmem_ld8_nowait(R0im + 8 * gg[0], ld[0][1]);
                        tmem_ld8_nowait(R1re + 8 * gg[0], ld[0][2]);
                        tmem_ld8_nowait(R1im + 8 * gg[0], ld[0][3]);
                        if (two) {
                            tmem_ld8_nowait(R0re + 8 * gg[1], ld[1][0]);
                            tmem_ld8_nowait(R0im + 8 * gg[1], ld[1][1]);
                            tmem_ld8_nowait(R1re + 8 * gg[1], ld[1][2]);
                            tmem_ld8_nowait(R1im + 8 * gg[1], ld[1][3]);
                        }
                        tmem_wait_ld();
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (h == 1 && !two) break;
                            float dr[8], di[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                const float xr = __uint_as_float(ld[h][2][c]), xi = __uint_as_float(ld[h][3][c]);
                                dr[c] = fmaf(__uint_as_float(ld[h][0][c]), f, c1 * xr) +
                                        ((8 * gg[h] + c == r && r < m) ? c0 : 0.f);
                                di[c] = fmaf(__uint_as_float(ld[h][1][c]), f, c1 * xi);
                            }
                            if (j > 0) {
                                if (r < NP) put8(sm, oA, plane, NP, r, gg[h], dr, di, sigS, bad);
                            } else {
                                finish8(gg[h], dr, di);
                            }
                        }
                    }
                    xt_sync();
                }
                if (failed) break;
            } else {
                // degree 1: T(X) = I + X
                for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                    float xr[8], xi[8];
                    ld_acc8(R1re + 8 * g, R1im + 8 * g, xr, xi);
#pragma unroll
                    for (int c = 0; c < 8; ++c) xr[c] += (8 * g + c == r && r < m) ? 1.f : 0.f;
                    finish8(g, xr, xi);
                }
                xt_sync();
            }

            // ---- squarings
            if (s > 0 && !sq64) {
                // S^T from the product with the identity, into the B^T planes (scale carried over)
                if (threadIdx.x == 0) {
                    tc_fence_after();
                    issue_ident(aBT, aA, plane, NP, T1re, T1im);
                    mma_commit(&bar);
                }
                if (!mma_wait()) { failed = true; break; }
                for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                    float dr[8], di[8];
                    ld_acc8(R1re + 8 * g, R1im + 8 * g, dr, di);
                    if (r < NP) put8(sm, oBT, plane, NP, r, g, dr, di, 1.f, bad);
                }
                xt_sync();
                const float f = ldexpf(1.f, -2 * eQ), sigQ = ldexpf(1.f, eQ);
                for (int i = 1; i <= s && !failed; ++i) {
                    const bool last = i == s;
                    if (threadIdx.x == 0) {
                        tc_fence_after();
                        issue_cprod(aA, aBT, plane, NP, T0re, T0im);                // S^2
                        if (!last) issue_cprod(aBT, aA, plane, NP, T1re, T1im);    // (S^2)^T
                        mma_commit(&bar);
                    }
                    if (!mma_wait()) { failed = true; break; }
                    for (int g = gq; g < nkg; g += XT_GSTRIDE) {
                        float dr[8], di[8];
                        ld_acc8(R0re + 8 * g, R0im + 8 * g, dr, di);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            dr[c] *= f;
                            di[c] *= f;
                        }
                        if (last) {
                            if (r < m) {
#pragma unroll
                                for (int c = 0; c < 8; ++c)
                                    if (8 * g + c < m) Uo[(size_t)r * m + 8 * g + c] = make_float2(dr[c], di[c]);
                            }
                        } else {
                            float tr[8], ti[8];
                            ld_acc8(R1re + 8 * g, R1im + 8 * g, tr, ti);
                            if (r < NP) {
                                put8(sm, oA, plane, NP, r, g, dr, di, sigQ, bad);
#pragma unroll
                                for (int c = 0; c < 8; ++c) {
                                    tr[c] *= f;
                                    ti[c] *= f;
                                }
                                put8(sm, oBT, plane, NP, r, g, tr, ti, sigQ, bad);
                            }
                        }
                    }
                    xt_sync();
                }
                if (failed) break;
            } else if (sq64) {
                // FP64 squaring chain on the CUDA cores
                double2* Da = D0;
                double2* Db = D1;
                for (int i = 0; i < s; ++i) {
                    for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                        const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
                        double2 acc = make_double2(0.0, 0.0);
                        for (int kk = 0; kk < m; ++kk) {
                            const double2 a = Da[(size_t)row * m + kk], b = Da[(size_t)kk * m + col];
                            acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
                            acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
                        }
                        Db[e] = acc;
                    }
                    __syncthreads();
                    double2* t = Da;
                    Da = Db;
                    Db = t;
                }
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Uo[e] = make_float2((float)Da[e].x, (float)Da[e].y);
                __syncthreads();
            }
        }
    }
    if (bad) atomicOr(P.status, ST_RANGE);
    if (failed) {
        // the commit never arrived: give the MMAs in flight another bounded wait before freeing TMEM
        if (threadIdx.x == 0) {
            atomicOr(P.status, ST_TIMEOUT);
            mbar_wait_bounded(&bar, phase, XT_WAIT_NS);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// Launch shape of a class whose largest block is m_max: dynamic shared memory (raised, if need be,
// so that no more CTAs share an SM than its tensor memory holds), TMEM columns, CTAs per SM.
struct XtConfig {
    size_t smem;
    uint32_t tmem_cols;
    int per_sm;
};

XtConfig xt_config(int m_max) {
    XtConfig c{};
    const int NP = xt_pad16(m_max);
    c.smem = xt_smem(NP);
    c.tmem_cols = 4u * (uint32_t)xt_cs(NP);
    const int by_tmem = (int)(512u / c.tmem_cols);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, expm_tc_kernel);
    const size_t per_sm_smem = 233472, reserved = 1024;  // 228 KB per SM, 1 KB reserved per CTA
    const size_t need = c.smem + fa.sharedSizeBytes + reserved;
    int by_smem = (int)(per_sm_smem / need);
    const int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * XT_THREADS) : 1;
    int k = std::min(std::min(by_tmem, by_smem), std::max(by_regs, 1));
    if (k < 1) k = 1;
    if (by_smem > k) {  // raise the request until only k CTAs fit
        const size_t want = per_sm_smem / (size_t)(k + 1) + 16;
        if (want > fa.sharedSizeBytes + reserved) c.smem = std::max(c.smem, want - fa.sharedSizeBytes - reserved);
    }
    c.per_sm = k;
    return c;
}

}  // namespace

int expm_tc_supported(int prec, int m) { return prec != QOC_PREC_F64 && m >= 1 && m <= XT_MAXM; }

size_t expm_tc_slot_bytes(int m_max) { return (size_t)2 * m_max * m_max * sizeof(double2); }

int expm_tc_grid_limit(int m_max) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * xt_config(m_max).per_sm;
}

int launch_expm_tc(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                   const int2* items, long long n_items, void* Uout, char* scratch, size_t slot_bytes, int m_max,
                   int grid, cudaStream_t st, int all_items) {
    if (m_max > XT_MAXM) return -1;
    const XtConfig c = xt_config(m_max);
    if (cudaFuncSetAttribute(expm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem) != cudaSuccess)
        return -1;
    expm_tc_kernel<<<grid, XT_THREADS, c.smem, st>>>(P, tabs, u, cls, n_cls, items, n_items, Uout, scratch, slot_bytes,
                                                     m_max, c.tmem_cols, all_items);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
