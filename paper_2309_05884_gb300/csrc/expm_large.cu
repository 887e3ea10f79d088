// Batched slice propagators of large blocks (m > 112, up to 2048) on the tcgen05 tensor cores
// (Sec. II.A, Eq. exppropagator), for the slices that need no squaring.
//
// The Taylor polynomial of odd degree 2q-1 is evaluated by Horner's rule in Y = X^2 (as in
// expm_tc.cu), T(X) = sum_{j<q} (c_{2j} I + c_{2j+1} X) Y^j, but a block no longer fits one CTA: every
// product is a batched tiled GEMM launch over (128 x 128 output tile, slice), with the matrices of
// a chunk of slices in a global scratch area (X, Y and two Horner iterates per slice, FP32).
//   xl_prep      per slice: norm bound, Taylor degree, power-of-two operand scales, ownership (slices
//                that need squarings are left to the CUDA-core tiles);
//   xl_assemble  X = -i tau (H0 + sum_j u_j Hc_j);
//   xl_gemm      Y = X X, then S <- S Y + c_{2j+1} X + c_{2j} I for j = q-2 .. 0 (a slice joins at its
//                own first step, where S = c_{2q-1} X + c_{2q-2} I is formed while staging);
//   xl_export    U = T(X) into the propagator store.
// GEMM tile: one CTA of 512 threads, M = N = 128, K in chunks of 32 through two shared-memory stages.
// Each stage holds the FP16 hi/lo split of a 128 x 32 slab of A (rows, K-major) and of B^T (rows of
// B^T, staged transposed from B's rows), with the power-of-two operand scales of the slice; the MMAs
// of a chunk run while the next chunk is staged.  The (hi,hi) products accumulate in one pair of TMEM
// accumulators and the three smaller split products in another, added in FP32 at the end: with K up
// to 2048 the small terms are never rounded against the large running sum.
#include <cuda_fp16.h>

#include <algorithm>

#include "../../include/qoc.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace qoc {
namespace {

constexpr int XL_THREADS = 512;
constexpr int XL_TM = 128, XL_TN = 128, XL_KC = 32;
constexpr uint64_t XL_WAIT_NS = 2000000000ull;
constexpr uint32_t XL_TMEM_COLS = 512;  // re, im of the (hi,hi) and of the correction accumulators

// 1/k!, k = 0..35 (Taylor coefficients)
__constant__ float xl_coef[36] = {
    1.000000000e+00f, 1.000000000e+00f, 5.000000000e-01f, 1.666666667e-01f,
    4.166666667e-02f, 8.333333333e-03f, 1.388888889e-03f, 1.984126984e-04f,
    2.480158730e-05f, 2.755731922e-06f, 2.755731922e-07f, 2.505210839e-08f,
    2.087675699e-09f, 1.605904384e-10f, 1.147074560e-11f, 7.647163732e-13f,
    4.779477332e-14f, 2.811457254e-15f, 1.561920697e-16f, 8.220635247e-18f,
    4.110317623e-19f, 1.957294106e-20f, 8.896791392e-22f, 3.868170171e-23f,
    1.611737571e-24f, 6.446950284e-26f, 2.479596263e-27f, 9.183689864e-29f,
    3.279889237e-30f, 1.130996289e-31f, 3.769987629e-33f, 1.216125042e-34f,
    3.800390755e-36f, 1.151633562e-37f, 3.387157536e-39f, 9.677592959e-41f};

// per slice of a chunk
struct XlItem {
    int bi, kw, k;   // block, window slot, slice (0-based)
    int q;           // Taylor degree 2q-1
    int own;         // 1: no squaring needed, this path owns the slice
    int eX, eY, eS;  // power-of-two scales of X, Y and the Horner iterates
    float sc;        // tau (no squarings)
};

// one FP16 plane slab [rows][XL_KC] in the K-major no-swizzle core layout: element (row, k)
__device__ __forceinline__ int xl_off(int row, int k) { return (((row >> 3) * (XL_KC >> 3) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7); }

__device__ __forceinline__ void xl_split(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// Prep: one thread per slice of the chunk [i0, i0 + n) of the class's item range.
__global__ void xl_prep_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks,
                               const int2* __restrict__ cls_items, long long i0, int n, XlItem* __restrict__ items) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long it = i0 + t;
    XlItem X{};
    if (P.nk < 0) {
        const int2 e = cls_items[it];
        X.bi = e.x;
        X.kw = e.y;
        X.k = e.y;
    } else {
        X.bi = cls_blocks[it / P.nk];
        X.kw = (int)(it % P.nk);
        X.k = P.k0 + X.kw;
    }
    const DevBlock& B = P.blocks[X.bi];
    const double beta = slice_beta(P, B, u, X.k);
    int nan = 0;
    for (int j = 0; j < P.nc; ++j) nan |= !isfinite(u[(size_t)(B.u_row + X.k) * P.nc + j]);
    const int s = slice_halvings(beta, tabs.theta_cap, P.max_sq);
    X.own = s == 0;
    if (X.own) {
        if (nan) atomicOr(P.status, ST_NAN_PULSE);
        int q = 1;
        while (q < 16 && tabs.theta_odd[q - 1] < beta) ++q;
        X.q = q;
        auto ex = [](double bound) {
            if (!(bound > 0.0)) return 40;
            int e2;
            const double mant = frexp(bound, &e2);
            const int e = 14 - (mant > 0.5 ? e2 : e2 - 1);
            return e < -30 ? -30 : (e > 40 ? 40 : e);
        };
        X.eX = ex(beta);
        X.eY = ex(beta * beta);
        const int lg = (int)ceil(beta * 1.4426950408889634);  // log2 e^beta
        X.eS = 14 - lg < -30 ? -30 : (14 - lg > 40 ? 40 : 14 - lg);
        X.sc = (float)B.dt;
        if (P.stats) {
            const unsigned long long m3 = (unsigned long long)B.m * B.m * B.m;
            atomicAdd(P.stats + 0, m3 * (unsigned long long)(q >= 2 ? q : 0));
            atomicAdd(P.stats + 2, 1ull);
        }
    }
    items[t] = X;
}

// X = -i sc (H0 + sum_j u_j Hc_j) for every owned slice: grid (chunks of entries, slice).
__global__ void xl_assemble_kernel(DevPlan P, const double* __restrict__ u, const XlItem* __restrict__ items,
                                   float2* __restrict__ scratch, size_t slot) {
    const XlItem& X = items[blockIdx.y];
    if (!X.own) return;
    const DevBlock& B = P.blocks[X.bi];
    const int m = B.m;
    const size_t mm = (size_t)m * m;
    const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;
    float uf[8];
    for (int j = 0; j < P.nc; ++j) {
        const double x = u[(size_t)(B.u_row + X.k) * P.nc + j];
        uf[j] = isfinite(x) ? (float)x : 0.f;
    }
    float2* Xm = scratch + (size_t)blockIdx.y * 4 * slot;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
        float2 h = H[e];
        for (int j = 0; j < P.nc; ++j) {
            const float2 hc = H[(size_t)(1 + j) * mm + e];
            h.x = fmaf(uf[j], hc.x, h.x);
            h.y = fmaf(uf[j], hc.y, h.y);
        }
        Xm[e] = make_float2(h.y * X.sc, -h.x * X.sc);
    }
}

// One K chunk [k0, k0 + XL_KC) of the A rows [row0, row0 + 128) and of the B^T rows (B columns)
// [col0, col0 + 128), held in registers between its load and its store into a stage: each thread
// loads 8 consecutive k of one A row (thread t: row t / 4) and 8 consecutive rows of B at one column
// (t % 128; coalesced along the columns).  Entries outside the m x m matrix are 0; A is
// S_init = c1 X + c0 I when init (X in Asrc).
struct XlRegs {
    float2 a[8], b[8];
};

__device__ __forceinline__ void xl_load(XlRegs& R, const float2* __restrict__ Asrc, const float2* __restrict__ Bsrc,
                                        int m, int row0, int col0, int k0, bool init, float c1, float c0) {
    const int t = threadIdx.x;
    {
        const int r = row0 + (t >> 2), kb = k0 + (t & 3) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = kb + c;
            float2 v = make_float2(0.f, 0.f);
            if (r < m && k < m) {
                v = Asrc[(size_t)r * m + k];
                if (init) {
                    v.x = c1 * v.x + (r == k ? c0 : 0.f);
                    v.y = c1 * v.y;
                }
            }
            R.a[c] = v;
        }
    }
    {
        const int n = col0 + (t & 127), kb = k0 + (t >> 7) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = kb + c;
            R.b[c] = (n < m && k < m) ? Bsrc[(size_t)k * m + n] : make_float2(0.f, 0.f);
        }
    }
}

// The registers of one chunk into the FP16 planes of a stage (A: planes 0..3 = re hi, re lo, im hi,
// im lo; B^T: planes 4..7), scaled by the power-of-two scales sA and sB.
__device__ __forceinline__ void xl_store(unsigned char* st, const XlRegs& R, float sA, float sB) {
    __half* pl = reinterpret_cast<__half*>(st);
    constexpr int PL = XL_TM * XL_KC;  // halves per plane
    const int t = threadIdx.x;
    {
        __half h[4][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            xl_split(R.a[c].x * sA, h[0][c], h[1][c]);
            xl_split(R.a[c].y * sA, h[2][c], h[3][c]);
        }
        const int off = xl_off(t >> 2, (t & 3) * 8);
#pragma unroll
        for (int p = 0; p < 4; ++p) *reinterpret_cast<uint4*>(pl + p * PL + off) = *reinterpret_cast<const uint4*>(h[p]);
    }
    {
        __half h[4][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            xl_split(R.b[c].x * sB, h[0][c], h[1][c]);
            xl_split(R.b[c].y * sB, h[2][c], h[3][c]);
        }
        const int off = xl_off(t & 127, (t >> 7) * 8);
#pragma unroll
        for (int p = 0; p < 4; ++p)
            *reinterpret_cast<uint4*>(pl + (4 + p) * PL + off) = *reinterpret_cast<const uint4*>(h[p]);
    }
}

// One thread: the MMAs of one staged chunk.  Corrections (lo lo, hi lo, lo hi) into (cre, cim), the
// (hi, hi) products into (hre, him); first: the first chunk (overwrite instead of accumulate).
__device__ __forceinline__ void xl_issue(uint32_t st, bool first, uint32_t hre, uint32_t him, uint32_t cre, uint32_t cim) {
    constexpr uint32_t PLB = XL_TM * XL_KC * 2;  // plane bytes
    const uint32_t lbo = 128, sbo = (XL_KC / 8) * 128;
    const uint32_t pos = idesc_f16(XL_TM, XL_TN, false), neg = idesc_f16(XL_TM, XL_TN, true);
    const uint64_t dA = smem_desc_u32(st, lbo, sbo), dB = smem_desc_u32(st + 4 * PLB, lbo, sbo);
    const uint64_t pl = PLB >> 4;
    const int ha[4] = {1, 0, 1, 0}, hb[4] = {1, 1, 0, 0};  // (lo,lo), (hi,lo), (lo,hi), (hi,hi)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const uint32_t dre = t < 3 ? cre : hre, dim = t < 3 ? cim : him;
        const uint64_t ar0 = dA + ha[t] * pl, ai0 = dA + (2 + ha[t]) * pl;
        const uint64_t br0 = dB + hb[t] * pl, bi0 = dB + (2 + hb[t]) * pl;
#pragma unroll
        for (int kk = 0; kk < XL_KC / 16; ++kk) {
            const uint64_t s = (uint64_t)kk * 16u;  // 256 bytes: two core matrices along K
            const int acc = !(first && kk == 0 && (t == 0 || t == 3));
            mma_f16(dre, ar0 + s, br0 + s, pos, acc);
            mma_f16(dim, ar0 + s, bi0 + s, pos, acc);
            mma_f16(dre, ai0 + s, bi0 + s, neg, 1);
            mma_f16(dim, ai0 + s, br0 + s, pos, 1);
        }
    }
}

// C = A B for every owned slice of the chunk: grid (output tiles of the largest block, slice).
// mode 0: Y = X X.  mode 1: Horner step j: S_out = S_in Y + c_{2j+1} X + c_{2j} I for slices with
// j <= q - 2 (at j = q - 2, S_in = c_{2q-1} X + c_{2q-2} I is formed while staging).
__global__ void __launch_bounds__(XL_THREADS, 1)
xl_gemm_kernel(DevPlan P, const XlItem* __restrict__ items, float2* __restrict__ scratch, size_t slot, int tiles_n,
               int mode, int j) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tslot;
    const XlItem& X = items[blockIdx.y];
    if (!X.own) return;
    if (mode == 1 && j > X.q - 2) return;
    const DevBlock& B = P.blocks[X.bi];
    const int m = B.m;
    const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    const int row0 = tm * XL_TM, col0 = tn * XL_TN;
    if (row0 >= m || col0 >= m) return;

    float2* base = scratch + (size_t)blockIdx.y * 4 * slot;
    float2* Xm = base;
    float2* Ym = base + slot;
    const float2* Asrc;
    const float2* Bsrc;
    float2* Cdst;
    float sA, sB, unscale, c1 = 0.f, c0 = 0.f, ic1 = 0.f, ic0 = 0.f;
    bool init = false;
    if (mode == 0) {
        Asrc = Xm;
        Bsrc = Xm;
        Cdst = Ym;
        sA = sB = ldexpf(1.f, X.eX);
        unscale = ldexpf(1.f, -2 * X.eX);
    } else {
        const int out = (X.q - 2 - j) & 1;
        init = j == X.q - 2;
        Asrc = init ? Xm : base + (size_t)(2 + (out ^ 1)) * slot;
        Bsrc = Ym;
        Cdst = base + (size_t)(2 + out) * slot;
        sA = ldexpf(1.f, X.eS);
        sB = ldexpf(1.f, X.eY);
        unscale = ldexpf(1.f, -(X.eS + X.eY));
        c1 = xl_coef[2 * j + 1];
        c0 = xl_coef[2 * j];
        ic1 = xl_coef[2 * X.q - 1];
        ic0 = xl_coef[2 * X.q - 2];
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        tmem_alloc(&tslot, XL_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const uint32_t hre = tmem, him = tmem + 128, cre = tmem + 256, cim = tmem + 384;
    constexpr uint32_t STAGE = 8 * XL_TM * XL_KC * 2;  // 8 planes of FP16
    const uint32_t sbase = smem_u32(sm);
    const int nch = (m + XL_KC - 1) / XL_KC;
    bool failed = false;
    // chunk ch + 1 is loaded into registers while the MMAs of chunks ch - 1 and ch run
    XlRegs R;
    xl_load(R, Asrc, Bsrc, m, row0, col0, 0, init, ic1, ic0);
    for (int ch = 0; ch < nch && !failed; ++ch) {
        const int stg = ch & 1;
        if (ch >= 2) {  // the MMAs of chunk ch - 2 read this stage
            const bool ok = mbar_wait_bounded(&bar[stg], (uint32_t)(((ch - 2) >> 1) & 1), XL_WAIT_NS);
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        xl_store(sm + stg * STAGE, R, sA, sB);
        if (ch + 1 < nch) xl_load(R, Asrc, Bsrc, m, row0, col0, (ch + 1) * XL_KC, init, ic1, ic0);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            xl_issue(sbase + stg * STAGE, ch == 0, hre, him, cre, cim);
            mma_commit(&bar[stg]);
        }
    }
    // every issued chunk has completed
    if (!failed) {
        bool ok = mbar_wait_bounded(&bar[(nch - 1) & 1], (uint32_t)(((nch - 1) >> 1) & 1), XL_WAIT_NS);
        if (nch >= 2) ok = ok && mbar_wait_bounded(&bar[(nch - 2) & 1], (uint32_t)(((nch - 2) >> 1) & 1), XL_WAIT_NS);
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (!failed) {
        tc_fence_after();
        // epilogue: warp w drains lanes 32 (w % 4).. (rows), columns 32 (w / 4) .. +31
        const int quarter = warp & 3, ch0 = (warp >> 2) * 32;
        const int r = row0 + 32 * quarter + lane;
        const uint32_t lb = (uint32_t)(32 * quarter) << 16;
        for (int g = 0; g < 4; ++g) {
            const int cl = ch0 + 8 * g;
            uint32_t a[8], b[8], cc[8], d[8];
            tmem_ld8_nowait(hre + lb + cl, a);
            tmem_ld8_nowait(him + lb + cl, b);
            tmem_ld8_nowait(cre + lb + cl, cc);
            tmem_ld8_nowait(cim + lb + cl, d);
            tmem_wait_ld();
            if (r < m) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = col0 + cl + c;
                    if (col < m) {
                        float2 v = make_float2((__uint_as_float(a[c]) + __uint_as_float(cc[c])) * unscale,
                                               (__uint_as_float(b[c]) + __uint_as_float(d[c])) * unscale);
                        if (mode == 1) {
                            const float2 x = Xm[(size_t)r * m + col];
                            v.x = fmaf(c1, x.x, v.x) + (r == col ? c0 : 0.f);
                            v.y = fmaf(c1, x.y, v.y);
                        }
                        Cdst[(size_t)r * m + col] = v;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(P.status, ST_TIMEOUT);
        // the commits never arrived: wait once more (bounded) before freeing the tensor memory
        mbar_wait_bounded(&bar[0], 0, XL_WAIT_NS);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, XL_TMEM_COLS);
}

// U of every owned slice: T(X) = I + X (q = 1) or the last Horner iterate.
__global__ void xl_export_kernel(DevPlan P, const XlItem* __restrict__ items, const float2* __restrict__ scratch,
                                 size_t slot, float2* __restrict__ Uout) {
    const XlItem& X = items[blockIdx.y];
    if (!X.own) return;
    const DevBlock& B = P.blocks[X.bi];
    const int m = B.m;
    const size_t mm = (size_t)m * m;
    const float2* base = scratch + (size_t)blockIdx.y * 4 * slot;
    const float2* src = X.q >= 2 ? base + (size_t)(2 + ((X.q - 2) & 1)) * slot : base;
    float2* Uo = Uout + B.u_off + (size_t)X.kw * B.mmp;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
        float2 v = src[e];
        if (X.q < 2) {
            const int r = (int)(e / m), c = (int)(e - (size_t)r * m);
            if (r == c) v.x += 1.f;
        }
        Uo[e] = v;
    }
}


}  // namespace

namespace {
size_t xl_slot(int m_max) { return (size_t)m_max * m_max; }  // float2 entries of one matrix
size_t xl_item_bytes(int m_max) { return 4 * xl_slot(m_max) * sizeof(float2); }

// slices per chunk: scratch of at most ~2 GiB, at most 256 slices, at least one
long long xl_chunk(int m_max, long long max_items) {
    long long c = (long long)((size_t)2 << 30) / (long long)xl_item_bytes(m_max);
    c = std::max(1LL, std::min(c, 256LL));
    return std::max(1LL, std::min(c, max_items));
}

size_t xl_items_bytes(long long chunk) { return ((size_t)chunk * sizeof(XlItem) + 255) / 256 * 256; }
}  // namespace

int expm_large_supported(int prec, int m) { return prec != QOC_PREC_F64 && m >= 1 && m <= 2048; }

size_t expm_large_scratch_bytes(int m_max, long long max_items) {
    const long long ch = xl_chunk(m_max, max_items);
    return xl_items_bytes(ch) + (size_t)ch * xl_item_bytes(m_max);
}

int launch_expm_large(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                      const int2* items, long long n_items, void* Uout, char* scratch, int m_max, cudaStream_t st) {
    const long long total = P.nk < 0 ? n_items : (long long)n_cls * P.nk;
    if (total <= 0) return 0;
    const long long ch = xl_chunk(m_max, total);
    XlItem* it = reinterpret_cast<XlItem*>(scratch);
    float2* mats = reinterpret_cast<float2*>(scratch + xl_items_bytes(ch));
    const size_t slot = xl_slot(m_max);
    const int tiles = (m_max + XL_TM - 1) / XL_TM;
    const size_t smem = (size_t)2 * 8 * XL_TM * XL_KC * 2;
    if (cudaFuncSetAttribute(xl_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    // the highest degree a slice without squarings can need (its norm is at most theta_cap)
    int qmax = 1;
    while (qmax < 16 && tabs.theta_odd[qmax - 1] < tabs.theta_cap) ++qmax;
    const int ew_blocks = (int)std::min<size_t>(64, (slot + 255) / 256);
    for (long long i0 = 0; i0 < total; i0 += ch) {
        const int n = (int)std::min(ch, total - i0);
        xl_prep_kernel<<<(n + 127) / 128, 128, 0, st>>>(P, tabs, u, cls, items, i0, n, it);
        xl_assemble_kernel<<<dim3(ew_blocks, n), 256, 0, st>>>(P, u, it, mats, slot);
        if (qmax >= 2) {
            xl_gemm_kernel<<<dim3(tiles * tiles, n), XL_THREADS, smem, st>>>(P, it, mats, slot, tiles, 0, 0);
            for (int j = qmax - 2; j >= 0; --j)
                xl_gemm_kernel<<<dim3(tiles * tiles, n), XL_THREADS, smem, st>>>(P, it, mats, slot, tiles, 1, j);
        }
        xl_export_kernel<<<dim3(ew_blocks, n), 256, 0, st>>>(P, it, mats, slot, reinterpret_cast<float2*>(Uout));
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

// launches of one call: per chunk prep, assembly, Y, qmax - 1 Horner steps, export
long long expm_large_launches(const ExpmTables& tabs, int m_max, long long total) {
    if (total <= 0) return 0;
    int qmax = 1;
    while (qmax < 16 && tabs.theta_odd[qmax - 1] < tabs.theta_cap) ++qmax;
    const long long ch = xl_chunk(m_max, total);
    const long long chunks = (total + ch - 1) / ch;
    return chunks * (3 + (qmax >= 2 ? qmax : 0));
}

}  // namespace qoc
