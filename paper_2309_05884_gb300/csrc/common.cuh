// Device-side helpers shared by the kernels: complex arithmetic on float2/double2, the device
// plan tables, and the launch-wrapper declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qoc {

template <class T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <class T> using cx = typename CT<T>::type;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T re, T im) { cx<T> z; z.x = re; z.y = im; return z; }
template <class T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <class T> __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class T> __device__ __forceinline__ void cfma_conj(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <class T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by -i*s
template <class T> __device__ __forceinline__ cx<T> cmul_mis(cx<T> a, T s) { return mk<T>(a.y * s, -a.x * s); }
template <class T, class U> __device__ __forceinline__ cx<T> ccast(cx<U> a) { return mk<T>((T)a.x, (T)a.y); }

// Status bits latched in the plan's device status word.
enum : int {
    ST_NAN_PULSE = 1,       // a non-finite pulse value
    ST_SQUARING_CAP = 2,    // a slice needed more squarings than the cap
    ST_SERIES_CAP = 4,      // a slice's gradient series did not reach its tolerance
    ST_TIMEOUT = 8,         // a bounded wait on an asynchronous copy gave up
    ST_RANGE = 16,          // a tensor-core operand left the range of its FP16 split
    ST_NORM = 32,           // an initial or target block state whose norm is not 1
};

// Per-active-block table, in device memory (one entry per active block of every problem).
struct DevBlock {
    int m;            // size
    int c;            // active copies
    int b;            // index in its problem's basis
    int prob;         // problem index
    int N;            // slices of the problem
    int pad;
    double dt;        // slice length tau of the problem
    int64_t u_row;    // first row of the problem in the concatenated pulse array [sum_p N_p][nc]
    int64_t part_off; // first row of this block in the slice-derivative array [sum_b N_b][nc]
    int64_t mmp;      // padded stride (elements) between consecutive U_b[k]: m*m rounded up to 4
    int64_t h_off;    // complex offset of H0_b in the packed Hamiltonian array; Hc_jb at h_off + (1+j)*m*m
    int64_t u_off;    // complex offset of U_b[slot 0] in the propagator area (slot i at u_off + i*mmp)
    int64_t s_off;    // complex offset of psi_b[slot 0] in the window state areas (slot i at s_off + i*c*m)
    int64_t v_off;    // complex offset of block b in a boundary-vector array [b][copy][m]
    double h0_norm;  // upper bound of the spectral norm of H0_b (hc_norm: of each Hc_jb)
    double hc_norm[8];
};

// GRAPE update rule applied by the reduction kernel (after F and dF/du of an iteration).
struct UpdateRule {
    int kind;         // 0: u += step * g;  1: Adam ascent with (beta1, beta2, eps)
    int freeze;       // 1: problems whose F reached f_target keep their pulses
    double step, beta1, beta2, eps, f_target;
    int* iter;        // device iteration counter (Adam bias correction, F history slot)
    int* reached;     // [n_prob] first iteration with F >= f_target (-1 = not yet), or null
    double* adam_m;   // [rows][nc] first moments
    double* adam_v;   // [rows][nc] second moments
    double* F_hist;   // [iters][n_prob] or null
    const double* gscale;  // [n_prob] factors applied to problem p's gradient (chain rule of a
                           // caller's dL/dF_p), or null for 1
};

// Everything a kernel needs about the plan, passed by value.
struct DevPlan {
    int N;            // slices (single-problem plans; batches use DevBlock::N)
    int k0;           // first slice (0-based) of the current window
    int nk;           // slices in the current window; < 0: every block's whole problem
    int nc;           // controls
    int nb;           // active blocks
    int n_prob;       // problems
    int prec;         // QOC_PREC_*
    int max_sq;       // squaring cap
    int grad_mode;
    double dt;        // tau (single-problem plans)
    const DevBlock* blocks;
    const int64_t* copy_src;   // [sum_b c_b] source offsets of active copies (complex elements), block-major
    const int64_t* copy_base;  // [nb] start of block b's entries in copy_src
    const int2* items;         // (block, slice) list over all blocks (whole-problem launches)
    long long n_items;
    const int* prob_blocks;    // active blocks of problem p at prob_blocks[prob_block_off[p] .. [p+1])
    const int* prob_block_off;
    const void* H;             // packed block Hamiltonians in the working precision
    const double2* H64;        // the same in FP64
    int* status;
    unsigned long long* stats; // work counters or null
};

// Norm bound of slice k (0-based) of block B: beta = tau (|H0|_2 + sum_j |u_kj| |Hc_j|_2) with the
// per-block bounds of the spectral norms, an upper bound of |A_k|_2 (triangle inequality) that fixes the squarings of the exponential and the series lengths (Sec. II.A).  Non-finite
// pulse values count as 0 (the kernels latch ST_NAN_PULSE).  Every kernel that decides which
// slices it owns uses this function, so that the decisions of different kernels agree exactly.
__device__ __forceinline__ double slice_beta(const DevPlan& P, const DevBlock& B, const double* u, long long k) {
    double beta = B.h0_norm;
    for (int j = 0; j < P.nc; ++j) {
        const double x = u[(size_t)(B.u_row + k) * P.nc + j];
        beta += fabs(isfinite(x) ? x : 0.0) * B.hc_norm[j];
    }
    return beta * B.dt;
}

// Halvings s that bring beta under cap, at most max_s; *scaled (may be null) receives beta / 2^s.
__device__ __forceinline__ int slice_halvings(double beta, double cap, int max_s, double* scaled = nullptr) {
    int s = 0;
    while (beta > cap && s < max_s) {
        beta *= 0.5;
        ++s;
    }
    if (scaled) *scaled = beta;
    return s;
}

// The items blockIdx.x + i * gridDim.x (i = 0, 1, ...) of a grid-stride loop over [0, total), tested
// blockDim.x at a time in parallel: want(item) decides on one thread, the kept ones are listed in
// increasing order in list (capacity blockDim.x) and counted in *n (wcnt: 32 ints of scratch).
// Returns false once the CTA has no items left.  Call from every thread; the caller walks
// list[0 .. *n) and then calls again with base += blockDim.x.
template <class Want>
__device__ __forceinline__ bool cta_select(long long total, long long base, Want want, int* list, int* n, int* wcnt) {
    if ((long long)blockIdx.x + base * gridDim.x >= total) return false;
    __syncthreads();  // every thread is done with the previous list
    const long long item = (long long)blockIdx.x + (base + threadIdx.x) * gridDim.x;
    const bool keep = item < total && want(item);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wcnt[w];
    if (keep) list[off + __popc(bal & ((1u << lane) - 1u))] = (int)threadIdx.x;
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wcnt[w];
        *n = t;
    }
    __syncthreads();
    return true;
}

}  // namespace qoc
