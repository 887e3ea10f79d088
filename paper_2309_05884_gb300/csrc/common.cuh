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
};

// Per-active-block table, in device memory (one entry per active block).
struct DevBlock {
    int m;            // size
    int c;            // active copies
    int b;            // index in the basis
    int pad;
    int64_t mmp;      // padded stride (elements) between consecutive U_b[k]: m*m rounded up to 4
    int64_t h_off;    // complex offset of H0_b in the packed Hamiltonian array; Hc_jb at h_off + (1+j)*m*m
    int64_t u_off;    // complex offset of U_b[k=0] in the propagator area (U_b[k] at u_off + k*mmp)
    int64_t s_off;    // complex offset of psi_b[slot 0] in the window state areas (slot i at s_off + i*c*m)
    int64_t v_off;    // complex offset of block b in a boundary-vector array [b][copy][m]
    double h0_norm1;  // max column 1-norm of H0_b
    double hc_norm1[8];
};

// Everything a kernel needs about the plan, passed by value.
struct DevPlan {
    int N;            // slices
    int k0;           // first slice (0-based) of the current window
    int nk;           // slices in the current window
    int nc;           // controls
    int nb;           // active blocks
    int prec;         // QOC_PREC_*
    double dt;        // tau
    int max_sq;       // squaring cap
    int grad_mode;
    const DevBlock* blocks;
    const int64_t* copy_src;   // [sum_b c_b] source offsets of active copies (complex elements), block-major
    const int64_t* copy_base;  // [nb] start of block b's entries in copy_src
    const void* H;             // packed block Hamiltonians in the working precision
    const double2* H64;        // the same in FP64
    int* status;
    unsigned long long* stats;  // work counters or null
};

}  // namespace qoc
