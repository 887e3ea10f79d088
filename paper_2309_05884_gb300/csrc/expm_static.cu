// Batched matrix exponential that allocates nothing: U_i = exp(A_i) for caller-provided complex
// FP64 matrices, with its working matrices in a fixed device array that lives in this library's
// module instead of in memory the caller or the library allocates.
//
// Who needs this: code that must not allocate device memory while it runs — a real-time control
// loop that forbids allocator calls after start-up, a host whose memory is handed out by a
// different runtime, or a library caller that has no allocator of its own and cannot create a
// plan workspace.  Such callers pass their input and output buffers and nothing else.
//
// The array (QOC_NOALLOC_SCRATCH_BYTES = 16 MiB) is part of the loaded module, so every GPU that
// loads libqoc.so holds it until the process exits.  Every call shares it: two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on it and give wrong
// results; serialise them.  Nothing in the array has to start at zero (each call writes every
// scratch element it reads).
//
// Host code may not use the array's name as a device address: on the host it names a stand-in
// object, and a kernel handed that pointer would fault or touch the wrong memory.  The device
// address is looked up once per device with cudaGetSymbolAddress (with that device current) on
// the first call made on it; make that first call before any stream capture begins.  Later calls
// check that the cached address is still device memory of the current device (a cudaDeviceReset
// tears the module down with its context) and look it up again if not.
#include <mutex>
#include <string>

#include "gemm.cuh"
#include "qoc_internal.h"

#define QOC_NOALLOC_SCRATCH_BYTES (16u << 20)
#define QOC_NOALLOC_MAX_M 128

namespace qoc {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QOC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
bool g_theta_ready = false;

__constant__ int c_sp[9] = {2, 2, 3, 3, 4, 4, 5, 5, 5};
__constant__ int c_sq[9] = {1, 2, 2, 3, 3, 4, 4, 5, 6};
// largest 1-norm per degree for FP64 truncation below 2^-53 (same bound as the plan's table)
struct Theta { double t[9]; };

// One CTA per matrix at a time (persistent over the batch); every scratch matrix of a slot is
// written before it is read.
template <int R>
__global__ void __launch_bounds__(GEMM_THREADS)
expm_noalloc_kernel(const double2* __restrict__ A, double2* __restrict__ U, int m, long long count,
                    unsigned char* __restrict__ scratch, size_t slot_bytes, Theta th) {
    __shared__ GemmSmem<double, R> sm;
    __shared__ double coef[8];
    __shared__ const double2* pw[8];
    __shared__ double s_if[32];
    __shared__ double s_red[GEMM_THREADS];
    __shared__ int s_sq, s_p, s_q;
    __shared__ double s_scale;
    const size_t mm = (size_t)m * m;
    double2* base = reinterpret_cast<double2*>(scratch + (size_t)blockIdx.x * slot_bytes);
    double2* S0 = base + 6 * mm;
    double2* S1 = base + 7 * mm;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { s_if[i] = f; f /= (double)(i + 1); }
    }
    if (threadIdx.x < 8) pw[threadIdx.x] = base + (size_t)(threadIdx.x < 6 ? threadIdx.x : 0) * mm;
    for (long long it = blockIdx.x; it < count; it += gridDim.x) {
        const double2* Ai = A + (size_t)it * mm;
        // 1-norm (max column sum)
        double best = 0.0;
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += hypot(Ai[(size_t)i * m + j].x, Ai[(size_t)i * m + j].y);
            best = fmax(best, s);
        }
        s_red[threadIdx.x] = best;
        __syncthreads();
        for (int s = GEMM_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) s_red[threadIdx.x] = fmax(s_red[threadIdx.x], s_red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double beta = s_red[0];
            int s = 0;
            while (beta > th.t[8] && s < 60) { beta *= 0.5; ++s; }
            int di = 0;
            while (di < 8 && th.t[di] < beta) ++di;
            s_sq = s;
            s_p = c_sp[di];
            s_q = c_sq[di];
            s_scale = ldexp(1.0, -s);
        }
        __syncthreads();
        const int s = s_sq, p = s_p, q = s_q, d = p * q;
        const double sc = s_scale;
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            const double2 a = Ai[e];
            base[mm + e] = mk<double>(a.x * sc, a.y * sc);
        }
        __syncthreads();
        for (int i = 2; i <= p; ++i) cta_gemm<double, R>(base + i * mm, base + (i - 1) * mm, base + mm, m, 0, nullptr, nullptr, sm);
        double2* S = S0;
        double2* Sn = S1;
        {
            const int b0 = (q - 1) * p;
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
                double2 v = cscale<double>(base[(size_t)p * mm + e], s_if[d]);
                if (row == col) v.x += s_if[b0];
                for (int l = 1; l < p; ++l) {
                    v.x = fma(s_if[b0 + l], pw[l][e].x, v.x);
                    v.y = fma(s_if[b0 + l], pw[l][e].y, v.y);
                }
                S[e] = v;
            }
        }
        __syncthreads();
        for (int kb = q - 2; kb >= 0; --kb) {
            if ((int)threadIdx.x < p) coef[threadIdx.x] = s_if[kb * p + threadIdx.x];
            __syncthreads();
            cta_gemm<double, R>(Sn, S, base + (size_t)p * mm, m, p, coef, pw, sm);
            double2* t = S; S = Sn; Sn = t;
        }
        for (int i = 0; i < s; ++i) {
            cta_gemm<double, R>(Sn, S, S, m, 0, nullptr, nullptr, sm);
            double2* t = S; S = Sn; Sn = t;
        }
        double2* Ui = U + (size_t)it * mm;
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Ui[e] = S[e];
        __syncthreads();
    }
}

double theta64(int d) {
    const double unit = std::ldexp(1.0, -53);
    auto bound = [&](double b) {
        double t = 1.0;
        for (int i = 1; i <= d + 1; ++i) t *= b / i;
        const double den = 1.0 - b / (d + 2);
        return den <= 0 ? 1e300 : t / den;
    };
    double lo = 0.0, hi = d + 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (bound(mid) <= unit) lo = mid; else hi = mid;
    }
    return lo;
}

Theta g_theta;

// The cached address is still this device's memory (false after a device reset, for instance).
bool still_valid(void* ptr, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace qoc

using namespace qoc;

extern "C" int qoc_expm_batch_noalloc(const double* A, double* U, int m, long long count, void* stream) {
    if (!A || !U) return set_error(QOC_EINVAL, "null matrix pointer");
    if (count < 0) return set_error(QOC_EINVAL, "count must be >= 0");
    if (m < 1 || m > QOC_NOALLOC_MAX_M)
        return set_error(QOC_EUNSUPPORTED, "qoc_expm_batch_noalloc: matrix size m must be 1.." +
                                               std::to_string(QOC_NOALLOC_MAX_M) + ", got " + std::to_string(m));
    if (count == 0) return QOC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(QOC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(QOC_EUNSUPPORTED, "device index beyond the library's table");
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_theta_ready) {
            const int degs[9] = {2, 4, 6, 9, 12, 16, 20, 25, 30};
            for (int i = 0; i < 9; ++i) g_theta.t[i] = theta64(degs[i]);
            g_theta_ready = true;
        }
        if (g_dev_ptr[dev] && !still_valid(g_dev_ptr[dev], dev)) g_dev_ptr[dev] = nullptr;
        if (!g_dev_ptr[dev]) {
            // first call on this device: look up the device address of the module's array
            e = cudaGetSymbolAddress(&g_dev_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_dev_ptr[dev] = nullptr;
                return set_error(QOC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        ptr = g_dev_ptr[dev];
    }
    const size_t slot = ((size_t)10 * m * m * sizeof(double2) + 255) / 256 * 256;
    const long long slots = (long long)(QOC_NOALLOC_SCRATCH_BYTES / slot);
    const int grid = (int)(count < slots ? count : slots);
    const Theta th = g_theta;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double2* a = reinterpret_cast<const double2*>(A);
    double2* u = reinterpret_cast<double2*>(U);
    unsigned char* sp = static_cast<unsigned char*>(ptr);
    if (m <= 16) expm_noalloc_kernel<1><<<grid, GEMM_THREADS, 0, st>>>(a, u, m, count, sp, slot, th);
    else if (m <= 32) expm_noalloc_kernel<2><<<grid, GEMM_THREADS, 0, st>>>(a, u, m, count, sp, slot, th);
    else if (m <= 48) expm_noalloc_kernel<3><<<grid, GEMM_THREADS, 0, st>>>(a, u, m, count, sp, slot, th);
    else expm_noalloc_kernel<4><<<grid, GEMM_THREADS, 0, st>>>(a, u, m, count, sp, slot, th);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QOC_ECUDA, std::string("expm_noalloc launch: ") + cudaGetErrorString(e));
    return QOC_OK;
}
