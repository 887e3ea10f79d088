// Dense layers, GELU, MSE loss and Adam for the learned warm-start network.
//
// The network maps a problem's parameters to initial pulses (a 3 x 256 hidden-layer MLP with GELU,
// BF16 weights, FP32 activations and accumulation); it is trained on pulses the GRAPE solver of this
// library optimised.  The paper has no such component: it is the warm start added around the
// method, scored by the method's own fidelity.
//
// All matrix products go through one tiled SIMT kernel, C[M][N] (+)= sum_k A(m,k) B(k,n), with
// arbitrary strides so that the forward product X W^T, the input gradient dZ W and the weight
// gradient dZ^T X share it; BF16 operands are widened to FP32 when staged in shared memory.
#include <cuda_bf16.h>
#include <math.h>

#include "../../include/qoc.h"
#include "qoc_internal.h"

namespace qoc {
namespace {

constexpr int MT = 64, KT = 16, MTH = 256;  // 64x64 output tile, 16-deep k chunk, 256 threads (4x4 each)

template <class TA>
__device__ __forceinline__ float ld(const TA* p);
template <>
__device__ __forceinline__ float ld<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[m][n] = (accumulate ? C : 0) + sum_k A[m*sam + k*sak] * B[k*sbk + n*sbn]
template <class TA, class TB>
__global__ void __launch_bounds__(MTH)
gemm_kernel(int M, int N, int K, const TA* __restrict__ A, long long sam, long long sak, const TB* __restrict__ B,
            long long sbk, long long sbn, float* __restrict__ C, long long ldc, int accumulate) {
    __shared__ float As[KT][MT + 1];
    __shared__ float Bs[KT][MT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * MT, n0 = blockIdx.x * MT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += KT) {
        for (int e = threadIdx.x; e < MT * KT; e += MTH) {
            const int mm = e / KT, kk = e % KT;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? ld<TA>(A + gm * sam + gk * sak) : 0.f;
        }
        for (int e = threadIdx.x; e < MT * KT; e += MTH) {
            const int kk = e / MT, nn = e % MT;
            const int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < K && gn < N) ? ld<TB>(B + gk * sbk + gn * sbn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float* c = C + (long long)gm * ldc + gn;
            *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
    }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    // d/dz [z Phi(z)] = Phi(z) + z phi(z)
    const float Phi = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
    return Phi + z * phi;
}

// Z[b][o] += bias[o]; Y = act(Z)
__global__ void bias_act_kernel(float* Z, float* Y, const float* bias, long long B, int out, int act) {
    const long long n = B * out;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float z = Z[e] + (bias ? bias[e % out] : 0.f);
        Z[e] = z;
        Y[e] = act == 1 ? gelu(z) : z;
    }
}

// dZ = dY * act'(Z)
__global__ void act_grad_kernel(const float* Z, const float* dY, float* dZ, long long n, int act) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dZ[e] = act == 1 ? dY[e] * gelu_grad(Z[e]) : dY[e];
}

// db[o] = sum_b dZ[b][o]
__global__ void colsum_kernel(const float* dZ, float* db, long long B, int out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    double s = 0.0;
    for (long long b = 0; b < B; ++b) s += dZ[b * out + o];
    db[o] = (float)s;
}

__global__ void adam_kernel(float* w, __nv_bfloat16* shadow, const float* g, float* m, float* v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float mm = b1 * m[e] + (1.f - b1) * g[e];
        const float vv = b2 * v[e] + (1.f - b2) * g[e] * g[e];
        m[e] = mm;
        v[e] = vv;
        const float x = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);  // descent on the loss
        w[e] = x;
        if (shadow) shadow[e] = __float2bfloat16_rn(x);
    }
}

// loss = mean (Y - T)^2 (FP64 accumulation), dY = 2 (Y - T) / n
__global__ void mse_kernel(const float* Y, const float* T, float* dY, double* loss, long long n) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = Y[e] - T[e];
        s += (double)d * d;
        if (dY) dY[e] = 2.f * d / (float)n;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)n);
}

__global__ void to_bf16_kernel(const float* x, __nv_bfloat16* y, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16_rn(x[e]);
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

int cuda_status(const char* what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QOC_OK : set_error(QOC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class TA, class TB>
void gemm(int M, int N, int K, const TA* A, long long sam, long long sak, const TB* B, long long sbk, long long sbn,
          float* C, long long ldc, int acc, cudaStream_t st) {
    dim3 grid((N + MT - 1) / MT, (M + MT - 1) / MT);
    gemm_kernel<TA, TB><<<grid, MTH, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, acc);
}

}  // namespace
}  // namespace qoc

using namespace qoc;

extern "C" {

int qoc_dense_forward(const float* X, const uint16_t* W, const float* bias, float* Z, float* Y, long long B, int in,
                      int out, int act, void* stream) {
    if (!X || !W || !Z || !Y || B < 0 || in < 1 || out < 1 || (act != 0 && act != 1))
        return set_error(QOC_EINVAL, "qoc_dense_forward: bad argument");
    if (B == 0) return QOC_OK;
    if (B > (1LL << 31)) return set_error(QOC_EUNSUPPORTED, "batch too large");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const auto* Wb = reinterpret_cast<const __nv_bfloat16*>(W);
    // Z[b][o] = sum_i X[b][i] W[o][i]
    gemm<float, __nv_bfloat16>((int)B, out, in, X, in, 1, Wb, 1, in, Z, out, 0, st);
    bias_act_kernel<<<grid_for(B * out), 256, 0, st>>>(Z, Y, bias, B, out, act);
    return cuda_status("qoc_dense_forward");
}

int qoc_dense_backward(const float* X, const uint16_t* W, const float* Z, const float* dY, float* dZ, float* dX,
                       float* dW, float* db, long long B, int in, int out, int act, void* stream) {
    if (!X || !W || !Z || !dY || !dZ || B < 1 || in < 1 || out < 1 || (act != 0 && act != 1))
        return set_error(QOC_EINVAL, "qoc_dense_backward: bad argument");
    if (B > (1LL << 31)) return set_error(QOC_EUNSUPPORTED, "batch too large");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const auto* Wb = reinterpret_cast<const __nv_bfloat16*>(W);
    act_grad_kernel<<<grid_for(B * out), 256, 0, st>>>(Z, dY, dZ, B * out, act);
    // dX[b][i] = sum_o dZ[b][o] W[o][i]
    if (dX) gemm<float, __nv_bfloat16>((int)B, in, out, dZ, out, 1, Wb, in, 1, dX, in, 0, st);
    // dW[o][i] = sum_b dZ[b][o] X[b][i]
    if (dW) gemm<float, float>(out, in, (int)B, dZ, 1, out, X, in, 1, dW, in, 0, st);
    if (db) colsum_kernel<<<(out + 255) / 256, 256, 0, st>>>(dZ, db, B, out);
    return cuda_status("qoc_dense_backward");
}

int qoc_adam_step(float* param, uint16_t* shadow_bf16, const float* grad, float* m, float* v, long long n, float lr,
                  float beta1, float beta2, float eps, int t, void* stream) {
    if (!param || !grad || !m || !v || n < 0 || t < 1) return set_error(QOC_EINVAL, "qoc_adam_step: bad argument");
    if (n == 0) return QOC_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    adam_kernel<<<grid_for(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        param, reinterpret_cast<__nv_bfloat16*>(shadow_bf16), grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return cuda_status("qoc_adam_step");
}

int qoc_mse(const float* Y, const float* T, float* dY, double* loss, long long n, void* stream) {
    if (!Y || !T || !loss || n < 1) return set_error(QOC_EINVAL, "qoc_mse: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    mse_kernel<<<grid_for(n) > 1024 ? 1024 : grid_for(n), 256, 0, st>>>(Y, T, dY, loss, n);
    return cuda_status("qoc_mse");
}

int qoc_to_bf16(const float* x, uint16_t* y, long long n, void* stream) {
    if (!x || !y || n < 0) return set_error(QOC_EINVAL, "qoc_to_bf16: bad argument");
    if (n == 0) return QOC_OK;
    to_bf16_kernel<<<grid_for(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        x, reinterpret_cast<__nv_bfloat16*>(y), n);
    return cuda_status("qoc_to_bf16");
}

}  // extern "C"
