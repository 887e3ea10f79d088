// Batched complex products on tcgen05 tensor cores (see tc_gemm.cuh): C[i] = A[i] B[i].
#include <string>

#include "../../include/qoc.h"
#include "kernels.h"
#include "qoc_internal.h"
#include "tc_gemm.cuh"

namespace qoc {
namespace {

constexpr uint64_t TC_WAIT_NS = 2000000000ull;

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_cgemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C, int m,
                long long count, TcLayout L, int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar_off());
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bar_off() + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        tmem_alloc(tslot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool failed = false;
    const size_t mm = (size_t)m * m;
    for (long long it = blockIdx.x; it < count; it += gridDim.x) {
        tc_stage_a(sm, L, A + it * mm, m);
        tc_stage_b(sm, L, B + it * mm, m);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            tc_issue(sm, L, tmem, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase, TC_WAIT_NS);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        const int row = 32 * warp + lane;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        for (int c0 = 0; c0 < L.NP; c0 += 16) {
            float vr[16], vi[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, vr);
            tmem_ld16(tmem + lane_base + 128u + (uint32_t)c0, vi);
            if (row < m) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = c0 + j;
                    if (col < m) C[it * mm + (size_t)row * m + col] = make_float2(vr[j], vi[j]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (failed) {
        // the commit never arrived: give the MMAs in flight another bounded wait before freeing TMEM
        if (threadIdx.x == 0) {
            if (status) atomicOr(status, ST_TIMEOUT);
            mbar_wait_bounded(bar, phase, TC_WAIT_NS);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

}  // namespace
}  // namespace qoc

using namespace qoc;

extern "C" int qoc_tc_cgemm(const float* A, const float* B, float* C, int m, long long count, int* status,
                            void* stream) {
    if (!A || !B || !C) return set_error(QOC_EINVAL, "qoc_tc_cgemm: null matrix pointer");
    if (m < 1 || m > TC_MAXM) return set_error(QOC_EUNSUPPORTED, "qoc_tc_cgemm: m must be 1..112");
    if (count < 0) return set_error(QOC_EINVAL, "qoc_tc_cgemm: count must be >= 0");
    if (count == 0) return QOC_OK;
    TcLayout L{tc_pad16(m), tc_pad16(m)};
    const size_t smem = L.total();
    cudaError_t e = cudaFuncSetAttribute(tc_cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(QOC_ECUDA, std::string("qoc_tc_cgemm: ") + cudaGetErrorString(e));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)(count < sms ? count : sms);
    tc_cgemm_kernel<<<grid, TC_THREADS, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(B), reinterpret_cast<float2*>(C), m, count,
        L, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QOC_ECUDA, std::string("qoc_tc_cgemm launch: ") + cudaGetErrorString(e));
    return QOC_OK;
}
