// Batched slice propagators on the tcgen05 tensor cores (Sec. II.A, Eq. exppropagator).
//
// The method is that of expm.cu — Taylor polynomial of degree p*q by Paterson-Stockmeyer on
// X = A/2^s, then s squarings — but every complex product runs on the tensor cores through the
// FP16-split scheme of tc_gemm.cuh (about FP32 accuracy).  One CTA of 128 threads owns one
// (slice, block) item at a time; X, its powers and the Horner iterates live in FP32 in the CTA's
// global scratch slot (they feed the Horner sums), the operands of each product are staged into
// shared memory from there.  The right-hand factor is staged once per run of products that share it
// (X for the powers, X^p for the Horner steps).  Squarings run on the tensor cores when the plan
// keeps them in FP32; plans with an FP64 squaring chain square in FP64 on the CUDA cores.
#include "../../include/qoc.h"
#include "kernels.h"
#include "tc_gemm.cuh"

namespace qoc {
namespace {

__constant__ int t_deg_p[9] = {2, 2, 3, 3, 4, 4, 5, 5, 5};
__constant__ int t_deg_q[9] = {1, 2, 2, 3, 3, 4, 4, 5, 6};
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

// C = (staged A)(staged B) into tmem; then out[e] = acc + sum_{l<nterm} coef_l P_l (P_0 = I) for
// the m x m entries.  Returns false if the commit did not arrive in time.
__device__ bool tc_product_out(unsigned char* sm, const TcLayout& L, uint32_t tmem, uint64_t* bar, uint32_t& phase,
                               float2* out, int m, int nterm, const float* coef, const float2* const* pw) {
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        tc_issue(sm, L, tmem, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase, TC_WAIT_NS);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u;
    tc_fence_after();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
                if (col >= m) continue;
                const size_t o = (size_t)row * m + col;
                float2 v = make_float2(vr[j], vi[j]);
                if (nterm > 0 && row == col) v.x += coef[0];
                for (int l = 1; l < nterm; ++l) {
                    const float2 x = pw[l][o];
                    v.x = fmaf(coef[l], x.x, v.x);
                    v.y = fmaf(coef[l], x.y, v.y);
                }
                out[o] = v;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
expm_tc_kernel(DevPlan P, ExpmTables tabs, const double* __restrict__ u, const int* __restrict__ cls_blocks, int n_cls,
               const int2* __restrict__ cls_items, long long n_cls_items, void* __restrict__ Uout,
               char* __restrict__ scratch, size_t slot_bytes, int m_max, TcLayout L) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar_off());
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bar_off() + 8);
    __shared__ float coef[8];
    __shared__ const float2* pw[8];
    __shared__ double s_if[32];
    __shared__ double s_uk[8];
    __shared__ double s_scale;
    __shared__ int s_sq, s_p, s_q;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        tmem_alloc(tslot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        double f = 1.0;
        for (int i = 0; i < 32; ++i) { s_if[i] = f; f /= (double)(i + 1); }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool failed = false;

    const size_t mm_max = (size_t)m_max * m_max;
    float2* base = reinterpret_cast<float2*>(scratch + (size_t)blockIdx.x * slot_bytes);
    float2* S0 = base + 6 * mm_max;
    float2* S1 = base + 7 * mm_max;
    double2* D0 = reinterpret_cast<double2*>(base + 8 * mm_max);
    double2* D1 = D0 + mm_max;
    if (threadIdx.x < 8) pw[threadIdx.x] = base + (size_t)(threadIdx.x < 6 ? threadIdx.x : 0) * mm_max;

    const bool whole = P.nk < 0;
    const long long total = whole ? n_cls_items : (long long)n_cls * P.nk;
    for (long long item = blockIdx.x; item < total && !failed; item += gridDim.x) {
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
        const int m = B.m;
        const size_t mm = (size_t)m * m;
        if (threadIdx.x == 0) {
            double beta = B.h0_norm1;
            int bad = 0;
            for (int j = 0; j < P.nc; ++j) {
                const double x = u[(size_t)(B.u_row + k) * P.nc + j];
                const int fin = isfinite(x);
                bad |= !fin;
                s_uk[j] = fin ? x : 0.0;
                beta += fabs(s_uk[j]) * B.hc_norm1[j];
            }
            if (bad) atomicOr(P.status, ST_NAN_PULSE);
            beta *= B.dt;
            int s = 0;
            while (beta > tabs.theta_cap && s < P.max_sq) { beta *= 0.5; ++s; }
            if (beta > tabs.theta_cap) atomicOr(P.status, ST_SQUARING_CAP);
            int di = 0;
            while (di < tabs.n_deg - 1 && tabs.theta[di] < beta) ++di;
            s_sq = s;
            s_p = t_deg_p[di];
            s_q = t_deg_q[di];
            s_scale = B.dt / (double)(1LL << s);
            if (P.stats) {
                const unsigned long long m3 = (unsigned long long)m * m * m;
                atomicAdd(P.stats + 0, m3 * (unsigned long long)(s_p + s_q - 2));
                atomicAdd(P.stats + 1, m3 * (unsigned long long)s);
                atomicAdd(P.stats + 2, 1ull);
            }
        }
        __syncthreads();
        const int s = s_sq, p = s_p, q = s_q, d = p * q;
        // X = -i (tau / 2^s)(H0 + sum_j u_j Hc_j)
        {
            const float2* H = reinterpret_cast<const float2*>(P.H) + B.h_off;
            const float sc = (float)s_scale;
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                float2 h = H[e];
                for (int j = 0; j < P.nc; ++j) {
                    const float2 hc = H[(size_t)(1 + j) * mm + e];
                    const float uj = (float)s_uk[j];
                    h.x = fmaf(uj, hc.x, h.x);
                    h.y = fmaf(uj, hc.y, h.y);
                }
                base[mm_max + e] = make_float2(h.y * sc, -h.x * sc);
            }
        }
        __syncthreads();
        // powers X^2..X^p: B = X staged once
        if (p >= 2) tc_stage_b(sm, L, base + mm_max, m);
        for (int l = 2; l <= p && !failed; ++l) {
            tc_stage_a(sm, L, base + (size_t)(l - 1) * mm_max, m);
            if (!tc_product_out(sm, L, tmem, bar, phase, base + (size_t)l * mm_max, m, 0, nullptr, nullptr))
                failed = true;
        }
        if (failed) break;
        // S = c_d X^p + sum_{l<p} c_{(q-1)p+l} X^l
        float2* S = S0;
        float2* Sn = S1;
        {
            const int b0 = (q - 1) * p;
            const float2* Xpp = base + (size_t)p * mm_max;
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                const int row = (int)(e / m), col = (int)(e - (size_t)row * m);
                float2 v = make_float2(Xpp[e].x * (float)s_if[d], Xpp[e].y * (float)s_if[d]);
                if (row == col) v.x += (float)s_if[b0];
                for (int l = 1; l < p; ++l) {
                    const float2 x = pw[l][e];
                    const float c = (float)s_if[b0 + l];
                    v.x = fmaf(c, x.x, v.x);
                    v.y = fmaf(c, x.y, v.y);
                }
                S[e] = v;
            }
        }
        __syncthreads();
        // Horner in X^p: B = X^p staged once
        if (q >= 2) tc_stage_b(sm, L, base + (size_t)p * mm_max, m);
        for (int kb = q - 2; kb >= 0 && !failed; --kb) {
            if (threadIdx.x < p) coef[threadIdx.x] = (float)s_if[kb * p + threadIdx.x];
            tc_stage_a(sm, L, S, m);
            if (!tc_product_out(sm, L, tmem, bar, phase, Sn, m, p, coef, pw)) failed = true;
            float2* t = S; S = Sn; Sn = t;
        }
        if (failed) break;
        float2* Uo = reinterpret_cast<float2*>(Uout) + B.u_off + (size_t)kw * B.mmp;
        if (s > 0 && !tabs.sq_f64) {
            for (int i = 0; i < s && !failed; ++i) {  // squarings on the tensor cores
                tc_stage_a(sm, L, S, m);
                tc_stage_b(sm, L, S, m);
                if (!tc_product_out(sm, L, tmem, bar, phase, Sn, m, 0, nullptr, nullptr)) failed = true;
                float2* t = S; S = Sn; Sn = t;
            }
            if (failed) break;
        } else if (s > 0) {
            // FP64 squaring chain on the CUDA cores (rare for the norms this path serves)
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) D0[e] = make_double2(S[e].x, S[e].y);
            __syncthreads();
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
                double2* t = Da; Da = Db; Db = t;
            }
            for (size_t e = threadIdx.x; e < mm; e += blockDim.x) S[e] = make_float2((float)Da[e].x, (float)Da[e].y);
            __syncthreads();
        }
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) Uo[e] = S[e];
        __syncthreads();
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(P.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, phase, TC_WAIT_NS);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

}  // namespace

int expm_tc_supported(int prec, int m) { return prec != QOC_PREC_F64 && m >= 1 && m <= TC_MAXM; }

size_t expm_tc_smem(int m_max) {
    TcLayout L{tc_pad16(m_max), tc_pad16(m_max)};
    return L.total();
}

int expm_tc_grid_limit() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;  // one CTA per SM (shared memory and half of TMEM each)
}

int launch_expm_tc(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                   const int2* items, long long n_items, void* Uout, char* scratch, size_t slot_bytes, int m_max,
                   int grid, cudaStream_t st) {
    TcLayout L{tc_pad16(m_max), tc_pad16(m_max)};
    const size_t smem = L.total();
    if (cudaFuncSetAttribute(expm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    expm_tc_kernel<<<grid, TC_THREADS, smem, st>>>(P, tabs, u, cls, n_cls, items, n_items, Uout, scratch, slot_bytes,
                                                   m_max, L);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
