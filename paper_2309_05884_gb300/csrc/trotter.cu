// Trotterised propagation with per-qubit controls (Sec. IV, Eqs. Hcprime, completeH_cpl,
// propagator_cpl and propagator_cpl_transformed).
//
// With a separate pulse pair on every qubit the Hamiltonian is no longer symmetric, so the state
// lives in the full 2^n space.  Slice j is approximated by the ordered product over qubits
//     U_j = prod_{i=1..n} exp(-i tau h_i^(j)) E,   E = exp(-i tau/n H_cpl)   (factor i = 1 leftmost),
//     h_i^(j) = 1/2 (Bz_ij sigma_z^(i) + Bx_ij sigma_x^(i) + By_ij sigma_y^(i)),
// where each single-qubit factor is one 2 x 2 exponential (the paper moves it to the last qubit by
// the swap A_(i,n); acting on qubit i directly is the same operator) and the coupling factor is
// constant: H_cpl commutes with the dihedral group, so E = A_D (direct sum of exp(-i tau/n H_cpl,b))
// A_D^dagger with one exponential per D_n block, computed once at creation.
//
// Kernel: one CTA per state column keeps the 2^n amplitudes in shared memory (two buffers) and walks
// every slice: for i = n .. 1: coordinates in the symmetry basis (A_D^dagger: each basis vector lives
// on one orbit, a short sparse row), the block products with E_b (read from L2), back to the full
// space (A_D, the transposed sparse rows), then the 2 x 2 factor on qubit i as a butterfly over the
// pairs of states that differ in that qubit's bit.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "qoc_internal.h"

using namespace qoc;

struct qoc_trotter {
    int n = 0;
    int dim = 0;
    double tau = 0.0;
    int device = 0;
    // A_D^dagger rows (block coordinate t -> full indices) and A_D rows (full index x -> coordinates)
    int* d_fwd_ptr = nullptr;
    int* d_fwd_idx = nullptr;
    double* d_fwd_val = nullptr;
    int* d_bwd_ptr = nullptr;
    int* d_bwd_idx = nullptr;
    double* d_bwd_val = nullptr;
    // per coordinate t: offset of row a of E_b, first coordinate of its copy, m
    long long* d_erow = nullptr;
    int2* d_xbase = nullptr;
    double2* d_E = nullptr;  // E_b = exp(-i tau/n H_cpl,b), blocks in basis order, m_b^2 each
};

namespace {

constexpr int TR_THREADS = 256;

__global__ void __launch_bounds__(TR_THREADS)
trotter_kernel(int n, int dim, int N, double tau, const double* __restrict__ pulses, const int* __restrict__ fptr,
               const int* __restrict__ fidx, const double* __restrict__ fval, const int* __restrict__ bptr,
               const int* __restrict__ bidx, const double* __restrict__ bval, const long long* __restrict__ erow,
               const int2* __restrict__ xbase, const double2* __restrict__ E, const double2* __restrict__ in,
               double2* __restrict__ out) {
    extern __shared__ __align__(16) double2 tsm[];
    double2* psi = tsm;
    double2* tmp = tsm + dim;
    const double2* src = in + (size_t)blockIdx.x * dim;
    for (int x = threadIdx.x; x < dim; x += blockDim.x) psi[x] = src[x];
    __syncthreads();
    for (int j = 0; j < N; ++j) {
        for (int i = n; i >= 1; --i) {
            // coordinates c = A_D^dagger psi
            for (int t = threadIdx.x; t < dim; t += blockDim.x) {
                double2 s = make_double2(0.0, 0.0);
                for (int q = fptr[t]; q < fptr[t + 1]; ++q) {
                    const double v = fval[q];
                    const double2 p = psi[fidx[q]];
                    s.x = fma(v, p.x, s.x);
                    s.y = fma(v, p.y, s.y);
                }
                tmp[t] = s;
            }
            __syncthreads();
            // block products y_t = sum_a' E_b[a][a'] c_{base + a'}, written over psi (free now)
            for (int t = threadIdx.x; t < dim; t += blockDim.x) {
                const int2 xb = xbase[t];  // (first coordinate of the copy, m)
                const double2* row = E + erow[t];
                double2 s = make_double2(0.0, 0.0);
                for (int a = 0; a < xb.y; ++a) cfma<double>(s, row[a], tmp[xb.x + a]);
                psi[t] = s;
            }
            __syncthreads();
            // back to the full space: phi = A_D y, into tmp
            for (int x = threadIdx.x; x < dim; x += blockDim.x) {
                double2 s = make_double2(0.0, 0.0);
                for (int q = bptr[x]; q < bptr[x + 1]; ++q) {
                    const double v = bval[q];
                    const double2 y = psi[bidx[q]];
                    s.x = fma(v, y.x, s.x);
                    s.y = fma(v, y.y, s.y);
                }
                tmp[x] = s;
            }
            __syncthreads();
            // the 2 x 2 factor exp(-i tau h_i) on qubit i (bit n - i; qubit 1 is the most significant)
            const double* pl = pulses + ((size_t)j * n + (i - 1)) * 3;
            const double bz = pl[0], bx = pl[1], by = pl[2];
            const double beta = sqrt(bz * bz + bx * bx + by * by);
            const double th = 0.5 * tau * beta;
            const double c = cos(th);
            const double S = beta > 0.0 ? sin(th) / beta : 0.5 * tau;  // sin(theta) / beta
            // e = cos(th) I - i sin(th) (b / beta) . sigma
            const double2 e00 = make_double2(c, -S * bz), e01 = make_double2(-S * by, -S * bx);
            const double2 e10 = make_double2(S * by, -S * bx), e11 = make_double2(c, S * bz);
            const int bit = n - i;
            const int lowmask = (1 << bit) - 1;
            for (int pidx = threadIdx.x; pidx < dim / 2; pidx += blockDim.x) {
                const int x0 = ((pidx & ~lowmask) << 1) | (pidx & lowmask);
                const int x1 = x0 | (1 << bit);
                const double2 a = tmp[x0], b = tmp[x1];
                double2 r0 = cmul<double>(e00, a), r1 = cmul<double>(e10, a);
                cfma<double>(r0, e01, b);
                cfma<double>(r1, e11, b);
                psi[x0] = r0;
                psi[x1] = r1;
            }
            __syncthreads();
        }
    }
    double2* dst = out + (size_t)blockIdx.x * dim;
    for (int x = threadIdx.x; x < dim; x += blockDim.x) dst[x] = psi[x];
}

int cuda_err(cudaError_t e, const char* what) {
    return set_error(QOC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

void qoc_trotter_free(qoc_trotter* T) {
    if (!T) return;
    cudaFree(T->d_fwd_ptr);
    cudaFree(T->d_fwd_idx);
    cudaFree(T->d_fwd_val);
    cudaFree(T->d_bwd_ptr);
    cudaFree(T->d_bwd_idx);
    cudaFree(T->d_bwd_val);
    cudaFree(T->d_erow);
    cudaFree(T->d_xbase);
    cudaFree(T->d_E);
    delete T;
}

int qoc_trotter_create(const qoc_basis* B, double tau, qoc_trotter** out) {
    if (!B || !out) return set_error(QOC_EINVAL, "null argument");
    *out = nullptr;
    if (B->group != QOC_GROUP_DN) return set_error(QOC_EINVAL, "the coupling basis must be a D_n basis");
    if (!B->has_vectors || B->state_len != B->full_dim)
        return set_error(QOC_EINVAL, "the coupling basis needs every block and its full-space vectors");
    if (B->n > 12) return set_error(QOC_EUNSUPPORTED, "Trotterised propagation keeps 2^n amplitudes per CTA: n <= 12");
    if (!(tau > 0.0) || !std::isfinite(tau)) return set_error(QOC_EINVAL, "tau must be positive and finite");
    const int n = B->n, dim = 1 << n;
    auto* T = new (std::nothrow) qoc_trotter();
    if (!T) return set_error(QOC_ENOMEM, "host allocation failed");
    T->n = n;
    T->dim = dim;
    T->tau = tau;
    cudaGetDevice(&T->device);

    // sparse rows of A_D^dagger (coordinate t) and of A_D (full index x)
    std::vector<int> fptr(dim + 1, 0), bptr(dim + 1, 0);
    std::vector<int> fidx, tmp_x;
    std::vector<double> fval;
    std::vector<long long> erow(dim);
    std::vector<int2> xbase(dim);
    long long eoff = 0;
    std::vector<std::vector<std::pair<int, double>>> cols(dim);
    for (const auto& blk : B->blocks) {
        for (int r = 0; r < blk.c; ++r)
            for (int a = 0; a < blk.m; ++a) {
                const int t = (int)(blk.offset + (int64_t)r * blk.m + a);
                const auto& v = blk.vecs[(size_t)r * blk.m + a];
                for (size_t q = 0; q < v.idx.size(); ++q) {
                    fidx.push_back((int)v.idx[q]);
                    fval.push_back(v.val[q]);
                    cols[v.idx[q]].push_back({t, v.val[q]});
                }
                fptr[t + 1] = (int)fidx.size();
                erow[t] = eoff + (long long)a * blk.m;
                xbase[t] = make_int2((int)(blk.offset + (int64_t)r * blk.m), blk.m);
            }
        eoff += (long long)blk.m * blk.m;
    }
    std::vector<int> bidx;
    std::vector<double> bval;
    for (int x = 0; x < dim; ++x) {
        for (const auto& e : cols[x]) {
            bidx.push_back(e.first);
            bval.push_back(e.second);
        }
        bptr[x + 1] = (int)bidx.size();
    }

    cudaError_t e = cudaSuccess;
    auto up = [&](auto** dst, const auto* src, size_t count) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, sizeof(*src) * (count ? count : 1));
        if (e == cudaSuccess && count) e = cudaMemcpy(*dst, src, sizeof(*src) * count, cudaMemcpyHostToDevice);
    };
    up(&T->d_fwd_ptr, fptr.data(), fptr.size());
    up(&T->d_fwd_idx, fidx.data(), fidx.size());
    up(&T->d_fwd_val, fval.data(), fval.size());
    up(&T->d_bwd_ptr, bptr.data(), bptr.size());
    up(&T->d_bwd_idx, bidx.data(), bidx.size());
    up(&T->d_bwd_val, bval.data(), bval.size());
    up(&T->d_erow, erow.data(), erow.size());
    up(&T->d_xbase, xbase.data(), xbase.size());
    if (e != cudaSuccess) {
        qoc_trotter_free(T);
        return cuda_err(e, "Trotter tables upload");
    }

    // E_b = exp(-i tau/n H_cpl,b): the library's FP64 exponential of every block, one slice of
    // length tau/n with the controls at zero
    qoc_plan* plan = nullptr;
    qoc_plan_opts o;
    qoc_plan_opts_default(&o);
    o.prec = QOC_PREC_F64;
    int rc = qoc_plan_create(B, 1, tau / n, &o, nullptr, &plan);
    if (rc) {
        qoc_trotter_free(T);
        return rc;
    }
    size_t wsb = 0;
    qoc_plan_workspace_bytes(plan, &wsb);
    void* ws = nullptr;
    double* u0 = nullptr;
    e = cudaMalloc(&ws, wsb ? wsb : 256);
    if (e == cudaSuccess) e = cudaMalloc(&u0, sizeof(double) * B->n_ctrl);
    if (e == cudaSuccess) e = cudaMemset(u0, 0, sizeof(double) * B->n_ctrl);
    if (e == cudaSuccess) e = cudaMalloc(&T->d_E, sizeof(double2) * (size_t)(eoff ? eoff : 1));
    if (e != cudaSuccess) {
        cudaFree(ws);
        cudaFree(u0);
        qoc_plan_free(plan);
        qoc_trotter_free(T);
        return cuda_err(e, "Trotter set-up allocation");
    }
    rc = qoc_expm_blocks(plan, u0, reinterpret_cast<double*>(T->d_E), ws, wsb, nullptr);
    if (rc == QOC_OK) rc = qoc_plan_sync_status(plan, nullptr);
    cudaFree(ws);
    cudaFree(u0);
    qoc_plan_free(plan);
    if (rc) {
        qoc_trotter_free(T);
        return rc;
    }
    *out = T;
    return QOC_OK;
}

int qoc_trotter_propagate(const qoc_trotter* T, const double* pulses, int N, const double* psi_in, double* psi_out,
                          long long ncols, void* stream) {
    if (!T || !pulses || !psi_in || !psi_out) return set_error(QOC_EINVAL, "null argument");
    if (N < 0 || ncols < 0) return set_error(QOC_EINVAL, "N and ncols must be >= 0");
    if (ncols == 0) return QOC_OK;
    if (ncols > 2147483647LL) return set_error(QOC_EUNSUPPORTED, "too many columns for one launch");
    if (psi_in == psi_out) return set_error(QOC_EINVAL, "psi_out must not alias psi_in");
    cudaSetDevice(T->device);
    const size_t smem = 2 * (size_t)T->dim * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(trotter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err(e, "Trotter kernel attribute");
    trotter_kernel<<<(unsigned)ncols, TR_THREADS, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        T->n, T->dim, N, T->tau, pulses, T->d_fwd_ptr, T->d_fwd_idx, T->d_fwd_val, T->d_bwd_ptr, T->d_bwd_idx,
        T->d_bwd_val, T->d_erow, T->d_xbase, T->d_E, reinterpret_cast<const double2*>(psi_in),
        reinterpret_cast<double2*>(psi_out));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "Trotter launch");
    return QOC_OK;
}

}  // extern "C"
