// Exact slice derivatives of the fidelity (Appendix B) and their reduction to dF/du.
//
// For slice k and block b, with A = -i tau (H0_b + sum_j u_kj Hc_jb), E_j = -i tau Hc_jb,
// psi = psi_{k-1} and lam = lam_k (costate), the Frechet derivative of exp gives
//     lam^dagger L(A, E_j) psi = sum_{p+q<=P} (A^dagger^p lam)^dagger E_j (A^q psi) / (p+q+1)!
// (the series L(A,E) = sum_{p,q} A^p E A^q / (p+q+1)!, truncated once beta^{P+1}/(P+1)! is below
// the tolerance, beta the slice's norm bound).  With v_q = A^q psi, w_p = (A^dagger)^p lam = (-A)^p
// lam and z_q = sum_{p<=P-q} w_p / (p+q+1)!, the sum is
//     -i tau sum_{a,b} Hc_j[a][b] * M[a][b],   M[a][b] = sum_q conj(z_q[a]) v_q[b],
// so every Hc_jb is read once per slice.  The paper's own slice derivative (Eq.
// propagator_differentiation) is the leading term -i tau Hc_j U_k; grad_mode 1 evaluates it as
// lam_k^dagger E_j psi_k with the same contraction (one term, z = lam_k, v = psi_k).
// dF/du_kj = 2 Re(conj(o) * sum_{b, copies} [...]), o = <psi_f|psi_N> (Eq. probability).
// A slice whose bound beta exceeds the series range is split into 2^s equal sub-slices
// (exp(A) = exp(A/2^s)^{2^s}, u_kj shared): the forward sub-states come from the Taylor action of
// exp(A/2^s), each sub-slice contributes its own series term with E_j/2^s, and the costate of the
// previous sub-slice is sum_p w_p / p!, a by-product of the w-chain.
#include "kernels.h"

namespace qoc {

namespace {

constexpr int GRAD_THREADS = 512;
// P: longest series; CG: copies processed together (2*CG right-hand sides per pass over A)
template <class T> struct GradCfg;
template <> struct GradCfg<float> { static constexpr int P = 24, CG = 2; };
template <> struct GradCfg<double> { static constexpr int P = 40, CG = 1; };
constexpr int MAX_SUB_LOG2 = 7;  // at most 128 sub-slices per slice
constexpr int REV_MIN_SUB = 3;   // slices needing >= 2^3 sub-slices go to reverse mode (grad_rev.cu)

// ys[v] = sgn[v] * M xs[v] for v < nv (nv <= NV); M is m x m row-major (shared or global), the
// vectors are in shared memory.  G threads share a row; M[o][j] is read once for all nv vectors.
template <class T, int NV>
__device__ __forceinline__ void cta_gemv_multi(cx<T>* const* ys, const cx<T>* M, const cx<T>* const* xs,
                                               const T* sgn, int nv, int m) {
    int G = 1;
    while (G < 32 && G * 2 * m <= (int)blockDim.x) G *= 2;
    const int outs = blockDim.x / G;
    const int part = threadIdx.x % G;
    for (int o0 = 0; o0 < m; o0 += outs) {
        const int o = o0 + threadIdx.x / G;
        cx<T> acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = mk<T>(0, 0);
        if (o < m) {
            const cx<T>* row = M + (size_t)o * m;
            for (int j = part; j < m; j += G) {
                const cx<T> a = row[j];
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    if (v < nv) cfma<T>(acc[v], a, xs[v][j]);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v >= nv) break;
            for (int off = G / 2; off > 0; off >>= 1) {
                acc[v].x += __shfl_xor_sync(0xffffffffu, acc[v].x, off);
                acc[v].y += __shfl_xor_sync(0xffffffffu, acc[v].y, off);
            }
            if (o < m && part == 0) ys[v][o] = mk<T>(sgn[v] * acc[v].x, sgn[v] * acc[v].y);
        }
    }
    __syncthreads();
}

template <class T>
__host__ __device__ constexpr size_t grad_vec_count(int max_m) {
    return (size_t)(2 * (GradCfg<T>::P + 1) * GradCfg<T>::CG + 3 * GradCfg<T>::CG) * max_m;
}

// Shared layout (elements of cx<T>): [A: m^2 if a_in_smem][V: (PM+1)*CG*m][Z: (PM+1)*CG*m][W: CG*m][Wn: CG*m]
template <class T>
__global__ void __launch_bounds__(GRAD_THREADS)
grad_kernel(DevPlan P, double tol, double theta, const double* __restrict__ u, const cx<T>* __restrict__ psi_st,
            const cx<T>* __restrict__ lam_st, double2* __restrict__ partial, char* __restrict__ scratch,
            size_t slot_bytes, int a_in_smem, int max_m, int fast_m, int gemm_min_m) {
    constexpr int PM = GradCfg<T>::P;
    constexpr int CG = GradCfg<T>::CG;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double s_if[PM + 2];
    __shared__ double s_uk[8];
    __shared__ int s_P;
    __shared__ double red[GRAD_THREADS / 32][8][2];

    const int NK = P.nk, nc = P.nc;
    const bool whole = P.nk < 0;
    const long long total = whole ? P.n_items : (long long)NK * P.nb;
    // a_in_smem: 1 = A and the vector families in shared memory; 0 = A in this CTA's global slot,
    // vectors in shared memory; -1 = both in the global slot (large blocks)
    cx<T>* gA = reinterpret_cast<cx<T>*>(scratch + (size_t)blockIdx.x * slot_bytes);
    cx<T>* sA = reinterpret_cast<cx<T>*>(dsm);
    cx<T>* A = a_in_smem == 1 ? sA : gA;
    cx<T>* V = a_in_smem == 1 ? sA + (size_t)max_m * max_m : a_in_smem == 0 ? sA : gA + (size_t)max_m * max_m;
    cx<T>* Z = V + (size_t)(PM + 1) * CG * max_m;
    cx<T>* W = Z + (size_t)(PM + 1) * CG * max_m;
    cx<T>* Wn = W + (size_t)CG * max_m;
    cx<T>* Ln = Wn + (size_t)CG * max_m;  // costate of the previous sub-slice
    // forward sub-states (only for slices that are split), in this CTA's global slot
    cx<T>* Psub = gA + (a_in_smem == 1 ? 0 : (size_t)max_m * max_m) +
                  (a_in_smem == -1 ? grad_vec_count<T>(max_m) : 0);
    __shared__ int s_sub;

    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int i = 0; i < PM + 2; ++i) { s_if[i] = f; f /= (double)(i + 1); }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    __shared__ int s_list[GRAD_THREADS];
    __shared__ int s_nl;
    __shared__ int s_wc[32];
    // slices this launch owns: not those of the reverse-mode kernel (>= 2^REV_MIN_SUB sub-slices) nor
    // the unsplit slices of register-sized blocks (grad_fast.cu) or of GEMM-path blocks (grad_gemm.cu)
    auto want = [&](long long it) -> bool {
        int bi;
        long long k;
        if (whole) {
            const int2 e = P.items[it];
            bi = e.x;
            k = e.y;
        } else {
            bi = (int)(it / NK);
            k = P.k0 + it % NK;
        }
        const DevBlock& Bw = P.blocks[bi];
        const int sub = P.grad_mode == 0 ? slice_halvings(slice_beta(P, Bw, u, k), theta, MAX_SUB_LOG2) : 0;
        return sub < REV_MIN_SUB && !(sub == 0 && (Bw.m <= fast_m || (gemm_min_m > 0 && Bw.m >= gemm_min_m)));
    };
    for (long long lb = 0; cta_select(total, lb, want, s_list, &s_nl, s_wc); lb += blockDim.x) {
        const int nl = s_nl;
        for (int li = 0; li < nl; ++li) {
            const long long item = (long long)blockIdx.x + (lb + s_list[li]) * gridDim.x;
            int bi, kw, k;  // block; window slot (psi_{k-1} in slot kw, lam_k in slot kw+1); slice 1..N
            if (whole) {
                const int2 it = P.items[item];
                bi = it.x;
                kw = it.y;
                k = it.y + 1;
            } else {
                bi = (int)(item / NK);
                kw = (int)(item % NK);
                k = P.k0 + kw + 1;
            }
            const DevBlock& B = P.blocks[bi];
            const int m = B.m, c = B.c;
            const size_t mm = (size_t)m * m;
            const T tau = (T)B.dt;
            if (threadIdx.x == 0) {
                double beta = B.h0_norm;
                for (int j = 0; j < nc; ++j) {
                    const double uk = u[(size_t)(B.u_row + k - 1) * nc + j];
                    s_uk[j] = isfinite(uk) ? uk : 0.0;
                    beta += fabs(s_uk[j]) * B.hc_norm[j];
                }
                beta *= B.dt;
                int Pt = 0, sub = 0;
                if (P.grad_mode == 0) {
                    while (beta > theta && sub < MAX_SUB_LOG2) { beta *= 0.5; ++sub; }
                    double term = beta;  // beta^{P+1}/(P+1)! at P = 0
                    while (Pt < PM && term > tol) { ++Pt; term *= beta / (double)(Pt + 1); }
                    if (term > tol || beta > theta) atomicOr(P.status, ST_SERIES_CAP);
                }
                s_P = Pt;
                s_sub = sub;
            }
            __syncthreads();
            const int Pt = s_P;
            const int nsub = 1 << s_sub;
            const T tau_s = tau / (T)nsub;
            const cx<T>* H = reinterpret_cast<const cx<T>*>(P.H) + B.h_off;
            if (P.grad_mode == 0) {
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    cx<T> h = H[e];
                    for (int j = 0; j < nc; ++j) {
                        const cx<T> hc = H[(size_t)(1 + j) * mm + e];
                        const T uj = (T)s_uk[j];
                        h.x = fma(uj, hc.x, h.x);
                        h.y = fma(uj, hc.y, h.y);
                    }
                    A[e] = cmul_mis<T>(h, tau_s);
                }
            }
            // per-thread partial sums in the working precision (a thread adds ~m^2/blockDim terms);
            // the cross-thread reduction below is FP64
            T accr[8], acci[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) accr[j] = acci[j] = (T)0;
            __syncthreads();
            for (int r0 = 0; r0 < c; r0 += CG) {
                const int cg = (c - r0) < CG ? (c - r0) : CG;
                // V[q][r] at V + (q*CG + r)*m ; Z likewise ; W[r] at W + r*m ; Psub[i][r] at Psub + (i*CG + r)*m
                const long long kpsi = P.grad_mode == 0 ? kw : kw + 1;
                for (int e = threadIdx.x; e < cg * m; e += blockDim.x) {
                    const int r = e / m, a = e - r * m;
                    const cx<T> x = psi_st[B.s_off + kpsi * c * m + (size_t)(r0 + r) * m + a];
                    if (nsub == 1) V[(size_t)r * m + a] = x; else Psub[(size_t)r * m + a] = x;
                    W[(size_t)r * m + a] = lam_st[B.s_off + (long long)(kw + 1) * c * m + (size_t)(r0 + r) * m + a];
                }
                __syncthreads();
                // forward sub-states psi^(i+1) = sum_q A^q psi^(i) / q!  (split slices only)
                for (int i = 0; i + 1 < nsub; ++i) {
                    for (int e = threadIdx.x; e < cg * m; e += blockDim.x) {
                        const int r = e / m, a = e - r * m;
                        const cx<T> x = Psub[((size_t)i * CG + r) * m + a];
                        V[(size_t)r * m + a] = x;
                        Psub[((size_t)(i + 1) * CG + r) * m + a] = x;
                    }
                    __syncthreads();
                    for (int q = 1; q <= Pt; ++q) {
                        cx<T>* ys[2 * CG];
                        const cx<T>* xs[2 * CG];
                        T sg[2 * CG];
#pragma unroll
                        for (int r = 0; r < 2 * CG; ++r) {
                            const int rr = r < cg ? r : 0;
                            xs[r] = V + ((size_t)(q - 1) * CG + rr) * m;
                            ys[r] = V + ((size_t)q * CG + rr) * m;
                            sg[r] = (T)1;
                        }
                        cta_gemv_multi<T, 2 * CG>(ys, A, xs, sg, cg, m);
                        const T cf = (T)s_if[q];
                        for (int e = threadIdx.x; e < cg * m; e += blockDim.x) {
                            const int r = e / m, a = e - r * m;
                            cx<T>& d = Psub[((size_t)(i + 1) * CG + r) * m + a];
                            const cx<T> v = V[((size_t)q * CG + r) * m + a];
                            d.x = fma(cf, v.x, d.x);
                            d.y = fma(cf, v.y, d.y);
                        }
                        __syncthreads();
                    }
                }
                for (int isub = nsub - 1; isub >= 0; --isub) {
                    if (nsub > 1) {
                        for (int e = threadIdx.x; e < cg * m; e += blockDim.x) {
                            const int r = e / m, a = e - r * m;
                            V[(size_t)r * m + a] = Psub[((size_t)isub * CG + r) * m + a];
                        }
                    }
                    for (int e = threadIdx.x; e < (Pt + 1) * CG * m; e += blockDim.x) Z[e] = mk<T>(0, 0);
                    for (int e = threadIdx.x; e < CG * m; e += blockDim.x) Ln[e] = mk<T>(0, 0);
                    __syncthreads();
                    for (int p = 0; p <= Pt; ++p) {
                        // z_q += w_p / (p+q+1)!  for q <= P-p ; the previous sub-slice's costate += w_p / p!
                        for (int e = threadIdx.x; e < (Pt - p + 1) * cg * m; e += blockDim.x) {
                            const int q = e / (cg * m);
                            const int ra = e - q * cg * m;
                            const T cf = (T)s_if[p + q + 1];
                            cx<T>& z = Z[(size_t)q * CG * m + ra];
                            const cx<T> w = W[ra];
                            z.x = fma(cf, w.x, z.x);
                            z.y = fma(cf, w.y, z.y);
                            if (q == 0 && nsub > 1) {
                                const T cl = (T)s_if[p];
                                Ln[ra].x = fma(cl, w.x, Ln[ra].x);
                                Ln[ra].y = fma(cl, w.y, Ln[ra].y);
                            }
                        }
                        __syncthreads();
                        if (p < Pt) {
                            // one pass over A: v_{p+1} = A v_p and w_{p+1} = -A w_p for every copy of the group
                            cx<T>* ys[2 * CG];
                            const cx<T>* xs[2 * CG];
                            T sg[2 * CG];
#pragma unroll
                            for (int r = 0; r < CG; ++r) {
                                // v vectors in slots [0, cg), w vectors in [cg, 2cg); unused slots are never read
                                const int rr = r < cg ? r : 0;
                                xs[r] = V + ((size_t)p * CG + rr) * m;
                                ys[r] = V + ((size_t)(p + 1) * CG + rr) * m;
                                sg[r] = (T)1;
                            }
#pragma unroll
                            for (int r = 0; r < CG; ++r) {
                                const int rr = r < cg ? r : 0;
                                xs[CG + r] = W + (size_t)rr * m;
                                ys[CG + r] = Wn + (size_t)rr * m;
                                sg[CG + r] = (T)-1;
                            }
                            if (cg < CG) {  // pack the w vectors right after the v vectors
                                for (int r = 0; r < cg; ++r) {
                                    xs[cg + r] = xs[CG + r];
                                    ys[cg + r] = ys[CG + r];
                                    sg[cg + r] = (T)-1;
                                }
                            }
                            cta_gemv_multi<T, 2 * CG>(ys, A, xs, sg, 2 * cg, m);
                            cx<T>* t = W; W = Wn; Wn = t;
                        }
                    }
                // contraction with every Hc_j: sum_{a,b} Hc_j[a][b] sum_{q,r} conj(Z_qr[a]) V_qr[b]
                for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
                    const int a = (int)(e / m), b = (int)(e - (size_t)a * m);
                    cx<T> Mab = mk<T>(0, 0);
                    for (int q = 0; q <= Pt; ++q)
                        for (int r = 0; r < cg; ++r)
                            cfma_conj<T>(Mab, Z[((size_t)q * CG + r) * m + a], V[((size_t)q * CG + r) * m + b]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j < nc) {
                            const cx<T> hc = H[(size_t)(1 + j) * mm + e];
                            accr[j] = fma(hc.x, Mab.x, fma(-hc.y, Mab.y, accr[j]));
                            acci[j] = fma(hc.x, Mab.y, fma(hc.y, Mab.x, acci[j]));
                        }
                    }
                }
                    __syncthreads();
                    if (nsub > 1) {  // costate at the start of this sub-slice
                        for (int e = threadIdx.x; e < cg * m; e += blockDim.x) W[e] = Ln[e];
                        __syncthreads();
                    }
                }
            }
            // block reduction of the nc complex sums; then multiply by -i tau / 2^s
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j >= nc) break;
                double xr = (double)accr[j], xi = (double)acci[j];
                for (int off = 16; off > 0; off >>= 1) {
                    xr += __shfl_xor_sync(0xffffffffu, xr, off);
                    xi += __shfl_xor_sync(0xffffffffu, xi, off);
                }
                if (lane == 0) { red[warp][j][0] = xr; red[warp][j][1] = xi; }
            }
            __syncthreads();
            if (threadIdx.x < nc) {
                double xr = 0.0, xi = 0.0;
                for (int w = 0; w < GRAD_THREADS / 32; ++w) { xr += red[w][threadIdx.x][0]; xi += red[w][threadIdx.x][1]; }
                // (-i tau) (xr + i xi) = tau xi - i tau xr
                const double ts = B.dt / (double)nsub;
                double2 o;
                o.x = ts * xi;
                o.y = -ts * xr;
                partial[(size_t)(B.part_off + k - 1) * nc + threadIdx.x] = o;
            }
            __syncthreads();
        }
    }
}

// grid (x: elements of problem p, y: p).  grad[k][j] = 2 Re(conj(o_p) sum over the problem's blocks of
// the slice derivative); then the update rule (none, fixed step or Adam) unless the problem is frozen.
__global__ void grad_reduce_kernel(DevPlan P, const double2* __restrict__ partial, const double2* __restrict__ o_ws,
                                   double* grad, double* u, UpdateRule rule, const double* out3) {
    const int p = blockIdx.y, nc = P.nc;
    const int t0 = P.prob_block_off[p], t1 = P.prob_block_off[p + 1];
    const DevBlock& B0 = P.blocks[P.prob_blocks[t0]];
    const int Np = B0.N;
    const long long row0 = B0.u_row;
    const double2 o = o_ws[p];
    const double Fp = out3[3 * p];
    const int it = rule.iter ? *rule.iter : 0;
    const bool reached_now = Fp >= rule.f_target;
    const bool frozen = rule.freeze && (reached_now || (rule.reached && rule.reached[p] >= 0));
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Np * nc; e += gridDim.x * blockDim.x) {
        const int k = e / nc, j = e - k * nc;
        double sr = 0.0, si = 0.0;
        for (int t = t0; t < t1; ++t) {
            const DevBlock& B = P.blocks[P.prob_blocks[t]];
            const double2 d = partial[(size_t)(B.part_off + k) * nc + j];
            sr += d.x;
            si += d.y;
        }
        const double gv = 2.0 * (o.x * sr + o.y * si) * (rule.gscale ? rule.gscale[p] : 1.0);
        const size_t idx = (size_t)row0 * nc + e;
        if (grad) grad[idx] = gv;
        if (u && rule.kind >= 0 && !frozen) {
            if (rule.kind == 0) {
                u[idx] += rule.step * gv;
            } else {
                const double m = rule.beta1 * rule.adam_m[idx] + (1.0 - rule.beta1) * gv;
                const double v = rule.beta2 * rule.adam_v[idx] + (1.0 - rule.beta2) * gv * gv;
                rule.adam_m[idx] = m;
                rule.adam_v[idx] = v;
                const double mh = m / (1.0 - pow(rule.beta1, it + 1));
                const double vh = v / (1.0 - pow(rule.beta2, it + 1));
                u[idx] += rule.step * mh / (sqrt(vh) + rule.eps);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rule.F_hist) rule.F_hist[(size_t)it * P.n_prob + p] = Fp;
        if (rule.reached && reached_now && rule.reached[p] < 0) rule.reached[p] = it;
    }
}

__global__ void tick_kernel(int* iter) { *iter += 1; }

__global__ void assemble_kernel(DevPlan P, const double* __restrict__ u, const double2* __restrict__ H64,
                                double2* __restrict__ A_out, const long long* __restrict__ a_off) {
    const int bi = blockIdx.y;
    const DevBlock& B = P.blocks[bi];
    const int m = B.m;
    const size_t mm = (size_t)m * m;
    const double2* H = H64 + B.h_off;
    for (int k = blockIdx.x; k < B.N; k += gridDim.x) {
        for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
            double2 h = H[e];
            for (int j = 0; j < P.nc; ++j) {
                const double uj = u[(size_t)(B.u_row + k) * P.nc + j];
                const double2 hc = H[(size_t)(1 + j) * mm + e];
                h.x = fma(uj, hc.x, h.x);
                h.y = fma(uj, hc.y, h.y);
            }
            double2 a;
            a.x = B.dt * h.y;
            a.y = -B.dt * h.x;
            A_out[a_off[bi] + (size_t)k * mm + e] = a;
        }
    }
}

template <class T>
size_t grad_vec_elems(int max_m) {
    return (size_t)(2 * (GradCfg<T>::P + 1) * GradCfg<T>::CG + 3 * GradCfg<T>::CG) * max_m;
}

template <class T>
size_t grad_psub_elems(int max_m) {
    return ((size_t)1 << MAX_SUB_LOG2) * GradCfg<T>::CG * max_m;
}

// placement mode (see grad_kernel): 1, 0 or -1
template <class T>
int grad_mode_of(int max_m) {
    const size_t limit = 220 * 1024;
    const size_t vec = grad_vec_elems<T>(max_m) * sizeof(cx<T>);
    const size_t a = (size_t)max_m * max_m * sizeof(cx<T>);
    if (vec + a <= limit) return 1;
    if (vec <= limit) return 0;
    return -1;
}

template <class T>
size_t grad_smem(int max_m) {
    const int md = grad_mode_of<T>(max_m);
    if (md == 1) return ((size_t)max_m * max_m + grad_vec_elems<T>(max_m)) * sizeof(cx<T>);
    if (md == 0) return grad_vec_elems<T>(max_m) * sizeof(cx<T>);
    return 0;
}

template <class T>
size_t grad_slot(int max_m) {
    const int md = grad_mode_of<T>(max_m);
    size_t e = (md == 1 ? 0 : (size_t)max_m * max_m) + (md == -1 ? grad_vec_elems<T>(max_m) : 0) +
               grad_psub_elems<T>(max_m);
    return e * sizeof(cx<T>) + 256;
}

}  // namespace

size_t grad_vector_smem(int prec, int max_m) {
    (void)prec;
    (void)max_m;
    return 0;  // the vector families fall back to global memory when they do not fit
}

size_t grad_slot_bytes(int prec, int max_m) { return prec == 0 ? grad_slot<double>(max_m) : grad_slot<float>(max_m); }

int grad_grid_limit(int prec, int max_m) {
    int dev = 0, sms = 0, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (prec == 0) {
        const size_t sm = grad_smem<double>(max_m);
        cudaFuncSetAttribute(grad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grad_kernel<double>, GRAD_THREADS, sm);
    } else {
        const size_t sm = grad_smem<float>(max_m);
        cudaFuncSetAttribute(grad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, grad_kernel<float>, GRAD_THREADS, sm);
    }
    if (occ < 1) occ = 1;
    return sms * occ;
}

int launch_grad_partials(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store,
                         double2* partial, char* scratch, size_t slot_bytes, int max_m, int grid,
                         cudaStream_t st, int gemm_min_m) {
    if (P.nc > 8) return -2;
    if (P.prec == 0) {
        const size_t sm = grad_smem<double>(max_m);
        cudaFuncSetAttribute(grad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        grad_kernel<double><<<grid, GRAD_THREADS, sm, st>>>(P, 1e-17, 3.8, u, (const double2*)psi_store,
                                                           (const double2*)lam_store, partial, scratch, slot_bytes,
                                                           grad_mode_of<double>(max_m), max_m, 0, 0);
    } else {
        const size_t sm = grad_smem<float>(max_m);
        cudaFuncSetAttribute(grad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        grad_kernel<float><<<grid, GRAD_THREADS, sm, st>>>(P, GF32_SERIES_TOL, 3.0, u, (const float2*)psi_store,
                                                          (const float2*)lam_store, partial, scratch, slot_bytes,
                                                          grad_mode_of<float>(max_m), max_m, grad_fast_max_m(P.prec),
                                                          gemm_min_m);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_grad_reduce(const DevPlan& P, const double2* partial, const double2* o_ws, double* grad, double* u,
                       const UpdateRule& rule, const double* out3, cudaStream_t st) {
    int maxN = P.N;
    dim3 grid(64, P.n_prob);
    (void)maxN;
    grad_reduce_kernel<<<grid, 256, 0, st>>>(P, partial, o_ws, grad, u, rule, out3);
    if (rule.iter) tick_kernel<<<1, 1, 0, st>>>(rule.iter);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_assemble(const DevPlan& P, const double* u, double2* A_out, const long long* a_off, cudaStream_t st) {
    dim3 grid(256, P.nb);
    assemble_kernel<<<grid, 256, 0, st>>>(P, u, P.H64, A_out, a_off);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace qoc
