// Launch wrappers of the CUDA kernels (host-callable, no templates in the interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace qoc {

// Degree table of the Taylor / Paterson-Stockmeyer scheme: theta[i] is the largest norm bound
// for which degree (p_i q_i) keeps the truncation below the working unit roundoff.
// FP32 exact-derivative series: terms below 2^-27 (about an eighth of the FP32 unit roundoff,
// relative to the leading term) are dropped
constexpr double GF32_SERIES_TOL = 7.450580596923828e-09;

struct ExpmTables {
    double theta[9];
    int n_deg;          // degrees allowed (prefix of the table)
    double theta_cap;   // largest norm the polynomial is evaluated at; larger norms are scaled
    int sq_f64;         // 1: squaring chain in FP64; 0: in the working precision
    double theta_odd[16];  // theta_odd[q-1]: norm bound of the odd Taylor degree 2q-1 (tensor-core kernel)
};

// ---- expm.cu
size_t expm_slot_bytes(int prec, int m_max);
int expm_r_for(int prec, int m);
int expm_grid_limit(int prec, int R);
// One launch per size class R: cls lists the class's blocks (windowed launches), items its
// (block, slice) pairs (whole-problem launches, P.nk < 0).
// skip_s0: leave the slices that need no squaring to the tensor-core kernel
int launch_expm(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                const int2* items, long long n_items, int R, void* Uout, char* scratch, size_t slot_bytes, int m_max,
                int grid, cudaStream_t st, int skip_s0 = 0);
// U_out[a_off[b] + k*m*m + e] (complex128, unpadded) <- the working-precision propagators.
int launch_export_u(const DevPlan& P, const void* U, double2* U_out, const long long* a_off, cudaStream_t st);

// ---- expm_warp.cu (m <= 32: warp-packed, 32/MP matrices per warp)
int expm_warp_mp(int prec, int m);             // MP (8, 16, 32) or 0 if the warp kernel does not apply
int expm_warp_grid_limit(int prec, int MP);
int launch_expm_warp(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                     const int2* items, long long n_items, int MP, int per_warp, void* Uout, int grid,
                     cudaStream_t st);

// ---- expm_large.cu (tcgen05 tiled GEMMs for blocks of up to 2048 states, slices without squaring)
int expm_large_supported(int prec, int m);
size_t expm_large_scratch_bytes(int m_max, long long max_items);
// hm, hcount (host, n_cls entries): size and item count of each class block, in the class's order
// (its items are contiguous: a whole problem's slices, or nk window slices); one block at a time.
int launch_expm_large(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                      const int2* items, long long n_items, void* Uout, char* scratch, int m_max, const int* hm,
                      const long long* hcount, cudaStream_t st);
long long expm_large_launches(const ExpmTables& tabs, int m_max, const int* hm, const long long* hcount, int n_cls);

// ---- grad_fast.cu (exact slice derivatives, FP32, m <= 128, unsplit slices; A in registers)
int grad_fast_max_m(int prec);
// gemm_min_m > 0: unsplit slices of blocks with m >= gemm_min_m belong to the GEMM path (grad_gemm.cu)
int launch_grad_fast(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store, double2* partial,
                     int max_m, int grid, cudaStream_t st, int gemm_min_m = 0);

// ---- grad_gemm.cu (exact slice derivatives of the blocks on the GEMM path, FP32 plans, unsplit slices:
// the series chains of every slice of a chunk as tall GEMMs with the stacked [H0; Hc_j])
constexpr int GG_PCAP = 19;  // longest series (beta <= 3: beta^20 / 20! < 7.5e-9)
struct GgBlock {
    int bi;          // active block index
    int m, c;        // size, active copies
    int ncol;        // 2 c S columns of the chunk layout
    long long x0, x1, y, z, w;  // complex offsets in the chunk scratch: X ping, X pong, Y, Z store, W store
    // tensor-core GEMM: split-FP16 slabs of the stacked H (plan memory, byte offset hp, scale 2^eH) and
    // of the columns X (chunk scratch, byte offset xp), per-column scale exponents at int offset cs
    long long hp, xp, cs;
    int rtc, ctc, kc, eH;  // row tiles of the stacked H, column tiles, K chunks of 32
};
enum { GG_OFF = 0, GG_CUDA = 1, GG_TC = 2 };
int grad_gemm_min_m();
// Offsets of every block for S slice slots per chunk, and the GEMM tile list (block, row tile, column
// tile) for the CUDA-core (tc = 0) or tensor-core (tc = 1) product; returns the tile count, *elems the
// complex elements of the FP32 chunk scratch, *xbytes the bytes of the column slabs that follow it.
int grad_gemm_layout(GgBlock* gb, int ngb, int nc, int S, int tc, int4* tiles, int max_tiles, size_t* elems,
                     size_t* xbytes);
// Slab layout of every block's stacked [H0; Hc_j] for the tensor-core path (host): fills hp, rtc, kc and
// the scale exponent eH from hmax[g] (a bound on the block's largest |entry|); *hbytes the total;
// launch_grad_gemm_hplanes writes the slabs.
int grad_gemm_hplanes(GgBlock* gb, int ngb, int nc, const double* hmax, size_t* hbytes);
// aux: 32 + 2 ngb S ints + the column scales of device scratch (grad_gemm_aux_ints); min_m: blocks below
// it are skipped (the other kernels own their slices); mode GG_CUDA or GG_TC
size_t grad_gemm_aux_ints(const GgBlock* gb, int ngb, int S);
// xplanes: the column slabs (grad_gemm_layout's xbytes); hplanes: the stacked-H slabs (GG_TC only)
int launch_grad_gemm(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store, double2* partial,
                     const GgBlock* gb, int ngb, const int4* tiles, int ntiles, int S, int* aux, void* scratch,
                     void* xplanes, const void* hplanes, int mode, int min_m, cudaStream_t st);
// Writes every block's stacked-H slabs (gb on the device, after grad_gemm_hplanes filled hp, rtc, kc, eH);
// h_off: device [ngb] complex offsets of each block's H0 in the FP32 H.
int launch_grad_gemm_hplanes(const GgBlock* gb, int ngb, int nc, const void* H32, const long long* h_off, void* hplanes,
                             int* status, cudaStream_t st);

// ---- persistent.cu (one GRAPE iteration of an FP64 plan in one cooperative launch)
int persistent_config(int max_m, int max_c, int* grid, size_t* slot, size_t* smem);
// u is read by the iteration and, with rule.kind >= 0, updated in place; sync: 4 device words (zeroed
// here before the launch); ts: 8 device words of global-timer stamps
int launch_persistent(const DevPlan& P, const ExpmTables& tabs, double* u, const double2* psi0, const double2* psif,
                      const int64_t* prob_state, double* out3, double2* o_ws, double2* partial, double* grad,
                      const UpdateRule& rule, void* U, void* psi_st, void* lam_st, void* fwd0, void* fwd1, void* bwd0,
                      void* bwd1, char* scratch, size_t slot_bytes, int m_max, int want_grad, unsigned* sync,
                      unsigned long long* ts, int grid, size_t smem, cudaStream_t st);

// ---- expm_tc.cu (tcgen05 tensor cores, FP16-split products; FP32 plans, m <= 112)
int expm_tc_supported(int prec, int m);
int expm_tc_grid_limit(int m_max);
size_t expm_tc_slot_bytes(int m_max);
// all_items: 1 = every slice on the tensor cores; 0 = only the slices that need no squaring
int launch_expm_tc(const DevPlan& P, const ExpmTables& tabs, const double* u, const int* cls, int n_cls,
                   const int2* items, long long n_items, void* Uout, char* scratch, size_t slot_bytes, int m_max,
                   int grid, cudaStream_t st, int all_items);

// ---- sweep.cu
// Forward (psi_{i+1} = U_i psi_i) and/or backward (lam_i = U_i^dagger lam_{i+1}) sweeps over the
// current slice window of every active block, one CTA per (direction, block); dirs: 1 = forward,
// 2 = backward, 3 = both.  Boundary vectors are [block][copy][m] arrays in the working precision.
// ---- sweep_cluster.cu (each chain over a thread-block cluster, DSMEM exchange per step)
int sweep_cluster_size(int prec, int nb, int max_m, int max_c);
int sweep_cluster_fits(int prec, int max_m, int max_c, int CL);
int launch_sweeps_cluster(const DevPlan& P, const void* U, const void* fwd_init, void* fwd_out, const void* bwd_init,
                          void* bwd_out, void* psi_store, void* lam_store, int dirs, int max_m, int max_c, int CL,
                          cudaStream_t st);
int launch_sweeps(const DevPlan& P, const void* U, const void* fwd_init, void* fwd_out, const void* bwd_init,
                  void* bwd_out, void* psi_store, void* lam_store, int dirs, int max_m, int max_c, cudaStream_t st);
// dst (boundary layout, working precision) <- the caller's block state (complex128).
int launch_gather(const DevPlan& P, const double2* src, void* dst, cudaStream_t st);
// o = sum_{active copies} <psif | psi_N> (FP64) with psi_N in boundary layout; out3 = {|o|^2, Re o, Im o}.
int launch_overlap(const DevPlan& P, const void* fin, const double2* psif, double* out3, double2* o_ws,
                   cudaStream_t st);
// Per problem p (prob_state[2p] = complex offset, [2p+1] = length of its block state): latch ST_NORM
// when | ||a_p|| - 1 | or | ||b_p|| - 1 | (b may be null) exceeds tol, FP64 sums.
int launch_norm_check(const int64_t* prob_state, int n_prob, const double2* a, const double2* b, double tol,
                      int* status, cudaStream_t st);
// A bounded wait on an mbarrier that nothing completes: gives up after limit_ns and latches
// ST_TIMEOUT, the path every bounded wait of the kernels takes when a copy or commit never lands.
int launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t st);
// psiN (caller's block state, complex128) <- fin (boundary layout); inactive copies are zeroed.
int launch_store_final(const DevPlan& P, const void* fin, double2* psiN, long long state_len, cudaStream_t st);

// ---- grad.cu
// Per-slice, per-block partial derivatives do[k][b][j] = sum_r lam_k^dagger dU_k/du_kj psi_{k-1}.
// gemm_min_m > 0: unsplit slices of blocks with m >= gemm_min_m belong to the GEMM path (grad_gemm.cu)
int launch_grad_partials(const DevPlan& P, const double* u, const void* psi_store, const void* lam_store,
                         double2* partial, char* scratch, size_t slot_bytes, int max_m, int grid,
                         cudaStream_t st, int gemm_min_m = 0);
size_t grad_slot_bytes(int prec, int max_m);
// Shared memory the slice-derivative kernel needs for its vector families (without A).
size_t grad_vector_smem(int prec, int max_m);
int grad_grid_limit(int prec, int max_m);
// ---- grad_rev.cu: reverse-mode slice derivatives of the slices with >= 3 squarings
int grad_rev_min_s();
size_t grad_rev_slot_bytes(int prec, int m_max);
// One launch per size class (cls: the class's blocks, items: its (block, slice) pairs).
int launch_grad_rev(const DevPlan& P, const ExpmTables& tabs, const double* u, const void* psi, const void* lam,
                    double2* partial, char* scratch, size_t slot, int m_max, int grid, const int* cls, int n_cls,
                    const int2* items, long long n_items, int class_m_max, cudaStream_t st);
// Per problem p: grad[k][j] = 2 Re(conj(o_p) sum over p's blocks of the slice derivatives); then
// the update rule on u (rule.kind < 0: none); advances rule.iter when it is set.
int launch_grad_reduce(const DevPlan& P, const double2* partial, const double2* o_ws, double* grad, double* u,
                       const UpdateRule& rule, const double* out3, cudaStream_t st);
// A_out[b][k] = -i dt (H0_b + sum_j u_kj Hc_jb) in complex128.
int launch_assemble(const DevPlan& P, const double* u, double2* A_out, const long long* a_off, cudaStream_t st);

}  // namespace qoc
