// GPU plan: the active blocks of one or many problems (each a basis with its own slice count N and
// slice length tau), their Hamiltonians resident in device memory, the workspace layout, and the C
// ABI entry points that chain the kernels:
//   gather states -> assembly + expm (one launch per size class) -> forward/backward sweeps ->
//   FP64 overlap per problem -> exact slice derivatives -> reduction (+ GRAPE update).
// With one problem and a checkpoint segment S < N the same kernels run on slice windows.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "qoc_internal.h"

using namespace qoc;

struct ExpmClass {
    int kind;            // 0: CTA tiles (param R), 1: warp-packed (param MP, per_warp matrices per warp)
    int per_warp;
    int R;
    int offset;          // into the class block list (windowed launches)
    int count;           // active blocks in the class
    long long item_off;  // into the class item list (whole-problem launches)
    long long n_items;
    int m_max;
    int grid;
    size_t slot_bytes;
    // tensor-core classes with R == 0 (slices without squarings only): the CUDA-core tile launch that
    // takes the class's other slices
    int R2 = 0;
    int grid2 = 0;
    size_t slot2 = 0;
};

// Kernel choice for blocks of size <= m_max (rules sorted by m_max; the first match wins).
struct ExpmRule {
    int m_max;
    int kind;   // 0 CTA tiles, 1 warp-packed, 2 tensor cores (m <= 112), 3 tiled tensor-core GEMMs
    int param;  // R (CTA) or matrices per warp (warp-packed; 0 = as many as fit)
};

struct Problem {
    const qoc_basis* basis;
    int N;
    double dt;
    int64_t state_off;  // complex offset of this problem's block state in the concatenated states
    int64_t state_len;  // its length (the basis' state length, or sum_b m_b^2 for the gate objective)
    int64_t u_row;      // first pulse row
};

struct GraphKey {
    const void* u;
    const void* psi0;
    const void* psif;
    const void* F_hist;
    const void* reached;
    const void* ws;
    double step, beta1, beta2, eps, f_target;
    int kind, freeze;
    cudaStream_t stream;
};

struct qoc_plan {
    std::vector<Problem> probs;
    int n_prob = 0;
    int64_t rows = 0;       // sum_p N_p (pulse rows)
    int64_t state_len = 0;  // concatenated block-state length
    int device = 0;
    int N = 0;              // slices of a single-problem plan (max over problems otherwise)
    double dt = 0.0;
    qoc_plan_opts opts{};
    int nc = 0;
    int nb = 0;
    int max_m = 0;
    int max_c = 0;
    std::vector<DevBlock> hblocks;
    std::vector<int64_t> copy_src, copy_base;
    std::vector<long long> a_off;  // export layout offsets (complex), per active block
    std::vector<int2> items;       // (block, slice) over all blocks
    std::vector<int> prob_blocks, prob_block_off;
    ExpmTables tabs{};
    std::vector<ExpmClass> classes;
    std::vector<int> h_cls;        // host copy of the class block lists
    std::vector<ExpmRule> rules;
    size_t expm_scratch = 0;
    int grad_grid = 0;
    int gf_grid = 0;  // register-tile gradient kernel
    int sweep_cl = 0;  // cluster size of the sweeps (0: one CTA per chain)
    size_t grad_slot = 0;
    int rev_grid = 0;
    size_t rev_slot = 0;
    // GEMM-path slice derivatives of large blocks (single-problem FP32 plans)
    std::vector<GgBlock> gg;       // blocks on the path (m >= gg_min_m)
    int gg_S = 0, gg_ntiles = 0;
    int gg_mode = GG_TC;           // GG_OFF, GG_CUDA (FP32 CUDA-core tiles) or GG_TC (tcgen05)
    int gg_min_m = 129;
    size_t gg_xbytes = 0;          // column slabs after the FP32 chunk scratch
    size_t gg_aux = 0;             // ints of device aux
    void* d_gg_hplanes = nullptr;  // stacked-H slabs (GG_TC)
    long long* d_gg_hoff = nullptr;
    // one persistent launch per iteration (FP64 plans without checkpointing)
    bool pk_on = false;
    mutable bool pk_last = false;  // the last call ran the persistent kernel (phase times from its stamps)
    int pk_grid = 0;
    size_t pk_slot = 0, pk_smem = 0;
    unsigned long long* d_pk_ts = nullptr;
    size_t gg_bytes = 0;
    GgBlock* d_gg = nullptr;
    int4* d_gg_tiles = nullptr;
    int seg = 0;                    // slices per checkpoint segment (single problem)
    int nseg = 1;                   // segments
    int64_t vlen = 0;               // complex elements of one boundary vector set (sum c*m)
    // device
    DevBlock* d_blocks = nullptr;
    int64_t* d_copy_src = nullptr;
    int64_t* d_copy_base = nullptr;
    long long* d_a_off = nullptr;
    void* d_H = nullptr;
    double2* d_H64 = nullptr;
    int* d_cls = nullptr;
    int2* d_cls_items = nullptr;
    int2* d_items = nullptr;
    int* d_prob_blocks = nullptr;
    int* d_prob_block_off = nullptr;
    int* d_status = nullptr;
    int64_t* d_prob_state = nullptr;  // [n_prob][2]: complex offset and length of each problem's block state
    int* h_status = nullptr;          // pinned host copy of d_status, written at the end of every call
    cudaEvent_t st_ev = nullptr;      // recorded after that copy
    mutable bool st_recorded = false;
    unsigned long long* d_stats = nullptr;
    bool profiling = false;
    bool capturing = false;
    // profiling: a pair of CUDA events around every phase launch of the last call (phase ids as in
    // qoc_plan_phase_times), summed per phase on request
    mutable std::vector<cudaEvent_t> sec_ev;
    mutable std::vector<int> sec_phase;
    cudaGraphExec_t graph = nullptr;
    GraphKey graph_key{};
    // workspace layout (bytes)
    size_t off_U = 0, off_psi = 0, off_lam = 0, off_partial = 0, off_o = 0, off_out3 = 0, off_expm = 0,
           off_grad = 0, off_ckpt = 0, off_lamb = 0, off_adam = 0, off_iter = 0, off_reached = 0, off_rev = 0,
           off_gg = 0, off_ggaux = 0, off_pk = 0, off_pksync = 0;
    size_t el = 16;
    size_t ws_bytes = 0;
    int64_t u_elems = 0, s_elems = 0, part_rows = 0;

    DevPlan dev(int k0 = 0, int nk = -1) const {
        DevPlan P{};
        P.N = N;
        P.k0 = k0;
        P.nk = nk;
        P.nc = nc;
        P.nb = nb;
        P.n_prob = n_prob;
        P.prec = opts.prec;
        P.dt = dt;
        P.max_sq = opts.max_squarings;
        P.grad_mode = opts.grad_mode;
        P.blocks = d_blocks;
        P.copy_src = d_copy_src;
        P.copy_base = d_copy_base;
        P.items = d_items;
        P.n_items = (long long)items.size();
        P.prob_blocks = d_prob_blocks;
        P.prob_block_off = d_prob_block_off;
        P.H = d_H;
        P.H64 = d_H64;
        P.status = d_status;
        P.stats = (profiling && !capturing) ? d_stats : nullptr;
        return P;
    }
};

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(QOC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Largest beta with beta^{d+1}/(d+1)! / (1 - beta/(d+2)) <= u  (Taylor remainder bound).
double theta_for(int d, double unit) {
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

cudaStream_t to_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_ws(const qoc_plan* p, void* ws, size_t bytes) {
    if (!ws && p->ws_bytes > 0) return set_error(QOC_EINVAL, "null workspace");
    if (bytes < p->ws_bytes)
        return set_error(QOC_ENOMEM, "workspace too small: need " + std::to_string(p->ws_bytes) + " bytes");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return set_error(QOC_EINVAL, "workspace must be 256-byte aligned");
    return QOC_OK;
}

// The error code of a set of latched status bits (the most severe first).
int status_error(int st) {
    if (st & ST_TIMEOUT) return set_error(QOC_ETIMEOUT, "a bounded device wait gave up");
    if (st & ST_NAN_PULSE) return set_error(QOC_EINVAL, "non-finite pulse value");
    if (st & ST_NORM)
        return set_error(QOC_EINVAL, "an initial or target block state has a norm that differs from 1 by more than 1e-8");
    if (st & ST_SQUARING_CAP) return set_error(QOC_EUNSUPPORTED, "a slice needed more squarings than max_squarings");
    if (st & ST_SERIES_CAP) return set_error(QOC_EUNSUPPORTED, "a slice's norm is beyond the gradient series' range");
    if (st & ST_RANGE)
        return set_error(QOC_EUNSUPPORTED, "a tensor-core expm operand left the FP16-split range (non-Hermitian H?)");
    return QOC_OK;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Status bits latched by earlier calls on the plan whose work has finished on the GPU: returned (and
// cleared) at the start of the next call.  Bits of calls still running are left for a later call or
// for qoc_plan_sync_status; nothing here waits for the GPU.
int take_latched(const qoc_plan* p, cudaStream_t st) {
    if (!p->st_recorded || p->capturing || stream_capturing(st)) return QOC_OK;
    const cudaError_t q = cudaEventQuery(p->st_ev);
    if (q == cudaErrorNotReady) {
        (void)cudaGetLastError();
        return QOC_OK;
    }
    if (q != cudaSuccess) return cuda_fail(q, "status event");
    const int bits = *reinterpret_cast<volatile int*>(p->h_status);
    p->st_recorded = false;
    if (!bits) return QOC_OK;
    *reinterpret_cast<volatile int*>(p->h_status) = 0;
    cudaMemsetAsync(p->d_status, 0, sizeof(int), st);
    return status_error(bits);
}

// Queue the copy of the status word that the next call reads (not inside a stream capture).
void record_status(const qoc_plan* p, cudaStream_t st) {
    if (p->capturing || stream_capturing(st)) return;
    if (cudaMemcpyAsync(p->h_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaEventRecord(p->st_ev, st) == cudaSuccess)
        p->st_recorded = true;
    else
        (void)cudaGetLastError();
}

// Norms of the caller's initial (and target, may be null) block states, checked on the device.
int check_norms(const qoc_plan* p, const double* a, const double* b, cudaStream_t st) {
    if (launch_norm_check(p->d_prob_state, p->n_prob, reinterpret_cast<const double2*>(a),
                          reinterpret_cast<const double2*>(b), 1e-8, p->d_status, st) != 0)
        return cuda_fail(cudaGetLastError(), "norm check launch");
    return QOC_OK;
}

// Start a call's phase log (profiling only).
void sections_begin(const qoc_plan* p) {
    if (p->profiling && !p->capturing) p->sec_phase.clear();
}

// Events on the launching stream around one phase's launches (profiling only, not while capturing).
struct Timed {
    const qoc_plan* p;
    cudaStream_t st;
    size_t idx = 0;
    bool on;
    Timed(const qoc_plan* p_, int phase, cudaStream_t s) : p(p_), st(s), on(p_->profiling && !p_->capturing) {
        if (!on) return;
        idx = 2 * p->sec_phase.size();
        while (p->sec_ev.size() < idx + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                (void)cudaGetLastError();
                on = false;
                return;
            }
            p->sec_ev.push_back(e);
        }
        p->sec_phase.push_back(phase);
        cudaEventRecord(p->sec_ev[idx], st);
    }
    ~Timed() {
        if (on) cudaEventRecord(p->sec_ev[idx + 1], st);
    }
};
enum { PH_EXPM = 0, PH_SWEEPS = 1, PH_OVERLAP = 2, PH_DERIV = 3, PH_REDUCE = 4 };

char* ckpt_vec(const qoc_plan* p, char* ws, int i) { return ws + p->off_ckpt + (size_t)i * p->vlen * p->el; }
char* lamb_vec(const qoc_plan* p, char* ws, int i) { return ws + p->off_lamb + (size_t)i * p->vlen * p->el; }

// nk < 0: whole-problem launches over every block; nk >= 0: slice window [k0, k0 + nk) of one problem
int run_expm(const qoc_plan* p, const double* u, char* ws, int k0, int nk, cudaStream_t st) {
    Timed tm(p, PH_EXPM, st);
    const DevPlan P = p->dev(k0, nk);
    for (const auto& c : p->classes) {
        int rc;
        if (c.kind == 1)
            rc = launch_expm_warp(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                  c.R, c.per_warp, ws + p->off_U, c.grid, st);
        else if (c.kind == 3) {
            std::vector<int> hm(c.count);
            std::vector<long long> hcount(c.count);
            for (int i = 0; i < c.count; ++i) {
                const DevBlock& hb = p->hblocks[p->h_cls[c.offset + i]];
                hm[i] = hb.m;
                hcount[i] = nk < 0 ? hb.N : nk;
            }
            rc = launch_expm_large(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                   ws + p->off_U, ws + p->off_expm, c.m_max, hm.data(), hcount.data(), st);
            if (rc == 0)
                rc = launch_expm(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                 c.R2, ws + p->off_U, ws + p->off_expm, c.slot2, c.m_max, c.grid2, st, 1);
        } else if (c.kind == 2) {
            rc = launch_expm_tc(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                ws + p->off_U, ws + p->off_expm, c.slot_bytes, c.m_max, c.grid, st, c.R);
            if (rc == 0 && c.R == 0)
                rc = launch_expm(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                 c.R2, ws + p->off_U, ws + p->off_expm, c.slot2, c.m_max, c.grid2, st, 1);
        }
        else
            rc = launch_expm(P, p->tabs, u, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items, c.R,
                             ws + p->off_U, ws + p->off_expm, c.slot_bytes, c.m_max, c.grid, st);
        if (rc != 0) return cuda_fail(cudaGetLastError(), "expm launch");
    }
    return QOC_OK;
}

int run_sweeps(const qoc_plan* p, char* ws, int k0, int nk, int dirs, const char* fwd_in, char* fwd_out,
               const char* bwd_in, char* bwd_out, cudaStream_t st) {
    Timed tm(p, PH_SWEEPS, st);
    const DevPlan P = p->dev(k0, nk);
    const int rc = p->sweep_cl > 0
                       ? launch_sweeps_cluster(P, ws + p->off_U, fwd_in, fwd_out, bwd_in, bwd_out, ws + p->off_psi,
                                               ws + p->off_lam, dirs, p->max_m, p->max_c, p->sweep_cl, st)
                       : launch_sweeps(P, ws + p->off_U, fwd_in, fwd_out, bwd_in, bwd_out, ws + p->off_psi,
                                       ws + p->off_lam, dirs, p->max_m, p->max_c, st);
    if (rc == -2) return set_error(QOC_EUNSUPPORTED, "block states do not fit in shared memory");
    if (rc != 0) return cuda_fail(cudaGetLastError(), "sweep launch");
    return QOC_OK;
}

int run_grad(const qoc_plan* p, const double* u, char* ws, int k0, int nk, cudaStream_t st) {
    Timed tm(p, PH_DERIV, st);
    const DevPlan P = p->dev(k0, nk);
    const bool gon = p->gg_mode != GG_OFF && !p->gg.empty();
    const int gmin = gon ? p->gg_min_m : 0;
    const int g = launch_grad_partials(P, u, ws + p->off_psi, ws + p->off_lam,
                                       reinterpret_cast<double2*>(ws + p->off_partial), ws + p->off_grad,
                                       p->grad_slot, p->max_m, p->grad_grid, st, gmin);
    if (g == -2) return set_error(QOC_EUNSUPPORTED, "gradient kernel limits exceeded");
    if (g != 0) return cuda_fail(cudaGetLastError(), "gradient launch");
    if (gon &&
        launch_grad_gemm(P, u, ws + p->off_psi, ws + p->off_lam, reinterpret_cast<double2*>(ws + p->off_partial),
                         p->d_gg, (int)p->gg.size(), p->d_gg_tiles, p->gg_ntiles, p->gg_S,
                         reinterpret_cast<int*>(ws + p->off_ggaux), ws + p->off_gg,
                         ws + p->off_gg + align_up(p->gg_bytes, 1024), p->d_gg_hplanes, p->gg_mode, p->gg_min_m, st) != 0)
        return cuda_fail(cudaGetLastError(), "gradient launch (GEMM path)");
    if (launch_grad_fast(P, u, ws + p->off_psi, ws + p->off_lam, reinterpret_cast<double2*>(ws + p->off_partial),
                         p->max_m, p->gf_grid, st, gmin) != 0)
        return cuda_fail(cudaGetLastError(), "gradient launch (register tiles)");
    if (P.grad_mode == 0) {
        // large-norm slices: reverse-mode kernel, one launch per size class with that class's tile
        for (const auto& c : p->classes) {
            if (launch_grad_rev(P, p->tabs, u, ws + p->off_psi, ws + p->off_lam,
                                reinterpret_cast<double2*>(ws + p->off_partial), ws + p->off_rev, p->rev_slot, p->max_m,
                                p->rev_grid, p->d_cls + c.offset, c.count, p->d_cls_items + c.item_off, c.n_items,
                                c.m_max, st) != 0)
                return cuda_fail(cudaGetLastError(), "reverse-mode gradient launch");
        }
    }
    return QOC_OK;
}

void window_of(const qoc_plan* p, int s, int* k0, int* nk) {
    *k0 = s * p->seg;
    *nk = std::min(p->seg, p->N - *k0);
}

// Forward pass: psi_0 (gathered into checkpoint 0) -> checkpoint nseg = psi_N.
int forward_pass(const qoc_plan* p, const double* u, const double* psi0, char* w, cudaStream_t st) {
    int rc;
    if (launch_gather(p->dev(), reinterpret_cast<const double2*>(psi0), ckpt_vec(p, w, 0), st) != 0)
        return cuda_fail(cudaGetLastError(), "gather launch");
    if (p->nseg == 1) {
        if ((rc = run_expm(p, u, w, 0, -1, st))) return rc;
        return run_sweeps(p, w, 0, -1, 1, ckpt_vec(p, w, 0), ckpt_vec(p, w, 1), nullptr, nullptr, st);
    }
    for (int s = 0; s < p->nseg; ++s) {
        int k0, nk;
        window_of(p, s, &k0, &nk);
        if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
        if ((rc = run_sweeps(p, w, k0, nk, 1, ckpt_vec(p, w, s), ckpt_vec(p, w, s + 1), nullptr, nullptr, st)))
            return rc;
    }
    return QOC_OK;
}

// Partition the active blocks into expm launches by the plan's rules; uploads the class lists.
int build_classes(qoc_plan* p) {
    const int wp = p->opts.prec;
    struct Key { int kind, param, per_warp; };
    std::vector<Key> keys(p->nb);
    for (int i = 0; i < p->nb; ++i) {
        const int m = p->hblocks[i].m;
        Key key{0, expm_r_for(wp == QOC_PREC_F64 ? 0 : 1, m), 0};
        for (const auto& r : p->rules) {
            if (m > r.m_max) continue;
            if (r.kind == 1) {
                const int MP = expm_warp_mp(wp, m);
                if (!MP) continue;  // not applicable: next rule
                key = {1, MP, r.param > 0 ? std::min(r.param, 32 / MP) : 32 / MP};
            } else if (r.kind == 2) {
                if (!expm_tc_supported(wp, m)) continue;
                key = {2, r.param > 0 ? 1 : 0, 0};
            } else if (r.kind == 3) {
                if (!expm_large_supported(wp, m)) continue;
                key = {3, 0, 0};
            } else {
                const int rmax = wp == QOC_PREC_F64 ? 4 : 7;
                key = {0, r.param > 0 ? std::min(r.param, rmax) : expm_r_for(wp == QOC_PREC_F64 ? 0 : 1, m), 0};
            }
            break;
        }
        keys[i] = key;
    }
    std::vector<int> cls_list;
    std::vector<int2> cls_items;
    p->classes.clear();
    p->expm_scratch = 0;
    std::vector<Key> seen;
    for (int i = 0; i < p->nb; ++i) {
        bool dup = false;
        for (const auto& s : seen)
            if (s.kind == keys[i].kind && s.param == keys[i].param && s.per_warp == keys[i].per_warp) dup = true;
        if (!dup) seen.push_back(keys[i]);
    }
    for (const auto& key : seen) {
        ExpmClass c{};
        c.kind = key.kind;
        c.R = key.param;
        c.per_warp = key.per_warp;
        c.offset = (int)cls_list.size();
        c.item_off = (long long)cls_items.size();
        for (int i = 0; i < p->nb; ++i)
            if (keys[i].kind == key.kind && keys[i].param == key.param && keys[i].per_warp == key.per_warp) {
                cls_list.push_back(i);
                c.count++;
                c.m_max = std::max(c.m_max, p->hblocks[i].m);
                for (int k = 0; k < p->hblocks[i].N; ++k) cls_items.push_back(make_int2(i, k));
            }
        c.n_items = (long long)cls_items.size() - c.item_off;
        const long long max_items = p->nseg == 1 ? c.n_items : (long long)c.count * p->seg;
        if (c.kind == 2) {
            c.grid = (int)std::max<long long>(1, std::min<long long>(max_items, expm_tc_grid_limit(c.m_max)));
            c.slot_bytes = align_up(expm_tc_slot_bytes(c.m_max), 256);
            p->expm_scratch = std::max(p->expm_scratch, c.slot_bytes * (size_t)c.grid);
            if (c.R == 0) {  // the launches run in turn on one stream and share the scratch
                c.R2 = expm_r_for(1, c.m_max);
                c.grid2 = (int)std::max<long long>(1, std::min<long long>(max_items, expm_grid_limit(1, c.R2)));
                c.slot2 = align_up(expm_slot_bytes(1, c.m_max), 256);
                p->expm_scratch = std::max(p->expm_scratch, c.slot2 * (size_t)c.grid2);
            }
        } else if (c.kind == 3) {
            // tiled tensor-core GEMMs for the slices without squarings, the CUDA-core tiles for the rest
            c.grid = 1;
            c.slot_bytes = align_up(expm_large_scratch_bytes(c.m_max, max_items), 256);
            p->expm_scratch = std::max(p->expm_scratch, c.slot_bytes);
            c.R2 = expm_r_for(1, c.m_max);
            c.grid2 = (int)std::max<long long>(1, std::min<long long>(max_items, expm_grid_limit(1, c.R2)));
            c.slot2 = align_up(expm_slot_bytes(1, c.m_max), 256);
            p->expm_scratch = std::max(p->expm_scratch, c.slot2 * (size_t)c.grid2);
        } else if (c.kind == 1) {
            const long long groups = (max_items + c.per_warp - 1) / c.per_warp;
            const long long ctas = (groups + (c.R == 32 ? 2 : 4) - 1) / (c.R == 32 ? 2 : 4);
            c.grid = (int)std::max<long long>(1, std::min<long long>(ctas, expm_warp_grid_limit(wp, c.R)));
            c.slot_bytes = 0;
        } else {
            c.grid = (int)std::min<long long>(max_items, expm_grid_limit(wp == QOC_PREC_F64 ? 0 : 1, c.R));
            c.slot_bytes = align_up(expm_slot_bytes(wp == QOC_PREC_F64 ? 0 : 1, c.m_max), 256);
            p->expm_scratch = std::max(p->expm_scratch, c.slot_bytes * (size_t)c.grid);
        }
        p->classes.push_back(c);
    }
    cudaFree(p->d_cls);
    cudaFree(p->d_cls_items);
    p->d_cls = nullptr;
    p->d_cls_items = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_cls, sizeof(int) * std::max<size_t>(1, cls_list.size()))) != cudaSuccess)
        return cuda_fail(e, "upload classes");
    if ((e = cudaMalloc(&p->d_cls_items, sizeof(int2) * std::max<size_t>(1, cls_items.size()))) != cudaSuccess)
        return cuda_fail(e, "upload classes");
    cudaMemcpy(p->d_cls, cls_list.data(), sizeof(int) * cls_list.size(), cudaMemcpyHostToDevice);
    p->h_cls = cls_list;
    cudaMemcpy(p->d_cls_items, cls_items.data(), sizeof(int2) * cls_items.size(), cudaMemcpyHostToDevice);
    return QOC_OK;
}

// Recompute the workspace layout from the plan's sizes (classes may change the expm scratch).
void layout_workspace(qoc_plan* p, int64_t u_elems, int64_t s_elems, int64_t part_rows) {
    const size_t el = p->el;
    size_t off = 0;
    p->off_U = off;       off = align_up(off + (size_t)u_elems * el, 256);
    p->off_psi = off;     off = align_up(off + (size_t)s_elems * el, 256);
    p->off_lam = off;     off = align_up(off + (size_t)s_elems * el, 256);
    p->off_partial = off; off = align_up(off + (size_t)part_rows * p->nc * 16, 256);
    p->off_o = off;       off = align_up(off + (size_t)p->n_prob * 16, 256);
    p->off_out3 = off;    off = align_up(off + (size_t)p->n_prob * 24, 256);
    p->off_expm = off;    off = align_up(off + p->expm_scratch, 256);
    p->off_grad = off;    off = align_up(off + p->grad_slot * (size_t)p->grad_grid, 256);
    p->off_rev = off;     off = align_up(off + p->rev_slot * (size_t)p->rev_grid, 256);
    p->off_gg = off;      off = align_up(off + (p->gg.empty() ? 0 : align_up(p->gg_bytes, 1024) + p->gg_xbytes), 1024);
    p->off_ggaux = off;   off = align_up(off + sizeof(int) * p->gg_aux, 256);
    p->off_pk = off;      off = align_up(off + (p->pk_on ? p->pk_slot * (size_t)p->pk_grid : 0), 256);
    p->off_pksync = off;  off = align_up(off + 64, 256);
    p->off_ckpt = off;    off = align_up(off + (size_t)(p->nseg + 1) * p->vlen * el, 256);
    p->off_lamb = off;    off = align_up(off + (size_t)2 * p->vlen * el, 256);
    p->off_adam = off;    off = align_up(off + (size_t)2 * p->rows * p->nc * sizeof(double), 256);
    p->off_iter = off;    off = align_up(off + sizeof(int), 256);
    p->off_reached = off; off = align_up(off + (size_t)p->n_prob * sizeof(int), 256);
    p->ws_bytes = off;
}

// The GEMM path of the slice derivatives (grad_gemm.cu) for the plan's mode and threshold: blocks,
// chunk size, layout, tile lists and (tensor cores) the stacked-H slabs.  Single-problem FP32 plans in
// exact mode only; the workspace layout must be recomputed afterwards.
int build_gg(qoc_plan* p) {
    cudaFree(p->d_gg);
    cudaFree(p->d_gg_tiles);
    cudaFree(p->d_gg_hplanes);
    cudaFree(p->d_gg_hoff);
    p->d_gg = nullptr;
    p->d_gg_tiles = nullptr;
    p->d_gg_hplanes = nullptr;
    p->d_gg_hoff = nullptr;
    p->gg.clear();
    p->gg_bytes = p->gg_xbytes = p->gg_aux = 0;
    p->gg_S = p->gg_ntiles = 0;
    if (p->opts.prec == QOC_PREC_F64 || p->opts.grad_mode != 0 || p->n_prob != 1 || p->gg_mode == GG_OFF) return QOC_OK;
    std::vector<double> hmax;
    std::vector<long long> hoff;
    for (int bi = 0; bi < p->nb; ++bi)
        if (p->hblocks[bi].m >= p->gg_min_m) {
            GgBlock G{};
            G.bi = bi;
            G.m = p->hblocks[bi].m;
            G.c = p->hblocks[bi].c;
            p->gg.push_back(G);
            const auto& blk = p->probs[0].basis->blocks[p->hblocks[bi].b];
            double mx = 0.0;
            for (const auto& z : blk.h0) mx = std::max(mx, std::max(std::fabs(z.real()), std::fabs(z.imag())));
            for (const auto& z : blk.hc) mx = std::max(mx, std::max(std::fabs(z.real()), std::fabs(z.imag())));
            hmax.push_back(mx);
            hoff.push_back(p->hblocks[bi].h_off);
        }
    if (p->gg.empty()) return QOC_OK;
    const int ngb = (int)p->gg.size();
    const int tc = p->gg_mode == GG_TC;
    // chunk slots: every slice of a window at once where about 1.5 GB of scratch allows, at most 512
    const int slots = p->nseg == 1 ? p->N : p->seg;
    size_t per_slot = 0;
    for (const auto& G : p->gg)
        per_slot += (size_t)G.c * G.m * sizeof(float2) * (4 + 2 * (1 + p->nc) + (GG_PCAP + 1) * (1 + p->nc)) +
                    (size_t)2 * G.c * ((G.m + 31) / 32 * 32) * 8;  // column slabs: 4 FP16 planes
    p->gg_S = (int)std::max<size_t>(1, std::min<size_t>({(size_t)slots, (size_t)512, ((size_t)3 << 29) / per_slot}));
    size_t elems = 0;
    if (tc) {
        size_t hbytes = 0;
        grad_gemm_hplanes(p->gg.data(), ngb, p->nc, hmax.data(), &hbytes);
        cudaError_t e = cudaMalloc(&p->d_gg_hplanes, hbytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc H slabs");
    }
    p->gg_ntiles = grad_gemm_layout(p->gg.data(), ngb, p->nc, p->gg_S, tc, nullptr, 0, &elems, &p->gg_xbytes);
    std::vector<int4> tl(p->gg_ntiles);
    grad_gemm_layout(p->gg.data(), ngb, p->nc, p->gg_S, tc, tl.data(), p->gg_ntiles, &elems, &p->gg_xbytes);
    p->gg_bytes = elems * sizeof(float2);
    p->gg_aux = grad_gemm_aux_ints(p->gg.data(), ngb, p->gg_S);
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_gg, sizeof(GgBlock) * ngb)) != cudaSuccess) return cuda_fail(e, "upload GEMM-path blocks");
    cudaMemcpy(p->d_gg, p->gg.data(), sizeof(GgBlock) * ngb, cudaMemcpyHostToDevice);
    if ((e = cudaMalloc(&p->d_gg_tiles, sizeof(int4) * tl.size())) != cudaSuccess) return cuda_fail(e, "upload GEMM-path tiles");
    cudaMemcpy(p->d_gg_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice);
    if (tc) {
        if ((e = cudaMalloc(&p->d_gg_hoff, sizeof(long long) * ngb)) != cudaSuccess) return cuda_fail(e, "upload H offsets");
        cudaMemcpy(p->d_gg_hoff, hoff.data(), sizeof(long long) * ngb, cudaMemcpyHostToDevice);
        if (launch_grad_gemm_hplanes(p->d_gg, ngb, p->nc, p->d_H, p->d_gg_hoff, p->d_gg_hplanes, p->d_status, nullptr) != 0)
            return cuda_fail(cudaGetLastError(), "H slabs launch");
        if ((e = cudaStreamSynchronize(nullptr)) != cudaSuccess) return cuda_fail(e, "H slabs");
    }
    return QOC_OK;
}

UpdateRule no_update() {
    UpdateRule r{};
    r.kind = -1;
    r.f_target = 2.0;
    return r;
}

// The whole evaluation (and update) in one persistent launch (qoc_plan_set_persistent).
int persistent_impl(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3,
                    double* grad, double* u_update, const UpdateRule& rule, char* w, cudaStream_t st) {
    const bool want_grad = grad || u_update;
    p->pk_last = !p->capturing;
    if (launch_persistent(p->dev(), p->tabs, u_update ? u_update : const_cast<double*>(u),
                          reinterpret_cast<const double2*>(psi0), reinterpret_cast<const double2*>(psif),
                          p->d_prob_state, out3, reinterpret_cast<double2*>(w + p->off_o),
                          reinterpret_cast<double2*>(w + p->off_partial), grad, rule, w + p->off_U, w + p->off_psi,
                          w + p->off_lam, ckpt_vec(p, w, 0), ckpt_vec(p, w, 1), lamb_vec(p, w, 0), lamb_vec(p, w, 1),
                          w + p->off_pk, p->pk_slot, p->max_m, want_grad ? 1 : 0,
                          reinterpret_cast<unsigned*>(w + p->off_pksync), p->d_pk_ts, p->pk_grid, p->pk_smem, st) != 0)
        return cuda_fail(cudaGetLastError(), "persistent launch");
    return QOC_OK;
}

// One F (+ gradient, + update) evaluation.  Without checkpointing the forward states and costates
// run in one sweep launch; with it, the costate pass recomputes each segment's propagators.
int fidelity_grad_impl(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3,
                       double* grad, double* u_update, const UpdateRule& rule, char* w, cudaStream_t st) {
    if (p->pk_on) return persistent_impl(p, u, psi0, psif, out3, grad, u_update, rule, w, st);
    p->pk_last = false;
    int rc;
    const DevPlan P = p->dev();
    sections_begin(p);
    const bool want_grad = grad || u_update;
    double2* o_ws = reinterpret_cast<double2*>(w + p->off_o);
    if (p->nseg == 1) {
        if (launch_gather(P, reinterpret_cast<const double2*>(psi0), ckpt_vec(p, w, 0), st) != 0 ||
            (want_grad && launch_gather(P, reinterpret_cast<const double2*>(psif), lamb_vec(p, w, 0), st) != 0))
            return cuda_fail(cudaGetLastError(), "gather launch");
        if ((rc = run_expm(p, u, w, 0, -1, st))) return rc;
        if ((rc = run_sweeps(p, w, 0, -1, want_grad ? 3 : 1, ckpt_vec(p, w, 0), ckpt_vec(p, w, 1), lamb_vec(p, w, 0),
                             lamb_vec(p, w, 1), st)))
            return rc;
        {
            Timed tm(p, PH_OVERLAP, st);
            if (launch_overlap(P, ckpt_vec(p, w, 1), reinterpret_cast<const double2*>(psif), out3, o_ws, st) != 0)
                return cuda_fail(cudaGetLastError(), "overlap launch");
        }
        if (want_grad && (rc = run_grad(p, u, w, 0, -1, st))) return rc;
    } else {
        if ((rc = forward_pass(p, u, psi0, w, st))) return rc;
        {
            Timed tm(p, PH_OVERLAP, st);
            if (launch_overlap(P, ckpt_vec(p, w, p->nseg), reinterpret_cast<const double2*>(psif), out3, o_ws, st) != 0)
                return cuda_fail(cudaGetLastError(), "overlap launch");
        }
        if (want_grad) {
            if (launch_gather(P, reinterpret_cast<const double2*>(psif), lamb_vec(p, w, 0), st) != 0)
                return cuda_fail(cudaGetLastError(), "gather launch");
            // costate pass: recompute each segment's propagators and states, newest segment first
            int cur = 0;
            for (int s = p->nseg - 1; s >= 0; --s) {
                int k0, nk;
                window_of(p, s, &k0, &nk);
                if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
                if ((rc = run_sweeps(p, w, k0, nk, 3, ckpt_vec(p, w, s), ckpt_vec(p, w, s + 1), lamb_vec(p, w, cur),
                                     lamb_vec(p, w, cur ^ 1), st)))
                    return rc;
                if ((rc = run_grad(p, u, w, k0, nk, st))) return rc;
                cur ^= 1;
            }
        }
    }
    if (want_grad) {
        Timed tm(p, PH_REDUCE, st);
        if (launch_grad_reduce(P, reinterpret_cast<const double2*>(w + p->off_partial), o_ws, grad, u_update, rule,
                               out3, st) != 0)
            return cuda_fail(cudaGetLastError(), "reduce launch");
    }
    return QOC_OK;
}

// The forward half of fidelity_grad_impl: propagators, forward states (every slice, or the segment
// boundaries when checkpointing) and the overlaps; the workspace keeps what backward_impl needs.
int forward_impl(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3, char* w,
                 cudaStream_t st) {
    int rc;
    sections_begin(p);
    if ((rc = forward_pass(p, u, psi0, w, st))) return rc;
    Timed tm(p, PH_OVERLAP, st);
    if (launch_overlap(p->dev(), ckpt_vec(p, w, p->nseg), reinterpret_cast<const double2*>(psif), out3,
                       reinterpret_cast<double2*>(w + p->off_o), st) != 0)
        return cuda_fail(cudaGetLastError(), "overlap launch");
    return QOC_OK;
}

// The backward half: costates from lam_N = psi_f, exact slice derivatives (recomputing each segment's
// propagators and states when checkpointing) and grad = gF_p dF_p/du.
int backward_impl(const qoc_plan* p, const double* u, const double* psif, const double* gF, double* grad, char* w,
                  cudaStream_t st) {
    int rc;
    sections_begin(p);
    const DevPlan P = p->dev();
    if (launch_gather(P, reinterpret_cast<const double2*>(psif), lamb_vec(p, w, 0), st) != 0)
        return cuda_fail(cudaGetLastError(), "gather launch");
    if (p->nseg == 1) {
        if ((rc = run_sweeps(p, w, 0, -1, 2, nullptr, nullptr, lamb_vec(p, w, 0), lamb_vec(p, w, 1), st))) return rc;
        if ((rc = run_grad(p, u, w, 0, -1, st))) return rc;
    } else {
        int cur = 0;
        for (int s = p->nseg - 1; s >= 0; --s) {
            int k0, nk;
            window_of(p, s, &k0, &nk);
            if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
            if ((rc = run_sweeps(p, w, k0, nk, 3, ckpt_vec(p, w, s), ckpt_vec(p, w, s + 1), lamb_vec(p, w, cur),
                                 lamb_vec(p, w, cur ^ 1), st)))
                return rc;
            if ((rc = run_grad(p, u, w, k0, nk, st))) return rc;
            cur ^= 1;
        }
    }
    UpdateRule rule = no_update();
    rule.gscale = gF;
    Timed tm(p, PH_REDUCE, st);
    if (launch_grad_reduce(P, reinterpret_cast<const double2*>(w + p->off_partial),
                           reinterpret_cast<const double2*>(w + p->off_o), grad, nullptr, rule,
                           reinterpret_cast<const double*>(w + p->off_out3), st) != 0)
        return cuda_fail(cudaGetLastError(), "reduce launch");
    return QOC_OK;
}

}  // namespace

extern "C" {

void qoc_plan_opts_default(qoc_plan_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec = QOC_PREC_F64;
    o->grad_mode = 0;
    o->max_squarings = 16;
    o->ckpt_segment = 0;
}

void qoc_plan_free(qoc_plan* p);

int qoc_plan_create_batch(const qoc_basis* const* bases, int n_problems, const int* Ns, const double* dts,
                          const qoc_plan_opts* opts, const uint8_t* const* actives, qoc_plan** out) {
    if (!bases || !Ns || !dts || !out || n_problems < 1) return set_error(QOC_EINVAL, "null argument or no problem");
    *out = nullptr;
    qoc_plan_opts o;
    if (opts) o = *opts; else qoc_plan_opts_default(&o);
    if (o.prec < QOC_PREC_F64 || o.prec > QOC_PREC_F32_ALL) return set_error(QOC_EINVAL, "unknown precision");
    if (o.grad_mode != 0 && o.grad_mode != 1) return set_error(QOC_EINVAL, "unknown grad_mode");
    if (o.max_squarings <= 0) o.max_squarings = 16;
    if (o.max_squarings > 40) return set_error(QOC_EINVAL, "max_squarings must be <= 40");
    if (o.ckpt_segment < -1) return set_error(QOC_EINVAL, "ckpt_segment must be -1, 0 or positive");
    if (o.ckpt_segment != 0 && n_problems > 1) return set_error(QOC_EINVAL, "checkpointing needs a single-problem plan");
    if (o.objective != QOC_OBJ_STATE && o.objective != QOC_OBJ_GATE) return set_error(QOC_EINVAL, "unknown objective");
    const bool gate = o.objective == QOC_OBJ_GATE;
    if (gate && actives)
        for (int i = 0; i < n_problems; ++i)
            if (actives[i]) return set_error(QOC_EINVAL, "the gate objective uses every column of every block: pass no active mask");
    const int nc = bases[0] ? bases[0]->n_ctrl : 0;
    for (int i = 0; i < n_problems; ++i) {
        if (!bases[i]) return set_error(QOC_EINVAL, "null basis");
        if (bases[i]->n_ctrl != nc) return set_error(QOC_EINVAL, "every problem needs the same number of controls");
        if (Ns[i] < 1) return set_error(QOC_EINVAL, "N must be >= 1");
        if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return set_error(QOC_EINVAL, "dt must be positive and finite");
    }
    if (nc < 1 || nc > 8) return set_error(QOC_EUNSUPPORTED, "1..8 controls");

    auto* p = new (std::nothrow) qoc_plan();
    if (!p) return set_error(QOC_ENOMEM, "host allocation failed");
    p->opts = o;
    p->nc = nc;
    p->n_prob = n_problems;
    cudaGetDevice(&p->device);
    // the FP32 paths store propagators and states in complex FP32
    const size_t el = o.prec == QOC_PREC_F64 ? 16 : 8;
    p->el = el;
    const int wp = o.prec == QOC_PREC_F64 ? 0 : 1;  // working precision passed to the kernels

    int64_t state_off = 0, u_row = 0;
    int maxN = 0;
    for (int i = 0; i < n_problems; ++i) {
        int64_t len = bases[i]->state_len;
        if (gate) {
            len = 0;
            for (const auto& blk : bases[i]->blocks) len += (int64_t)blk.m * blk.m;
        }
        p->probs.push_back({bases[i], Ns[i], dts[i], state_off, len, u_row});
        state_off += len;
        u_row += Ns[i];
        maxN = std::max(maxN, Ns[i]);
    }
    p->rows = u_row;
    p->state_len = state_off;
    p->N = maxN;
    p->dt = dts[0];
    p->seg = o.ckpt_segment == 0 ? Ns[0]
             : o.ckpt_segment < 0 ? std::max(1, (int)std::ceil(std::sqrt((double)Ns[0])))
                                  : std::min(o.ckpt_segment, Ns[0]);
    p->nseg = n_problems == 1 ? (Ns[0] + p->seg - 1) / p->seg : 1;
    if (n_problems > 1) p->seg = 0;

    // active blocks of every problem, ordered by size (largest first) for load balance
    struct Act { int prob; int b; std::vector<int> copies; };
    std::vector<Act> acts;
    for (int i = 0; i < n_problems; ++i) {
        const qoc_basis* B = bases[i];
        int64_t copy_counter = 0;
        for (int b = 0; b < (int)B->blocks.size(); ++b) {
            const auto& blk = B->blocks[b];
            Act a{i, b, {}};
            if (gate) {  // the m columns of the block's unitary
                for (int r = 0; r < blk.m; ++r) a.copies.push_back(r);
                acts.push_back(std::move(a));
                continue;
            }
            for (int r = 0; r < blk.c; ++r, ++copy_counter)
                if (!actives || !actives[i] || actives[i][copy_counter]) a.copies.push_back(r);
            if (!a.copies.empty()) acts.push_back(std::move(a));
        }
    }
    if (acts.empty()) {
        delete p;
        return set_error(QOC_EINVAL, "no active block copy");
    }
    std::stable_sort(acts.begin(), acts.end(), [&](const Act& x, const Act& y) {
        return bases[x.prob]->blocks[x.b].m > bases[y.prob]->blocks[y.b].m;
    });
    p->nb = (int)acts.size();

    int64_t h_off = 0, u_off = 0, s_off = 0, v_off = 0, part_off = 0;
    std::vector<cplx> H64;
    std::vector<std::vector<int>> per_prob(n_problems);
    for (int bi = 0; bi < p->nb; ++bi) {
        const auto& a = acts[bi];
        const auto& pr = p->probs[a.prob];
        const auto& blk = pr.basis->blocks[a.b];
        const int slots = p->nseg == 1 ? pr.N : p->seg;
        DevBlock d{};
        d.m = blk.m;
        d.c = (int)a.copies.size();
        d.b = a.b;
        d.prob = a.prob;
        d.N = pr.N;
        d.dt = pr.dt;
        d.u_row = pr.u_row;
        d.part_off = part_off;
        d.mmp = ((int64_t)blk.m * blk.m + 3) / 4 * 4;
        d.h_off = h_off;
        d.u_off = u_off;
        d.s_off = s_off;
        d.v_off = v_off;
        d.h0_norm = blk.h0_norm;
        for (int j = 0; j < nc; ++j) d.hc_norm[j] = blk.hc_norm[j];
        p->copy_base.push_back((int64_t)p->copy_src.size());
        int64_t boff = blk.offset;
        if (gate) {  // block-state layout of the gate objective: [block][column][m]
            boff = 0;
            for (int b2 = 0; b2 < a.b; ++b2) boff += (int64_t)pr.basis->blocks[b2].m * pr.basis->blocks[b2].m;
        }
        for (int r : a.copies) p->copy_src.push_back(pr.state_off + boff + (int64_t)r * blk.m);
        H64.insert(H64.end(), blk.h0.begin(), blk.h0.end());
        H64.insert(H64.end(), blk.hc.begin(), blk.hc.end());
        h_off += (int64_t)(1 + nc) * blk.m * blk.m;
        u_off += (int64_t)slots * d.mmp;
        s_off += (int64_t)(slots + 1) * d.c * d.m;
        v_off += (int64_t)d.c * d.m;
        part_off += pr.N;
        p->max_m = std::max(p->max_m, d.m);
        p->max_c = std::max(p->max_c, d.c);
        p->hblocks.push_back(d);
        per_prob[a.prob].push_back(bi);
        for (int k = 0; k < pr.N; ++k) p->items.push_back(make_int2(bi, k));
    }
    p->vlen = v_off;
    p->prob_block_off.push_back(0);
    for (int i = 0; i < n_problems; ++i) {
        p->prob_blocks.insert(p->prob_blocks.end(), per_prob[i].begin(), per_prob[i].end());
        p->prob_block_off.push_back((int)p->prob_blocks.size());
    }
    // export layout (assemble / expm outputs): problem by problem, active blocks in basis order
    {
        std::vector<int> order(p->nb);
        for (int i = 0; i < p->nb; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            const auto& X = p->hblocks[x];
            const auto& Y = p->hblocks[y];
            return X.prob != Y.prob ? X.prob < Y.prob : X.b < Y.b;
        });
        p->a_off.assign(p->nb, 0);
        long long acc = 0;
        for (int i : order) {
            p->a_off[i] = acc;
            acc += (long long)p->hblocks[i].N * p->hblocks[i].m * p->hblocks[i].m;
        }
    }

    // Taylor degree table: FP64 unit roundoff for the FP64 path, FP32 otherwise
    const int degs[9] = {2, 4, 6, 9, 12, 16, 20, 25, 30};
    const double unit = o.prec == QOC_PREC_F64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    for (int i = 0; i < 9; ++i) p->tabs.theta[i] = theta_for(degs[i], unit);
    // tensor-core degrees: its products round at about 2^-23 (two FP16 halves, FP32 accumulation), so
    // the truncation bound is matched to that rather than to FP32's 2^-24
    const double tc_unit = o.prec == QOC_PREC_F64 ? unit : std::ldexp(1.0, -23);
    for (int q = 1; q <= 16; ++q) p->tabs.theta_odd[q - 1] = theta_for(2 * q - 1, tc_unit);
    if (o.prec == QOC_PREC_F64) {
        p->tabs.n_deg = 9;
        p->tabs.theta_cap = p->tabs.theta[8];
    } else {
        p->tabs.n_deg = 7;
        p->tabs.theta_cap = std::min(p->tabs.theta[6], 3.0);
    }
    p->tabs.sq_f64 = o.prec == QOC_PREC_F32_ALL ? 0 : 1;

    // expm size classes.  In plans with the FP64 squaring chain the slices of blocks with 25..2048
    // states that need no squaring go to the tensor cores (one CTA per slice up to 112 states, tiled
    // GEMMs beyond); a tensor-core product errs up to about 2x
    // an FP32 one, so slices whose squarings would amplify that stay on the tiled CUDA-core kernels,
    // as do all other blocks.  All-FP32 plans (typically large norms, where most slices are squared)
    // keep the tiled kernels; the autotuner may pick warp-packed or tensor-core rules.
    if (o.prec == QOC_PREC_F32) {
        p->rules.push_back({24, 0, 0});
        p->rules.push_back({112, 2, 0});
        p->rules.push_back({2048, 3, 0});  // larger blocks: tiled tensor-core GEMMs
    }
    p->rules.push_back({1 << 30, 0, 0});
    {
        const int rc = build_classes(p);
        if (rc) {
            qoc_plan_free(p);
            return rc;
        }
    }
    // gradient kernel
    p->grad_slot = align_up(grad_slot_bytes(wp, p->max_m), 256);
    const long long grad_items = p->nseg == 1 ? (long long)p->items.size() : (long long)p->seg * p->nb;
    p->grad_grid = (int)std::min<long long>(grad_items, grad_grid_limit(wp, p->max_m));
    p->sweep_cl = sweep_cluster_size(wp, p->nb, p->max_m, p->max_c);
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        p->gf_grid = (int)std::max<long long>(1, std::min<long long>(grad_items, sms));
    }
    // reverse-mode kernel for large-norm slices: one scratch slot per CTA, at most 256 MiB in total
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        p->rev_slot = align_up(grad_rev_slot_bytes(wp == QOC_PREC_F64 ? 0 : 1, p->max_m), 256);
        const long long by_mem = std::max<long long>(1, (256LL << 20) / (long long)p->rev_slot);
        p->rev_grid = (int)std::max<long long>(1, std::min<long long>({grad_items, (long long)sms, by_mem}));
    }

    // workspace layout
    p->u_elems = u_off;
    p->s_elems = s_off;
    p->part_rows = part_off;
    layout_workspace(p, u_off, s_off, part_off);

    // device uploads
    auto fail = [&](cudaError_t e, const char* what) {
        int rc = cuda_fail(e, what);
        qoc_plan_free(p);
        return rc;
    };
    cudaError_t e;
#define QOC_UP(dst, src, n, what)                                                             \
    do {                                                                                      \
        if ((e = cudaMalloc(&(dst), sizeof(*(src)) * std::max<size_t>(1, (n)))) != cudaSuccess) \
            return fail(e, what);                                                             \
        if ((n) > 0 && (e = cudaMemcpy((dst), (src), sizeof(*(src)) * (n), cudaMemcpyHostToDevice)) != cudaSuccess) \
            return fail(e, what);                                                             \
    } while (0)
    QOC_UP(p->d_blocks, p->hblocks.data(), p->hblocks.size(), "upload blocks");
    QOC_UP(p->d_copy_src, p->copy_src.data(), p->copy_src.size(), "upload copies");
    QOC_UP(p->d_copy_base, p->copy_base.data(), p->copy_base.size(), "upload copies");
    QOC_UP(p->d_a_off, p->a_off.data(), p->a_off.size(), "upload offsets");
    QOC_UP(p->d_items, p->items.data(), p->items.size(), "upload items");
    QOC_UP(p->d_prob_blocks, p->prob_blocks.data(), p->prob_blocks.size(), "upload problems");
    QOC_UP(p->d_prob_block_off, p->prob_block_off.data(), p->prob_block_off.size(), "upload problems");
    QOC_UP(p->d_H64, reinterpret_cast<double2*>(H64.data()), H64.size(), "upload H");
    {
        std::vector<int64_t> ps;
        for (const auto& pr : p->probs) {
            ps.push_back(pr.state_off);
            ps.push_back(pr.state_len);
        }
        QOC_UP(p->d_prob_state, ps.data(), ps.size(), "upload problems");
    }
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc status");
    if ((e = cudaHostAlloc(&p->h_status, sizeof(int), cudaHostAllocDefault)) != cudaSuccess)
        return fail(e, "cudaHostAlloc status");
    *p->h_status = 0;
    if ((e = cudaEventCreateWithFlags(&p->st_ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e, "cudaEventCreate");
    if ((e = cudaMalloc(&p->d_stats, 8 * sizeof(unsigned long long))) != cudaSuccess) return fail(e, "cudaMalloc stats");
    cudaMemset(p->d_stats, 0, 8 * sizeof(unsigned long long));
    cudaMemset(p->d_status, 0, sizeof(int));
#undef QOC_UP
    if (o.prec == QOC_PREC_F64) {
        p->d_H = p->d_H64;
    } else {
        std::vector<float> H32(2 * H64.size());
        for (size_t i = 0; i < H64.size(); ++i) {
            H32[2 * i] = (float)H64[i].real();
            H32[2 * i + 1] = (float)H64[i].imag();
        }
        if ((e = cudaMalloc(&p->d_H, sizeof(float) * H32.size())) != cudaSuccess) return fail(e, "cudaMalloc H32");
        cudaMemcpy(p->d_H, H32.data(), sizeof(float) * H32.size(), cudaMemcpyHostToDevice);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "plan upload");
    {
        const int rc = build_gg(p);
        if (rc) {
            qoc_plan_free(p);
            return rc;
        }
        layout_workspace(p, p->u_elems, p->s_elems, p->part_rows);
    }
    *out = p;
    return QOC_OK;
}

int qoc_plan_create(const qoc_basis* B, int N, double dt, const qoc_plan_opts* opts, const uint8_t* active,
                    qoc_plan** out) {
    if (!B) return set_error(QOC_EINVAL, "null basis");
    const uint8_t* acts[1] = {active};
    return qoc_plan_create_batch(&B, 1, &N, &dt, opts, acts, out);
}

void qoc_plan_free(qoc_plan* p) {
    if (!p) return;
    cudaFree(p->d_blocks);
    cudaFree(p->d_copy_src);
    cudaFree(p->d_copy_base);
    cudaFree(p->d_a_off);
    if (p->d_H && p->d_H != p->d_H64) cudaFree(p->d_H);
    cudaFree(p->d_H64);
    cudaFree(p->d_cls);
    cudaFree(p->d_cls_items);
    cudaFree(p->d_items);
    cudaFree(p->d_prob_blocks);
    cudaFree(p->d_prob_block_off);
    cudaFree(p->d_gg);
    cudaFree(p->d_gg_tiles);
    cudaFree(p->d_gg_hplanes);
    cudaFree(p->d_gg_hoff);
    cudaFree(p->d_pk_ts);
    cudaFree(p->d_status);
    cudaFree(p->d_prob_state);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->st_ev) cudaEventDestroy(p->st_ev);
    cudaFree(p->d_stats);
    for (auto& ev : p->sec_ev)
        if (ev) cudaEventDestroy(ev);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    delete p;
}

int qoc_plan_info(const qoc_plan* p, int* n_problems, int64_t* pulse_rows, int64_t* state_len) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    if (n_problems) *n_problems = p->n_prob;
    if (pulse_rows) *pulse_rows = p->rows;
    if (state_len) *state_len = p->state_len;
    return QOC_OK;
}

int qoc_plan_workspace_bytes(const qoc_plan* p, size_t* bytes) {
    if (!p || !bytes) return set_error(QOC_EINVAL, "null argument");
    *bytes = p->ws_bytes;
    return QOC_OK;
}

int qoc_plan_sync_status(qoc_plan* p, void* stream) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    cudaSetDevice(p->device);
    cudaError_t e = cudaStreamSynchronize(to_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    cudaMemset(p->d_status, 0, sizeof(int));
    *reinterpret_cast<volatile int*>(p->h_status) = 0;
    p->st_recorded = false;
    return status_error(st);
}

int qoc_plan_selftest_wait(qoc_plan* p, double limit_ms, void* stream) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    if (!(limit_ms >= 0.001 && limit_ms <= 1000.0)) return set_error(QOC_EINVAL, "limit_ms must be in [0.001, 1000]");
    cudaSetDevice(p->device);
    cudaStream_t st = to_stream(stream);
    if (launch_wait_selftest((unsigned long long)(limit_ms * 1e6), p->d_status, st) != 0)
        return cuda_fail(cudaGetLastError(), "self-test launch");
    record_status(p, st);
    return QOC_OK;
}

int qoc_plan_set_profiling(qoc_plan* p, int on) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    cudaSetDevice(p->device);
    p->profiling = on != 0;
    if (on) cudaMemset(p->d_stats, 0, 8 * sizeof(unsigned long long));
    return QOC_OK;
}

int qoc_plan_phase_times(qoc_plan* p, float* ms, int n) {
    if (!p || !ms) return set_error(QOC_EINVAL, "null argument");
    if (!p->profiling) return set_error(QOC_EINVAL, "profiling is off");
    if (p->pk_last) {
        cudaSetDevice(p->device);
        unsigned long long t[8];
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(t, p->d_pk_ts, sizeof(t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "persistent phase stamps");
        for (int i = 0; i < n && i < 5; ++i) ms[i] = (float)((double)(t[i + 2] - t[i + 1]) * 1e-6);
        return QOC_OK;
    }
    if (p->sec_phase.empty()) return set_error(QOC_EINVAL, "no call was timed since profiling was enabled");
    cudaSetDevice(p->device);
    const size_t last = 2 * p->sec_phase.size() - 1;
    cudaError_t e = cudaEventSynchronize(p->sec_ev[last]);
    if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (size_t i = 0; i < p->sec_phase.size(); ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->sec_ev[2 * i], p->sec_ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event elapsed");
        acc[p->sec_phase[i]] += t;
    }
    for (int i = 0; i < n && i < 5; ++i) ms[i] = acc[i];
    return QOC_OK;
}

int qoc_plan_work_counts(qoc_plan* p, long long* out, int n) {
    if (!p || !out) return set_error(QOC_EINVAL, "null argument");
    cudaSetDevice(p->device);
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(h, p->d_stats, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats read");
    for (int i = 0; i < n && i < 6; ++i) out[i] = (long long)h[i];
    return QOC_OK;
}

int qoc_plan_kernel_launches(const qoc_plan* p, int with_grad, int* launches) {
    if (!p || !launches) return set_error(QOC_EINVAL, "null argument");
    // gathers, one expm launch per size class, sweeps, overlap, slice derivatives, reduction
    // (+ the iteration counter when optimising); propagate: gather, expm, sweep, memset, store
    const int nrev = (int)p->classes.size();  // reverse-mode derivative launches: one per class
    int ncls = 0;                               // exponential launches per pass over all slices
    for (const auto& c : p->classes) {
        if (c.kind == 3) {
            std::vector<int> hm(c.count);
            std::vector<long long> hcount(c.count);
            for (int i = 0; i < c.count; ++i) {
                const DevBlock& hb = p->hblocks[p->h_cls[c.offset + i]];
                hm[i] = hb.m;
                hcount[i] = p->nseg == 1 ? hb.N : p->seg;
            }
            ncls += (int)expm_large_launches(p->tabs, c.m_max, hm.data(), hcount.data(), c.count) + 1;
        } else {
            ncls += (c.kind == 2 && c.R == 0) ? 2 : 1;
        }
    }
    // register-tile derivative launch per gradient pass (FP32 plans), plus the GEMM path's chunks:
    // prep, load, (GG_PCAP + 1) GEMM + combine steps, contraction
    if (p->pk_on && with_grad) {  // one cooperative launch (its counters are zeroed by a memset)
        *launches = 1;
        return QOC_OK;
    }
    int gfl = (grad_fast_max_m(p->opts.prec) > 0 && p->nc <= 8) ? 1 : 0;
    if (p->gg_mode != GG_OFF && !p->gg.empty() && p->opts.grad_mode == 0) {
        const int slots = p->nseg == 1 ? p->N : p->seg;
        gfl += ((slots + p->gg_S - 1) / p->gg_S) * (3 + (p->gg_mode == GG_TC ? 3 : 2) * (GG_PCAP + 1));
    }
    if (p->nseg == 1)
        *launches = with_grad ? 2 + ncls + 1 + 1 + 1 + gfl + nrev + 1 : 1 + ncls + 1 + 1;
    else
        *launches = with_grad ? 1 + p->nseg * (ncls + 1) + 1 + 1 + p->nseg * (ncls + nrev + 2 + gfl) + 1
                              : 1 + p->nseg * (ncls + 1) + 1;
    return QOC_OK;
}

int qoc_plan_set_sweep_cluster(qoc_plan* p, int cl) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    if (cl == -1) {
        p->sweep_cl = sweep_cluster_size(p->opts.prec, p->nb, p->max_m, p->max_c);
        return QOC_OK;
    }
    if (cl != 0 && (cl < 2 || cl > 8)) return set_error(QOC_EINVAL, "cluster size must be -1, 0 or 2..8");
    if (cl > 0 && !sweep_cluster_fits(p->opts.prec, p->max_m, p->max_c, cl))
        return set_error(QOC_EUNSUPPORTED, "cluster sweep buffers do not fit in shared memory");
    p->sweep_cl = cl;
    return QOC_OK;
}

int qoc_plan_set_deriv_gemm(qoc_plan* p, int mode, int min_m) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    if (mode < GG_OFF || mode > GG_TC) return set_error(QOC_EINVAL, "mode must be 0 (off), 1 (CUDA cores) or 2 (tensor cores)");
    if (min_m != 0 && (min_m < 8 || min_m > 4096)) return set_error(QOC_EINVAL, "min_m must be 0 (keep) or 8..4096");
    cudaSetDevice(p->device);
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->gg_mode = mode;
    if (min_m) p->gg_min_m = min_m;
    const int rc = build_gg(p);
    if (rc) return rc;
    layout_workspace(p, p->u_elems, p->s_elems, p->part_rows);
    return QOC_OK;
}

int qoc_plan_deriv_gemm(const qoc_plan* p, int* blocks) {
    if (!p || !blocks) return set_error(QOC_EINVAL, "null argument");
    *blocks = p->gg_mode != GG_OFF ? (int)p->gg.size() : 0;
    return QOC_OK;
}

int qoc_plan_set_persistent(qoc_plan* p, int on) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    if (on != 0 && on != 1) return set_error(QOC_EINVAL, "on must be 0 or 1");
    cudaSetDevice(p->device);
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    if (!on) {
        p->pk_on = false;
        p->pk_last = false;
        layout_workspace(p, p->u_elems, p->s_elems, p->part_rows);
        return QOC_OK;
    }
    if (p->opts.prec != QOC_PREC_F64) return set_error(QOC_EUNSUPPORTED, "the persistent iteration runs FP64 plans");
    if (p->nseg != 1) return set_error(QOC_EUNSUPPORTED, "the persistent iteration keeps every propagator (no checkpointing)");
    if (p->opts.grad_mode != 0) return set_error(QOC_EUNSUPPORTED, "the persistent iteration computes the exact derivative");
    int grid = 0;
    size_t slot = 0, smem = 0;
    if (!persistent_config(p->max_m, p->max_c, &grid, &slot, &smem))
        return set_error(QOC_EUNSUPPORTED, "the persistent kernel's buffers do not fit in shared memory");
    if (!p->d_pk_ts) {
        cudaError_t e = cudaMalloc(&p->d_pk_ts, 8 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc stamps");
        cudaMemset(p->d_pk_ts, 0, 8 * sizeof(unsigned long long));
    }
    p->pk_grid = grid;
    p->pk_slot = slot;
    p->pk_smem = smem;
    p->pk_on = true;
    layout_workspace(p, p->u_elems, p->s_elems, p->part_rows);
    return QOC_OK;
}


int qoc_plan_sweep_cluster(const qoc_plan* p, int* cl) {
    if (!p || !cl) return set_error(QOC_EINVAL, "null argument");
    *cl = p->sweep_cl;
    return QOC_OK;
}

int qoc_plan_set_expm_rules(qoc_plan* p, int n_rules, const int* m_max, const int* kind, const int* param) {
    if (!p || n_rules < 1 || !m_max || !kind || !param) return set_error(QOC_EINVAL, "null argument or no rule");
    std::vector<ExpmRule> rules;
    for (int i = 0; i < n_rules; ++i) {
        if (kind[i] < 0 || kind[i] > 3)
            return set_error(QOC_EINVAL,
                             "rule kind must be 0 (CTA tiles), 1 (warp-packed), 2 (tensor cores) or 3 (tiled tensor cores)");
        if (param[i] < 0) return set_error(QOC_EINVAL, "rule parameter must be >= 0");
        if (kind[i] == 2 && param[i] > 1)
            return set_error(QOC_EINVAL, "tensor-core rule parameter must be 0 (unsquared slices) or 1 (all)");
        rules.push_back({m_max[i], kind[i], param[i]});
    }
    std::stable_sort(rules.begin(), rules.end(), [](const ExpmRule& a, const ExpmRule& b) { return a.m_max < b.m_max; });
    rules.push_back({1 << 30, 0, 0});  // fallback: CTA tiles sized by m
    cudaSetDevice(p->device);
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->rules = rules;
    const int rc = build_classes(p);
    if (rc) return rc;
    layout_workspace(p, p->u_elems, p->s_elems, p->part_rows);
    return QOC_OK;
}

int qoc_plan_expm_classes(const qoc_plan* p, int max_out, int* n_classes, int* kind, int* param, int* per_warp,
                          int* m_max, int* n_blocks) {
    if (!p || !n_classes) return set_error(QOC_EINVAL, "null argument");
    *n_classes = (int)p->classes.size();
    for (int i = 0; i < (int)p->classes.size() && i < max_out; ++i) {
        const auto& c = p->classes[i];
        if (kind) kind[i] = c.kind;
        if (param) param[i] = c.R;
        if (per_warp) per_warp[i] = c.per_warp;
        if (m_max) m_max[i] = c.m_max;
        if (n_blocks) n_blocks[i] = c.count;
    }
    return QOC_OK;
}

int qoc_assemble_blocks(const qoc_plan* p, const double* u, double* A_out, void* stream) {
    if (!p || !u || !A_out) return set_error(QOC_EINVAL, "null argument");
    cudaSetDevice(p->device);
    if (launch_assemble(p->dev(), u, reinterpret_cast<double2*>(A_out), p->d_a_off, to_stream(stream)) != 0)
        return cuda_fail(cudaGetLastError(), "assemble launch");
    return QOC_OK;
}

int qoc_expm_blocks(const qoc_plan* p, const double* u, double* U_out, void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !U_out) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    char* w = static_cast<char*>(ws);
    cudaStream_t st = to_stream(stream);
    if ((rc = take_latched(p, st))) return rc;
    if (p->nseg == 1) {
        if ((rc = run_expm(p, u, w, 0, -1, st))) return rc;
        if (launch_export_u(p->dev(), w + p->off_U, reinterpret_cast<double2*>(U_out), p->d_a_off, st) != 0)
            return cuda_fail(cudaGetLastError(), "export launch");
        record_status(p, st);
        return QOC_OK;
    }
    for (int s = 0; s < p->nseg; ++s) {
        int k0, nk;
        window_of(p, s, &k0, &nk);
        if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
        if (launch_export_u(p->dev(k0, nk), w + p->off_U, reinterpret_cast<double2*>(U_out), p->d_a_off, st) != 0)
            return cuda_fail(cudaGetLastError(), "export launch");
    }
    record_status(p, st);
    return QOC_OK;
}

int qoc_propagate(const qoc_plan* p, const double* u, const double* psi0, double* psiN, void* ws, size_t ws_bytes,
                  void* stream) {
    if (!p || !u || !psi0 || !psiN) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    char* w = static_cast<char*>(ws);
    cudaStream_t st = to_stream(stream);
    if ((rc = take_latched(p, st))) return rc;
    if ((rc = check_norms(p, psi0, nullptr, st))) return rc;
    if ((rc = forward_pass(p, u, psi0, w, st))) return rc;
    if (launch_store_final(p->dev(), ckpt_vec(p, w, p->nseg), reinterpret_cast<double2*>(psiN), p->state_len, st) != 0)
        return cuda_fail(cudaGetLastError(), "store launch");
    record_status(p, st);
    return QOC_OK;
}

int qoc_fidelity_and_grad(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3,
                          double* grad, void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !psi0 || !psif || !out3) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    cudaStream_t st = to_stream(stream);
    if ((rc = take_latched(p, st))) return rc;
    if (!p->pk_on && (rc = check_norms(p, psi0, psif, st))) return rc;
    rc = fidelity_grad_impl(p, u, psi0, psif, out3, grad, nullptr, no_update(), static_cast<char*>(ws), st);
    if (rc == QOC_OK) record_status(p, st);
    return rc;
}

int qoc_fidelity_forward(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3,
                         void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !psi0 || !psif || !out3) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    cudaStream_t st = to_stream(stream);
    if ((rc = take_latched(p, st))) return rc;
    if ((rc = check_norms(p, psi0, psif, st))) return rc;
    p->pk_last = false;
    rc = forward_impl(p, u, psi0, psif, out3, static_cast<char*>(ws), st);
    if (rc == QOC_OK) record_status(p, st);
    return rc;
}

int qoc_fidelity_backward(const qoc_plan* p, const double* u, const double* psif, const double* gF, double* grad,
                          void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !psif || !grad) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    cudaStream_t st = to_stream(stream);
    if ((rc = take_latched(p, st))) return rc;
    p->pk_last = false;
    rc = backward_impl(p, u, psif, gF, grad, static_cast<char*>(ws), st);
    if (rc == QOC_OK) record_status(p, st);
    return rc;
}

void qoc_opt_opts_default(qoc_opt_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->iters = 100;
    o->rule = QOC_RULE_FIXED;
    o->step = 0.1;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->f_target = 2.0;
    o->check_every = 10;
    o->use_graph = 0;
    o->freeze_converged = 1;
}

int qoc_optimize_pulses(qoc_plan* p, double* u, const double* psi0, const double* psif, const qoc_opt_opts* oo,
                        double* F_hist, int* reached, int* iters_done, void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !psi0 || !psif || !F_hist || !oo) return set_error(QOC_EINVAL, "null argument");
    const qoc_opt_opts o = *oo;
    if (o.iters < 0) return set_error(QOC_EINVAL, "iters must be >= 0");
    if (o.rule != QOC_RULE_FIXED && o.rule != QOC_RULE_ADAM) return set_error(QOC_EINVAL, "unknown update rule");
    if (!std::isfinite(o.step)) return set_error(QOC_EINVAL, "step must be finite");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    char* w = static_cast<char*>(ws);
    cudaStream_t st = to_stream(stream);
    if (o.use_graph && st == nullptr) return set_error(QOC_EINVAL, "graph replay needs a non-default stream");
    if ((rc = take_latched(p, st))) return rc;
    if (!p->pk_on && (rc = check_norms(p, psi0, psif, st))) return rc;
    double* out3 = reinterpret_cast<double*>(w + p->off_out3);
    int* d_iter = reinterpret_cast<int*>(w + p->off_iter);
    int* d_reached = reached ? reached : reinterpret_cast<int*>(w + p->off_reached);
    UpdateRule rule{};
    rule.kind = o.rule;
    rule.freeze = o.freeze_converged && o.f_target <= 1.0;
    rule.step = o.step;
    rule.beta1 = o.beta1;
    rule.beta2 = o.beta2;
    rule.eps = o.eps;
    rule.f_target = o.f_target;
    rule.iter = d_iter;
    rule.reached = d_reached;
    rule.adam_m = reinterpret_cast<double*>(w + p->off_adam);
    rule.adam_v = rule.adam_m + p->rows * p->nc;
    rule.F_hist = F_hist;
    // fresh optimiser state
    cudaMemsetAsync(d_iter, 0, sizeof(int), st);
    cudaMemsetAsync(d_reached, 0xFF, sizeof(int) * p->n_prob, st);
    cudaMemsetAsync(rule.adam_m, 0, sizeof(double) * 2 * p->rows * p->nc, st);

    const bool stop_early = o.f_target <= 1.0;
    const int check_every = o.check_every < 1 ? 1 : o.check_every;
    std::vector<int> h_reached(p->n_prob);
    // every convergence check also reads the status word: a latched error ends the optimisation
    auto all_reached = [&](bool* all) -> int {
        cudaError_t e = cudaMemcpyAsync(h_reached.data(), d_reached, sizeof(int) * p->n_prob, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "convergence read");
        const int bits = *reinterpret_cast<volatile int*>(p->h_status);
        if (bits) {
            *reinterpret_cast<volatile int*>(p->h_status) = 0;
            p->st_recorded = false;
            cudaMemsetAsync(p->d_status, 0, sizeof(int), st);
            return status_error(bits);
        }
        *all = true;
        for (int v : h_reached)
            if (v < 0) *all = false;
        return QOC_OK;
    };

    if (o.use_graph) {
        GraphKey key{};
        key.u = u; key.psi0 = psi0; key.psif = psif; key.F_hist = F_hist; key.reached = d_reached; key.ws = ws;
        key.step = o.step; key.beta1 = o.beta1; key.beta2 = o.beta2; key.eps = o.eps; key.f_target = o.f_target;
        key.kind = rule.kind; key.freeze = rule.freeze; key.stream = st;
        if (!p->graph || std::memcmp(&key, &p->graph_key, sizeof(GraphKey)) != 0) {
            if (p->graph) {
                cudaGraphExecDestroy(p->graph);
                p->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "begin capture");
            p->capturing = true;
            rc = fidelity_grad_impl(p, u, psi0, psif, out3, nullptr, u, rule, w, st);
            p->capturing = false;
            e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&p->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                p->graph = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
            p->graph_key = key;
        }
    }
    int done = 0;
    for (int it = 0; it < o.iters; ++it) {
        if (o.use_graph) {
            cudaError_t e = cudaGraphLaunch(p->graph, st);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        } else {
            rc = fidelity_grad_impl(p, u, psi0, psif, out3, nullptr, u, rule, w, st);
            if (rc) return rc;
        }
        done = it + 1;
        if (stop_early && (done % check_every == 0)) {
            bool all = false;
            if ((rc = all_reached(&all))) return rc;
            if (all) break;
        }
    }
    if (iters_done) *iters_done = done;
    if (stop_early) {
        bool all = false;
        if ((rc = all_reached(&all))) return rc;
        if (!all) return set_error(QOC_ENOTCONVERGED, "F_target not reached by every problem");
    }
    record_status(p, st);
    return QOC_OK;
}

}  // extern "C"
