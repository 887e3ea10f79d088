// GPU plan: the active blocks of a basis for a fixed slice count and slice length, their
// Hamiltonians resident in device memory, the workspace layout, and the C ABI entry points that
// chain the kernels (assembly + expm -> sweeps -> overlap -> slice derivatives -> reduction).
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
    int R;
    int offset;   // into the class-list array
    int count;    // active blocks in the class
    int m_max;
    int grid;
    size_t slot_bytes;
};

struct qoc_plan {
    const qoc_basis* basis = nullptr;
    int device = 0;
    int N = 0;
    double dt = 0.0;
    qoc_plan_opts opts{};
    int nc = 0;
    int nb = 0;
    int max_m = 0;
    int max_c = 0;
    std::vector<DevBlock> hblocks;
    std::vector<int64_t> copy_src, copy_base;
    std::vector<long long> a_off;  // export layout offsets (complex), per active block
    int64_t export_elems = 0;      // N * sum m^2 over active blocks
    ExpmTables tabs{};
    std::vector<ExpmClass> classes;
    int grad_grid = 0;
    size_t grad_slot = 0;
    int seg = 0;                    // slices per checkpoint segment (== N without checkpointing)
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
    int* d_status = nullptr;
    unsigned long long* d_stats = nullptr;
    bool profiling = false;
    cudaEvent_t ev[6] = {};
    // workspace layout (bytes)
    size_t off_U = 0, off_psi = 0, off_lam = 0, off_partial = 0, off_o = 0, off_out3 = 0, off_expm = 0,
           off_grad = 0, off_ckpt = 0, off_lamb = 0;
    size_t el = 16;
    size_t ws_bytes = 0;

    DevPlan dev(char* ws, int k0 = 0, int nk = -1) const {
        DevPlan P{};
        P.N = N;
        P.k0 = k0;
        P.nk = nk < 0 ? N : nk;
        P.nc = nc;
        P.nb = nb;
        P.prec = opts.prec;
        P.dt = dt;
        P.max_sq = opts.max_squarings;
        P.grad_mode = opts.grad_mode;
        P.blocks = d_blocks;
        P.copy_src = d_copy_src;
        P.copy_base = d_copy_base;
        P.H = d_H;
        P.H64 = d_H64;
        P.status = d_status;
        P.stats = profiling ? d_stats : nullptr;
        (void)ws;
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

int run_expm(const qoc_plan* p, const double* u, char* ws, int k0, int nk, cudaStream_t st) {
    const DevPlan P = p->dev(ws, k0, nk);
    for (const auto& c : p->classes) {
        if (launch_expm(P, p->tabs, u, p->d_cls + c.offset, c.count, c.R, ws + p->off_U, ws + p->off_expm,
                        c.slot_bytes, c.m_max, c.grid, st) != 0)
            return cuda_fail(cudaGetLastError(), "expm launch");
    }
    return QOC_OK;
}

char* ckpt_vec(const qoc_plan* p, char* ws, int i) { return ws + p->off_ckpt + (size_t)i * p->vlen * p->el; }
char* lamb_vec(const qoc_plan* p, char* ws, int i) { return ws + p->off_lamb + (size_t)i * p->vlen * p->el; }

int run_sweeps(const qoc_plan* p, char* ws, int k0, int nk, int dirs, const char* fwd_in, char* fwd_out,
               const char* bwd_in, char* bwd_out, cudaStream_t st) {
    const DevPlan P = p->dev(ws, k0, nk);
    const int rc = launch_sweeps(P, ws + p->off_U, fwd_in, fwd_out, bwd_in, bwd_out, ws + p->off_psi,
                                 ws + p->off_lam, dirs, p->max_m, p->max_c, st);
    if (rc == -2) return set_error(QOC_EUNSUPPORTED, "block states do not fit in shared memory");
    if (rc != 0) return cuda_fail(cudaGetLastError(), "sweep launch");
    return QOC_OK;
}

int run_grad(const qoc_plan* p, const double* u, char* ws, int k0, int nk, cudaStream_t st) {
    const DevPlan P = p->dev(ws, k0, nk);
    const int g = launch_grad_partials(P, u, ws + p->off_psi, ws + p->off_lam,
                                       reinterpret_cast<double2*>(ws + p->off_partial), ws + p->off_grad,
                                       p->grad_slot, p->max_m, p->grad_grid, st);
    if (g == -2) return set_error(QOC_EUNSUPPORTED, "gradient kernel limits exceeded");
    if (g != 0) return cuda_fail(cudaGetLastError(), "gradient launch");
    return QOC_OK;
}

// Forward pass over all segments: psi_0 (gathered into checkpoint 0) -> checkpoint nseg = psi_N.
int forward_pass(const qoc_plan* p, const double* u, const double* psi0, char* w, cudaStream_t st) {
    int rc;
    if (launch_gather(p->dev(w), reinterpret_cast<const double2*>(psi0), ckpt_vec(p, w, 0), st) != 0)
        return cuda_fail(cudaGetLastError(), "gather launch");
    for (int s = 0; s < p->nseg; ++s) {
        const int k0 = s * p->seg, nk = std::min(p->seg, p->N - k0);
        if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
        if ((rc = run_sweeps(p, w, k0, nk, 1, ckpt_vec(p, w, s), ckpt_vec(p, w, s + 1), nullptr, nullptr, st)))
            return rc;
    }
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
}

int qoc_plan_create(const qoc_basis* B, int N, double dt, const qoc_plan_opts* opts, const uint8_t* active,
                    qoc_plan** out) {
    if (!B || !out) return set_error(QOC_EINVAL, "null argument");
    *out = nullptr;
    if (N < 1) return set_error(QOC_EINVAL, "N must be >= 1");
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(QOC_EINVAL, "dt must be positive and finite");
    qoc_plan_opts o;
    if (opts) o = *opts; else qoc_plan_opts_default(&o);
    if (o.prec != QOC_PREC_F64 && o.prec != QOC_PREC_F32) return set_error(QOC_EINVAL, "unknown precision");
    if (o.grad_mode != 0 && o.grad_mode != 1) return set_error(QOC_EINVAL, "unknown grad_mode");
    if (o.max_squarings <= 0) o.max_squarings = 16;
    if (o.max_squarings > 40) return set_error(QOC_EINVAL, "max_squarings must be <= 40");
    if (B->n_ctrl > 8) return set_error(QOC_EUNSUPPORTED, "at most 8 controls");

    auto* p = new (std::nothrow) qoc_plan();
    if (!p) return set_error(QOC_ENOMEM, "host allocation failed");
    p->basis = B;
    p->N = N;
    p->dt = dt;
    p->opts = o;
    p->nc = B->n_ctrl;
    cudaGetDevice(&p->device);
    const size_t el = o.prec == QOC_PREC_F64 ? 16 : 8;
    p->el = el;
    if (o.ckpt_segment < -1) {
        delete p;
        return set_error(QOC_EINVAL, "ckpt_segment must be -1, 0 or positive");
    }
    p->seg = o.ckpt_segment == 0 ? N
             : o.ckpt_segment < 0 ? std::max(1, (int)std::ceil(std::sqrt((double)N)))
                                  : std::min(o.ckpt_segment, N);
    p->nseg = (N + p->seg - 1) / p->seg;

    // active blocks, ordered by size (largest first) for load balance
    struct Act { int b; std::vector<int> copies; };
    std::vector<Act> acts;
    int64_t copy_counter = 0;
    for (int b = 0; b < (int)B->blocks.size(); ++b) {
        const auto& blk = B->blocks[b];
        Act a{b, {}};
        for (int r = 0; r < blk.c; ++r, ++copy_counter)
            if (!active || active[copy_counter]) a.copies.push_back(r);
        if (!a.copies.empty()) acts.push_back(std::move(a));
    }
    if (acts.empty()) {
        delete p;
        return set_error(QOC_EINVAL, "no active block copy");
    }
    std::stable_sort(acts.begin(), acts.end(),
                     [&](const Act& x, const Act& y) { return B->blocks[x.b].m > B->blocks[y.b].m; });
    p->nb = (int)acts.size();

    int64_t h_off = 0, u_off = 0, s_off = 0, v_off = 0;
    std::vector<cplx> H64;
    for (const auto& a : acts) {
        const auto& blk = B->blocks[a.b];
        DevBlock d{};
        d.m = blk.m;
        d.c = (int)a.copies.size();
        d.b = a.b;
        d.mmp = ((int64_t)blk.m * blk.m + 3) / 4 * 4;
        d.h_off = h_off;
        d.u_off = u_off;
        d.s_off = s_off;
        d.v_off = v_off;
        d.h0_norm1 = blk.h0_norm1;
        for (int j = 0; j < p->nc; ++j) d.hc_norm1[j] = blk.hc_norm1[j];
        p->copy_base.push_back((int64_t)p->copy_src.size());
        for (int r : a.copies) p->copy_src.push_back(blk.offset + (int64_t)r * blk.m);
        H64.insert(H64.end(), blk.h0.begin(), blk.h0.end());
        H64.insert(H64.end(), blk.hc.begin(), blk.hc.end());
        h_off += (int64_t)(1 + p->nc) * blk.m * blk.m;
        u_off += (int64_t)p->seg * d.mmp;
        s_off += (int64_t)(p->seg + 1) * d.c * d.m;
        v_off += (int64_t)d.c * d.m;
        p->max_m = std::max(p->max_m, d.m);
        p->max_c = std::max(p->max_c, d.c);
        p->hblocks.push_back(d);
    }
    // export layout (assemble / expm outputs): active blocks in basis order
    {
        std::vector<int> order(p->nb);
        for (int i = 0; i < p->nb; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return p->hblocks[x].b < p->hblocks[y].b; });
        p->a_off.assign(p->nb, 0);
        long long acc = 0;
        for (int i : order) {
            p->a_off[i] = acc;
            acc += (long long)N * p->hblocks[i].m * p->hblocks[i].m;
        }
        p->export_elems = acc;
    }

    // Taylor degree table
    const int degs[9] = {2, 4, 6, 9, 12, 16, 20, 25, 30};
    const double unit = o.prec == QOC_PREC_F64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    for (int i = 0; i < 9; ++i) p->tabs.theta[i] = theta_for(degs[i], unit);
    if (o.prec == QOC_PREC_F64) {
        p->tabs.n_deg = 9;
        p->tabs.theta_cap = p->tabs.theta[8];
    } else {
        p->tabs.n_deg = 7;
        p->tabs.theta_cap = std::min(p->tabs.theta[6], 3.0);
    }

    // expm size classes
    std::vector<int> cls_list;
    size_t expm_scratch = 0;
    for (int R = 1; R <= 7; ++R) {
        ExpmClass c{R, (int)cls_list.size(), 0, 0, 0, 0};
        for (int i = 0; i < p->nb; ++i)
            if (expm_r_for(o.prec, p->hblocks[i].m) == R) {
                cls_list.push_back(i);
                c.count++;
                c.m_max = std::max(c.m_max, p->hblocks[i].m);
            }
        if (c.count == 0) continue;
        const long long items = (long long)c.count * p->seg;
        c.grid = (int)std::min<long long>(items, expm_grid_limit(o.prec, R));
        c.slot_bytes = align_up(expm_slot_bytes(o.prec, c.m_max), 256);
        expm_scratch = std::max(expm_scratch, c.slot_bytes * (size_t)c.grid);
        p->classes.push_back(c);
    }
    // gradient kernel
    p->grad_slot = align_up(grad_slot_bytes(o.prec, p->max_m), 256);
    p->grad_grid = (int)std::min<long long>((long long)p->seg * p->nb, grad_grid_limit(o.prec, p->max_m));
    p->vlen = v_off;
    if (grad_vector_smem(o.prec, p->max_m) > 220 * 1024) {
        delete p;
        return set_error(QOC_EUNSUPPORTED, "block too large for the gradient kernel's shared-memory series");
    }

    // workspace layout
    size_t off = 0;
    p->off_U = off;       off = align_up(off + (size_t)u_off * el, 256);
    p->off_psi = off;     off = align_up(off + (size_t)s_off * el, 256);
    p->off_lam = off;     off = align_up(off + (size_t)s_off * el, 256);
    p->off_partial = off; off = align_up(off + (size_t)N * p->nb * p->nc * 16, 256);
    p->off_o = off;       off = align_up(off + 16, 256);
    p->off_out3 = off;    off = align_up(off + 32, 256);
    p->off_expm = off;    off = align_up(off + expm_scratch, 256);
    p->off_grad = off;    off = align_up(off + p->grad_slot * (size_t)p->grad_grid, 256);
    p->off_ckpt = off;    off = align_up(off + (size_t)(p->nseg + 1) * p->vlen * el, 256);
    p->off_lamb = off;    off = align_up(off + (size_t)2 * p->vlen * el, 256);
    p->ws_bytes = off;

    // device uploads
    auto fail = [&](cudaError_t e, const char* what) {
        int rc = cuda_fail(e, what);
        qoc_plan_free(p);
        return rc;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_blocks, sizeof(DevBlock) * p->nb)) != cudaSuccess) return fail(e, "cudaMalloc blocks");
    if ((e = cudaMalloc(&p->d_copy_src, sizeof(int64_t) * p->copy_src.size())) != cudaSuccess) return fail(e, "cudaMalloc copies");
    if ((e = cudaMalloc(&p->d_copy_base, sizeof(int64_t) * p->nb)) != cudaSuccess) return fail(e, "cudaMalloc copies");
    if ((e = cudaMalloc(&p->d_a_off, sizeof(long long) * p->nb)) != cudaSuccess) return fail(e, "cudaMalloc offsets");
    if ((e = cudaMalloc(&p->d_H64, sizeof(cplx) * H64.size())) != cudaSuccess) return fail(e, "cudaMalloc H");
    if ((e = cudaMalloc(&p->d_cls, sizeof(int) * std::max<size_t>(1, cls_list.size()))) != cudaSuccess) return fail(e, "cudaMalloc classes");
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc status");
    if ((e = cudaMalloc(&p->d_stats, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e, "cudaMalloc stats");
    cudaMemset(p->d_stats, 0, 4 * sizeof(unsigned long long));
    for (auto& ev : p->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e, "cudaEventCreate");
    cudaMemcpy(p->d_blocks, p->hblocks.data(), sizeof(DevBlock) * p->nb, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_copy_src, p->copy_src.data(), sizeof(int64_t) * p->copy_src.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_copy_base, p->copy_base.data(), sizeof(int64_t) * p->nb, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_a_off, p->a_off.data(), sizeof(long long) * p->nb, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_H64, H64.data(), sizeof(cplx) * H64.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_cls, cls_list.data(), sizeof(int) * cls_list.size(), cudaMemcpyHostToDevice);
    cudaMemset(p->d_status, 0, sizeof(int));
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
    *out = p;
    return QOC_OK;
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
    cudaFree(p->d_status);
    cudaFree(p->d_stats);
    for (auto& ev : p->ev)
        if (ev) cudaEventDestroy(ev);
    delete p;
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
    if (st & ST_TIMEOUT) return set_error(QOC_ETIMEOUT, "a bounded device wait gave up");
    if (st & ST_NAN_PULSE) return set_error(QOC_EINVAL, "non-finite pulse value");
    if (st & ST_SQUARING_CAP) return set_error(QOC_EUNSUPPORTED, "a slice needed more squarings than max_squarings");
    if (st & ST_SERIES_CAP) return set_error(QOC_EUNSUPPORTED, "a slice's norm is beyond the gradient series' range");
    return QOC_OK;
}

int qoc_plan_set_profiling(qoc_plan* p, int on) {
    if (!p) return set_error(QOC_EINVAL, "null plan");
    cudaSetDevice(p->device);
    p->profiling = on != 0;
    if (on) cudaMemset(p->d_stats, 0, 4 * sizeof(unsigned long long));
    return QOC_OK;
}

int qoc_plan_phase_times(qoc_plan* p, float* ms, int n) {
    if (!p || !ms) return set_error(QOC_EINVAL, "null argument");
    if (!p->profiling) return set_error(QOC_EINVAL, "profiling is off");
    cudaSetDevice(p->device);
    cudaError_t e = cudaEventSynchronize(p->ev[5]);
    if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
    for (int i = 0; i < n && i < 5; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event elapsed");
        ms[i] = t;
    }
    return QOC_OK;
}

int qoc_plan_work_counts(qoc_plan* p, long long* out, int n) {
    if (!p || !out) return set_error(QOC_EINVAL, "null argument");
    cudaSetDevice(p->device);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(h, p->d_stats, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats read");
    for (int i = 0; i < n && i < 3; ++i) out[i] = (long long)h[i];
    return QOC_OK;
}

int qoc_plan_kernel_launches(const qoc_plan* p, int with_grad, int* launches) {
    if (!p || !launches) return set_error(QOC_EINVAL, "null argument");
    // expm: one launch per size class; then sweeps, overlap, slice derivatives, reduction
    // (propagate: sweeps and the final-state store after a memset)
    const int ncls = (int)p->classes.size();
    if (p->nseg == 1)
        *launches = with_grad ? 2 + ncls + 1 + 1 + 1 + 1 : 1 + ncls + 1 + 1;  // gathers, expm, sweeps, overlap, grad, reduce
    else
        *launches = with_grad ? 1 + p->nseg * (ncls + 1) + 1 + 1 + p->nseg * (ncls + 2) + 1
                              : 1 + p->nseg * (ncls + 1) + 1;
    return QOC_OK;
}

int qoc_assemble_blocks(const qoc_plan* p, const double* u, double* A_out, void* stream) {
    if (!p || !u || !A_out) return set_error(QOC_EINVAL, "null argument");
    cudaSetDevice(p->device);
    const DevPlan P = p->dev(nullptr);
    if (launch_assemble(P, u, reinterpret_cast<double2*>(A_out), p->d_a_off, to_stream(stream)) != 0)
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
    for (int s = 0; s < p->nseg; ++s) {
        const int k0 = s * p->seg, nk = std::min(p->seg, p->N - k0);
        if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
        if (launch_export_u(p->dev(w, k0, nk), w + p->off_U, reinterpret_cast<double2*>(U_out), p->d_a_off, st) != 0)
            return cuda_fail(cudaGetLastError(), "export launch");
    }
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
    if ((rc = forward_pass(p, u, psi0, w, st))) return rc;
    if (launch_store_final(p->dev(w), ckpt_vec(p, w, p->nseg), reinterpret_cast<double2*>(psiN), p->basis->state_len,
                           st) != 0)
        return cuda_fail(cudaGetLastError(), "store launch");
    return QOC_OK;
}

// Phase events: [0]..[1] propagators (+ forward sweeps when checkpointing), [1]..[2] sweeps (costate
// pass when checkpointing: recomputed propagators, both sweeps and slice derivatives), [2]..[3]
// overlap, [3]..[4] slice derivatives (0 when checkpointing), [4]..[5] reduction / update.
static int fidelity_grad_impl(const qoc_plan* p, const double* u, const double* psi0, const double* psif,
                              double* out3, double* grad, double* u_update, double step, double* F_slot, char* w,
                              cudaStream_t st) {
    int rc;
    const DevPlan P = p->dev(w);
    auto mark = [&](int i) {
        if (p->profiling) cudaEventRecord(p->ev[i], st);
    };
    const bool want_grad = grad || u_update;
    double2* o_ws = reinterpret_cast<double2*>(w + p->off_o);
    mark(0);
    if (p->nseg == 1) {
        if (launch_gather(P, reinterpret_cast<const double2*>(psi0), ckpt_vec(p, w, 0), st) != 0 ||
            (want_grad && launch_gather(P, reinterpret_cast<const double2*>(psif), lamb_vec(p, w, 0), st) != 0))
            return cuda_fail(cudaGetLastError(), "gather launch");
        if ((rc = run_expm(p, u, w, 0, p->N, st))) return rc;
        mark(1);
        if ((rc = run_sweeps(p, w, 0, p->N, want_grad ? 3 : 1, ckpt_vec(p, w, 0), ckpt_vec(p, w, 1),
                             lamb_vec(p, w, 0), lamb_vec(p, w, 1), st)))
            return rc;
        mark(2);
        if (launch_overlap(P, ckpt_vec(p, w, 1), reinterpret_cast<const double2*>(psif), out3, o_ws, st) != 0)
            return cuda_fail(cudaGetLastError(), "overlap launch");
        mark(3);
        if (want_grad && (rc = run_grad(p, u, w, 0, p->N, st))) return rc;
    } else {
        if ((rc = forward_pass(p, u, psi0, w, st))) return rc;
        mark(1);
        if (launch_overlap(P, ckpt_vec(p, w, p->nseg), reinterpret_cast<const double2*>(psif), out3, o_ws, st) != 0)
            return cuda_fail(cudaGetLastError(), "overlap launch");
        mark(2);
        if (want_grad) {
            if (launch_gather(P, reinterpret_cast<const double2*>(psif), lamb_vec(p, w, 0), st) != 0)
                return cuda_fail(cudaGetLastError(), "gather launch");
            // costate pass: recompute each segment's propagators and states, newest segment first
            int cur = 0;
            for (int s = p->nseg - 1; s >= 0; --s) {
                const int k0 = s * p->seg, nk = std::min(p->seg, p->N - k0);
                if ((rc = run_expm(p, u, w, k0, nk, st))) return rc;
                if ((rc = run_sweeps(p, w, k0, nk, 3, ckpt_vec(p, w, s), ckpt_vec(p, w, s + 1), lamb_vec(p, w, cur),
                                     lamb_vec(p, w, cur ^ 1), st)))
                    return rc;
                if ((rc = run_grad(p, u, w, k0, nk, st))) return rc;
                cur ^= 1;
            }
        }
        mark(3);
    }
    mark(4);
    if (want_grad) {
        if (launch_grad_reduce(P, reinterpret_cast<const double2*>(w + p->off_partial), o_ws, grad, u_update, step,
                               F_slot, out3, st) != 0)
            return cuda_fail(cudaGetLastError(), "reduce launch");
    }
    mark(5);
    return QOC_OK;
}

int qoc_fidelity_and_grad(const qoc_plan* p, const double* u, const double* psi0, const double* psif, double* out3,
                          double* grad, void* ws, size_t ws_bytes, void* stream) {
    if (!p || !u || !psi0 || !psif || !out3) return set_error(QOC_EINVAL, "null argument");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    return fidelity_grad_impl(p, u, psi0, psif, out3, grad, nullptr, 0.0, nullptr, static_cast<char*>(ws),
                              to_stream(stream));
}

int qoc_optimize_pulses(const qoc_plan* p, double* u, const double* psi0, const double* psif, int iters, double step,
                        double f_target, int check_every, double* F_hist, int* iters_done, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!p || !u || !psi0 || !psif || !F_hist) return set_error(QOC_EINVAL, "null argument");
    if (iters < 0) return set_error(QOC_EINVAL, "iters must be >= 0");
    if (!std::isfinite(step)) return set_error(QOC_EINVAL, "step must be finite");
    int rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaSetDevice(p->device);
    char* w = static_cast<char*>(ws);
    cudaStream_t st = to_stream(stream);
    double* out3 = reinterpret_cast<double*>(w + p->off_out3);
    const bool stop_early = f_target <= 1.0;
    if (check_every < 1) check_every = 1;
    int done = 0;
    for (int it = 0; it < iters; ++it) {
        double* trip = F_hist + it;  // F at the current pulses, copied here by the reduction kernel
        rc = fidelity_grad_impl(p, u, psi0, psif, out3, nullptr, u, step, trip, w, st);
        if (rc) return rc;
        done = it + 1;
        if (stop_early && (done % check_every == 0)) {
            double F = 0.0;
            cudaError_t e = cudaMemcpyAsync(&F, trip, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "fidelity read");
            if (F >= f_target) break;
        }
    }
    if (iters_done) *iters_done = done;
    if (stop_early && done > 0) {
        double F = 0.0;
        cudaMemcpyAsync(&F, F_hist + done - 1, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (!(F >= f_target)) return set_error(QOC_ENOTCONVERGED, "F_target not reached");
    }
    return QOC_OK;
}

}  // extern "C"
