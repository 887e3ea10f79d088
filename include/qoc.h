/*
 * qoc.h — C ABI of the symmetry-block GRAPE library (libqoc.so).
 *
 * Method: Wang, Okyay, Kumar, Wong, "Accelerating Quantum Optimal Control of Multi-Qubit
 * Systems with Symmetry-Based Hamiltonian Transformations" (arXiv 2309.05884).
 *   - n qubits, H(t) = H0 + sum_j u_j(t) Hc_j                         (Sec. II.A, Eq. schrodingerEq)
 *   - piecewise-constant slices, tau = T/N,
 *     psi_k = exp(-i tau (H0 + sum_j u_kj Hc_j)) psi_{k-1}            (Sec. II.A, Eq. exppropagator)
 *   - objective F = |<psi_f|psi_N>|^2                                 (Sec. II.A, Eq. probability)
 *   - the S_n / D_n symmetry makes A^dagger H A block diagonal; every block evolves on its own
 *                                                                     (Sec. II.A, Fig. 2; Appendix A)
 *   - gradient of F through the slice derivative of exp and the costates lambda_{k-1} = U_k^dagger
 *     lambda_k                                                        (Appendix B, Eq. propagator_differentiation)
 *
 * Conventions
 *   - Qubit 1 is the most significant bit of a computational-basis index; |0> = |up>, sigma_z = +1.
 *   - Complex numbers are interleaved (re, im) doubles.  A "block state" is the concatenation over
 *     blocks b = 0..n_blocks-1 of c_b copies of an m_b-vector (copy-major: [copy][index]); block b
 *     starts at complex offset offset_b (see qoc_basis_block).
 *   - Pulses u are [N][n_ctrl] doubles, row-major; the gradient has the same layout.
 *   - "dev" = device pointer (CUDA global memory), "host" = host pointer.  The caller owns every
 *     buffer it passes; the library owns qoc_basis / qoc_plan objects and the device copies of the
 *     block Hamiltonians they hold.
 *   - Stream arguments are cudaStream_t passed as void* (NULL = legacy default stream).  Calls that
 *     take a stream are asynchronous on it; argument errors are returned synchronously before any
 *     launch.  Kernel-side errors (a NaN pulse, an initial or target state whose norm is not 1, an
 *     exhausted iteration cap, a bounded wait that gave up) are latched in a device status word of
 *     the plan.  Every call on the plan ends by queueing a copy of that word to pinned host memory;
 *     the next call that starts after that copy has completed on the GPU returns the latched error
 *     (and clears it) before it launches anything.  qoc_plan_sync_status() waits and returns it at
 *     once.  No call waits for the GPU to find out (inside a stream capture neither step runs).
 *
 * Every function returns QOC_OK (0) or a negative error code; qoc_last_error() gives a message for
 * the calling thread's last failure.
 */
#ifndef QOC_H
#define QOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- error codes */
enum {
    QOC_OK = 0,
    QOC_EINVAL = -1,          /* bad argument, shape, NaN/Inf input, unnormalised state (|norm - 1| > 1e-8) */
    QOC_ENOMEM = -2,          /* host or device allocation failed, or workspace too small */
    QOC_ECUDA = -3,           /* a CUDA runtime call failed */
    QOC_ETIMEOUT = -4,        /* a bounded device wait gave up */
    QOC_EUNSUPPORTED = -5,    /* a size or option beyond what the library builds */
    QOC_ENOTCONVERGED = -6    /* optimisation stopped before reaching its target */
};

/* ---------------------------------------------------------------- Hamiltonian terms */
/* Operator kinds (coefficient 1); sigma_a^(i) acts on qubit i (Sec. II.A):
 *   QOC_SUM_a       : sum_i sigma_a^(i)                     (H_x, H_y, H_z of Sec. II.A)
 *   QOC_ALLPAIRS_aa : sum_{i<j} sigma_a^(i) sigma_a^(j)     (S_n-invariant pair coupling)
 *   QOC_RING_aa     : sum_{i=1..n} sigma_a^(i) sigma_a^(i+dist), indices mod n
 *                     (H_{z,cpl} of Sec. II.A for dist = 1; Eq. H0MoreCoupling1 for dist > 1) */
enum qoc_term_kind {
    QOC_SUM_X = 0, QOC_SUM_Y = 1, QOC_SUM_Z = 2,
    QOC_ALLPAIRS_XX = 3, QOC_ALLPAIRS_YY = 4, QOC_ALLPAIRS_ZZ = 5,
    QOC_RING_XX = 6, QOC_RING_YY = 7, QOC_RING_ZZ = 8
};

enum { QOC_GROUP_SN = 0, QOC_GROUP_DN = 1 };

typedef struct qoc_term {
    int kind;      /* enum qoc_term_kind */
    int dist;      /* ring distance (RING_* only), 1 <= dist <= n/2 */
    double coeff;  /* real coefficient */
} qoc_term;

typedef struct qoc_system_desc {
    int n;                       /* qubits: S_n 1..64, D_n 3..16 */
    int group;                   /* QOC_GROUP_SN or QOC_GROUP_DN; every term must be invariant */
    int n_h0_terms;
    const qoc_term* h0;          /* host, n_h0_terms entries */
    int n_ctrl;                  /* number of control fields, 1..8 */
    const int* n_hc_terms;       /* host, n_ctrl entries */
    const qoc_term* const* hc;   /* host, hc[j] has n_hc_terms[j] entries */
} qoc_system_desc;

/* ---------------------------------------------------------------- symmetry basis (host, once) */
typedef struct qoc_basis qoc_basis;

/* Flags for qoc_build_symmetry_basis. */
enum {
    QOC_BASIS_FIRST_BLOCK_ONLY = 1,  /* keep only the block of |0...0> (Sec. II.B: H_1 suffices
                                        when the initial and target states lie in it) */
    QOC_BASIS_NO_VECTORS = 2         /* do not keep full-space basis vectors (no state conversion) */
};

/* Build the symmetry-adapted block decomposition of H0 and every Hc_j (Appendix A).
 * S_n: blocks are the spin sectors J = n/2, n/2-1, ... of size 2J+1 with C(n,n/2-J)-C(n,n/2-J-1)
 *      identical copies (the |J,M> route of Appendix A); for n > 12 only J = n/2 is built.
 * D_n: blocks are the irreps A1, A2, (B1, B2), E1, ... of the dihedral group acting on qubit
 *      indices (Eq. groupAlgebraElementsDn); 2-dimensional irreps have 2 identical copies.
 * Checks every term's invariance under the group and returns QOC_EINVAL if one is not.
 * out: receives a basis owned by the library (free with qoc_basis_free).
 * Errors: QOC_EINVAL (bad desc), QOC_EUNSUPPORTED (n out of range), QOC_ENOMEM. */
int qoc_build_symmetry_basis(const qoc_system_desc* sys, int flags, qoc_basis** out);
void qoc_basis_free(qoc_basis* basis);

/* n_blocks, n_ctrl, total block-state length (complex elements), full-space dimension (0 if n>62). */
int qoc_basis_info(const qoc_basis* basis, int* n_blocks, int* n_ctrl, int64_t* state_len,
                   int64_t* full_dim);

/* Block b: size m_b, copies c_b, complex offset in the block state, label ("A1", "E2", "J=3/2"...;
 * label must hold 16 bytes, may be NULL). */
int qoc_basis_block(const qoc_basis* basis, int b, int* size, int* copies, int64_t* offset,
                    char* label);

/* Host copies of block b's H0_b (m*m complex) and Hc_jb (n_ctrl*m*m complex), row-major.  Either
 * pointer may be NULL. */
int qoc_basis_block_matrices(const qoc_basis* basis, int b, double* h0, double* hc);

/* Upper bounds of the spectral norms of block b's H0_b (out[0]) and Hc_jb (out[1 + j]), host,
 * 1 + n_ctrl doubles.  The slice norm bound tau (|H0_b| + sum_j |u_kj| |Hc_jb|) built from them fixes
 * the Taylor degree, the squarings and the derivative-series lengths (Sec. II.A; the paper states
 * the truncated series, not the norm).  Each is the Collatz-Wielandt value max_i (|M| x)_i / x_i of
 * the entrywise moduli along power iterations from x = 1: never below ||M||_2, never above the 1-norm. */
int qoc_basis_norm_bounds(const qoc_basis* basis, int b, double* out);

/* full (host, 2^n complex) -> blk (host, state_len complex): coordinates <v_{b,r,a}|psi>.
 * Needs the basis vectors (D_n n <= 16, S_n n <= 12, built without QOC_BASIS_NO_VECTORS). */
int qoc_state_to_blocks(const qoc_basis* basis, const double* full, double* blk);
/* blk (host) -> full (host): the inverse map. */
int qoc_blocks_to_state(const qoc_basis* basis, const double* blk, double* full);

/* The Dicke state |D(n,k)> (k ones, symmetric) in block coordinates (host, state_len complex).
 * S_n only; it is the basis vector |J=n/2, M=n/2-k> of block 0. */
int qoc_dicke_state(const qoc_basis* basis, int k, double* blk);

/* ---------------------------------------------------------------- GPU plan */
typedef struct qoc_plan qoc_plan;

enum {
    QOC_PREC_F64 = 0,     /* all steps in FP64 */
    QOC_PREC_F32 = 1,     /* complex FP32 Taylor polynomial and sweeps; FP64 squaring chain,
                             overlap, fidelity and gradient accumulation */
    QOC_PREC_F32_ALL = 2  /* as QOC_PREC_F32 but the squaring chain in FP32 too (small blocks with
                             few squarings; FP64 overlap and accumulation) */
};

/* Options of a plan; zero-initialise and set what you need (qoc_plan_opts_default fills it). */
typedef struct qoc_plan_opts {
    int prec;             /* QOC_PREC_F64 or QOC_PREC_F32 */
    int grad_mode;        /* 0 = exact slice derivative (Frechet derivative of exp);
                             1 = the paper's first-order form -i tau Hc_j U_k (Eq. propagator_differentiation) */
    int max_squarings;    /* cap on the scaling-and-squaring count s (default 16) */
    int ckpt_segment;     /* 0 = keep every propagator of a call in the workspace (default);
                             S > 0 = checkpointing: keep the state at every S-th slice and only S
                             slices of propagators; the costate pass recomputes each segment's
                             propagators and states (twice the exponentials, workspace ~ N/S + S
                             states and S propagators per block); -1 = S = ceil(sqrt(N)) */
    int objective;        /* QOC_OBJ_STATE (default) or QOC_OBJ_GATE, see below */
    int reserved[3];
} qoc_plan_opts;

/* Objectives.
 *   QOC_OBJ_STATE: state transfer, F = |<psi_f|psi_N>|^2 (Sec. II.A, Eq. probability); block states
 *     as described under Conventions, the copies selected by the active mask.
 *   QOC_OBJ_GATE: gate (unitary) fidelity, the trace fidelity of Sec. IV with a target gate W:
 *     F = |Tr(W^dagger U_N ... U_1) / d|^2, d = 2^n.  For a symmetric W (one that commutes with the
 *     group, as the gates of Sec. III do) both are block diagonal and every copy of block b carries
 *     the same W_b, so Tr(W^dagger U) = sum_b c_b Tr(W_b^dagger U_b).  The plan propagates every column
 *     of every block: block states have the layout [block b][column r][m_b] (length sum_b m_b^2), the
 *     caller passes psi0 = sqrt(c_b / d) times the identity columns and psif = sqrt(c_b / d) times the
 *     columns of W_b, so that sum_b sum_r <psif_br|psi_N,br> = Tr(W^dagger U) / d and out3, the
 *     gradient and the optimiser work unchanged.  No active mask (every column takes part). */
enum { QOC_OBJ_STATE = 0, QOC_OBJ_GATE = 1 };

void qoc_plan_opts_default(qoc_plan_opts* opts);

/* A plan fixes the basis, the number of slices N, the slice length dt = tau, the options and the
 * copies that take part.  active (host, one byte per block copy in block-state order, may be NULL
 * for "all"): copies whose initial or target component is zero cannot contribute to the overlap
 * and may be left out (Sec. II.B, "only the first block").  Uploads the block Hamiltonians once.
 * Errors: QOC_EINVAL, QOC_EUNSUPPORTED (a block larger than the kernels support), QOC_ECUDA. */
int qoc_plan_create(const qoc_basis* basis, int N, double dt, const qoc_plan_opts* opts,
                    const uint8_t* active, qoc_plan** out);

/* A plan over many independent problems that run together in every launch (batched GRAPE):
 * problem i has basis bases[i], Ns[i] slices of length dts[i] and active copies actives[i] (host,
 * may be NULL, as may the array itself).  Every basis must have the same number of controls.
 * Device buffers of a batch plan concatenate the problems in order: pulses and gradients
 * [sum_i Ns[i]][n_ctrl], block states [sum_i state_len_i], out3 [n_problems][3].  Checkpointing
 * (ckpt_segment != 0) needs a single problem. */
int qoc_plan_create_batch(const qoc_basis* const* bases, int n_problems, const int* Ns, const double* dts,
                          const qoc_plan_opts* opts, const uint8_t* const* actives, qoc_plan** out);

/* Problems, total pulse rows (sum of N) and concatenated block-state length of a plan. */
int qoc_plan_info(const qoc_plan* plan, int* n_problems, int64_t* pulse_rows, int64_t* state_len);
void qoc_plan_free(qoc_plan* plan);

/* Bytes of device workspace the plan's calls need (propagators, states and costates, partial
 * sums).  The caller allocates it (any allocator) and passes it to every call; calls on one plan
 * and one workspace must not overlap in time. */
int qoc_plan_workspace_bytes(const qoc_plan* plan, size_t* bytes);

/* Return and clear the plan's device status word (synchronises the given stream). */
int qoc_plan_sync_status(qoc_plan* plan, void* stream);

/* Failure-path self-test of the bounded waits (no counterpart in the paper): launches one kernel
 * that waits on a shared-memory mbarrier that nothing completes, with the same bounded-wait routine
 * the propagator and sweep kernels use on their bulk copies and tensor-core commits.  The wait gives
 * up after limit_ms (0.001..1000) and latches the timeout bit, so that qoc_plan_sync_status (or the
 * next call on the plan, once this one has finished) returns QOC_ETIMEOUT; the context stays usable.
 * Asynchronous on stream. */
int qoc_plan_selftest_wait(qoc_plan* plan, double limit_ms, void* stream);

/* Block assembly (Eq. exppropagator's exponent): A_out[b][k] = -i dt (H0_b + sum_j u_kj Hc_jb) for
 * every active block b and slice k, as m_b*m_b complex128 row-major matrices packed block-major
 * (block b at complex offset N * sum_{b'<b} m_b'^2).
 * u: dev [N][n_ctrl] doubles.  A_out: dev.  Errors: QOC_EINVAL. */
int qoc_assemble_blocks(const qoc_plan* plan, const double* u, double* A_out, void* stream);

/* Batched propagators U[b][k] = exp(A[b][k]) by scaling and squaring with a Taylor polynomial
 * (Sec. II.A, Eq. exppropagator), written as complex128 in the layout of qoc_assemble_blocks. */
int qoc_expm_blocks(const qoc_plan* plan, const double* u, double* U_out, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Forward propagation of every active block copy: psiN = U_N ... U_1 psi0 (Eq. exppropagator).
 * psi0, psiN: dev block states (state_len complex128); inactive copies of psiN are set to 0. */
int qoc_propagate(const qoc_plan* plan, const double* u, const double* psi0, double* psiN,
                  void* workspace, size_t workspace_bytes, void* stream);

/* Fidelity and gradient (Eq. probability; Appendix B):
 *   out3 (dev, 3 doubles per problem) = { F, Re o, Im o },  o = sum over the problem's active copies
 *   <psif|psi_N>,  F = |o|^2
 *   grad (dev [N][n_ctrl], may be NULL) = dF/du_kj = 2 Re(conj(o) sum lam_k^dagger dU_k/du_kj psi_{k-1})
 * psi0, psif: dev block states (state_len complex128), each of norm 1 per problem (checked on the
 * device to 1e-8: QOC_EINVAL, latched).  The forward states and the costates run concurrently. */
int qoc_fidelity_and_grad(const qoc_plan* plan, const double* u, const double* psi0,
                          const double* psif, double* out3, double* grad, void* workspace,
                          size_t workspace_bytes, void* stream);

/* The same computation in two halves, for reverse-mode differentiation (a framework's backward runs
 * only when a gradient is asked for):
 *   qoc_fidelity_forward: propagators, forward states psi_k = U_k psi_{k-1} (Eq. exppropagator) and
 *     out3 as above.  The workspace keeps the states of every slice (with checkpointing: of every
 *     segment boundary), the propagators (without checkpointing) and the overlaps o_p.
 *   qoc_fidelity_backward: costates lam_N = psif, lam_{k-1} = U_k^dagger lam_k (Appendix B), the exact
 *     slice derivatives (with checkpointing each segment's propagators and states are recomputed, as
 *     in qoc_fidelity_and_grad) and grad[k][j] = gF_p * dF_p/du_kj for the rows of problem p;
 *     gF: dev [n_problems] doubles (a caller's dL/dF_p), NULL for 1.
 * qoc_fidelity_backward needs the workspace exactly as the last qoc_fidelity_forward on the same
 * plan left it (same u, psif; no other call on that workspace in between); the library cannot check
 * this. */
int qoc_fidelity_forward(const qoc_plan* plan, const double* u, const double* psi0, const double* psif,
                         double* out3, void* workspace, size_t workspace_bytes, void* stream);
int qoc_fidelity_backward(const qoc_plan* plan, const double* u, const double* psif, const double* gF,
                          double* grad, void* workspace, size_t workspace_bytes, void* stream);

/* Gradient ascent (GRAPE, Sec. II.A) on every problem of the plan. */
enum { QOC_RULE_FIXED = 0,   /* u <- u + step * dF/du */
       QOC_RULE_ADAM = 1 };  /* Adam ascent: moments of dF/du with beta1, beta2, eps; u <- u + step * m^/(sqrt(v^)+eps) */

typedef struct qoc_opt_opts {
    int iters;             /* iterations at most */
    int rule;              /* QOC_RULE_FIXED or QOC_RULE_ADAM */
    double step, beta1, beta2, eps;
    double f_target;       /* <= 1: stop once every problem reached F >= f_target (checked on the host
                              every check_every iterations); > 1: run all iterations */
    int check_every;
    int use_graph;         /* 1: capture one iteration into a CUDA graph once and replay it (needs a
                              non-default stream; the graph is kept while the arguments stay the same) */
    int freeze_converged;  /* 1 (default): a problem that reached f_target keeps its pulses */
    int reserved[3];
} qoc_opt_opts;

void qoc_opt_opts_default(qoc_opt_opts* opts);

/* For it = 0..iters-1: F and dF/du of every problem, F_hist[it][p] = F_p (dev, iters*n_problems
 * doubles), then the update of u (dev [rows][n_ctrl], in place) unless problem p is frozen.
 * The initial pulses are u as the caller passes it: a warm start is the caller writing proposed
 * pulses (for instance the warm-start network's output, qoc_dense_forward) into u first, and a
 * fallback is a second call on the problems that did not converge, from other pulses.
 * Every convergence check also reads the status word: a latched error ends the loop with its code.
 * reached (dev, n_problems ints, may be NULL): first iteration whose F_p >= f_target, -1 if none.
 * *iters_done (host, may be NULL) receives the iterations run.  Returns QOC_ENOTCONVERGED if
 * f_target <= 1 and some problem did not reach it. */
int qoc_optimize_pulses(qoc_plan* plan, double* u, const double* psi0, const double* psif, const qoc_opt_opts* opts,
                        double* F_hist, int* reached, int* iters_done, void* workspace, size_t workspace_bytes,
                        void* stream);

/* ---------------------------------------------------------------- tuning */
/* Sweep kernel of the forward/backward passes (Sec. II.A, Eq. exppropagator; costates through
 * U_k^dagger as in Appendix B).  cl = 2..8 splits each (direction, block) chain over a
 * thread-block cluster of cl CTAs (rows of U_k per CTA, streamed through shared memory in sub-blocks
 * when they do not fit at once; state exchanged through distributed shared memory each step); 0 runs
 * one CTA per chain; -1 restores the automatic choice made at plan creation (the largest cluster,
 * 8 down to 2, for which every chain's cluster can be resident at once; blocks of m >= 24).
 * Returns QOC_EINVAL for other values, QOC_EUNSUPPORTED if the cluster buffers of the plan's largest
 * block do not fit in shared memory.  The paper has no counterpart: it is a launch-shape choice. */
int qoc_plan_set_sweep_cluster(qoc_plan* plan, int cl);
/* Current cluster size of the sweeps (0: one CTA per chain). */
int qoc_plan_sweep_cluster(const qoc_plan* plan, int* cl);

/* Slice derivatives as tall GEMMs (Appendix B, Eq. propagator_differentiation, exact form), for
 * single-problem FP32 plans in exact mode: the derivative series of every unsplit slice of the blocks
 * with at least min_m states runs as GEMMs shared by all slices of a chunk: A_k x = -i tau (H0 x +
 * sum_j u_kj Hc_j x) with H0, Hc_j the same for every slice, so one step of the power chains of all
 * slices is [H0; Hc_1; ...] times a matrix of their vectors, and the Hc_j v products it yields are the
 * ones the series contracts with.  mode 0: off (per-slice series kernels); 1: FP32 CUDA-core tiles;
 * 2 (default): tcgen05 tensor cores with both operands split into FP16 hi/lo planes (the products as
 * in qoc_tc_cgemm, FP32 accumulation; the columns scaled per slice by the chain bound beta^p).
 * min_m: 0 keeps the current threshold (default 129: smaller blocks use the register-tile kernel),
 * else 8..4096.  The workspace size may change: query qoc_plan_workspace_bytes again.  The results
 * agree to rounding.  The paper has no counterpart: it is a choice of kernels.
 * qoc_plan_deriv_gemm: number of blocks on the GEMM path (0 if off or none qualifies). */
int qoc_plan_set_deriv_gemm(qoc_plan* plan, int mode, int min_m);
int qoc_plan_deriv_gemm(const qoc_plan* plan, int* blocks);

/* One persistent launch per iteration (FP64 plans without checkpointing, exact derivative): on = 1
 * makes qoc_fidelity_and_grad and every iteration of qoc_optimize_pulses a single cooperative kernel
 * launch (preceded by a 16-byte memset of its counters) over all problems and blocks: norm check and
 * gathers, propagators (Eq. exppropagator), forward states and costates, overlaps (Eq. probability),
 * slice derivatives (Appendix B; reverse mode through the computed propagator for every slice), the
 * gradient and the update rule, separated by grid barriers whose waits give up after 2 s (status
 * QOC_ETIMEOUT).  Work inside a phase is handed out by atomic queues.  The workspace grows by one
 * scratch slot per resident CTA: query qoc_plan_workspace_bytes again.  Graph replay
 * (qoc_opt_opts.use_graph) captures the one launch.  Errors: QOC_EUNSUPPORTED (FP32 plan,
 * checkpointing, first-order mode, blocks too large for the kernel's shared memory).  The qoc_fidelity_forward /
 * qoc_fidelity_backward halves keep their own launches.  The paper has no counterpart. */
int qoc_plan_set_persistent(qoc_plan* plan, int on);

/* Kernel choice of the batched exponentials (Sec. II.A, Eq. exppropagator, as in qoc_expm_blocks):
 * rule i applies to blocks of size m <= m_max[i] (rules are tried in increasing m_max; the first
 * that applies wins): kind 0 = tiled CTA kernel, param = register tile R (1..7 FP32, 1..4 FP64; 0 =
 * by size); kind 1 = warp-packed kernel (m <= 32 FP32, <= 16 FP64, not with QOC_PREC_F32), param =
 * matrices per warp (0 = as many as fit); kind 2 = tcgen05 tensor-core kernel (FP32 plans, m <= 112;
 * products as in qoc_tc_cgemm), param 0 = only the slices that need no squaring (the block's other
 * slices run on the tiled kernel in a second launch), param 1 = every slice; kind 3 = tcgen05 tiled
 * batched GEMMs for large blocks (FP32 plans, m <= 2048; 128 x 128 output tiles, one launch per
 * product over a chunk of slices, operands kept in the workspace as pre-split FP16 planes) for the
 * slices that need no squaring, the tiled kernel for the rest (param ignored).  Blocks no rule
 * covers use the tiled kernel.  At plan creation QOC_PREC_F32 plans use kind 2, param 0 for blocks
 * of 25..112 states, kind 3 for 113..2048 and the tiled kernel for the rest; QOC_PREC_F32_ALL and
 * FP64 plans use the tiled kernel.  A tensor-core product (two FP16 halves per operand, all four
 * split products) errs up to about 2x an FP32 one, which the squarings of large-norm slices would
 * amplify.  The plan's workspace size may change: query qoc_plan_workspace_bytes again.  An
 * autotuner times candidate rules (paper_2309_05884_gb300/autotune.py). */
int qoc_plan_set_expm_rules(qoc_plan* plan, int n_rules, const int* m_max, const int* kind, const int* param);
/* The plan's current exponential launches: kind, param (R or MP), matrices per warp, largest block
 * and block count of each; arrays of max_out entries (may be NULL). */
int qoc_plan_expm_classes(const qoc_plan* plan, int max_out, int* n_classes, int* kind, int* param, int* per_warp,
                          int* m_max, int* n_blocks);

/* ---------------------------------------------------------------- measurement */
/* Phase timing: when enabled, every later call records CUDA events on its stream around each
 * phase's launches.  qoc_plan_phase_times waits for the last call and writes up to n_out sums of its
 * launch durations in ms, over every segment of a checkpointed call:
 *   [0] assembly + batched exponentials (both passes when checkpointing), [1] forward/backward
 *   sweeps, [2] overlap, [3] slice derivatives, [4] gradient reduction / update.
 * Work counters (reset by enabling): counts[0] = sum over (slice, block) items of m^3 times the
 * polynomial products taken (working precision), counts[1] = sum of m^3 times the squarings,
 * counts[2] = (slice, block) items exponentiated, counts[3] = complex multiply-adds of the exact
 * slice-derivative series done by the register-tile kernel (FP32 plans, unsplit slices): per item
 * (c (3P + 1) + n_ctrl) m^2 for c copies and series length P (2P matrix-vector products per copy,
 * the (P+1)-term M tile, the contraction with each Hc_j); counts[4] = complex multiply-adds of the
 * slice-derivative series of large blocks done as tall GEMMs (FP32 plans, m > 128, unsplit slices):
 * per item (1 + n_ctrl) m^2 2c (P + 1) for the chains and c n_ctrl m (P + 1)(P + 2)/2 for the
 * contraction; counts[5] = sum over (slice, block) items of m^3 times the tensor-core products taken
 * with three split terms instead of four (the Horner steps; counts[0] + counts[1] - counts[5] of the
 * tensor-core products keep all four). */
int qoc_plan_set_profiling(qoc_plan* plan, int on);
int qoc_plan_phase_times(qoc_plan* plan, float* ms_out, int n_out);
int qoc_plan_work_counts(qoc_plan* plan, long long* counts_out, int n_out);
/* Number of kernel launches one qoc_fidelity_and_grad (with_grad = 1) or qoc_propagate (0) call makes. */
int qoc_plan_kernel_launches(const qoc_plan* plan, int with_grad, int* launches);

/* ---------------------------------------------------------------- tensor-core products */
/* Batched complex products C[i] = A[i] B[i] on the 5th-generation tensor cores (tcgen05, kind::f16)
 * at about FP32 accuracy: every real part is split into two FP16 numbers (hi + lo) and the products
 * keep hi*hi + hi*lo + lo*hi with FP32 accumulation.  This is the building block of the matrix
 * exponentials of Eq. exppropagator (Sec. II.A) on the tensor cores.  A, B, C: dev, count complex64
 * (interleaved float) m x m row-major matrices each; m <= 112.  status (dev int, may be NULL): a
 * bounded wait that gave up sets bit 8.  Asynchronous on stream. */
int qoc_tc_cgemm(const float* A, const float* B, float* C, int m, long long count, int* status, void* stream);

/* ---------------------------------------------------------------- learned warm start */
/* Dense layers of the warm-start network (not part of the paper: a small MLP that proposes initial
 * pulses from a problem's parameters, trained on pulses optimised by this library's GRAPE).
 * Row-major device arrays; W is BF16 (uint16 bits) [out][in]; activations, biases and gradients
 * FP32; products accumulate in FP32.  act: 0 = identity, 1 = GELU(z) = z Phi(z) (exact, erf form).
 *   forward : Z = X W^T + bias (pre-activation, kept for backward), Y = act(Z); X [B][in], Z, Y [B][out]
 *   backward: dZ = dY * act'(Z); dX = dZ W (may be NULL); dW = dZ^T X [out][in]; db = column sums of dZ
 * Adam (descent): m, v and param FP32 [n]; shadow (BF16, may be NULL) receives the rounded param;
 * t counts steps from 1.  MSE: loss (dev double) = mean (Y - T)^2, dY = 2 (Y - T)/n (may be NULL). */
int qoc_dense_forward(const float* X, const uint16_t* W, const float* bias, float* Z, float* Y, long long B, int in,
                      int out, int act, void* stream);
int qoc_dense_backward(const float* X, const uint16_t* W, const float* Z, const float* dY, float* dZ, float* dX,
                       float* dW, float* db, long long B, int in, int out, int act, void* stream);
int qoc_adam_step(float* param, uint16_t* shadow_bf16, const float* grad, float* m, float* v, long long n, float lr,
                  float beta1, float beta2, float eps, int t, void* stream);
int qoc_mse(const float* Y, const float* T, float* dY, double* loss, long long n, void* stream);
int qoc_to_bf16(const float* x, uint16_t* y, long long n, void* stream);

/* ---------------------------------------------------------------- Trotterised per-qubit controls */
/* Sec. IV (Eqs. Hcprime, completeH_cpl, propagator_cpl, propagator_cpl_transformed): with one pulse
 * pair per qubit the Hamiltonian H_j = sum_i h_i^(j) + H_cpl has no symmetry left, and the slice
 * propagator is approximated by the ordered product (factor i = 1 leftmost)
 *     U_j = prod_{i=1..n} exp(-i tau h_i^(j)) E,   E = exp(-i tau/n H_cpl),
 *     h_i^(j) = 1/2 (Bz_ij sigma_z^(i) + Bx_ij sigma_x^(i) + By_ij sigma_y^(i)),
 * i.e. one 2 x 2 exponential per qubit and slice and a constant coupling factor that, H_cpl being
 * D_n symmetric, is E = A_D (direct sum over blocks of exp(-i tau/n H_cpl,b)) A_D^dagger: one block
 * exponential each, computed once by qoc_trotter_create.  States live in the full 2^n space.
 *
 * qoc_trotter_create: cpl is a D_n basis (every block, with vectors) whose H0 is H_cpl (its controls
 *   are not used); tau the slice length.  n <= 12 (QOC_EUNSUPPORTED beyond: the kernel keeps two
 *   2^n-amplitude buffers per CTA in shared memory).  Allocates device tables; free with
 *   qoc_trotter_free.  Errors: QOC_EINVAL (not D_n, missing blocks or vectors, bad tau), QOC_ECUDA.
 * qoc_trotter_propagate: psi_out[c] = U_N ... U_1 psi_in[c] for ncols full-space states (dev,
 *   [ncols][2^n] complex128, psi_out must not alias psi_in); pulses dev [N][n][3] doubles
 *   (Bz, Bx, By of qubit i in slice j at ((j * n) + i) * 3).  Columns = the identity gives the
 *   propagator K.  FP64.  Asynchronous on stream. */
typedef struct qoc_trotter qoc_trotter;
int qoc_trotter_create(const qoc_basis* cpl, double tau, qoc_trotter** out);
int qoc_trotter_propagate(const qoc_trotter* tr, const double* pulses, int N, const double* psi_in, double* psi_out,
                          long long ncols, void* stream);
void qoc_trotter_free(qoc_trotter* tr);

/* ---------------------------------------------------------------- allocation-free variant */
/* The paper has no counterpart to this entry point; it serves callers that cannot allocate device
 * memory while they run (a real-time loop that forbids allocator calls after start-up, a host whose
 * device memory is owned by another runtime, a caller without an allocator for a plan workspace).
 *
 * U[i] = exp(A[i]) for count complex FP64 m x m matrices (dev, row-major, interleaved re/im, A and
 * U of count*m*m complex each; U must not overlap A), by scaling and squaring with a Taylor
 * polynomial in FP64 (the method of qoc_expm_blocks, applied to arbitrary matrices).  Allocates
 * nothing: its working matrices live in a 16 MiB array inside the loaded library, which every GPU
 * that loads libqoc.so keeps until the process exits.
 *   - m must be 1..128, else QOC_EUNSUPPORTED with a message; count >= 0 (0 is a no-op).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture starts.  If the device
 *     is reset (cudaDeviceReset) the next call finds the cached address stale and looks it up again.
 *   - All calls share the array: calls whose kernels overlap on the GPU (other streams, other host
 *     threads) race and return wrong results; serialise them.
 *   - Asynchronous on 'stream'; errors of the launch itself are returned. */
int qoc_expm_batch_noalloc(const double* A, double* U, int m, long long count, void* stream);

/* ---------------------------------------------------------------- misc */
const char* qoc_strerror(int code);
const char* qoc_last_error(void);
int qoc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QOC_H */
