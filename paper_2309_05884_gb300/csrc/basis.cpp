// Host-side symmetry basis builder (runs once per system).
//
// Paper, Sec. II.A and Appendix A: the n-qubit space splits into orthogonal subspaces labelled by
// irreps of S_n or D_n, and A^dagger H A is block diagonal for every group-invariant H.
//
// S_n: blocks are spin sectors; the collective operators act on |J, M> by the standard
//      angular-momentum matrices (Appendix A, Clebsch-Gordan route), so the blocks are written
//      down analytically:  sum Z = 2 Jz,  sum X = J+ + J-,  sum Y = -i (J+ - J-),
//      sum_{i<j} a_i a_j = ((sum a)^2 - n)/2.  Full-space vectors (n <= 12) come from pivoted
//      Gram-Schmidt of each weight space against the vectors lowered from higher spin, then
//      repeated lowering |J, M-1> = J- |J, M> / sqrt(J(J+1) - M(M-1)).
// D_n: for each irrep theta (real orthogonal form) and each orbit of computational states under
//      rotations and reflections of the ring, the projector P_11 = (d/2n) sum_g D_11(g) rho(g)
//      (Eq. groupAlgebraElementsDn) is formed on the orbit span and its range orthonormalised by
//      pivoted Gram-Schmidt; the second copy of a 2-dimensional irrep is P_21 applied to row 1,
//      which makes both copies' blocks identical.  Block entries <e_a|H|e_b> use the sparse action
//      of the Pauli terms on basis states.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <new>
#include <stdexcept>

#include "qoc_internal.h"

namespace qoc {

namespace {

thread_local std::string g_last_error;

struct Err : std::runtime_error {
    int code;
    Err(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline int bit_at(uint64_t x, int p, int n) { return int((x >> (n - 1 - p)) & 1ULL); }
inline uint64_t mask_at(int p, int n) { return 1ULL << (n - 1 - p); }

// Apply sigma_a at position p to basis state x: returns new state, multiplies amp.
inline uint64_t pauli_apply(char a, int p, int n, uint64_t x, cplx& amp) {
    int b = bit_at(x, p, n);
    switch (a) {
        case 'x': return x ^ mask_at(p, n);
        case 'y': amp *= (b == 0) ? cplx(0, 1) : cplx(0, -1); return x ^ mask_at(p, n);
        default: if (b) amp = -amp; return x;
    }
}

char axis_of(int kind) {
    switch (kind) {
        case QOC_SUM_X: case QOC_ALLPAIRS_XX: case QOC_RING_XX: return 'x';
        case QOC_SUM_Y: case QOC_ALLPAIRS_YY: case QOC_RING_YY: return 'y';
        default: return 'z';
    }
}

// H|x> for a term list: calls emit(y, amplitude) for every produced component.
void apply_terms(const std::vector<qoc_term>& terms, int n, uint64_t x,
                 const std::function<void(uint64_t, cplx)>& emit) {
    for (const auto& t : terms) {
        char a = axis_of(t.kind);
        if (t.kind <= QOC_SUM_Z) {
            for (int p = 0; p < n; ++p) {
                cplx amp = t.coeff;
                uint64_t y = pauli_apply(a, p, n, x, amp);
                emit(y, amp);
            }
        } else if (t.kind <= QOC_ALLPAIRS_ZZ) {
            for (int p = 0; p < n; ++p)
                for (int q = p + 1; q < n; ++q) {
                    cplx amp = t.coeff;
                    uint64_t y = pauli_apply(a, q, n, x, amp);
                    y = pauli_apply(a, p, n, y, amp);
                    emit(y, amp);
                }
        } else {
            for (int p = 0; p < n; ++p) {
                int q = (p + t.dist) % n;
                cplx amp = t.coeff;
                uint64_t y = pauli_apply(a, q, n, x, amp);
                y = pauli_apply(a, p, n, y, amp);
                emit(y, amp);
            }
        }
    }
}

// An upper bound of the spectral norm of a Hermitian block M (m x m, row-major): for the entrywise
// moduli P = |M|, ||M||_2 = rho(M) <= rho(P) <= max_i (P x)_i / x_i for every positive x
// (Collatz-Wielandt).  Evaluated along power iterations on P + s I from x = 1 (the first bound is the
// max row sum, i.e. the 1-norm of a Hermitian matrix; the shift s, half of it, keeps the iteration
// from oscillating when P is bipartite, e.g. a hopping term, and leaves the ratios of P as they are),
// kept positive by a small floor; the smallest bound met is returned.  P is scanned once into its
// nonzeros, so an iteration costs their number.
double spectral_bound(const std::vector<cplx>& M, int m) {
    std::vector<int> ptr(m + 1, 0), col;
    std::vector<double> val;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) {
            const double a = std::abs(M[(size_t)i * m + j]);
            if (a > 0.0) {
                col.push_back(j);
                val.push_back(a);
            }
        }
        ptr[i + 1] = (int)col.size();
    }
    if (col.empty()) return 0.0;
    std::vector<double> x(m, 1.0), y(m);
    double best = std::numeric_limits<double>::infinity(), shift = -1.0;
    for (int it = 0; it < 300; ++it) {
        double hi = 0.0, lo = std::numeric_limits<double>::infinity(), ymax = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * x[col[k]];
            y[i] = s;
            hi = std::max(hi, s / x[i]);
            lo = std::min(lo, s / x[i]);
            ymax = std::max(ymax, s);
        }
        best = std::min(best, hi);
        if (hi - lo <= 1e-4 * hi || ymax <= 0.0) break;
        if (shift < 0.0) shift = 0.5 * hi;
        double zmax = 0.0;
        for (int i = 0; i < m; ++i) {
            y[i] += shift * x[i];
            zmax = std::max(zmax, y[i]);
        }
        for (int i = 0; i < m; ++i) x[i] = y[i] / zmax + 1e-6;
    }
    return best;
}

// Pivoted Gram-Schmidt: from candidate columns cand[k] (dense, length L), pick an orthonormal
// set spanning their span, orthogonal to the given 'against' vectors.  Stops at 'want' vectors or
// when every residual is below tol * max(1, largest initial norm) (an absolute floor, so that an
// all-zero candidate set yields nothing).
std::vector<std::vector<double>> pivoted_gs(std::vector<std::vector<double>> cand,
                                            const std::vector<std::vector<double>>& against,
                                            int want, double tol) {
    auto dot = [](const std::vector<double>& a, const std::vector<double>& b) {
        double s = 0.0;
        for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
        return s;
    };
    auto proj_out = [&](std::vector<double>& v, const std::vector<double>& q) {
        double d = dot(q, v);
        for (size_t i = 0; i < v.size(); ++i) v[i] -= d * q[i];
    };
    double scale = 0.0;
    for (auto& v : cand) scale = std::max(scale, std::sqrt(dot(v, v)));
    for (int pass = 0; pass < 2; ++pass)
        for (auto& v : cand)
            for (const auto& q : against) proj_out(v, q);
    std::vector<std::vector<double>> out;
    std::vector<char> used(cand.size(), 0);
    while (want < 0 || (int)out.size() < want) {
        int best = -1;
        double bn = 0.0;
        for (size_t k = 0; k < cand.size(); ++k) {
            if (used[k]) continue;
            double nn = std::sqrt(dot(cand[k], cand[k]));
            if (nn > bn) { bn = nn; best = (int)k; }
        }
        if (best < 0 || bn <= tol * std::max(scale, 1.0)) break;
        used[best] = 1;
        std::vector<double> q = cand[best];
        for (const auto& p : out) proj_out(q, p);  // re-orthogonalise
        double qn = std::sqrt(dot(q, q));
        for (auto& e : q) e /= qn;
        for (size_t k = 0; k < cand.size(); ++k)
            if (!used[k]) proj_out(cand[k], q);
        out.push_back(std::move(q));
    }
    return out;
}

uint64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

// ------------------------------------------------------------------------------------- S_n
void build_sn(qoc_basis& B, const std::vector<qoc_term>& h0,
              const std::vector<std::vector<qoc_term>>& hc, bool first_only, bool want_vectors) {
    const int n = B.n;
    auto check = [&](const std::vector<qoc_term>& ts) {
        for (const auto& t : ts)
            if (t.kind >= QOC_RING_XX && n >= 4)
                throw Err(QOC_EINVAL, "ring couplings are not S_n-invariant for n >= 4; use group D_n");
    };
    check(h0);
    for (auto& l : hc) check(l);

    // Analytic block of a term list in the |J, M = J - a> basis.
    auto block_of = [&](const std::vector<qoc_term>& ts, int J2) {
        const int m = J2 + 1;
        const double J = 0.5 * J2;
        std::vector<cplx> Jz(m * m), Jp(m * m), Jm(m * m);
        for (int a = 0; a < m; ++a) {
            double M = J - a;
            Jz[a * m + a] = M;
            if (a + 1 < m) {
                double c = std::sqrt(J * (J + 1) - M * (M - 1));
                Jm[(a + 1) * m + a] = c;  // J- |J,M> = c |J,M-1>
                Jp[a * m + (a + 1)] = c;
            }
        }
        auto mul = [&](const std::vector<cplx>& X, const std::vector<cplx>& Y) {
            std::vector<cplx> Z(m * m);
            for (int i = 0; i < m; ++i)
                for (int k = 0; k < m; ++k)
                    for (int j = 0; j < m; ++j) Z[i * m + j] += X[i * m + k] * Y[k * m + j];
            return Z;
        };
        std::vector<cplx> Sx(m * m), Sy(m * m), Sz(m * m);
        for (int i = 0; i < m * m; ++i) {
            Sz[i] = 2.0 * Jz[i];
            Sx[i] = Jp[i] + Jm[i];
            Sy[i] = cplx(0, -1) * (Jp[i] - Jm[i]);
        }
        std::vector<cplx> out(m * m);
        for (const auto& t : ts) {
            const std::vector<cplx>& S = (axis_of(t.kind) == 'x') ? Sx : (axis_of(t.kind) == 'y') ? Sy : Sz;
            if (t.kind <= QOC_SUM_Z) {
                for (int i = 0; i < m * m; ++i) out[i] += t.coeff * S[i];
            } else {
                // ALLPAIRS: ((sum a)^2 - n)/2; RING with n <= 3 equals ALLPAIRS (n = 3) or twice it (n = 2)
                double mult = 1.0;
                if (t.kind >= QOC_RING_XX) {
                    if (n == 3) mult = 1.0;
                    else if (n == 2) mult = 2.0;
                    else mult = 0.0;
                }
                std::vector<cplx> S2 = mul(S, S);
                for (int i = 0; i < m * m; ++i) out[i] += mult * t.coeff * 0.5 * S2[i];
                for (int a = 0; a < m; ++a) out[a * m + a] -= mult * t.coeff * 0.5 * n;
            }
        }
        return out;
    };

    const bool vectors = want_vectors && n <= 12;
    const bool only_first = first_only || n > 12;
    B.has_vectors = vectors;

    // Weight spaces for the vectors.
    std::vector<std::vector<uint64_t>> states;  // by weight
    std::vector<int64_t> pos;
    if (vectors) {
        states.resize(n + 1);
        pos.assign((size_t)1 << n, -1);
        for (uint64_t x = 0; x < (1ULL << n); ++x) {
            int w = __builtin_popcountll(x);
            pos[x] = (int64_t)states[w].size();
            states[w].push_back(x);
        }
    }
    std::vector<std::vector<std::vector<double>>> lowered(n + 1);  // by weight, dense over states[w]

    int64_t off = 0;
    for (int w = 0; w <= n / 2; ++w) {
        uint64_t copies = binom(n, w) - (w >= 1 ? binom(n, w - 1) : 0);
        if (copies == 0) continue;
        const int J2 = n - 2 * w;
        Block blk;
        blk.m = J2 + 1;
        blk.c = (int)std::min<uint64_t>(copies, 1ULL << 30);
        blk.label = (J2 % 2 == 0) ? ("J=" + std::to_string(J2 / 2)) : ("J=" + std::to_string(J2) + "/2");
        blk.h0 = block_of(h0, J2);
        blk.h0_norm = spectral_bound(blk.h0, blk.m);
        for (auto& l : hc) {
            auto M = block_of(l, J2);
            blk.hc_norm.push_back(spectral_bound(M, blk.m));
            blk.hc.insert(blk.hc.end(), M.begin(), M.end());
        }
        if (vectors) {
            const size_t L = states[w].size();
            std::vector<std::vector<double>> cand(L, std::vector<double>(L, 0.0));
            for (size_t k = 0; k < L; ++k) cand[k][k] = 1.0;
            auto hw = pivoted_gs(cand, lowered[w], (int)copies, 1e-8);
            if ((uint64_t)hw.size() != copies) throw Err(QOC_EINVAL, "S_n highest-weight construction failed");
            blk.vecs.resize((size_t)blk.c * blk.m);
            for (int r = 0; r < blk.c; ++r) {
                std::vector<double> cur = hw[r];
                const double J = 0.5 * J2;
                for (int a = 0; a <= J2; ++a) {
                    const int wa = w + a;
                    SparseVec sv;
                    for (size_t i = 0; i < cur.size(); ++i)
                        if (cur[i] != 0.0) { sv.idx.push_back((int64_t)states[wa][i]); sv.val.push_back(cur[i]); }
                    blk.vecs[(size_t)r * blk.m + a] = sv;
                    if (a > 0) lowered[wa].push_back(cur);
                    if (a == J2) break;
                    const double M = J - a;
                    const double c = std::sqrt(J * (J + 1) - M * (M - 1));
                    std::vector<double> nxt(states[wa + 1].size(), 0.0);
                    for (size_t i = 0; i < cur.size(); ++i) {
                        if (cur[i] == 0.0) continue;
                        uint64_t x = states[wa][i];
                        for (int p = 0; p < n; ++p)
                            if (!bit_at(x, p, n)) nxt[pos[x | mask_at(p, n)]] += cur[i];
                    }
                    for (auto& e : nxt) e /= c;
                    cur.swap(nxt);
                }
            }
        }
        blk.offset = off;
        off += (int64_t)blk.m * blk.c;
        B.blocks.push_back(std::move(blk));
        if (only_first) break;
    }
    B.state_len = off;
}

// ------------------------------------------------------------------------------------- D_n
struct GroupEl { int t, e; std::vector<int> perm; };

std::vector<GroupEl> dn_group(int n) {
    std::vector<GroupEl> G;
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < n; ++t) {
            GroupEl g{t, e, std::vector<int>(n)};
            for (int i = 0; i < n; ++i) g.perm[i] = (((e ? -i : i) + t) % n + n) % n;
            G.push_back(std::move(g));
        }
    return G;
}

uint64_t dn_act(const std::vector<int>& perm, uint64_t x, int n) {
    uint64_t y = 0;
    for (int i = 0; i < n; ++i)
        if (bit_at(x, i, n)) y |= mask_at(perm[i], n);
    return y;
}

struct Irrep { std::string label; int d; int kind; int mfreq; };

// D(t, e) of an irrep into out[d*d] (row-major), real orthogonal form.
void irrep_matrix(const Irrep& ir, int n, int t, int e, double* out) {
    switch (ir.kind) {
        case 0: out[0] = 1.0; return;                                  // A1
        case 1: out[0] = e ? -1.0 : 1.0; return;                       // A2
        case 2: out[0] = (t % 2) ? -1.0 : 1.0; return;                 // B1
        case 3: out[0] = ((t + e) % 2) ? -1.0 : 1.0; return;           // B2
        default: {                                                     // E_m: R(2 pi m t / n) diag(1, -1)^e
            double a = 2.0 * M_PI * ir.mfreq * t / n;
            double c = std::cos(a), s = std::sin(a);
            double f = e ? -1.0 : 1.0;
            out[0] = c; out[1] = -s * f;
            out[2] = s; out[3] = c * f;
        }
    }
}

void build_dn(qoc_basis& B, const std::vector<qoc_term>& h0,
              const std::vector<std::vector<qoc_term>>& hc, bool first_only, bool want_vectors) {
    const int n = B.n;
    const uint64_t dim = 1ULL << n;
    auto G = dn_group(n);
    std::vector<Irrep> irreps = {{"A1", 1, 0, 0}, {"A2", 1, 1, 0}};
    if (n % 2 == 0) { irreps.push_back({"B1", 1, 2, 0}); irreps.push_back({"B2", 1, 3, 0}); }
    for (int m = 1; m <= (n - 1) / 2; ++m) irreps.push_back({"E" + std::to_string(m), 2, 4, m});

    // Orbits ordered by smallest element.
    std::vector<int32_t> orbit_of(dim, -1), pos_in_orbit(dim, -1);
    std::vector<std::vector<uint64_t>> orbits;
    for (uint64_t x = 0; x < dim; ++x) {
        if (orbit_of[x] >= 0) continue;
        std::vector<uint64_t> orb;
        for (auto& g : G) orb.push_back(dn_act(g.perm, x, n));
        std::sort(orb.begin(), orb.end());
        orb.erase(std::unique(orb.begin(), orb.end()), orb.end());
        for (size_t i = 0; i < orb.size(); ++i) { orbit_of[orb[i]] = (int32_t)orbits.size(); pos_in_orbit[orb[i]] = (int32_t)i; }
        orbits.push_back(std::move(orb));
    }

    B.has_vectors = want_vectors;
    int64_t off = 0;
    std::vector<cplx> scratch(dim);
    std::vector<uint64_t> touched;
    std::vector<char> is_touched(dim, 0);
    for (const auto& ir : irreps) {
        const int d = ir.d;
        // Row vectors of this irrep, per orbit: rows[r] = list of (orbit id, dense coeffs).
        std::vector<std::vector<std::pair<int, std::vector<double>>>> rows(d);
        std::vector<std::vector<int>> orbit_vecs(orbits.size());  // indices into rows[0]
        double D[4];
        for (size_t o = 0; o < orbits.size(); ++o) {
            const auto& orb = orbits[o];
            const size_t L = orb.size();
            std::vector<double> P11(L * L, 0.0), P21(d == 2 ? L * L : 0, 0.0);
            for (auto& g : G) {
                irrep_matrix(ir, n, g.t, g.e, D);
                for (size_t i = 0; i < L; ++i) {
                    size_t j = (size_t)pos_in_orbit[dn_act(g.perm, orb[i], n)];
                    P11[j * L + i] += D[0];
                    if (d == 2) P21[j * L + i] += D[2];
                }
            }
            const double scale = double(d) / (2.0 * n);
            for (auto& v : P11) v *= scale;
            for (auto& v : P21) v *= scale;
            std::vector<std::vector<double>> cols(L, std::vector<double>(L));
            for (size_t i = 0; i < L; ++i)
                for (size_t j = 0; j < L; ++j) cols[i][j] = P11[j * L + i];
            auto q = pivoted_gs(cols, {}, -1, 1e-7);
            for (auto& v : q) {
                orbit_vecs[o].push_back((int)rows[0].size());
                if (d == 2) {
                    std::vector<double> v2(L, 0.0);
                    for (size_t j = 0; j < L; ++j)
                        for (size_t i = 0; i < L; ++i) v2[j] += P21[j * L + i] * v[i];
                    rows[1].push_back({(int)o, v2});
                }
                rows[0].push_back({(int)o, std::move(v)});
            }
        }
        const int m = (int)rows[0].size();
        if (m == 0) continue;
        Block blk;
        blk.m = m;
        blk.c = d;
        blk.label = ir.label;
        auto block_of = [&](const std::vector<qoc_term>& ts) {
            std::vector<cplx> M((size_t)m * m);
            for (int b = 0; b < m; ++b) {
                const auto& ob = rows[0][b];
                const auto& orb = orbits[ob.first];
                touched.clear();
                for (size_t i = 0; i < orb.size(); ++i) {
                    double cb = ob.second[i];
                    if (cb == 0.0) continue;
                    apply_terms(ts, n, orb[i], [&](uint64_t y, cplx amp) {
                        if (!is_touched[y]) { is_touched[y] = 1; touched.push_back(y); scratch[y] = 0.0; }
                        scratch[y] += amp * cb;
                    });
                }
                for (uint64_t y : touched) {
                    is_touched[y] = 0;
                    int o = orbit_of[y];
                    int p = pos_in_orbit[y];
                    for (int a : orbit_vecs[o]) M[(size_t)a * m + b] += rows[0][a].second[p] * scratch[y];
                }
            }
            return M;
        };
        blk.h0 = block_of(h0);
        blk.h0_norm = spectral_bound(blk.h0, m);
        for (auto& l : hc) {
            auto M = block_of(l);
            blk.hc_norm.push_back(spectral_bound(M, m));
            blk.hc.insert(blk.hc.end(), M.begin(), M.end());
        }
        if (want_vectors) {
            blk.vecs.resize((size_t)d * m);
            for (int r = 0; r < d; ++r)
                for (int a = 0; a < m; ++a) {
                    SparseVec sv;
                    const auto& ov = rows[r][a];
                    const auto& orb = orbits[ov.first];
                    for (size_t i = 0; i < orb.size(); ++i)
                        if (ov.second[i] != 0.0) { sv.idx.push_back((int64_t)orb[i]); sv.val.push_back(ov.second[i]); }
                    blk.vecs[(size_t)r * m + a] = std::move(sv);
                }
        }
        blk.offset = off;
        off += (int64_t)m * d;
        B.blocks.push_back(std::move(blk));
        if (first_only) break;
    }
    B.state_len = off;
}

}  // namespace

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

const char* last_error_cstr() { return g_last_error.c_str(); }

}  // namespace qoc

// ===================================================================================== C ABI
using namespace qoc;

extern "C" {

const char* qoc_last_error(void) { return qoc::last_error_cstr(); }

const char* qoc_strerror(int code) {
    switch (code) {
        case QOC_OK: return "ok";
        case QOC_EINVAL: return "invalid argument";
        case QOC_ENOMEM: return "out of memory";
        case QOC_ECUDA: return "CUDA error";
        case QOC_ETIMEOUT: return "device wait timed out";
        case QOC_EUNSUPPORTED: return "unsupported size or option";
        case QOC_ENOTCONVERGED: return "not converged";
        default: return "unknown error";
    }
}

int qoc_version(void) { return 100; }

int qoc_build_symmetry_basis(const qoc_system_desc* sys, int flags, qoc_basis** out) {
    if (!sys || !out) return set_error(QOC_EINVAL, "null argument");
    *out = nullptr;
    try {
        if (sys->group != QOC_GROUP_SN && sys->group != QOC_GROUP_DN)
            return set_error(QOC_EINVAL, "group must be QOC_GROUP_SN or QOC_GROUP_DN");
        if (sys->group == QOC_GROUP_SN && (sys->n < 1 || sys->n > 64))
            return set_error(QOC_EUNSUPPORTED, "S_n builds need 1 <= n <= 64");
        if (sys->group == QOC_GROUP_DN && (sys->n < 3 || sys->n > 16))
            return set_error(QOC_EUNSUPPORTED, "D_n builds need 3 <= n <= 16");
        if (sys->n_ctrl < 1 || sys->n_ctrl > 8) return set_error(QOC_EINVAL, "n_ctrl must be 1..8");
        if (sys->n_h0_terms < 0 || (sys->n_h0_terms > 0 && !sys->h0) || !sys->n_hc_terms || !sys->hc)
            return set_error(QOC_EINVAL, "null term list");
        auto copy_terms = [&](const qoc_term* t, int cnt) {
            std::vector<qoc_term> v(t, t + cnt);
            for (auto& e : v) {
                if (e.kind < QOC_SUM_X || e.kind > QOC_RING_ZZ) throw Err(QOC_EINVAL, "unknown term kind");
                if (!std::isfinite(e.coeff)) throw Err(QOC_EINVAL, "non-finite term coefficient");
                if (e.kind >= QOC_RING_XX && (e.dist < 1 || e.dist >= sys->n))
                    throw Err(QOC_EINVAL, "ring distance must be 1..n-1");
            }
            return v;
        };
        std::vector<qoc_term> h0 = copy_terms(sys->h0, sys->n_h0_terms);
        std::vector<std::vector<qoc_term>> hc;
        for (int j = 0; j < sys->n_ctrl; ++j) {
            if (sys->n_hc_terms[j] < 1 || !sys->hc[j]) return set_error(QOC_EINVAL, "empty control term list");
            hc.push_back(copy_terms(sys->hc[j], sys->n_hc_terms[j]));
        }
        auto* B = new qoc_basis();
        B->n = sys->n;
        B->group = sys->group;
        B->n_ctrl = sys->n_ctrl;
        B->full_dim = sys->n <= 62 ? (int64_t(1) << sys->n) : 0;
        const bool first = flags & QOC_BASIS_FIRST_BLOCK_ONLY;
        const bool vecs = !(flags & QOC_BASIS_NO_VECTORS);
        try {
            if (sys->group == QOC_GROUP_SN) build_sn(*B, h0, hc, first, vecs);
            else build_dn(*B, h0, hc, first, vecs);
        } catch (...) {
            delete B;
            throw;
        }
        *out = B;
        return QOC_OK;
    } catch (const Err& e) {
        return set_error(e.code, e.what());
    } catch (const std::bad_alloc&) {
        return set_error(QOC_ENOMEM, "host allocation failed while building the basis");
    } catch (const std::exception& e) {
        return set_error(QOC_EINVAL, e.what());
    }
}

int qoc_basis_info(const qoc_basis* B, int* n_blocks, int* n_ctrl, int64_t* state_len, int64_t* full_dim) {
    if (!B) return set_error(QOC_EINVAL, "null basis");
    if (n_blocks) *n_blocks = (int)B->blocks.size();
    if (n_ctrl) *n_ctrl = B->n_ctrl;
    if (state_len) *state_len = B->state_len;
    if (full_dim) *full_dim = B->full_dim;
    return QOC_OK;
}

int qoc_basis_block(const qoc_basis* B, int b, int* size, int* copies, int64_t* offset, char* label) {
    if (!B || b < 0 || b >= (int)B->blocks.size()) return set_error(QOC_EINVAL, "bad block index");
    const auto& blk = B->blocks[b];
    if (size) *size = blk.m;
    if (copies) *copies = blk.c;
    if (offset) *offset = blk.offset;
    if (label) {
        std::strncpy(label, blk.label.c_str(), 15);
        label[15] = 0;
    }
    return QOC_OK;
}

int qoc_basis_block_matrices(const qoc_basis* B, int b, double* h0, double* hc) {
    if (!B || b < 0 || b >= (int)B->blocks.size()) return set_error(QOC_EINVAL, "bad block index");
    const auto& blk = B->blocks[b];
    if (h0) std::memcpy(h0, blk.h0.data(), blk.h0.size() * sizeof(cplx));
    if (hc) std::memcpy(hc, blk.hc.data(), blk.hc.size() * sizeof(cplx));
    return QOC_OK;
}

int qoc_basis_norm_bounds(const qoc_basis* B, int b, double* out) {
    if (!B || !out || b < 0 || b >= (int)B->blocks.size()) return set_error(QOC_EINVAL, "bad argument");
    const auto& blk = B->blocks[b];
    out[0] = blk.h0_norm;
    for (size_t j = 0; j < blk.hc_norm.size(); ++j) out[1 + j] = blk.hc_norm[j];
    return QOC_OK;
}

int qoc_state_to_blocks(const qoc_basis* B, const double* full, double* blk) {
    if (!B || !full || !blk) return set_error(QOC_EINVAL, "null argument");
    if (!B->has_vectors) return set_error(QOC_EUNSUPPORTED, "basis was built without full-space vectors");
    const cplx* f = reinterpret_cast<const cplx*>(full);
    cplx* o = reinterpret_cast<cplx*>(blk);
    for (const auto& b : B->blocks)
        for (int r = 0; r < b.c; ++r)
            for (int a = 0; a < b.m; ++a) {
                const auto& v = b.vecs[(size_t)r * b.m + a];
                cplx s = 0.0;
                for (size_t i = 0; i < v.idx.size(); ++i) s += v.val[i] * f[v.idx[i]];
                o[b.offset + (int64_t)r * b.m + a] = s;
            }
    return QOC_OK;
}

int qoc_blocks_to_state(const qoc_basis* B, const double* blk, double* full) {
    if (!B || !full || !blk) return set_error(QOC_EINVAL, "null argument");
    if (!B->has_vectors) return set_error(QOC_EUNSUPPORTED, "basis was built without full-space vectors");
    const cplx* in = reinterpret_cast<const cplx*>(blk);
    cplx* f = reinterpret_cast<cplx*>(full);
    for (int64_t i = 0; i < B->full_dim; ++i) f[i] = 0.0;
    for (const auto& b : B->blocks)
        for (int r = 0; r < b.c; ++r)
            for (int a = 0; a < b.m; ++a) {
                const auto& v = b.vecs[(size_t)r * b.m + a];
                cplx c = in[b.offset + (int64_t)r * b.m + a];
                for (size_t i = 0; i < v.idx.size(); ++i) f[v.idx[i]] += v.val[i] * c;
            }
    return QOC_OK;
}

int qoc_dicke_state(const qoc_basis* B, int k, double* blk) {
    if (!B || !blk) return set_error(QOC_EINVAL, "null argument");
    if (B->group != QOC_GROUP_SN) return set_error(QOC_EINVAL, "Dicke states are defined for S_n bases");
    if (k < 0 || k > B->n) return set_error(QOC_EINVAL, "Dicke index out of range");
    for (int64_t i = 0; i < 2 * B->state_len; ++i) blk[i] = 0.0;
    blk[2 * (B->blocks[0].offset + k)] = 1.0;
    return QOC_OK;
}

void qoc_basis_free(qoc_basis* B) { delete B; }

}  // extern "C"
