// Internal structures shared by the host builder (basis.cpp) and the CUDA plan (plan.cu).
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qoc.h"

namespace qoc {

using cplx = std::complex<double>;

// A sparse full-space vector supported on few computational states (one D_n orbit, or one
// S_n weight space); coefficients are real for both groups in the gauges used here.
struct SparseVec {
    std::vector<int64_t> idx;
    std::vector<double> val;
};

struct Block {
    int m = 0;                 // block size
    int c = 0;                 // identical copies
    int64_t offset = 0;        // complex offset of copy 0 in a block state
    std::string label;
    std::vector<cplx> h0;      // m*m row-major
    std::vector<cplx> hc;      // n_ctrl*m*m
    double h0_norm = 0.0;     // upper bound of the spectral norm of H0_b (basis.cpp: spectral_bound)
    std::vector<double> hc_norm;
    std::vector<SparseVec> vecs;  // c*m basis vectors (copy-major), empty without vectors
};

}  // namespace qoc

struct qoc_basis {
    int n = 0;
    int group = 0;
    int n_ctrl = 0;
    bool has_vectors = false;
    int64_t state_len = 0;
    int64_t full_dim = 0;
    std::vector<qoc::Block> blocks;
};

namespace qoc {
// Thread-local last-error message (set by every failing entry point).
int set_error(int code, const std::string& msg);
}  // namespace qoc
