// Host-side one-time analysis for the refactorization solver.
//
// The paper's CPU/GPU split (Section 1.3, refactorization; Section 3.1.1:
// the first matrices are factorized with pivoting on the CPU, and only
// numeric refactorization runs on the GPU afterwards): everything in this
// file runs once per sparsity pattern on the host, in C++.
//
//   * canonicalize      -- validate the caller's CSR pattern and sort it;
//   * order_colamd_like -- fill-reducing column order: approximate minimum
//                          degree on the column-intersection graph (pattern
//                          of A^T A), using the rows of A as the initial
//                          elements of a quotient graph, with element
//                          absorption and supervariables;
//   * pivot_lu          -- first numeric LU of A(:,Q) with threshold partial
//                          pivoting (diagonal preference), which fixes P;
//   * symbolic          -- L/U structure of A(P,Q) for a fixed P (no numeric
//                          work), used when the caller supplies P;
//   * build_layout      -- the row-major combined factor layout the GPU
//                          kernels use, with the value gather map.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kkt {

struct Csr {
    int32_t n = 0;
    std::vector<int32_t> rowptr, colind;   // sorted, duplicate free
    std::vector<int64_t> src;              // canonical entry -> caller entry
    bool identity_src = true;              // caller order was already canonical
};

// Returns 0 or a negative KKT_ERR_* code.
int canonicalize(int32_t n, const int32_t* rowptr, const int32_t* colind, Csr* out, std::string* why);

// Column order Q (Q[j] = original column placed j-th).
int order_colamd_like(const Csr& A, std::vector<int32_t>* Q);

// Column-oriented structure of the factors in the permuted space:
// for column j, L rows (> j) and U rows (<= j, diagonal included).
struct ColStructure {
    std::vector<int64_t> Lp, Up;
    std::vector<int32_t> Li, Ui;
};

// Threshold partial pivoting LU on the values of A (canonical order).
// Outputs P (P[i] = original row of the i-th pivot) and the structure.
int pivot_lu(const Csr& A, const double* vals, const std::vector<int32_t>& Q, double tol,
             std::vector<int32_t>* P, ColStructure* S, int32_t* bad_col);

// Structure of A(P,Q) = LU for a given P (validates that every pivot is
// structurally present).
int symbolic(const Csr& A, const std::vector<int32_t>& P, const std::vector<int32_t>& Q,
             ColStructure* S, int32_t* bad_col);

// Row-major combined factor F = L + U - I in the permuted space.
// Row i holds, columns ascending: L(i, k<i), U(i,i), U(i, j>i).
struct Layout {
    int32_t n = 0;
    std::vector<int64_t> Fp;       // n+1 row pointers
    std::vector<int32_t> Fj;       // column indices
    std::vector<int64_t> Fdiag;    // position of the diagonal in each row
    std::vector<int64_t> Fsrc;     // F slot -> canonical A entry, -1 for fill
    int64_t nnzL = 0, nnzU = 0;    // strict lower, upper incl. diagonal
    int32_t levelsL = 0, levelsU = 0;
    std::vector<int32_t> levL;     // L-solve DAG level of each row (rows ascending)
    std::vector<int32_t> levU;     // U-solve DAG level of each row (rows descending)
    double updates = 0;            // multiply-adds of one refactorization
};

int build_layout(const Csr& A, const std::vector<int32_t>& P, const std::vector<int32_t>& Q,
                 const ColStructure& S, Layout* out);

}  // namespace kkt
