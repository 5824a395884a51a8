// Small dense FP64 linear algebra for the operator precomputation.
// Matrices are row-major std::vector<double> with explicit dimensions.
#pragma once
#include <cstdint>
#include <vector>

namespace kifmm {

struct Svd {
    int m = 0, n = 0;           // A is m x n, m >= n
    std::vector<double> u;      // m x n, columns = left singular vectors
    std::vector<double> s;      // n, descending
    std::vector<double> v;      // n x n, columns = right singular vectors
};

// One-sided (Hestenes) Jacobi SVD of a row-major m x n matrix, m >= n.
// Rotations are applied to column pairs until every pair is orthogonal to
// a relative 1e-15; singular values are the final column norms.
Svd jacobi_svd(const std::vector<double> &a, int m, int n);

// R factor (n x n, upper triangular, row-major) of the Householder QR of a
// tall matrix given as a sequence of row blocks, each `rows_per_block x n`
// row-major.  Blocks are folded in one group at a time (R <- qr([R; B]).R),
// so memory stays O(n^2 + block).
class TallQR {
public:
    explicit TallQR(int n);
    void add_rows(const double *rows, int count); // count x n row-major
    void finish() { fold(); }                     // fold remaining rows
    const std::vector<double> &r() const { return r_; }
private:
    int n_;
    bool have_r_ = false;
    std::vector<double> r_;
    std::vector<double> pending_; // rows waiting to be folded in
    int npending_ = 0;
    void fold();
};

// y = A x for row-major A (m x n).
void matvec(const std::vector<double> &a, int m, int n, const double *x,
            double *y);

// C = A B, row-major; A m x k, B k x n.
std::vector<double> matmul(const std::vector<double> &a,
                           const std::vector<double> &b, int m, int k, int n);

// Transpose of a row-major m x n matrix.
std::vector<double> transpose(const std::vector<double> &a, int m, int n);

} // namespace kifmm
