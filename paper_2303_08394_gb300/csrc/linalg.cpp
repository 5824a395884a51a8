// FP64 Jacobi SVD and blocked Householder QR (see linalg.h).
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace kifmm {

Svd jacobi_svd(const std::vector<double> &a, int m, int n) {
    // Work on columns: store A column-major so a column is contiguous.
    std::vector<double> col((size_t)m * n), v((size_t)n * n, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) col[(size_t)j * m + i] = a[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) v[(size_t)j * n + j] = 1.0;  // column-major V
    std::vector<double> norm2(n);
    for (int j = 0; j < n; ++j) {
        double s = 0;
        const double *cj = &col[(size_t)j * m];
        for (int i = 0; i < m; ++i) s += cj[i] * cj[i];
        norm2[j] = s;
    }
    const double tol = 1e-15;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *cp = &col[(size_t)p * m], *cq = &col[(size_t)q * m];
                double alpha = norm2[p], beta = norm2[q], gamma = 0.0;
                for (int i = 0; i < m; ++i) gamma += cp[i] * cq[i];
                if (alpha == 0.0 || beta == 0.0) continue;
                double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
                if (rel <= tol) continue;
                off = std::max(off, rel);
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) /
                           (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < m; ++i) {
                    double x = cp[i], y = cq[i];
                    cp[i] = c * x - s * y;
                    cq[i] = s * x + c * y;
                }
                double *vp = &v[(size_t)p * n], *vq = &v[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
                // recompute norms of the two rotated columns exactly
                double np = 0, nq = 0;
                for (int i = 0; i < m; ++i) { np += cp[i] * cp[i]; nq += cq[i] * cq[i]; }
                norm2[p] = np;
                norm2[q] = nq;
            }
        }
        if (off <= tol) break;
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return norm2[x] > norm2[y]; });
    Svd out;
    out.m = m;
    out.n = n;
    out.u.assign((size_t)m * n, 0.0);
    out.s.assign(n, 0.0);
    out.v.assign((size_t)n * n, 0.0);
    for (int jj = 0; jj < n; ++jj) {
        int j = order[jj];
        double sv = std::sqrt(norm2[j]);
        out.s[jj] = sv;
        const double *cj = &col[(size_t)j * m];
        for (int i = 0; i < m; ++i)
            out.u[(size_t)i * n + jj] = sv > 0 ? cj[i] / sv : 0.0;
        const double *vj = &v[(size_t)j * n];
        for (int i = 0; i < n; ++i) out.v[(size_t)i * n + jj] = vj[i];
    }
    return out;
}

TallQR::TallQR(int n) : n_(n) {}

void TallQR::add_rows(const double *rows, int count) {
    pending_.insert(pending_.end(), rows, rows + (size_t)count * n_);
    npending_ += count;
    if (npending_ >= 16 * n_) fold();
}

// Householder QR of [R; pending] (column-major work array), keep R.
void TallQR::fold() {
    if (npending_ == 0) return;
    const int n = n_;
    const int m = (have_r_ ? n : 0) + npending_;
    std::vector<double> w((size_t)m * n);  // column-major
    int row = 0;
    if (have_r_) {
        for (int i = 0; i < n; ++i, ++row)
            for (int j = 0; j < n; ++j) w[(size_t)j * m + row] = r_[(size_t)i * n + j];
    }
    for (int i = 0; i < npending_; ++i, ++row)
        for (int j = 0; j < n; ++j) w[(size_t)j * m + row] = pending_[(size_t)i * n + j];
    std::vector<double> vh(m);
    for (int j = 0; j < n && j < m; ++j) {
        double *cj = &w[(size_t)j * m];
        double nrm = 0;
        for (int i = j; i < m; ++i) nrm += cj[i] * cj[i];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = cj[j] > 0 ? -nrm : nrm;
        for (int i = j; i < m; ++i) vh[i] = cj[i];
        vh[j] -= alpha;
        double vn2 = 0;
        for (int i = j; i < m; ++i) vn2 += vh[i] * vh[i];
        cj[j] = alpha;
        for (int i = j + 1; i < m; ++i) cj[i] = 0.0;
        if (vn2 == 0.0) continue;
#pragma omp parallel for schedule(static)
        for (int c = j + 1; c < n; ++c) {
            double *cc = &w[(size_t)c * m];
            double d = 0;
            for (int i = j; i < m; ++i) d += vh[i] * cc[i];
            double f = 2.0 * d / vn2;
            for (int i = j; i < m; ++i) cc[i] -= f * vh[i];
        }
    }
    r_.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n && i < m; ++i)
        for (int j = i; j < n; ++j) r_[(size_t)i * n + j] = w[(size_t)j * m + i];
    have_r_ = true;
    pending_.clear();
    npending_ = 0;
}

void matvec(const std::vector<double> &a, int m, int n, const double *x,
            double *y) {
    for (int i = 0; i < m; ++i) {
        double s = 0;
        for (int j = 0; j < n; ++j) s += a[(size_t)i * n + j] * x[j];
        y[i] = s;
    }
}

std::vector<double> matmul(const std::vector<double> &a,
                           const std::vector<double> &b, int m, int k, int n) {
    std::vector<double> c((size_t)m * n, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double *ci = &c[(size_t)i * n];
        for (int l = 0; l < k; ++l) {
            double ail = a[(size_t)i * k + l];
            if (ail == 0.0) continue;
            const double *bl = &b[(size_t)l * n];
            for (int j = 0; j < n; ++j) ci[j] += ail * bl[j];
        }
    }
    return c;
}

std::vector<double> transpose(const std::vector<double> &a, int m, int n) {
    std::vector<double> t((size_t)n * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) t[(size_t)j * m + i] = a[(size_t)i * n + j];
    return t;
}

} // namespace kifmm
