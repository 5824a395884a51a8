// FP64 precomputation of the KIFMM operators ("Parallelization strategies
// for FMM operators": the M2M and L2L matrices are precomputed once and
// rescaled per level; "Computational structure of FMM operators": check and
// equivalent surfaces of 6(p-1)^2 + 2 points).
//
// Everything is computed for the unit box with the kernel 1/r; the 1/(4 pi)
// factor and the physical length scale are applied once per potential.
//
// Pseudo-inverses are kept in factored form A^+ = V diag(1/s) U^T with the
// singular values below rcond * s_max dropped.  The GPU applies U^T, then
// 1/s, then V in FP32; an explicitly formed A^+ would carry eps * cond(A)
// of rounding in every direction (cond ~ 1e9 at p = 6), while the factored
// form keeps the rounding in the directions the next operator damps.
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>

#include "linalg.h"
#include "plan.h"

namespace kifmm {

int offset_index(int tx, int ty, int tz) {
    if (tx < -3 || tx > 3 || ty < -3 || ty > 3 || tz < -3 || tz > 3) return -1;
    if (std::abs(tx) <= 1 && std::abs(ty) <= 1 && std::abs(tz) <= 1) return -1;
    int idx = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                if (std::abs(a) <= 1 && std::abs(b) <= 1 && std::abs(c) <= 1) continue;
                if (a == tx && b == ty && c == tz) return idx;
                ++idx;
            }
    return -1;
}

namespace {

std::vector<double> unit_surface(int p) {
    std::vector<double> s;
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b)
            for (int c = 0; c < p; ++c) {
                bool boundary = a == 0 || b == 0 || c == 0 || a == p - 1 ||
                                b == p - 1 || c == p - 1;
                if (!boundary) continue;
                s.push_back(-1.0 + 2.0 * a / (p - 1));
                s.push_back(-1.0 + 2.0 * b / (p - 1));
                s.push_back(-1.0 + 2.0 * c / (p - 1));
            }
    return s;
}

// K[i][j] = 1 / |t_i - s_j| (0 if coincident); t_i = tc + ta * surf_i,
// s_j = sc + sa * surf_j.
std::vector<double> surface_kernel(const std::vector<double> &surf, int ns,
                                   const double tc[3], double ta,
                                   const double sc[3], double sa) {
    std::vector<double> k((size_t)ns * ns);
    for (int i = 0; i < ns; ++i) {
        double tx = tc[0] + ta * surf[3 * i], ty = tc[1] + ta * surf[3 * i + 1],
               tz = tc[2] + ta * surf[3 * i + 2];
        for (int j = 0; j < ns; ++j) {
            double dx = tx - (sc[0] + sa * surf[3 * j]);
            double dy = ty - (sc[1] + sa * surf[3 * j + 1]);
            double dz = tz - (sc[2] + sa * surf[3 * j + 2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            k[(size_t)i * ns + j] = r2 > 0 ? 1.0 / std::sqrt(r2) : 0.0;
        }
    }
    return k;
}

// Truncated SVD factors of a square ns x ns matrix.
void truncated_svd(const std::vector<double> &a, int ns, double rcond,
                   std::vector<double> &u, std::vector<double> &s,
                   std::vector<double> &v, int &rank) {
    Svd d = jacobi_svd(a, ns, ns);
    rank = 0;
    while (rank < ns && d.s[rank] > rcond * d.s[0]) ++rank;
    if (rank == 0) throw std::runtime_error("check-to-equivalent matrix is zero");
    u.assign((size_t)ns * rank, 0.0);
    v.assign((size_t)ns * rank, 0.0);
    s.assign(d.s.begin(), d.s.begin() + rank);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < rank; ++j) {
            u[(size_t)i * rank + j] = d.u[(size_t)i * ns + j];
            v[(size_t)i * rank + j] = d.v[(size_t)i * ns + j];
        }
}

std::shared_ptr<Operators> compute(int p, double ai, double ao, double rcond,
                                   double eps_svd) {
    auto op = std::make_shared<Operators>();
    op->p = p;
    op->ai = ai;
    op->ao = ao;
    op->rcond = rcond;
    op->eps_svd = eps_svd;
    op->surf = unit_surface(p);
    const int ns = (int)op->surf.size() / 3;
    op->ns = ns;
    const double zero[3] = {0, 0, 0};

    truncated_svd(surface_kernel(op->surf, ns, zero, ao, zero, ai), ns, rcond,
                  op->Pu, op->Ps, op->Pv, op->rP);
    truncated_svd(surface_kernel(op->surf, ns, zero, ai, zero, ao), ns, rcond,
                  op->Qu, op->Qs, op->Qv, op->rQ);
    const int rP = op->rP, rQ = op->rQ;
    auto PuT = transpose(op->Pu, ns, rP);   // rP x ns
    auto QuT = transpose(op->Qu, ns, rQ);   // rQ x ns

    op->M2M.assign((size_t)8 * rP * ns, 0.0);
    op->L2L.assign((size_t)8 * rQ * ns, 0.0);
    for (int sg = 0; sg < 8; ++sg) {
        double c[3] = {(sg & 1) - 0.5, ((sg >> 1) & 1) - 0.5, ((sg >> 2) & 1) - 0.5};
        // parent (h = 1) upward check surface <- child (h = 1/2) equivalent
        auto k_up = surface_kernel(op->surf, ns, zero, ao, c, 0.5 * ai);
        auto m = matmul(PuT, k_up, rP, ns, ns);
        std::copy(m.begin(), m.end(), op->M2M.begin() + (size_t)sg * rP * ns);
        // child downward check surface <- parent downward equivalent; the
        // factor 1/2 converts the potential to child-normalised units
        auto k_dn = surface_kernel(op->surf, ns, c, 0.5 * ai, zero, ao);
        for (auto &x : k_dn) x *= 0.5;
        auto l = matmul(QuT, k_dn, rQ, ns, ns);
        std::copy(l.begin(), l.end(), op->L2L.begin() + (size_t)sg * rQ * ns);
    }

    // M2L operators K_t for the 316 offsets
    std::vector<std::vector<double>> kt(kNumOffsets);
    int idx = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                if (std::abs(a) <= 1 && std::abs(b) <= 1 && std::abs(c) <= 1) continue;
                double sc[3] = {2.0 * a, 2.0 * b, 2.0 * c};
                kt[idx++] = surface_kernel(op->surf, ns, zero, ai, sc, ai);
            }
    if (eps_svd > 0) {
        // left factor: row space of H^T = [K_1^T; ...; K_316^T]
        TallQR qh(ns), qw(ns);
        for (int t = 0; t < kNumOffsets; ++t) {
            auto ktt = transpose(kt[t], ns, ns);
            qh.add_rows(ktt.data(), ns);
            qw.add_rows(kt[t].data(), ns);
        }
        qh.finish();
        qw.finish();
        Svd sh = jacobi_svd(qh.r(), ns, ns);
        Svd sw = jacobi_svd(qw.r(), ns, ns);
        // A tall M = Q R with R = U S V^T has right singular vectors V.
        int kh = 0, kw = 0;
        while (kh < ns && sh.s[kh] > eps_svd * sh.s[0]) ++kh;
        while (kw < ns && sw.s[kw] > eps_svd * sw.s[0]) ++kw;
        int k = std::max(kh, kw);
        op->k = k;
        op->sigmaH = sh.s;
        op->sigmaW = sw.s;
        op->Uk.assign((size_t)ns * k, 0.0);
        op->Vk.assign((size_t)ns * k, 0.0);
        for (int i = 0; i < ns; ++i)
            for (int j = 0; j < k; ++j) {
                op->Uk[(size_t)i * k + j] = sh.v[(size_t)i * ns + j];
                op->Vk[(size_t)i * k + j] = sw.v[(size_t)i * ns + j];
            }
    } else {
        op->k = ns;
        op->Uk.assign((size_t)ns * ns, 0.0);
        op->Vk.assign((size_t)ns * ns, 0.0);
        for (int i = 0; i < ns; ++i) op->Uk[(size_t)i * ns + i] = op->Vk[(size_t)i * ns + i] = 1.0;
    }
    const int k = op->k;
    auto UkT = transpose(op->Uk, ns, k);
    op->S.assign((size_t)kNumOffsets * k * k, 0.0);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < kNumOffsets; ++t) {
        auto kv = matmul(kt[t], op->Vk, ns, ns, k);     // ns x k
        auto s = matmul(UkT, kv, k, ns, k);             // k x k
        std::copy(s.begin(), s.end(), op->S.begin() + (size_t)t * k * k);
    }
    op->QUk = matmul(QuT, op->Uk, rQ, ns, k);
    return op;
}

} // namespace

std::shared_ptr<const Operators> get_operators(int p, double ai, double ao,
                                               double rcond, double eps_svd) {
    static std::mutex mu;
    static std::map<std::tuple<int, double, double, double, double>,
                    std::shared_ptr<const Operators>> cache;
    auto key = std::make_tuple(p, ai, ao, rcond, eps_svd);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    auto op = compute(p, ai, ao, rcond, eps_svd);
    std::lock_guard<std::mutex> g(mu);
    cache[key] = op;
    return op;
}

} // namespace kifmm
