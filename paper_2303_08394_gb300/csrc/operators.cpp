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
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
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

// ------------------------------------------------------------ file cache
// The precomputation depends only on (p, ai, ao, rcond, eps_svd), so it is
// done once and kept: the paper precomputes the M2M and L2L matrices
// ("Parallelization strategies for FMM operators") and keeps its
// precomputed quantities in a database ("Data-oriented design of
// PyExaFMM").  A cache file holds, little-endian:
//   "KIFMMOPS", u32 format, u32 byte-order mark 0x01020304,
//   i32 p, f64 ai, ao, rcond, eps_svd (the key, compared bit for bit),
//   i32 ns, rP, rQ, k, then each array as i64 count + f64 values, in the
//   order of the Operators members, and last an FNV-1a 64 checksum of
//   every byte before it.
// A file that fails any check (magic, format, byte order, key, sizes,
// checksum, length) is ignored and replaced; writes go to a temporary file
// renamed into place, so readers see a whole file or none.  The cache is
// best effort: a directory that cannot be written only costs the write.

namespace {

std::mutex g_dir_mu;
std::string g_dir;   // empty: no file cache

constexpr char kMagic[8] = {'K', 'I', 'F', 'M', 'M', 'O', 'P', 'S'};
constexpr uint32_t kFormat = 1;
constexpr uint32_t kByteOrder = 0x01020304u;

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Out {
    std::vector<unsigned char> b;
    void raw(const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        b.insert(b.end(), c, c + n);
    }
    template <class T> void val(T v) { raw(&v, sizeof v); }
    void vec(const std::vector<double> &v) {
        val<int64_t>((int64_t)v.size());
        raw(v.data(), v.size() * sizeof(double));
    }
};

struct In {
    const unsigned char *p;
    size_t n, at = 0;
    bool ok = true;
    bool raw(void *dst, size_t k) {
        if (!ok || k > n - at) return ok = false;
        std::memcpy(dst, p + at, k);
        at += k;
        return true;
    }
    template <class T> T val() {
        T v{};
        raw(&v, sizeof v);
        return v;
    }
    void vec(std::vector<double> &v, size_t want) {
        const int64_t c = val<int64_t>();
        if (!ok || c < 0 || (size_t)c != want) {
            ok = false;
            return;
        }
        v.resize(want);
        raw(v.data(), want * sizeof(double));
    }
};

std::string cache_file(const std::string &dir, int p, double ai, double ao, double rcond,
                       double eps_svd) {
    const double key[4] = {ai, ao, rcond, eps_svd};
    char name[96];
    std::snprintf(name, sizeof name, "kifmm_ops_v%u_p%d_%016llx.bin", kFormat, p,
                  (unsigned long long)fnv1a(reinterpret_cast<const unsigned char *>(key),
                                            sizeof key));
    return dir + "/" + name;
}

std::vector<unsigned char> serialise(const Operators &o) {
    Out w;
    w.raw(kMagic, sizeof kMagic);
    w.val<uint32_t>(kFormat);
    w.val<uint32_t>(kByteOrder);
    w.val<int32_t>(o.p);
    w.val<double>(o.ai);
    w.val<double>(o.ao);
    w.val<double>(o.rcond);
    w.val<double>(o.eps_svd);
    w.val<int32_t>(o.ns);
    w.val<int32_t>(o.rP);
    w.val<int32_t>(o.rQ);
    w.val<int32_t>(o.k);
    for (const std::vector<double> *v : {&o.surf, &o.Pu, &o.Ps, &o.Pv, &o.Qu, &o.Qs, &o.Qv,
                                         &o.M2M, &o.L2L, &o.Uk, &o.Vk, &o.S, &o.QUk,
                                         &o.sigmaH, &o.sigmaW})
        w.vec(*v);
    w.val<uint64_t>(fnv1a(w.b.data(), w.b.size()));
    return std::move(w.b);
}

bool same_bits(double a, double b) { return std::memcmp(&a, &b, sizeof a) == 0; }

// The operators in `bytes` if they are a whole, intact file for this key.
std::shared_ptr<Operators> deserialise(const std::vector<unsigned char> &bytes, int p, double ai,
                                       double ao, double rcond, double eps_svd) {
    if (bytes.size() < sizeof(uint64_t)) return nullptr;
    const size_t body = bytes.size() - sizeof(uint64_t);
    uint64_t sum;
    std::memcpy(&sum, bytes.data() + body, sizeof sum);
    if (sum != fnv1a(bytes.data(), body)) return nullptr;
    In r{bytes.data(), body};
    char magic[8];
    r.raw(magic, sizeof magic);
    if (!r.ok || std::memcmp(magic, kMagic, sizeof magic) != 0) return nullptr;
    if (r.val<uint32_t>() != kFormat || r.val<uint32_t>() != kByteOrder) return nullptr;
    auto o = std::make_shared<Operators>();
    o->p = r.val<int32_t>();
    o->ai = r.val<double>();
    o->ao = r.val<double>();
    o->rcond = r.val<double>();
    o->eps_svd = r.val<double>();
    if (!r.ok || o->p != p || !same_bits(o->ai, ai) || !same_bits(o->ao, ao) ||
        !same_bits(o->rcond, rcond) || !same_bits(o->eps_svd, eps_svd))
        return nullptr;
    o->ns = r.val<int32_t>();
    o->rP = r.val<int32_t>();
    o->rQ = r.val<int32_t>();
    o->k = r.val<int32_t>();
    const int ns = o->ns;
    if (!r.ok || ns != 6 * (p - 1) * (p - 1) + 2 || o->rP < 1 || o->rP > ns || o->rQ < 1 ||
        o->rQ > ns || o->k < 1 || o->k > ns)
        return nullptr;
    const size_t n = (size_t)ns, rP = (size_t)o->rP, rQ = (size_t)o->rQ, k = (size_t)o->k;
    const size_t sig = eps_svd > 0 ? n : 0;
    r.vec(o->surf, 3 * n);
    r.vec(o->Pu, n * rP);
    r.vec(o->Ps, rP);
    r.vec(o->Pv, n * rP);
    r.vec(o->Qu, n * rQ);
    r.vec(o->Qs, rQ);
    r.vec(o->Qv, n * rQ);
    r.vec(o->M2M, 8 * rP * n);
    r.vec(o->L2L, 8 * rQ * n);
    r.vec(o->Uk, n * k);
    r.vec(o->Vk, n * k);
    r.vec(o->S, (size_t)kNumOffsets * k * k);
    r.vec(o->QUk, rQ * k);
    r.vec(o->sigmaH, sig);
    r.vec(o->sigmaW, sig);
    if (!r.ok || r.at != body) return nullptr;
    return o;
}

std::vector<unsigned char> read_file(const std::string &path) {
    std::vector<unsigned char> b;
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return b;
    unsigned char chunk[1 << 16];
    size_t got;
    while ((got = std::fread(chunk, 1, sizeof chunk, f)) > 0) b.insert(b.end(), chunk, chunk + got);
    std::fclose(f);
    return b;
}

void write_file_atomic(const std::string &path, const std::vector<unsigned char> &b) {
    static std::atomic<unsigned> counter{0};
    const std::string tmp = path + ".tmp." + std::to_string((long long)getpid()) + "." +
                            std::to_string(counter++);
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
    if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path.c_str()) != 0)
        std::remove(tmp.c_str());
}

} // namespace

bool set_operator_cache_dir(const char *dir) {
    std::string d = dir ? dir : "";
    if (!d.empty()) {
        struct stat st;
        if (stat(d.c_str(), &st) != 0 || !S_ISDIR(st.st_mode)) return false;
    }
    std::lock_guard<std::mutex> g(g_dir_mu);
    g_dir = d;
    return true;
}

std::shared_ptr<const Operators> get_operators(int p, double ai, double ao, double rcond,
                                               double eps_svd, int *source) {
    static std::mutex mu;
    static std::map<std::tuple<int, double, double, double, double>,
                    std::shared_ptr<const Operators>> cache;
    auto key = std::make_tuple(p, ai, ao, rcond, eps_svd);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            if (source) *source = kOpsFromMemory;
            return it->second;
        }
    }
    std::string dir;
    {
        std::lock_guard<std::mutex> g(g_dir_mu);
        dir = g_dir;
    }
    std::shared_ptr<Operators> op;
    int from = kOpsComputed;
    if (!dir.empty()) {
        const std::string path = cache_file(dir, p, ai, ao, rcond, eps_svd);
        op = deserialise(read_file(path), p, ai, ao, rcond, eps_svd);
        if (op) {
            from = kOpsFromFile;
        } else {
            op = compute(p, ai, ao, rcond, eps_svd);
            write_file_atomic(path, serialise(*op));
        }
    } else {
        op = compute(p, ai, ao, rcond, eps_svd);
    }
    if (source) *source = from;
    std::lock_guard<std::mutex> g(mu);
    cache[key] = op;
    return op;
}

} // namespace kifmm
