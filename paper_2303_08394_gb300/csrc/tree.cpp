// Linear octree, 2:1 balance and interaction lists ("The Fast Multipole
// Method": root cube split into 8 equal children until a box holds at most
// ncrit points; "Computational structure of FMM operators": U, V, W, X lists
// and the balance condition; "Data-oriented design": nodes are ids in flat
// arrays, points sorted so every box owns a contiguous range).
//
// Readings of what the paper leaves open:
//  * root: smallest cube around all points, centred on the bounding box,
//    half-width inflated by a relative 1e-6 (0.5 when all points coincide);
//  * integer coordinate of a point: floor((x - corner) / (2 hw) * 2^16)
//    clamped to [0, 2^16 - 1]; the box of level l holding it has index
//    coordinate >> (16 - l), so a point on a split plane goes upward;
//  * a split creates all 8 children, empty ones included, and the balance
//    condition is enforced over all leaves; boxes without points are then
//    dropped from every list and operator (their expansions are zero);
//  * lists, for boxes holding points ("adjacent" = closed boxes touch):
//    U(B) leaf: adjacent leaves, B included; V(B), level >= 2: children of
//    the boxes adjacent to B's parent at the parent's level (the parent
//    included) that are not adjacent to B; W(B) leaf: descendants of B's
//    adjacent same-level boxes that are not adjacent to B but whose parent
//    is; X(B) = {A : B in W(A)}.
#include <algorithm>
#include <queue>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>
#include <stdexcept>

#include "plan.h"

namespace kifmm {

namespace {

inline uint64_t spread3(uint64_t v) {  // 16 bits -> every third bit
    v &= 0xFFFF;
    v = (v | (v << 16)) & 0x0000FF0000FFULL;
    v = (v | (v << 8)) & 0x00F00F00F00FULL;
    v = (v | (v << 4)) & 0x0C30C30C30C3ULL;
    v = (v | (v << 2)) & 0x249249249249ULL;
    return v;
}
inline uint64_t morton(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}
inline uint64_t pack(int l, int x, int y, int z) {
    return ((uint64_t)l << 60) | ((uint64_t)(uint32_t)x << 40) |
           ((uint64_t)(uint32_t)y << 20) | (uint64_t)(uint32_t)z;
}

struct BNode {        // construction node (empty boxes included)
    int l, x, y, z;
    int64_t b, e;     // sorted point range
    int32_t first_child = -1;
};

// closed boxes touch or overlap
inline bool adjacent(int la, int xa, int ya, int za, int lb, int xb, int yb,
                     int zb) {
    int L = std::max(la, lb);
    int sa = L - la, sb = L - lb;
    int64_t a[3] = {xa, ya, za}, b[3] = {xb, yb, zb};
    for (int d = 0; d < 3; ++d) {
        int64_t loa = a[d] << sa, hia = (a[d] + 1) << sa;
        int64_t lob = b[d] << sb, hib = (b[d] + 1) << sb;
        if (loa > hib || lob > hia) return false;
    }
    return true;
}

} // namespace

double Tree::node_half_width(int64_t node) const {
    return std::ldexp(1.0, -key[4 * node]);
}
double Tree::node_centre(int64_t node, int d) const {
    int l = key[4 * node];
    return -1.0 + (2.0 * key[4 * node + 1 + d] + 1.0) * std::ldexp(1.0, -l);
}

void root_cube(const double lo[3], const double hi[3], double centre[3], double &hw) {
    double ext = 0;
    for (int d = 0; d < 3; ++d) {
        centre[d] = 0.5 * (lo[d] + hi[d]);
        ext = std::max(ext, hi[d] - lo[d]);
    }
    const double h = 0.5 * ext * (1.0 + 1e-6);
    hw = h > 0 ? h : 0.5;
}

void build_tree(const double *xyz, int64_t n, const TreeOptions &opt,
                Tree &t) {
    if (n < 1) throw std::runtime_error("n must be >= 1");
    if (opt.ncrit < 1) throw std::runtime_error("ncrit must be >= 1");
    if (opt.max_level < 0 || opt.max_level > kKeyBits)
        throw std::runtime_error("max_level must be in [0, 16]");
    t = Tree();
    t.n = n;
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = xyz[d];
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double v = xyz[3 * i + d];
            if (!std::isfinite(v)) throw std::runtime_error("non-finite coordinate");
            lo[d] = std::min(lo[d], v);
            hi[d] = std::max(hi[d], v);
        }
    root_cube(lo, hi, t.centre, t.hw);
    double corner[3];
    for (int d = 0; d < 3; ++d) corner[d] = t.centre[d] - t.hw;

    // integer coordinates and Morton order
    std::vector<uint32_t> ic((size_t)3 * n);
    std::vector<uint64_t> mk(n);
    const double scale = (double)(1 << kKeyBits);
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            double u = (xyz[3 * i + d] - corner[d]) / (2.0 * t.hw);
            double f = std::floor(u * scale);
            int64_t k = (int64_t)f;
            k = std::min<int64_t>(std::max<int64_t>(k, 0), (1 << kKeyBits) - 1);
            ic[3 * i + d] = (uint32_t)k;
        }
        mk[i] = morton(ic[3 * i], ic[3 * i + 1], ic[3 * i + 2]);
    }
    t.perm.resize(n);
    std::iota(t.perm.begin(), t.perm.end(), 0);
    std::stable_sort(t.perm.begin(), t.perm.end(),
                     [&](int64_t a, int64_t b) { return mk[a] < mk[b]; });
    std::vector<uint64_t> smk(n);
    for (int64_t i = 0; i < n; ++i) smk[i] = mk[t.perm[i]];

    // construction tree (all 8 children of every split box)
    std::vector<BNode> bn;
    std::unordered_map<uint64_t, int32_t> where;
    auto split = [&](int32_t id) {
        BNode nd = bn[id];
        int l = nd.l;
        int shift = 3 * (kKeyBits - l - 1);
        int32_t first = (int32_t)bn.size();
        int64_t b = nd.b;
        for (int c = 0; c < 8; ++c) {
            // points of child c: digit at this level == c
            int64_t e = b;
            if (nd.e > nd.b) {
                e = std::partition_point(smk.begin() + b, smk.begin() + nd.e,
                                         [&](uint64_t k) { return (int)((k >> shift) & 7) <= c; }) -
                    smk.begin();
            }
            BNode ch;
            ch.l = l + 1;
            ch.x = 2 * nd.x + (c & 1);
            ch.y = 2 * nd.y + ((c >> 1) & 1);
            ch.z = 2 * nd.z + ((c >> 2) & 1);
            ch.b = b;
            ch.e = e;
            b = e;
            where[pack(ch.l, ch.x, ch.y, ch.z)] = (int32_t)bn.size();
            bn.push_back(ch);
        }
        bn[id].first_child = first;
    };
    BNode root;
    root.l = root.x = root.y = root.z = 0;
    root.b = 0;
    root.e = n;
    bn.push_back(root);
    where[pack(0, 0, 0, 0)] = 0;
    for (size_t i = 0; i < bn.size(); ++i) {
        if (bn[i].e - bn[i].b > opt.ncrit && bn[i].l < opt.max_level) split((int32_t)i);
    }
    if (opt.balance) {
        // A leaf at level l must split when an internal box at level l+1
        // touches it.  After a split, the new children and the leaves one
        // level up that touch the split box are examined again.
        std::deque<int32_t> work;
        for (size_t i = 0; i < bn.size(); ++i)
            if (bn[i].first_child < 0) work.push_back((int32_t)i);
        while (!work.empty()) {
            int32_t id = work.front();
            work.pop_front();
            const BNode nd = bn[id];
            if (nd.first_child >= 0 || nd.l >= opt.max_level) continue;
            bool must = false;
            for (int a = 2 * nd.x - 1; a <= 2 * nd.x + 2 && !must; ++a)
                for (int b = 2 * nd.y - 1; b <= 2 * nd.y + 2 && !must; ++b)
                    for (int c = 2 * nd.z - 1; c <= 2 * nd.z + 2 && !must; ++c) {
                        if (a >> 1 == nd.x && b >> 1 == nd.y && c >> 1 == nd.z &&
                            a >= 0 && b >= 0 && c >= 0)
                            continue;
                        if (a < 0 || b < 0 || c < 0) continue;
                        auto it = where.find(pack(nd.l + 1, a, b, c));
                        if (it != where.end() && bn[it->second].first_child >= 0) must = true;
                    }
            if (!must) continue;
            split(id);
            int32_t first = bn[id].first_child;
            for (int c = 0; c < 8; ++c) work.push_back(first + c);
            if (nd.l >= 1) {
                int px = nd.x >> 1, py = nd.y >> 1, pz = nd.z >> 1;
                for (int a = px - 1; a <= px + 1; ++a)
                    for (int b = py - 1; b <= py + 1; ++b)
                        for (int c = pz - 1; c <= pz + 1; ++c) {
                            if (a < 0 || b < 0 || c < 0) continue;
                            auto it = where.find(pack(nd.l - 1, a, b, c));
                            if (it == where.end()) continue;
                            const BNode &m = bn[it->second];
                            if (m.first_child < 0 &&
                                adjacent(m.l, m.x, m.y, m.z, nd.l, nd.x, nd.y, nd.z))
                                work.push_back(it->second);
                        }
            }
        }
    }

    // keep boxes holding points, ordered by level then Morton key
    std::vector<int32_t> keep;
    for (size_t i = 0; i < bn.size(); ++i)
        if (bn[i].e > bn[i].b) keep.push_back((int32_t)i);
    std::sort(keep.begin(), keep.end(), [&](int32_t a, int32_t b) {
        if (bn[a].l != bn[b].l) return bn[a].l < bn[b].l;
        return morton(bn[a].x, bn[a].y, bn[a].z) < morton(bn[b].x, bn[b].y, bn[b].z);
    });
    std::vector<int32_t> newid(bn.size(), -1);
    for (size_t i = 0; i < keep.size(); ++i) newid[keep[i]] = (int32_t)i;
    const int64_t nn = (int64_t)keep.size();
    t.key.resize(4 * nn);
    t.begin.resize(nn);
    t.end.resize(nn);
    t.parent.assign(nn, -1);
    t.child.assign(8 * nn, -1);
    t.leaf.assign(nn, 0);
    t.depth = 0;
    for (int64_t i = 0; i < nn; ++i) {
        const BNode &nd = bn[keep[i]];
        t.key[4 * i] = nd.l;
        t.key[4 * i + 1] = nd.x;
        t.key[4 * i + 2] = nd.y;
        t.key[4 * i + 3] = nd.z;
        t.begin[i] = nd.b;
        t.end[i] = nd.e;
        t.depth = std::max(t.depth, nd.l);
        if (nd.first_child < 0) {
            t.leaf[i] = 1;
        } else {
            bool any = false;
            for (int c = 0; c < 8; ++c) {
                int32_t ch = newid[nd.first_child + c];
                t.child[8 * i + c] = ch;
                if (ch >= 0) {
                    t.parent[ch] = (int32_t)i;
                    any = true;
                }
            }
            if (!any) t.leaf[i] = 1;  // cannot happen for a box with points
        }
        if (t.leaf[i]) t.leaves.push_back((int32_t)i);
    }
    t.level_ptr.assign(t.depth + 2, 0);
    for (int64_t i = 0; i < nn; ++i) t.level_ptr[t.key[4 * i] + 1]++;
    for (int l = 0; l <= t.depth; ++l) t.level_ptr[l + 1] += t.level_ptr[l];

    // point positions relative to their leaf centre, in root units
    t.rel.assign((size_t)4 * n, 0.0f);
    t.rel_lo.assign((size_t)4 * n, 0.0f);
    for (int32_t lf : t.leaves) {
        double c[3];
        for (int d = 0; d < 3; ++d) c[d] = t.node_centre(lf, d);
        for (int64_t s = t.begin[lf]; s < t.end[lf]; ++s) {
            int64_t i = t.perm[s];
            for (int d = 0; d < 3; ++d)
            {
                const double v = (xyz[3 * i + d] - t.centre[d]) / t.hw - c[d];
                const float hi = (float)v;
                t.rel[4 * s + d] = hi;
                t.rel_lo[4 * s + d] = (float)(v - (double)hi);
            }
        }
    }
}

void build_lists(Tree &t) {
    const int64_t nn = t.nodes();
    std::unordered_map<uint64_t, int32_t> where;
    where.reserve(nn * 2);
    for (int64_t i = 0; i < nn; ++i)
        where[pack(t.key[4 * i], t.key[4 * i + 1], t.key[4 * i + 2], t.key[4 * i + 3])] =
            (int32_t)i;
    auto K = [&](int32_t i, int d) { return t.key[4 * i + d]; };
    auto adj = [&](int32_t a, int32_t b) {
        return adjacent(K(a, 0), K(a, 1), K(a, 2), K(a, 3), K(b, 0), K(b, 1), K(b, 2), K(b, 3));
    };
    auto lookup = [&](int l, int x, int y, int z) -> int32_t {
        if (x < 0 || y < 0 || z < 0) return -1;
        auto it = where.find(pack(l, x, y, z));
        return it == where.end() ? -1 : it->second;
    };

    std::vector<std::vector<int32_t>> U(nn), V(nn), W(nn), X(nn);
    // U: descend from the root into every box touching the leaf
    for (int32_t b : t.leaves) {
        std::vector<int32_t> stack = {0};
        while (!stack.empty()) {
            int32_t nd = stack.back();
            stack.pop_back();
            if (!adj(nd, b)) continue;
            if (t.leaf[nd]) {
                U[b].push_back(nd);
            } else {
                for (int c = 0; c < 8; ++c)
                    if (t.child[8 * nd + c] >= 0) stack.push_back(t.child[8 * nd + c]);
            }
        }
        std::sort(U[b].begin(), U[b].end());
    }
    // V: children of the parent's colleagues, not adjacent
    for (int64_t b = 0; b < nn; ++b) {
        if (K(b, 0) < 2) continue;
        int32_t par = t.parent[b];
        int pl = K(par, 0), px = K(par, 1), py = K(par, 2), pz = K(par, 3);
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c)
                for (int e = -1; e <= 1; ++e) {
                    int32_t col = lookup(pl, px + a, py + c, pz + e);
                    if (col < 0 || t.leaf[col]) continue;
                    for (int s = 0; s < 8; ++s) {
                        int32_t ch = t.child[8 * col + s];
                        if (ch >= 0 && !adj(ch, (int32_t)b)) V[b].push_back(ch);
                    }
                }
        std::sort(V[b].begin(), V[b].end());
    }
    // W (and X): descendants of the colleagues
    for (int32_t b : t.leaves) {
        int l = K(b, 0), x = K(b, 1), y = K(b, 2), z = K(b, 3);
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c)
                for (int e = -1; e <= 1; ++e) {
                    if (a == 0 && c == 0 && e == 0) continue;
                    int32_t col = lookup(l, x + a, y + c, z + e);
                    if (col < 0 || t.leaf[col]) continue;
                    std::vector<int32_t> stack;
                    for (int s = 0; s < 8; ++s)
                        if (t.child[8 * col + s] >= 0) stack.push_back(t.child[8 * col + s]);
                    while (!stack.empty()) {
                        int32_t d = stack.back();
                        stack.pop_back();
                        if (!adj(d, b)) {
                            W[b].push_back(d);
                        } else if (!t.leaf[d]) {
                            for (int s = 0; s < 8; ++s)
                                if (t.child[8 * d + s] >= 0) stack.push_back(t.child[8 * d + s]);
                        }
                    }
                }
        std::sort(W[b].begin(), W[b].end());
        for (int32_t a : W[b]) X[a].push_back(b);
    }
    for (auto &xs : X) std::sort(xs.begin(), xs.end());

    auto to_csr = [&](std::vector<std::vector<int32_t>> &L, std::vector<int64_t> &ptr,
                      std::vector<int32_t> &idx) {
        ptr.assign(nn + 1, 0);
        for (int64_t i = 0; i < nn; ++i) ptr[i + 1] = ptr[i] + (int64_t)L[i].size();
        idx.resize(ptr[nn]);
        for (int64_t i = 0; i < nn; ++i)
            std::copy(L[i].begin(), L[i].end(), idx.begin() + ptr[i]);
    };
    to_csr(U, t.u_ptr, t.u_idx);
    to_csr(V, t.v_ptr, t.v_idx);
    to_csr(W, t.w_ptr, t.w_idx);
    to_csr(X, t.x_ptr, t.x_idx);
    t.v_off.resize(t.v_idx.size());
    for (int64_t b = 0; b < nn; ++b)
        for (int64_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; ++e) {
            int32_t a = t.v_idx[e];
            int o = offset_index(K(a, 1) - K(b, 1), K(a, 2) - K(b, 2), K(a, 3) - K(b, 3));
            if (o < 0) throw std::runtime_error("internal: V entry outside the offset set");
            t.v_off[e] = (int16_t)o;
        }
    t.p2p_pairs = 0;
    for (int32_t b : t.leaves)
        for (int64_t e = t.u_ptr[b]; e < t.u_ptr[b + 1]; ++e) {
            int32_t a = t.u_idx[e];
            t.p2p_pairs += (t.end[b] - t.begin[b]) * (t.end[a] - t.begin[a]);
        }
}

void set_point_roles(Tree &t, int64_t nsrc, bool distinct) {
    t.qidx.resize(t.n);
    t.oidx.resize(t.n);
    for (int64_t s = 0; s < t.n; ++s) {
        const int64_t c = t.perm[s];
        if (!distinct) {
            t.qidx[s] = t.oidx[s] = c;
        } else {
            t.qidx[s] = c < nsrc ? c : -1;
            t.oidx[s] = c >= nsrc ? c - nsrc : -1;
        }
    }
    t.nproblems = 1;
    t.roots = {t.centre[0], t.centre[1], t.centre[2], t.hw};
    t.node_problem.assign(t.nodes(), 0);
}

void merge_forest(const std::vector<Tree> &parts, const std::vector<int64_t> &row_offset,
                  Tree &m) {
    const int np = (int)parts.size();
    if (np < 1 || (int)row_offset.size() != np)
        throw std::runtime_error("merge_forest: bad arguments");
    m = Tree();
    m.nproblems = np;
    int depth = 0;
    std::vector<int64_t> pt_base(np + 1, 0);
    for (int i = 0; i < np; ++i) {
        depth = std::max(depth, parts[i].depth);
        pt_base[i + 1] = pt_base[i] + parts[i].n;
    }
    m.depth = depth;
    m.n = pt_base[np];
    // new node ids: level-major, then problem, then the problem's order
    std::vector<std::vector<int32_t>> newid(np);
    int64_t nn = 0;
    m.level_ptr.assign(depth + 2, 0);
    for (int l = 0; l <= depth; ++l) {
        m.level_ptr[l] = (int32_t)nn;
        for (int i = 0; i < np; ++i) {
            const Tree &t = parts[i];
            if ((int)newid[i].size() != t.nodes()) newid[i].assign(t.nodes(), -1);
            if (l > t.depth) continue;
            for (int32_t b = t.level_ptr[l]; b < t.level_ptr[l + 1]; ++b) newid[i][b] = (int32_t)nn++;
        }
    }
    m.level_ptr[depth + 1] = (int32_t)nn;
    if (nn > INT32_MAX / 8) throw std::runtime_error("merge_forest: too many nodes");
    m.key.assign((size_t)4 * nn, 0);
    m.begin.assign(nn, 0);
    m.end.assign(nn, 0);
    m.parent.assign(nn, -1);
    m.child.assign((size_t)8 * nn, -1);
    m.leaf.assign(nn, 0);
    m.node_problem.assign(nn, 0);
    m.perm.resize(m.n);
    m.rel.resize((size_t)4 * m.n);
    m.rel_lo.resize((size_t)4 * m.n);
    m.qidx.resize(m.n);
    m.oidx.resize(m.n);
    for (int i = 0; i < np; ++i) {
        const Tree &t = parts[i];
        const int64_t pb = pt_base[i], ro = row_offset[i];
        m.roots.insert(m.roots.end(), {t.centre[0], t.centre[1], t.centre[2], t.hw});
        for (int64_t s = 0; s < t.n; ++s) {
            m.perm[pb + s] = pb + t.perm[s];
            m.qidx[pb + s] = t.qidx[s] >= 0 ? ro + t.qidx[s] : -1;
            m.oidx[pb + s] = t.oidx[s] >= 0 ? ro + t.oidx[s] : -1;
        }
        std::copy(t.rel.begin(), t.rel.end(), m.rel.begin() + 4 * pb);
        std::copy(t.rel_lo.begin(), t.rel_lo.end(), m.rel_lo.begin() + 4 * pb);
        const auto &id = newid[i];
        for (int64_t b = 0; b < t.nodes(); ++b) {
            const int32_t q = id[b];
            for (int d = 0; d < 4; ++d) m.key[4 * (size_t)q + d] = t.key[4 * b + d];
            m.begin[q] = pb + t.begin[b];
            m.end[q] = pb + t.end[b];
            m.parent[q] = t.parent[b] >= 0 ? id[t.parent[b]] : -1;
            for (int c = 0; c < 8; ++c) {
                const int32_t ch = t.child[8 * b + c];
                m.child[8 * (size_t)q + c] = ch >= 0 ? id[ch] : -1;
            }
            m.leaf[q] = t.leaf[b];
            m.node_problem[q] = i;
        }
        m.p2p_pairs += t.p2p_pairs;
    }
    for (int64_t q = 0; q < nn; ++q)
        if (m.leaf[q]) m.leaves.push_back((int32_t)q);
    // lists: each node keeps its own problem's list, renumbered (the map is
    // increasing within a problem, so sorted lists stay sorted)
    std::vector<int32_t> owner_problem(nn), owner_local(nn);
    for (int i = 0; i < np; ++i)
        for (int64_t b = 0; b < parts[i].nodes(); ++b) {
            owner_problem[newid[i][b]] = i;
            owner_local[newid[i][b]] = (int32_t)b;
        }
    auto merge_list = [&](std::vector<int64_t> Tree::*ptr, std::vector<int32_t> Tree::*idx,
                          std::vector<int16_t> *off) {
        std::vector<int64_t> &mp = m.*ptr;
        std::vector<int32_t> &mi = m.*idx;
        mp.assign(nn + 1, 0);
        for (int64_t q = 0; q < nn; ++q) {
            const Tree &t = parts[owner_problem[q]];
            const int32_t b = owner_local[q];
            mp[q + 1] = mp[q] + ((t.*ptr)[b + 1] - (t.*ptr)[b]);
        }
        mi.resize(mp[nn]);
        if (off) off->resize(mp[nn]);
        for (int64_t q = 0; q < nn; ++q) {
            const int i = owner_problem[q];
            const Tree &t = parts[i];
            const int32_t b = owner_local[q];
            int64_t o = mp[q];
            for (int64_t e = (t.*ptr)[b]; e < (t.*ptr)[b + 1]; ++e, ++o) {
                mi[o] = newid[i][(t.*idx)[e]];
                if (off) (*off)[o] = t.v_off[e];
            }
        }
    };
    merge_list(&Tree::u_ptr, &Tree::u_idx, nullptr);
    merge_list(&Tree::v_ptr, &Tree::v_idx, &m.v_off);
    merge_list(&Tree::w_ptr, &Tree::w_idx, nullptr);
    merge_list(&Tree::x_ptr, &Tree::x_idx, nullptr);
}

void build_m2l_table(const Tree &t, M2LTable &m) {
    m = M2LTable();
    // targets of every (level, parity class) in node order; tiles of
    // kTileRows consecutive targets of one class
    std::vector<std::vector<int32_t>> lists;
    std::vector<int> list_level;
    for (int l = 2; l <= t.depth; ++l)
        for (int cls = 0; cls < 8; ++cls) {
            std::vector<int32_t> targets;
            for (int32_t b = t.level_ptr[l]; b < t.level_ptr[l + 1]; ++b) {
                int c = (t.key[4 * b + 1] & 1) | ((t.key[4 * b + 2] & 1) << 1) |
                        ((t.key[4 * b + 3] & 1) << 2);
                if (c == cls && t.v_ptr[b + 1] > t.v_ptr[b]) targets.push_back(b);
            }
            lists.push_back(std::move(targets));
            list_level.push_back(l);
        }
    std::vector<std::pair<int, size_t>> tiles;  // (list, first target)
    for (size_t i = 0; i < lists.size(); ++i)
        for (size_t s0 = 0; s0 < lists[i].size(); s0 += kTileRows) tiles.push_back({(int)i, s0});
    const int64_t nt = (int64_t)tiles.size();
    // every tile independently: the offsets its targets use and, per offset,
    // the source of each row; then concatenated in tile order
    std::vector<std::vector<int32_t>> t_off(nt), t_src(nt);
    m.tile_level.resize(nt);
    m.tile_target.assign((size_t)nt * kTileRows, -1);
#pragma omp parallel
    {
        std::vector<int32_t> src((size_t)kNumOffsets * kTileRows, -1);
        std::vector<char> used(kNumOffsets, 0);
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < nt; ++i) {
            const std::vector<int32_t> &targets = lists[tiles[i].first];
            const size_t s0 = tiles[i].second;
            const size_t cnt = std::min<size_t>(kTileRows, targets.size() - s0);
            m.tile_level[i] = list_level[tiles[i].first];
            for (size_t r = 0; r < cnt; ++r) {
                const int32_t b = targets[s0 + r];
                m.tile_target[(size_t)i * kTileRows + r] = b;
                for (int64_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; ++e) {
                    const int o = t.v_off[e];
                    src[(size_t)o * kTileRows + r] = t.v_idx[e];
                    used[o] = 1;
                }
            }
            for (int o = 0; o < kNumOffsets; ++o) {
                if (!used[o]) continue;
                t_off[i].push_back(o);
                int32_t *row = src.data() + (size_t)o * kTileRows;
                t_src[i].insert(t_src[i].end(), row, row + kTileRows);
                std::fill(row, row + kTileRows, -1);
                used[o] = 0;
            }
        }
    }
    size_t ne = 0;
    for (int64_t i = 0; i < nt; ++i) ne += t_off[i].size();
    m.entry_offset.reserve(ne);
    m.entry_src.reserve(ne * kTileRows);
    m.tile_entry_ptr.push_back(0);
    for (int64_t i = 0; i < nt; ++i) {
        m.entry_offset.insert(m.entry_offset.end(), t_off[i].begin(), t_off[i].end());
        m.entry_src.insert(m.entry_src.end(), t_src[i].begin(), t_src[i].end());
        m.tile_entry_ptr.push_back((int32_t)m.entry_offset.size());
    }
}

void build_m2l_schedule(int ncta, M2LTable &m) {
    m.ncta = 0;
    m.cta_ptr.clear();
    m.cta_tiles.clear();
    const int nt = (int)m.tile_level.size();
    if (ncta <= 0 || nt < ncta) return;
    std::vector<int32_t> order(nt);
    for (int i = 0; i < nt; ++i) order[i] = i;
    auto cost = [&](int i) { return m.tile_entry_ptr[i + 1] - m.tile_entry_ptr[i]; };
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return cost(a) > cost(b); });
    // (load, block) min-heap: ties go to the lower block, so it is deterministic
    std::priority_queue<std::pair<int64_t, int>, std::vector<std::pair<int64_t, int>>,
                        std::greater<std::pair<int64_t, int>>>
        heap;
    for (int c = 0; c < ncta; ++c) heap.push({0, c});
    std::vector<std::vector<int32_t>> per(ncta);
    for (int i : order) {
        auto top = heap.top();
        heap.pop();
        per[top.second].push_back(i);
        // an entry is two K chunks of MMAs; a tile also pays its epilogue
        heap.push({top.first + cost(i) + 1, top.second});
    }
    m.ncta = ncta;
    m.cta_ptr.push_back(0);
    for (int c = 0; c < ncta; ++c) {
        m.cta_tiles.insert(m.cta_tiles.end(), per[c].begin(), per[c].end());
        m.cta_ptr.push_back((int32_t)m.cta_tiles.size());
    }
}

void build_m2l_windows(const Tree &t, int ncta, M2LWindows &w) {
    w = M2LWindows();
    w.ncta = std::max(1, ncta);
    std::vector<int32_t> tg;
    for (int64_t b = 0; b < t.nodes(); ++b)
        if (t.v_ptr[b + 1] > t.v_ptr[b]) tg.push_back((int32_t)b);
    const int64_t ntg = (int64_t)tg.size();
    // cost of a window: per item a fixed share (its operator tile), per
    // pair column its 16-wide share of the product
    constexpr int64_t kItemCost = kItemCols;
    auto r16 = [](int64_t n) { return (n + 15) / 16 * 16; };
    auto items = [](int64_t n) { return (n + kItemCols - 1) / kItemCols; };
    std::vector<int32_t> cnt(kNumOffsets, 0);
    std::vector<int> touched;
    auto delta = [&](int32_t b) {
        int64_t d = 0;
        for (int64_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; ++e) {
            const int64_t n = cnt[t.v_off[e]];
            d += (items(n + 1) - items(n)) * kItemCost + r16(n + 1) - r16(n);
        }
        return d;
    };
    auto add = [&](int32_t b) {
        for (int64_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; ++e) {
            const int o = t.v_off[e];
            if (cnt[o]++ == 0) touched.push_back(o);
        }
    };
    auto reset = [&]() {
        for (int o : touched) cnt[o] = 0;
        touched.clear();
    };
    // greedy cut in plan order under a cost cap (and kWinTargets boxes)
    auto greedy = [&](int64_t cap, std::vector<int32_t> *starts, std::vector<int64_t> *costs) {
        reset();
        int64_t nwin = 0, cost = 0, size = 0;
        for (int64_t i = 0; i < ntg; ++i) {
            int64_t d = delta(tg[i]);
            if (size > 0 && (size == kWinTargets || cost + d > cap)) {
                if (costs) costs->push_back(cost);
                reset();
                cost = size = 0;
                d = delta(tg[i]);
            }
            if (size == 0) {
                ++nwin;
                if (starts) starts->push_back((int32_t)i);
            }
            add(tg[i]);
            cost += d;
            ++size;
        }
        if (size > 0 && costs) costs->push_back(cost);
        reset();
        return nwin;
    };
    w.win_target_ptr.push_back(0);
    w.win_item_ptr.push_back(0);
    w.item_pair_ptr.push_back(0);
    w.cta_ptr.assign(w.ncta + 1, 0);
    if (ntg == 0) return;
    // as many windows as a whole number of rounds over the blocks needs, so
    // that every block gets the same number of windows of about equal cost
    const int64_t rounds = (ntg + (int64_t)kWinTargets * w.ncta - 1) / ((int64_t)kWinTargets * w.ncta);
    const int64_t want = std::min<int64_t>(ntg, rounds * w.ncta);
    int64_t lo = 1, hi = 1;
    while (greedy(hi, nullptr, nullptr) > want) hi *= 2;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (greedy(mid, nullptr, nullptr) <= want) hi = mid;
        else lo = mid + 1;
    }
    std::vector<int32_t> starts;
    std::vector<int64_t> costs;
    greedy(hi, &starts, &costs);
    const int64_t nwin = (int64_t)starts.size();
    starts.push_back((int32_t)ntg);
    // items: per window, per offset in increasing order, pairs in window order
    std::vector<std::vector<std::pair<int32_t, int32_t>>> bucket(kNumOffsets);
    for (int64_t wi = 0; wi < nwin; ++wi) {
        for (int32_t i = starts[wi]; i < starts[wi + 1]; ++i) {
            const int32_t b = tg[i];
            w.win_targets.push_back(b);
            for (int64_t e = t.v_ptr[b]; e < t.v_ptr[b + 1]; ++e)
                bucket[t.v_off[e]].push_back({i - starts[wi], t.v_idx[e]});
        }
        w.win_target_ptr.push_back((int32_t)w.win_targets.size());
        for (int o = 0; o < kNumOffsets; ++o) {
            std::vector<std::pair<int32_t, int32_t>> &v = bucket[o];
            for (size_t a = 0; a < v.size(); a += kItemCols) {
                const size_t z = std::min(v.size(), a + (size_t)kItemCols);
                w.item_offset.push_back(o);
                for (size_t k = a; k < z; ++k) {
                    w.pair_slot.push_back(v[k].first);
                    w.pair_src.push_back(v[k].second);
                }
                w.item_pair_ptr.push_back((int32_t)w.pair_src.size());
            }
            v.clear();
        }
        w.win_item_ptr.push_back((int32_t)w.item_offset.size());
    }
    // longest window first to the least loaded block
    std::vector<int32_t> order(nwin);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return costs[a] > costs[b]; });
    std::vector<int64_t> load(w.ncta, 0);
    std::vector<std::vector<int32_t>> per(w.ncta);
    for (int32_t wi : order) {
        const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        per[c].push_back(wi);
        load[c] += costs[wi];
    }
    for (int c = 0; c < w.ncta; ++c) {
        std::sort(per[c].begin(), per[c].end());
        w.cta_win.insert(w.cta_win.end(), per[c].begin(), per[c].end());
        w.cta_ptr[c + 1] = (int32_t)w.cta_win.size();
    }
}

void build_schedules(const Tree &t, int chunk, int direct_max, Schedules &s) {
    s = Schedules();
    for (int32_t lf : t.leaves)
        if (t.key[4 * lf] >= 2) s.p2m_nodes.push_back(lf);
    s.m2m_level_ptr.assign(t.depth + 2, 0);
    s.down_level_ptr.assign(t.depth + 2, 0);
    s.down_chunk_level_ptr.assign(t.depth + 2, 0);
    for (int l = 0; l <= t.depth; ++l) {
        s.m2m_level_ptr[l] = (int32_t)s.m2m_nodes.size();
        if (l >= 2)
            for (int32_t b = t.level_ptr[l]; b < t.level_ptr[l + 1]; ++b)
                if (!t.leaf[b]) s.m2m_nodes.push_back(b);
        s.down_level_ptr[l] = (int32_t)s.down_nodes.size();
        s.down_chunk_level_ptr[l] = (int32_t)(s.down_chunk.size() / 4);
        if (l >= 2) {
            for (int sg = 0; sg < 8; ++sg) {
                size_t start = s.down_nodes.size();
                for (int32_t b = t.level_ptr[l]; b < t.level_ptr[l + 1]; ++b) {
                    int c = (t.key[4 * b + 1] & 1) | ((t.key[4 * b + 2] & 1) << 1) |
                            ((t.key[4 * b + 3] & 1) << 2);
                    if (c == sg) s.down_nodes.push_back(b);
                }
                for (size_t p = start; p < s.down_nodes.size(); p += chunk) {
                    int cnt = (int)std::min<size_t>(chunk, s.down_nodes.size() - p);
                    s.down_chunk.push_back((int32_t)p);
                    s.down_chunk.push_back(cnt);
                    s.down_chunk.push_back(sg);
                    s.down_chunk.push_back(l);
                }
            }
        }
    }
    s.m2m_level_ptr[t.depth + 1] = (int32_t)s.m2m_nodes.size();
    s.down_level_ptr[t.depth + 1] = (int32_t)s.down_nodes.size();
    s.down_chunk_level_ptr[t.depth + 1] = (int32_t)(s.down_chunk.size() / 4);
    // The leaf pass takes the points of a W-list box directly when it is a
    // leaf of at most direct_max points, and those of a leaf's X list when
    // the leaf itself has at most direct_max points; P2L serves every other
    // box with an X list.
    s.w_direct.assign(t.nodes(), 0);
    for (int32_t lf : t.leaves)
        if (t.end[lf] - t.begin[lf] <= direct_max) s.w_direct[lf] = 1;
    s.x_slot.assign(t.nodes(), -1);
    s.x_level_count.assign(t.depth + 1, 0);
    for (int64_t b = 0; b < t.nodes(); ++b)
        if (t.x_ptr[b + 1] > t.x_ptr[b] && !(t.leaf[b] && s.w_direct[b])) {
            s.x_slot[b] = (int32_t)s.x_nodes.size();
            s.x_nodes.push_back((int32_t)b);
            ++s.x_level_count[t.key[4 * b]];
        }
}

namespace {

// Index of the first element of v outside [lo, hi), or -1.
template <class T> int64_t first_outside(const std::vector<T> &v, int64_t lo, int64_t hi) {
    int64_t bad = INT64_MAX;
#pragma omp parallel for reduction(min : bad) schedule(static)
    for (int64_t i = 0; i < (int64_t)v.size(); ++i)
        if ((int64_t)v[i] < lo || (int64_t)v[i] >= hi) bad = std::min(bad, i);
    return bad == INT64_MAX ? -1 : bad;
}

std::string outside(const char *name, int64_t i, int64_t lo, int64_t hi) {
    return std::string(name) + "[" + std::to_string(i) + "] outside [" + std::to_string(lo) +
           ", " + std::to_string(hi) + ")";
}

// CSR offsets: size rows + 1, start 0, non-decreasing, end at nidx, and
// (uploaded as int32) at most INT32_MAX.
template <class T>
std::string check_csr(const char *name, const std::vector<T> &ptr, int64_t rows, int64_t nidx) {
    if ((int64_t)ptr.size() != rows + 1) return std::string(name) + ": wrong size";
    if (ptr[0] != 0 || (int64_t)ptr[rows] != nidx)
        return std::string(name) + ": does not span its index array";
    if (nidx > INT32_MAX) return std::string(name) + ": too many entries for 32-bit offsets";
    for (int64_t i = 0; i < rows; ++i)
        if (ptr[i + 1] < ptr[i]) return std::string(name) + ": decreasing at " + std::to_string(i);
    return "";
}

} // namespace

std::string check_windows(const Tree &t, const M2LWindows &w) {
    const int64_t nn = t.nodes();
    auto csr = [](const std::vector<int32_t> &ptr, size_t count, const char *name) -> std::string {
        if (ptr.empty() || ptr.front() != 0 || (size_t)ptr.back() != count)
            return std::string(name) + ": offsets do not span their array";
        for (size_t k = 1; k < ptr.size(); ++k)
            if (ptr[k] < ptr[k - 1]) return std::string(name) + ": offsets decrease";
        return std::string();
    };
    const int64_t nwin = (int64_t)w.win_item_ptr.size() - 1;
    std::string e;
    if ((int64_t)w.win_target_ptr.size() != nwin + 1) return "m2l windows: inconsistent sizes";
    if (!(e = csr(w.win_target_ptr, w.win_targets.size(), "m2l window targets")).empty()) return e;
    if (!(e = csr(w.win_item_ptr, w.item_offset.size(), "m2l window items")).empty()) return e;
    if ((int64_t)w.item_pair_ptr.size() != (int64_t)w.item_offset.size() + 1)
        return "m2l items: inconsistent sizes";
    if (!(e = csr(w.item_pair_ptr, w.pair_src.size(), "m2l item pairs")).empty()) return e;
    if (w.pair_slot.size() != w.pair_src.size()) return "m2l pairs: inconsistent sizes";
    if ((int64_t)w.cta_ptr.size() != (int64_t)w.ncta + 1) return "m2l blocks: inconsistent sizes";
    if (!(e = csr(w.cta_ptr, w.cta_win.size(), "m2l block windows")).empty()) return e;
    for (int32_t x : w.cta_win)
        if (x < 0 || x >= nwin) return "m2l block windows: window out of range";
    for (int32_t x : w.win_targets)
        if (x < 0 || x >= nn) return "m2l window targets: node out of range";
    for (int32_t x : w.pair_src)
        if (x < 0 || x >= nn) return "m2l pairs: source out of range";
    for (int32_t x : w.item_offset)
        if (x < 0 || x >= kNumOffsets) return "m2l items: offset out of range";
    for (int64_t wi = 0; wi < nwin; ++wi) {
        const int32_t ntw = w.win_target_ptr[wi + 1] - w.win_target_ptr[wi];
        if (ntw > kWinTargets) return "m2l window: too many targets";
        for (int32_t it = w.win_item_ptr[wi]; it < w.win_item_ptr[wi + 1]; ++it) {
            const int32_t np = w.item_pair_ptr[it + 1] - w.item_pair_ptr[it];
            if (np < 1 || np > kItemCols) return "m2l item: pair count out of range";
            for (int32_t k = w.item_pair_ptr[it]; k < w.item_pair_ptr[it + 1]; ++k)
                if (w.pair_slot[k] < 0 || w.pair_slot[k] >= ntw)
                    return "m2l pairs: slot outside its window";
        }
    }
    return std::string();
}

std::string check_tables(const Tree &t, const Schedules &s, const M2LTable &m, int64_t rows) {
    const int64_t nn = t.nodes(), n = t.n;
    std::string e;
    int64_t i;
#define CHECK(expr) \
    if (!(e = (expr)).empty()) return e;
#define RANGE(vec, lo, hi) \
    if ((i = first_outside(vec, lo, hi)) >= 0) return outside(#vec, i, lo, hi);
    if (n > INT32_MAX || nn > INT32_MAX / 8) return "tree too large for 32-bit indices";
    if ((int64_t)t.begin.size() != nn || (int64_t)t.end.size() != nn ||
        (int64_t)t.child.size() != 8 * nn || (int64_t)t.key.size() != 4 * nn ||
        (int64_t)t.leaf.size() != nn || (int64_t)t.node_problem.size() != nn ||
        (int64_t)t.qidx.size() != n || (int64_t)t.oidx.size() != n ||
        (int64_t)t.rel.size() != 4 * n || (int64_t)t.rel_lo.size() != 4 * n)
        return "tree arrays of inconsistent sizes";
    RANGE(t.begin, 0, n + 1);
    RANGE(t.end, 0, n + 1);
    for (int64_t b = 0; b < nn; ++b)
        if (t.begin[b] > t.end[b]) return "node " + std::to_string(b) + ": begin > end";
    RANGE(t.parent, -1, nn);
    RANGE(t.child, -1, nn);
    RANGE(t.leaves, 0, nn);
    RANGE(t.node_problem, 0, t.nproblems);
    if ((int64_t)t.roots.size() != 4 * (int64_t)t.nproblems) return "roots: wrong size";
    RANGE(t.qidx, -1, rows);
    RANGE(t.oidx, -1, rows);
    if ((int64_t)t.level_ptr.size() != t.depth + 2 || t.level_ptr[0] != 0 ||
        t.level_ptr[t.depth + 1] != nn)
        return "level_ptr does not span the nodes";
    CHECK(check_csr("u_ptr", t.u_ptr, nn, (int64_t)t.u_idx.size()));
    CHECK(check_csr("v_ptr", t.v_ptr, nn, (int64_t)t.v_idx.size()));
    CHECK(check_csr("w_ptr", t.w_ptr, nn, (int64_t)t.w_idx.size()));
    CHECK(check_csr("x_ptr", t.x_ptr, nn, (int64_t)t.x_idx.size()));
    RANGE(t.u_idx, 0, nn);
    RANGE(t.v_idx, 0, nn);
    RANGE(t.w_idx, 0, nn);
    RANGE(t.x_idx, 0, nn);
    if (t.v_off.size() != t.v_idx.size()) return "v_off: wrong size";
    RANGE(t.v_off, 0, kNumOffsets);
    // schedules
    RANGE(s.p2m_nodes, 0, nn);
    RANGE(s.m2m_nodes, 0, nn);
    RANGE(s.down_nodes, 0, nn);
    RANGE(s.x_nodes, 0, nn);
    if ((int64_t)s.x_slot.size() != nn) return "x_slot: wrong size";
    RANGE(s.x_slot, -1, (int64_t)s.x_nodes.size());
    if ((int64_t)s.w_direct.size() != nn) return "w_direct: wrong size";
    RANGE(s.w_direct, 0, 2);
    CHECK(check_csr("m2m_level_ptr", s.m2m_level_ptr, t.depth + 1, (int64_t)s.m2m_nodes.size()));
    CHECK(check_csr("down_level_ptr", s.down_level_ptr, t.depth + 1,
                    (int64_t)s.down_nodes.size()));
    if (s.down_chunk.size() % 4 != 0) return "down_chunk: not whole chunks";
    CHECK(check_csr("down_chunk_level_ptr", s.down_chunk_level_ptr, t.depth + 1,
                    (int64_t)s.down_chunk.size() / 4));
    for (size_t c = 0; c < s.down_chunk.size(); c += 4) {
        const int64_t start = s.down_chunk[c], cnt = s.down_chunk[c + 1];
        if (start < 0 || cnt < 1 || start + cnt > (int64_t)s.down_nodes.size() ||
            s.down_chunk[c + 2] < 0 || s.down_chunk[c + 2] > 7 || s.down_chunk[c + 3] < 0 ||
            s.down_chunk[c + 3] > t.depth)
            return "down_chunk " + std::to_string(c / 4) + ": out of range";
    }
    // M2L work table
    const int64_t nt = (int64_t)m.tile_level.size();
    if ((int64_t)m.tile_target.size() != nt * kTileRows) return "tile_target: wrong size";
    CHECK(check_csr("tile_entry_ptr", m.tile_entry_ptr, nt, (int64_t)m.entry_offset.size()));
    if (m.entry_src.size() != m.entry_offset.size() * kTileRows) return "entry_src: wrong size";
    RANGE(m.tile_level, 2, t.depth + 1);
    RANGE(m.tile_target, -1, nn);
    RANGE(m.entry_offset, 0, kNumOffsets);
    RANGE(m.entry_src, -1, nn);
    if (m.ncta > 0) {
        // the block schedule: every tile exactly once
        CHECK(check_csr("m2l cta_ptr", m.cta_ptr, m.ncta, (int64_t)m.cta_tiles.size()));
        if ((int64_t)m.cta_tiles.size() != nt) return "m2l cta_tiles: wrong size";
        RANGE(m.cta_tiles, 0, nt);
        std::vector<char> seen(nt, 0);
        for (int32_t i : m.cta_tiles)
            if (seen[i]++) return "m2l cta_tiles: tile " + std::to_string(i) + " twice";
    }
#undef RANGE
#undef CHECK
    return "";
}

} // namespace kifmm
