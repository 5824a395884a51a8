// Level-synchronous plan build: the octree, its 2:1 balance and the U, V, W,
// X lists from whole-level passes ("The Fast Multipole Method": the root cube
// is split into 8 children until a box holds at most ncrit points;
// "Computational structure of FMM operators": the four lists and the balance
// condition; "Data-oriented design": flat arrays, points sorted so that every
// box owns a contiguous range).
//
// The same step sequence runs on the device (element-wise kernels, CUB radix
// sorts and prefix sums) or on the host (the same element functions in
// OpenMP loops, std sorts).  Both give the arrays of the recursive builder
// (build_tree + build_lists) bit for bit: the sort is stable on the same
// Morton keys, the FP64 arithmetic is the same sequence of correctly rounded
// operations, and every list is sorted by node index.
//
// Split sets.  S0_l = boxes of level l < max_level holding more than ncrit
// points, the boxes the plain construction splits.  With the balance
// condition the split set of level l is
//     S_l = S0_l  u  { B of level l : B touches some D in S_{l+1} },
// taken from the deepest level upward.  A box this adds must split in every
// 2:1-balanced refinement (left a leaf, it would touch a box two levels
// finer: a child of D), and the sets are balanced by construction, so they
// are the least balanced refinement, the one the worklist builder reaches.
// The boxes of level l+1 are the 8 children of every box in S_l; those
// holding points are the nodes, and a node is a leaf when it is not in S_l.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "plan.h"

namespace kifmm {
namespace {

#define HD __host__ __device__

constexpr int kStack = 128;  // DFS stack: 8 + 7 per level below the start

HD inline uint64_t spread(uint64_t v) {  // 16 bits -> every third bit
    v &= 0xFFFF;
    v = (v | (v << 16)) & 0x0000FF0000FFULL;
    v = (v | (v << 8)) & 0x00F00F00F00FULL;
    v = (v | (v << 4)) & 0x0C30C30C30C3ULL;
    v = (v | (v << 2)) & 0x249249249249ULL;
    return v;
}
HD inline uint32_t compact(uint64_t v) {  // every third bit -> 16 bits
    v &= 0x249249249249ULL;
    v = (v | (v >> 2)) & 0x0C30C30C30C3ULL;
    v = (v | (v >> 4)) & 0x00F00F00F00FULL;
    v = (v | (v >> 8)) & 0x0000FF0000FFULL;
    v = (v | (v >> 16)) & 0xFFFFULL;
    return (uint32_t)v;
}
HD inline uint64_t morton(uint32_t x, uint32_t y, uint32_t z) {
    return spread(x) | (spread(y) << 1) | (spread(z) << 2);
}
HD inline int64_t lower_bound(const uint64_t *a, int64_t lo, int64_t hi, uint64_t v) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        if (a[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}
HD inline bool contains(const uint64_t *a, int64_t lo, int64_t hi, uint64_t v) {
    const int64_t i = lower_bound(a, lo, hi, v);
    return i < hi && a[i] == v;
}
// closed boxes (level, integer coordinates) touch or overlap
HD inline bool touch(int la, int xa, int ya, int za, int lb, int xb, int yb, int zb) {
    const int L = la > lb ? la : lb;
    const int sa = L - la, sb = L - lb;
    const int64_t a[3] = {xa, ya, za}, b[3] = {xb, yb, zb};
    for (int d = 0; d < 3; ++d) {
        const int64_t loa = a[d] << sa, hia = (a[d] + 1) << sa;
        const int64_t lob = b[d] << sb, hib = (b[d] + 1) << sb;
        if (loa > hib || lob > hia) return false;
    }
    return true;
}
// offset t in {-3..3}^3 without {-1..1}^3 -> 0..315, lexicographic with tz
// fastest; -1 outside that set
HD inline int offset_slot(int tx, int ty, int tz) {
    if (tx < -3 || tx > 3 || ty < -3 || ty > 3 || tz < -3 || tz > 3) return -1;
    if (tx >= -1 && tx <= 1 && ty >= -1 && ty <= 1 && tz >= -1 && tz <= 1) return -1;
    const int lin = (tx + 3) * 49 + (ty + 3) * 7 + (tz + 3);
    int inner = 0;  // near offsets that come earlier in the same order
    for (int a = 2; a <= 4; ++a)
        for (int b = 2; b <= 4; ++b)
            for (int c = 2; c <= 4; ++c) inner += (a * 49 + b * 7 + c) < lin;
    return lin - inner;
}
// 2^-l, exactly
HD inline double pow2m(int l) {
    double s = 1.0;
    for (int i = 0; i < l; ++i) s *= 0.5;
    return s;
}

struct Levels {
    int32_t p[kKeyBits + 2];
};

// Read-only view of the finished node arrays (nodes ordered by level, then
// level Morton key).
struct NodeView {
    const uint64_t *mk;     // Morton key of the box at its own level
    const int32_t *lvl;
    const int32_t *child;   // 8 per node, -1 absent
    const uint8_t *leaf;
    Levels lp;              // first node of each level
    int depth;

    HD int32_t find(int l, int x, int y, int z) const {
        if (l > depth) return -1;
        const int side = 1 << l;
        if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
        const uint64_t k = morton((uint32_t)x, (uint32_t)y, (uint32_t)z);
        const int64_t i = lower_bound(mk, lp.p[l], lp.p[l + 1], k);
        return (i < lp.p[l + 1] && mk[i] == k) ? (int32_t)i : -1;
    }
    HD void coords(int32_t i, int &l, int &x, int &y, int &z) const {
        l = lvl[i];
        x = (int)compact(mk[i]);
        y = (int)compact(mk[i] >> 1);
        z = (int)compact(mk[i] >> 2);
    }
    HD bool touches(int32_t a, int lb, int xb, int yb, int zb) const {
        int l, x, y, z;
        coords(a, l, x, y, z);
        return touch(l, x, y, z, lb, xb, yb, zb);
    }
};

template <bool FILL>
struct Emit {
    int32_t *out;
    int64_t pos;
    HD void operator()(int32_t v) {
        if (FILL) out[pos] = v;
        ++pos;
    }
};

// ---------------------------------------------------------------- functors

struct FKeys {  // integer coordinates -> Morton key; payload = input index
    const double *x;
    double c0, c1, c2, two_hw;
    uint64_t *key;
    uint32_t *idx;
    HD void operator()(int64_t i) const {
        const double corner[3] = {c0, c1, c2};
        uint32_t ic[3];
        for (int d = 0; d < 3; ++d) {
            const double u = (x[3 * i + d] - corner[d]) / two_hw;
            const double f = floor(u * (double)(1 << kKeyBits));
            int64_t k = (int64_t)f;
            k = k < 0 ? 0 : (k > (1 << kKeyBits) - 1 ? (1 << kKeyBits) - 1 : k);
            ic[d] = (uint32_t)k;
        }
        key[i] = morton(ic[0], ic[1], ic[2]);
        idx[i] = (uint32_t)i;
    }
};

// children of the boxes par[] (level lc - 1): key, point range, and a flag:
// split-worthy (mode 0: more than ncrit points below max_level) or
// non-empty (mode 1)
struct FChildren {
    const uint64_t *par;
    int lc, mode, ncrit, max_level;
    const uint64_t *smk;
    int64_t n;
    uint64_t *ck;
    int64_t *b, *e, *flag;
    HD void operator()(int64_t i) const {
        const uint64_t c = par[i >> 3] * 8 + (uint64_t)(i & 7);
        const int shift = 3 * (kKeyBits - lc);
        const int64_t lo = lower_bound(smk, 0, n, c << shift);
        const int64_t hi = lower_bound(smk, lo, n, (c + 1) << shift);
        ck[i] = c;
        if (b) {
            b[i] = lo;
            e[i] = hi;
        }
        flag[i] = mode == 0 ? (hi - lo > ncrit && lc < max_level) : (hi > lo);
    }
};

// the boxes of level l touching box d[i >> 3] of level l + 1: two
// candidates per axis
struct FTouch {
    const uint64_t *d;
    int l;
    uint64_t *out;
    int64_t *flag;
    HD void operator()(int64_t i) const {
        const uint64_t k = d[i >> 3];
        const int j = (int)(i & 7);
        const int c[3] = {(int)compact(k), (int)compact(k >> 1), (int)compact(k >> 2)};
        int b[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            const int lo = c[a] >= 1 ? (c[a] - 1) / 2 : -1;
            b[a] = lo + ((j >> a) & 1);
            ok = ok && b[a] >= 0 && b[a] < (1 << l);
        }
        out[i] = ok ? morton((uint32_t)b[0], (uint32_t)b[1], (uint32_t)b[2]) : 0;
        flag[i] = ok;
    }
};

struct FUniqueFlag {  // first of every run of equal sorted keys
    const uint64_t *k;
    int64_t *flag;
    HD void operator()(int64_t i) const { flag[i] = i == 0 || k[i] != k[i - 1]; }
};

template <class T>
struct FScatter {  // out[pos[i]] = in[i] where flag[i]
    const T *in;
    const int64_t *flag, *pos;
    T *out;
    HD void operator()(int64_t i) const {
        if (flag[i]) out[pos[i]] = in[i];
    }
};

// new nodes of one level from the compacted candidates
struct FPlaceNodes {
    const uint64_t *ck;
    const int64_t *b, *e, *flag, *pos;
    int32_t first, l;
    uint64_t *mk;
    int32_t *lvl;
    int64_t *nb, *ne;
    HD void operator()(int64_t i) const {
        if (!flag[i]) return;
        const int64_t j = first + pos[i];
        mk[j] = ck[i];
        lvl[j] = l;
        nb[j] = b[i];
        ne[j] = e[i];
    }
};

// parent, child slot, leaf flag and (level, x, y, z) of every node
struct FLink {
    NodeView t;
    const uint64_t *sk;  // split sets, level-concatenated
    Levels sp;
    int nsplit_levels;
    int32_t *parent, *child, *key4;
    uint8_t *leaf;
    HD void operator()(int64_t j) const {
        int l, x, y, z;
        t.coords((int32_t)j, l, x, y, z);
        key4[4 * j] = l;
        key4[4 * j + 1] = x;
        key4[4 * j + 2] = y;
        key4[4 * j + 3] = z;
        const bool split = l < nsplit_levels && contains(sk, sp.p[l], sp.p[l + 1], t.mk[j]);
        leaf[j] = split ? 0 : 1;
        if (l == 0) {
            parent[j] = -1;
            return;
        }
        const int32_t p = t.find(l - 1, x >> 1, y >> 1, z >> 1);  // holds points too
        parent[j] = p;
        if (p >= 0) child[8 * (int64_t)p + (int)(t.mk[j] & 7)] = (int32_t)j;
    }
};

struct FLeafFlag {
    const uint8_t *leaf;
    int64_t *flag;
    HD void operator()(int64_t j) const { flag[j] = leaf[j]; }
};

struct FLeafIds {
    const int64_t *flag, *pos;
    int32_t *leaves;
    HD void operator()(int64_t j) const {
        if (flag[j]) leaves[pos[j]] = (int32_t)j;
    }
};

// positions relative to the leaf centre in root units, with the residual
struct FRel {
    NodeView t;
    const int32_t *leaves;
    const int64_t *nb, *ne;
    const uint32_t *perm;
    const double *x;
    double c0, c1, c2, hw;
    float *rel, *rel_lo;
    HD void operator()(int64_t i) const {
        const int32_t lf = leaves[i];
        int l, k[3];
        t.coords(lf, l, k[0], k[1], k[2]);
        const double centre[3] = {c0, c1, c2};
        const double h = pow2m(l);
        double c[3];
        for (int d = 0; d < 3; ++d) c[d] = -1.0 + (2.0 * k[d] + 1.0) * h;
        for (int64_t s = nb[lf]; s < ne[lf]; ++s) {
            const int64_t p = perm[s];
            for (int d = 0; d < 3; ++d) {
                const double v = (x[3 * p + d] - centre[d]) / hw - c[d];
                const float hi = (float)v;
                rel[4 * s + d] = hi;
                rel_lo[4 * s + d] = (float)(v - (double)hi);
            }
            rel[4 * s + 3] = 0.0f;
            rel_lo[4 * s + 3] = 0.0f;
        }
    }
};

struct FWiden {
    const uint32_t *in;
    int64_t *out;
    HD void operator()(int64_t i) const { out[i] = in[i]; }
};

// U(b), b a leaf: every leaf touching b, b included.  A touching leaf at b's
// level or coarser is the deepest node holding one of the 26 neighbour
// positions of b's level; a finer one lies below a same-level neighbour and
// is reached by descending through the boxes that touch b.
template <bool FILL>
struct FListU {
    NodeView t;
    const int32_t *leaves;
    const int64_t *ptr;
    int32_t *idx;
    int64_t *cnt;
    HD void operator()(int64_t i) const {
        const int32_t b = leaves[i];
        int l, x, y, z;
        t.coords(b, l, x, y, z);
        Emit<FILL> em{idx, FILL ? ptr[b] : 0};
        int32_t coarse[26];
        int nc = 0;
        int32_t stack[kStack];
        const int side = 1 << l;
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c)
                for (int e = -1; e <= 1; ++e) {
                    if (a == 0 && c == 0 && e == 0) {
                        em(b);
                        continue;
                    }
                    const int X = x + a, Y = y + c, Z = z + e;
                    if (X < 0 || Y < 0 || Z < 0 || X >= side || Y >= side || Z >= side) continue;
                    int lev = l;
                    int32_t nd = -1;
                    for (; lev >= 0; --lev) {
                        nd = t.find(lev, X >> (l - lev), Y >> (l - lev), Z >> (l - lev));
                        if (nd >= 0) break;
                    }
                    if (nd < 0) continue;
                    if (lev < l) {  // a coarser leaf, or empty space under an internal box
                        if (!t.leaf[nd]) continue;
                        bool seen = false;
                        for (int k = 0; k < nc; ++k) seen = seen || coarse[k] == nd;
                        if (!seen) {
                            coarse[nc++] = nd;
                            em(nd);
                        }
                        continue;
                    }
                    if (t.leaf[nd]) {
                        em(nd);
                        continue;
                    }
                    int sp = 0;
                    stack[sp++] = nd;
                    while (sp > 0) {
                        const int32_t d = stack[--sp];
                        for (int s = 0; s < 8; ++s) {
                            const int32_t ch = t.child[8 * (int64_t)d + s];
                            if (ch < 0 || !t.touches(ch, l, x, y, z)) continue;
                            if (t.leaf[ch]) em(ch);
                            else if (sp < kStack) stack[sp++] = ch;
                        }
                    }
                }
        if (!FILL) cnt[b] = em.pos;
    }
};

// V(b), level >= 2: children of the boxes touching b's parent at the
// parent's level (the parent included) that do not touch b
template <bool FILL>
struct FListV {
    NodeView t;
    const int32_t *parent;
    int32_t first;
    const int64_t *ptr;
    int32_t *idx;
    int64_t *cnt;
    HD void operator()(int64_t i) const {
        const int32_t b = first + (int32_t)i;
        int l, x, y, z, pl, px, py, pz;
        t.coords(b, l, x, y, z);
        t.coords(parent[b], pl, px, py, pz);
        Emit<FILL> em{idx, FILL ? ptr[b] : 0};
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c)
                for (int e = -1; e <= 1; ++e) {
                    const int32_t col = t.find(pl, px + a, py + c, pz + e);
                    if (col < 0 || t.leaf[col]) continue;
                    for (int s = 0; s < 8; ++s) {
                        const int32_t ch = t.child[8 * (int64_t)col + s];
                        if (ch >= 0 && !t.touches(ch, l, x, y, z)) em(ch);
                    }
                }
        if (!FILL) cnt[b] = em.pos;
    }
};

// W(b), b a leaf: descendants of b's same-level neighbours that do not touch
// b while their parent does
template <bool FILL>
struct FListW {
    NodeView t;
    const int32_t *leaves;
    const int64_t *ptr;
    int32_t *idx;
    int64_t *cnt;
    HD void operator()(int64_t i) const {
        const int32_t b = leaves[i];
        int l, x, y, z;
        t.coords(b, l, x, y, z);
        Emit<FILL> em{idx, FILL ? ptr[b] : 0};
        int32_t stack[kStack];
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c)
                for (int e = -1; e <= 1; ++e) {
                    if (a == 0 && c == 0 && e == 0) continue;
                    const int32_t col = t.find(l, x + a, y + c, z + e);
                    if (col < 0 || t.leaf[col]) continue;
                    int sp = 0;
                    for (int s = 0; s < 8; ++s) {
                        const int32_t ch = t.child[8 * (int64_t)col + s];
                        if (ch >= 0) stack[sp++] = ch;
                    }
                    while (sp > 0) {
                        const int32_t d = stack[--sp];
                        if (!t.touches(d, l, x, y, z)) {
                            em(d);
                        } else if (!t.leaf[d]) {
                            for (int s = 0; s < 8; ++s) {
                                const int32_t ch = t.child[8 * (int64_t)d + s];
                                if (ch >= 0 && sp < kStack) stack[sp++] = ch;
                            }
                        }
                    }
                }
        if (!FILL) cnt[b] = em.pos;
    }
};

struct FXPairs {  // (a, b) for every a in W(b), as a << 32 | b
    const int32_t *leaves;
    const int64_t *wptr;
    const int32_t *widx;
    uint64_t *key;
    HD void operator()(int64_t i) const {
        const int32_t b = leaves[i];
        for (int64_t e = wptr[b]; e < wptr[b + 1]; ++e)
            key[e] = ((uint64_t)(uint32_t)widx[e] << 32) | (uint32_t)b;
    }
};

struct FXPtr {
    const uint64_t *key;
    int64_t m;
    int64_t *xptr;
    HD void operator()(int64_t a) const { xptr[a] = lower_bound(key, 0, m, (uint64_t)a << 32); }
};

struct FXIdx {
    const uint64_t *key;
    int32_t *xidx;
    HD void operator()(int64_t e) const { xidx[e] = (int32_t)(uint32_t)(key[e] & 0xFFFFFFFFULL); }
};

struct FVOff {
    NodeView t;
    int32_t first;
    const int64_t *vptr;
    const int32_t *vidx;
    int16_t *voff;
    int *bad;
    HD void operator()(int64_t i) const {
        const int32_t b = first + (int32_t)i;
        int l, x, y, z;
        t.coords(b, l, x, y, z);
        for (int64_t e = vptr[b]; e < vptr[b + 1]; ++e) {
            int la, xa, ya, za;
            t.coords(vidx[e], la, xa, ya, za);
            const int o = offset_slot(xa - x, ya - y, za - z);
            voff[e] = (int16_t)o;
            if (o < 0) *bad = 1;
        }
    }
};

struct FP2P {  // near-field pairs of leaf b: |b| * sum over U(b) of |a|
    const int32_t *leaves;
    const int64_t *nb, *ne, *uptr;
    const int32_t *uidx;
    int64_t *val;
    HD void operator()(int64_t i) const {
        const int32_t b = leaves[i];
        int64_t s = 0;
        for (int64_t e = uptr[b]; e < uptr[b + 1]; ++e) s += ne[uidx[e]] - nb[uidx[e]];
        val[b] = s * (ne[b] - nb[b]);
    }
};

// ---------------------------------------------------------------- backends

template <class F>
__global__ void k_for_each(int64_t n, F f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f(i);
}

__global__ void k_bbox(const double *x, int64_t n3, double *part, int *bad) {
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
    }
    int nf = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 3 * i < n3;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const double v = x[3 * i + d];
            if (!isfinite(v)) nf = 1;
            else {
                lo[d] = fmin(lo[d], v);
                hi[d] = fmax(hi[d], v);
            }
        }
    __shared__ double red[6][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            red[d][w] = lo[d];
            red[3 + d][w] = hi[d];
        }
    if (__any_sync(0xffffffffu, nf) && lane == 0) atomicOr(bad, 1);
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = red[threadIdx.x][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            v = threadIdx.x < 3 ? fmin(v, red[threadIdx.x][k]) : fmax(v, red[threadIdx.x][k]);
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

// every segment of idx sorted ascending: a warp per segment ranks its
// entries in shared memory (entries are distinct node ids); longer segments
// fall back to an insertion sort by one lane
__global__ void k_sort_segments(const int64_t *ptr, int32_t *idx, int64_t nseg) {
    constexpr int kCap = 512, kW = 4;
    __shared__ int32_t buf[kW][kCap];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t g = blockIdx.x * (int64_t)kW + w; g < nseg; g += (int64_t)gridDim.x * kW) {
        const int64_t b = ptr[g], n = ptr[g + 1] - b;
        if (n <= 1) continue;
        if (n <= kCap) {
            for (int j = lane; j < n; j += 32) buf[w][j] = idx[b + j];
            __syncwarp();
            for (int j = lane; j < n; j += 32) {
                const int32_t v = buf[w][j];
                int r = 0;
                for (int k = 0; k < n; ++k) r += buf[w][k] < v;
                idx[b + r] = v;
            }
            __syncwarp();
        } else if (lane == 0) {
            for (int64_t j = 1; j < n; ++j) {
                const int32_t v = idx[b + j];
                int64_t k = j;
                for (; k > 0 && idx[b + k - 1] > v; --k) idx[b + k] = idx[b + k - 1];
                idx[b + k] = v;
            }
        }
        __syncwarp();
    }
}

void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess)
        throw CudaFailure((int)e, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceBackend {
    cudaStream_t s = nullptr;
    std::vector<void *> owned;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;

    DeviceBackend() { cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream"); }
    ~DeviceBackend() {
        if (s) cudaStreamSynchronize(s);
        for (void *p : owned) cudaFree(p);
        if (tmp) cudaFree(tmp);
        if (s) cudaStreamDestroy(s);
    }
    template <class T>
    T *alloc(int64_t n) {
        void *p = nullptr;
        cuda_check(cudaMalloc(&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T)), "cudaMalloc");
        owned.push_back(p);
        return (T *)p;
    }
    void *scratch(size_t bytes) {
        if (bytes > tmp_bytes) {
            if (tmp) cuda_check(cudaFree(tmp), "cudaFree");
            tmp = nullptr;
            cuda_check(cudaMalloc(&tmp, bytes), "cudaMalloc");
            tmp_bytes = bytes;
        }
        return tmp;
    }
    template <class F>
    void run(int64_t n, const F &f) {
        if (n <= 0) return;
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 32);
        k_for_each<F><<<(unsigned)blocks, 256, 0, s>>>(n, f);
        cuda_check(cudaGetLastError(), "launch");
    }
    void fill(void *p, int byte, size_t bytes) {
        cuda_check(cudaMemsetAsync(p, byte, bytes, s), "memset");
    }
    void put(void *dst, const void *src, size_t bytes) {
        cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s), "copy");
    }
    template <class T>
    T get(const T *p, int64_t i) {
        T v;
        cuda_check(cudaMemcpyAsync(&v, p + i, sizeof(T), cudaMemcpyDeviceToHost, s), "copy");
        cuda_check(cudaStreamSynchronize(s), "sync");
        return v;
    }
    template <class T>
    void to_host(const T *p, int64_t n, T *dst) {
        if (n > 0)
            cuda_check(cudaMemcpyAsync(dst, p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, s),
                       "copy");
    }
    void sync() { cuda_check(cudaStreamSynchronize(s), "sync"); }
    // stable sort of (key, value) by the key bits [0, end_bit); results in
    // place of the inputs
    void sort_pairs(uint64_t *&k, uint32_t *&v, int64_t n, int end_bit) {
        if (n <= 1 || end_bit <= 0) return;
        uint64_t *k2 = alloc<uint64_t>(n);
        uint32_t *v2 = alloc<uint32_t>(n);
        size_t bytes = 0;
        cuda_check(cub::DeviceRadixSort::SortPairs(nullptr, bytes, k, k2, v, v2, n, 0, end_bit, s),
                   "sort");
        void *t = scratch(bytes);
        cuda_check(cub::DeviceRadixSort::SortPairs(t, bytes, k, k2, v, v2, n, 0, end_bit, s), "sort");
        k = k2;
        v = v2;
    }
    void sort_keys(uint64_t *&k, int64_t n, int end_bit) {
        if (n <= 1 || end_bit <= 0) return;
        uint64_t *k2 = alloc<uint64_t>(n);
        size_t bytes = 0;
        cuda_check(cub::DeviceRadixSort::SortKeys(nullptr, bytes, k, k2, n, 0, end_bit, s), "sort");
        void *t = scratch(bytes);
        cuda_check(cub::DeviceRadixSort::SortKeys(t, bytes, k, k2, n, 0, end_bit, s), "sort");
        k = k2;
    }
    void scan(const int64_t *in, int64_t *out, int64_t n) {
        if (n <= 0) return;
        size_t bytes = 0;
        cuda_check(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, s), "scan");
        void *t = scratch(bytes);
        cuda_check(cub::DeviceScan::ExclusiveSum(t, bytes, in, out, n, s), "scan");
    }
    void bbox(const double *x, int64_t n, double lo[3], double hi[3], bool &bad) {
        const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
        double *part = alloc<double>(6 * blocks);
        int *flag = alloc<int>(1);
        fill(flag, 0, sizeof(int));
        k_bbox<<<blocks, 256, 0, s>>>(x, 3 * n, part, flag);
        cuda_check(cudaGetLastError(), "launch");
        std::vector<double> h(6 * blocks);
        to_host(part, 6 * blocks, h.data());
        int f = get(flag, 0);
        bad = f != 0;
        for (int d = 0; d < 3; ++d) {
            lo[d] = h[d];
            hi[d] = h[3 + d];
            for (int b = 1; b < blocks; ++b) {
                lo[d] = std::min(lo[d], h[6 * b + d]);
                hi[d] = std::max(hi[d], h[6 * b + 3 + d]);
            }
        }
    }
    void sort_segments(const int64_t *ptr, int32_t *idx, int64_t nseg) {
        if (nseg <= 0) return;
        const int64_t blocks = std::min<int64_t>((nseg + 3) / 4, 152 * 16);
        k_sort_segments<<<(unsigned)blocks, 128, 0, s>>>(ptr, idx, nseg);
        cuda_check(cudaGetLastError(), "launch");
    }
};

struct HostBackend {
    std::vector<void *> owned;
    ~HostBackend() {
        for (void *p : owned) std::free(p);
    }
    template <class T>
    T *alloc(int64_t n) {
        void *p = std::malloc((size_t)std::max<int64_t>(n, 1) * sizeof(T));
        if (!p) throw std::bad_alloc();
        owned.push_back(p);
        return (T *)p;
    }
    template <class F>
    void run(int64_t n, const F &f) {
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) f(i);
    }
    void fill(void *p, int byte, size_t bytes) { std::memset(p, byte, bytes); }
    void put(void *dst, const void *src, size_t bytes) { std::memcpy(dst, src, bytes); }
    template <class T>
    T get(const T *p, int64_t i) { return p[i]; }
    template <class T>
    void to_host(const T *p, int64_t n, T *dst) {
        if (n > 0) std::memcpy(dst, p, (size_t)n * sizeof(T));
    }
    void sync() {}
    void sort_pairs(uint64_t *&k, uint32_t *&v, int64_t n, int end_bit) {
        if (n <= 1 || end_bit <= 0) return;
        const uint64_t mask = end_bit >= 64 ? ~0ULL : ((1ULL << end_bit) - 1);
        std::vector<int64_t> o(n);
        std::iota(o.begin(), o.end(), 0);
        std::stable_sort(o.begin(), o.end(),
                         [&](int64_t a, int64_t b) { return (k[a] & mask) < (k[b] & mask); });
        uint64_t *k2 = alloc<uint64_t>(n);
        uint32_t *v2 = alloc<uint32_t>(n);
        for (int64_t i = 0; i < n; ++i) {
            k2[i] = k[o[i]];
            v2[i] = v[o[i]];
        }
        k = k2;
        v = v2;
    }
    void sort_keys(uint64_t *&k, int64_t n, int end_bit) {
        if (n <= 1 || end_bit <= 0) return;
        std::sort(k, k + n);
    }
    void scan(const int64_t *in, int64_t *out, int64_t n) {
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t v = in[i];
            out[i] = s;
            s += v;
        }
    }
    void bbox(const double *x, int64_t n, double lo[3], double hi[3], bool &bad) {
        bad = false;
        for (int d = 0; d < 3; ++d) lo[d] = hi[d] = x[d];
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                const double v = x[3 * i + d];
                if (!std::isfinite(v)) bad = true;
                lo[d] = std::min(lo[d], v);
                hi[d] = std::max(hi[d], v);
            }
    }
    void sort_segments(const int64_t *ptr, int32_t *idx, int64_t nseg) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t g = 0; g < nseg; ++g) std::sort(idx + ptr[g], idx + ptr[g + 1]);
    }
};

// ---------------------------------------------------------------- driver

// Compact the flagged entries of in[0, m) (flags as 0/1 int64) into a new
// array; returns it and sets count.
template <class B, class T>
T *keep_flagged(B &be, const T *in, const int64_t *flag, int64_t m, int64_t &count) {
    count = 0;
    if (m <= 0) return be.template alloc<T>(1);
    int64_t *pos = be.template alloc<int64_t>(m);
    be.scan(flag, pos, m);
    count = be.get(pos, m - 1) + be.get(flag, m - 1);
    T *out = be.template alloc<T>(count);
    be.run(m, FScatter<T>{in, flag, pos, out});
    return out;
}

struct LevelSet {
    uint64_t *k = nullptr;  // sorted level Morton keys
    int64_t n = 0;
};

// CSR list of one kind: count pass, prefix sum, fill pass, per-node sort
template <class B, template <bool> class F, class Make>
void list_csr(B &be, int64_t nn, int64_t nitems, Make make, std::vector<int64_t> &ptr_h,
              std::vector<int32_t> &idx_h, int64_t **ptr_d = nullptr, int32_t **idx_d = nullptr) {
    int64_t *cnt = be.template alloc<int64_t>(nn + 1);
    be.fill(cnt, 0, (size_t)(nn + 1) * sizeof(int64_t));
    be.run(nitems, make(F<false>{}, nullptr, nullptr, cnt));
    int64_t *ptr = be.template alloc<int64_t>(nn + 1);
    be.scan(cnt, ptr, nn + 1);
    const int64_t total = be.get(ptr, nn);
    int32_t *idx = be.template alloc<int32_t>(total);
    be.run(nitems, make(F<true>{}, ptr, idx, nullptr));
    be.sort_segments(ptr, idx, nn);
    ptr_h.resize(nn + 1);
    idx_h.resize(total);
    be.to_host(ptr, nn + 1, ptr_h.data());
    be.to_host(idx, total, idx_h.data());
    if (ptr_d) *ptr_d = ptr;
    if (idx_d) *idx_d = idx;
}

template <class B>
void build(B &be, const double *xs, const double *xt, int64_t n, const TreeOptions &opt,
           Tree &t) {
    if (n < 1) throw std::runtime_error("n must be >= 1");
    if (opt.ncrit < 1) throw std::runtime_error("ncrit must be >= 1");
    if (opt.max_level < 0 || opt.max_level > kKeyBits)
        throw std::runtime_error("max_level must be in [0, 16]");
    const int64_t np = xt ? 2 * n : n;
    t = Tree();
    t.n = np;
    double *x = be.template alloc<double>(3 * np);
    be.put(x, xs, (size_t)3 * n * sizeof(double));
    if (xt) be.put(x + 3 * n, xt, (size_t)3 * n * sizeof(double));

    // root cube
    double lo[3], hi[3];
    bool bad = false;
    be.bbox(x, np, lo, hi, bad);
    if (bad) throw std::runtime_error("non-finite coordinate");
    root_cube(lo, hi, t.centre, t.hw);
    const double corner[3] = {t.centre[0] - t.hw, t.centre[1] - t.hw, t.centre[2] - t.hw};

    // Morton order (stable: equal keys keep the input order)
    uint64_t *smk = be.template alloc<uint64_t>(np);
    uint32_t *perm = be.template alloc<uint32_t>(np);
    be.run(np, FKeys{x, corner[0], corner[1], corner[2], 2.0 * t.hw, smk, perm});
    be.sort_pairs(smk, perm, np, 3 * kKeyBits);

    // S0: boxes holding more than ncrit points, top down
    std::vector<LevelSet> S0;
    {
        LevelSet root;
        if (np > opt.ncrit && opt.max_level > 0) {
            root.k = be.template alloc<uint64_t>(1);
            be.fill(root.k, 0, sizeof(uint64_t));
            root.n = 1;
        }
        S0.push_back(root);
        while (S0.back().n > 0) {
            const int lc = (int)S0.size();
            const int64_t m = 8 * S0.back().n;
            uint64_t *ck = be.template alloc<uint64_t>(m);
            int64_t *flag = be.template alloc<int64_t>(m);
            be.run(m, FChildren{S0.back().k, lc, 0, opt.ncrit, opt.max_level, smk, np, ck, nullptr,
                                nullptr, flag});
            LevelSet nx;
            nx.k = keep_flagged(be, ck, flag, m, nx.n);
            S0.push_back(nx);
        }
        S0.pop_back();  // the last level is empty
    }
    // S: with the balance condition, S0 plus the boxes touching a split box
    // one level finer, from the deepest level up
    const int nsl = (int)S0.size();
    std::vector<LevelSet> S(S0);
    if (opt.balance) {
        for (int l = nsl - 2; l >= 0; --l) {
            const LevelSet &D = S[l + 1];
            const int64_t m = 8 * D.n;
            uint64_t *tk = be.template alloc<uint64_t>(m);
            int64_t *flag = be.template alloc<int64_t>(m);
            be.run(m, FTouch{D.k, l, tk, flag});
            int64_t nt = 0;
            uint64_t *touched = keep_flagged(be, tk, flag, m, nt);
            const int64_t nc = S0[l].n + nt;
            uint64_t *all = be.template alloc<uint64_t>(nc);
            if (S0[l].n) be.put(all, S0[l].k, (size_t)S0[l].n * sizeof(uint64_t));
            if (nt) be.put(all + S0[l].n, touched, (size_t)nt * sizeof(uint64_t));
            be.sort_keys(all, nc, 3 * l);
            int64_t *uf = be.template alloc<int64_t>(nc);
            be.run(nc, FUniqueFlag{all, uf});
            LevelSet u;
            u.k = keep_flagged(be, all, uf, nc, u.n);
            S[l] = u;
        }
    }
    // concatenated split sets for the leaf test
    Levels sp{};
    int64_t stot = 0;
    for (int l = 0; l < nsl; ++l) {
        sp.p[l] = (int32_t)stot;
        stot += S[l].n;
    }
    sp.p[nsl] = (int32_t)stot;
    uint64_t *sk = be.template alloc<uint64_t>(stot);
    for (int l = 0; l < nsl; ++l)
        if (S[l].n) be.put(sk + sp.p[l], S[l].k, (size_t)S[l].n * sizeof(uint64_t));

    // nodes: the root, then the non-empty children of every split box
    int64_t cap = 1;
    for (int l = 0; l < nsl; ++l) cap += 8 * S[l].n;
    if (cap > INT32_MAX) throw std::runtime_error("too many boxes");
    uint64_t *mk = be.template alloc<uint64_t>(cap);
    int32_t *lvl = be.template alloc<int32_t>(cap);
    int64_t *nb = be.template alloc<int64_t>(cap);
    int64_t *ne = be.template alloc<int64_t>(cap);
    {
        const uint64_t z = 0;
        const int32_t zl = 0;
        const int64_t zb = 0;
        be.put(mk, &z, sizeof z);
        be.put(lvl, &zl, sizeof zl);
        be.put(nb, &zb, sizeof zb);
        be.put(ne, &np, sizeof np);
        be.sync();
    }
    Levels lp{};
    lp.p[0] = 0;
    lp.p[1] = 1;
    int depth = 0;
    for (int l = 0; l < nsl; ++l) {
        if (S[l].n == 0) break;
        const int64_t m = 8 * S[l].n;
        uint64_t *ck = be.template alloc<uint64_t>(m);
        int64_t *b = be.template alloc<int64_t>(m);
        int64_t *e = be.template alloc<int64_t>(m);
        int64_t *flag = be.template alloc<int64_t>(m);
        be.run(m, FChildren{S[l].k, l + 1, 1, opt.ncrit, opt.max_level, smk, np, ck, b, e, flag});
        int64_t *pos = be.template alloc<int64_t>(m);
        be.scan(flag, pos, m);
        const int64_t cnt = be.get(pos, m - 1) + be.get(flag, m - 1);
        if (cnt == 0) break;
        be.run(m, FPlaceNodes{ck, b, e, flag, pos, lp.p[l + 1], l + 1, mk, lvl, nb, ne});
        lp.p[l + 2] = lp.p[l + 1] + (int32_t)cnt;
        depth = l + 1;
    }
    const int64_t nn = lp.p[depth + 1];
    t.depth = depth;
    int32_t *parent = be.template alloc<int32_t>(nn);
    int32_t *child = be.template alloc<int32_t>(8 * nn);
    int32_t *key4 = be.template alloc<int32_t>(4 * nn);
    uint8_t *leaf = be.template alloc<uint8_t>(nn);
    be.fill(child, 0xFF, (size_t)8 * nn * sizeof(int32_t));
    NodeView tv{mk, lvl, child, leaf, lp, depth};
    be.run(nn, FLink{tv, sk, sp, nsl, parent, child, key4, leaf});
    int64_t *lflag = be.template alloc<int64_t>(nn);
    be.run(nn, FLeafFlag{leaf, lflag});
    int64_t *lpos = be.template alloc<int64_t>(nn);
    be.scan(lflag, lpos, nn);
    const int64_t nleaves = be.get(lpos, nn - 1) + be.get(lflag, nn - 1);
    int32_t *leaves = be.template alloc<int32_t>(nleaves);
    be.run(nn, FLeafIds{lflag, lpos, leaves});

    // sorted point data
    float *rel = be.template alloc<float>(4 * np);
    float *rel_lo = be.template alloc<float>(4 * np);
    be.run(nleaves, FRel{tv, leaves, nb, ne, perm, x, t.centre[0], t.centre[1], t.centre[2], t.hw,
                         rel, rel_lo});
    int64_t *perm64 = be.template alloc<int64_t>(np);
    be.run(np, FWiden{perm, perm64});

    // lists
    int64_t *uptr = nullptr, *wptr = nullptr, *vptr = nullptr;
    int32_t *uidx = nullptr, *widx = nullptr, *vidx = nullptr;
    list_csr<B, FListU>(
        be, nn, nleaves,
        [&](auto f, const int64_t *ptr, int32_t *idx, int64_t *cnt) {
            f.t = tv;
            f.leaves = leaves;
            f.ptr = ptr;
            f.idx = idx;
            f.cnt = cnt;
            return f;
        },
        t.u_ptr, t.u_idx, &uptr, &uidx);
    const int32_t first2 = depth >= 2 ? lp.p[2] : (int32_t)nn;
    list_csr<B, FListV>(
        be, nn, nn - first2,
        [&](auto f, const int64_t *ptr, int32_t *idx, int64_t *cnt) {
            f.t = tv;
            f.parent = parent;
            f.first = first2;
            f.ptr = ptr;
            f.idx = idx;
            f.cnt = cnt;
            return f;
        },
        t.v_ptr, t.v_idx, &vptr, &vidx);
    list_csr<B, FListW>(
        be, nn, nleaves,
        [&](auto f, const int64_t *ptr, int32_t *idx, int64_t *cnt) {
            f.t = tv;
            f.leaves = leaves;
            f.ptr = ptr;
            f.idx = idx;
            f.cnt = cnt;
            return f;
        },
        t.w_ptr, t.w_idx, &wptr, &widx);
    // X = the transpose of W, sorted by (a, b)
    {
        const int64_t m = (int64_t)t.w_idx.size();
        uint64_t *pk = be.template alloc<uint64_t>(m);
        be.run(nleaves, FXPairs{leaves, wptr, widx, pk});
        be.sort_keys(pk, m, 64);
        int64_t *xptr = be.template alloc<int64_t>(nn + 1);
        int32_t *xidx = be.template alloc<int32_t>(m);
        be.run(nn + 1, FXPtr{pk, m, xptr});
        be.run(m, FXIdx{pk, xidx});
        t.x_ptr.resize(nn + 1);
        t.x_idx.resize(m);
        be.to_host(xptr, nn + 1, t.x_ptr.data());
        be.to_host(xidx, m, t.x_idx.data());
    }
    {
        const int64_t m = (int64_t)t.v_idx.size();
        int16_t *voff = be.template alloc<int16_t>(m);
        int *vbad = be.template alloc<int>(1);
        be.fill(vbad, 0, sizeof(int));
        be.run(nn - first2, FVOff{tv, first2, vptr, vidx, voff, vbad});
        t.v_off.resize(m);
        be.to_host(voff, m, t.v_off.data());
        if (be.get(vbad, 0)) throw std::runtime_error("internal: V entry outside the offset set");
    }
    {
        int64_t *val = be.template alloc<int64_t>(nn + 1);
        be.fill(val, 0, (size_t)(nn + 1) * sizeof(int64_t));
        be.run(nleaves, FP2P{leaves, nb, ne, uptr, uidx, val});
        int64_t *acc = be.template alloc<int64_t>(nn + 1);
        be.scan(val, acc, nn + 1);
        t.p2p_pairs = be.get(acc, nn);
    }

    // node and point arrays to the host tree
    t.key.resize(4 * nn);
    t.begin.resize(nn);
    t.end.resize(nn);
    t.parent.resize(nn);
    t.child.resize(8 * nn);
    t.leaf.resize(nn);
    t.leaves.resize(nleaves);
    t.perm.resize(np);
    t.rel.resize(4 * np);
    t.rel_lo.resize(4 * np);
    be.to_host(key4, 4 * nn, t.key.data());
    be.to_host(nb, nn, t.begin.data());
    be.to_host(ne, nn, t.end.data());
    be.to_host(parent, nn, t.parent.data());
    be.to_host(child, 8 * nn, t.child.data());
    be.to_host(leaf, nn, t.leaf.data());
    be.to_host(leaves, nleaves, t.leaves.data());
    be.to_host(perm64, np, t.perm.data());
    be.to_host(rel, 4 * np, t.rel.data());
    be.to_host(rel_lo, 4 * np, t.rel_lo.data());
    be.sync();
    t.level_ptr.assign(lp.p, lp.p + depth + 2);
}

} // namespace

void build_tree_levels(const double *xs, const double *xt, int64_t n, const TreeOptions &opt,
                       bool on_device, Tree &t) {
    if (on_device) {
        DeviceBackend be;
        build(be, xs, xt, n, opt, t);
    } else {
        HostBackend be;
        build(be, xs, xt, n, opt, t);
    }
}

} // namespace kifmm
