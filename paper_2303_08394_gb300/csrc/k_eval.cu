// Leaf evaluation: near field over U ("P2P"), L2P from the leaf's own
// downward density, and M2P from the upward densities of its W list
// ("Computational structure of FMM operators": all three are evaluations of
// Eq. (1) between point sets, so they share one loop).
//
// One block of 128 threads owns one target leaf B.  Its sources form a list
// of segments: B's own points, the points of the other leaves in U(B), B's
// downward equivalent surface (charges = downward density), the upward
// equivalent surface of every box in W(B) (charges = upward density) -- or,
// for a W box that is a leaf with no more points than a surface, its points
// -- and, when B itself has no more points than a surface, the points of
// the leaves in X(B) (their P2L is then skipped).  The
// segment table is built in shared memory with a block scan; then all 128
// threads copy up to CAP sources at once into shared memory, positions
// shifted into B's frame (leaf-relative coordinates plus the exact dyadic
// difference of box centres, so no precision is lost at deep levels).
//
// Compute: the block works on a chunk of 16 T targets, T = 1..8 chosen per
// leaf from its size (the plan groups the leaves by T and each group runs as
// its own kernel, so the narrow widths keep fewer registers and more
// resident blocks; many charge columns cap T at 4 and take several chunks):
// lane l holds targets (l mod 16) + 16 i, i < T, and the two half-warps
// take alternate staged sources, so one shared-memory access (two adjacent
// 16-byte words) feeds 2 T pairs per lane.  The four warps always split the
// sources of a chunk between them, whatever T, so the rounding does not
// depend on T.
// The staged count is padded with zero charges far away so the inner loop
// is unrolled; the r > 0 test that drops the self pair runs only over B's
// own points.
//
// Precision: FP32 rsqrt/FMA per pair.  Each run of 32 sources per lane is
// summed in plain FP32 and added into a per-target Kahan (sum,
// compensation) pair; the pairs of the two half-warps and of the source
// slices are merged with further Kahan additions in a fixed order, and the
// potential is formed in FP64 (sum - compensation), scaled by 1/(4 pi hw)
// of the leaf's problem and written in the caller's row order (points that
// are sources only are not written).  Runs are assigned from the
// source order alone, so every right-hand side gets bit-identical
// arithmetic whatever NR it is batched in.
//
// Gradient variant (kGrad, one charge column per launch): each pair also
// adds q (y - x) / r^3 (y the source, x the target), the target-gradient of
// q / r, into three more Kahan sums; the close-pair correction covers it,
// and it is scaled by 1 / (4 pi hw^2) (positions are in root units).
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int kWarps = 4, kThreads = 32 * kWarps;
constexpr int kSegCap = 256;       // segments per table window
constexpr float kFar = 1.0e15f;    // position of padding sources (charge 0)

// Targets per lane the register budget allows for NR columns (or the
// gradient); wider leaves take one pass per chunk of 16 TMax targets.
template <int NR, bool kGrad> struct TMax {
    static constexpr int v = (NR == 1 && !kGrad) ? kLeafWidths : 4;
};
// minb: resident blocks per SM the register allocation must allow.
// sums per target and launch: NR potentials, or potential + gradient
template <int NR, bool kGrad> struct Sums {
    static_assert(!kGrad || NR == 1, "gradients are evaluated one column per launch");
    static constexpr int n = kGrad ? 4 : NR;
};

// minb: resident blocks per SM the register allocation must allow (the
// largest counts that compile without spills, and measured faster than the
// register-rich ones: the leaf pass is latency-bound, so more warps help).
template <int NR, int T> struct Cfg {
    // sources per block-staged round (several columns; a multiple of 256,
    // see run()); one column stages per warp and does not use it
    static constexpr int cap = NR == 1 ? 256 : (NR == 2 ? 768 : 512);
    static constexpr int minb = NR == 1 ? (T <= 3 ? 7 : (T <= 5 ? 6 : (T <= 7 ? 5 : 4)))
                                        : (NR == 2 ? (T <= 2 ? 5 : 4) : 1);
};

// s = fl(a + b); err receives the exact rounding error (a + b = s + err).
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// asynchronous 16- and 4-byte copies global -> shared (cp.async), their
// commit and waits
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_one() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    // merge another (sum, compensation) pair
    __device__ __forceinline__ void merge(float s2, float c2) {
        add(s2);
        add(-c2);
    }
};

template <int NR> struct Charges;
template <> struct Charges<2> {
    __device__ static void get(const float *sq, int j, float (&q)[2]) {
        const float2 v = reinterpret_cast<const float2 *>(sq)[j];
        q[0] = v.x; q[1] = v.y;
    }
};
template <> struct Charges<4> {
    __device__ static void get(const float *sq, int j, float (&q)[4]) {
        const float4 v = reinterpret_cast<const float4 *>(sq)[j];
        q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
    }
};
template <> struct Charges<8> {
    __device__ static void get(const float *sq, int j, float (&q)[8]) {
        const float4 a = reinterpret_cast<const float4 *>(sq)[2 * j];
        const float4 b = reinterpret_cast<const float4 *>(sq)[2 * j + 1];
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
        q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
    }
};

// Pairs closer than this fraction of the target leaf's half-width are
// recomputed from the position residuals (see run()).
constexpr float kCloseFrac = 0.125f;

template <int NR, int CAP> struct Smem;

template <bool kSelf>
__device__ __forceinline__ void pair_terms(float4 p, float3 x, float &r2, float &inv) {
    const float dx = p.x - x.x, dy = p.y - x.y, dz = p.z - x.z;
    // Outside B's own points a pair is never coincident in exact arithmetic;
    // the 1e-30 floor keeps one that rounds to r = 0 in FP32 finite.
    r2 = fmaf(dx, dx, fmaf(dy, dy, kSelf ? dz * dz : fmaf(dz, dz, 1e-30f)));
    inv = KIFMM_RSQRT(r2);
    if (kSelf) inv = r2 > 0.f ? inv : 0.f;
}

// Close pairs.  Positions are FP32 offsets from the target leaf's centre, so
// a pair at distance r << h (leaf half-width) computed from them alone has
// relative error ~ eps h / r.  Every staged source carries, beside its FP32
// position in B's frame, what that position dropped (the rounding of the
// move into B's frame plus the point's own residual, position = hi + lo to
// about 2^-48 h).  After a source's T pairs, a lane whose smallest r^2 (the
// target itself excluded) is below thr2 = (kCloseFrac h)^2 sets the
// source's bit in a 32-bit mask of the run (a run is at most 32 sources per
// lane); at the end of the run the lane recomputes the close pairs of its
// marked sources from the exact difference (p - x) + (p_lo - x_lo) and adds
// q (1/r_accurate - 1/r_fp32).  Distinct points that coincide in FP32 are so
// resolved as in FP64 (exact duplicates keep r = 0 and drop out).  On points
// spread over a surface most sources have a close target somewhere in the
// leaf, but few for any one lane, so marking costs a predicated OR per
// source and the corrections are paid per close source of the lane only.
template <int NR, int T, bool kSelf, bool kGrad>
__device__ __forceinline__ void fix_source(const float4 *spos, const float4 *sres,
                                           const float *sq, const float4 *xlo, int k, int base,
                                           const float3 (&x)[T], int t0, int tl, float thr2,
                                           float (&part)[T][Sums<NR, kGrad>::n]) {
    const float4 p = spos[k], pl = sres[k];
    float q[NR];
    if constexpr (NR == 1) {
        q[0] = p.w;
    } else {
        Charges<NR>::get(sq, k, q);
    }
#pragma unroll
    for (int i = 0; i < T; ++i) {
        float r2, inv;
        pair_terms<kSelf>(p, x[i], r2, inv);
        if (!(r2 < thr2) || (kSelf && base + k == t0 + 16 * i)) continue;
        // a close pair has a valid target: padding targets are far
        const float4 xl = xlo[tl + 16 * i];
        const float dx = (p.x - x[i].x) + (pl.x - xl.x);
        const float dy = (p.y - x[i].y) + (pl.y - xl.y);
        const float dz = (p.z - x[i].z) + (pl.z - xl.z);
        const float r2a = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float ia = r2a > 0.f ? KIFMM_RSQRT(r2a) : 0.f;
        const float d = ia - inv;
        if constexpr (kGrad) {
            // replace the main loop's FP32 term w3 (p - x) by the accurate one
            part[i][0] = fmaf(q[0], d, part[i][0]);
            const float w3 = q[0] * (inv * inv * inv);
            const float wa = q[0] * (ia * ia * ia);
            part[i][1] = fmaf(wa, dx, fmaf(-w3, p.x - x[i].x, part[i][1]));
            part[i][2] = fmaf(wa, dy, fmaf(-w3, p.y - x[i].y, part[i][2]));
            part[i][3] = fmaf(wa, dz, fmaf(-w3, p.z - x[i].z, part[i][3]));
        } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) part[i][r] = fmaf(q[r], d, part[i][r]);
        }
    }
}

// Staged sources j = a + 2u + h (j < e; a and e multiples of 16) against
// this lane's T targets; h is the lane's half-warp.  base + j is the
// source's index in the window's source list; t0: index of the lane's first
// target among B's points (target i is t0 + 16 i), and tl its slot in the
// staged target residuals.  B's own points are listed first, in order, so
// in the self run a target meets itself at source index t0 + 16 i.
// kClose = false: every source of [a, e) is provably farther than
// kCloseFrac h from every target (see far_from in leaf()), so the close
// marking is left out; the sums are those of kClose = true.
template <int NR, int T, bool kSelf, bool kGrad, bool kClose>
__device__ __forceinline__ void run(const float4 *spos, const float4 *sres, const float *sq,
                                    const float4 *xlo, int base, int a, int e, int h,
                                    const float3 (&x)[T], int t0, int tl, float thr2,
                                    float (&part)[T][Sums<NR, kGrad>::n]) {
    uint32_t close = 0;  // bit 4 it + u: source a + h + 8 it + 2 u has a close target
    int it = 0;
    for (int j = a + h; j < e; j += 8, ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = j + 2 * u;
            const float4 p = spos[k];
            float q[NR];
            if constexpr (NR == 1) {
                q[0] = p.w;
            } else {
                Charges<NR>::get(sq, k, q);
            }
            float r2min = 3.0e38f;
#pragma unroll
            for (int i = 0; i < T; ++i) {
                float r2, inv;
                pair_terms<kSelf>(p, x[i], r2, inv);
                if constexpr (kClose) {
                    if (!kSelf || base + k != t0 + 16 * i) r2min = fminf(r2min, r2);
                }
                if constexpr (kGrad) {
                    const float w3 = q[0] * (inv * inv * inv);
                    part[i][0] = fmaf(q[0], inv, part[i][0]);
                    part[i][1] = fmaf(w3, p.x - x[i].x, part[i][1]);
                    part[i][2] = fmaf(w3, p.y - x[i].y, part[i][2]);
                    part[i][3] = fmaf(w3, p.z - x[i].z, part[i][3]);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) part[i][r] = fmaf(q[r], inv, part[i][r]);
                }
            }
            if constexpr (kClose) {
                if (r2min < thr2) close |= 1u << (4 * it + u);
            }
        }
    }
    if constexpr (kClose) {
        // a run spans at most 64 staged sources, so eight iterations of four
#pragma unroll 1
        while (close) {
            const int bit = __ffs(close) - 1;
            close &= close - 1;
            const int k = a + h + 8 * (bit >> 2) + 2 * (bit & 3);
            fix_source<NR, T, kSelf, kGrad>(spos, sres, sq, xlo, k, base, x, t0, tl, thr2, part);
        }
    }
}

// Segment table of one window and the residuals of a pass's targets.
struct SegTable {
    float4 xlo[128];          // residuals of the chunk's 16 T <= 128 targets
    float4 seg_off[kSegCap];  // centre offset, surface radius
    int seg_node[kSegCap], seg_kind[kSegCap], seg_start[kSegCap + 1];
    int warp_sum[kWarps], warp_nf[kWarps];
};

// Several columns: the block stages rounds of CAP sources together.
template <int NR, int CAP> struct Smem : SegTable {
    union {
        struct {
            float4 spos[CAP];
            float4 sres[CAP];   // what each staged position dropped (see fix_source)
            float sq[CAP * NR];
        } st;
        // partial sums of the source slices (used after the last round)
        float2 red[kWarps][4 * (NR > 4 ? NR : 4)][16];
    } u;
    __device__ float2 *red(int w, int row) { return u.red[w][row]; }
};

// One column: every warp stages its own runs of 64 sources, double
// buffered: cp.async copies the raw data of the warp's next run while it
// computes the current one; each lane then moves its own two slots into B's
// frame in place (position, charge in w; residual), so no block barrier
// separates the runs.
template <int CAP> struct Smem<1, CAP> : SegTable {
    union {
        struct {
            float4 pos[kWarps][2][64];  // raw position, then staged position + charge
            float4 lo[kWarps][2][64];   // raw point residual, then staged residual
            float q[kWarps][2][64];     // raw charge or density
        } w;
        // partial sums of the source slices: T x sums per target, up to
        // 8 x 1 (potentials) or 4 x 4 (gradients)
        float2 red[kWarps][16][16];
    } u;
    __device__ float2 *red(int w, int row) { return u.red[w][row]; }
};

template <int NR, int T, bool kGrad>
__device__ __forceinline__ void leaf(const DevTree &t, const DevOps &o, const DevWork &w, int r0,
                                     Smem<NR, Cfg<NR, T>::cap> &sm, int b, int2 rb, int nt) {
    constexpr int NQ = Sums<NR, kGrad>::n;
    constexpr int CAP = Cfg<NR, T>::cap;
    static_assert(CAP % (64 * kWarps) == 0, "rounds must hold whole runs for every slicing");
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int tl = lane & 15, half = lane >> 4;
    const float4 gb = t.geom[b];
    const int u0 = t.u_ptr[b], nu = t.u_ptr[b + 1] - u0;
    const int w0 = t.w_ptr[b], nw = t.w_ptr[b + 1] - w0;
    const int nl2p = t.level[b] >= 2 ? 1 : 0;
    // X leaves taken directly (no P2L slot for B)
    const int x0 = t.x_ptr[b], nxd = t.x_slot[b] < 0 ? t.x_ptr[b + 1] - x0 : 0;
    const int nseg = nu + nl2p + nw + nxd;
    const int ns = o.ns, nsp = (o.ns + 3) & ~3;

    // the four warps are the source slices of one target chunk per pass
    constexpr int CH = 16 * T;
    const int nchunk = (nt + CH - 1) / CH;
    const int split = wid;
    const int self_end16 = (nt + 15) & ~15;
    const float thr = kCloseFrac * gb.w, thr2 = thr * thr;
    // a source at least this far (L-infinity, root units) from B's cube is
    // farther than thr from every target, with room for FP32 rounding
    const float far_sep = 1.01f * thr;

    for (int chunk = 0; chunk < nchunk; ++chunk) {
        float3 x[T];
        bool valid[T];
        const int t0 = chunk * CH + tl;  // target i is B's point t0 + 16 i
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const int tt = t0 + 16 * i;
            valid[i] = tt < nt;
            x[i] = make_float3(-kFar, -kFar, -kFar);
            if (valid[i]) {
                const float4 p = t.pts[rb.x + tt];
                x[i] = make_float3(p.x, p.y, p.z);
            }
        }
        if (tid < CH) {
            const int tt = chunk * CH + tid;
            sm.xlo[tid] = tt < nt ? t.pts_lo[rb.x + tt] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        Kahan acc[T][NQ];

        for (int sw = 0; sw < nseg; sw += kSegCap) {
            const int nsegw = min(kSegCap, nseg - sw);
            // ---- segment table: logical order [B] + U\{B} + [DE(B)] + W
            // (surfaces, or points of the small leaves) + X taken directly
            int cnt2[2];
            int nf = -1;  // last segment of this thread that may hold a close source
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int s = 2 * tid + hh;
                int c = 0;
                if (s < nsegw) {
                    const int ls = sw + s;
                    int node, kind;
                    if (ls < nu) {
                        node = ls == 0 ? b : t.u_idx[u0 + ls];
                        if (ls > 0 && node == b) node = t.u_idx[u0];
                        kind = 0;
                    } else if (ls < nu + nl2p) {
                        node = b;
                        kind = 1;
                    } else if (ls < nu + nl2p + nw) {
                        node = t.w_idx[w0 + ls - nu - nl2p];
                        kind = t.w_direct[node] ? 0 : 2;
                    } else {
                        node = t.x_idx[x0 + ls - nu - nl2p - nw];
                        kind = 0;
                    }
                    const float4 ga = t.geom[node];
                    float rad = 0.f;
                    const float ox = ga.x - gb.x, oy = ga.y - gb.y, oz = ga.z - gb.z;
                    bool far = false;
                    if (kind == 0) {
                        const int2 ra = t.range[node];
                        c = ra.y - ra.x;
                        sm.seg_node[s] = ra.x;
                        // a W or X leaf does not touch B: its points are at
                        // least max|offset| - h_A - h from B's cube
                        if (ls >= nu)
                            far = fmaxf(fabsf(ox), fmaxf(fabsf(oy), fabsf(oz))) - ga.w - gb.w >=
                                  far_sep;
                    } else {
                        c = ns;
                        sm.seg_node[s] = node;
                        rad = kind == 1 ? o.ao * gb.w : o.ai * ga.w;
                        // surface points lie on the cube of half-width rad
                        // about the box centre: B's own downward surface
                        // encloses B with a gap rad - h; a W box's surface
                        // is at least max|offset| - rad - h from B's cube
                        const float sep =
                            kind == 1 ? rad - gb.w
                                      : fmaxf(fabsf(ox), fmaxf(fabsf(oy), fabsf(oz))) - rad - gb.w;
                        far = sep >= far_sep;
                    }
                    if (!far) nf = s;
                    sm.seg_kind[s] = kind;
                    sm.seg_off[s] = make_float4(ox, oy, oz, rad);
                }
                cnt2[hh] = c;
            }
            // block exclusive scan of the per-thread pair sums
            const int mine = cnt2[0] + cnt2[1];
            int incl = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            nf = __reduce_max_sync(0xffffffffu, nf);
            if (lane == 31) {
                sm.warp_sum[wid] = incl;
                sm.warp_nf[wid] = nf;
            }
            __syncthreads();
            int base_w = 0, total = 0, nfmax = -1;
#pragma unroll
            for (int k = 0; k < kWarps; ++k) {
                const int v = sm.warp_sum[k];
                if (k < wid) base_w += v;
                total += v;
                nfmax = max(nfmax, sm.warp_nf[k]);
            }
            const int excl = base_w + incl - mine;
            if (2 * tid < nsegw) sm.seg_start[2 * tid] = excl;
            if (2 * tid + 1 < nsegw) sm.seg_start[2 * tid + 1] = excl + cnt2[0];
            if (tid == 0) sm.seg_start[nsegw] = total;
            __syncthreads();
            // sources from far_from on are far from every target
            const int far_from = sm.seg_start[nfmax + 1];
            const int self_hi = sw == 0 ? self_end16 : 0;

            // Runs of 64 sources (32 per half-warp) go round-robin to the
            // slices: run r of the window (sources 64 r ..) to warp r mod 4,
            // whatever the staging, so the rounding depends on the source
            // order only.  run_sources: the sources [g0, g0 + e) of run g0 / 64
            // are staged at spos[0 .. e).
            auto run_sources = [&](const float4 *spos, const float4 *sres, const float *sq,
                                   int g0, int e) {
                const int js = min(max(self_hi - g0, 0), e);
                float part[T][NQ];
#pragma unroll
                for (int i = 0; i < T; ++i)
#pragma unroll
                    for (int r = 0; r < NQ; ++r) part[i][r] = 0.f;
                if (js > 0)
                    run<NR, T, true, kGrad, true>(spos, sres, sq, sm.xlo, g0, 0, js, half, x, t0,
                                                  tl, thr2, part);
                if (g0 >= far_from)
                    run<NR, T, false, kGrad, false>(spos, sres, sq, sm.xlo, g0, js, e, half, x,
                                                    t0, tl, thr2, part);
                else
                    run<NR, T, false, kGrad, true>(spos, sres, sq, sm.xlo, g0, js, e, half, x,
                                                   t0, tl, thr2, part);
#pragma unroll
                for (int i = 0; i < T; ++i)
#pragma unroll
                    for (int r = 0; r < NQ; ++r) acc[i][r].add(part[i][r]);
            };

            int seg = 0;  // segment of this thread's next source (sources ascend)
            if constexpr (NR == 1) {
                // ---- warp-private runs r = wid, wid + 4, ...; lane l stages
                // slots l and l + 32 of each
                const int nrun = (total + 63) >> 6;
                float4(*wpos)[64] = sm.u.w.pos[wid];
                float4(*wlo)[64] = sm.u.w.lo[wid];
                float(*wq)[64] = sm.u.w.q[wid];
                int sg_next[2];
                auto issue = [&](int r, int bb) {
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int k = lane + 32 * h2, f = 64 * r + k;
                        int sg = -1;
                        if (f < total) {
                            // f < total = seg_start[nsegw], so the scan stops
                            // at a segment index below nsegw
                            while (sm.seg_start[seg + 1] <= f) ++seg;
                            sg = seg;
                            const int off = f - sm.seg_start[seg];
                            const int kind = sm.seg_kind[seg];
                            if (kind == 0) {
                                const int i = sm.seg_node[seg] + off;
                                cp_async16(&wpos[bb][k], t.pts + i);
                                cp_async16(&wlo[bb][k], t.pts_lo + i);
                                cp_async4(&wq[bb][k], w.qs + (size_t)i * w.nrhs + r0);
                            } else {
                                const float *dens = kind == 1 ? w.down : w.up;
                                cp_async16(&wpos[bb][k], o.surf + off);
                                cp_async4(&wq[bb][k],
                                          dens + ((size_t)sm.seg_node[seg] * w.nrhs + r0) * nsp +
                                              off);
                            }
                        }
                        sg_next[h2] = sg;
                    }
                    cp_async_commit();
                };
                int r = wid, bb = 0;
                if (r < nrun) issue(r, 0);
                for (; r < nrun; r += kWarps, bb ^= 1) {
                    const int sg_cur[2] = {sg_next[0], sg_next[1]};
                    if (r + kWarps < nrun) {
                        issue(r + kWarps, bb ^ 1);
                        cp_async_wait_one();
                    } else {
                        cp_async_wait_all();
                    }
                    // this lane's two slots into B's frame, in place
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int k = lane + 32 * h2, sg = sg_cur[h2];
                        float4 pos = make_float4(kFar, kFar, kFar, 0.f);
                        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (sg >= 0) {
                            const float4 so = sm.seg_off[sg], p = wpos[bb][k];
                            const float q = wq[bb][k];
                            if (sm.seg_kind[sg] == 0) {
                                const float4 pl = wlo[bb][k];
                                float ex, ey, ez;
                                pos = make_float4(two_sum(p.x, so.x, ex), two_sum(p.y, so.y, ey),
                                                  two_sum(p.z, so.z, ez), q);
                                res = make_float4(ex + pl.x, ey + pl.y, ez + pl.z, 0.f);
                            } else {
                                pos = make_float4(fmaf(so.w, p.x, so.x), fmaf(so.w, p.y, so.y),
                                                  fmaf(so.w, p.z, so.z), q);
                            }
                        }
                        wpos[bb][k] = pos;
                        wlo[bb][k] = res;
                    }
                    __syncwarp();
                    const int g0 = 64 * r;
                    run_sources(wpos[bb], wlo[bb], nullptr, g0,
                                (min(64, total - g0) + 15) & ~15);
                    __syncwarp();
                }
                // the next window's table replaces this one
                __syncthreads();
            } else {
                // ---- rounds of at most CAP sources staged by the block
                for (int base = 0; base < total; base += CAP) {
                    const int m = min(CAP, total - base);
                    const int mp = (m + 15) & ~15;
#pragma unroll 4
                    for (int it = 0; it < CAP / kThreads; ++it) {
                        const int k = tid + it * kThreads;
                        if ((k & ~31) >= mp) break;  // whole warp past the end
                        float4 pos = make_float4(kFar, kFar, kFar, 0.f);
                        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
                        float q[NR];
#pragma unroll
                        for (int r = 0; r < NR; ++r) q[r] = 0.f;
                        if (k < m) {
                            const int f = base + k;
                            while (sm.seg_start[seg + 1] <= f) ++seg;
                            const int off = f - sm.seg_start[seg];
                            const float4 so = sm.seg_off[seg];
                            const int kind = sm.seg_kind[seg];
                            if (kind == 0) {
                                const int i = sm.seg_node[seg] + off;
                                const float4 p = __ldg(t.pts + i), pl = __ldg(t.pts_lo + i);
                                float ex, ey, ez;
                                pos = make_float4(two_sum(p.x, so.x, ex), two_sum(p.y, so.y, ey),
                                                  two_sum(p.z, so.z, ez), 0.f);
                                res = make_float4(ex + pl.x, ey + pl.y, ez + pl.z, 0.f);
                                const float *qi = w.qs + (size_t)i * w.nrhs + r0;
#pragma unroll
                                for (int r = 0; r < NR; ++r) q[r] = __ldg(qi + r);
                            } else {
                                const float4 sp = __ldg(o.surf + off);
                                pos = make_float4(fmaf(so.w, sp.x, so.x), fmaf(so.w, sp.y, so.y),
                                                  fmaf(so.w, sp.z, so.z), 0.f);
                                const float *dens = kind == 1 ? w.down : w.up;
                                const float *d =
                                    dens + ((size_t)sm.seg_node[seg] * w.nrhs + r0) * nsp + off;
#pragma unroll
                                for (int r = 0; r < NR; ++r) q[r] = __ldg(d + (size_t)r * nsp);
                            }
                        }
                        if (k < mp) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) sm.u.st.sq[k * NR + r] = q[r];
                            sm.u.st.spos[k] = pos;
                            sm.u.st.sres[k] = res;
                        }
                    }
                    __syncthreads();
                    for (int j0 = 64 * split; j0 < mp; j0 += 64 * kWarps)
                        run_sources(sm.u.st.spos + j0, sm.u.st.sres + j0, sm.u.st.sq + j0 * NR,
                                    base + j0, min(64, mp - j0));
                    __syncthreads();
                }
            }
        }

        // ---- merge the upper half-warp into the lower, then the slices
#pragma unroll
        for (int i = 0; i < T; ++i)
#pragma unroll
            for (int r = 0; r < NQ; ++r) {
                const float s2 = __shfl_down_sync(0xffffffffu, acc[i][r].s, 16);
                const float c2 = __shfl_down_sync(0xffffffffu, acc[i][r].c, 16);
                if (half == 0) acc[i][r].merge(s2, c2);
            }
        if (split > 0 && half == 0) {
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int r = 0; r < NQ; ++r)
                    sm.red(wid, i * NQ + r)[tl] = make_float2(acc[i][r].s, acc[i][r].c);
        }
        __syncthreads();
        if (split == 0 && half == 0) {
            for (int s = 1; s < kWarps; ++s) {
#pragma unroll
                for (int i = 0; i < T; ++i)
#pragma unroll
                    for (int r = 0; r < NQ; ++r) {
                        const float2 v = sm.red(s, i * NQ + r)[tl];
                        acc[i][r].merge(v.x, v.y);
                    }
            }
            const double scale = t.node_scale[b];
#pragma unroll
            for (int i = 0; i < T; ++i) {
                if (!valid[i]) continue;
                const int64_t row = t.oidx[rb.x + chunk * CH + tl + 16 * i];
                if (row < 0) continue;  // a source only
                if constexpr (kGrad) {
                    if (w.pot_user)
                        w.pot_user[(size_t)row * w.nrhs + r0] =
                            ((double)acc[i][0].s - (double)acc[i][0].c) * scale;
                    // d/dx of 1 / (4 pi hw r_root): 1 / (4 pi hw^2) per root-unit term
                    const double gscale = scale * scale * (4.0 * 3.14159265358979323846);
                    double *g = w.grad_user + ((size_t)row * w.nrhs + r0) * 3;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        g[k] = ((double)acc[i][1 + k].s - (double)acc[i][1 + k].c) * gscale;
                } else {
                    double *out = w.pot_user + (size_t)row * w.nrhs + r0;
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        out[r] = ((double)acc[i][r].s - (double)acc[i][r].c) * scale;
                }
            }
        }
        __syncthreads();
    }
}

template <int NR, int T, bool kGrad>
struct Occupancy {
    static constexpr int minb = kGrad ? (T <= 2 ? 6 : (T == 3 ? 5 : 4)) : Cfg<NR, T>::minb;
};

template <int NR, int T, bool kGrad>
__global__ void __launch_bounds__(kThreads, (Occupancy<NR, T, kGrad>::minb))
    k_eval(DevTree t, DevOps o, DevWork w, int r0, int first) {
    // The width groups of one pass read only what the passes before them
    // wrote and write disjoint rows, so the next group may start as soon as
    // every block of this one has started (it fills this group's last
    // wave).  Each block ends by waiting for its programmatic predecessor
    // (the previous group; nothing for the first), so a group completes
    // only after all groups before it, and the work after the pass sees
    // every row.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ __align__(16) Smem<NR, Cfg<NR, T>::cap> sm;
    const int b = t.leaves[first + blockIdx.x];
    const int2 rb = t.range[b];
    const int nt = rb.y - rb.x;
    if (nt > 0) leaf<NR, T, kGrad>(t, o, w, r0, sm, b, rb, nt);
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// one launch per non-empty width group, widest first (longest blocks start
// first) or narrowest first (the autotuner's choice; the groups write
// disjoint rows, so the order changes no result); group Tg runs with
// min(Tg, TMax) targets per lane
template <int NR, bool kGrad, int T>
void launch_width(const DevTree &t, const DevOps &o, const DevWork &w, int r0, int first,
                  int n, cudaStream_t s, bool pdl) {
    if (!pdl) {
        k_eval<NR, T, kGrad><<<n, kThreads, 0, s>>>(t, o, w, r0, first);
        return;
    }
    // a programmatic dependent of the previous width group (see k_eval)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_eval<NR, T, kGrad>, t, o, w, r0, first);
}

template <int NR, bool kGrad = false>
cudaError_t launch_eval_nr(const DevTree &t, const DevOps &o, const DevWork &w, int r0,
                           cudaStream_t s, int *launches, bool narrow_first) {
    int launched = 0;  // groups of this pass launched so far
    for (int step = 0; step < kLeafWidths; ++step) {
        const int Tg = narrow_first ? 1 + step : kLeafWidths - step;
        const int n = t.t_first[Tg - 1] - t.t_first[Tg], first = t.t_first[Tg];
        if (n <= 0) continue;
        const int T = Tg < TMax<NR, kGrad>::v ? Tg : TMax<NR, kGrad>::v;
        const bool pdl = launched > 0;
        switch (T) {
        case 1: launch_width<NR, kGrad, 1>(t, o, w, r0, first, n, s, pdl); break;
        case 2: launch_width<NR, kGrad, 2>(t, o, w, r0, first, n, s, pdl); break;
        case 3: launch_width<NR, kGrad, 3>(t, o, w, r0, first, n, s, pdl); break;
        case 4: launch_width<NR, kGrad, 4>(t, o, w, r0, first, n, s, pdl); break;
        default:
            if constexpr (TMax<NR, kGrad>::v > 4) {
                switch (T) {
                case 5: launch_width<NR, kGrad, 5>(t, o, w, r0, first, n, s, pdl); break;
                case 6: launch_width<NR, kGrad, 6>(t, o, w, r0, first, n, s, pdl); break;
                case 7: launch_width<NR, kGrad, 7>(t, o, w, r0, first, n, s, pdl); break;
                default: launch_width<NR, kGrad, 8>(t, o, w, r0, first, n, s, pdl); break;
                }
            }
            break;
        }
        ++launched;
        ++*launches;
    }
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_eval(const DevTree &t, const DevOps &o, const DevWork &w, cudaStream_t s,
                        int *launches, bool narrow_first) {
    *launches = 0;
    if (w.grad_user) {
        // potentials (if w.pot_user) and gradients, one column per launch
        cudaError_t e = cudaSuccess;
        for (int r0 = 0; r0 < w.nrhs && e == cudaSuccess; ++r0)
            e = launch_eval_nr<1, true>(t, o, w, r0, s, launches, narrow_first);
        return e;
    }
    int r0 = 0;
    cudaError_t e = cudaSuccess;
    while (r0 < w.nrhs && e == cudaSuccess) {
        int left = w.nrhs - r0;
        if (left >= 8) { e = launch_eval_nr<8>(t, o, w, r0, s, launches, narrow_first); r0 += 8; }
        else if (left >= 4) { e = launch_eval_nr<4>(t, o, w, r0, s, launches, narrow_first); r0 += 4; }
        else if (left >= 2) { e = launch_eval_nr<2>(t, o, w, r0, s, launches, narrow_first); r0 += 2; }
        else { e = launch_eval_nr<1>(t, o, w, r0, s, launches, narrow_first); r0 += 1; }
    }
    return e;
}

} // namespace kifmm
