// Batched matrix x gathered-vector products for the upward and downward
// passes (P2M, M2M, L2L, the downward check-to-equivalent step and the M2L
// projections).  Every one of them is, for all boxes of a level at once,
//
//   Y[dst(v)][i] = scale[i] * ( sum_s sum_j A_s[i][j] X_s[src_s(v)][j] )
//                  + add[add(v)][i]
//
// with v running over (list position, right-hand side) pairs.  Segment s
// pairs an operator A_s (stored as its transpose, rows padded to a multiple
// of 4 floats) with a source array whose row for vector v is chosen through
// an index list (a child, the parent, the box itself, ...; -1 reads zeros).
//
// Tiling: a block of 128 threads computes BM output rows x BV vectors, each
// thread an RP x 4 register tile (rows RP*tr.., vectors tv + TV q).  Five
// shapes are compiled -- 64 x 32, 32 x 64 and 128 x 16 with 4 x 4 tiles,
// 64 x 64 and 128 x 32 with 8 x 4 tiles -- and the plan's autotuner picks
// one per call site; every shape computes each output with the same
// K-ordered FMA chain, so the choice never changes a bit of the result.
// K advances in chunks of 32, copied global -> shared with cp.async,
// Stages chunks in flight (as many as 48 KB of shared memory holds, up to
// three), so the per-chunk L2 round trip is paid once per Stages chunks;
// the source row of each vector is looked up once per segment, not per
// chunk.  Missing sources and the ragged end of K are zero-filled by the
// copies themselves (source size below 16 bytes).  Every source and
// operator row stride is a multiple of 4 floats, so each 16-byte copy is
// aligned.
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int BK = 32;
constexpr int XLD = BK + 4;  // padded row of the vector tile (floats)
// chunks in flight: three where they fit the 48 KB of static shared memory
template <int BM, int BV> struct Stages {
    static constexpr int bytes = (BK * BM + BV * XLD) * 4;
    static constexpr int v = 3 * bytes <= 48 * 1024 ? 3 : 2;
};
// The split-K decision uses this reference shape whatever shape runs, so it
// (and the rounding it implies) is the same for every variant.
constexpr int kRefBM = 64, kRefBV = 32;

__device__ __forceinline__ void cp16(void *dst, const void *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kStages> __device__ __forceinline__ void cp_wait_stages() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int BM, int RP>
__global__ void __launch_bounds__(128) k_vgemm(VGemm g) {
    constexpr int TR = BM / RP;         // row groups of RP
    constexpr int TV = 128 / TR;        // vector lanes
    constexpr int BV = 4 * TV;          // vectors per block
    constexpr int kStages = Stages<BM, BV>::v;
    static_assert(RP % 4 == 0 && TR * TV == 128, "whole row groups and vector lanes");
    constexpr int XQ = BK / 4;          // 16-byte pieces of one vector's chunk
    constexpr int XP = BV * XQ;         // 16-byte pieces of one X chunk
    constexpr int AP = BM * BK / 4;     // 16-byte pieces of one A chunk
    constexpr int XH = (XP + 127) / 128, AH = AP / 128;
    static_assert(AP % 128 == 0, "whole A pieces per thread");
    __shared__ __align__(16) float As[kStages][BK][BM];     // As[.][j][i]
    __shared__ __align__(16) float Xs[kStages][BV][XLD];    // Xs[.][v][j]
    const int tid = threadIdx.x;
    const int tr = tid / TV, tv = tid % TV;
    const int i0 = blockIdx.y * BM;
    const int v0 = blockIdx.x * BV;
    const int nvec = g.count * g.nrhs;
    const int mp = (g.m + 3) & ~3;

    // the X pieces this thread copies: vector lv[h], quarter lq[h]
    int lv[XH], lq[XH], pos_l[XH], rhs_l[XH];
#pragma unroll
    for (int h = 0; h < XH; ++h) {
        const int q = tid + h * 128;
        lv[h] = q / XQ;
        lq[h] = q % XQ;
        const int vload = v0 + lv[h];
        const bool in = q < XP && vload < nvec;
        pos_l[h] = in ? vload / g.nrhs : -1;
        rhs_l[h] = in ? vload - pos_l[h] * g.nrhs : 0;
    }

    // split-K: block z computes segment z alone
    const bool split = g.part != nullptr;
    const int s_first = split ? (int)blockIdx.z : 0;
    const int s_end = split ? s_first + 1 : g.nseg;
    // A segment with no source row for any vector of this block adds only
    // exact zeros (each of its FMAs adds a * 0 to the sum), so the block
    // skips its chunks and the sums are bit for bit those of the full walk.
    // Only the segments the caller marks sparse are checked (the downward
    // step's X-list segment has rows for a few boxes of a level).  The index
    // tables are constant, so this runs before the programmatic-dependence
    // wait.
    __shared__ uint32_t live_s;
    uint32_t mine = 0, listed = 0;  // checked segments with a row here / checked
    for (int s = s_first; s < s_end; ++s) {
        const VSeg &sg = g.seg[s];
        if (!sg.src_idx || !((g.sparse >> s) & 1u)) continue;
        listed |= 1u << s;
#pragma unroll
        for (int h = 0; h < XH; ++h)
            if (tid + h * 128 < XP && pos_l[h] >= 0 && sg.src_idx[pos_l[h]] >= 0)
                mine |= 1u << s;
    }
    uint32_t live = ((1u << s_end) - 1u) & ~((1u << s_first) - 1u);
    if (listed) {
        if (tid == 0) live_s = 0;
        __syncthreads();
        mine = __reduce_or_sync(0xffffffffu, mine);
        if ((tid & 31) == 0 && mine) atomicOr(&live_s, mine);
        __syncthreads();
        live = (live & ~listed) | live_s;
    }
    int total_chunks = 0;
    for (int s = s_first; s < s_end; ++s)
        if ((live >> s) & 1u) total_chunks += (g.seg[s].n + BK - 1) / BK;

    // the issue side walks the chunks of the live segments in order:
    // segment is_, chunk icc of it, and each X piece's source row for that
    // segment
    int is_ = s_first;
    while (is_ < s_end && !((live >> is_) & 1u)) ++is_;
    int icc = 0, inch = is_ < s_end ? (g.seg[is_].n + BK - 1) / BK : 0;
    const float *xrow[XH];
    auto set_rows = [&](int s) {
        const VSeg &sg = g.seg[s];
#pragma unroll
        for (int h = 0; h < XH; ++h) {
            xrow[h] = nullptr;
            if (tid + h * 128 < XP && pos_l[h] >= 0) {
                const int node = sg.src_idx ? sg.src_idx[pos_l[h]] : sg.src_base + pos_l[h];
                if (node >= 0) xrow[h] = sg.src + ((size_t)node * g.nrhs + rhs_l[h]) * sg.src_ld;
            }
        }
    };
    if (is_ < s_end) set_rows(is_);
    // copy the next chunk (the c-th, flattened over the segments) into stage c % kStages
    auto issue = [&](int c) {
        if (c < total_chunks) {
            while (icc == inch) {
                do {
                    ++is_;
                } while (!((live >> is_) & 1u));
                icc = 0;
                inch = (g.seg[is_].n + BK - 1) / BK;
                set_rows(is_);
            }
            const VSeg &sg = g.seg[is_];
            const int st = c % kStages;
            const int j0 = icc * BK;
#pragma unroll
            for (int h = 0; h < AH; ++h) {
                const int q = tid + h * 128;            // BK rows x BM/4 pieces
                const int jj = q / (BM / 4), ii = (q % (BM / 4)) * 4;
                const int j = j0 + jj, i = i0 + ii;
                const bool in = j < sg.n && i < mp;
                cp16(&As[st][jj][ii], in ? sg.AT + (size_t)j * mp + i : sg.AT, in ? 16 : 0);
            }
#pragma unroll
            for (int h = 0; h < XH; ++h) {
                if (tid + h * 128 >= XP) continue;
                int bytes = 0;
                const float *src = sg.src;
                const int j = j0 + lq[h] * 4;
                if (xrow[h] && j < sg.n) {
                    src = xrow[h] + j;
                    bytes = 4 * min(4, sg.n - j);
                }
                cp16(&Xs[st][lv[h]][lq[h] * 4], src, bytes);
            }
            ++icc;
        }
        cp_commit();
    };

    float acc[RP][4];
#pragma unroll
    for (int a = 0; a < RP; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

    // Launched as a programmatic dependent of the previous kernel in the
    // stream: everything above reads only kernel parameters and the plan's
    // constant index tables, so it overlaps that kernel's tail; the vectors
    // and add rows it produced are read only after this wait.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int c = 0; c < kStages - 1; ++c) issue(c);
    for (int c = 0; c < total_chunks; ++c) {
        issue(c + kStages - 1);
        cp_wait_stages<kStages>();
        __syncthreads();
        const int st = c % kStages;
#pragma unroll
        for (int k4 = 0; k4 < BK; k4 += 4) {
            float x[4][4];  // x[vec][kk]
            if constexpr (RP == 4) {
                float a[4][4];  // a[kk][row]
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 t = *reinterpret_cast<const float4 *>(&As[st][k4 + e][tr * 4]);
                    a[e][0] = t.x; a[e][1] = t.y; a[e][2] = t.z; a[e][3] = t.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4 *>(&Xs[st][tv + TV * q][k4]);
                    x[q][0] = t.x; x[q][1] = t.y; x[q][2] = t.z; x[q][3] = t.w;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[e][p], x[q][e], acc[p][q]);
            } else {
                // wide tiles: the vectors first, then one k of A rows at a time
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4 *>(&Xs[st][tv + TV * q][k4]);
                    x[q][0] = t.x; x[q][1] = t.y; x[q][2] = t.z; x[q][3] = t.w;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float a[RP];
#pragma unroll
                    for (int g4 = 0; g4 < RP / 4; ++g4) {
                        const float4 t = *reinterpret_cast<const float4 *>(
                            &As[st][k4 + e][tr * RP + 4 * g4]);
                        a[4 * g4] = t.x; a[4 * g4 + 1] = t.y;
                        a[4 * g4 + 2] = t.z; a[4 * g4 + 3] = t.w;
                    }
#pragma unroll
                    for (int p = 0; p < RP; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], x[q][e], acc[p][q]);
                }
            }
        }
        __syncthreads();
    }
    cp_wait_all();

    // epilogue
    if (split) {
        // partial product of segment z (scaled: the scale is per row, linear)
        float *pz = g.part + (size_t)blockIdx.z * nvec * mp;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int v = v0 + tv + TV * q;
            if (v >= nvec) continue;
#pragma unroll
            for (int p = 0; p < RP; ++p) {
                const int i = i0 + tr * RP + p;
                if (i >= g.m) continue;
                pz[(size_t)v * mp + i] = g.scale ? acc[p][q] * __ldg(g.scale + i) : acc[p][q];
            }
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = v0 + tv + TV * q;
        if (v >= nvec) continue;
        const int pos = v / g.nrhs, rhs = v - pos * g.nrhs;
        const int dnode = g.dst_idx ? g.dst_idx[pos] : g.dst_base + pos;
        if (dnode < 0) continue;
        float *drow = g.dst + ((size_t)dnode * g.nrhs + rhs) * g.dst_ld;
        const float *arow = nullptr;
        if (g.add) {
            const int an = g.add_idx ? g.add_idx[pos] : pos;
            if (an >= 0)
                arow = g.add + ((size_t)an * g.nrhs + rhs) * g.add_ld + (g.add_off ? g.add_off[pos] : 0);
        }
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            const int i = i0 + tr * RP + p;
            if (i >= g.m) continue;
            float r = acc[p][q];
            if (g.scale) r *= __ldg(g.scale + i);
            if (arow) r += arow[i];
            drow[i] = r;
        }
    }
}

// Sum of the nseg partial products in segment order, then the add row and
// the scatter of the unsplit epilogue.
__global__ void k_vreduce(VGemm g) {
    const int nvec = g.count * g.nrhs;
    const int mp = (g.m + 3) & ~3;
    const int64_t total = (int64_t)nvec * g.m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / g.m), i = (int)(t - (int64_t)v * g.m);
        float r = 0.f;
        for (int z = 0; z < g.nseg; ++z) r += g.part[((size_t)z * nvec + v) * mp + i];
        const int pos = v / g.nrhs, rhs = v - pos * g.nrhs;
        const int dnode = g.dst_idx ? g.dst_idx[pos] : g.dst_base + pos;
        if (dnode < 0) continue;
        if (g.add) {
            const int an = g.add_idx ? g.add_idx[pos] : pos;
            if (an >= 0)
                r += g.add[((size_t)an * g.nrhs + rhs) * g.add_ld + (g.add_off ? g.add_off[pos] : 0) + i];
        }
        g.dst[((size_t)dnode * g.nrhs + rhs) * g.dst_ld + i] = r;
    }
}

// The decision looks at the box count only, not at nrhs, so every column of
// an evaluation gets the same summation order whatever nrhs it is batched in.
bool wants_split(int m, int count, int nseg) {
    const int64_t blocks = (((int64_t)count + kRefBV - 1) / kRefBV) * ((m + kRefBM - 1) / kRefBM);
    return nseg > 1 && blocks < kSplitBlocks;
}

template <int BM, int RP>
cudaError_t launch_shape(const VGemm &g, int nvec, bool split, cudaStream_t s) {
    constexpr int BV = 4 * (128 / (BM / RP));
    const dim3 grid((nvec + BV - 1) / BV, (g.m + BM - 1) / BM, split ? g.nseg : 1);
    if (grid.y > 65535u || grid.x > 2147483647u) return cudaErrorInvalidValue;
    // programmatic dependent launch: the blocks may start (and run their
    // prologue) while the previous kernel of the stream finishes
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_vgemm<BM, RP>, g);
}

} // namespace

size_t vgemm_split_floats(int m, int count, int nrhs, int nseg) {
    if (!wants_split(m, count, nseg)) return 0;
    return (size_t)nseg * count * nrhs * ((m + 3) & ~3);
}

cudaError_t launch_vgemm(const VGemm &g0, cudaStream_t s, int shape) {
    if (g0.count == 0) return cudaSuccess;
    if (g0.nseg < 1 || g0.nseg > kMaxSeg) return cudaErrorInvalidValue;
    for (int k = 0; k < g0.nseg; ++k)
        if ((g0.seg[k].src_ld & 3) != 0) return cudaErrorInvalidValue;  // 16-byte rows
    VGemm g = g0;
    const bool split = g.part && wants_split(g.m, g.count, g.nseg);
    if (!split) g.part = nullptr;
    const int nvec = g.count * g.nrhs;
    cudaError_t e = shape == 1   ? launch_shape<32, 4>(g, nvec, split, s)
                    : shape == 2 ? launch_shape<128, 4>(g, nvec, split, s)
                    : shape == 3 ? launch_shape<64, 8>(g, nvec, split, s)
                    : shape == 4 ? launch_shape<128, 8>(g, nvec, split, s)
                                 : launch_shape<64, 4>(g, nvec, split, s);
    if (!split || e != cudaSuccess) return e;
    const int64_t total = (int64_t)nvec * g.m;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_vreduce<<<blocks, 256, 0, s>>>(g);
    return cudaGetLastError();
}

} // namespace kifmm
