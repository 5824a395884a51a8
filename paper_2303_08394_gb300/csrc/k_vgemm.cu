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
// Tiling: a block computes 64 output rows x 32 vectors, 128 threads, each a
// 4 x 4 register tile; K advances in chunks of 16 through shared memory
// (operands read as float4).  The next chunk is loaded into registers while
// the current one is multiplied.
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int BM = 64, BV = 32, BK = 16;

__device__ __forceinline__ float4 load_vec4(const float *row, int j, int n) {
    // four consecutive elements of a source row, zero past its end
    if (j + 4 <= n && ((reinterpret_cast<uintptr_t>(row + j) & 15) == 0))
        return __ldg(reinterpret_cast<const float4 *>(row + j));
    float4 r;
    r.x = j + 0 < n ? __ldg(row + j + 0) : 0.f;
    r.y = j + 1 < n ? __ldg(row + j + 1) : 0.f;
    r.z = j + 2 < n ? __ldg(row + j + 2) : 0.f;
    r.w = j + 3 < n ? __ldg(row + j + 3) : 0.f;
    return r;
}

__global__ void __launch_bounds__(128) k_vgemm(VGemm g) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Xs[2][BK][BV + 4];
    const int tid = threadIdx.x;
    const int tr = tid >> 3, tv = tid & 7;         // 16 row groups x 8 vector groups
    const int i0 = blockIdx.y * BM;
    const int v0 = blockIdx.x * BV;
    const int nvec = g.count * g.nrhs;

    // the vector this thread loads for the X tile, and its list position
    const int lv = tid >> 2, lq = tid & 3;          // 32 vectors x 4 float4 pieces
    const int vload = v0 + lv;
    const int pos_l = vload < nvec ? vload / g.nrhs : -1;
    const int rhs_l = vload < nvec ? vload - pos_l * g.nrhs : 0;

    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

    // flattened K chunks over all segments
    int total_chunks = 0;
    for (int s = 0; s < g.nseg; ++s) total_chunks += (g.seg[s].n + BK - 1) / BK;

    float4 ra[2], rx;
    auto fetch = [&](int chunk) {
        int s = 0, c = chunk;
        while (c >= (g.seg[s].n + BK - 1) / BK) {
            c -= (g.seg[s].n + BK - 1) / BK;
            ++s;
        }
        const VSeg &sg = g.seg[s];
        const int j0 = c * BK;
        const int mp = (g.m + 3) & ~3;
        // A: 16 rows (j) x 64 columns (i) of AT, 2 float4 per thread
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = tid + h * 128;            // 0..255
            const int jj = q >> 4, ii = (q & 15) * 4;
            const int j = j0 + jj, i = i0 + ii;
            if (j < sg.n && i < mp)
                ra[h] = __ldg(reinterpret_cast<const float4 *>(sg.AT + (size_t)j * mp + i));
            else
                ra[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // X: 32 vectors x 16 elements, 1 float4 per thread
        rx = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pos_l >= 0) {
            const int node = sg.src_idx ? sg.src_idx[pos_l] : sg.src_base + pos_l;
            if (node >= 0) {
                const float *row = sg.src + ((size_t)node * g.nrhs + rhs_l) * sg.src_ld;
                rx = load_vec4(row, j0 + lq * 4, sg.n);
            }
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = tid + h * 128;
            *reinterpret_cast<float4 *>(&As[buf][q >> 4][(q & 15) * 4]) = ra[h];
        }
        Xs[buf][lq * 4 + 0][lv] = rx.x;
        Xs[buf][lq * 4 + 1][lv] = rx.y;
        Xs[buf][lq * 4 + 2][lv] = rx.z;
        Xs[buf][lq * 4 + 3][lv] = rx.w;
    };

    if (total_chunks > 0) {
        fetch(0);
        stash(0);
        __syncthreads();
    }
    for (int c = 0; c < total_chunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < total_chunks) fetch(c + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[buf][kk][tr * 4]);
            const float4 x = *reinterpret_cast<const float4 *>(&Xs[buf][kk][tv * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], xv[q], acc[p][q]);
        }
        if (c + 1 < total_chunks) {
            stash(buf ^ 1);
            __syncthreads();
        }
    }

    // epilogue
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = v0 + tv * 4 + q;
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
        for (int p = 0; p < 4; ++p) {
            const int i = i0 + tr * 4 + p;
            if (i >= g.m) continue;
            float r = acc[p][q];
            if (g.scale) r *= __ldg(g.scale + i);
            if (arow) r += arow[i];
            drow[i] = r;
        }
    }
}

} // namespace

cudaError_t launch_vgemm(const VGemm &g, cudaStream_t s) {
    if (g.count == 0) return cudaSuccess;
    if (g.nseg < 1 || g.nseg > kMaxSeg) return cudaErrorInvalidValue;
    const int nvec = g.count * g.nrhs;
    const dim3 grid((nvec + BV - 1) / BV, (g.m + BM - 1) / BM);
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    k_vgemm<<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

} // namespace kifmm
