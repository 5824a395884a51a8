// Point-to-surface evaluations of the upward and downward passes
// ("Computational structure of FMM operators"):
//   P2M check  leaf points -> upward check potential (radius ao)
//   P2L        X-list points -> downward check potential (radius ai)
// both in coordinates normalised by the receiving box's half-width; the
// matrix products that follow them run in k_vgemm.cu.  Also the gather of
// the caller's charges into tree order (points that are targets only get
// charge 0).
#include <algorithm>

#include "device.cuh"

namespace kifmm {

namespace {

// Upward check potential of leaf nodes[pos] at its ns check points for NR
// right-hand sides from r0: one block per leaf, one thread per check point
// (the block is ns rounded up to a warp).  The leaf's points are staged in
// shared memory, scaled to leaf units (an exact power-of-two scaling), with
// the charge in the w slot when NR is 1; each check point sums them in
// order.  No pair coincides: the points lie in the leaf's cube (half-width
// 1 in leaf units) and the check surface on the cube of half-width
// alpha_outer > 1, at least alpha_outer - 1 away.
template <int NR>
__global__ void __launch_bounds__(512) k_p2m_check(DevTree t, DevOps o, DevWork w,
                                                   const int *nodes, int count, float *chk,
                                                   int ld, int r0) {
    extern __shared__ float4 p2m_smem[];
    float4 *spos = p2m_smem;                                     // blockDim
    float *sq = reinterpret_cast<float *>(spos + blockDim.x);    // blockDim x NR (NR > 1)
    const int ns = o.ns;
    const int j = threadIdx.x;
    const float4 s = o.surf[min(j, ns - 1)];
    const float cx = o.ao * s.x, cy = o.ao * s.y, cz = o.ao * s.z;
    for (int pos = blockIdx.x; pos < count; pos += gridDim.x) {
        const int node = nodes[pos];
        const float inv_h = 1.f / t.geom[node].w;
        const int2 rg = t.range[node];
        float acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = 0.f;
        for (int i0 = rg.x; i0 < rg.y; i0 += blockDim.x) {
            __syncthreads();
            const int i = i0 + threadIdx.x;
            if (i < rg.y) {
                const float4 p = __ldg(t.pts + i);
                float4 v = make_float4(p.x * inv_h, p.y * inv_h, p.z * inv_h, 0.f);
                const float *qi = w.qs + (size_t)i * w.nrhs + r0;
                if constexpr (NR == 1) {
                    v.w = __ldg(qi);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) sq[threadIdx.x * NR + r] = __ldg(qi + r);
                }
                spos[threadIdx.x] = v;
            }
            __syncthreads();
            const int cnt = min((int)blockDim.x, rg.y - i0);
#pragma unroll 4
            for (int c = 0; c < cnt; ++c) {
                const float4 v = spos[c];
                const float dx = cx - v.x, dy = cy - v.y, dz = cz - v.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float inv = KIFMM_RSQRT(r2);
                if constexpr (NR == 1) {
                    acc[0] = fmaf(v.w, inv, acc[0]);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] = fmaf(sq[c * NR + r], inv, acc[r]);
                }
            }
        }
        if (j < ns) {
#pragma unroll
            for (int r = 0; r < NR; ++r) chk[((size_t)pos * w.nrhs + r0 + r) * ld + j] = acc[r];
        }
    }
}

// P2L: downward check potential of box B (radius ai, normalised by h_B)
// from the points of every leaf in X(B), for NR right-hand sides from r0.
// One block per box; thread j holds the check points j + nthr i (i < T).
// The X leaves are laid end to end as segments of one source list, staged
// in rounds of up to kXCap sources into shared memory, shifted into B's
// frame (charges in the w slot when NR is 1), one barrier pair per round
// however many leaves; each check point sums its sources in list order.  No
// pair coincides: an X(B) leaf does not touch B, so it lies at least one
// B-width from it, and the check surface reaches only 0.05 h_B beyond B.
constexpr int kXCap = 512;      // staged sources per round
constexpr int kXSegCap = 64;    // X leaves per table window (at most one per thread)
constexpr int kXMaxWarps = 16;

template <int NR> struct P2LSmem {
    float4 spos[kXCap];                    // position in B's units, charge in w (NR = 1)
    float sq[NR > 1 ? kXCap * NR : 1];     // charges (NR > 1)
    float4 seg_shift[kXSegCap];            // (leaf centre - B's centre) / h_B
    int seg_first[kXSegCap], seg_start[kXSegCap + 1];
    int warp_sum[kXMaxWarps];
};

template <int NR, int T>
__global__ void __launch_bounds__(512) k_p2l(DevTree t, DevOps o, DevWork w, const int *nodes,
                                             int r0) {
    __shared__ __align__(16) P2LSmem<NR> sm;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    const int b = nodes[blockIdx.x];
    const float4 gb = t.geom[b];
    const float inv_h = 1.f / gb.w;
    const int ns = o.ns, nsp = (o.ns + 3) & ~3;
    float cx[T], cy[T], cz[T], acc[T][NR];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const float4 s = o.surf[min(tid + nthr * i, ns - 1)];
        cx[i] = o.ai * s.x;
        cy[i] = o.ai * s.y;
        cz[i] = o.ai * s.z;
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[i][r] = 0.f;
    }
    const int l0 = t.x_ptr[b], nlist = t.x_ptr[b + 1] - l0;
    const int segcap = min(kXSegCap, nthr);
    for (int sw = 0; sw < nlist; sw += segcap) {
        const int nsegw = min(segcap, nlist - sw);
        // ---- segment table: the window's X leaves, shifts and offsets
        int c = 0;
        if (tid < nsegw) {
            const int a = t.x_idx[l0 + sw + tid];
            const int2 ra = t.range[a];
            const float4 ga = t.geom[a];
            c = ra.y - ra.x;
            sm.seg_first[tid] = ra.x;
            sm.seg_shift[tid] = make_float4((ga.x - gb.x) * inv_h, (ga.y - gb.y) * inv_h,
                                            (ga.z - gb.z) * inv_h, 0.f);
        }
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) sm.warp_sum[wid] = incl;
        __syncthreads();
        int base_w = 0, total = 0;
        for (int k = 0; k < nwarps; ++k) {
            const int v = sm.warp_sum[k];
            if (k < wid) base_w += v;
            total += v;
        }
        if (tid < nsegw) sm.seg_start[tid] = base_w + incl - c;
        if (tid == 0) sm.seg_start[nsegw] = total;
        __syncthreads();

        // ---- rounds of at most kXCap staged sources
        int seg = 0;  // segment of this thread's next source (sources ascend)
        for (int base = 0; base < total; base += kXCap) {
            const int m = min(kXCap, total - base);
            for (int k = tid; k < m; k += nthr) {
                // f < total = seg_start[nsegw], so the scan stops below nsegw
                const int f = base + k;
                while (sm.seg_start[seg + 1] <= f) ++seg;
                const int i = sm.seg_first[seg] + f - sm.seg_start[seg];
                const float4 p = __ldg(t.pts + i);
                const float4 sh = sm.seg_shift[seg];
                float4 v = make_float4(fmaf(p.x, inv_h, sh.x), fmaf(p.y, inv_h, sh.y),
                                       fmaf(p.z, inv_h, sh.z), 0.f);
                const float *qi = w.qs + (size_t)i * w.nrhs + r0;
                if constexpr (NR == 1) {
                    v.w = __ldg(qi);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) sm.sq[k * NR + r] = __ldg(qi + r);
                }
                sm.spos[k] = v;
            }
            __syncthreads();
#pragma unroll 2
            for (int cc = 0; cc < m; ++cc) {
                const float4 v = sm.spos[cc];
                float q[NR];
                if constexpr (NR == 1) {
                    q[0] = v.w;
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) q[r] = sm.sq[cc * NR + r];
                }
#pragma unroll
                for (int i = 0; i < T; ++i) {
                    const float dx = cx[i] - v.x, dy = cy[i] - v.y, dz = cz[i] - v.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float inv = KIFMM_RSQRT(r2);
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[i][r] = fmaf(q[r], inv, acc[i][r]);
                }
            }
            __syncthreads();
        }
    }
    const size_t slot = (size_t)t.x_slot[b];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const int j = tid + nthr * i;
        if (j >= ns) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r) w.xchk[(slot * w.nrhs + r0 + r) * nsp + j] = acc[i][r];
    }
}

__global__ void k_gather_charges(DevTree t, DevWork w) {
    const int64_t total = t.n * (int64_t)w.nrhs;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / w.nrhs, r = idx - i * w.nrhs;
        const int64_t c = t.qidx[i];
        w.qs[idx] = c >= 0 ? w.charges_user[c * w.nrhs + r] : 0.f;
    }
}

} // namespace

cudaError_t launch_gather_charges(const DevTree &t, const DevWork &w, cudaStream_t s) {
    const int64_t total = t.n * (int64_t)w.nrhs;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_gather_charges<<<blocks, 256, 0, s>>>(t, w);
    return cudaGetLastError();
}

template <int NR>
cudaError_t p2m_check_nr(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                         int count, float *chk, int ld, int r0, cudaStream_t s) {
    const int threads = (o.ns + 31) & ~31;
    if (threads > 512) return cudaErrorInvalidValue;
    const size_t smem = (size_t)threads * 16 + (NR > 1 ? (size_t)threads * NR * 4 : 0);
    const int blocks = count < 152 * 64 ? count : 152 * 64;
    k_p2m_check<NR><<<blocks, threads, smem, s>>>(t, o, w, nodes, count, chk, ld, r0);
    return cudaGetLastError();
}

cudaError_t launch_p2m_check(const DevTree &t, const DevOps &o, const DevWork &w,
                             const int *nodes, int count, float *chk, int ld, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int r0 = 0; r0 < w.nrhs && e == cudaSuccess;) {
        const int left = w.nrhs - r0;
        if (left >= 8) { e = p2m_check_nr<8>(t, o, w, nodes, count, chk, ld, r0, s); r0 += 8; }
        else if (left >= 4) { e = p2m_check_nr<4>(t, o, w, nodes, count, chk, ld, r0, s); r0 += 4; }
        else if (left >= 2) { e = p2m_check_nr<2>(t, o, w, nodes, count, chk, ld, r0, s); r0 += 2; }
        else { e = p2m_check_nr<1>(t, o, w, nodes, count, chk, ld, r0, s); r0 += 1; }
    }
    return e;
}

cudaError_t launch_p2l(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    // two check points per thread
    constexpr int T = 2;
    const int threads = ((o.ns + T - 1) / T + 31) & ~31;
    if (threads > 32 * kXMaxWarps) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int r0 = 0; r0 < w.nrhs && e == cudaSuccess;) {
        const int left = w.nrhs - r0;
        const int nr = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        if (nr == 8) k_p2l<8, T><<<count, threads, 0, s>>>(t, o, w, nodes, r0);
        else if (nr == 4) k_p2l<4, T><<<count, threads, 0, s>>>(t, o, w, nodes, r0);
        else if (nr == 2) k_p2l<2, T><<<count, threads, 0, s>>>(t, o, w, nodes, r0);
        else k_p2l<1, T><<<count, threads, 0, s>>>(t, o, w, nodes, r0);
        e = cudaGetLastError();
        r0 += nr;
    }
    return e;
}

} // namespace kifmm
