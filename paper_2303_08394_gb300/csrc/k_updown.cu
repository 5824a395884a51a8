// Upward and downward passes ("Computational structure of FMM operators"):
//   P2M  leaf points -> upward check potential -> upward equivalent density
//   M2M  children's upward densities -> parent's upward density
//   P2L  X-list points -> downward check potential
//   down M2L output + P2L + L2L from the parent -> downward density
// Each pseudo-inverse is applied in factored form (U^T, 1/s, V) in FP32.
// Densities of a box of half-width h are computed in h-normalised
// coordinates; with the 1/r kernel they are then independent of h.
#include "device.cuh"

namespace kifmm {

namespace {

// ys[v*ldy + i] (+)= scale[i] * sum_j AT[j*m + i] * xs[v*ldx + j], i < m, v < nv.
__device__ __forceinline__ void block_mv(const float *__restrict__ AT, int m, int n,
                                         const float *xs, int ldx, int nv, float *ys,
                                         int ldy, const float *__restrict__ scale,
                                         bool accumulate) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float acc[kMaxVec];
#pragma unroll
        for (int v = 0; v < kMaxVec; ++v) acc[v] = 0.f;
        for (int j = 0; j < n; ++j) {
            const float a = __ldg(AT + (size_t)j * m + i);
#pragma unroll
            for (int v = 0; v < kMaxVec; ++v)
                if (v < nv) acc[v] = fmaf(a, xs[v * ldx + j], acc[v]);
        }
        const float sc = scale ? __ldg(scale + i) : 1.f;
#pragma unroll
        for (int v = 0; v < kMaxVec; ++v)
            if (v < nv) {
                float r = sc * acc[v];
                ys[v * ldy + i] = accumulate ? ys[v * ldy + i] + r : r;
            }
    }
}

__device__ __forceinline__ int vec_node(const int *nodes, int first, int count, int v,
                                        int nr) {
    int g = v / nr;
    return first + g < count ? nodes[first + g] : -1;
}

// Writes densities rho (smem, V x ns) to the node arrays and projects them
// on Vk for the M2L: qhat = Vk^T rho.
__device__ void finish_upward(const DevOps &o, const DevWork &w, const int *nodes,
                              int first, int count, int r0, int nr, int nrr, int nv,
                              float *rho, float *tmp) {
    const int ns = o.ns, kp = o.kpad;
    for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
        int v = idx / ns, i = idx - v * ns;
        int node = vec_node(nodes, first, count, v, nr);
        if (node >= 0 && v % nr < nrr)
            w.up[((size_t)node * w.nrhs + r0 + v % nr) * ns + i] = rho[v * ns + i];
    }
    block_mv(o.Vk, kp, ns, rho, ns, nv, tmp, kp, nullptr, false);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nv * kp; idx += blockDim.x) {
        int v = idx / kp, i = idx - v * kp;
        int node = vec_node(nodes, first, count, v, nr);
        if (node >= 0 && v % nr < nrr)
            w.qhat[((size_t)node * w.nrhs + r0 + v % nr) * kp + i] = tmp[v * kp + i];
    }
}

// P2M for a chunk of leaves: check potential of the leaf's points on its
// upward check surface (radius ao, normalised), then y = Pu^T chk / Ps,
// rho = Pv y.
__global__ void __launch_bounds__(256) k_p2m(DevTree t, DevOps o, DevWork w,
                                             const int *nodes, int count, int G, int nr) {
    extern __shared__ float smem[];
    const int ns = o.ns, wide = max(max(ns, o.kpad), o.rP);
    float *bufA = smem;                       // V x wide
    float *bufB = smem + kMaxVec * wide;      // V x wide
    const int first = blockIdx.x * G;
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const int nv = G * nr;
    // 1. check potentials into bufA[v*ns + j]
    for (int idx = threadIdx.x; idx < G * ns; idx += blockDim.x) {
        int g = idx / ns, j = idx - g * ns;
        float acc[kMaxVec];
#pragma unroll
        for (int v = 0; v < kMaxVec; ++v) acc[v] = 0.f;
        if (first + g < count) {
            int node = nodes[first + g];
            float4 gm = t.geom[node];
            float inv_h = 1.f / gm.w;
            int2 rg = t.range[node];
            float4 s = o.surf[j];
            float cx = o.ao * s.x, cy = o.ao * s.y, cz = o.ao * s.z;
            for (int i = rg.x; i < rg.y; ++i) {
                float4 p = t.pts[i];
                float dx = cx - p.x * inv_h, dy = cy - p.y * inv_h, dz = cz - p.z * inv_h;
                float r2 = dx * dx + dy * dy + dz * dz;
                float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                const float *q = w.qs + (size_t)i * w.nrhs + r0;
#pragma unroll
                for (int r = 0; r < kMaxVec; ++r)
                    if (r < nrr) acc[r] = fmaf(__ldg(q + r), inv, acc[r]);
            }
        }
        for (int r = 0; r < nr; ++r) bufA[(g * nr + r) * ns + j] = r < nrr ? acc[r] : 0.f;
    }
    __syncthreads();
    block_mv(o.Pu, o.rP, ns, bufA, ns, nv, bufB, o.rP, o.Ps_inv, false);
    __syncthreads();
    block_mv(o.PvT, ns, o.rP, bufB, o.rP, nv, bufA, ns, nullptr, false);
    __syncthreads();
    finish_upward(o, w, nodes, first, count, r0, nr, nrr, nv, bufA, bufB);
}

// M2M for a chunk of internal nodes of one level: y = sum_sigma M2M_sigma
// rho_child(sigma), then rho = Pv (y / Ps).
__global__ void __launch_bounds__(256) k_m2m(DevTree t, DevOps o, DevWork w,
                                             const int *nodes, int count, int G, int nr) {
    extern __shared__ float smem[];
    const int ns = o.ns, wide = max(max(ns, o.kpad), o.rP);
    float *bufA = smem, *bufB = smem + kMaxVec * wide, *bufC = bufB + kMaxVec * wide;
    const int first = blockIdx.x * G;
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const int nv = G * nr;
    for (int sg = 0; sg < 8; ++sg) {
        for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
            int v = idx / ns, j = idx - v * ns;
            int node = vec_node(nodes, first, count, v, nr);
            int r = v % nr;
            float x = 0.f;
            if (node >= 0 && r < nrr) {
                int ch = t.child[node * 8 + sg];
                if (ch >= 0) x = w.up[((size_t)ch * w.nrhs + r0 + r) * ns + j];
            }
            bufA[v * ns + j] = x;
        }
        __syncthreads();
        block_mv(o.M2M + (size_t)sg * ns * o.rP, o.rP, ns, bufA, ns, nv, bufB, o.rP,
                 nullptr, sg > 0);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nv * o.rP; idx += blockDim.x)
        bufB[idx] *= o.Ps_inv[idx % o.rP];
    __syncthreads();
    block_mv(o.PvT, ns, o.rP, bufB, o.rP, nv, bufA, ns, nullptr, false);
    __syncthreads();
    finish_upward(o, w, nodes, first, count, r0, nr, nrr, nv, bufA, bufC);
}

// P2L: downward check potential of box B (radius ai, normalised by h_B)
// from the points of every leaf in X(B).
__global__ void __launch_bounds__(128) k_p2l(DevTree t, DevOps o, DevWork w,
                                             const int *nodes, int nr) {
    __shared__ float4 spos[128];
    __shared__ float sq[kMaxVec][128];
    const int b = nodes[blockIdx.x];
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const float4 gb = t.geom[b];
    const float inv_h = 1.f / gb.w;
    const int ns = o.ns;
    const int slot = t.x_slot[b];
    for (int j0 = 0; j0 < ns; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        float4 s = o.surf[min(j, ns - 1)];
        const float cx = o.ai * s.x, cy = o.ai * s.y, cz = o.ai * s.z;
        float acc[kMaxVec];
#pragma unroll
        for (int r = 0; r < kMaxVec; ++r) acc[r] = 0.f;
        for (int e = t.x_ptr[b]; e < t.x_ptr[b + 1]; ++e) {
            const int a = t.x_idx[e];
            const float4 ga = t.geom[a];
            const float sx = (ga.x - gb.x) * inv_h, sy = (ga.y - gb.y) * inv_h,
                        sz = (ga.z - gb.z) * inv_h;
            const int2 rg = t.range[a];
            for (int i0 = rg.x; i0 < rg.y; i0 += blockDim.x) {
                __syncthreads();
                const int i = i0 + threadIdx.x;
                if (i < rg.y) {
                    float4 p = t.pts[i];
                    spos[threadIdx.x] = make_float4(p.x * inv_h + sx, p.y * inv_h + sy,
                                                    p.z * inv_h + sz, 0.f);
                    for (int r = 0; r < nrr; ++r)
                        sq[r][threadIdx.x] = w.qs[(size_t)i * w.nrhs + r0 + r];
                }
                __syncthreads();
                const int cnt = min((int)blockDim.x, rg.y - i0);
                for (int q = 0; q < cnt; ++q) {
                    float dx = cx - spos[q].x, dy = cy - spos[q].y, dz = cz - spos[q].z;
                    float r2 = dx * dx + dy * dy + dz * dz;
                    float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
#pragma unroll
                    for (int r = 0; r < kMaxVec; ++r)
                        if (r < nrr) acc[r] = fmaf(sq[r][q], inv, acc[r]);
                }
            }
        }
        if (j < ns)
            for (int r = 0; r < nrr; ++r)
                w.xchk[((size_t)slot * w.nrhs + r0 + r) * ns + j] = acc[r];
    }
}

// Downward step for a chunk of same-level nodes sharing child position
// sigma: y = (Qu^T Uk) chat + Qu^T xchk + L2L_sigma rho_parent,
// rho = Qv (y / Qs).
__global__ void __launch_bounds__(256) k_down(DevTree t, DevOps o, DevWork w,
                                              const int *chunks, const int *nodes, int nr) {
    extern __shared__ float smem[];
    const int ns = o.ns, kp = o.kpad, rQ = o.rQ;
    const int wide = max(max(ns, kp), rQ);
    float *bufA = smem, *bufB = smem + kMaxVec * wide;
    const int *ch = chunks + 4 * blockIdx.x;
    const int sg = ch[2], level = ch[3];
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const int G = kMaxVec / nr;
    const int nv = G * nr;
    for (int g0 = 0; g0 < ch[1]; g0 += G) {
        const int *my = nodes + ch[0] + g0;
        const int count = min(G, ch[1] - g0);
        // M2L output, projected out: y = (Qu^T Uk) chat
        for (int idx = threadIdx.x; idx < nv * kp; idx += blockDim.x) {
            int v = idx / kp, j = idx - v * kp;
            int g = v / nr, r = v % nr;
            float x = 0.f;
            if (g < count && r < nrr) {
                int b = my[g];
                if (t.v_ptr[b + 1] > t.v_ptr[b])
                    x = w.chat[((size_t)b * w.nrhs + r0 + r) * kp + j];
            }
            bufA[v * kp + j] = x;
        }
        __syncthreads();
        block_mv(o.QUkT, rQ, kp, bufA, kp, nv, bufB, rQ, nullptr, false);
        __syncthreads();
        // P2L check potentials: y += Qu^T xchk
        bool any_x = false;
        for (int g = 0; g < count; ++g) any_x |= t.x_slot[my[g]] >= 0;
        if (any_x) {
            for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
                int v = idx / ns, j = idx - v * ns;
                int g = v / nr, r = v % nr;
                float x = 0.f;
                if (g < count && r < nrr) {
                    int slot = t.x_slot[my[g]];
                    if (slot >= 0) x = w.xchk[((size_t)slot * w.nrhs + r0 + r) * ns + j];
                }
                bufA[v * ns + j] = x;
            }
            __syncthreads();
            block_mv(o.Qu, rQ, ns, bufA, ns, nv, bufB, rQ, nullptr, true);
            __syncthreads();
        }
        // L2L from the parent (local expansions exist from level 2 on)
        if (level >= 3) {
            for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
                int v = idx / ns, j = idx - v * ns;
                int g = v / nr, r = v % nr;
                float x = 0.f;
                if (g < count && r < nrr) {
                    int par = t.parent[my[g]];
                    x = w.down[((size_t)par * w.nrhs + r0 + r) * ns + j];
                }
                bufA[v * ns + j] = x;
            }
            __syncthreads();
            block_mv(o.L2L + (size_t)sg * ns * rQ, rQ, ns, bufA, ns, nv, bufB, rQ, nullptr,
                     true);
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < nv * rQ; idx += blockDim.x)
            bufB[idx] *= o.Qs_inv[idx % rQ];
        __syncthreads();
        block_mv(o.QvT, ns, rQ, bufB, rQ, nv, bufA, ns, nullptr, false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
            int v = idx / ns, j = idx - v * ns;
            int g = v / nr, r = v % nr;
            if (g < count && r < nrr)
                w.down[((size_t)my[g] * w.nrhs + r0 + r) * ns + j] = bufA[v * ns + j];
        }
        __syncthreads();
    }
}

__global__ void k_gather_charges(DevTree t, DevWork w) {
    const int64_t total = t.n * (int64_t)w.nrhs;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / w.nrhs, r = idx - i * w.nrhs;
        w.qs[idx] = w.charges_user[t.perm[i] * w.nrhs + r];
    }
}

inline int rhs_chunk(int nrhs) { return nrhs < kMaxVec ? nrhs : kMaxVec; }

size_t mv_smem(const DevOps &o, int bufs) {
    int wide = o.ns;
    if (o.kpad > wide) wide = o.kpad;
    if (o.rP > wide) wide = o.rP;
    if (o.rQ > wide) wide = o.rQ;
    return (size_t)bufs * kMaxVec * wide * sizeof(float);
}

} // namespace

cudaError_t launch_gather_charges(const DevTree &t, const DevWork &w, cudaStream_t s) {
    int64_t total = t.n * (int64_t)w.nrhs;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_gather_charges<<<blocks, 256, 0, s>>>(t, w);
    return cudaGetLastError();
}

cudaError_t launch_p2m(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    int nr = rhs_chunk(w.nrhs), G = kMaxVec / nr;
    dim3 grid((count + G - 1) / G, (w.nrhs + nr - 1) / nr);
    size_t sm = mv_smem(o, 2);
    cudaError_t e = cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_p2m<<<grid, 256, sm, s>>>(t, o, w, nodes, count, G, nr);
    return cudaGetLastError();
}

cudaError_t launch_m2m(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    int nr = rhs_chunk(w.nrhs), G = kMaxVec / nr;
    dim3 grid((count + G - 1) / G, (w.nrhs + nr - 1) / nr);
    size_t sm = mv_smem(o, 3);
    cudaError_t e = cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_m2m<<<grid, 256, sm, s>>>(t, o, w, nodes, count, G, nr);
    return cudaGetLastError();
}

cudaError_t launch_p2l(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    int nr = rhs_chunk(w.nrhs);
    dim3 grid(count, (w.nrhs + nr - 1) / nr);
    k_p2l<<<grid, 128, 0, s>>>(t, o, w, nodes, nr);
    return cudaGetLastError();
}

cudaError_t launch_down(const DevTree &t, const DevOps &o, const DevWork &w, const int *chunks,
                        const int *nodes, int nchunks, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    int nr = rhs_chunk(w.nrhs);
    dim3 grid(nchunks, (w.nrhs + nr - 1) / nr);
    size_t sm = mv_smem(o, 2);
    cudaError_t e = cudaFuncSetAttribute(k_down, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_down<<<grid, 256, sm, s>>>(t, o, w, chunks, nodes, nr);
    return cudaGetLastError();
}

} // namespace kifmm
