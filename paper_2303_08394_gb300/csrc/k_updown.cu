// Upward and downward passes ("Computational structure of FMM operators"):
//   P2M  leaf points -> upward check potential -> upward equivalent density
//   M2M  children's upward densities -> parent's upward density
//   P2L  X-list points -> downward check potential
//   down M2L output + P2L + L2L from the parent -> downward density
// Each pseudo-inverse is applied in factored form (U^T, 1/s, V) in FP32.
// Densities of a box of half-width h are computed in h-normalised
// coordinates; with the 1/r kernel they are then independent of h.
//
// A block handles up to kMaxVec vectors (node x right-hand side).  In
// shared memory every vector occupies `ld` floats (smem_width(), a multiple
// of 4), so vector rows are 16-byte aligned.
#include "device.cuh"

namespace kifmm {

namespace {

__host__ __device__ inline int smem_width(const DevOps &o) {
    int w = o.ns;
    if (o.kpad > w) w = o.kpad;
    if (o.rP > w) w = o.rP;
    if (o.rQ > w) w = o.rQ;
    return (w + 3) & ~3;
}

// ys[v*ld + i] (+)= scale[i] * sum_j AT[j*m + i] * xs[v*ld + j], i < m, v < nv.
// Work items are (row i, group of 8 vectors); four matrix loads are issued
// before their FMAs so each thread keeps several L2 requests in flight, and
// the vector operands are read from shared memory as float4.  Rows of xs
// beyond nv may hold stale data: their sums are never stored.
__device__ __forceinline__ void block_mv(const float *__restrict__ AT, int m, int n,
                                         const float *xs, int nv, float *ys, int ld,
                                         const float *__restrict__ scale, bool accumulate) {
    const int ngroups = (nv + 7) >> 3;
    for (int item = threadIdx.x; item < m * ngroups; item += blockDim.x) {
        const int g = item / m, i = item - g * m;
        const float *x0 = xs + (size_t)(g * 8) * ld;
        float acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0.f;
        int j = 0;
        for (; j + 4 <= n; j += 4) {
            const float a0 = __ldg(AT + (size_t)(j + 0) * m + i);
            const float a1 = __ldg(AT + (size_t)(j + 1) * m + i);
            const float a2 = __ldg(AT + (size_t)(j + 2) * m + i);
            const float a3 = __ldg(AT + (size_t)(j + 3) * m + i);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float4 x = *reinterpret_cast<const float4 *>(x0 + v * ld + j);
                acc[v] = fmaf(a0, x.x, acc[v]);
                acc[v] = fmaf(a1, x.y, acc[v]);
                acc[v] = fmaf(a2, x.z, acc[v]);
                acc[v] = fmaf(a3, x.w, acc[v]);
            }
        }
        for (; j < n; ++j) {
            const float a = __ldg(AT + (size_t)j * m + i);
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[v] = fmaf(a, x0[v * ld + j], acc[v]);
        }
        const float sc = scale ? __ldg(scale + i) : 1.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int vv = g * 8 + v;
            if (vv < nv) {
                const float r = sc * acc[v];
                ys[vv * ld + i] = accumulate ? ys[vv * ld + i] + r : r;
            }
        }
    }
}

// Node of vector v in a block whose vectors are (node g, rhs r), v = g*nr + r.
__device__ __forceinline__ int vec_node(const int *nodes, int first, int count, int v,
                                        int nr) {
    const int g = v / nr;
    return first + g < count ? nodes[first + g] : -1;
}

// Stores densities rho (smem) to the node arrays and projects them on Vk for
// the M2L: qhat = Vk^T rho.
__device__ void finish_upward(const DevOps &o, const DevWork &w, const int *nodes, int first,
                              int count, int r0, int nr, int nrr, int nv, int ld,
                              const float *rho, float *tmp) {
    const int ns = o.ns, kp = o.kpad;
    for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
        const int v = idx / ns, i = idx - v * ns;
        const int node = vec_node(nodes, first, count, v, nr);
        if (node >= 0 && v % nr < nrr)
            w.up[((size_t)node * w.nrhs + r0 + v % nr) * ns + i] = rho[v * ld + i];
    }
    block_mv(o.Vk, kp, ns, rho, nv, tmp, ld, nullptr, false);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nv * kp; idx += blockDim.x) {
        const int v = idx / kp, i = idx - v * kp;
        const int node = vec_node(nodes, first, count, v, nr);
        if (node >= 0 && v % nr < nrr)
            w.qhat[((size_t)node * w.nrhs + r0 + v % nr) * kp + i] = tmp[v * ld + i];
    }
}

// P2M for a chunk of leaves: check potential of the leaf's points on its
// upward check surface (radius ao, normalised), then y = Pu^T chk / Ps,
// rho = Pv y.
__global__ void __launch_bounds__(256) k_p2m(DevTree t, DevOps o, DevWork w,
                                             const int *nodes, int count, int G, int nr) {
    extern __shared__ __align__(16) float smem[];
    const int ns = o.ns, ld = smem_width(o);
    float *bufA = smem, *bufB = smem + kMaxVec * ld;
    const int first = blockIdx.x * G;
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const int nv = G * nr;
    for (int idx = threadIdx.x; idx < G * ns; idx += blockDim.x) {
        const int g = idx / ns, j = idx - g * ns;
        float acc[kMaxRhs];
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r) acc[r] = 0.f;
        if (first + g < count) {
            const int node = nodes[first + g];
            const float inv_h = 1.f / t.geom[node].w;
            const int2 rg = t.range[node];
            const float4 s = o.surf[j];
            const float cx = o.ao * s.x, cy = o.ao * s.y, cz = o.ao * s.z;
            for (int i = rg.x; i < rg.y; ++i) {
                const float4 p = t.pts[i];
                const float dx = cx - p.x * inv_h, dy = cy - p.y * inv_h, dz = cz - p.z * inv_h;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float inv = r2 > 0.f ? KIFMM_RSQRT(r2) : 0.f;
                const float *q = w.qs + (size_t)i * w.nrhs + r0;
#pragma unroll
                for (int r = 0; r < kMaxRhs; ++r)
                    if (r < nrr) acc[r] = fmaf(__ldg(q + r), inv, acc[r]);
            }
        }
        for (int r = 0; r < nr; ++r) bufA[(g * nr + r) * ld + j] = r < nrr ? acc[r] : 0.f;
    }
    __syncthreads();
    block_mv(o.Pu, o.rP, ns, bufA, nv, bufB, ld, o.Ps_inv, false);
    __syncthreads();
    block_mv(o.PvT, ns, o.rP, bufB, nv, bufA, ld, nullptr, false);
    __syncthreads();
    finish_upward(o, w, nodes, first, count, r0, nr, nrr, nv, ld, bufA, bufB);
}

// M2M for a chunk of internal nodes of one level: y = sum_sigma M2M_sigma
// rho_child(sigma), then rho = Pv (y / Ps).
__global__ void __launch_bounds__(256) k_m2m(DevTree t, DevOps o, DevWork w,
                                             const int *nodes, int count, int G, int nr) {
    extern __shared__ __align__(16) float smem[];
    const int ns = o.ns, ld = smem_width(o);
    float *bufA = smem, *bufB = smem + kMaxVec * ld, *bufC = bufB + kMaxVec * ld;
    const int first = blockIdx.x * G;
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const int nv = G * nr;
    for (int sg = 0; sg < 8; ++sg) {
        for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
            const int v = idx / ns, j = idx - v * ns;
            const int node = vec_node(nodes, first, count, v, nr);
            const int r = v % nr;
            float x = 0.f;
            if (node >= 0 && r < nrr) {
                const int ch = t.child[node * 8 + sg];
                if (ch >= 0) x = w.up[((size_t)ch * w.nrhs + r0 + r) * ns + j];
            }
            bufA[v * ld + j] = x;
        }
        __syncthreads();
        block_mv(o.M2M + (size_t)sg * ns * o.rP, o.rP, ns, bufA, nv, bufB, ld, nullptr, sg > 0);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nv * o.rP; idx += blockDim.x) {
        const int v = idx / o.rP, i = idx - v * o.rP;
        bufB[v * ld + i] *= o.Ps_inv[i];
    }
    __syncthreads();
    block_mv(o.PvT, ns, o.rP, bufB, nv, bufA, ld, nullptr, false);
    __syncthreads();
    finish_upward(o, w, nodes, first, count, r0, nr, nrr, nv, ld, bufA, bufC);
}

// P2L: downward check potential of box B (radius ai, normalised by h_B)
// from the points of every leaf in X(B).
__global__ void __launch_bounds__(128) k_p2l(DevTree t, DevOps o, DevWork w, const int *nodes,
                                             int nr) {
    __shared__ float4 spos[128];
    __shared__ float sq[kMaxRhs][128];
    const int b = nodes[blockIdx.x];
    const int r0 = blockIdx.y * nr;
    const int nrr = min(nr, w.nrhs - r0);
    const float4 gb = t.geom[b];
    const float inv_h = 1.f / gb.w;
    const int ns = o.ns;
    const int slot = t.x_slot[b];
    for (int j0 = 0; j0 < ns; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const float4 s = o.surf[min(j, ns - 1)];
        const float cx = o.ai * s.x, cy = o.ai * s.y, cz = o.ai * s.z;
        float acc[kMaxRhs];
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r) acc[r] = 0.f;
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
                    const float4 p = t.pts[i];
                    spos[threadIdx.x] = make_float4(p.x * inv_h + sx, p.y * inv_h + sy,
                                                    p.z * inv_h + sz, 0.f);
                    for (int r = 0; r < nrr; ++r)
                        sq[r][threadIdx.x] = w.qs[(size_t)i * w.nrhs + r0 + r];
                }
                __syncthreads();
                const int cnt = min((int)blockDim.x, rg.y - i0);
                for (int c = 0; c < cnt; ++c) {
                    const float dx = cx - spos[c].x, dy = cy - spos[c].y, dz = cz - spos[c].z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float inv = r2 > 0.f ? KIFMM_RSQRT(r2) : 0.f;
#pragma unroll
                    for (int r = 0; r < kMaxRhs; ++r)
                        if (r < nrr) acc[r] = fmaf(sq[r][c], inv, acc[r]);
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
    extern __shared__ __align__(16) float smem[];
    const int ns = o.ns, kp = o.kpad, rQ = o.rQ;
    const int ld = smem_width(o);
    float *bufA = smem, *bufB = smem + kMaxVec * ld;
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
            const int v = idx / kp, j = idx - v * kp;
            const int g = v / nr, r = v % nr;
            float x = 0.f;
            if (g < count && r < nrr) {
                const int b = my[g];
                if (t.v_ptr[b + 1] > t.v_ptr[b])
                    x = w.chat[((size_t)b * w.nrhs + r0 + r) * kp + j];
            }
            bufA[v * ld + j] = x;
        }
        __syncthreads();
        block_mv(o.QUkT, rQ, kp, bufA, nv, bufB, ld, nullptr, false);
        __syncthreads();
        // P2L check potentials: y += Qu^T xchk
        bool any_x = false;
        for (int g = 0; g < count; ++g) any_x |= t.x_slot[my[g]] >= 0;
        if (any_x) {
            for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
                const int v = idx / ns, j = idx - v * ns;
                const int g = v / nr, r = v % nr;
                float x = 0.f;
                if (g < count && r < nrr) {
                    const int slot = t.x_slot[my[g]];
                    if (slot >= 0) x = w.xchk[((size_t)slot * w.nrhs + r0 + r) * ns + j];
                }
                bufA[v * ld + j] = x;
            }
            __syncthreads();
            block_mv(o.Qu, rQ, ns, bufA, nv, bufB, ld, nullptr, true);
            __syncthreads();
        }
        // L2L from the parent (local expansions exist from level 2 on)
        if (level >= 3) {
            for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
                const int v = idx / ns, j = idx - v * ns;
                const int g = v / nr, r = v % nr;
                float x = 0.f;
                if (g < count && r < nrr) {
                    const int par = t.parent[my[g]];
                    x = w.down[((size_t)par * w.nrhs + r0 + r) * ns + j];
                }
                bufA[v * ld + j] = x;
            }
            __syncthreads();
            block_mv(o.L2L + (size_t)sg * ns * rQ, rQ, ns, bufA, nv, bufB, ld, nullptr, true);
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < nv * rQ; idx += blockDim.x) {
            const int v = idx / rQ, i = idx - v * rQ;
            bufB[v * ld + i] *= o.Qs_inv[i];
        }
        __syncthreads();
        block_mv(o.QvT, ns, rQ, bufB, nv, bufA, ld, nullptr, false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nv * ns; idx += blockDim.x) {
            const int v = idx / ns, j = idx - v * ns;
            const int g = v / nr, r = v % nr;
            if (g < count && r < nrr)
                w.down[((size_t)my[g] * w.nrhs + r0 + r) * ns + j] = bufA[v * ld + j];
        }
        __syncthreads();
    }
}

__global__ void k_gather_charges(DevTree t, DevWork w) {
    const int64_t total = t.n * (int64_t)w.nrhs;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / w.nrhs, r = idx - i * w.nrhs;
        w.qs[idx] = w.charges_user[t.perm[i] * w.nrhs + r];
    }
}

// Right-hand sides per block of the matrix-vector kernels.
inline int rhs_chunk(int nrhs) { return nrhs < kMaxRhs ? nrhs : kMaxRhs; }

size_t mv_smem(const DevOps &o, int bufs) {
    return (size_t)bufs * kMaxVec * smem_width(o) * sizeof(float);
}

template <class K> cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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

cudaError_t launch_p2m(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int nr = rhs_chunk(w.nrhs), G = kMaxVec / nr;
    const dim3 grid((count + G - 1) / G, (w.nrhs + nr - 1) / nr);
    const size_t sm = mv_smem(o, 2);
    cudaError_t e = allow_smem(k_p2m, sm);
    if (e != cudaSuccess) return e;
    k_p2m<<<grid, 256, sm, s>>>(t, o, w, nodes, count, G, nr);
    return cudaGetLastError();
}

cudaError_t launch_m2m(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int nr = rhs_chunk(w.nrhs), G = kMaxVec / nr;
    const dim3 grid((count + G - 1) / G, (w.nrhs + nr - 1) / nr);
    const size_t sm = mv_smem(o, 3);
    cudaError_t e = allow_smem(k_m2m, sm);
    if (e != cudaSuccess) return e;
    k_m2m<<<grid, 256, sm, s>>>(t, o, w, nodes, count, G, nr);
    return cudaGetLastError();
}

cudaError_t launch_p2l(const DevTree &t, const DevOps &o, const DevWork &w, const int *nodes,
                       int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int nr = rhs_chunk(w.nrhs);
    const dim3 grid(count, (w.nrhs + nr - 1) / nr);
    k_p2l<<<grid, 128, 0, s>>>(t, o, w, nodes, nr);
    return cudaGetLastError();
}

cudaError_t launch_down(const DevTree &t, const DevOps &o, const DevWork &w, const int *chunks,
                        const int *nodes, int nchunks, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    const int nr = rhs_chunk(w.nrhs);
    const dim3 grid(nchunks, (w.nrhs + nr - 1) / nr);
    const size_t sm = mv_smem(o, 2);
    cudaError_t e = allow_smem(k_down, sm);
    if (e != cudaSuccess) return e;
    k_down<<<grid, 256, sm, s>>>(t, o, w, chunks, nodes, nr);
    return cudaGetLastError();
}

} // namespace kifmm
