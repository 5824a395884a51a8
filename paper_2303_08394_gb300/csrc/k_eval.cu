// Leaf evaluation: near field over U ("P2P"), L2P from the leaf's own
// downward density, and M2P from the upward densities of its W list
// ("Computational structure of FMM operators": all three are evaluations of
// Eq. (1) between point sets).  One warp owns one target leaf and 32 of its
// targets at a time (one per lane); sources are staged 32 at a time in the
// warp's shared memory and read as broadcasts.
//
// Precision: FP32 rsqrt/FMA per pair; each 32-source batch is summed in
// plain FP32 and added into a per-target Kahan (sum, compensation) pair;
// the final potential is formed in FP64, scaled by 1/(4 pi hw) and written
// in the caller's point order.
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int kWarpsPerBlock = 8;

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// One batch of up to 32 staged sources against this lane's target.
template <int NR>
__device__ __forceinline__ void batch(const float4 *spos, const float (*sq)[32], int cnt,
                                      float tx, float ty, float tz, Kahan *acc) {
    float part[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) part[r] = 0.f;
    for (int j = 0; j < cnt; ++j) {
        const float4 p = spos[j];
        const float dx = p.x - tx, dy = p.y - ty, dz = p.z - tz;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float inv = r2 > 0.f ? KIFMM_RSQRT(r2) : 0.f;
        if (NR == 1) {
            part[0] = fmaf(p.w, inv, part[0]);
        } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) part[r] = fmaf(sq[r][j], inv, part[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r].add(part[r]);
}

template <int NR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_eval(DevTree t, DevOps o, DevWork w, int r0) {
    __shared__ float4 s_pos[kWarpsPerBlock][32];
    __shared__ float s_q[kWarpsPerBlock][NR][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *spos = s_pos[wid];
    float(*sq)[32] = s_q[wid];
    const int gwarp = blockIdx.x * kWarpsPerBlock + wid;
    const int nwarps = gridDim.x * kWarpsPerBlock;
    const int ns = o.ns, nsp = (o.ns + 3) & ~3;  // surface rows are padded to nsp
    for (int li = gwarp; li < t.nleaves; li += nwarps) {
        const int b = t.leaves[li];
        const float4 gb = t.geom[b];
        const int2 rb = t.range[b];
        const int lvl = t.level[b];
        for (int t0 = rb.x; t0 < rb.y; t0 += 32) {
            const int ti = t0 + lane;
            const bool valid = ti < rb.y;
            float4 xt = valid ? t.pts[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
            Kahan acc[NR];
            // near field: U list (the leaf itself included)
            for (int e = t.u_ptr[b]; e < t.u_ptr[b + 1]; ++e) {
                const int a = t.u_idx[e];
                const float4 ga = t.geom[a];
                const float sx = ga.x - gb.x, sy = ga.y - gb.y, sz = ga.z - gb.z;
                const int2 ra = t.range[a];
                for (int s0 = ra.x; s0 < ra.y; s0 += 32) {
                    const int si = s0 + lane;
                    __syncwarp();
                    if (si < ra.y) {
                        float4 p = t.pts[si];
                        const float *q = w.qs + (size_t)si * w.nrhs + r0;
                        spos[lane] = make_float4(p.x + sx, p.y + sy, p.z + sz,
                                                 NR == 1 ? __ldg(q) : 0.f);
                        if (NR > 1) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) sq[r][lane] = __ldg(q + r);
                        }
                    }
                    __syncwarp();
                    batch<NR>(spos, sq, min(32, ra.y - s0), xt.x, xt.y, xt.z, acc);
                }
            }
            // L2P: the leaf's downward density on its downward equivalent surface
            if (lvl >= 2) {
                const float rad = o.ao * gb.w;
                for (int s0 = 0; s0 < ns; s0 += 32) {
                    const int j = s0 + lane;
                    __syncwarp();
                    if (j < ns) {
                        float4 s = o.surf[j];
                        const float *d = w.down + ((size_t)b * w.nrhs + r0) * nsp + j;
                        spos[lane] = make_float4(rad * s.x, rad * s.y, rad * s.z,
                                                 NR == 1 ? d[0] : 0.f);
                        if (NR > 1) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) sq[r][lane] = d[(size_t)r * nsp];
                        }
                    }
                    __syncwarp();
                    batch<NR>(spos, sq, min(32, ns - s0), xt.x, xt.y, xt.z, acc);
                }
            }
            // M2P: upward densities of the W list on their upward equivalent surfaces
            for (int e = t.w_ptr[b]; e < t.w_ptr[b + 1]; ++e) {
                const int a = t.w_idx[e];
                const float4 ga = t.geom[a];
                const float sx = ga.x - gb.x, sy = ga.y - gb.y, sz = ga.z - gb.z;
                const float rad = o.ai * ga.w;
                for (int s0 = 0; s0 < ns; s0 += 32) {
                    const int j = s0 + lane;
                    __syncwarp();
                    if (j < ns) {
                        float4 s = o.surf[j];
                        const float *d = w.up + ((size_t)a * w.nrhs + r0) * nsp + j;
                        spos[lane] = make_float4(sx + rad * s.x, sy + rad * s.y,
                                                 sz + rad * s.z, NR == 1 ? d[0] : 0.f);
                        if (NR > 1) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) sq[r][lane] = d[(size_t)r * nsp];
                        }
                    }
                    __syncwarp();
                    batch<NR>(spos, sq, min(32, ns - s0), xt.x, xt.y, xt.z, acc);
                }
            }
            if (valid) {
                double *out = w.pot_user + (size_t)t.perm[ti] * w.nrhs + r0;
#pragma unroll
                for (int r = 0; r < NR; ++r) out[r] = acc[r].value() * w.scale;
            }
        }
    }
}

template <int NR>
cudaError_t launch_eval_nr(const DevTree &t, const DevOps &o, const DevWork &w, int r0,
                           cudaStream_t s) {
    int blocks = (t.nleaves + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks < 1) blocks = 1;
    k_eval<NR><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(t, o, w, r0);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_eval(const DevTree &t, const DevOps &o, const DevWork &w, cudaStream_t s) {
    int r0 = 0;
    cudaError_t e = cudaSuccess;
    while (r0 < w.nrhs && e == cudaSuccess) {
        int left = w.nrhs - r0;
        if (left >= 8) { e = launch_eval_nr<8>(t, o, w, r0, s); r0 += 8; }
        else if (left >= 4) { e = launch_eval_nr<4>(t, o, w, r0, s); r0 += 4; }
        else if (left >= 2) { e = launch_eval_nr<2>(t, o, w, r0, s); r0 += 2; }
        else { e = launch_eval_nr<1>(t, o, w, r0, s); r0 += 1; }
    }
    return e;
}

} // namespace kifmm
