// V-list M2L in FP32 on the CUDA cores ("Computational structure of FMM
// operators": M2L over V is a matrix-vector product per (target, source)
// pair; here the products of one tile of 128 targets and one offset t are
// batched into a 128 x k by k x k product).
//
// chat[target] = sum_{A in V(target)} S_t(A,target) qhat[A]
//
// A block owns 128 rows (target, rhs) of one tile.  For every offset the
// tile uses it gathers the 128 source vectors (zero where a target has no
// source at that offset) and multiplies them by S_t, accumulating in
// registers: thread (tr, tc) holds rows 8 tr .. 8 tr + 7 and columns
// tc + 16 c.
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int kKc = 16;  // K chunk

template <int CPT>
__global__ void __launch_bounds__(256) k_m2l_simt(DevM2L m, DevOps o, DevWork w) {
    __shared__ float xs[kKc][128 + 4];
    __shared__ __align__(16) float ss[kKc][16 * CPT];
    __shared__ int rowsrc[128];
    const int tile = blockIdx.x;
    const int chunk = blockIdx.y;
    const int kp = o.kpad;  // == 16 * CPT
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int nrhs = w.nrhs;
    float acc[8][CPT];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[i][c] = 0.f;

    const int e0 = m.tile_entry_ptr[tile], e1 = m.tile_entry_ptr[tile + 1];
    for (int e = e0; e < e1; ++e) {
        const int off = m.entry_offset[e];
        __syncthreads();
        if (tid < 128) {
            const int g = chunk * 128 + tid;
            const int slot = g / nrhs, r = g - slot * nrhs;
            const int src = m.entry_src[(size_t)e * 128 + slot];
            rowsrc[tid] = src >= 0 ? src * nrhs + r : -1;
        }
        const float *St = o.St + (size_t)off * kp * kp;
        for (int kc = 0; kc < kp; kc += kKc) {
            __syncthreads();
            {   // gather 128 rows x 16 columns of qhat, stored transposed
                const int row = tid >> 1, half = tid & 1;
                const int rs = rowsrc[row];
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                if (rs >= 0) {
                    const float4 *src = reinterpret_cast<const float4 *>(
                        w.qhat + (size_t)rs * kp + kc + half * 8);
                    a = __ldg(src);
                    b = __ldg(src + 1);
                }
                const int c0 = half * 8;
                xs[c0 + 0][row] = a.x; xs[c0 + 1][row] = a.y;
                xs[c0 + 2][row] = a.z; xs[c0 + 3][row] = a.w;
                xs[c0 + 4][row] = b.x; xs[c0 + 5][row] = b.y;
                xs[c0 + 6][row] = b.z; xs[c0 + 7][row] = b.w;
            }
            // 16 rows of St (j = kc..kc+15), all kp columns
            for (int idx = tid; idx < kKc * kp / 4; idx += 256) {
                const int j = idx / (kp / 4), q = idx - j * (kp / 4);
                reinterpret_cast<float4 *>(&ss[j][0])[q] =
                    __ldg(reinterpret_cast<const float4 *>(St + (size_t)(kc + j) * kp) + q);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kKc; ++kk) {
                float a[8], bcol[CPT];
                const float4 a0 = *reinterpret_cast<const float4 *>(&xs[kk][tr * 8]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&xs[kk][tr * 8 + 4]);
                a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
                a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
                for (int c = 0; c < CPT; ++c) bcol[c] = ss[kk][tc + 16 * c];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) acc[i][c] = fmaf(a[i], bcol[c], acc[i][c]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int g = chunk * 128 + tr * 8 + i;
        const int slot = g / nrhs, r = g - slot * nrhs;
        const int tgt = m.tile_target[(size_t)tile * 128 + slot];
        if (tgt < 0) continue;
        float *out = w.chat + ((size_t)tgt * nrhs + r) * kp;
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[tc + 16 * c] = acc[i][c];
    }
}

template <int CPT>
cudaError_t launch_cpt(const DevM2L &m, const DevOps &o, const DevWork &w, cudaStream_t s) {
    dim3 grid(m.ntiles, w.nrhs);
    k_m2l_simt<CPT><<<grid, 256, 0, s>>>(m, o, w);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_m2l_simt(const DevM2L &m, const DevOps &o, const DevWork &w, cudaStream_t s) {
    if (m.ntiles == 0) return cudaSuccess;
    switch (o.kpad / 16) {
    case 1: return launch_cpt<1>(m, o, w, s);
    case 2: return launch_cpt<2>(m, o, w, s);
    case 3: return launch_cpt<3>(m, o, w, s);
    case 4: return launch_cpt<4>(m, o, w, s);
    case 5: return launch_cpt<5>(m, o, w, s);
    case 6: return launch_cpt<6>(m, o, w, s);
    case 7: return launch_cpt<7>(m, o, w, s);
    case 8: return launch_cpt<8>(m, o, w, s);
    case 9: return launch_cpt<9>(m, o, w, s);
    case 10: return launch_cpt<10>(m, o, w, s);
    case 11: return launch_cpt<11>(m, o, w, s);
    case 12: return launch_cpt<12>(m, o, w, s);
    case 13: return launch_cpt<13>(m, o, w, s);
    case 14: return launch_cpt<14>(m, o, w, s);
    case 15: return launch_cpt<15>(m, o, w, s);
    case 16: return launch_cpt<16>(m, o, w, s);
    case 17: return launch_cpt<17>(m, o, w, s);
    case 18: return launch_cpt<18>(m, o, w, s);
    case 19: return launch_cpt<19>(m, o, w, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace kifmm
