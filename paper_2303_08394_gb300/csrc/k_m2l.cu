// V-list M2L in FP32 on the CUDA cores ("Computational structure of FMM
// operators": M2L over V is a matrix-vector product per (target, source)
// pair; here the products of one tile of targets and one offset t are
// batched into a rows x k by k x k product).
//
// chat[target] = sum_{A in V(target)} S_t(A,target) qhat[A]
//
// A block owns 16*RPT rows (target, rhs) of one tile.  For every offset the
// tile uses it gathers the source vectors (zero where a target has no source
// at that offset) and multiplies them by S_t.  Thread (tr, tc) holds rows
// RPT*tr .. RPT*tr + RPT - 1 and columns tc + 16 c.
//
// Summation order: each offset's product is summed in a fresh partial and
// then added to the running total.  One accumulator over all ~189 k terms
// of a target loses about 5x more accuracy in FP32 (the far field then
// misses the 1e-6 bar against the FP64 oracle).
#include "device.cuh"

namespace kifmm {

namespace {

constexpr int kKc = 16;  // K chunk

template <int CPT, int RPT>
__global__ void __launch_bounds__(256) k_m2l_simt(DevM2L m, DevOps o, DevWork w) {
    constexpr int RB = 16 * RPT;  // rows per block
    __shared__ __align__(16) float xs[kKc][RB + 4];
    __shared__ __align__(16) float ss[kKc][16 * CPT];
    __shared__ int rowsrc[RB];
    const int tile = blockIdx.x;
    const int chunk = blockIdx.y;
    const int kp = o.kpad;  // == 16 * CPT
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int nrhs = w.nrhs;
    float acc[RPT][CPT], part[RPT][CPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[i][c] = 0.f;

    const int e0 = m.tile_entry_ptr[tile], e1 = m.tile_entry_ptr[tile + 1];
    for (int e = e0; e < e1; ++e) {
        const int off = m.entry_offset[e];
        __syncthreads();
        if (tid < RB) {
            const int g = chunk * RB + tid;
            const int slot = g / nrhs, r = g - slot * nrhs;
            int src = -1;
            if (slot < kTileRows) src = m.entry_src[(size_t)e * kTileRows + slot];
            rowsrc[tid] = src >= 0 ? src * nrhs + r : -1;
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int c = 0; c < CPT; ++c) part[i][c] = 0.f;
        const float *St = o.St + (size_t)off * kp * kp;
        for (int kc = 0; kc < kp; kc += kKc) {
            __syncthreads();
            {   // gather RB rows x 16 columns of qhat, stored transposed
                constexpr int PER = kKc * RB / 256;  // floats per thread: 8 or 4
                const int row = tid / (kKc / PER), part_c = (tid % (kKc / PER)) * PER;
                const int rs = rowsrc[row];
                float v[PER];
#pragma unroll
                for (int q = 0; q < PER; ++q) v[q] = 0.f;
                if (rs >= 0) {
                    const float4 *src = reinterpret_cast<const float4 *>(
                        w.qhat + (size_t)rs * kp + kc + part_c);
#pragma unroll
                    for (int q = 0; q < PER / 4; ++q) {
                        const float4 a = __ldg(src + q);
                        v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
                    }
                }
#pragma unroll
                for (int q = 0; q < PER; ++q) xs[part_c + q][row] = v[q];
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
                float a[RPT], bcol[CPT];
#pragma unroll
                for (int q = 0; q < RPT / 4; ++q) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(&xs[kk][tr * RPT + 4 * q]);
                    a[4 * q] = a4.x; a[4 * q + 1] = a4.y; a[4 * q + 2] = a4.z; a[4 * q + 3] = a4.w;
                }
#pragma unroll
                for (int c = 0; c < CPT; ++c) bcol[c] = ss[kk][tc + 16 * c];
#pragma unroll
                for (int i = 0; i < RPT; ++i)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) part[i][c] = fmaf(a[i], bcol[c], part[i][c]);
            }
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[i][c] += part[i][c];
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int g = chunk * RB + tr * RPT + i;
        const int slot = g / nrhs, r = g - slot * nrhs;
        if (slot >= kTileRows) continue;
        const int tgt = m.tile_target[(size_t)tile * kTileRows + slot];
        if (tgt < 0) continue;
        float *out = w.chat + ((size_t)tgt * nrhs + r) * kp;
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[tc + 16 * c] = acc[i][c];
    }
}

template <int CPT>
cudaError_t launch_cpt(const DevM2L &m, const DevOps &o, const DevWork &w, cudaStream_t s) {
    constexpr int RPT = CPT <= 12 ? 8 : 4;
    constexpr int RB = 16 * RPT;
    const int rows = kTileRows * w.nrhs;
    dim3 grid(m.ntiles, (rows + RB - 1) / RB);
    k_m2l_simt<CPT, RPT><<<grid, 256, 0, s>>>(m, o, w);
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
