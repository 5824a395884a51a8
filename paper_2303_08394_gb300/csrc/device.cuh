// Device-side views of a plan and the kernel launchers.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "constants.h"

// Reciprocal square root used by every kernel evaluation 1/r: the PTX
// rsqrt.approx.ftz.f32 instruction (relative error about 2^-23; squared
// distances below the smallest normal float are flushed to zero, which only
// the self pairs reach).  A build may define KIFMM_RSQRT to trade speed for
// rounding.
#ifndef KIFMM_RSQRT
#define KIFMM_RSQRT(x) ::kifmm::rsqrt_approx(x)
#endif

namespace kifmm {

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tree and lists on the device (all indices are node ids in plan order).
struct DevTree {
    int64_t n;
    int nnodes, depth;
    const float4 *pts;      // n: position relative to the leaf centre (root units)
    const float4 *pts_lo;   // n: rounding residual of pts (pts + pts_lo ~ FP64)
    const int64_t *qidx;    // n: charge row of each sorted point (-1 none)
    const int64_t *oidx;    // n: potential row of each sorted point (-1 none)
    const double *node_scale;  // nodes: 1 / (4 pi root half-width) of the
                               // box's problem (positions are in root units)
    const float4 *geom;     // nodes: centre x, y, z (root units), half-width
    const int2 *range;      // nodes: sorted point range [x, y)
    const int *level;       // nodes
    const int *parent;      // nodes
    const int *child;       // nodes x 8
    const int *leaves;      // nleaves, grouped by the leaf pass's width
                            // T = min(kLeafWidths, ceil(points / 16)): the
                            // widest group first (plan order within each)
    int nleaves;
    int t_first[kLeafWidths + 1];  // leaves[t_first[T] .. t_first[T - 1]) have
                                   // width T (t_first[kLeafWidths] = 0,
                                   // t_first[0] = nleaves)
    const int *u_ptr, *u_idx, *w_ptr, *w_idx, *x_ptr, *x_idx, *v_ptr;
    const int *x_slot;      // nodes: row block in the P2L buffer or -1; a
                            // leaf with an X list and no slot takes the X
                            // leaves' points in the leaf pass
    const int *w_direct;    // nodes: 1 if the box, as a W-list entry, acts
                            // on the leaf through its points instead of its
                            // upward equivalent surface
};

// FP32 operators.  Every matrix is stored as the transpose AT (n x m) of
// the m x n operator A it applies, rows padded to round4(m) floats so each
// row is 16-byte aligned; consecutive threads own consecutive output rows i
// and read AT[j*round4(m) + i].
struct DevOps {
    int ns, rP, rQ, k, kpad;
    float ai, ao;
    const float4 *surf;     // ns unit surface points
    const float *Pu;        // AT of Pu^T:  ns x rP
    const float *Ps_inv;    // rP
    const float *PvT;       // AT of Pv:    rP x ns
    const float *M2M;       // 8 x AT of M2M_sigma: ns x rP each
    const float *Vk;        // AT of Vk^T:  ns x kpad (zero padded)
    const float *QUkT;      // AT of Qu^T Uk: kpad x rQ (zero padded)
    const float *Qu;        // AT of Qu^T:  ns x rQ
    const float *L2L;       // AT of [L2L_0; ..; L2L_7] / Qs: ns x 8 rQ
    const float *Qs_inv;    // rQ
    const float *QvT;       // AT of Qv:    rQ x ns
    const float *St;        // 316 x kpad x kpad: St[t][j][i] = S_t[i][j]
};

// M2L tiles (see plan.h).
struct DevM2L {
    int ntiles;
    const int *tile_target;     // ntiles x 128
    const int *tile_entry_ptr;  // ntiles + 1
    const int *entry_offset;    // entries
    const int *entry_src;       // entries x 128
    int ncta;                   // blocks of the schedule (0: none, round robin)
    const int *cta_ptr;         // ncta + 1
    const int *cta_tiles;       // ntiles: the tiles of each block
};

// Pair-column M2L tables (plan.h, M2LWindows).
struct DevM2LPc {
    int ncta;
    const int *cta_ptr, *cta_win;
    const int *win_target_ptr, *win_targets, *win_item_ptr;
    const int *item_offset, *item_pair_ptr;
    const int *pair_src, *pair_slot;
};

// Buffers of one evaluation.  Densities: [node][rhs][round4(ns)];
// compressed M2L vectors: [node][rhs][kpad]; P2L check potentials:
// [x slot][rhs][round4(ns)].
struct DevWork {
    int nrhs;
    const float *charges_user;  // rows x nrhs, caller order
    float *qs;                  // n x nrhs, sorted order
    float *up, *down;           // nodes x nrhs x ns
    float *qhat, *chat;         // nodes x nrhs x kpad
    float *xchk;                // x nodes x nrhs x ns
    double *pot_user;           // rows x nrhs, caller order (may be null when
                                // grad_user is set)
    double *grad_user;          // rows x nrhs x 3, caller order: gradient of the
                                // potential at each target (null: potentials only)
};

// Batched operator x gathered-vector products (k_vgemm.cu):
//   Y[dst(v)][i] = scale[i] * sum_s sum_j A_s[i][j] X_s[src_s(v)][j] + add(v)[i]
// for v = pos * nrhs + r, pos < count, i < m.  A_s is stored as its transpose
// AT (n x round4(m)).  Source row of segment s for v: (src_idx[pos] or
// src_base + pos) * nrhs + r in rows of src_ld floats (index < 0 reads
// zeros).  Destination row: (dst_idx[pos] or dst_base + pos) * nrhs + r.
// Optional add row: (add_idx[pos]) * nrhs + r in rows of add_ld floats,
// offset by add_off[pos] floats.
constexpr int kMaxSeg = 8;
struct VSeg {
    const float *AT;
    int n;
    const float *src;
    int src_ld;
    const int *src_idx;
    int src_base;
};
struct VGemm {
    int m, count, nrhs, nseg;
    VSeg seg[kMaxSeg];
    // Segments (bit s) whose index list names a row for few vectors: a
    // block skips such a segment when none of its vectors has a row (the
    // sums are unchanged: the skipped terms are exact zeros).
    uint32_t sparse;
    const float *scale;
    float *dst;
    int dst_ld;
    const int *dst_idx;
    int dst_base;
    const float *add;
    int add_ld;
    const int *add_idx;
    const int *add_off;
    // Optional split-K scratch of nseg x count*nrhs x round4(m) floats: a
    // product of several segments that would run on few blocks (one block's
    // K loop then walks every segment in turn) is computed one segment per
    // block instead, and the partial products are summed in segment order.
    float *part;
};
// A product with a split-K scratch splits its segments when it has fewer
// than this many blocks for one right-hand side.
constexpr int kSplitBlocks = 4 * 152;
size_t vgemm_split_floats(int m, int count, int nrhs, int nseg);  // 0: no split
// Tile shapes of the level products (rows x vectors per block): 0 = 64 x 32,
// 1 = 32 x 64, 2 = 128 x 16 (4 x 4 per thread), 3 = 64 x 64, 4 = 128 x 32
// (8 x 4 per thread).  Bit-identical results; speed differs by shape.
constexpr int kGemmShapes = 5;
cudaError_t launch_vgemm(const VGemm &g, cudaStream_t s, int shape = 0);

// Upward check potentials of leaves (k_updown.cu): chk[pos*nrhs + r][j] for
// pos < count, rows of `ld` floats.
cudaError_t launch_p2m_check(const DevTree &t, const DevOps &o, const DevWork &w,
                             const int *nodes, int count, float *chk, int ld, cudaStream_t s);

cudaError_t launch_gather_charges(const DevTree &t, const DevWork &w, cudaStream_t s);
cudaError_t launch_p2l(const DevTree &t, const DevOps &o, const DevWork &w,
                       const int *nodes, int count, cudaStream_t s);
cudaError_t launch_m2l_simt(const DevM2L &m, const DevOps &o, const DevWork &w,
                            cudaStream_t s);
// Leaf pass (k_eval.cu): near field, L2P and M2P into the caller's rows;
// *launches receives the kernels it enqueued.  narrow_first: launch the
// width groups narrowest first instead of widest first (same results).
cudaError_t launch_eval(const DevTree &t, const DevOps &o, const DevWork &w,
                        cudaStream_t s, int *launches, bool narrow_first = false);

// Tensor-core M2L (k_m2l_tc.cu).  qh_hi/qh_lo hold (nnodes*nrhs + 1) rows of
// kpad operand elements (BF16, or TF32 in 32-bit words), the last row zero;
// s_hi/s_lo map the split S_t arrays [316*kpad rows][kpad] with 128-byte
// swizzled boxes of 128 bytes x kpad rows.  *err is set nonzero if a bounded
// wait expired.
size_t m2l_tc_smem(int kpad, int *stages);
// Opt the kernel into its dynamic shared memory (once per process and
// format, before the first launch; not stream-ordered, so outside captures).
cudaError_t configure_m2l_tc(int kpad, bool tf32);
cudaError_t launch_m2l_tc(const DevM2L &m, const DevOps &o, const DevWork &w, int nnodes,
                          bool tf32, const CUtensorMap &s_hi, const CUtensorMap &s_lo,
                          void *qh_hi, void *qh_lo, int *err, bool test_stall, int num_sms,
                          cudaStream_t st);

// Split qhat (nrows rows of kpad FP32) into hi/lo operand rows (BF16, or
// TF32 in 32-bit words), plus one zero row after the last.
cudaError_t launch_split_qhat(const float *qhat, int64_t nrows, int kp, bool tf32, void *hi,
                              void *lo, cudaStream_t st);
// Pair-column tensor-core M2L (k_m2l_pc.cu): the same operands as
// launch_m2l_tc (it splits qhat itself), work from the window tables; kpad
// at most 128.  ncta persistent blocks.
cudaError_t launch_m2l_pc(const DevM2LPc &m, const DevOps &o, const DevWork &w, int nnodes,
                          bool tf32, const CUtensorMap &s_hi, const CUtensorMap &s_lo,
                          void *qh_hi, void *qh_lo, int *err, bool test_stall, cudaStream_t st);
cudaError_t configure_m2l_pc(bool tf32);

// Nodes per down-pass chunk (chunks never mix child positions).
constexpr int kDownChunk = 32;

} // namespace kifmm
