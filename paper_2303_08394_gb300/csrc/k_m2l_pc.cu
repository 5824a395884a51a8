// V-list M2L on the 5th-generation tensor cores, one column per V pair.
//
// The compressed M2L ("Computational structure of FMM operators": M2L over
// V, compressed by a two-sided SVD) is c_B += S_t q_A over every pair
// (B, A) of the V lists, t the offset of A from B.  Here the products are
// grouped by offset: within a window of up to 256 target boxes, the pairs of
// offset t form an item, and the item is one tensor-core product
//     D[kpad x N] = S_t[kpad x kpad] * [q_A1 q_A2 ... q_AN],
// M = 128 rows (the output coefficients, S_t zero padded), N = the item's
// pairs rounded up to 16, K = kpad.  An adaptive tree uses few pairs per
// offset and target tile, so putting the pairs in N (steps of 16) instead of
// M (128 target rows) keeps the products filled.  Operands are split
// x = x_hi + x_lo in BF16 (kind::f16) or TF32 (kind::tf32) and every K step
// issues S_hi q_hi + S_hi q_lo + S_lo q_hi with FP32 accumulation in TMEM.
//
// The epilogue adds column j of D (the product for pair j, a fresh partial
// of one offset) into the running total of its target, which lives in TMEM
// column `slot` of the window (lanes = coefficients): totals are summed in
// offset order, so results do not depend on timing.  At the end of a window
// the totals are written to chat.  TMEM: 256 total columns, then two
// 128-column product buffers (the epilogue drains one while the MMAs fill
// the other).
//
// Warp roles (448 threads), as in the target-tile kernel:
//   0-3, 10-13  gather the item's source rows q_A (one 128-byte K chunk of
//        every column per stage) into the 128-byte swizzled K-major layout;
//        the two sets take chunks in turn;
//   4-7  epilogue (TMEM lane quarter = warp - 4);
//   8    TMA loads of the S_t chunks (hi and lo) into the A tiles;
//   9    allocates TMEM, issues the MMAs (one thread), frees TMEM.
// Every wait is bounded; on expiry the block records its role in *err
// (bits as in the target-tile kernel: 0 gatherers, 1 epilogue, 2 TMA, 3 and
// 4 MMA thread, 5 the test hook), drains what it issued and frees TMEM.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>

#include "constants.h"
#include "device.cuh"
#include "tc_ptx.cuh"

namespace kifmm {

namespace {

constexpr int kSets = 2;
constexpr int kThreads = 32 * (10 + 4 * (kSets - 1));
constexpr int kStages = 3;
constexpr uint32_t kTotCols = 256;      // window totals (kWinTargets)
constexpr uint32_t kAccCol = 256;       // first product buffer
constexpr uint32_t kAccCols = 128;      // per product buffer (kItemCols)
constexpr uint64_t kWaitLimit = 2000000000ull;      // 2 s per wait
constexpr uint64_t kTestStallLimit = 100000000ull;  // 0.1 s (test hook)
static_assert(kTotCols >= 256 && kAccCols >= 128, "TMEM columns must hold a window and an item");

struct PcArgs {
    DevM2LPc m;
    int nrhs, kpad, nch;
    const uint4 *qh_hi, *qh_lo;   // rows of kpad elements (16-byte pieces)
    float *chat;
    int *err;
    int test_stall;
};

template <bool kTF32> struct Fmt {
    static constexpr int esize = kTF32 ? 4 : 2;
    static constexpr int kc = 128 / esize;        // elements per 128-byte K chunk
    static constexpr int kstep = kTF32 ? 8 : 16;  // K per MMA instruction (32 bytes)
    static constexpr uint32_t ab = kTF32 ? 2u : 1u;
};

constexpr uint32_t kTile = 128 * 128;             // one split of a 128-row chunk tile
constexpr uint32_t kStageBytes = 4 * kTile;       // A hi, A lo, B hi, B lo

template <bool kTF32>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_pc(const __grid_constant__ CUtensorMap s_hi, const __grid_constant__ CUtensorMap s_lo,
             PcArgs a) {
    using F = Fmt<kTF32>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int kp = a.kpad, S = kStages;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)S * kStageBytes);
    uint64_t *full = bars, *empty = bars + S;
    uint64_t *acc_full = bars + 2 * S, *acc_empty = acc_full + 2, *done = acc_full + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *never = abort_flag + 1;  // stays 0: drains ignore the abort flag

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 128 + 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 128);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        *never = 0;
        tc::fence_mbar_init();
    }
    auto a_tile = [&](int s, int split) { return smem + (size_t)s * kStageBytes + split * kTile; };
    auto b_tile = [&](int s, int split) {
        return smem + (size_t)s * kStageBytes + 2 * kTile + split * kTile;
    };
    // rows kpad..127 of the S_t tiles stay zero (the TMA box has kpad rows)
    if (kp < 128) {
        for (int s = 0; s < S; ++s)
            for (int split = 0; split < 2; ++split) {
                uint4 *z = reinterpret_cast<uint4 *>(a_tile(s, split) + (size_t)kp * 128);
                for (int i = tid; i < (128 - kp) * 8; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
            }
        tc::fence_proxy_async_smem();
    }
    if (warp == 9) tc::tmem_alloc(tmem_slot, 512);
    if (warp == 8 && lane == 0) {
        tc::prefetch_tmap(&s_hi);
        tc::prefetch_tmap(&s_lo);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int w0 = a.m.cta_ptr[blockIdx.x], w1 = a.m.cta_ptr[blockIdx.x + 1];
    auto fail = [&](int role) {
        *abort_flag = 1;
        atomicOr(a.err, 1 << role);
    };

    if (warp < 4 || warp >= 10) {
        // ------------------------------------------------ pair-column gatherers
        // Eight lanes share a column (one 16-byte piece each), so one
        // warp-wide load reads four whole 128-byte row chunks; a thread
        // covers the columns (4 wi + i) * 4 + sub, i < 8, of its warp wi.
        const int set = warp < 4 ? 0 : 1 + (warp - 10) / 4;
        const int wi = warp < 4 ? warp : (warp - 10) % 4;
        const int piece = lane & 7, sub = lane >> 3;
        const int row16 = kp * F::esize / 16;
        uint32_t j = 0;
        bool ok = true;
        for (int u = w0; u < w1 && ok; ++u)
            for (int r = 0; r < a.nrhs && ok; ++r) {
                const int win = a.m.cta_win[u];
                const int i0 = a.m.win_item_ptr[win], i1 = a.m.win_item_ptr[win + 1];
                // the source rows of an item's columns are loaded one item
                // ahead (and its pair range two ahead), so those loads
                // overlap the previous item's copies
                int src[8], srcn[8];
                int p0n = 0, nn = 0;  // next item's pairs
                auto load_src = [&](int p0x, int nx, int (&sx)[8]) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int col = (wi * 8 + i) * 4 + sub;
                        sx[i] = col < nx ? a.m.pair_src[p0x + col] : -1;
                    }
                };
                if (i0 < i1) {
                    const int p0 = a.m.item_pair_ptr[i0], n = a.m.item_pair_ptr[i0 + 1] - p0;
                    load_src(p0, n, src);
                    if (i0 + 1 < i1) {
                        p0n = a.m.item_pair_ptr[i0 + 1];
                        nn = a.m.item_pair_ptr[i0 + 2] - p0n;
                    }
                }
                for (int it = i0; it < i1 && ok; ++it) {
                    if (it + 1 < i1) load_src(p0n, nn, srcn);
                    int p0nn = 0, nnn = 0;
                    if (it + 2 < i1) {
                        p0nn = a.m.item_pair_ptr[it + 2];
                        nnn = a.m.item_pair_ptr[it + 3] - p0nn;
                    }
                    uint32_t qoff[8];   // < 2^32: checked by the launcher
                    bool have[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        have[i] = src[i] >= 0;
                        qoff[i] = ((uint32_t)(have[i] ? src[i] : 0) * (uint32_t)a.nrhs + (uint32_t)r) *
                                      (uint32_t)row16 +
                                  (uint32_t)piece;
                    }
                    for (int c = 0; c < a.nch && ok; ++c, ++j) {
                        if ((int)(j % kSets) != set) continue;
                        const int s = j % S;
                        const int valid = min(F::kc, kp - c * F::kc);
                        const bool mine = piece * 16 < valid * F::esize;
                        uint4 vh[8], vl[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (mine && have[i]) {
                                vh[i] = __ldg(a.qh_hi + qoff[i] + c * 8);
                                vl[i] = __ldg(a.qh_lo + qoff[i] + c * 8);
                            }
                        ok = tc::mbar_wait(&empty[s], ((j / S) & 1) ^ 1, abort_flag, kWaitLimit);
                        if (!ok) {
                            if (!*abort_flag) fail(0);
                            break;
                        }
                        unsigned char *th = b_tile(s, 0), *tl = b_tile(s, 1);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (mine && have[i]) {
                                const int col = (wi * 8 + i) * 4 + sub;
                                const uint32_t off = (col >> 3) * 1024 + (col & 7) * 128 +
                                                     ((piece ^ (col & 7)) << 4);
                                *reinterpret_cast<uint4 *>(th + off) = vh[i];
                                *reinterpret_cast<uint4 *>(tl + off) = vl[i];
                            }
                        tc::fence_proxy_async_smem();
                        tc::mbar_arrive(&full[s]);
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) src[i] = srcn[i];
                    p0n = p0nn;
                    nn = nnn;
                }
            }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ epilogue
        const int q = warp - 4;               // TMEM lane quarter
        const int row = q * 32 + lane;        // output coefficient of this thread
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t gi = 0;
        bool ok = true;
        for (int u = w0; u < w1 && ok; ++u)
            for (int r = 0; r < a.nrhs && ok; ++r) {
                const int win = a.m.cta_win[u];
                const int t0 = a.m.win_target_ptr[win], nt = a.m.win_target_ptr[win + 1] - t0;
                const int i0 = a.m.win_item_ptr[win], i1 = a.m.win_item_ptr[win + 1];
                // totals start at zero
                {
                    float z[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) z[i] = 0.f;
                    for (int c0 = 0; c0 < nt; c0 += 16) tc::tmem_st16(lane_addr + c0, z);
                    tc::tmem_wait_st();
                }
                // the slots of an item's columns, lane l holding columns
                // l + 32 k: loaded one item ahead, so the loads overlap the
                // previous item's products
                int p0 = 0, n = 0, sl[4] = {0, 0, 0, 0};
                auto load_item = [&](int it, int &p0x, int &nx, int (&slx)[4]) {
                    p0x = a.m.item_pair_ptr[it];
                    nx = a.m.item_pair_ptr[it + 1] - p0x;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int c = lane + 32 * k;
                        slx[k] = c < nx ? a.m.pair_slot[p0x + c] : 0;
                    }
                };
                if (i0 < i1) load_item(i0, p0, n, sl);
                for (int it = i0; it < i1; ++it, ++gi) {
                    const int buf = gi & 1;
                    const uint32_t acc = kAccCol + (uint32_t)buf * kAccCols;
                    int p0n = 0, nn = 0, sln[4] = {0, 0, 0, 0};
                    if (it + 1 < i1) load_item(it + 1, p0n, nn, sln);
                    ok = tc::mbar_wait(&acc_full[buf], (gi >> 1) & 1, abort_flag, kWaitLimit);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) {
                        if (lane == 0 && !*abort_flag) fail(1);
                        break;
                    }
                    tc::tc_fence_after();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (32 * k >= n) break;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int c0 = 32 * k + 16 * h;
                            if (c0 >= n) break;
                            float v[16], tot[16];
                            int slot[16];
                            tc::tmem_ld16(lane_addr + acc + c0, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                slot[i] = __shfl_sync(0xffffffffu, sl[k], 16 * h + i);
                                if (c0 + i < n) tot[i] = tc::tmem_ld1(lane_addr + (uint32_t)slot[i]);
                            }
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (c0 + i < n)
                                    tc::tmem_st1(lane_addr + (uint32_t)slot[i], tot[i] + v[i]);
                        }
                    }
                    // the totals are read again by the next item
                    tc::tmem_wait_st();
                    tc::tc_fence_before();
                    tc::mbar_arrive(&acc_empty[buf]);
                    p0 = p0n;
                    n = nn;
#pragma unroll
                    for (int k = 0; k < 4; ++k) sl[k] = sln[k];
                }
                if (!ok) break;
                // the window's totals to chat (coefficient `row` of each target)
                for (int c0 = 0; c0 < nt; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(lane_addr + c0, v);
                    tc::tmem_wait_ld();
                    if (row < kp) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < nt) {
                                const int tgt = a.m.win_targets[t0 + c0 + i];
                                a.chat[((size_t)tgt * a.nrhs + r) * kp + row] = v[i];
                            }
                    }
                }
            }
    } else if (warp == 8) {
        // ------------------------------------------------ TMA for S_t chunks
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)kp * 128;   // one split of a chunk
            uint32_t j = 0;
            bool ok = true;
            for (int u = w0; u < w1 && ok; ++u)
                for (int r = 0; r < a.nrhs && ok; ++r) {
                    const int win = a.m.cta_win[u];
                    const int i0 = a.m.win_item_ptr[win], i1 = a.m.win_item_ptr[win + 1];
                    for (int it = i0; it < i1 && ok; ++it) {
                        const int row0 = a.m.item_offset[it] * kp;
                        for (int c = 0; c < a.nch; ++c, ++j) {
                            const int s = j % S;
                            ok = tc::mbar_wait(&empty[s], ((j / S) & 1) ^ 1, abort_flag,
                                               kWaitLimit);
                            if (!ok) {
                                if (!*abort_flag) fail(2);
                                break;
                            }
                            tc::mbar_arrive_expect_tx(&full[s], 2 * bytes);
                            tc::tma_load_2d(a_tile(s, 0), &s_hi, &full[s], c * F::kc, row0);
                            tc::tma_load_2d(a_tile(s, 1), &s_lo, &full[s], c * F::kc, row0);
                        }
                    }
                }
            // on abort, let the copies already issued land before the block exits
            if (!ok && j > 0) {
                const uint32_t last = j - 1;
                tc::mbar_wait(&full[last % S], (last / S) & 1, never, kWaitLimit);
            }
        }
    } else {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t s = 0, ph = 0, gi = 0;
            bool ready = false, ok = true;
            const int ks_last = (kp - (a.nch - 1) * F::kc) / F::kstep;
            // operand descriptors of stage 0; stage s is kStageBytes * s further
            const uint64_t da_hi0 = tc::sdesc_k128(tc::smem_u32(a_tile(0, 0)), 1024);
            const uint64_t da_lo0 = tc::sdesc_k128(tc::smem_u32(a_tile(0, 1)), 1024);
            const uint64_t db_hi0 = tc::sdesc_k128(tc::smem_u32(b_tile(0, 0)), 1024);
            const uint64_t db_lo0 = tc::sdesc_k128(tc::smem_u32(b_tile(0, 1)), 1024);
            if (a.test_stall && blockIdx.x == 0) {
                ok = tc::mbar_wait(done, 0, abort_flag, kTestStallLimit);
                if (!ok && !*abort_flag) fail(5);
            }
            for (int u = w0; u < w1 && ok; ++u)
                for (int r = 0; r < a.nrhs && ok; ++r) {
                    const int win = a.m.cta_win[u];
                    const int i0 = a.m.win_item_ptr[win], i1 = a.m.win_item_ptr[win + 1];
                    for (int it = i0; it < i1 && ok; ++it, ++gi) {
                        const int buf = gi & 1;
                        const uint32_t acc = tmem + kAccCol + (uint32_t)buf * kAccCols;
                        ok = tc::mbar_wait(&acc_empty[buf], ((gi >> 1) & 1) ^ 1, abort_flag,
                                           kWaitLimit);
                        if (!ok) {
                            if (!*abort_flag) fail(3);
                            break;
                        }
                        tc::tc_fence_after();
                        const int n = a.m.item_pair_ptr[it + 1] - a.m.item_pair_ptr[it];
                        const uint32_t N = (uint32_t)((n + 15) & ~15);
                        const uint32_t id = tc::idesc(F::ab, 128, N);
                        for (int c = 0; c < a.nch; ++c) {
                            if (!ready) {
                                ok = tc::mbar_wait(&full[s], ph, abort_flag, kWaitLimit);
                                if (!ok) {
                                    if (!*abort_flag) fail(4);
                                    break;
                                }
                            }
                            tc::tc_fence_after();
                            const uint32_t s1 = s + 1 == (uint32_t)S ? 0 : s + 1;
                            const uint32_t ph1 = s1 == 0 ? ph ^ 1 : ph;
                            const bool ready1 = tc::mbar_try_wait(&full[s1], ph1);
                            const int ksteps = c == a.nch - 1 ? ks_last : F::kc / F::kstep;
                            const uint32_t so = s * kStageBytes;
                            const uint64_t dah = tc::sdesc_advance(da_hi0, so);
                            const uint64_t dal = tc::sdesc_advance(da_lo0, so);
                            const uint64_t dbh = tc::sdesc_advance(db_hi0, so);
                            const uint64_t dbl = tc::sdesc_advance(db_lo0, so);
                            // K steps of 32 bytes; the first product of the
                            // item overwrites the accumulator
                            if (c == 0) {
                                tc::mma_c<kTF32, false>(acc, dah, dbh, id);
                            } else {
                                tc::mma_c<kTF32, true>(acc, dah, dbh, id);
                            }
                            tc::mma_c<kTF32, true>(acc, dah, dbl, id);
                            tc::mma_c<kTF32, true>(acc, dal, dbh, id);
#pragma unroll
                            for (int k = 1; k < 4; ++k) {
                                if (k >= ksteps) break;
                                const uint32_t kb = 32u * k;
                                tc::mma_c<kTF32, true>(acc, tc::sdesc_advance(dah, kb),
                                                       tc::sdesc_advance(dbh, kb), id);
                                tc::mma_c<kTF32, true>(acc, tc::sdesc_advance(dah, kb),
                                                       tc::sdesc_advance(dbl, kb), id);
                                tc::mma_c<kTF32, true>(acc, tc::sdesc_advance(dal, kb),
                                                       tc::sdesc_advance(dbh, kb), id);
                            }
                            tc::mma_commit(&empty[s]);
                            s = s1;
                            ph = ph1;
                            ready = ready1;
                        }
                        if (ok) tc::mma_commit(&acc_full[buf]);
                    }
                }
            // every MMA this thread issued has completed before TMEM is freed
            tc::mma_commit(done);
            tc::mbar_wait(done, 0, never, kWaitLimit);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 9) tc::tmem_dealloc(tmem, 512);
}

size_t pc_smem() { return 1024 + (size_t)kStages * kStageBytes + 256; }

} // namespace

cudaError_t launch_m2l_pc(const DevM2LPc &m, const DevOps &o, const DevWork &w, int nnodes,
                          bool tf32, const CUtensorMap &s_hi, const CUtensorMap &s_lo,
                          void *qh_hi, void *qh_lo, int *err, bool test_stall, cudaStream_t st) {
    if (m.ncta == 0) return cudaSuccess;
    const int kp = o.kpad;
    if (kp > 128) return cudaErrorInvalidValue;
    const int64_t nrows = (int64_t)nnodes * w.nrhs;
    // the gatherers address operand rows in 32-bit units of 16 bytes
    if ((nrows + 1) * (int64_t)kp * (tf32 ? 4 : 2) / 16 >= (int64_t)UINT32_MAX)
        return cudaErrorInvalidValue;
    cudaError_t e = launch_split_qhat(w.qhat, nrows, kp, tf32, qh_hi, qh_lo, st);
    if (e != cudaSuccess) return e;
    PcArgs a;
    a.m = m;
    a.nrhs = w.nrhs;
    a.kpad = kp;
    a.nch = (kp * (tf32 ? 4 : 2) + 127) / 128;
    a.qh_hi = static_cast<const uint4 *>(qh_hi);
    a.qh_lo = static_cast<const uint4 *>(qh_lo);
    a.chat = w.chat;
    a.err = err;
    a.test_stall = test_stall ? 1 : 0;
    if (tf32)
        k_m2l_pc<true><<<m.ncta, kThreads, pc_smem(), st>>>(s_hi, s_lo, a);
    else
        k_m2l_pc<false><<<m.ncta, kThreads, pc_smem(), st>>>(s_hi, s_lo, a);
    return cudaGetLastError();
}

cudaError_t configure_m2l_pc(bool tf32) {
    const int sm = (int)pc_smem();
    return tf32 ? cudaFuncSetAttribute(k_m2l_pc<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : cudaFuncSetAttribute(k_m2l_pc<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

} // namespace kifmm
