// V-list M2L on the 5th-generation tensor cores (tcgen05), split precision.
//
// Per M2L tile (128 target rows) and per offset t the tile uses:
//     D[128 x kpad] += X_t[128 x kpad] * S_t^T,   X_t row r = qhat of the
// source at offset t from target r (zero row if none).  Operands are split
// x = x_hi + x_lo in BF16 (kind::f16) or TF32 (kind::tf32) and every K step
// issues x_hi*S_hi + x_hi*S_lo + x_lo*S_hi with FP32 accumulation in TMEM.
// For kpad <= 128 ("wide" products) the first two are one MMA of N = 2 kpad,
// x_hi * [S_hi; S_lo], whose second half accumulates the tile's x_hi*S_lo
// correction over all of its offsets in TMEM columns of its own: two MMAs per
// K step instead of three, the same products.  The correction is 2^-8 (BF16)
// or 2^-11 (TF32) of the total, so its long accumulation adds nothing
// measurable to the error.
//
// Warp roles (448 threads):
//   0-3, 10-13  two sets that gather the 128 rows of X_t for one
//        128-byte K chunk into shared memory in the 128-byte swizzled
//        K-major layout (eight lanes per row, so each warp-wide load covers
//        four whole row chunks); the sets take chunks in turn and issue a
//        chunk's loads before waiting for its stage, so loads overlap the
//        MMAs;
//   4-7  epilogue: every group of offsets, add the TMEM accumulator into a
//        TMEM running total; after the tile's last offset add the wide
//        products' correction columns, zero them for the next tile (and
//        say so on an mbarrier the MMA thread waits on before the next
//        tile) and write the total (FP32) to chat.  The two-level sum keeps
//        the FP32 rounding of the ~189 k products per target at the level
//        the FP32 path reaches;
//   8    TMA loads of the S_t chunks (hi and lo) for the same K chunk, in
//        the order the wide product of the chunk's accumulator reads them;
//   9    allocates TMEM, issues the MMAs (one thread), frees TMEM.
// Roles in the error word: 0 gatherers, 1 epilogue, 2 TMA, 3 and 4 MMA
// thread (accumulator, stage), 5 the test hook's stall.
// Stages of shared memory are recycled through mbarriers: producers wait
// for `empty`, the MMA thread waits for `full` (gatherers and S_t bytes)
// and releases the stage with tcgen05.commit.  Every wait is bounded; on expiry the block
// records the failing role in *err, sets a block-wide abort flag, drains
// what it issued and frees its TMEM before returning.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "tc_ptx.cuh"

namespace kifmm {

namespace {

// Gather sets of 128 threads (warps 0-3, then 10-13, 14-17, ...).  A set
// holds a whole 32 KB K chunk (hi and lo) in registers, 64 per thread; a
// third set would push the shared register count below what the roles need.
constexpr int kSets = 2;
constexpr int kThreads = 32 * (10 + 4 * (kSets - 1));
// Offsets summed in one TMEM accumulator before it is added to the running
// total: the tensor core's FP32 accumulation over long sums loses accuracy
// (all ~189 offsets of a tile in one accumulator: 2.4e-5 relative error
// with BF16x3), so sums are kept short.  BF16x3 uses 4 (its error, 5.5e-6
// against the direct sum, is set by the BF16 split itself); TF32x3 uses 1,
// which its 1e-6 bar needs (4 gave 1.5e-6 against the oracle).  This holds
// for the main terms; the small x_hi*S_lo correction of wide products is
// drained once per tile.
inline int group_for(bool tf32) { return tf32 ? 1 : 4; }
constexpr uint64_t kWaitLimit = 2000000000ull;  // 2 s per wait
constexpr uint32_t kNoRow = 0xFFFFFFFFu;  // gather offset of a row with no source
// Test hook: with TcArgs::test_stall set, block 0's MMA thread first waits
// on `done`, which nothing completes before the thread's own final commit,
// with this shorter limit, so that its expiry (role 5) comes first and the
// block leaves through the same abort path as a real expired wait.
constexpr uint64_t kTestStallLimit = 100000000ull;  // 0.1 s

struct TcArgs {
    DevM2L m;
    int nrhs, kpad, nch, stages, row_chunks, nitems, nbuf, group;
    int wide;  // hi x [S_hi; S_lo] as one N = 2 kpad product (see the MMA issuer)
    uint32_t tmem_cols;
    const uint4 *qh_hi, *qh_lo;   // rows of kpad elements (16-byte pieces)
    int zero_row;                 // index of an all-zero qhat row
    float *chat;
    int *err;                     // device-visible error word (0 = ok)
    int test_stall;               // failure-detection test hook (see below)
};

template <bool kTF32> struct Fmt {
    static constexpr int esize = kTF32 ? 4 : 2;
    static constexpr int kc = 128 / esize;        // elements per 128-byte K chunk
    static constexpr int kstep = kTF32 ? 8 : 16;  // K per MMA instruction (32 bytes)
    static constexpr uint32_t ab = kTF32 ? 2u : 1u;
};

// The (tile, row chunk) items of this block, in the order every role walks
// them: with a schedule, the block's tiles (dealt longest first on the
// host) times all row chunks; without one, every gridDim-th item.
__device__ __forceinline__ int block_items(const TcArgs &a) {
    if (a.m.cta_ptr)
        return (a.m.cta_ptr[blockIdx.x + 1] - a.m.cta_ptr[blockIdx.x]) * a.row_chunks;
    return (int)blockIdx.x < a.nitems ? (a.nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                                       : 0;
}
__device__ __forceinline__ int block_item(const TcArgs &a, int k) {
    if (a.m.cta_ptr) {
        const int tile = a.m.cta_tiles[a.m.cta_ptr[blockIdx.x] + k / a.row_chunks];
        return tile * a.row_chunks + k % a.row_chunks;
    }
    return (int)blockIdx.x + k * (int)gridDim.x;
}

// A read-only 32-bit load issued where it stands in the program (volatile
// asm keeps the compiler from sinking it towards its first use).
__device__ __forceinline__ int ld_nc_s32(const int *p) {
    int v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

template <bool kTF32>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap s_hi, const __grid_constant__ CUtensorMap s_lo,
             TcArgs a) {
    using F = Fmt<kTF32>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int kp = a.kpad, S = a.stages;
    const uint32_t a_bytes = 128 * 128;                // one split of X_t chunk
    const uint32_t b_bytes = (uint32_t)kp * 128;       // one split of S_t chunk
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)S * stage_bytes);
    // full[s]: 128 gatherer arrivals + the TMA thread's arrival with the
    // S_t chunk's bytes, so the MMA thread waits once per stage
    uint64_t *full = bars, *empty = bars + 2 * S;
    uint64_t *acc_full = bars + 3 * S, *acc_empty = acc_full + 2, *done = acc_full + 4;
    // corr_empty: the epilogue has added a tile's correction columns into
    // its total and zeroed them (wide products only)
    uint64_t *corr_empty = done + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(corr_empty + 1);
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
        tc::mbar_init(corr_empty, 128);
        *abort_flag = 0;
        *never = 0;
        tc::fence_mbar_init();
    }
    if (warp == 9) tc::tmem_alloc(tmem_slot, a.tmem_cols);
    if (warp == 8 && lane == 0) {
        tc::prefetch_tmap(&s_hi);
        tc::prefetch_tmap(&s_lo);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // TMEM columns: nbuf accumulators of kp columns, then the running total.
    // With two accumulators the epilogue drains one while the MMAs fill the
    // other.  Wide products: main accumulator 0 at 0, the correction
    // columns at kp, main accumulator 1 at 2 kp, the total at 3 kp, so that
    // either main accumulator and the correction are kp-column neighbours
    // (0 and 1: [main0 | corr], [corr | main1]).
    const int nbuf = a.nbuf;
    const uint32_t tot_col = a.wide ? (uint32_t)(3 * kp) : (uint32_t)(nbuf * kp);
    auto main_col = [&](int buf) {
        return a.wide ? (uint32_t)(buf ? 2 * kp : 0) : (uint32_t)(buf * kp);
    };
    const uint32_t corr_col = (uint32_t)kp;

    auto a_tile = [&](int s, int split) { return smem + (size_t)s * stage_bytes + split * a_bytes; };
    auto b_tile = [&](int s, int split) {
        return smem + (size_t)s * stage_bytes + 2 * a_bytes + split * b_bytes;
    };
    auto fail = [&](int role) {
        *abort_flag = 1;
        atomicOr(a.err, 1 << role);
    };

    if (warp < 4 || warp >= 10) {
        // ------------------------------------------------ X_t row gatherers
        // kSets sets of 128 threads take K chunks in turn, so kSets chunks'
        // loads are in flight while the MMAs consume earlier stages.  Within
        // a set, eight lanes share a row (one 16-byte piece each), so one
        // warp-wide load reads four whole 128-byte row chunks; a thread
        // covers the rows (4 wi + i) * 4 + sub, i < 8, of its warp wi.
        const int set = warp < 4 ? 0 : 1 + (warp - 10) / 4;
        const int wi = warp < 4 ? warp : (warp - 10) % 4;   // warp within the set
        const int piece = lane & 7, sub = lane >> 3;
        uint32_t j = 0;
        bool ok = true;
        const int row16 = kp * F::esize / 16;
        for (int k = 0, nk = block_items(a); k < nk && ok; ++k) {
            const int item = block_item(a, k);
            const int tile = item / a.row_chunks, rc = item - tile * a.row_chunks;
            const int e0 = a.m.tile_entry_ptr[tile], e1 = a.m.tile_entry_ptr[tile + 1];
            // tile slot of each of this thread's eight rows (row g of the
            // item is slot g / nrhs, right-hand side g mod nrhs)
            int slot[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) slot[i] = (rc * 128 + (wi * 8 + i) * 4 + sub) / a.nrhs;
            // source boxes of the rows for the current entry; the next
            // entry's are loaded one entry ahead (in program order, so their
            // latency overlaps this entry's copies)
            int src[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                src[i] = e0 < e1 ? ld_nc_s32(a.m.entry_src + (size_t)e0 * kTileRows + slot[i]) : -1;
            for (int e = e0; e < e1 && ok; ++e) {
                int nsrc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    nsrc[i] = e + 1 < e1
                                  ? ld_nc_s32(a.m.entry_src + (size_t)(e + 1) * kTileRows + slot[i])
                                  : -1;
                // source row of each of this thread's eight tile rows, as an
                // offset in 16-byte pieces; kNoRow where the target has no
                // source at this offset (the row is zero and is not loaded:
                // on adaptive trees most tile rows of an entry are such rows)
                uint32_t qoff[8];   // < 2^32 - 1: checked by the launcher
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rhs = rc * 128 + (wi * 8 + i) * 4 + sub - slot[i] * a.nrhs;
                    qoff[i] = src[i] >= 0 ? (uint32_t)(src[i] * a.nrhs + rhs) * (uint32_t)row16 +
                                                (uint32_t)piece
                                          : kNoRow;
                }
                for (int c = 0; c < a.nch && ok; ++c, ++j) {
                    if ((int)(j % kSets) != set) continue;
                    const int s = j % S;
                    const int valid = min(F::kc, kp - c * F::kc);   // elements in this chunk
                    const bool mine = piece * 16 < valid * F::esize; // this lane's piece exists
                    uint4 vh[8], vl[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        vh[i] = vl[i] = make_uint4(0u, 0u, 0u, 0u);
                        if (mine && qoff[i] != kNoRow) {
                            vh[i] = __ldg(a.qh_hi + qoff[i] + c * 8);
                            vl[i] = __ldg(a.qh_lo + qoff[i] + c * 8);
                        }
                    }
                    ok = tc::mbar_wait(&empty[s], ((j / S) & 1) ^ 1, abort_flag, kWaitLimit);
                    if (!ok) {
                        if (!*abort_flag) fail(0);
                        break;
                    }
                    unsigned char *th = a_tile(s, 0), *tl = a_tile(s, 1);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (mine) {
                            const int r = (wi * 8 + i) * 4 + sub;
                            const uint32_t off = (r >> 3) * 1024 + (r & 7) * 128 +
                                                 ((piece ^ (r & 7)) << 4);
                            *reinterpret_cast<uint4 *>(th + off) = vh[i];
                            *reinterpret_cast<uint4 *>(tl + off) = vl[i];
                        }
                    tc::fence_proxy_async_smem();
                    tc::mbar_arrive(&full[s]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) src[i] = nsrc[i];
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ epilogue
        const int q = warp - 4;               // TMEM lane quarter
        const int row = q * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t gi = 0;
        bool ok = true;
        const float zero16[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f,
                                  0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (a.wide) {
            // the correction columns start at zero
            for (int cc = 0; cc < kp; cc += 16) tc::tmem_st16(lane_addr + corr_col + cc, zero16);
            tc::tmem_wait_st();
            tc::tc_fence_before();
            tc::mbar_arrive(corr_empty);
        }
        for (int k = 0, nk = block_items(a); k < nk && ok; ++k) {
            const int item = block_item(a, k);
            const int tile = item / a.row_chunks, rc = item - tile * a.row_chunks;
            const int g = rc * 128 + row;
            const int slot = g / a.nrhs, rhs = g - slot * a.nrhs;
            const int tgt = a.m.tile_target[(size_t)tile * kTileRows + slot];
            const int ne = a.m.tile_entry_ptr[tile + 1] - a.m.tile_entry_ptr[tile];
            const int ngroups = (ne + a.group - 1) / a.group;
            for (int grp = 0; grp < ngroups; ++grp, ++gi) {
                const int buf = gi % nbuf;
                const uint32_t acc_col = main_col(buf);
                ok = tc::mbar_wait(&acc_full[buf], (gi / nbuf) & 1, abort_flag, kWaitLimit);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0 && !*abort_flag) fail(1);
                    break;
                }
                tc::tc_fence_after();
                const bool first = grp == 0, last = grp == ngroups - 1;
                for (int cc = 0; cc < kp; cc += 16) {
                    float v[16], t[16], u[16];
                    tc::tmem_ld16(lane_addr + acc_col + cc, v);
                    if (!first) tc::tmem_ld16(lane_addr + tot_col + cc, t);
                    if (last && a.wide) tc::tmem_ld16(lane_addr + corr_col + cc, u);
                    tc::tmem_wait_ld();
                    if (first) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) t[i] = v[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) t[i] += v[i];
                    }
                    if (last && a.wide) {
                        // the tile's hi x lo correction, then zero it for the next tile
#pragma unroll
                        for (int i = 0; i < 16; ++i) t[i] += u[i];
                        tc::tmem_st16(lane_addr + corr_col + cc, zero16);
                    }
                    if (last) {
                        if (slot < kTileRows && tgt >= 0) {
                            float4 *out = reinterpret_cast<float4 *>(
                                a.chat + ((size_t)tgt * a.nrhs + rhs) * kp + cc);
                            out[0] = make_float4(t[0], t[1], t[2], t[3]);
                            out[1] = make_float4(t[4], t[5], t[6], t[7]);
                            out[2] = make_float4(t[8], t[9], t[10], t[11]);
                            out[3] = make_float4(t[12], t[13], t[14], t[15]);
                        }
                    } else {
                        tc::tmem_st16(lane_addr + tot_col + cc, t);
                    }
                }
                tc::tmem_wait_st();
                tc::tc_fence_before();
                tc::mbar_arrive(&acc_empty[buf]);
                if (last && a.wide) tc::mbar_arrive(corr_empty);
            }
        }
    } else if (warp == 8) {
        // ------------------------------------------------ TMA for S_t chunks
        if (lane == 0) {
            uint32_t j = 0, gbase = 0;
            bool ok = true;
            for (int k = 0, nk = block_items(a); k < nk && ok; ++k) {
                const int item = block_item(a, k);
                const int tile = item / a.row_chunks;
                const int e0 = a.m.tile_entry_ptr[tile], e1 = a.m.tile_entry_ptr[tile + 1];
                const uint32_t gfirst = gbase;
                gbase += (uint32_t)((e1 - e0 + a.group - 1) / a.group);
                for (int e = e0; e < e1 && ok; ++e) {
                    const int row0 = a.m.entry_offset[e] * kp;
                    // wide products: S_hi first for accumulator 0, S_lo first
                    // for accumulator 1 (see the MMA issuer)
                    const int p = a.wide ? (int)((gfirst + (uint32_t)((e - e0) / a.group)) & 1u) : 0;
                    for (int c = 0; c < a.nch; ++c, ++j) {
                        const int s = j % S;
                        ok = tc::mbar_wait(&empty[s], ((j / S) & 1) ^ 1, abort_flag, kWaitLimit);
                        if (!ok) {
                            if (!*abort_flag) fail(2);
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&full[s], 2 * b_bytes);
                        tc::tma_load_2d(b_tile(s, p), &s_hi, &full[s], c * F::kc, row0);
                        tc::tma_load_2d(b_tile(s, 1 - p), &s_lo, &full[s], c * F::kc, row0);
                    }
                }
            }
            // on abort, let the copies already issued land before the block
            // exits (the phase may also lack gatherer arrivals, so this wait
            // can run to its limit; the copies take microseconds)
            if (!ok && j > 0) {
                const uint32_t last = j - 1;
                tc::mbar_wait(&full[last % S], (last / S) & 1, never, kWaitLimit);
            }
        }
    } else {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id = tc::idesc(F::ab, 128, (uint32_t)kp);
            const uint32_t id2 = tc::idesc(F::ab, 128, 2u * (uint32_t)kp);
            // The MMA thread is the critical path: tcgen05.mma issue proceeds
            // at the tensor pipe's pace, so everything else it does per stage
            // adds to the kernel's time.  Stage and phase advance by counting;
            // the next stage's barrier is polled before this stage's MMAs are
            // issued, so that poll's latency overlaps the issue.
            uint32_t s = 0, ph = 0, gi = 0, citem = 0;
            bool ready = false;
            bool ok = true;
            const int ks_last = (kp - (a.nch - 1) * F::kc) / F::kstep;
            // operand descriptors of stage 0; stage s is stage_bytes * s further
            const uint64_t da_hi0 = tc::sdesc_k128(tc::smem_u32(a_tile(0, 0)), 1024);
            const uint64_t da_lo0 = tc::sdesc_k128(tc::smem_u32(a_tile(0, 1)), 1024);
            const uint64_t db_hi0 = tc::sdesc_k128(tc::smem_u32(b_tile(0, 0)), 1024);
            const uint64_t db_lo0 = tc::sdesc_k128(tc::smem_u32(b_tile(0, 1)), 1024);
            if (a.test_stall && blockIdx.x == 0) {
                ok = tc::mbar_wait(done, 0, abort_flag, kTestStallLimit);
                if (!ok && !*abort_flag) fail(5);
            }
            for (int k = 0, nk = block_items(a); k < nk && ok; ++k) {
                const int item = block_item(a, k);
                const int tile = item / a.row_chunks;
                const int e0 = a.m.tile_entry_ptr[tile], e1 = a.m.tile_entry_ptr[tile + 1];
                if (a.wide && e1 > e0) {
                    // the previous tile's correction columns are drained and zero
                    ok = tc::mbar_wait(corr_empty, citem & 1u, abort_flag, kWaitLimit);
                    if (!ok) {
                        if (!*abort_flag) fail(3);
                        break;
                    }
                    ++citem;
                }
                for (int eg = e0; eg < e1 && ok; eg += a.group, ++gi) {
                    const int buf = gi % nbuf;
                    const uint32_t acc_col = main_col(buf);
                    ok = tc::mbar_wait(&acc_empty[buf], ((gi / nbuf) & 1) ^ 1, abort_flag,
                                       kWaitLimit);
                    if (!ok) {
                        if (!*abort_flag) fail(3);
                        break;
                    }
                    tc::tc_fence_after();
                    bool first = true;  // the group's first product overwrites the accumulator
                    const int eend = min(e1, eg + a.group);
                    for (int e = eg; e < eend && ok; ++e) {
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
                            const uint32_t so = s * stage_bytes;
                            const uint64_t dah = tc::sdesc_advance(da_hi0, so);
                            const uint64_t dal = tc::sdesc_advance(da_lo0, so);
                            const uint64_t dbh = tc::sdesc_advance(db_hi0, so);
                            const uint64_t dbl = tc::sdesc_advance(db_lo0, so);
                            const uint32_t d = tmem + acc_col;
                            if (a.wide) {
                                // per K step: lo x S_hi into the main accumulator
                                // (the group's first overwrites it), then
                                // hi x [S_hi; S_lo] (or [S_lo; S_hi] for accumulator 1)
                                // as one N = 2 kp product into the main accumulator
                                // and the tile's correction columns
                                const uint32_t dw = tmem + (buf ? (uint32_t)kp : 0u);
                                const uint64_t db2 = dbh;
                                const uint64_t dbx = buf ? dbl : dbh;   // where S_hi is
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    if (kk >= ksteps) break;
                                    const uint32_t kb = 32u * kk;
                                    if (first) {
                                        tc::mma_c<kTF32, false>(d, tc::sdesc_advance(dal, kb),
                                                                tc::sdesc_advance(dbx, kb), id);
                                        first = false;
                                    } else {
                                        tc::mma_c<kTF32, true>(d, tc::sdesc_advance(dal, kb),
                                                               tc::sdesc_advance(dbx, kb), id);
                                    }
                                    tc::mma_c<kTF32, true>(dw, tc::sdesc_advance(dah, kb),
                                                           tc::sdesc_advance(db2, kb), id2);
                                }
                                tc::mma_commit(&empty[s]);
                                s = s1;
                                ph = ph1;
                                ready = ready1;
                                continue;
                            }
                            if (first) {
                                tc::mma_c<kTF32, false>(d, dah, dbh, id);
                                first = false;
                            } else {
                                tc::mma_c<kTF32, true>(d, dah, dbh, id);
                            }
                            tc::mma_c<kTF32, true>(d, dah, dbl, id);
                            tc::mma_c<kTF32, true>(d, dal, dbh, id);
#pragma unroll
                            for (int k = 1; k < 4; ++k) {
                                if (k >= ksteps) break;
                                const uint32_t kb = 32u * k;
                                tc::mma_c<kTF32, true>(d, tc::sdesc_advance(dah, kb),
                                                       tc::sdesc_advance(dbh, kb), id);
                                tc::mma_c<kTF32, true>(d, tc::sdesc_advance(dah, kb),
                                                       tc::sdesc_advance(dbl, kb), id);
                                tc::mma_c<kTF32, true>(d, tc::sdesc_advance(dal, kb),
                                                       tc::sdesc_advance(dbh, kb), id);
                            }
                            tc::mma_commit(&empty[s]);
                            s = s1;
                            ph = ph1;
                            ready = ready1;
                        }
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
    if (warp == 9) tc::tmem_dealloc(tmem, a.tmem_cols);
}

// Split qhat (FP32) into hi/lo rows in the operand format; the row after the
// last is all zero (the source of rows that have none).
template <bool kTF32>
__global__ void k_split_qhat(const float *__restrict__ qhat, int64_t nrows, int kp, void *hi,
                             void *lo) {
    const int64_t total = (nrows + 1) * kp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = i < nrows * kp ? qhat[i] : 0.f;
        if (kTF32) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
            const float r = x - __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
            static_cast<uint32_t *>(hi)[i] = h;
            static_cast<uint32_t *>(lo)[i] = l;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
            static_cast<__nv_bfloat16 *>(hi)[i] = h;
            static_cast<__nv_bfloat16 *>(lo)[i] = l;
        }
    }
}

} // namespace

cudaError_t launch_split_qhat(const float *qhat, int64_t nrows, int kp, bool tf32, void *hi,
                              void *lo, cudaStream_t st) {
    const int64_t total = (nrows + 1) * kp;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)152 * 16);
    if (tf32)
        k_split_qhat<true><<<blocks, 256, 0, st>>>(qhat, nrows, kp, hi, lo);
    else
        k_split_qhat<false><<<blocks, 256, 0, st>>>(qhat, nrows, kp, hi, lo);
    return cudaGetLastError();
}

size_t m2l_tc_smem(int kpad, int *stages) {
    const size_t stage = 2 * 128 * 128 + 2 * (size_t)kpad * 128;
    const size_t budget = 227 * 1024 - 1024 - 256;
    int s = (int)(budget / stage);
    if (s > 4) s = 4;
    if (stages) *stages = s;
    return 1024 + (size_t)s * stage + 256;
}

cudaError_t launch_m2l_tc(const DevM2L &m, const DevOps &o, const DevWork &w, int nnodes,
                          bool tf32, const CUtensorMap &s_hi, const CUtensorMap &s_lo,
                          void *qh_hi, void *qh_lo, int *err, bool test_stall, int num_sms,
                          cudaStream_t st) {
    if (m.ntiles == 0) return cudaSuccess;
    const int kp = o.kpad;
    const int64_t nrows = (int64_t)nnodes * w.nrhs;
    // the gatherers address operand rows in 32-bit units of 16 bytes
    if ((nrows + 1) * (int64_t)kp * (tf32 ? 4 : 2) / 16 >= (int64_t)UINT32_MAX)
        return cudaErrorInvalidValue;
    // 1. operand split of the compressed multipoles
    {
        cudaError_t e = launch_split_qhat(w.qhat, nrows, kp, tf32, qh_hi, qh_lo, st);
        if (e != cudaSuccess) return e;
    }
    TcArgs a;
    a.m = m;
    a.nrhs = w.nrhs;
    a.kpad = kp;
    a.nch = (kp * (tf32 ? 4 : 2) + 127) / 128;
    a.row_chunks = w.nrhs;
    a.nitems = m.ntiles * a.row_chunks;
    a.nbuf = 3 * kp <= 512 ? 2 : 1;
    a.wide = 4 * kp <= 512 ? 1 : 0;
    a.group = group_for(tf32);
    uint32_t cols = 32;
    while (cols < (uint32_t)((a.wide ? 4 : a.nbuf + 1) * kp)) cols <<= 1;
    a.tmem_cols = cols;
    a.qh_hi = static_cast<const uint4 *>(qh_hi);
    a.qh_lo = static_cast<const uint4 *>(qh_lo);
    a.zero_row = (int)nrows;
    a.chat = w.chat;
    a.err = err;
    a.test_stall = test_stall ? 1 : 0;
    const size_t sm = m2l_tc_smem(kp, &a.stages);
    // the plan's block schedule, when it was made for this many blocks
    if (a.m.ncta != num_sms) a.m.cta_ptr = a.m.cta_tiles = nullptr;
    const int grid = a.m.cta_ptr ? a.m.ncta : std::min(a.nitems, num_sms);
    if (tf32)
        k_m2l_tc<true><<<grid, kThreads, sm, st>>>(s_hi, s_lo, a);
    else
        k_m2l_tc<false><<<grid, kThreads, sm, st>>>(s_hi, s_lo, a);
    return cudaGetLastError();
}

cudaError_t configure_m2l_tc(int kpad, bool tf32) {
    const int sm = (int)m2l_tc_smem(kpad, nullptr);
    return tf32 ? cudaFuncSetAttribute(k_m2l_tc<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                : cudaFuncSetAttribute(k_m2l_tc<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

} // namespace kifmm
