// C ABI of the library (include/kifmm.h): plan creation, evaluation and
// inspection.  The evaluation enqueues, on the caller's stream:
//   gather charges into tree order -> P2M -> M2M (levels depth-1 .. 2)
//   -> M2L over V (all levels, one launch) -> P2L over X
//   -> downward step (levels 2 .. depth) -> leaf evaluation (U, L2P, W)
// which is the operator order of "Computational structure of FMM operators"
// with the near field fused into the leaf pass.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "device.cuh"
#include "kifmm.h"
#include "linalg.h"
#include "plan.h"
#include "plan_impl.h"

using namespace kifmm;

namespace {

thread_local std::string g_error;

fmm_status fail(fmm_status s, const std::string &msg) {
    g_error = msg;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

std::vector<float> to_f32(const std::vector<double> &v) {
    return std::vector<float>(v.begin(), v.end());
}

} // namespace

struct fmm_plan_s {
    fmm_options opts;
    int p = 0, ncrit = 0, device = 0;
    int64_t rows = 0;             // caller rows of charges and potentials
    int device_trees = 0;         // problems whose tree was built on the device
    Tree tree;
    M2LTable m2l;
    M2LWindows m2lw;              // pair-column M2L work table
    Schedules sched;
    std::shared_ptr<const Operators> ops;
    int ops_source = kOpsComputed;   // FMM_INFO_OPERATOR_SOURCE
    int kpad = 0;
    bool timing = false;
    std::vector<void *> allocs;   // plan-lifetime device memory
    DevTree dt{};
    DevOps dops{};
    DevM2L dm{};
    DevM2LPc dpc{};
    int *d_p2m = nullptr, *d_m2m = nullptr, *d_down = nullptr, *d_chunks = nullptr,
        *d_xnodes = nullptr;
    // index lists of the level products: children of every internal box
    // (sigma-major over m2m_nodes), M2L source of each box (itself or -1),
    // parent's position within its level's internal boxes, child offset
    // (sigma * rQ) into the parent's stacked L2L output
    int *d_m2m_child = nullptr, *d_chat_src = nullptr, *d_ppos = nullptr, *d_poff = nullptr;
    int max_level_nodes = 0, max_level_internal = 0;
    // workspace, sized for nrhs_cap right-hand sides
    int nrhs_cap = 0;
    float *qs = nullptr, *up = nullptr, *down = nullptr, *qhat = nullptr, *chat = nullptr,
          *xchk = nullptr, *charges_stage = nullptr, *chk = nullptr, *ybuf = nullptr,
          *yp = nullptr, *part = nullptr;
    double *pot_stage = nullptr, *grad_stage = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    cudaStream_t last_stream = nullptr;
    int last_nrhs = 0;               // nrhs of the last fmm_evaluate(_gradient)
    int64_t last_launches = 0;
    int num_sms = 0;
    // tensor-core M2L: split S_t arrays and their TMA maps, per mode
    // (index 0: BF16x3, 1: TF32x3)
    void *s_split[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    CUtensorMap tmap[2][2];
    bool tc_ready[2] = {false, false};
    float *qh_hi = nullptr, *qh_lo = nullptr;   // split qhat (4-byte slots)
    int qh_cap = 0;                             // nrhs the split buffers hold
    int *err_host = nullptr, *err_dev = nullptr;  // mapped pinned error word
    int test_m2l_stall = 0;                     // FMM_OPT_TEST_M2L_STALL
    int m2l_kernel = 1;                         // FMM_OPT_M2L_KERNEL
    // side stream of the upward pass: each level's M2L projection (qhat =
    // Vk^T rho, needed only by the M2L) runs there while the next level's
    // M2M proceeds; joined before the M2L
    cudaStream_t s_side = nullptr;
    cudaEvent_t ev_side[2] = {nullptr, nullptr};
    // Autotuner: tile shape per level-product call site (in enqueue order),
    // chosen by timing every shape during the first evaluation of each nrhs
    // and kept per nrhs; forced_shape >= 0 applies one shape everywhere
    // instead.  gemm_shape holds the choices of the evaluation being
    // enqueued.
    bool autotune = true;
    int forced_shape = -1;
    bool tuning = false;
    std::map<int, std::vector<int>> tuned_shapes;   // nrhs -> shapes per site
    std::vector<int> gemm_shape;
    std::vector<float> gemm_ms;   // best time per site (ms) of the last tuning
    // Two more tuned choices that keep every summation order (so the results
    // are the same bits either way), kept per nrhs like the shapes:
    // knob[0] the target-tile M2L's block schedule (1 longest-first tiles,
    // 0 round robin), knob[1] the leaf pass's launch order (0 widest group
    // first, 1 narrowest first).  forced_knobs >= 0 sets both (bit 0, bit 1).
    int knob[2] = {1, 0};
    int forced_knobs = -1;
    std::map<int, std::array<int, 2>> tuned_knobs;
    // CUDA graphs of recent evaluations, each replayed while its key holds:
    // the caller's buffers, nrhs, the M2L mode and kernel, and the workspace
    // generation; the least recently used of kGraphCache is dropped first
    bool use_graph = true;
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        const void *charges = nullptr, *pot = nullptr, *grad = nullptr;
        int nrhs = 0, mode = -1, kernel = -1;
        uint64_t ws_gen = 0, used = 0;
    };
    static constexpr int kGraphCache = 4;
    GraphEntry graphs[kGraphCache];
    uint64_t graph_clock = 0;
    uint64_t ws_gen = 0;
    void drop_graph() {
        for (GraphEntry &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = GraphEntry();
        }
    }

    ~fmm_plan_s() {
        if (opts.host_only) return;
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        for (void *a : allocs) cudaFree(a);
        free_workspace();
        for (auto &m : s_split)
            for (void *a : m)
                if (a) cudaFree(a);
        if (qh_hi) cudaFree(qh_hi);
        if (qh_lo) cudaFree(qh_lo);
        if (err_host) cudaFreeHost(err_host);
        drop_graph();
        for (auto &e : ev_side)
            if (e) cudaEventDestroy(e);
        if (s_side) cudaStreamDestroy(s_side);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (auto &e : tune_ev)
            if (e) cudaEventDestroy(e);
        cudaSetDevice(prev);
    }
    void free_workspace() {
        ++ws_gen;
        void *w[] = {qs,    up,        down,       qhat, chat, xchk, charges_stage,
                     pot_stage, grad_stage, chk, ybuf, yp,   part};
        for (void *a : w)
            if (a) cudaFree(a);
        qs = up = down = qhat = chat = xchk = charges_stage = chk = ybuf = yp = part = nullptr;
        pot_stage = grad_stage = nullptr;
        nrhs_cap = 0;
    }
    template <class T> fmm_status upload(const std::vector<T> &v, T **out) {
        *out = nullptr;
        size_t bytes = v.size() * sizeof(T);
        if (bytes == 0) bytes = sizeof(T);
        void *d = nullptr;
        CK(cudaMalloc(&d, bytes));
        allocs.push_back(d);
        if (!v.empty()) CK(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        *out = static_cast<T *>(d);
        return FMM_OK;
    }
};

namespace {

uint16_t bf16_rn(float f) {  // round to nearest even, finite inputs
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
float tf32_rn(float f) {  // 10-bit mantissa, round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up
// once; no link against the driver library).
fmm_status encode_fn(EncodeTiledFn *out) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                            &q));
        if (!f || q != cudaDriverEntryPointSuccess)
            return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    *out = fn;
    return FMM_OK;
}

// Split S_t (FP64) into hi/lo operand arrays [316][kpad][kpad] (row n holds
// S_t[n][0..kpad)) and encode their TMA maps (boxes of 128 bytes x kpad rows,
// 128-byte swizzle).
fmm_status prepare_tc(fmm_plan_s *P, int mode) {
    const int idx = mode == FMM_M2L_TF32X3 ? 1 : 0;
    if (P->tc_ready[idx]) return FMM_OK;
    const int kp = P->kpad, k = P->ops->k;
    if (kp > 256)
        return fail(FMM_ERR_UNSUPPORTED, "tensor-core M2L needs rank k <= 256 (raise eps_svd)");
    const bool tf = idx == 1;
    const size_t esize = tf ? 4 : 2;
    const size_t count = (size_t)kNumOffsets * kp * kp;
    std::vector<uint16_t> bh, bl;
    std::vector<float> th, tl;
    if (tf) {
        th.assign(count, 0.f);
        tl.assign(count, 0.f);
    } else {
        bh.assign(count, 0);
        bl.assign(count, 0);
    }
    const std::vector<double> &S = P->ops->S;
    for (int t = 0; t < kNumOffsets; ++t)
        for (int n = 0; n < k; ++n)
            for (int j = 0; j < k; ++j) {
                const double x = S[(size_t)t * k * k + (size_t)n * k + j];
                const size_t o = (size_t)t * kp * kp + (size_t)n * kp + j;
                if (tf) {
                    const float h = tf32_rn((float)x);
                    th[o] = h;
                    tl[o] = tf32_rn((float)(x - (double)h));
                } else {
                    const uint16_t h = bf16_rn((float)x);
                    bh[o] = h;
                    bl[o] = bf16_rn((float)(x - (double)bf16_val(h)));
                }
            }
    for (int sp = 0; sp < 2; ++sp) {
        CK(cudaMalloc(&P->s_split[idx][sp], count * esize));
        const void *src = tf ? (const void *)(sp ? tl.data() : th.data())
                             : (const void *)(sp ? bl.data() : bh.data());
        CK(cudaMemcpy(P->s_split[idx][sp], src, count * esize, cudaMemcpyHostToDevice));
    }
    EncodeTiledFn fn = nullptr;
    if (fmm_status st = encode_fn(&fn)) return st;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)kNumOffsets * kp};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * esize};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)kp};
    const cuuint32_t estr[2] = {1, 1};
    for (int sp = 0; sp < 2; ++sp) {
        CUresult r = fn(
            &P->tmap[idx][sp], tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
            2, P->s_split[idx][sp], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    }
    CK(configure_m2l_tc(kp, tf));
    CK(configure_m2l_pc(tf));
    P->tc_ready[idx] = true;
    return FMM_OK;
}

// The tensor-core modes run the pair-column kernel when the option asks for
// it and the operand width fits its 128 rows, else the target-tile kernel.
bool m2l_uses_pair_columns(const fmm_plan_s *P) {
    return P->m2l_kernel == 0 && P->kpad <= 128 && P->dpc.ncta > 0;
}

fmm_status upload_plan(fmm_plan_s *P) {
    const Tree &t = P->tree;
    const Operators &o = *P->ops;
    const int64_t nn = t.nodes();
    // points and nodes
    std::vector<float4> pts(t.n), pts_lo(t.n);
    for (int64_t i = 0; i < t.n; ++i) {
        pts[i] = make_float4(t.rel[4 * i], t.rel[4 * i + 1], t.rel[4 * i + 2], 0.f);
        pts_lo[i] = make_float4(t.rel_lo[4 * i], t.rel_lo[4 * i + 1], t.rel_lo[4 * i + 2], 0.f);
    }
    std::vector<float4> geom(nn);
    std::vector<int2> range(nn);
    std::vector<int> level(nn);
    for (int64_t b = 0; b < nn; ++b) {
        geom[b] = make_float4((float)t.node_centre(b, 0), (float)t.node_centre(b, 1),
                              (float)t.node_centre(b, 2), (float)t.node_half_width(b));
        range[b] = make_int2((int)t.begin[b], (int)t.end[b]);
        level[b] = t.key[4 * b];
    }
    auto to32 = [](const std::vector<int64_t> &v) { return std::vector<int>(v.begin(), v.end()); };
    DevTree &d = P->dt;
    d.n = t.n;
    d.nnodes = (int)nn;
    d.depth = t.depth;
    d.nleaves = (int)t.leaves.size();
    fmm_status s;
    float4 *dp;
    if ((s = P->upload(pts, &dp))) return s;
    d.pts = dp;
    if ((s = P->upload(pts_lo, &dp))) return s;
    d.pts_lo = dp;
    int64_t *dq, *dout;
    if ((s = P->upload(t.qidx, &dq))) return s;
    if (t.oidx == t.qidx) {
        dout = dq;
    } else if ((s = P->upload(t.oidx, &dout))) {
        return s;
    }
    d.qidx = dq;
    d.oidx = dout;
    {
        // 1 / (4 pi hw) of each box's problem (positions are in root units)
        std::vector<double> sc(nn);
        for (int64_t b = 0; b < nn; ++b)
            sc[b] = 1.0 / (4.0 * M_PI * t.roots[4 * (size_t)t.node_problem[b] + 3]);
        double *dsc;
        if ((s = P->upload(sc, &dsc))) return s;
        d.node_scale = dsc;
    }
    float4 *dg;
    if ((s = P->upload(geom, &dg))) return s;
    d.geom = dg;
    int2 *dr;
    if ((s = P->upload(range, &dr))) return s;
    d.range = dr;
    int *tmp;
#define UP32(vec, field)                                  \
    if ((s = P->upload(vec, &tmp))) return s;             \
    d.field = tmp;
    UP32(level, level);
    UP32(t.parent, parent);
    UP32(t.child, child);
    {
        // leaves grouped by the leaf pass's targets per lane (one kernel per
        // group, so each gets the register budget and occupancy of its width)
        std::vector<int> by_t;
        by_t.reserve(t.leaves.size());
        d.t_first[kLeafWidths] = 0;
        for (int w = kLeafWidths; w >= 1; --w) {
            for (int32_t lf : t.leaves) {
                const int64_t np = t.end[lf] - t.begin[lf];
                const int tw = (int)std::min<int64_t>(kLeafWidths,
                                                      std::max<int64_t>(1, (np + 15) / 16));
                if (tw == w) by_t.push_back(lf);
            }
            d.t_first[w - 1] = (int)by_t.size();
        }
        UP32(by_t, leaves);
    }
    UP32(to32(t.u_ptr), u_ptr);
    UP32(t.u_idx, u_idx);
    UP32(to32(t.w_ptr), w_ptr);
    UP32(t.w_idx, w_idx);
    UP32(to32(t.x_ptr), x_ptr);
    UP32(t.x_idx, x_idx);
    UP32(to32(t.v_ptr), v_ptr);
    UP32(P->sched.x_slot, x_slot);
    UP32(P->sched.w_direct, w_direct);
#undef UP32
    if ((s = P->upload(P->sched.p2m_nodes, &P->d_p2m))) return s;
    if ((s = P->upload(P->sched.m2m_nodes, &P->d_m2m))) return s;
    if ((s = P->upload(P->sched.down_nodes, &P->d_down))) return s;
    if ((s = P->upload(P->sched.down_chunk, &P->d_chunks))) return s;
    if ((s = P->upload(P->sched.x_nodes, &P->d_xnodes))) return s;
    {
        const Schedules &sc = P->sched;
        const int total = (int)sc.m2m_nodes.size();
        std::vector<int> child((size_t)8 * total), chat_src(nn, -1), ppos(nn, -1), poff(nn, 0);
        std::vector<int> pos_in_level(nn, -1);
        for (int l = 0; l <= t.depth; ++l)
            for (int q = sc.m2m_level_ptr[l]; q < sc.m2m_level_ptr[l + 1]; ++q) {
                const int b = sc.m2m_nodes[q];
                pos_in_level[b] = q - sc.m2m_level_ptr[l];
                for (int sg = 0; sg < 8; ++sg) child[(size_t)sg * total + q] = t.child[8 * b + sg];
            }
        for (int64_t b = 0; b < nn; ++b) {
            if (t.v_ptr[b + 1] > t.v_ptr[b]) chat_src[b] = (int)b;
            const int l = t.key[4 * b];
            if (l >= 3) ppos[b] = pos_in_level[t.parent[b]];
            const int sg = (t.key[4 * b + 1] & 1) | ((t.key[4 * b + 2] & 1) << 1) |
                           ((t.key[4 * b + 3] & 1) << 2);
            poff[b] = sg * o.rQ;
        }
        if ((s = P->upload(child, &P->d_m2m_child))) return s;
        if ((s = P->upload(chat_src, &P->d_chat_src))) return s;
        if ((s = P->upload(ppos, &P->d_ppos))) return s;
        if ((s = P->upload(poff, &P->d_poff))) return s;
        for (int l = 0; l <= t.depth; ++l) {
            P->max_level_nodes = std::max(P->max_level_nodes, t.level_ptr[l + 1] - t.level_ptr[l]);
            P->max_level_internal =
                std::max(P->max_level_internal, sc.m2m_level_ptr[l + 1] - sc.m2m_level_ptr[l]);
        }
        P->max_level_nodes = std::max(P->max_level_nodes, (int)sc.p2m_nodes.size());
    }

    // M2L tables
    DevM2L &m = P->dm;
    m.ntiles = (int)P->m2l.tile_level.size();
    int *mt;
    if ((s = P->upload(P->m2l.tile_target, &mt))) return s;
    m.tile_target = mt;
    if ((s = P->upload(P->m2l.tile_entry_ptr, &mt))) return s;
    m.tile_entry_ptr = mt;
    if ((s = P->upload(P->m2l.entry_offset, &mt))) return s;
    m.entry_offset = mt;
    if ((s = P->upload(P->m2l.entry_src, &mt))) return s;
    m.entry_src = mt;
    m.ncta = P->m2l.ncta;
    m.cta_ptr = m.cta_tiles = nullptr;
    if (m.ncta > 0) {
        if ((s = P->upload(P->m2l.cta_ptr, &mt))) return s;
        m.cta_ptr = mt;
        if ((s = P->upload(P->m2l.cta_tiles, &mt))) return s;
        m.cta_tiles = mt;
    }
    {
        const M2LWindows &wt = P->m2lw;
        DevM2LPc &pc = P->dpc;
        pc.ncta = wt.win_targets.empty() ? 0 : wt.ncta;
#define UPW(vec, field)                                   \
    if ((s = P->upload(wt.vec, &mt))) return s;           \
    pc.field = mt;
        UPW(cta_ptr, cta_ptr);
        UPW(cta_win, cta_win);
        UPW(win_target_ptr, win_target_ptr);
        UPW(win_targets, win_targets);
        UPW(win_item_ptr, win_item_ptr);
        UPW(item_offset, item_offset);
        UPW(item_pair_ptr, item_pair_ptr);
        UPW(pair_src, pair_src);
        UPW(pair_slot, pair_slot);
#undef UPW
    }

    // operators (FP32, transposed for coalesced row access)
    const int ns = o.ns, rP = o.rP, rQ = o.rQ, k = o.k, kp = P->kpad;
    DevOps &op = P->dops;
    op.ns = ns;
    op.rP = rP;
    op.rQ = rQ;
    op.k = k;
    op.kpad = kp;
    op.ai = (float)o.ai;
    op.ao = (float)o.ao;
    std::vector<float4> surf(ns);
    for (int j = 0; j < ns; ++j)
        surf[j] = make_float4((float)o.surf[3 * j], (float)o.surf[3 * j + 1],
                              (float)o.surf[3 * j + 2], 0.f);
    float4 *ds;
    if ((s = P->upload(surf, &ds))) return s;
    op.surf = ds;
    float *f;
#define UPF(vec, field)                                   \
    if ((s = P->upload(vec, &f))) return s;               \
    op.field = f;
    // AT (n x m row-major, FP64) -> FP32 with rows padded to round4(m)
    auto padded = [](const std::vector<double> &at, int n, int m) {
        const int mp = (m + 3) & ~3;
        std::vector<float> out((size_t)n * mp, 0.f);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < m; ++i) out[(size_t)j * mp + i] = (float)at[(size_t)j * m + i];
        return out;
    };
    auto append = [](std::vector<float> &dst, const std::vector<float> &src) {
        dst.insert(dst.end(), src.begin(), src.end());
    };
    UPF(padded(o.Pu, ns, rP), Pu);                       // AT of Pu^T
    {
        std::vector<float> inv(rP);
        for (int i = 0; i < rP; ++i) inv[i] = (float)(1.0 / o.Ps[i]);
        UPF(inv, Ps_inv);
    }
    UPF(padded(transpose(o.Pv, ns, rP), rP, ns), PvT);   // AT of Pv
    {
        std::vector<float> mm;
        for (int sg = 0; sg < 8; ++sg) {
            std::vector<double> m1(o.M2M.begin() + (size_t)sg * rP * ns,
                                   o.M2M.begin() + (size_t)(sg + 1) * rP * ns);
            append(mm, padded(transpose(m1, rP, ns), ns, rP));
        }
        UPF(mm, M2M);
    }
    {
        std::vector<double> vk((size_t)ns * kp, 0.0);        // AT of Vk^T, zero padded
        for (int j = 0; j < ns; ++j)
            for (int i = 0; i < k; ++i) vk[(size_t)j * kp + i] = o.Vk[(size_t)j * k + i];
        UPF(padded(vk, ns, kp), Vk);
    }
    {
        std::vector<double> q((size_t)kp * rQ, 0.0);         // AT of Qu^T Uk
        for (int i = 0; i < rQ; ++i)
            for (int j = 0; j < k; ++j) q[(size_t)j * rQ + i] = o.QUk[(size_t)i * k + j];
        UPF(padded(q, kp, rQ), QUkT);
    }
    UPF(padded(o.Qu, ns, rQ), Qu);                       // AT of Qu^T
    {
        // AT of [L2L_0; ...; L2L_7] with row (sigma, i) divided by Qs[i]:
        // ns x 8 rQ, so one product gives all eight children's contributions
        // already scaled for the downward pseudo-inverse
        std::vector<double> at((size_t)ns * 8 * rQ);
        for (int sg = 0; sg < 8; ++sg)
            for (int i = 0; i < rQ; ++i)
                for (int j = 0; j < ns; ++j)
                    at[(size_t)j * 8 * rQ + (size_t)sg * rQ + i] =
                        o.L2L[(size_t)sg * rQ * ns + (size_t)i * ns + j] / o.Qs[i];
        UPF(padded(at, ns, 8 * rQ), L2L);
    }
    {
        std::vector<float> inv(rQ);
        for (int i = 0; i < rQ; ++i) inv[i] = (float)(1.0 / o.Qs[i]);
        UPF(inv, Qs_inv);
    }
    UPF(padded(transpose(o.Qv, ns, rQ), rQ, ns), QvT);   // AT of Qv
    {
        std::vector<float> st((size_t)kNumOffsets * kp * kp, 0.f);
        for (int tt = 0; tt < kNumOffsets; ++tt)
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j)
                    st[(size_t)tt * kp * kp + (size_t)j * kp + i] =
                        (float)o.S[(size_t)tt * k * k + (size_t)i * k + j];
        UPF(st, St);
    }
#undef UPF
    if (P->timing)
        for (auto &e : P->ev) CK(cudaEventCreate(&e));
    for (auto &e : P->tune_ev) CK(cudaEventCreate(&e));
    CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));
    CK(cudaStreamCreateWithFlags(&P->s_side, cudaStreamNonBlocking));
    for (auto &e : P->ev_side) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaHostAlloc((void **)&P->err_host, sizeof(int), cudaHostAllocMapped));
    *P->err_host = 0;
    CK(cudaHostGetDevicePointer((void **)&P->err_dev, P->err_host, 0));
    if (P->opts.m2l_mode != FMM_M2L_FP32) {
        fmm_status s2 = prepare_tc(P, P->opts.m2l_mode);
        if (s2 != FMM_OK) return s2;
    }
    return FMM_OK;
}

fmm_status ensure_workspace(fmm_plan_s *P, int nrhs) {
    if (nrhs <= P->nrhs_cap) return FMM_OK;
    P->free_workspace();
    WorkspaceBytes wb;
    kifmm::plan_workspace_bytes(P, nrhs, &wb);
    auto alloc = [&](float **p, size_t bytes) -> cudaError_t {
        return cudaMalloc((void **)p, bytes ? bytes : 16);
    };
    CK(alloc(&P->qs, wb.qs));
    CK(alloc(&P->up, wb.up));
    CK(alloc(&P->down, wb.down));
    CK(alloc(&P->qhat, wb.qhat));
    CK(alloc(&P->chat, wb.chat));
    CK(alloc(&P->xchk, wb.xchk));
    CK(alloc(&P->chk, wb.chk));
    CK(alloc(&P->ybuf, wb.ybuf));
    CK(alloc(&P->yp, wb.yp));
    if (wb.part) CK(alloc(&P->part, wb.part));
    P->nrhs_cap = nrhs;
    return FMM_OK;
}

// Split-operand copies of qhat for the tensor-core M2L (4-byte slots, so the
// same buffers serve BF16 and TF32).
fmm_status ensure_split(fmm_plan_s *P, int nrhs) {
    if (P->opts.m2l_mode == FMM_M2L_FP32 || nrhs <= P->qh_cap) return FMM_OK;
    if (P->qh_hi) cudaFree(P->qh_hi);
    if (P->qh_lo) cudaFree(P->qh_lo);
    P->qh_hi = P->qh_lo = nullptr;
    P->qh_cap = 0;
    ++P->ws_gen;
    const size_t bytes = ((size_t)P->tree.nodes() * nrhs + 1) * P->kpad * 4;
    CK(cudaMalloc((void **)&P->qh_hi, bytes));
    CK(cudaMalloc((void **)&P->qh_lo, bytes));
    P->qh_cap = nrhs;
    return FMM_OK;
}

fmm_status enqueue(fmm_plan_s *P, const float *charges, int nrhs, double *pot, double *grad,
                   cudaStream_t st) {
    WorkBuffers b;
    b.qs = P->qs;
    b.up = P->up;
    b.down = P->down;
    b.qhat = P->qhat;
    b.chat = P->chat;
    b.xchk = P->xchk;
    b.chk = P->chk;
    b.ybuf = P->ybuf;
    b.yp = P->yp;
    b.part = P->part;
    b.qh_hi = P->qh_hi;
    b.qh_lo = P->qh_lo;
    return kifmm::plan_enqueue(P, charges, nrhs, pot, grad, b, st);
}

// One evaluation on `st`: replay the plan's graph when its key holds,
// otherwise capture the enqueue into a new graph and launch it.  The legacy
// default stream cannot be captured; there (and with the graph option off)
// the kernels are launched directly.
fmm_status run_evaluation(fmm_plan_s *P, const float *charges, int nrhs, double *pot,
                          double *grad, cudaStream_t st) {
    if (P->autotune && P->forced_shape < 0) {
        auto it = P->tuned_shapes.find(nrhs);
        if (it == P->tuned_shapes.end()) {
            // this evaluation tunes the level products (direct launches,
            // timed one by one) and is itself the result
            P->tuning = true;
            P->knob[0] = 1;
            P->knob[1] = 0;
            fmm_status s = enqueue(P, charges, nrhs, pot, grad, st);
            P->tuning = false;
            if (s != FMM_OK) return s;
            P->tuned_shapes[nrhs] = P->gemm_shape;
            P->tuned_knobs[nrhs] = {P->knob[0], P->knob[1]};
            return FMM_OK;
        }
        P->gemm_shape = it->second;
        const auto kn = P->tuned_knobs.find(nrhs);
        P->knob[0] = kn != P->tuned_knobs.end() ? kn->second[0] : 1;
        P->knob[1] = kn != P->tuned_knobs.end() ? kn->second[1] : 0;
    } else if (!P->autotune) {
        P->gemm_shape.clear();  // the default shape everywhere
        P->knob[0] = 1;
        P->knob[1] = 0;
    }
    if (P->forced_knobs >= 0) {
        P->knob[0] = P->forced_knobs & 1;
        P->knob[1] = (P->forced_knobs >> 1) & 1;
    }
    const bool legacy = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
    if (!P->use_graph || legacy) return enqueue(P, charges, nrhs, pot, grad, st);
    const int mode = P->opts.m2l_mode;
    ++P->graph_clock;
    for (fmm_plan_s::GraphEntry &g : P->graphs)
        if (g.exec && g.charges == charges && g.pot == pot && g.grad == grad && g.nrhs == nrhs &&
            g.mode == mode && g.kernel == P->m2l_kernel && g.ws_gen == P->ws_gen) {
            g.used = P->graph_clock;
            CK(cudaGraphLaunch(g.exec, st));
            return FMM_OK;
        }
    // a free entry, else the least recently used one
    fmm_plan_s::GraphEntry *slot = &P->graphs[0];
    for (fmm_plan_s::GraphEntry &g : P->graphs) {
        if (!g.exec) {
            slot = &g;
            break;
        }
        if (g.used < slot->used) slot = &g;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = fmm_plan_s::GraphEntry();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int64_t before = P->last_launches;
    fmm_status s = enqueue(P, charges, nrhs, pot, grad, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != FMM_OK) {
        if (g) cudaGraphDestroy(g);
        P->last_launches = before;
        return s;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(FMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return fail(FMM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    slot->exec = exec;
    slot->charges = charges;
    slot->pot = pot;
    slot->grad = grad;
    slot->nrhs = nrhs;
    slot->mode = mode;
    slot->kernel = P->m2l_kernel;
    slot->ws_gen = P->ws_gen;
    slot->used = P->graph_clock;
    CK(cudaGraphLaunch(exec, st));
    return FMM_OK;
}

} // namespace

namespace {
// Phase timing events: an external event record node when `st` is being
// captured into a graph, a plain record otherwise.
cudaError_t record_phase(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
               : cudaEventRecord(ev, st);
}
} // namespace

// Enqueue every kernel of one evaluation on `st`, using the given
// per-evaluation buffers (sized for nrhs, see plan_workspace_bytes).
// Autotuning of a two-way choice that changes no result: runs each
// alternative twice on `st` and times the second run; *best receives the
// faster one (ties keep *best).
template <class F>
static cudaError_t time_choice(fmm_plan_s *P, cudaStream_t st, F &&run, int *best) {
    float ms[2] = {0.f, 0.f};
    for (int c = 0; c < 2; ++c)
        for (int rep = 0; rep < 2; ++rep) {
            cudaError_t e;
            if ((e = cudaEventRecord(P->tune_ev[0], st)) != cudaSuccess) return e;
            if ((e = run(c)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(P->tune_ev[1], st)) != cudaSuccess) return e;
            if ((e = cudaEventSynchronize(P->tune_ev[1])) != cudaSuccess) return e;
            if ((e = cudaEventElapsedTime(&ms[c], P->tune_ev[0], P->tune_ev[1])) != cudaSuccess)
                return e;
        }
    if (ms[0] < ms[1]) *best = 0;
    else if (ms[1] < ms[0]) *best = 1;
    return cudaSuccess;
}

fmm_status kifmm::plan_enqueue(fmm_plan_s *P, const float *charges, int nrhs, double *pot,
                               double *grad, const WorkBuffers &b, cudaStream_t st) {
    const Tree &t = P->tree;
    const Schedules &sc = P->sched;
    DevWork w{};
    w.nrhs = nrhs;
    w.charges_user = charges;
    w.qs = b.qs;
    w.up = b.up;
    w.down = b.down;
    w.qhat = b.qhat;
    w.chat = b.chat;
    w.xchk = b.xchk;
    w.pot_user = pot;
    w.grad_user = grad;
    if (!b.chk || !b.ybuf || !b.yp)
        return fail(FMM_ERR_INVALID_ARG, "workspace is incomplete");
    int64_t launches = 0;
    if (P->timing) CK(record_phase(P->ev[0], st));
    CK(launch_gather_charges(P->dt, w, st));
    ++launches;
    const DevOps &o = P->dops;
    const int ns = o.ns, rP = o.rP, rQ = o.rQ, kp = o.kpad;
    // row strides of the per-box arrays, all 16-byte aligned
    const int nsp = (ns + 3) & ~3, rPp = (rP + 3) & ~3, rQp = (rQ + 3) & ~3;
    int site = 0;
    if (P->tuning) {
        P->gemm_shape.clear();
        P->gemm_ms.clear();
    }
    auto gemm = [&](VGemm &g, cudaStream_t gs) -> fmm_status {
        g.nrhs = nrhs;
        const int my = site++;
        if (g.count > 0) {
            ++launches;
            if (g.part && vgemm_split_floats(g.m, g.count, nrhs, g.nseg) > 0) ++launches;
        }
        if (P->tuning) {
            // time every shape (second of two runs each); no product reads
            // its own output, so the reruns are idempotent and every shape
            // writes the same bits
            int best = 0;
            float best_ms = 0.f;
            for (int sh = 0; sh < kGemmShapes && g.count > 0; ++sh) {
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {
                    CK(cudaEventRecord(P->tune_ev[0], gs));
                    CK(launch_vgemm(g, gs, sh));
                    CK(cudaEventRecord(P->tune_ev[1], gs));
                    CK(cudaEventSynchronize(P->tune_ev[1]));
                    CK(cudaEventElapsedTime(&ms, P->tune_ev[0], P->tune_ev[1]));
                }
                if (sh == 0 || ms < best_ms) {
                    best = sh;
                    best_ms = ms;
                }
            }
            P->gemm_shape.push_back(best);
            P->gemm_ms.push_back(best_ms);
            CK(launch_vgemm(g, gs, best));
            return FMM_OK;
        }
        const int shape = P->forced_shape >= 0 ? P->forced_shape
                          : my < (int)P->gemm_shape.size() ? P->gemm_shape[my] : 0;
        CK(launch_vgemm(g, gs, shape));
        return FMM_OK;
    };
    auto seg = [](const float *AT, int n, const float *src, int src_ld, const int *idx, int base) {
        VSeg s{};
        s.AT = AT;
        s.n = n;
        s.src = src;
        s.src_ld = src_ld;
        s.src_idx = idx;
        s.src_base = base;
        return s;
    };
    // side stream for the projections (not while tuning: timed one by one)
    const bool side = P->s_side && !P->tuning;
    bool side_used = false;
    // rho = Pv y (y already divided by Ps), written to up[node]; then the
    // M2L projection qhat[node] = Vk^T rho
    auto finish_up = [&](const int *nodes, int count) -> fmm_status {
        VGemm g{};
        g.m = ns;
        g.count = count;
        g.nseg = 1;
        g.seg[0] = seg(o.PvT, rP, b.ybuf, rPp, nullptr, 0);
        g.dst = b.up;
        g.dst_ld = nsp;
        g.dst_idx = nodes;
        if (fmm_status e = gemm(g, st)) return e;
        VGemm h{};
        h.m = kp;
        h.count = count;
        h.nseg = 1;
        h.seg[0] = seg(o.Vk, ns, b.up, nsp, nodes, 0);
        h.dst = b.qhat;
        h.dst_ld = kp;
        h.dst_idx = nodes;
        if (!side) return gemm(h, st);
        // reads this level's rho, writes its qhat rows: nothing the rest of
        // the upward pass touches
        CK(cudaEventRecord(P->ev_side[0], st));
        CK(cudaStreamWaitEvent(P->s_side, P->ev_side[0], 0));
        side_used = true;
        return gemm(h, P->s_side);
    };
    if (t.depth >= 2) {
        // P2M: check potentials, y = Pu^T chk / Ps, rho, qhat
        const int np = (int)sc.p2m_nodes.size();
        if (np > 0) {
            ++launches;
            CK(launch_p2m_check(P->dt, o, w, P->d_p2m, np, b.chk, nsp, st));
            VGemm g{};
            g.m = rP;
            g.count = np;
            g.nseg = 1;
            g.seg[0] = seg(o.Pu, ns, b.chk, nsp, nullptr, 0);
            g.scale = o.Ps_inv;
            g.dst = b.ybuf;
            g.dst_ld = rPp;
            if (fmm_status e = gemm(g, st)) return e;
            if (fmm_status e = finish_up(P->d_p2m, np)) return e;
        }
        // M2M, bottom-up: y = sum_sigma M2M_sigma up[child_sigma] / Ps
        const int total = (int)sc.m2m_nodes.size();
        const int mp = (rP + 3) & ~3;
        for (int l = t.depth - 1; l >= 2; --l) {
            const int a0 = sc.m2m_level_ptr[l], cnt = sc.m2m_level_ptr[l + 1] - a0;
            if (cnt == 0) continue;
            VGemm g{};
            g.m = rP;
            g.count = cnt;
            g.nseg = 8;
            for (int sg = 0; sg < 8; ++sg)
                g.seg[sg] = seg(o.M2M + (size_t)sg * ns * mp, ns, b.up, nsp,
                                P->d_m2m_child + (size_t)sg * total + a0, 0);
            g.scale = o.Ps_inv;
            g.dst = b.ybuf;
            g.dst_ld = rPp;
            g.part = b.part;
            if (fmm_status e = gemm(g, st)) return e;
            if (fmm_status e = finish_up(P->d_m2m + a0, cnt)) return e;
        }
    }
    if (side_used) {
        CK(cudaEventRecord(P->ev_side[1], P->s_side));
        CK(cudaStreamWaitEvent(st, P->ev_side[1], 0));
    }
    if (P->timing) CK(record_phase(P->ev[1], st));
    if (t.depth >= 2 && P->dm.ntiles > 0) {
        const int mode = P->opts.m2l_mode;
        if (mode == FMM_M2L_FP32) {
            CK(launch_m2l_simt(P->dm, P->dops, w, st));
            ++launches;
        } else {
            const int idx = mode == FMM_M2L_TF32X3 ? 1 : 0;
            if (!P->tc_ready[idx] || !b.qh_hi || !b.qh_lo)
                return fail(FMM_ERR_INVALID_ARG, "tensor-core M2L buffers are not prepared");
            if (m2l_uses_pair_columns(P))
                CK(launch_m2l_pc(P->dpc, P->dops, w, (int)t.nodes(), idx == 1, P->tmap[idx][0],
                                 P->tmap[idx][1], b.qh_hi, b.qh_lo, P->err_dev,
                                 P->test_m2l_stall != 0, st));
            else {
                auto m2l = [&](int sched) {
                    DevM2L dm = P->dm;
                    if (!sched) dm.ncta = 0;  // round robin over the tiles
                    return launch_m2l_tc(dm, P->dops, w, (int)t.nodes(), idx == 1,
                                         P->tmap[idx][0], P->tmap[idx][1], b.qh_hi, b.qh_lo,
                                         P->err_dev, P->test_m2l_stall != 0, P->num_sms, st);
                };
                if (P->tuning && P->forced_knobs < 0 && !P->test_m2l_stall && P->dm.ncta > 0) {
                    // both schedules give the same bits: keep the faster
                    int best = 1;
                    CK(time_choice(P, st, m2l, &best));
                    P->knob[0] = best;
                }
                CK(m2l(P->knob[0]));
            }
            launches += 2;
        }
    }
    if (P->timing) CK(record_phase(P->ev[2], st));
    if (t.depth >= 2) {
        if (!sc.x_nodes.empty())  // one launch per charge-column group of 8, 4, 2, 1
            launches += nrhs / 8 + ((nrhs % 8) >> 2) + ((nrhs % 4) >> 1) + (nrhs % 2);
        CK(launch_p2l(P->dt, o, w, P->d_xnodes, (int)sc.x_nodes.size(), st));
        const int total = (int)sc.m2m_nodes.size();
        (void)total;
        for (int l = 2; l <= t.depth; ++l) {
            const int b0 = t.level_ptr[l], cnt = t.level_ptr[l + 1] - b0;
            if (cnt == 0) continue;
            // L2L: all eight children's (scaled) check potentials from the
            // parents' downward densities, one product over the parent level
            if (l >= 3) {
                const int a0 = sc.m2m_level_ptr[l - 1], pc = sc.m2m_level_ptr[l] - a0;
                VGemm g{};
                g.m = 8 * rQ;
                g.count = pc;
                g.nseg = 1;
                g.seg[0] = seg(o.L2L, ns, b.down, nsp, P->d_m2m + a0, 0);
                g.dst = b.yp;
                g.dst_ld = 8 * rQ;
                if (fmm_status e = gemm(g, st)) return e;
            }
            // y = ((Qu^T Uk) chat + Qu^T xchk) / Qs + L2L part
            VGemm g{};
            g.m = rQ;
            g.count = cnt;
            g.nseg = 1;
            g.seg[0] = seg(o.QUkT, kp, b.chat, kp, P->d_chat_src + b0, 0);
            if (sc.x_level_count[l] > 0) {  // boxes of this level with a P2L slot
                g.seg[1] = seg(o.Qu, ns, b.xchk, nsp, P->dt.x_slot + b0, 0);
                g.nseg = 2;
                g.sparse = 1u << 1;  // a few boxes of the level have a slot
            }
            g.scale = o.Qs_inv;
            if (l >= 3) {
                g.add = b.yp;
                g.add_ld = 8 * rQ;
                g.add_idx = P->d_ppos + b0;
                g.add_off = P->d_poff + b0;
            }
            g.dst = b.ybuf;
            g.dst_ld = rQp;
            if (fmm_status e = gemm(g, st)) return e;
            // rho = Qv y -> down[node]
            VGemm h{};
            h.m = ns;
            h.count = cnt;
            h.nseg = 1;
            h.seg[0] = seg(o.QvT, rQ, b.ybuf, rQp, nullptr, 0);
            h.dst = b.down;
            h.dst_ld = nsp;
            h.dst_base = b0;
            if (fmm_status e = gemm(h, st)) return e;
        }
    }
    if (P->timing) CK(record_phase(P->ev[3], st));
    {
        int leaf_launches = 0;
        auto leafpass = [&](int narrow_first) {
            leaf_launches = 0;
            return launch_eval(P->dt, P->dops, w, st, &leaf_launches, narrow_first != 0);
        };
        if (P->tuning && P->forced_knobs < 0) {
            // both orders give the same bits: keep the faster
            int best = 0;
            CK(time_choice(P, st, leafpass, &best));
            P->knob[1] = best;
        }
        CK(leafpass(P->knob[1]));
        launches += leaf_launches;
    }
    if (P->timing) CK(record_phase(P->ev[4], st));
    P->last_launches = launches;
    return FMM_OK;
}

// Bytes of each per-evaluation buffer of plan P for nrhs right-hand sides.
void kifmm::plan_workspace_bytes(const fmm_plan_s *P, int nrhs, WorkspaceBytes *out) {
    const Tree &t = P->tree;
    const size_t nn = (size_t)t.nodes(), ns = (P->ops->ns + 3) & ~3, kp = P->kpad;
    const size_t nx = P->sched.x_nodes.size();
    out->qs = (size_t)t.n * nrhs * sizeof(float);
    out->up = out->down = nn * nrhs * ns * sizeof(float);
    out->qhat = out->chat = nn * nrhs * kp * sizeof(float);
    out->xchk = nx * nrhs * ns * sizeof(float);
    out->qh = P->opts.m2l_mode == FMM_M2L_FP32 ? 0 : (nn * nrhs + 1) * kp * 4;
    const size_t rmax = (size_t)((std::max(P->ops->rP, P->ops->rQ) + 3) & ~3);
    out->chk = P->sched.p2m_nodes.size() * nrhs * ns * sizeof(float);
    out->ybuf = (size_t)P->max_level_nodes * nrhs * rmax * sizeof(float);
    out->yp = (size_t)P->max_level_internal * nrhs * 8 * P->ops->rQ * sizeof(float);
    // split-K scratch of the M2M level products (levels depth-1 .. 2)
    size_t part = 0;
    for (int l = t.depth - 1; l >= 2; --l) {
        const int cnt = P->sched.m2m_level_ptr[l + 1] - P->sched.m2m_level_ptr[l];
        if (cnt > 0) part = std::max(part, vgemm_split_floats(P->ops->rP, cnt, nrhs, 8));
    }
    out->part = part * sizeof(float);
}

int kifmm::plan_device(const fmm_plan_s *P) { return P->device; }
int kifmm::plan_m2l_mode(const fmm_plan_s *P) { return P->opts.m2l_mode; }

// A bounded device-side wait that expired sets the plan's mapped error word;
// it is reported once, by the next call that looks, and then cleared.
fmm_status kifmm::plan_check_device_error(fmm_plan_s *P) {
    if (!P->err_host) return FMM_OK;
    const int e = *(volatile int *)P->err_host;
    if (e == 0) return FMM_OK;
    *(volatile int *)P->err_host = 0;
    return fail(FMM_ERR_TIMEOUT, "a bounded wait in the tensor-core M2L expired (roles mask " +
                                     std::to_string(e) + "); results of that evaluation are invalid");
}
fmm_status kifmm::plan_set_error(fmm_status s, const std::string &msg) { return fail(s, msg); }
bool kifmm::plan_host_only(const fmm_plan_s *P) { return P->opts.host_only != 0; }

namespace {

// Host copy of n x 3 positions (device pointers are copied down).
fmm_status host_points(const double *src, int64_t n, bool may_be_device,
                       std::vector<double> &buf, const double **out) {
    *out = src;
    if (may_be_device && is_device_pointer(src)) {
        buf.resize((size_t)3 * n);
        CK(cudaMemcpy(buf.data(), src, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
        *out = buf.data();
    }
    return FMM_OK;
}

// Problems of at least this many points build their tree on the device
// under FMM_TREE_AUTO.
constexpr int64_t kDeviceTreeMin = 65536;

// Tree, lists and point roles of one problem (optional distinct targets:
// the tree is built on their union).  FMM_TREE_DEVICE takes host or device
// positions, the host builders host positions.
void build_problem(const double *xs, const double *xt, int64_t n, const TreeOptions &to,
                   int how, Tree &t) {
    if (how == FMM_TREE_DEVICE || how == FMM_TREE_LEVELS_HOST) {
        build_tree_levels(xs, xt, n, to, how == FMM_TREE_DEVICE, t);
    } else if (xt) {
        std::vector<double> all((size_t)6 * n);
        std::copy(xs, xs + 3 * n, all.begin());
        std::copy(xt, xt + 3 * n, all.begin() + 3 * n);
        build_tree(all.data(), 2 * n, to, t);
        build_lists(t);
    } else {
        build_tree(xs, n, to, t);
        build_lists(t);
    }
    set_point_roles(t, n, xt != nullptr);
}

// Host fault-injection hook for the table check's tests (environment
// variable FMM_TEST_CORRUPT_TABLE=<table>): one out-of-range value is put
// into the named table before the check runs, so a test can see the check
// refuse the plan before anything reaches the device.  Unset in normal use.
void corrupt_table_for_test(fmm_plan_s *P, const std::string &name) {
    Tree &t = P->tree;
    const int32_t nn = (int32_t)t.nodes();
    if (name == "u_idx" && !t.u_idx.empty()) t.u_idx[t.u_idx.size() / 2] = nn;
    else if (name == "v_ptr" && t.v_ptr.size() > 2) t.v_ptr[1] = t.v_ptr.back() + 1;
    else if (name == "entry_src" && !P->m2l.entry_src.empty()) P->m2l.entry_src.back() = nn;
    else if (name == "tile_target" && !P->m2l.tile_target.empty()) P->m2l.tile_target[0] = -2;
    else if (name == "qidx" && !t.qidx.empty()) t.qidx[0] = P->rows;
    else if (name == "down_chunk" && !P->sched.down_chunk.empty()) P->sched.down_chunk[1] = 1 << 30;
    else if (name == "begin" && !t.begin.empty()) t.begin[0] = t.n + 1;
    else if (name == "child" && !t.child.empty()) t.child[0] = nn + 7;
}

fmm_status create_plan(const double *const *sources, const double *const *targets,
                       const int64_t *n, int nproblems, int p, int ncrit,
                       const fmm_options *opts, fmm_plan_t *out) {
    if (!out) return fail(FMM_ERR_INVALID_ARG, "out is NULL");
    if (!sources || !n) return fail(FMM_ERR_INVALID_ARG, "sources or n is NULL");
    if (nproblems < 1 || nproblems > 65536)
        return fail(FMM_ERR_INVALID_ARG, "nproblems must be in [1, 65536]");
    int64_t rows = 0, points = 0;
    for (int i = 0; i < nproblems; ++i) {
        if (!sources[i]) return fail(FMM_ERR_INVALID_ARG, "sources is NULL");
        if (n[i] < 1) return fail(FMM_ERR_INVALID_ARG, "n must be >= 1");
        const bool distinct = targets && targets[i] && targets[i] != sources[i];
        rows += n[i];
        points += distinct ? 2 * n[i] : n[i];
        if (points > INT32_MAX / 2)
            return fail(FMM_ERR_UNSUPPORTED, "too many points for 32-bit ranges");
    }
    if (p < 2 || p > 10) return fail(FMM_ERR_INVALID_ARG, "p must be in [2, 10]");
    if (ncrit < 1) return fail(FMM_ERR_INVALID_ARG, "ncrit must be >= 1");
    fmm_options o;
    fmm_options_init(&o);
    if (opts) o = *opts;
    if (!(o.alpha_inner > 1.0) || !(o.alpha_outer > o.alpha_inner) || !(o.alpha_outer < 3.0))
        return fail(FMM_ERR_INVALID_ARG, "need 1 < alpha_inner < alpha_outer < 3");
    if (!(o.rcond > 0.0 && o.rcond < 1.0)) return fail(FMM_ERR_INVALID_ARG, "rcond in (0,1)");
    if (!(o.eps_svd >= 0.0 && o.eps_svd < 1.0))
        return fail(FMM_ERR_INVALID_ARG, "eps_svd in [0,1)");
    if (o.max_level < 0 || o.max_level > kKeyBits)
        return fail(FMM_ERR_INVALID_ARG, "max_level in [0,16]");
    if (o.m2l_mode != FMM_M2L_FP32 && o.m2l_mode != FMM_M2L_BF16X3 &&
        o.m2l_mode != FMM_M2L_TF32X3)
        return fail(FMM_ERR_INVALID_ARG, "unknown M2L mode");
    if (o.tree_build < FMM_TREE_AUTO || o.tree_build > FMM_TREE_LEVELS_HOST)
        return fail(FMM_ERR_INVALID_ARG, "unknown tree_build");
    if (o.direct_wx != 0 && o.direct_wx != 1)
        return fail(FMM_ERR_INVALID_ARG, "direct_wx is 0 or 1");
    if (o.tree_build == FMM_TREE_DEVICE && o.host_only)
        return fail(FMM_ERR_INVALID_ARG, "FMM_TREE_DEVICE needs a device (host_only is set)");
    fmm_plan_s *P = nullptr;
    kifmm::DeviceGuard dg_;  // the caller's device is current again on return
    try {
        P = new fmm_plan_s();
        P->opts = o;
        P->p = p;
        P->ncrit = ncrit;
        P->rows = rows;
        const char *tm = std::getenv("FMM_TIMING");
        P->timing = tm && tm[0] == '1' && !o.host_only;
        if (!o.host_only) {
            int dev = o.device;
            if (dev < 0) {
                cudaError_t e = cudaGetDevice(&dev);
                if (e != cudaSuccess) {
                    delete P;
                    return fail(FMM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
                }
            }
            P->device = dev;
            cudaError_t e = dg_.set(dev);
            if (e != cudaSuccess) {
                delete P;
                return fail(FMM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
            }
        }
        TreeOptions to;
        to.ncrit = ncrit;
        to.max_level = o.max_level;
        to.balance = o.balance != 0;
        // builder of every problem; host views of the points of those built
        // on the host (device arrays copied down)
        std::vector<int> how(nproblems);
        std::vector<std::vector<double>> buf(2 * (size_t)nproblems);
        std::vector<const double *> xs(nproblems), xt(nproblems, nullptr);
        for (int i = 0; i < nproblems; ++i) {
            const bool distinct = targets && targets[i] && targets[i] != sources[i];
            const int64_t pts = distinct ? 2 * n[i] : n[i];
            how[i] = o.tree_build == FMM_TREE_AUTO
                         ? (!o.host_only && pts >= kDeviceTreeMin ? FMM_TREE_DEVICE : FMM_TREE_HOST)
                         : o.tree_build;
            fmm_status e = FMM_OK;
            if (how[i] == FMM_TREE_DEVICE) {
                xs[i] = sources[i];
                xt[i] = distinct ? targets[i] : nullptr;
                P->device_trees++;
                continue;
            }
            e = host_points(sources[i], n[i], !o.host_only, buf[2 * i], &xs[i]);
            if (e == FMM_OK && distinct)
                e = host_points(targets[i], n[i], !o.host_only, buf[2 * i + 1], &xt[i]);
            if (e != FMM_OK) {
                delete P;
                return e;
            }
        }
        if (nproblems == 1) {
            build_problem(xs[0], xt[0], n[0], to, how[0], P->tree);
        } else {
            std::vector<Tree> parts(nproblems);
            std::vector<int64_t> row_off(nproblems, 0);
            for (int i = 1; i < nproblems; ++i) row_off[i] = row_off[i - 1] + n[i - 1];
            std::vector<std::string> msg(nproblems);
            // device builds one after another, then the host builds in parallel
            for (int i = 0; i < nproblems; ++i)
                if (how[i] == FMM_TREE_DEVICE) build_problem(xs[i], xt[i], n[i], to, how[i], parts[i]);
            bool bad = false;
#pragma omp parallel for schedule(dynamic, 1) reduction(|| : bad)
            for (int i = 0; i < nproblems; ++i) {
                if (how[i] == FMM_TREE_DEVICE) continue;
                try {
                    build_problem(xs[i], xt[i], n[i], to, how[i], parts[i]);
                } catch (const std::exception &ex) {
                    msg[i] = std::string("problem ") + std::to_string(i) + ": " + ex.what();
                    bad = true;
                }
            }
            if (bad)
                for (int i = 0; i < nproblems; ++i)
                    if (!msg[i].empty()) throw std::runtime_error(msg[i]);
            merge_forest(parts, row_off, P->tree);
        }
        build_m2l_table(P->tree, P->m2l);
        {
            // one persistent block per SM of the plan's device
            int nsm = 152;
            if (!o.host_only &&
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device) !=
                    cudaSuccess) {
                cudaGetLastError();
                nsm = 152;
            }
            build_m2l_windows(P->tree, nsm, P->m2lw);
            build_m2l_schedule(nsm, P->m2l);
        }
        // points on a check or equivalent surface: 6 (p - 1)^2 + 2
        const int nsurf = 6 * (p - 1) * (p - 1) + 2;
        build_schedules(P->tree, kDownChunk, o.direct_wx ? nsurf : -1, P->sched);
        if (const char *hook = std::getenv("FMM_TEST_CORRUPT_TABLE"))
            corrupt_table_for_test(P, hook);
        std::string bad = check_tables(P->tree, P->sched, P->m2l, P->rows);
        if (bad.empty()) bad = check_windows(P->tree, P->m2lw);
        if (!bad.empty()) {
            delete P;
            return fail(FMM_ERR_UNSUPPORTED, "plan tables failed their check: " + bad);
        }
        P->ops = get_operators(p, o.alpha_inner, o.alpha_outer, o.rcond, o.eps_svd,
                               &P->ops_source);
        P->kpad = (P->ops->k + 15) / 16 * 16;
        if (!o.host_only) {
            fmm_status s = upload_plan(P);
            if (s != FMM_OK) {
                delete P;
                return s;
            }
        }
    } catch (const std::bad_alloc &) {
        delete P;
        return fail(FMM_ERR_OOM, "host allocation failed");
    } catch (const CudaFailure &ex) {
        delete P;
        return fail(ex.code == (int)cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA,
                    std::string("device tree build: ") + ex.what());
    } catch (const std::exception &ex) {
        delete P;
        return fail(FMM_ERR_INVALID_ARG, ex.what());
    }
    *out = P;
    return FMM_OK;
}

// fmm_evaluate / fmm_evaluate_gradient: host buffers are staged through
// plan-owned device memory; potentials may be NULL when gradients are asked.
fmm_status evaluate_impl(fmm_plan_s *P, const float *charges, int nrhs, double *potentials,
                         double *gradients, void *stream) {
    if (!P) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (P->opts.host_only) return fail(FMM_ERR_INVALID_ARG, "host-only plan cannot evaluate");
    if (!charges) return fail(FMM_ERR_INVALID_ARG, "NULL charges or potentials");
    if (nrhs < 1) return fail(FMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    kifmm::DeviceGuard dg_;
    CK(dg_.set(P->device));
    if (fmm_status e = kifmm::plan_check_device_error(P)) return e;
    const bool dq = is_device_pointer(charges);
    const bool dp = !potentials || is_device_pointer(potentials);
    const bool dg = !gradients || is_device_pointer(gradients);
    fmm_status s = ensure_workspace(P, nrhs);
    if (s != FMM_OK) return s;
    s = ensure_split(P, nrhs);
    if (s != FMM_OK) return s;
    const size_t nq = (size_t)P->rows * nrhs;
    const float *dq_ptr = charges;
    double *dp_ptr = potentials, *dg_ptr = gradients;
    if (!dq) {
        if (!P->charges_stage) CK(cudaMalloc((void **)&P->charges_stage, (size_t)P->rows * P->nrhs_cap * sizeof(float)));
        CK(cudaMemcpyAsync(P->charges_stage, charges, nq * sizeof(float), cudaMemcpyHostToDevice, st));
        dq_ptr = P->charges_stage;
    }
    if (!dp) {
        if (!P->pot_stage) CK(cudaMalloc((void **)&P->pot_stage, (size_t)P->rows * P->nrhs_cap * sizeof(double)));
        dp_ptr = P->pot_stage;
    }
    if (!dg) {
        if (!P->grad_stage) CK(cudaMalloc((void **)&P->grad_stage, (size_t)P->rows * P->nrhs_cap * 3 * sizeof(double)));
        dg_ptr = P->grad_stage;
    }
    s = run_evaluation(P, dq_ptr, nrhs, dp_ptr, dg_ptr, st);
    if (s != FMM_OK) return s;
    P->last_stream = st;
    P->last_nrhs = nrhs;
    if (!dp) CK(cudaMemcpyAsync(potentials, dp_ptr, nq * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!dg) CK(cudaMemcpyAsync(gradients, dg_ptr, 3 * nq * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!dq || !dp || !dg) {
        CK(cudaStreamSynchronize(st));
        return kifmm::plan_check_device_error(P);
    }
    return FMM_OK;
}

} // namespace

extern "C" {

void fmm_options_init(fmm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->alpha_inner = 1.05;
    o->alpha_outer = 2.95;
    o->rcond = 1e-7;
    o->eps_svd = 1e-7;
    o->max_level = kKeyBits;
    o->balance = 1;
    o->m2l_mode = FMM_M2L_FP32;
    o->host_only = 0;
    o->device = -1;
    o->tree_build = FMM_TREE_AUTO;
    o->direct_wx = 1;
}

fmm_status fmm_plan_create(const double *sources, const double *targets, int64_t n, int p,
                           int ncrit, fmm_plan_t *out) {
    return create_plan(&sources, &targets, &n, 1, p, ncrit, nullptr, out);
}

fmm_status fmm_plan_create_ex(const double *sources, const double *targets, int64_t n, int p,
                              int ncrit, const fmm_options *opts, fmm_plan_t *out) {
    return create_plan(&sources, &targets, &n, 1, p, ncrit, opts, out);
}

fmm_status fmm_plan_create_batch(const double *const *sources, const double *const *targets,
                                 const int64_t *n, int nproblems, int p, int ncrit,
                                 fmm_plan_t *out) {
    return create_plan(sources, targets, n, nproblems, p, ncrit, nullptr, out);
}

fmm_status fmm_plan_create_batch_ex(const double *const *sources,
                                    const double *const *targets, const int64_t *n,
                                    int nproblems, int p, int ncrit, const fmm_options *opts,
                                    fmm_plan_t *out) {
    return create_plan(sources, targets, n, nproblems, p, ncrit, opts, out);
}

fmm_status fmm_plan_set_option(fmm_plan_t plan, int key, double value) {
    if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (key == FMM_OPT_M2L_MODE) {
        const int mode = (int)value;
        if (mode != FMM_M2L_FP32 && mode != FMM_M2L_BF16X3 && mode != FMM_M2L_TF32X3)
            return fail(FMM_ERR_INVALID_ARG, "unknown M2L mode");
        if (mode != FMM_M2L_FP32 && !plan->opts.host_only) {
            kifmm::DeviceGuard dg_;
            CK(dg_.set(plan->device));
            fmm_status s = prepare_tc(plan, mode);
            if (s != FMM_OK) return s;
        }
        plan->opts.m2l_mode = mode;
        return FMM_OK;
    }
    if (key == FMM_OPT_AUTOTUNE) {
        plan->autotune = value != 0.0;
        plan->tuned_shapes.clear();
        plan->tuned_knobs.clear();
        plan->drop_graph();
        return FMM_OK;
    }
    if (key == FMM_OPT_GEMM_SHAPE) {
        const int sh = (int)value;
        if (sh < -1 || sh >= kGemmShapes) return fail(FMM_ERR_INVALID_ARG, "shape in [-1, 4]");
        plan->forced_shape = sh;
        plan->drop_graph();
        return FMM_OK;
    }
    if (key == FMM_OPT_FORCE_KNOBS) {
        const int v = (int)value;
        if ((double)v != value || v < -1 || v > 3)
            return fail(FMM_ERR_INVALID_ARG, "value -1 or 0..3");
        plan->forced_knobs = v;
        plan->drop_graph();
        return FMM_OK;
    }
    if (key == FMM_OPT_M2L_KERNEL) {
        if (value != 0.0 && value != 1.0) return fail(FMM_ERR_INVALID_ARG, "value 0 or 1");
        plan->m2l_kernel = (int)value;
        plan->drop_graph();
        return FMM_OK;
    }
    if (key == FMM_OPT_TEST_M2L_STALL) {
        if (value != 0.0 && value != 1.0) return fail(FMM_ERR_INVALID_ARG, "value 0 or 1");
        plan->test_m2l_stall = (int)value;
        plan->drop_graph();
        return FMM_OK;
    }
    if (key == FMM_OPT_GRAPH) {
        plan->use_graph = value != 0.0;
        if (!plan->use_graph) plan->drop_graph();
        return FMM_OK;
    }
    return fail(FMM_ERR_INVALID_ARG, "unknown option key");
}

fmm_status fmm_evaluate(fmm_plan_t P, const float *charges, int nrhs, double *potentials,
                        void *stream) {
    if (!potentials) return fail(FMM_ERR_INVALID_ARG, "NULL charges or potentials");
    return evaluate_impl(P, charges, nrhs, potentials, nullptr, stream);
}

fmm_status fmm_evaluate_gradient(fmm_plan_t P, const float *charges, int nrhs,
                                 double *potentials, double *gradients, void *stream) {
    if (!gradients) return fail(FMM_ERR_INVALID_ARG, "NULL gradients");
    return evaluate_impl(P, charges, nrhs, potentials, gradients, stream);
}

void fmm_destroy(fmm_plan_t plan) { delete plan; }

fmm_status fmm_set_operator_cache(const char *dir) {
    if (!set_operator_cache_dir(dir))
        return fail(FMM_ERR_INVALID_ARG, std::string("not an existing directory: ") + dir);
    return FMM_OK;
}

const char *fmm_last_error(void) { return g_error.c_str(); }

fmm_status fmm_plan_info(fmm_plan_t P, int key, int64_t *value) {
    if (!P || !value) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    const Tree &t = P->tree;
    switch (key) {
    case FMM_INFO_N: *value = P->rows; break;
    case FMM_INFO_POINTS: *value = t.n; break;
    case FMM_INFO_PROBLEMS: *value = t.nproblems; break;
    case FMM_INFO_DEVICE_TREES: *value = P->device_trees; break;
    case FMM_INFO_OPERATOR_SOURCE: *value = P->ops_source; break;
    case FMM_INFO_NODES: *value = t.nodes(); break;
    case FMM_INFO_LEAVES: *value = (int64_t)t.leaves.size(); break;
    case FMM_INFO_DEPTH: *value = t.depth; break;
    case FMM_INFO_NSURF: *value = P->ops->ns; break;
    case FMM_INFO_RANK_M2L: *value = P->ops->k; break;
    case FMM_INFO_RANK_UP: *value = P->ops->rP; break;
    case FMM_INFO_RANK_DOWN: *value = P->ops->rQ; break;
    case FMM_INFO_U_PAIRS: *value = (int64_t)t.u_idx.size(); break;
    case FMM_INFO_V_PAIRS: *value = (int64_t)t.v_idx.size(); break;
    case FMM_INFO_W_PAIRS: *value = (int64_t)t.w_idx.size(); break;
    case FMM_INFO_X_PAIRS: *value = (int64_t)t.x_idx.size(); break;
    case FMM_INFO_P2P_PAIRS: *value = t.p2p_pairs; break;
    case FMM_INFO_SURF_PAIRS:
    case FMM_INFO_WX_DIRECT_PAIRS: {
        // the leaf pass's L2P (own downward surface, levels >= 2) and M2P
        // (W boxes' upward surfaces) pairs, and its direct W / X pairs,
        // counted like the near field
        int64_t surf = 0, direct = 0;
        for (int64_t b : t.leaves) {
            const int64_t nb = t.end[b] - t.begin[b];
            int64_t nsurf = t.key[4 * b] >= 2 ? 1 : 0;
            for (int64_t e = t.w_ptr[b]; e < t.w_ptr[b + 1]; ++e) {
                const int64_t a = t.w_idx[e];
                if (P->sched.w_direct[a]) direct += nb * (t.end[a] - t.begin[a]);
                else ++nsurf;
            }
            if (P->sched.x_slot[b] < 0)
                for (int64_t e = t.x_ptr[b]; e < t.x_ptr[b + 1]; ++e) {
                    const int64_t a = t.x_idx[e];
                    direct += nb * (t.end[a] - t.begin[a]);
                }
            surf += nb * nsurf;
        }
        *value = key == FMM_INFO_SURF_PAIRS ? surf * P->ops->ns : direct;
        break;
    }
    case FMM_INFO_M2L_TILES: *value = (int64_t)P->m2l.tile_level.size(); break;
    case FMM_INFO_M2L_ENTRIES: *value = (int64_t)P->m2l.entry_offset.size(); break;
    case FMM_INFO_LAST_LAUNCHES: *value = P->last_launches; break;
    case FMM_INFO_TUNINGS: *value = (int64_t)P->tuned_shapes.size(); break;
    case FMM_INFO_M2L_WINDOWS: *value = (int64_t)P->m2lw.win_item_ptr.size() - 1; break;
    case FMM_INFO_M2L_ITEMS: *value = (int64_t)P->m2lw.item_offset.size(); break;
    case FMM_INFO_M2L_KERNEL:
        *value = P->opts.m2l_mode == FMM_M2L_FP32 ? 0 : (m2l_uses_pair_columns(P) ? 2 : 1);
        break;
    default: return fail(FMM_ERR_INVALID_ARG, "unknown info key");
    }
    return FMM_OK;
}

fmm_status fmm_plan_get_array(fmm_plan_t P, int which, void *dst, int64_t bytes,
                              int64_t *needed) {
    if (!P) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    const Tree &t = P->tree;
    const Operators &o = *P->ops;
    const void *src = nullptr;
    size_t size = 0;
    std::vector<int64_t> range;
    std::vector<int32_t> leaf32, shapes;
    switch (which) {
    case FMM_ARRAY_NODE_KEYS: src = t.key.data(); size = t.key.size() * 4; break;
    case FMM_ARRAY_NODE_RANGE:
        range.resize(2 * t.nodes());
        for (int64_t b = 0; b < t.nodes(); ++b) {
            range[2 * b] = t.begin[b];
            range[2 * b + 1] = t.end[b];
        }
        src = range.data();
        size = range.size() * 8;
        break;
    case FMM_ARRAY_LEAF_FLAG:
        leaf32.assign(t.leaf.begin(), t.leaf.end());
        src = leaf32.data();
        size = leaf32.size() * 4;
        break;
    case FMM_ARRAY_PERM: src = t.perm.data(); size = t.perm.size() * 8; break;
    case FMM_ARRAY_U_PTR: src = t.u_ptr.data(); size = t.u_ptr.size() * 8; break;
    case FMM_ARRAY_U_IDX: src = t.u_idx.data(); size = t.u_idx.size() * 4; break;
    case FMM_ARRAY_V_PTR: src = t.v_ptr.data(); size = t.v_ptr.size() * 8; break;
    case FMM_ARRAY_V_IDX: src = t.v_idx.data(); size = t.v_idx.size() * 4; break;
    case FMM_ARRAY_W_PTR: src = t.w_ptr.data(); size = t.w_ptr.size() * 8; break;
    case FMM_ARRAY_W_IDX: src = t.w_idx.data(); size = t.w_idx.size() * 4; break;
    case FMM_ARRAY_X_PTR: src = t.x_ptr.data(); size = t.x_ptr.size() * 8; break;
    case FMM_ARRAY_X_IDX: src = t.x_idx.data(); size = t.x_idx.size() * 4; break;
    case FMM_ARRAY_SURFACE: src = o.surf.data(); size = o.surf.size() * 8; break;
    case FMM_ARRAY_M2L_U: src = o.Uk.data(); size = o.Uk.size() * 8; break;
    case FMM_ARRAY_M2L_V: src = o.Vk.data(); size = o.Vk.size() * 8; break;
    case FMM_ARRAY_M2L_S: src = o.S.data(); size = o.S.size() * 8; break;
    case FMM_ARRAY_ROOT: src = t.roots.data(); size = t.roots.size() * 8; break;
    case FMM_ARRAY_CHARGE_ROW: src = t.qidx.data(); size = t.qidx.size() * 8; break;
    case FMM_ARRAY_OUTPUT_ROW: src = t.oidx.data(); size = t.oidx.size() * 8; break;
    case FMM_ARRAY_GEMM_SHAPES:
        shapes.assign(P->gemm_shape.begin(), P->gemm_shape.end());
        src = shapes.data();
        size = shapes.size() * 4;
        break;
    case FMM_ARRAY_NODE_PROBLEM:
        src = t.node_problem.data();
        size = t.node_problem.size() * 4;
        break;
    case FMM_ARRAY_OP_PU: src = o.Pu.data(); size = o.Pu.size() * 8; break;
    case FMM_ARRAY_OP_PS: src = o.Ps.data(); size = o.Ps.size() * 8; break;
    case FMM_ARRAY_OP_PV: src = o.Pv.data(); size = o.Pv.size() * 8; break;
    case FMM_ARRAY_OP_QU: src = o.Qu.data(); size = o.Qu.size() * 8; break;
    case FMM_ARRAY_OP_QS: src = o.Qs.data(); size = o.Qs.size() * 8; break;
    case FMM_ARRAY_OP_QV: src = o.Qv.data(); size = o.Qv.size() * 8; break;
    case FMM_ARRAY_OP_M2M: src = o.M2M.data(); size = o.M2M.size() * 8; break;
    case FMM_ARRAY_OP_L2L: src = o.L2L.data(); size = o.L2L.size() * 8; break;
    case FMM_ARRAY_OP_QUK: src = o.QUk.data(); size = o.QUk.size() * 8; break;
    case FMM_ARRAY_M2L_TILE_LEVEL:
        src = P->m2l.tile_level.data();
        size = P->m2l.tile_level.size() * 4;
        break;
    case FMM_ARRAY_M2L_TILE_TARGET:
        src = P->m2l.tile_target.data();
        size = P->m2l.tile_target.size() * 4;
        break;
    case FMM_ARRAY_M2L_TILE_ENTRY_PTR:
        src = P->m2l.tile_entry_ptr.data();
        size = P->m2l.tile_entry_ptr.size() * 4;
        break;
    case FMM_ARRAY_M2L_ENTRY_OFFSET:
        src = P->m2l.entry_offset.data();
        size = P->m2l.entry_offset.size() * 4;
        break;
    case FMM_ARRAY_M2L_ENTRY_SRC:
        src = P->m2l.entry_src.data();
        size = P->m2l.entry_src.size() * 4;
        break;
#define WARR(id, vec)                       \
    case id:                                \
        src = P->m2lw.vec.data();           \
        size = P->m2lw.vec.size() * 4;      \
        break;
    WARR(FMM_ARRAY_M2L_WIN_TARGET_PTR, win_target_ptr)
    WARR(FMM_ARRAY_M2L_WIN_TARGETS, win_targets)
    WARR(FMM_ARRAY_M2L_WIN_ITEM_PTR, win_item_ptr)
    WARR(FMM_ARRAY_M2L_ITEM_OFFSET, item_offset)
    WARR(FMM_ARRAY_M2L_ITEM_PAIR_PTR, item_pair_ptr)
    WARR(FMM_ARRAY_M2L_PAIR_SRC, pair_src)
    WARR(FMM_ARRAY_M2L_PAIR_SLOT, pair_slot)
    WARR(FMM_ARRAY_M2L_CTA_PTR, cta_ptr)
    WARR(FMM_ARRAY_M2L_CTA_WIN, cta_win)
#undef WARR
    case FMM_ARRAY_M2L_TILE_CTA_PTR:
        src = P->m2l.cta_ptr.data();
        size = P->m2l.cta_ptr.size() * 4;
        break;
    case FMM_ARRAY_M2L_TILE_CTA_TILES:
        src = P->m2l.cta_tiles.data();
        size = P->m2l.cta_tiles.size() * 4;
        break;
    case FMM_ARRAY_TUNED_KNOBS:
        src = P->knob;
        size = sizeof(P->knob);
        break;
    default: return fail(FMM_ERR_INVALID_ARG, "unknown array");
    }
    if (needed) *needed = (int64_t)size;
    if (!dst) return FMM_OK;
    if (bytes < (int64_t)size) return fail(FMM_ERR_INVALID_ARG, "destination too small");
    if (size) std::memcpy(dst, src, size);
    return FMM_OK;
}

fmm_status fmm_plan_get_workspace(fmm_plan_t P, int which, void *dst, int64_t bytes,
                                  int64_t *needed) {
    if (!P) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (P->opts.host_only || P->last_nrhs < 1)
        return fail(FMM_ERR_INVALID_ARG, "no evaluation on this plan yet");
    const size_t nn = (size_t)P->tree.nodes(), nr = (size_t)P->last_nrhs;
    const size_t nsp = (size_t)((P->ops->ns + 3) & ~3), kp = (size_t)P->kpad;
    const float *src = nullptr;
    size_t ld = 0;
    switch (which) {
    case FMM_WORK_UP: src = P->up; ld = nsp; break;
    case FMM_WORK_DOWN: src = P->down; ld = nsp; break;
    case FMM_WORK_QHAT: src = P->qhat; ld = kp; break;
    case FMM_WORK_CHAT: src = P->chat; ld = kp; break;
    default: return fail(FMM_ERR_INVALID_ARG, "unknown workspace array");
    }
    const size_t size = nn * nr * ld * sizeof(float);
    if (needed) *needed = (int64_t)size;
    if (!dst) return FMM_OK;
    if (bytes < (int64_t)size) return fail(FMM_ERR_INVALID_ARG, "destination too small");
    if (!src) return fail(FMM_ERR_INVALID_ARG, "no workspace");
    kifmm::DeviceGuard dg_;
    CK(dg_.set(P->device));
    CK(cudaStreamSynchronize(P->last_stream));
    if (size) CK(cudaMemcpy(dst, src, size, cudaMemcpyDeviceToHost));
    return FMM_OK;
}

fmm_status fmm_plan_phase_ms(fmm_plan_t P, int phase, double *ms) {
    if (!P || !ms) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    if (!P->timing) return fail(FMM_ERR_INVALID_ARG, "timing is off (set FMM_TIMING=1)");
    if (phase < 0 || phase > 3) return fail(FMM_ERR_INVALID_ARG, "phase in [0,3]");
    CK(cudaEventSynchronize(P->ev[4]));
    float v = 0;
    CK(cudaEventElapsedTime(&v, P->ev[phase], P->ev[phase + 1]));
    *ms = v;
    return FMM_OK;
}

} // extern "C"
