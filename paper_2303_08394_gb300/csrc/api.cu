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
    Tree tree;
    M2LTable m2l;
    Schedules sched;
    std::shared_ptr<const Operators> ops;
    int kpad = 0;
    bool timing = false;
    std::vector<void *> allocs;   // plan-lifetime device memory
    DevTree dt{};
    DevOps dops{};
    DevM2L dm{};
    int *d_p2m = nullptr, *d_m2m = nullptr, *d_down = nullptr, *d_chunks = nullptr,
        *d_xnodes = nullptr;
    // workspace, sized for nrhs_cap right-hand sides
    int nrhs_cap = 0;
    float *qs = nullptr, *up = nullptr, *down = nullptr, *qhat = nullptr, *chat = nullptr,
          *xchk = nullptr, *charges_stage = nullptr;
    double *pot_stage = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t last_stream = nullptr;
    int64_t last_launches = 0;

    ~fmm_plan_s() {
        if (opts.host_only) return;
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        for (void *a : allocs) cudaFree(a);
        free_workspace();
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        cudaSetDevice(prev);
    }
    void free_workspace() {
        void *w[] = {qs, up, down, qhat, chat, xchk, charges_stage, pot_stage};
        for (void *a : w)
            if (a) cudaFree(a);
        qs = up = down = qhat = chat = xchk = charges_stage = nullptr;
        pot_stage = nullptr;
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

fmm_status upload_plan(fmm_plan_s *P) {
    const Tree &t = P->tree;
    const Operators &o = *P->ops;
    const int64_t nn = t.nodes();
    // points and nodes
    std::vector<float4> pts(t.n);
    for (int64_t i = 0; i < t.n; ++i)
        pts[i] = make_float4(t.rel[4 * i], t.rel[4 * i + 1], t.rel[4 * i + 2], 0.f);
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
    int64_t *dperm;
    if ((s = P->upload(t.perm, &dperm))) return s;
    d.perm = dperm;
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
    UP32(t.leaves, leaves);
    UP32(to32(t.u_ptr), u_ptr);
    UP32(t.u_idx, u_idx);
    UP32(to32(t.w_ptr), w_ptr);
    UP32(t.w_idx, w_idx);
    UP32(to32(t.x_ptr), x_ptr);
    UP32(t.x_idx, x_idx);
    UP32(to32(t.v_ptr), v_ptr);
    UP32(P->sched.x_slot, x_slot);
#undef UP32
    if ((s = P->upload(P->sched.p2m_nodes, &P->d_p2m))) return s;
    if ((s = P->upload(P->sched.m2m_nodes, &P->d_m2m))) return s;
    if ((s = P->upload(P->sched.down_nodes, &P->d_down))) return s;
    if ((s = P->upload(P->sched.down_chunk, &P->d_chunks))) return s;
    if ((s = P->upload(P->sched.x_nodes, &P->d_xnodes))) return s;

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
    UPF(to_f32(o.Pu), Pu);
    {
        std::vector<float> inv(rP);
        for (int i = 0; i < rP; ++i) inv[i] = (float)(1.0 / o.Ps[i]);
        UPF(inv, Ps_inv);
    }
    UPF(to_f32(transpose(o.Pv, ns, rP)), PvT);
    {
        std::vector<float> mm((size_t)8 * ns * rP);
        for (int sg = 0; sg < 8; ++sg)
            for (int i = 0; i < rP; ++i)
                for (int j = 0; j < ns; ++j)
                    mm[(size_t)sg * ns * rP + (size_t)j * rP + i] =
                        (float)o.M2M[(size_t)sg * rP * ns + (size_t)i * ns + j];
        UPF(mm, M2M);
    }
    {
        std::vector<float> vk((size_t)ns * kp, 0.f);
        for (int j = 0; j < ns; ++j)
            for (int i = 0; i < k; ++i) vk[(size_t)j * kp + i] = (float)o.Vk[(size_t)j * k + i];
        UPF(vk, Vk);
    }
    {
        std::vector<float> q((size_t)kp * rQ, 0.f);
        for (int i = 0; i < rQ; ++i)
            for (int j = 0; j < k; ++j) q[(size_t)j * rQ + i] = (float)o.QUk[(size_t)i * k + j];
        UPF(q, QUkT);
    }
    UPF(to_f32(o.Qu), Qu);
    {
        std::vector<float> ll((size_t)8 * ns * rQ);
        for (int sg = 0; sg < 8; ++sg)
            for (int i = 0; i < rQ; ++i)
                for (int j = 0; j < ns; ++j)
                    ll[(size_t)sg * ns * rQ + (size_t)j * rQ + i] =
                        (float)o.L2L[(size_t)sg * rQ * ns + (size_t)i * ns + j];
        UPF(ll, L2L);
    }
    {
        std::vector<float> inv(rQ);
        for (int i = 0; i < rQ; ++i) inv[i] = (float)(1.0 / o.Qs[i]);
        UPF(inv, Qs_inv);
    }
    UPF(to_f32(transpose(o.Qv, ns, rQ)), QvT);
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
    return FMM_OK;
}

fmm_status ensure_workspace(fmm_plan_s *P, int nrhs) {
    if (nrhs <= P->nrhs_cap) return FMM_OK;
    P->free_workspace();
    const Tree &t = P->tree;
    const size_t nn = (size_t)t.nodes(), ns = P->ops->ns, kp = P->kpad;
    const size_t nx = P->sched.x_nodes.size();
    auto alloc = [&](void **p, size_t bytes) -> cudaError_t {
        return cudaMalloc(p, bytes ? bytes : 16);
    };
    CK(alloc((void **)&P->qs, (size_t)t.n * nrhs * sizeof(float)));
    CK(alloc((void **)&P->up, nn * nrhs * ns * sizeof(float)));
    CK(alloc((void **)&P->down, nn * nrhs * ns * sizeof(float)));
    CK(alloc((void **)&P->qhat, nn * nrhs * kp * sizeof(float)));
    CK(alloc((void **)&P->chat, nn * nrhs * kp * sizeof(float)));
    CK(alloc((void **)&P->xchk, nx * nrhs * ns * sizeof(float)));
    P->nrhs_cap = nrhs;
    return FMM_OK;
}

fmm_status enqueue(fmm_plan_s *P, const float *charges, int nrhs, double *pot,
                   cudaStream_t st) {
    WorkBuffers b;
    b.qs = P->qs;
    b.up = P->up;
    b.down = P->down;
    b.qhat = P->qhat;
    b.chat = P->chat;
    b.xchk = P->xchk;
    return kifmm::plan_enqueue(P, charges, nrhs, pot, b, st);
}

} // namespace

// Enqueue every kernel of one evaluation on `st`, using the given
// per-evaluation buffers (sized for nrhs, see plan_workspace_bytes).
fmm_status kifmm::plan_enqueue(fmm_plan_s *P, const float *charges, int nrhs, double *pot,
                               const WorkBuffers &b, cudaStream_t st) {
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
    w.scale = 1.0 / (4.0 * M_PI * t.hw);
    int64_t launches = 0;
    if (P->timing) CK(cudaEventRecord(P->ev[0], st));
    CK(launch_gather_charges(P->dt, w, st));
    ++launches;
    if (t.depth >= 2) {
        if (!sc.p2m_nodes.empty()) ++launches;
        CK(launch_p2m(P->dt, P->dops, w, P->d_p2m, (int)sc.p2m_nodes.size(), st));
        for (int l = t.depth - 1; l >= 2; --l) {
            int a = sc.m2m_level_ptr[l], b = sc.m2m_level_ptr[l + 1];
            if (b > a) ++launches;
            CK(launch_m2m(P->dt, P->dops, w, P->d_m2m + a, b - a, st));
        }
    }
    if (P->timing) CK(cudaEventRecord(P->ev[1], st));
    if (t.depth >= 2 && P->dm.ntiles > 0) {
        CK(launch_m2l_simt(P->dm, P->dops, w, st));
        ++launches;
    }
    if (P->timing) CK(cudaEventRecord(P->ev[2], st));
    if (t.depth >= 2) {
        if (!sc.x_nodes.empty()) ++launches;
        CK(launch_p2l(P->dt, P->dops, w, P->d_xnodes, (int)sc.x_nodes.size(), st));
        for (int l = 2; l <= t.depth; ++l) {
            int a = sc.down_chunk_level_ptr[l], b = sc.down_chunk_level_ptr[l + 1];
            if (b > a) ++launches;
            CK(launch_down(P->dt, P->dops, w, P->d_chunks + 4 * a, P->d_down, b - a, st));
        }
    }
    if (P->timing) CK(cudaEventRecord(P->ev[3], st));
    CK(launch_eval(P->dt, P->dops, w, st));
    launches += nrhs / 8 + ((nrhs % 8) >> 2) + ((nrhs % 4) >> 1) + (nrhs % 2);
    if (P->timing) CK(cudaEventRecord(P->ev[4], st));
    P->last_launches = launches;
    return FMM_OK;
}

// Bytes of each per-evaluation buffer of plan P for nrhs right-hand sides.
void kifmm::plan_workspace_bytes(const fmm_plan_s *P, int nrhs, WorkspaceBytes *out) {
    const Tree &t = P->tree;
    const size_t nn = (size_t)t.nodes(), ns = P->ops->ns, kp = P->kpad;
    const size_t nx = P->sched.x_nodes.size();
    out->qs = (size_t)t.n * nrhs * sizeof(float);
    out->up = out->down = nn * nrhs * ns * sizeof(float);
    out->qhat = out->chat = nn * nrhs * kp * sizeof(float);
    out->xchk = nx * nrhs * ns * sizeof(float);
}

int kifmm::plan_device(const fmm_plan_s *P) { return P->device; }
fmm_status kifmm::plan_set_error(fmm_status s, const std::string &msg) { return fail(s, msg); }
bool kifmm::plan_host_only(const fmm_plan_s *P) { return P->opts.host_only != 0; }

namespace {

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
}

fmm_status fmm_plan_create(const double *sources, const double *targets, int64_t n, int p,
                           int ncrit, fmm_plan_t *out) {
    return fmm_plan_create_ex(sources, targets, n, p, ncrit, nullptr, out);
}

fmm_status fmm_plan_create_ex(const double *sources, const double *targets, int64_t n, int p,
                              int ncrit, const fmm_options *opts, fmm_plan_t *out) {
    if (!out) return fail(FMM_ERR_INVALID_ARG, "out is NULL");
    if (!sources) return fail(FMM_ERR_INVALID_ARG, "sources is NULL");
    if (targets && targets != sources)
        return fail(FMM_ERR_UNSUPPORTED, "targets distinct from sources are not supported");
    if (n < 1) return fail(FMM_ERR_INVALID_ARG, "n must be >= 1");
    if (n > INT32_MAX / 2) return fail(FMM_ERR_UNSUPPORTED, "n too large for 32-bit ranges");
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
    if (o.m2l_mode != FMM_M2L_FP32)
        return fail(FMM_ERR_UNSUPPORTED, "only the FP32 M2L is built in this library version");
    fmm_plan_s *P = nullptr;
    try {
        P = new fmm_plan_s();
        P->opts = o;
        P->p = p;
        P->ncrit = ncrit;
        const char *tm = std::getenv("FMM_TIMING");
        P->timing = tm && tm[0] == '1' && !o.host_only;
        std::vector<double> host;
        const double *xyz = sources;
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
            cudaError_t e = cudaSetDevice(dev);
            if (e != cudaSuccess) {
                delete P;
                return fail(FMM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
            }
            if (is_device_pointer(sources)) {
                host.resize((size_t)3 * n);
                e = cudaMemcpy(host.data(), sources, host.size() * sizeof(double),
                               cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    delete P;
                    return fail(FMM_ERR_CUDA, std::string("copy sources: ") + cudaGetErrorString(e));
                }
                xyz = host.data();
            }
        }
        TreeOptions to;
        to.ncrit = ncrit;
        to.max_level = o.max_level;
        to.balance = o.balance != 0;
        build_tree(xyz, n, to, P->tree);
        build_lists(P->tree);
        build_m2l_table(P->tree, P->m2l);
        build_schedules(P->tree, kDownChunk, P->sched);
        P->ops = get_operators(p, o.alpha_inner, o.alpha_outer, o.rcond, o.eps_svd);
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
    } catch (const std::exception &ex) {
        delete P;
        return fail(FMM_ERR_INVALID_ARG, ex.what());
    }
    *out = P;
    return FMM_OK;
}

fmm_status fmm_plan_set_option(fmm_plan_t plan, int key, double value) {
    if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (key == FMM_OPT_M2L_MODE) {
        int mode = (int)value;
        if (mode == FMM_M2L_FP32) {
            plan->opts.m2l_mode = mode;
            return FMM_OK;
        }
        if (mode == FMM_M2L_BF16X3 || mode == FMM_M2L_TF32X3)
            return fail(FMM_ERR_UNSUPPORTED, "tensor-core M2L is not built in this version");
        return fail(FMM_ERR_INVALID_ARG, "unknown M2L mode");
    }
    return fail(FMM_ERR_INVALID_ARG, "unknown option key");
}

fmm_status fmm_evaluate(fmm_plan_t P, const float *charges, int nrhs, double *potentials,
                        void *stream) {
    if (!P) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (P->opts.host_only) return fail(FMM_ERR_INVALID_ARG, "host-only plan cannot evaluate");
    if (!charges || !potentials) return fail(FMM_ERR_INVALID_ARG, "NULL charges or potentials");
    if (nrhs < 1) return fail(FMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(P->device));
    const bool dq = is_device_pointer(charges), dp = is_device_pointer(potentials);
    fmm_status s = ensure_workspace(P, nrhs);
    if (s != FMM_OK) return s;
    const size_t nq = (size_t)P->tree.n * nrhs;
    const float *dq_ptr = charges;
    double *dp_ptr = potentials;
    if (!dq) {
        if (!P->charges_stage) CK(cudaMalloc((void **)&P->charges_stage, (size_t)P->tree.n * P->nrhs_cap * sizeof(float)));
        CK(cudaMemcpyAsync(P->charges_stage, charges, nq * sizeof(float), cudaMemcpyHostToDevice, st));
        dq_ptr = P->charges_stage;
    }
    if (!dp) {
        if (!P->pot_stage) CK(cudaMalloc((void **)&P->pot_stage, (size_t)P->tree.n * P->nrhs_cap * sizeof(double)));
        dp_ptr = P->pot_stage;
    }
    s = enqueue(P, dq_ptr, nrhs, dp_ptr, st);
    if (s != FMM_OK) return s;
    P->last_stream = st;
    if (!dp) CK(cudaMemcpyAsync(potentials, dp_ptr, nq * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!dq || !dp) CK(cudaStreamSynchronize(st));
    return FMM_OK;
}

void fmm_destroy(fmm_plan_t plan) { delete plan; }

const char *fmm_last_error(void) { return g_error.c_str(); }

fmm_status fmm_plan_info(fmm_plan_t P, int key, int64_t *value) {
    if (!P || !value) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    const Tree &t = P->tree;
    switch (key) {
    case FMM_INFO_N: *value = t.n; break;
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
    case FMM_INFO_M2L_TILES: *value = (int64_t)P->m2l.tile_level.size(); break;
    case FMM_INFO_M2L_ENTRIES: *value = (int64_t)P->m2l.entry_offset.size(); break;
    case FMM_INFO_LAST_LAUNCHES: *value = P->last_launches; break;
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
    std::vector<int32_t> leaf32;
    std::vector<double> root;
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
    case FMM_ARRAY_ROOT:
        root = {t.centre[0], t.centre[1], t.centre[2], t.hw};
        src = root.data();
        size = 32;
        break;
    default: return fail(FMM_ERR_INVALID_ARG, "unknown array");
    }
    if (needed) *needed = (int64_t)size;
    if (!dst) return FMM_OK;
    if (bytes < (int64_t)size) return fail(FMM_ERR_INVALID_ARG, "destination too small");
    if (size) std::memcpy(dst, src, size);
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
