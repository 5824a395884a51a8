// Internal host-side structures of a KIFMM plan.
#pragma once
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "constants.h"
#include "kifmm.h"

namespace kifmm {

// Offset t = (tx, ty, tz) -> index 0..315 (lexicographic, tz fastest),
// or -1 for |t|_inf <= 1 or out of range.
int offset_index(int tx, int ty, int tz);

// FP64 operators for the unit box (half-width 1, centre 0) and the kernel
// 1/r.  All of them are level independent: the Laplace kernel is homogeneous
// of degree -1, so a box of half-width h has K_h = K / h and its
// pseudo-inverse h K^+, which cancel in every composite below.
struct Operators {
    int p = 0, ns = 0;                 // order, surface points 6(p-1)^2+2
    double ai = 0, ao = 0, rcond = 0, eps_svd = 0;
    std::vector<double> surf;          // ns x 3 unit surface
    // Upward check-to-equivalent matrix K(ao s, ai s) = Pu diag(Ps) Pv^T,
    // truncated to the rP singular values above rcond * sigma_max.
    int rP = 0;
    std::vector<double> Pu, Ps, Pv;    // ns x rP, rP, ns x rP
    // Downward check-to-equivalent matrix K(ai s, ao s) = Qu diag(Qs) Qv^T.
    int rQ = 0;
    std::vector<double> Qu, Qs, Qv;    // ns x rQ, rQ, ns x rQ
    // M2M: parent upward check potential of child sigma's density, already
    // projected on Pu: 8 x (rP x ns) = Pu^T K(ao s, c_sigma + ai/2 s).
    std::vector<double> M2M;
    // L2L: child downward check potential from the parent's downward
    // density, in child-normalised units and projected on Qu:
    // 8 x (rQ x ns) = Qu^T (1/2) K(c_sigma + ai/2 s, ao s).
    std::vector<double> L2L;
    // M2L: K_t = K(ai s, 2t + ai s), t in the 316 offsets, compressed as
    // K_t ~ Uk S_t Vk^T with Uk, Vk from the SVDs of [K_1 ... K_316] and
    // [K_1; ...; K_316].  eps_svd == 0 keeps K_t dense (Uk = Vk = I).
    int k = 0;
    std::vector<double> Uk, Vk;        // ns x k
    std::vector<double> S;             // 316 x k x k
    std::vector<double> QUk;           // rQ x k = Qu^T Uk
    std::vector<double> sigmaH, sigmaW;// singular values of the stacks
};

// Operators for (p, radii, cutoffs): from this process's memory, else from
// the file cache directory when one is set, else computed (and then written
// there).  *source (may be NULL) receives which.
enum { kOpsComputed = 0, kOpsFromMemory = 1, kOpsFromFile = 2 };
std::shared_ptr<const Operators> get_operators(int p, double ai, double ao,
                                               double rcond, double eps_svd,
                                               int *source = nullptr);
// Directory of the operator file cache; NULL or "" turns it off.  False if
// `dir` is not an existing directory.
bool set_operator_cache_dir(const char *dir);

// Octree over the (sorted) points plus interaction lists and schedules.
struct Tree {
    int64_t n = 0;
    double centre[3] = {0, 0, 0}, hw = 0;   // root cube
    int depth = 0;
    std::vector<int64_t> perm;              // sorted position -> caller index
    std::vector<float> rel_lo;              // n x 4: rounding residual of rel
                                            // (rel + rel_lo is the FP64 value
                                            // to about 2^-48 of the leaf size)
    std::vector<float> rel;                 // n x 4: position relative to its
                                            // leaf centre, root units, w = 0
    // nodes that hold points, ordered by level then Morton key
    std::vector<int32_t> key;               // nodes x 4 (level, ix, iy, iz)
    std::vector<int64_t> begin, end;        // sorted point range
    std::vector<int32_t> parent;            // -1 for the root
    std::vector<int32_t> child;             // nodes x 8, -1 if absent
    std::vector<uint8_t> leaf;
    std::vector<int32_t> level_ptr;         // depth + 2 entries
    std::vector<int32_t> leaves;            // node indices of leaves
    // interaction lists, CSR over all nodes (sorted by node index)
    std::vector<int64_t> u_ptr, v_ptr, w_ptr, x_ptr;
    std::vector<int32_t> u_idx, v_idx, w_idx, x_idx;
    std::vector<int16_t> v_off;             // offset index of each V entry
    int64_t p2p_pairs = 0;
    // caller rows of each sorted point: charge row (-1: a target only) and
    // output row (-1: a source only)
    std::vector<int64_t> qidx, oidx;
    // independent problems sharing the tree arrays (a forest): root cube of
    // each (centre x, y, z, half-width) and the problem of every node
    int nproblems = 1;
    std::vector<double> roots;
    std::vector<int32_t> node_problem;

    int64_t nodes() const { return (int64_t)parent.size(); }
    double node_centre(int64_t node, int d) const;   // root units
    double node_half_width(int64_t node) const;      // root units
};

struct TreeOptions {
    int ncrit = 64;
    int max_level = kKeyBits;
    bool balance = true;
};

// Build the tree (throws std::runtime_error on bad input).
void build_tree(const double *xyz, int64_t n, const TreeOptions &opt,
                Tree &tree);
// Root cube from the coordinate bounds: centred on the bounding box, the
// half-width of its largest extent inflated by a relative 1e-6 (0.5 when
// every point coincides).
void root_cube(const double lo[3], const double hi[3], double centre[3], double &hw);

// A CUDA call failed while building a plan on the device.
struct CudaFailure : std::runtime_error {
    int code;
    CudaFailure(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};
// The level-synchronous builder: the tree, the sorted point data and the
// U, V, W, X lists that build_tree + build_lists give, bit for bit, from
// whole-level passes (Morton sort, split sets per level, 2:1 balance as a
// closed form over the levels, lists by per-node neighbour lookups).  It
// runs on the current CUDA device (on_device; xs and xt may be host or
// device pointers) or on the host (host pointers).  With xt the tree is
// built on the union of the n sources and the n targets.
void build_tree_levels(const double *xs, const double *xt, int64_t n, const TreeOptions &opt,
                       bool on_device, Tree &tree);
// Fill U, V, W, X lists.
void build_lists(Tree &tree);
// Point roles and the single root of a one-problem tree.  With
// distinct = false every point is a source and a target (qidx = oidx =
// perm); otherwise the first nsrc input points are the sources and the next
// nsrc the targets.
void set_point_roles(Tree &tree, int64_t nsrc, bool distinct);
// Merge trees of independent problems (lists built, roles set) into one
// forest.  Nodes are ordered by level, then problem, then the problem's own
// order, so every per-level range still covers one contiguous block; point
// ranges, lists and schedules are renumbered and the caller rows of problem
// i are shifted by row_offset[i].
void merge_forest(const std::vector<Tree> &parts, const std::vector<int64_t> &row_offset,
                  Tree &out);

// M2L work decomposition: per level, targets grouped by parity class and
// chunked into tiles of kTileRows; each tile lists the offsets any of its
// targets uses and, per offset, the source node of every row (-1: none).
struct M2LTable {
    std::vector<int32_t> tile_level;      // tiles
    std::vector<int32_t> tile_target;     // tiles x kTileRows (-1 pad)
    std::vector<int32_t> tile_entry_ptr;  // tiles + 1
    std::vector<int32_t> entry_offset;    // entries
    std::vector<int32_t> entry_src;       // entries x kTileRows (-1 none)
    // tiles of each persistent block (empty when there are fewer tiles
    // than blocks): cta_ptr[ncta + 1], cta_tiles[tiles]
    int ncta = 0;
    std::vector<int32_t> cta_ptr, cta_tiles;
};
void build_m2l_table(const Tree &tree, M2LTable &table);
// Deals the tiles to `ncta` persistent blocks, longest first (cost: the
// tile's entries), each to the least loaded block; no schedule when there
// are fewer tiles than blocks.
void build_m2l_schedule(int ncta, M2LTable &table);

// M2L work decomposition of the pair-column tensor-core kernel: the boxes
// with a V list, in plan order, are cut into windows of at most
// kWinTargets boxes with about equal cost; within a window, the (target,
// source) pairs of each offset t form items of at most kItemCols pairs, in
// offset order and, within an item, in target order.  Each item is one
// product S_t [q_A ...] whose columns are its pairs.  The windows are dealt
// to `ncta` persistent blocks, longest first, to the least loaded block.
constexpr int kWinTargets = 256;
constexpr int kItemCols = 128;
struct M2LWindows {
    int ncta = 0;
    std::vector<int32_t> cta_ptr, cta_win;      // ncta + 1; windows per block
    std::vector<int32_t> win_target_ptr;        // windows + 1
    std::vector<int32_t> win_targets;           // target boxes, window by window
    std::vector<int32_t> win_item_ptr;          // windows + 1
    std::vector<int32_t> item_offset;           // items: offset index t
    std::vector<int32_t> item_pair_ptr;         // items + 1
    std::vector<int32_t> pair_src;              // pairs: source box
    std::vector<int32_t> pair_slot;             // pairs: target's place in its window
};
void build_m2l_windows(const Tree &tree, int ncta, M2LWindows &w);

// Node schedules for the up and down passes.
struct Schedules {
    std::vector<int32_t> p2m_nodes;       // leaves at level >= 2
    std::vector<int32_t> m2m_nodes;       // internal nodes, by level
    std::vector<int32_t> m2m_level_ptr;   // depth + 2
    std::vector<int32_t> down_nodes;      // nodes at level >= 2, by level,
                                          // then child position, then order
    std::vector<int32_t> down_level_ptr;  // depth + 2
    std::vector<int32_t> down_chunk;      // chunks x 4: start, count, sigma,
                                          // level (chunks never mix sigma)
    std::vector<int32_t> down_chunk_level_ptr; // depth + 2
    std::vector<int32_t> x_nodes;         // nodes whose X list goes through P2L
    std::vector<int32_t> x_slot;          // nodes: slot in x_nodes or -1
    std::vector<int32_t> x_level_count;   // depth + 1: x_nodes per level
    std::vector<int32_t> w_direct;        // nodes: 1 for a leaf small enough
                                          // to interact through its points
                                          // in W and X lists
};
// direct_max: leaves of at most this many points take their X lists'
// points in the leaf pass instead of through P2L (-1: none)
void build_schedules(const Tree &tree, int chunk, int direct_max, Schedules &s);

// Check every index table the kernels read before any of it reaches the
// device: CSR offsets non-decreasing and ending at their index count, every
// node, point, row, offset and schedule index inside its array, and every
// value the upload narrows to 32 bits representable.  Empty when the plan
// is sound, else a message naming the first table that is not.
std::string check_tables(const Tree &t, const Schedules &s, const M2LTable &m, int64_t rows);
// The same for the pair-column M2L table (every index inside its array,
// window and item sizes within the kernel's limits).
std::string check_windows(const Tree &t, const M2LWindows &w);

} // namespace kifmm

// Host-side plan (the opaque fmm_plan_t).
struct fmm_plan_s;
