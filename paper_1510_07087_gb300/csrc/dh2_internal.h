// Internal structures shared by the host code (tree builder, C ABI) and the
// CUDA kernels.  Nothing here is part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dh2.h"

namespace dh2 {

constexpr int kSideRow = 0;
constexpr int kSideCol = 1;

// Largest number of rows of a factor (leaf cluster size, or k_t1c' + k_t2c'
// for a non-leaf pair) the pair kernels accept, per real type.
constexpr int kPmaxF32 = 128;
constexpr int kPmaxF64 = 96;
// Singular values stored per pair: kSigValues values (the largest factor
// size), then the number resolved individually and the energy of the rest.
constexpr int kSigValues = 128;
constexpr int kSigStride = kSigValues + 2;

// Launch codes of the pair kernel: problem (6 bits) | side (1 bit) | pair (25 bits).
constexpr int kCodeSideShift = 25;
constexpr int kCodeProbShift = 26;
constexpr uint32_t kCodePairMask = (1u << 25) - 1u;
constexpr int kMaxBatch = 64;
constexpr int kRTile = 32;  // columns per tile of the R = Q^* A kernel
constexpr int kNormCols = 64;  // columns of a piece of the admissible blocks' norms pass (by 32 rows)

// Device status bits (OR-ed by kernels into one word).
constexpr uint32_t kStatusNoConv = 1u;
constexpr uint32_t kStatusTooLarge = 2u;
constexpr uint32_t kStatusTimeout = 4u;
constexpr uint32_t kStatusNaN = 8u;

struct Block {
  int32_t t, s;
  int32_t adm;
  int32_t cb;
};

// One used (cluster, direction) pair of one side.
struct Pair {
  int32_t cluster;
  int32_t dir;
  int32_t level;
  int32_t leaf;
  int64_t ncols;                    // #F_tc
  std::vector<int32_t> own;         // own admissible blocks, column order
  // parent segments: (parent pair id, column offset of that segment in this pair)
  std::vector<std::pair<int64_t, int64_t>> parents;
  int64_t son_pair[2] = {-1, -1};   // non-leaf: pairs (t_j, sd(c))
  int64_t son_off[2] = {0, 0};      // column offset of this pair's columns inside the son pair
};

struct Side {
  std::vector<Pair> pairs;                      // ordered by level descending, leaves first per level
  std::vector<int64_t> level_begin;             // depth+2 entries: pairs of level l in [begin[d-l].. ) (see tree.cpp)
  std::vector<int64_t> leaf_pairs;              // ids of leaf pairs
  std::vector<std::vector<int64_t>> nonleaf_by_level;  // per level l: non-leaf pair ids
  std::vector<int64_t> block_pair;              // per block: pair id of this side (-1 if inadmissible)
  std::vector<int64_t> block_off;               // per block: column offset of the block in its own pair
  // leaf column maps (concatenated over leaf pairs): G index of the column and
  // block id, kept as segments (one per block of a leaf pair's F_tc, in column
  // order) and expanded on the device when the tree is uploaded
  std::vector<int64_t> leaf_colmap_off;         // per pair (only leaf pairs meaningful), npairs+1
  std::vector<int64_t> seg_dst;                 // per segment: first entry in the column map
  std::vector<int32_t> seg_col0;                // first column of G (the other cluster's start)
  std::vector<int32_t> seg_w;                   // number of columns
  std::vector<int32_t> seg_blk;                 // block id
  std::vector<int64_t> seg_begin;               // per pair: its first segment (npairs+1; leaf pairs only non-empty)
  int64_t ncols_total = 0, nleafcols = 0;
};

struct Tree {
  int64_t n = 0;
  dh2_tree_params params{};
  std::vector<int64_t> perm;
  std::vector<int32_t> start, size, level, parent, son0, son1;
  std::vector<double> lo, hi, center, diam;  // 3 per cluster for lo/hi/center
  int32_t depth = 0;
  std::vector<double> delta;
  std::vector<std::vector<double>> dirs;     // per level, 3 * |D_l|
  std::vector<std::vector<int32_t>> sd;      // per level, |D_l| (lazy, -2 = not computed)
  std::vector<Block> blocks;
  int64_t nadm = 0;
  double adm_fraction = 0.0;
  int32_t max_leaf = 0;
  Side side[2];

  int32_t sd_of(int32_t lvl, int32_t c);     // son map with lazy evaluation
  int32_t nclusters() const { return (int32_t)start.size(); }
  bool is_leaf(int32_t t) const { return son0[t] < 0; }

  // device copies (uploaded on first use)
  struct Dev;
  Dev* dev = nullptr;
  int dev_id = -1;
};

dh2_status build_tree(const double* pts, int64_t n, const dh2_tree_params& p, Tree& tr);
void free_tree_device(Tree& tr);

// Column panels of a host-resident G (dh2_compress_host): whole clusters of
// the shallowest level that holds an admissible block (or leaves above it),
// grouped into ranges of similar width.  Every admissible block's column
// cluster lies in one panel, and so does every column-basis leaf pair
// together with the blocks it inherits from its ancestors; a row-basis leaf
// pair can start once the last panel its columns touch has arrived.  Launch
// codes as in the compression schedule (side << 25 | pair, or block).
struct PanelPlan {
  std::vector<int64_t> col;                                  // panel k: columns [col[k], col[k+1])
  std::vector<std::vector<uint32_t>> blk;                    // per panel: blocks whose columns lie in it
  std::vector<uint32_t> blk_rest;                            // blocks across panels (inadmissible only)
  std::vector<std::vector<std::vector<uint32_t>>> col_leaf;  // per panel, per size class: column-basis leaves
  // per panel k, per size class: row-basis leaves whose columns (own and
  // inherited blocks) all lie in panels 0..k
  std::vector<std::vector<std::vector<uint32_t>>> row_leaf;
};

}  // namespace dh2

struct dh2_tree {
  dh2::Tree tr;
  // host-input compression: the panel plan and the device buffer G is copied
  // into (built and allocated on first use, reused by later calls)
  dh2::PanelPlan plan;
  bool plan_built = false;
  void* g_stage = nullptr;
  size_t g_stage_bytes = 0;
};
