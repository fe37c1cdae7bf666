// Internal plan representation shared by the host plan compiler, the C ABI
// and the kernels.  Not part of the public ABI (see include/fmm.h).
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/fmm.h"

namespace fmm {

// Upper bound on the flattened terms of one leaf (Eq. 4.4): the number of
// A blocks summed into S_r, of B blocks summed into T_r, and of C blocks the
// product M_r is added into.
constexpr int kMaxTerms = 64;

// One leaf of the flattened plan: S = sum a_coef[t] A(a_blk[t]),
// T = sum b_coef[t] B(b_blk[t]), C(c_blk[t]) += c_coef[t] * S T.
// Blocks are packed (row_block << 16) | col_block in the block grid of the
// operand (A: pm x pk blocks, B: pk x pn, C: pm x pn).  c_first[t] is 1 when
// this leaf is the first (in leaf order) to touch C block c_blk[t], so the
// epilogue stores instead of accumulating.
constexpr int32_t kFirstBit = (int32_t)0x80000000u;

// Largest pm x pn for which the plan carries per-C-block term lists.
constexpr int64_t kMaxGatherBlocks = (int64_t)1 << 20;

struct LeafDesc {
  int32_t na, nb, nc, pad;
  int32_t a_blk[kMaxTerms];
  float a_coef[kMaxTerms];
  int32_t b_blk[kMaxTerms];
  float b_coef[kMaxTerms];
  int32_t c_blk[kMaxTerms];
  float c_coef[kMaxTerms];
  int32_t c_first[kMaxTerms];
};

// A rule re-indexed so that A, B and C blocks are all enumerated row-major.
struct CanonRule {
  int m0, k0, n0, r;
  std::vector<double> U, V, W;  // (m0 k0) x r, (k0 n0) x r, (m0 n0) x r, row-major
  double Q = 0, E = 0;
  int64_t nnz = 0;
  // per product r: alpha_r, beta_r (nonzeros of column r of U, V) and
  // a_r, b_r (their 1-norms); per C block k: gamma_k (nonzeros of row k of W)
  std::vector<double> alpha, beta, a, b, gamma;
};

struct Plan {
  int levels = 0;
  int leaf_format = FMM_LEAF_BF16;
  int schedule = FMM_SCHEDULE_AUTO;  // where S_r / T_r are formed (fmm_plan_set_schedule)
  std::vector<CanonRule> rules;
  int64_t pm = 1, pk = 1, pn = 1;  // products of m0, k0, n0 over the levels
  int64_t leaves = 1;
  double q_sum = 0, e_prod = 1;
  int64_t nnz = 0;
  int max_terms = 0;  // max over leaves of na, nb, nc
  std::vector<LeafDesc> host;
  // The same terms as compact per-side lists (what the bandwidth passes
  // read): for side s (0 = A, 1 = B, 2 = C), int32 words at list_off[s]:
  // start[leaves + 1], then blk[list_nnz[s]], then coef[list_nnz[s]] (float
  // bits); leaf r's terms are [start[r], start[r + 1]).  C blocks carry
  // kFirstBit when the leaf is the first to touch the block.
  std::vector<int32_t> lists;
  int64_t list_off[3] = {0, 0, 0};
  int64_t list_nnz[3] = {0, 0, 0};
  // The C terms again, grouped by C block (what the gather output pass
  // reads): int32 words at gather_off: start[pm pn + 1], then leaf[nnz],
  // then coef[nnz] (float bits); block k's terms are [start[k], start[k+1])
  // in leaf order.  gather_off < 0 when pm pn exceeds kMaxGatherBlocks.
  int64_t gather_off = -1;
  // Device copy (on `device`): the LeafDesc array followed by `lists`.
  LeafDesc* dev = nullptr;
  int device = -1;
  // Non-uniform plans (Sec. 3.4): one rule per node of the recursion tree.
  // table holds the distinct rules and node_rule each node's rule index,
  // level by level, the children of a node in product order (r = 0..R-1).
  // Both empty for uniform plans, whose levels are `rules`.  For a tree,
  // rules[l] is the first node's rule of level l+1 (all nodes of a level
  // partition alike), q_sum is max_k delta_k and e_prod max_k xi_k (Sec. 4.5).
  std::vector<CanonRule> table;
  std::vector<int> node_rule;
  bool level_r_uniform = true;  // all nodes of each level have the same R
  int between = 0;           // scaling between recursive steps (fmm_plan_set_between_scaling)
  Plan* level1 = nullptr;    // the first level alone (its sums give the between-steps exponents)
  Plan* grad_a = nullptr;  // plan for dA = dC B^T  (lazily built)
  Plan* grad_b = nullptr;  // plan for dB = A^T dC
};

// Host plan compiler (plan.cpp).
fmm_status canonicalize(const fmm_rule& in, CanonRule* out);
int brent_violations(const CanonRule& r);
void principal_quantities(CanonRule* r);
fmm_status build_plan(const std::vector<CanonRule>& rules, int leaf_format, Plan** out);
fmm_status build_tree_plan(const std::vector<CanonRule>& table, int levels, const std::vector<int>& node_rule,
                           int leaf_format, Plan** out);
void destroy_plan(Plan* p);
CanonRule rule_for_grad_a(const CanonRule& r);  // <m0, n0, k0>: [[W, V^T, U]]
CanonRule rule_for_grad_b(const CanonRule& r);  // <k0, m0, n0>: [[U^T, W, V]]

}  // namespace fmm
