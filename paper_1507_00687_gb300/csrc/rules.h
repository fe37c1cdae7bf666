// Rule algebra and the Castrapel-Gustafson variant trees (rules.cpp).
// Internal to the library; the C ABI wraps these in capi.cu.
#pragma once

#include <cstdint>
#include <vector>

#include "plan.h"

namespace fmm {

fmm_status rule_rotate(const fmm_rule& in, double* U, double* V, double* W, fmm_rule* out);
fmm_status rule_compose(const fmm_rule& outer, const fmm_rule& inner, double* U, double* V, double* W,
                        fmm_rule* out);
fmm_status rule_transform(const fmm_rule& in, const double* XU, const double* XV, const double* XW, double* U,
                          double* V, double* W, fmm_rule* out);
fmm_status rule_permute(const fmm_rule& in, const int32_t* pi, const int32_t* pk, const int32_t* pj, double* U,
                        double* V, double* W, fmm_rule* out);

// Variant v (0..7) of a canonical <2,2,2> rule: bit 0 exchanges the i
// blocks, bit 1 the k blocks, bit 2 the j blocks.
CanonRule cg_variant(const CanonRule& c, int v);
uint64_t splitmix64_at(uint64_t seed, uint64_t n);
// Each node's variant index, level by level from the root (the node order
// of fmm_plan_tree), by FMM_SELECT_*.
fmm_status cg_select(const CanonRule& base, int levels, int selection, uint64_t seed, const float* block_max_a,
                     const float* block_max_b, std::vector<int>* node_rule);

}  // namespace fmm
